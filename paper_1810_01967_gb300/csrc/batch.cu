// Many slices of different sizes through whole BLIP iterations at once (the batching form).
//
// All slices stay resident in HBM, stacked voxel-major: X, A^H Y, the gradient output Z and the
// BF16 query operand are [sum n_s][...] with per-slice offsets.  One iteration runs the
// gradient step of every slice -- one launch over all stacked slices when every Ny factors into
// 2, 3 and 5 (mixed-radix y-transforms in shared memory, a descriptor table locating each
// slice's rows and masks), else per slice with its own y-FFT plan -- writing the rows of Z and of
// the packed operand, and then one projection over all stacked voxels: a single persistent
// launch of the search kernel against the shared dictionary, however uneven the slices.  With
// `use_graph` the iteration is captured once into a CUDA graph on an internal stream and
// replayed; the first iteration runs eagerly so that cuFFT plans and scratch are created
// outside the capture, and a graph is captured again when any scratch buffer it references has
// been reallocated since (the scratch epoch).  Only projections without host synchronisation
// can be captured: FP32, BF16 or FP8 without certification, and -- with the dictionary's BF16
// operand -- the cover-tree and learned forms, whose exhaustive fallback then takes its voxel
// count from the device (mrf_dict::sync_free) instead of reading it back.
#include <cstring>
#include <vector>

#include "mrf_internal.cuh"

struct mrf_batch {
    mrf_dict* D = nullptr;
    std::vector<mrf_op> ops;
    std::vector<int64_t> off;   // [ns + 1] voxel offsets
    int64_t n_total = 0;
    float2* X = nullptr;        // [n_total][L]
    float2* AHY = nullptr;      // [n_total][L]
    int32_t* idx = nullptr;     // [n_total]
    float2* rho = nullptr;      // [n_total]
    cudaStream_t cs = nullptr;  // capture / replay stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    mrf_proj_opts gopts = {};
    float gmu = 0.f;
    uint64_t gepoch = 0;        // scratch epoch the graph was captured at
    void* gtable = nullptr;     // descriptor table of the one-launch gradient (device)
    int64_t gtiles = 0;         // its CTA tiles; 0: per-slice gradient steps
    int gmaxNy = 0;
};

namespace {

mrf_status bfail(mrf_status s, const std::string& m) {
    mrf_set_error(m);
    return s;
}

bool capturable(const mrf_dict* D, const mrf_proj_opts& o) {
    if (o.certify) return false;
    if (o.mode == MRF_PROJ_FP32_EXACT || o.mode == MRF_PROJ_BF16 || o.mode == MRF_PROJ_FP8)
        return true;
    // the tensor-core tree search reads nothing back to the host when uncertified
    if (o.mode == MRF_PROJ_TREE_TC) return D->ttc != nullptr;
    return (o.mode == MRF_PROJ_COVERTREE || o.mode == MRF_PROJ_LEARNED) && D->bop != nullptr;
}

// Sets the dictionary's sync-free mode for the lifetime of a graph run.
struct SyncFree {
    mrf_dict* D;
    bool prev;
    SyncFree(mrf_dict* d, bool on) : D(d), prev(d->sync_free) { if (on) D->sync_free = true; }
    ~SyncFree() { D->sync_free = prev; }
};

mrf_status iterate(mrf_batch* B, float mu, const mrf_proj_opts* o, cudaStream_t st) {
    mrf_dict* D = B->D;
    const int L = D->L;
    MRF_TRY(dict_ensure_scratch(D, B->n_total));     // a no-op unless another call shrank it
    const bool zq = (o->mode == MRF_PROJ_BF16);
    if (B->gtiles > 0) {
        ProfScope ps0(0, 1, st);
        MRF_TRY(launch_grad_multi(B->gtable, static_cast<int>(B->ops.size()), B->gtiles,
                                  B->gmaxNy, B->X, B->AHY, L, mu, D->zbuf, zq ? D->zq : nullptr,
                                  D->Kp, D->err, st));
    } else {
        for (size_t s = 0; s < B->ops.size(); ++s) {
            const int64_t a = B->off[s];
            MRF_TRY(gradient_to(&B->ops[s], B->AHY + a * L, B->X + a * L, mu, D->zbuf + a * L,
                                D->wbuf, zq ? D->zq + a * D->Kp : nullptr, D->Kp, D->err, st));
        }
    }
    return project_core(D, D->zbuf, B->n_total, o, B->idx, B->idx, B->rho, B->X, zq, st);
}

void drop_graph(mrf_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
}

}  // namespace

extern "C" {

void mrf_batch_free(mrf_batch* B) {
    if (!B) return;
    drop_graph(B);
    if (B->cs) cudaStreamDestroy(B->cs);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    void* ptrs[] = {B->X, B->AHY, B->idx, B->rho, B->gtable};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete B;
}

mrf_status mrf_batch_create(mrf_dict* D, int32_t n_slices, const mrf_op* ops, mrf_batch** out) {
    if (!D || !ops || !out || n_slices < 1) return bfail(MRF_EINVAL, "bad batch arguments");
    *out = nullptr;
    mrf_batch* B = new mrf_batch();
    B->D = D;
    B->off.push_back(0);
    int64_t max_n = 0;
    for (int32_t s = 0; s < n_slices; ++s) {
        mrf_status st = check_op_public(&ops[s]);
        if (st != MRF_OK) { mrf_batch_free(B); return st; }
        if (ops[s].L != D->L) { mrf_batch_free(B); return bfail(MRF_EINVAL, "slice L differs from the dictionary's"); }
        B->ops.push_back(ops[s]);
        const int64_t n = static_cast<int64_t>(ops[s].Ny) * ops[s].Nx;
        max_n = n > max_n ? n : max_n;
        B->off.push_back(B->off.back() + n);
    }
    B->n_total = B->off.back();
    if (B->n_total > INT32_MAX) { mrf_batch_free(B); return bfail(MRF_EINVAL, "too many voxels"); }
    const size_t nl = static_cast<size_t>(B->n_total) * D->L;
    cudaError_t e = cudaMalloc(&B->X, nl * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&B->AHY, nl * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&B->idx, B->n_total * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&B->rho, B->n_total * sizeof(float2));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mrf_batch_free(B);
        return bfail(MRF_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    mrf_status st = dict_ensure_scratch(D, B->n_total);
    if (st != MRF_OK) { mrf_batch_free(B); return st; }
    (void)max_n;
    bool all_multi = true;
    for (const mrf_op& o : B->ops) all_multi = all_multi && grad_multi_supported(o.Ny);
    if (all_multi) {
        st = grad_multi_table(B->ops.data(), B->off.data(), n_slices, &B->gtable, &B->gtiles,
                              &B->gmaxNy, nullptr);
        if (st != MRF_OK) { mrf_batch_free(B); return st; }
    }
    *out = B;
    return MRF_OK;
}

mrf_status mrf_batch_load(mrf_batch* B, const void* const* Y, void* stream) {
    if (!B || !Y) return bfail(MRF_EINVAL, "batch and Y are required");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int L = B->D->L;
    for (size_t s = 0; s < B->ops.size(); ++s) {
        if (!Y[s]) return bfail(MRF_EINVAL, "a slice's k-space pointer is NULL");
        MRF_TRY(mrf_adjoint(&B->ops[s], Y[s], B->AHY + B->off[s] * L, stream));
    }
    MRF_CUDA_TRY(cudaMemsetAsync(B->X, 0, sizeof(float2) * B->n_total * L, st));
    MRF_CUDA_TRY(cudaMemsetAsync(B->idx, 0, sizeof(int32_t) * B->n_total, st));
    return MRF_OK;
}

mrf_status mrf_batch_run(mrf_batch* B, int32_t iters, float mu, const mrf_proj_opts* opts,
                         int32_t use_graph, void* stream) {
    if (!B || iters < 0 || !std::isfinite(mu)) return bfail(MRF_EINVAL, "bad batch run arguments");
    mrf_proj_opts o;
    if (opts) o = *opts; else mrf_default_proj_opts(&o);
    MRF_TRY(check_proj_public(B->D, &o));
    if (use_graph && !capturable(B->D, o))
        return bfail(MRF_EUNSUPPORTED, "graph replay needs a projection without host "
                                       "synchronisation (certify = 0; the cover-tree and learned "
                                       "forms also need the BF16 operand)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SyncFree guard(B->D, use_graph != 0);
    for (int32_t it = 0; it < iters; ++it) {
        if (!use_graph || it == 0) {
            MRF_TRY(iterate(B, mu, &o, st));
            continue;
        }
        // the graph holds the addresses of the dictionary's scratch buffers: replay it only
        // while none of them has been reallocated since the capture (another batch or
        // projection may have grown them), else capture again
        const bool same = B->exec && B->gmu == mu && B->gepoch == scratch_epoch() &&
                          std::memcmp(&B->gopts, &o, sizeof(o)) == 0;
        if (!same) {
            drop_graph(B);
            MRF_CUDA_TRY(cudaEventRecord(B->ev_in, st));
            MRF_CUDA_TRY(cudaStreamWaitEvent(B->cs, B->ev_in, 0));
            const bool prof = profiler_suspend();
            cudaError_t e = cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeRelaxed);
            mrf_status s = (e == cudaSuccess) ? iterate(B, mu, &o, B->cs) : MRF_ECUDA;
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(B->cs, &g);
            profiler_resume(prof);
            if (s != MRF_OK || e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return bfail(s != MRF_OK ? s : MRF_ECUDA, "capturing the batch iteration failed");
            }
            B->graph = g;
            MRF_CUDA_TRY(cudaGraphInstantiate(&B->exec, g, 0));
            B->gopts = o;
            B->gmu = mu;
            B->gepoch = scratch_epoch();
        }
        MRF_CUDA_TRY(cudaEventRecord(B->ev_in, st));
        MRF_CUDA_TRY(cudaStreamWaitEvent(B->cs, B->ev_in, 0));
        MRF_CUDA_TRY(cudaGraphLaunch(B->exec, B->cs));
        MRF_CUDA_TRY(cudaEventRecord(B->ev_out, B->cs));
        MRF_CUDA_TRY(cudaStreamWaitEvent(st, B->ev_out, 0));
    }
    return MRF_OK;
}

mrf_status mrf_batch_slice(mrf_batch* B, int32_t s, void** X, int32_t** idx, void** rho,
                           int64_t* n, int64_t* offset) {
    if (!B || s < 0 || s >= static_cast<int32_t>(B->ops.size())) return bfail(MRF_EINVAL, "bad slice");
    const int64_t a = B->off[s];
    if (X) *X = B->X + a * B->D->L;
    if (idx) *idx = B->idx + a;
    if (rho) *rho = B->rho + a;
    if (n) *n = B->off[s + 1] - a;
    if (offset) *offset = a;
    return MRF_OK;
}

mrf_status mrf_batch_lut(mrf_batch* B, float* params_out, void* stream) {
    if (!B || !params_out) return bfail(MRF_EINVAL, "batch and params_out are required");
    return mrf_lut(B->D, B->idx, B->n_total, params_out, stream);
}

}  // extern "C"
