// Host side of the C ABI (include/mrf.h): argument checks, dictionary index, scratch
// management, cuFFT plans of the sampling operator and the BLIP / CoverBLIP driver loop
// (§3.2 eq. blip, Algorithm 2 with the step rule eq. steprule and the kappa rescale).
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <atomic>
#include <tuple>

#include "mrf_internal.cuh"

static thread_local std::string g_last_error;

void mrf_set_error(const std::string& msg) { g_last_error = msg; }

namespace {

cudaStream_t S_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

mrf_status fail(mrf_status s, const std::string& msg) {
    mrf_set_error(msg);
    return s;
}


// Fault injection (mrf_debug_fail_alloc): the number of allocations still to succeed before one
// is refused, or -1.
std::atomic<int64_t> g_fail_alloc_after{-1};

std::atomic<uint64_t> g_scratch_epoch{0};

template <typename T>
mrf_status dalloc(T** p, size_t count) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        scratch_epoch_bump();
    }
    if (count == 0) return MRF_OK;
    int64_t left = g_fail_alloc_after.load();
    while (left >= 0 && !g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {}
    if (left == 0) return fail(MRF_ENOMEM, "injected allocation failure (mrf_debug_fail_alloc)");
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(MRF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return MRF_OK;
}

// ------------------------------------------------------------------------------ cuFFT plans
// Plans are cached per (kind, Ny, Nx, L) and re-bound to the caller's stream on every use.
std::mutex g_plan_mu;
std::map<std::tuple<int, int, int, int>, cufftHandle> g_plans;

}  // namespace

uint64_t scratch_epoch() { return g_scratch_epoch.load(); }
void scratch_epoch_bump() { g_scratch_epoch.fetch_add(1); }

mrf_status get_plan(int kind, int Ny, int Nx, int L, cudaStream_t st, cufftHandle* out) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto key = std::make_tuple(kind, Ny, Nx, L);
    auto it = g_plans.find(key);
    cufftHandle h;
    if (it == g_plans.end()) {
        cufftResult r;
        if (kind == 0) {   // 1-D along y of [Ny][Nx*L]: stride Nx*L, batches adjacent
            int nn[1] = {Ny};
            int emb[1] = {Ny};
            long long stride = static_cast<long long>(Nx) * L;
            r = cufftPlanMany(&h, 1, nn, emb, static_cast<int>(stride), 1, emb,
                              static_cast<int>(stride), 1, CUFFT_C2C, static_cast<int>(stride));
        } else {           // 2-D over (y, x) of [Ny][Nx][L]: element stride L, batch L
            int nn[2] = {Ny, Nx};
            int emb[2] = {Ny, Nx};
            r = cufftPlanMany(&h, 2, nn, emb, L, 1, emb, L, 1, CUFFT_C2C, L);
        }
        if (r != CUFFT_SUCCESS)
            return fail(MRF_ECUDA, "cufftPlanMany failed: " + std::to_string(static_cast<int>(r)));
        g_plans[key] = h;
    } else {
        h = it->second;
    }
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) return fail(MRF_ECUDA, "cufftSetStream failed");
    *out = h;
    return MRF_OK;
}

mrf_status fft_exec(cufftHandle h, const float2* in, float2* out, int dir) {
    cufftResult r = cufftExecC2C(h, reinterpret_cast<cufftComplex*>(const_cast<float2*>(in)),
                                 reinterpret_cast<cufftComplex*>(out), dir);
    if (r != CUFFT_SUCCESS)
        return fail(MRF_ECUDA, "cufftExecC2C failed: " + std::to_string(static_cast<int>(r)));
    return MRF_OK;
}

namespace {

mrf_status check_op(const mrf_op* op) {
    if (!op || !op->mask) return fail(MRF_EINVAL, "op or op->mask is NULL");
    if (op->Ny < 1 || op->Nx < 1 || op->L < 1) return fail(MRF_EINVAL, "op sizes must be >= 1");
    if (static_cast<int64_t>(op->Nx) * op->L > INT32_MAX)
        return fail(MRF_EINVAL, "Nx * L too large for the FFT batch");
    return MRF_OK;
}

// ------------------------------------------------------------------------------ scratch
int topk_slots(const mrf_proj_opts* o) {
    const bool k32 = o->mode == MRF_PROJ_FP8 || o->mode == MRF_PROJ_BF16X3 ||
                     (o->mode == MRF_PROJ_TREE_TC && o->certify);
    const int def = o->mode == MRF_PROJ_FP32_EXACT ? 8 : (k32 ? 32 : 16);
    const int k = o->topk > 0 ? o->topk : def;
    if (o->mode == MRF_PROJ_FP32_EXACT) return k <= 8 ? 8 : 16;   // FP32 scores: at most 16
    return k <= 8 ? 8 : (k <= 16 ? 16 : 32);
}

mrf_status ensure_scratch(mrf_dict* D, int64_t n) {
    if (n <= D->cap_n) return MRF_OK;
    const int64_t L = D->L;
    // a growth that fails part way leaves no scratch (the next call reallocates all of it)
    D->cap_n = 0;
    MRF_TRY(dalloc(&D->zbuf, static_cast<size_t>(n * L)));
    MRF_TRY(dalloc(&D->wbuf, static_cast<size_t>(n * L)));
    MRF_TRY(dalloc(&D->vlist, static_cast<size_t>(n)));
    MRF_TRY(dalloc(&D->vlist2, static_cast<size_t>(n)));
    if (D->bop) MRF_TRY(dalloc(&D->zq, static_cast<size_t>(n * D->Kp)));
    if (D->fop) {
        MRF_TRY(dalloc(&D->zq8, static_cast<size_t>(n * D->Kp8)));
        MRF_TRY(dalloc(&D->qs8, static_cast<size_t>(n)));
    }
    if (D->bop3) {
        MRF_TRY(dalloc(&D->zq3, static_cast<size_t>(n * D->Kp3)));
        MRF_TRY(dalloc(&D->zmarg, static_cast<size_t>(n)));
    }
    if (D->xprev) MRF_TRY(dalloc(&D->xprev, static_cast<size_t>(n * L)));
    if (D->aligned) MRF_TRY(dalloc(&D->qph, static_cast<size_t>(n)));
    D->cap_n = n;
    return MRF_OK;
}

mrf_status ensure_part(mrf_dict* D, int64_t n, int S, int K) {
    size_t need = static_cast<size_t>(S) * n * K * (sizeof(float) + sizeof(int32_t));
    if (need <= D->part_bytes) return MRF_OK;
    if (D->part) {
        cudaFree(D->part);
        scratch_epoch_bump();
    }
    D->part = nullptr;
    D->part_bytes = 0;
    cudaError_t e = cudaMalloc(&D->part, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MRF_ENOMEM, std::string("cudaMalloc(partials): ") + cudaGetErrorString(e));
    }
    D->part_bytes = need;
    return MRF_OK;
}

mrf_status check_proj_opts(const mrf_dict* D, const mrf_proj_opts* o) {
    if (!o) return fail(MRF_EINVAL, "proj opts is NULL");
    if (o->cone != MRF_CONE_COMPLEX && o->cone != MRF_CONE_REAL_POS)
        return fail(MRF_EINVAL, "unknown cone");
    if (o->topk < 0 || o->topk > 32) return fail(MRF_EINVAL, "topk must be in 0..32");
    if (!(o->tie_tol >= 0.f && o->tie_tol < 0.5f)) return fail(MRF_EINVAL, "tie_tol out of range");
    switch (o->mode) {
        case MRF_PROJ_FP32_EXACT: return MRF_OK;
        case MRF_PROJ_BF16:
            if (!D->bop) return fail(MRF_EUNSUPPORTED, "dictionary built without the BF16 operand");
            return MRF_OK;
        case MRF_PROJ_COVERTREE:
            if (!D->tree) return fail(MRF_EUNSUPPORTED, "dictionary built without a cover tree");
            if (!(o->eps >= 0.f) || !std::isfinite(o->eps)) return fail(MRF_EINVAL, "eps must be >= 0");
            return MRF_OK;
        case MRF_PROJ_LEARNED:
            if (!D->mlp) return fail(MRF_EUNSUPPORTED, "no learned model attached to the dictionary");
            return MRF_OK;
        case MRF_PROJ_FP8:
            if (!D->fop) return fail(MRF_EUNSUPPORTED, "dictionary built without the FP8 operand");
            return MRF_OK;
        case MRF_PROJ_BF16X3:
            if (!D->bop3)
                return fail(MRF_EUNSUPPORTED, "dictionary built without the split-BF16 operand");
            return MRF_OK;
        case MRF_PROJ_TREE_TC:
            if (!D->ttc)
                return fail(MRF_EUNSUPPORTED,
                            "dictionary built without the tensor-core tree search (tree_tc)");
            if (!(o->eps >= 0.f) || !std::isfinite(o->eps)) return fail(MRF_EINVAL, "eps must be >= 0");
            if ((o->cone == MRF_CONE_COMPLEX) != (ct_metric(D) == 0))
                return fail(MRF_EINVAL, "the tree's metric does not match the cone (tree_cone)");
            return MRF_OK;
        default: return fail(MRF_EINVAL, "unknown projection mode");
    }
}

mrf_status read_stats(mrf_dict* D, int64_t n, mrf_stats* stats, cudaStream_t st) {
    unsigned long long c[CNT_N];
    uint32_t e = 0;
    MRF_CUDA_TRY(cudaMemcpyAsync(c, D->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaMemcpyAsync(&e, D->err, sizeof(e), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats) {
        stats->n_voxels = n;
        stats->n_zero = static_cast<int64_t>(c[CNT_ZERO]);
        stats->n_tie_rescored = static_cast<int64_t>(c[CNT_TIE_RESCORED]);
        stats->n_tie_overflow = static_cast<int64_t>(c[CNT_TIE_OVERFLOW]);
        stats->n_uncertified = static_cast<int64_t>(c[CNT_UNCERT]);
        stats->n_fallback = static_cast<int64_t>(c[CNT_FALLBACK]);
        stats->n_dist_evals = static_cast<int64_t>(c[CNT_DIST]);
        stats->device_error = static_cast<int32_t>(e);
    }
    if (e & MRF_DERR_TIMEOUT) return fail(MRF_ETIMEOUT, "a device-side wait bound expired");
    if (e & MRF_DERR_NONFINITE) return fail(MRF_ENONFINITE, "non-finite value in an input");
    if (e & MRF_DERR_BOUNDS) return fail(MRF_EINTERNAL, "device-side index out of range");
    return MRF_OK;
}

}  // namespace

// ------------------------------------------------------------------------------ profiler
namespace {
struct ProfEntry {
    int stage;
    int launches;
    cudaEvent_t a, b;
};
bool g_prof_on = false;
std::vector<ProfEntry> g_prof_pending;
double g_prof_ms[MRF_PROFILE_STAGES];
int64_t g_prof_launch[MRF_PROFILE_STAGES];

void prof_clear() {
    for (auto& e : g_prof_pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    g_prof_pending.clear();
    for (int i = 0; i < MRF_PROFILE_STAGES; ++i) { g_prof_ms[i] = 0.0; g_prof_launch[i] = 0; }
}

}  // namespace

// Stage names of the NVTX ranges (tools such as ncu and Nsight Systems show them; without a tool
// attached the calls return at once).
const char* const kStageName[MRF_PROFILE_STAGES] = {
    "mrf:gradient", "mrf:pack_queries", "mrf:search_tc", "mrf:search_fp32",
    "mrf:merge", "mrf:fallback", "mrf:lut", "mrf:search_proposal"};

ProfScope::ProfScope(int stage, int launches, cudaStream_t s) : on(g_prof_on), st(s) {
    nvtxRangePushA(stage >= 0 && stage < MRF_PROFILE_STAGES ? kStageName[stage] : "mrf:stage");
    if (!on) return;
    stage_ = stage;
    launches_ = launches;
    cudaEventCreate(&a_);
    cudaEventCreate(&b_);
    cudaEventRecord(a_, st);
}

ProfScope::~ProfScope() {
    nvtxRangePop();
    if (!on) return;
    cudaEventRecord(b_, st);
    g_prof_pending.push_back(ProfEntry{stage_, launches_, a_, b_});
}

namespace {
// Options whose cert_margin selects the rigorous bound (for the merge's rescore window).
const mrf_proj_opts kRigorous = [] {
    mrf_proj_opts o;
    mrf_default_proj_opts(&o);
    o.cert_margin = 0.f;
    return o;
}();

mrf_status bf16_margin(const mrf_dict* D, const mrf_proj_opts* o, float* m) {
    // |c~ - c| <= (2u + u^2) ||d|| ||z|| for BF16 operand rounding (8 significant bits:
    // u = 2^-8) plus the FP32 accumulation of 2L products; in normalised-correlation units
    *m = o->cert_margin > 0.f ? o->cert_margin
                              : static_cast<float>(std::ldexp(1.0, -7) + std::ldexp(1.0, -16) +
                                                   2.0 * D->L * std::ldexp(1.0, -24));
    return MRF_OK;
}

// FP8 counterpart.  A row scaled into (224, 448] and rounded to E4M3 has error at most
// 2^-4 |x_i| per normal entry and 2^-10 per subnormal one, so relative to the row norm
// (>= 224) u8 = 2^-4 + sqrt(2L) 2^-10 / 224.  The MMA's internal accumulation width for FP8
// inputs is not documented; the margin assumes partial sums rounded to 13 bits (2L 2^-13),
// which is far above the FP32 figure.  The result (about 0.37 at L = 1000) makes certification
// flag almost every voxel: certified FP8 is a correctness mode, the FP8 form is meant to run
// uncertified with its agreement rate measured.
mrf_status fp8_margin(const mrf_dict* D, const mrf_proj_opts* o, float* m) {
    if (o->cert_margin > 0.f) { *m = o->cert_margin; return MRF_OK; }
    const double u8 = std::ldexp(1.0, -4) + std::sqrt(2.0 * D->L) * std::ldexp(1.0, -10) / 224.0;
    const double b = 2.0 * u8 + u8 * u8 + 2.0 * D->L * std::ldexp(1.0, -13);
    *m = static_cast<float>(b < 2.0 ? b : 2.0);
    return MRF_OK;
}

// Bound of the merge's FP32 rescore of one candidate, in normalised-correlation units: each lane
// accumulates 2 ceil(L/32) fused multiply-adds, five butterfly additions join the lanes, and a
// few roundings form the score (unit roundoff 2^-24 each, relative to sum |terms| <= ||z||).
float rescore_bound(int L) {
    return static_cast<float>((2.0 * ((L + 31) / 32) + 9.0) * std::ldexp(1.0, -24));
}

// Largest per-voxel bound of the split-BF16 form (the split.cu formula at the worst query
// split, ||z_lo|| = u (1 + u), ||e_z|| = u^2, ||z_hi|| = 1 + u, u = 2^-8): the rescore window.
float x3_bound_worst(const mrf_dict* D) {
    const double u = std::ldexp(1.0, -8), Al = D->x3_al, Ae = D->x3_ae;
    const double zl = u * (1 + u), ze = u * u, zh = 1 + u, dh = 1 + Al + Ae;
    const double Kp = D->Kp3 / 3;
    const double e_op = zl * Al + (1 + ze) * Ae + ze;
    const double m_lo = zl * dh + zh * Al, m_hi = m_lo + zh * dh;
    const double eps = std::ldexp(1.0, -23);
    const double e_acc = eps * (2.0 * Kp / 16.0 * m_lo + Kp / 16.0 * m_hi);
    return static_cast<float>((e_op + std::sqrt(2.0) * e_acc + eps) * (1.0 + 1e-6));
}

}  // namespace

mrf_status dict_ensure_scratch(mrf_dict* D, int64_t n) { return ensure_scratch(D, n); }

bool profiler_suspend() {
    const bool was = g_prof_on;
    g_prof_on = false;
    return was;
}
void profiler_resume(bool was) { g_prof_on = was; }

mrf_status check_op_public(const mrf_op* op) { return check_op(op); }
mrf_status check_proj_public(const mrf_dict* D, const mrf_proj_opts* o) {
    return check_proj_opts(D, o);
}

// Exhaustive projection of the voxels listed in D->vlist (cnt of them, length in D->nlist[0]):
// BF16 tensor cores with certification (second list D->vlist2) when the operand exists, else
// FP32.  Results go to the listed voxels' entries of the outputs.
mrf_status exhaustive_on_list(mrf_dict* D, const float2* Z, int32_t cnt, const mrf_proj_opts* o,
                              int32_t* idx_out, float2* rho_out, float2* X_out, cudaStream_t st) {
    ProfScope ps5(5, 0, st);
    if (D->bop && D->sync_free && !o->certify) {
        // the list's length stays on the device: cnt is its capacity, the kernels read the
        // count and skip what lies past it
        const int K = 16;
        MRF_TRY(launch_pack_gather(Z, D->vlist, cnt, D->L, D->Kp, D->zq, st, D->nlist));
        const int S = bf16_choose_splits(D, cnt);
        MRF_TRY(ensure_part(D, cnt, S, K));
        float* qs = static_cast<float*>(D->part);
        int32_t* qi = reinterpret_cast<int32_t*>(qs + static_cast<size_t>(S) * cnt * K);
        MRF_TRY(launch_bf16_topk(D->zq, cnt, D, o->cone, K, S, qs, qi, st, D->nlist));
        float bound;
        bf16_margin(D, &kRigorous, &bound);
        return launch_merge(Z, cnt, D, o->cone, K, S, qs, qi, D->vlist, D->nlist, o->tie_tol, 0,
                            0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err, D->counters,
                            st, 2.f * bound + o->tie_tol);
    }
    if (D->bop) {
        const int K = 16;
        MRF_TRY(launch_pack_gather(Z, D->vlist, cnt, D->L, D->Kp, D->zq, st));
        const int S = bf16_choose_splits(D, cnt);
        MRF_TRY(ensure_part(D, cnt, S, K));
        float* qs = static_cast<float*>(D->part);
        int32_t* qi = reinterpret_cast<int32_t*>(qs + static_cast<size_t>(S) * cnt * K);
        MRF_TRY(launch_bf16_topk(D->zq, cnt, D, o->cone, K, S, qs, qi, st));
        float margin;
        bf16_margin(D, o, &margin);
        float bound;
        bf16_margin(D, &kRigorous, &bound);
        MRF_TRY(launch_merge(Z, cnt, D, o->cone, K, S, qs, qi, D->vlist, D->nlist, o->tie_tol,
                             o->certify, margin, idx_out, rho_out, X_out, D->vlist2,
                             D->nlist + 1, D->err, D->counters, st,
                             2.f * bound + o->tie_tol));
        if (!o->certify) return MRF_OK;
        int32_t c2 = 0;
        MRF_CUDA_TRY(cudaMemcpyAsync(&c2, D->nlist + 1, sizeof(c2), cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        if (c2 == 0) return MRF_OK;
        const int S2 = fp32_choose_splits(c2, D->d, D->num_sms);
        MRF_TRY(ensure_part(D, c2, S2, 8));
        float* rs = static_cast<float*>(D->part);
        int32_t* ri = reinterpret_cast<int32_t*>(rs + static_cast<size_t>(S2) * c2 * 8);
        MRF_TRY(launch_fp32_topk(Z, D->vlist2, D->nlist + 1, c2, D, o->cone, 8, S2, rs, ri, st));
        return launch_merge(Z, c2, D, o->cone, 8, S2, rs, ri, D->vlist2, D->nlist + 1,
                            o->tie_tol, 0, 0.f, idx_out, rho_out, X_out, nullptr, nullptr,
                            D->err, D->counters, st);
    }
    const int S2 = fp32_choose_splits(cnt, D->d, D->num_sms);
    MRF_TRY(ensure_part(D, cnt, S2, 8));
    float* qs = static_cast<float*>(D->part);
    int32_t* qi = reinterpret_cast<int32_t*>(qs + static_cast<size_t>(S2) * cnt * 8);
    MRF_TRY(launch_fp32_topk(Z, D->vlist, D->nlist, cnt, D, o->cone, 8, S2, qs, qi, st));
    return launch_merge(Z, cnt, D, o->cone, 8, S2, qs, qi, D->vlist, D->nlist, o->tie_tol, 0,
                        0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err, D->counters, st);
}

namespace {
// FP32 exhaustive search of the voxels the merge listed as uncertified (D->vlist, length in
// D->nlist[0]), then their merge: the exact answer for those voxels.
mrf_status research_uncertified(mrf_dict* D, const float2* Z, int K, const mrf_proj_opts* o,
                                int32_t* idx_out, float2* rho_out, float2* X_out,
                                cudaStream_t st) {
    int32_t cnt = 0;
    MRF_CUDA_TRY(cudaMemcpyAsync(&cnt, D->nlist, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    if (cnt == 0) return MRF_OK;
    ProfScope ps5(5, 2, st);
    const int K2 = K > 16 ? 16 : K;      // FP32 scores: 16 candidates suffice
    const int S2 = fp32_choose_splits(cnt, D->d, D->num_sms);
    MRF_TRY(ensure_part(D, cnt, S2, K2));
    float* qs = static_cast<float*>(D->part);
    int32_t* qi = reinterpret_cast<int32_t*>(qs + static_cast<size_t>(S2) * cnt * K2);
    MRF_TRY(launch_fp32_topk(Z, D->vlist, D->nlist, cnt, D, o->cone, K2, S2, qs, qi, st));
    return launch_merge(Z, cnt, D, o->cone, K2, S2, qs, qi, D->vlist, D->nlist, o->tie_tol, 0,
                        0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err, D->counters, st);
}

// The projection proper.  `zq_ready` says the BF16 operand of Z is already in D->zq.
mrf_status project_impl(mrf_dict* D, const float2* Z, int64_t n, const mrf_proj_opts* o,
                        const int32_t* warm, int32_t* idx_out, float2* rho_out, float2* X_out,
                        bool zq_ready, cudaStream_t st) {
    (void)warm;
    const int K = topk_slots(o);
    if (n == 0) return MRF_OK;
    MRF_TRY(ensure_scratch(D, n));
    if (o->mode == MRF_PROJ_FP32_EXACT) {
        const int S = D->tune.fp32_splits > 0 ? D->tune.fp32_splits
                                              : fp32_choose_splits(n, D->d, D->num_sms);
        D->tune.last_fp32_splits = S;
        MRF_TRY(ensure_part(D, n, S, K));
        float* ps = static_cast<float*>(D->part);
        int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(S) * n * K);
        {
            ProfScope ps3(3, 1, st);
            MRF_TRY(launch_fp32_topk(Z, nullptr, nullptr, n, D, o->cone, K, S, ps, pi, st));
        }
        ProfScope ps4(4, 1, st);
        MRF_TRY(launch_merge(Z, n, D, o->cone, K, S, ps, pi, nullptr, nullptr, o->tie_tol, 0,
                             0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err,
                             D->counters, st));
        return MRF_OK;
    }
    if (o->mode == MRF_PROJ_BF16 || o->mode == MRF_PROJ_FP8) {
        const bool f8 = (o->mode == MRF_PROJ_FP8);
        if (f8) {
            ProfScope ps1(1, 1, st);
            MRF_TRY(launch_pack_queries_fp8(Z, nullptr, n, D->L, D->Kp8, D->zq8, D->qs8, st));
        } else if (!zq_ready) {
            ProfScope ps1(1, 1, st);
            MRF_TRY(launch_pack_queries(Z, n, D->L, D->Kp, D->zq, st));
        }
        const int S = bf16_choose_splits(D, n);
        MRF_TRY(ensure_part(D, n, S, K));
        float* ps = static_cast<float*>(D->part);
        int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(S) * n * K);
        {
            ProfScope ps2(2, 1, st);
            if (f8) MRF_TRY(launch_fp8_topk(D->zq8, D->qs8, n, D, o->cone, K, S, ps, pi, st));
            else MRF_TRY(launch_bf16_topk(D->zq, n, D, o->cone, K, S, ps, pi, st));
        }
        if (o->certify) MRF_CUDA_TRY(cudaMemsetAsync(D->nlist, 0, sizeof(int32_t), st));
        float margin;
        if (f8) fp8_margin(D, o, &margin);
        else bf16_margin(D, o, &margin);
        {
            ProfScope ps4(4, 1, st);
            // rescore window: twice the rigorous bound of the kernel's error, plus tie_tol
            float bound;
            if (f8) fp8_margin(D, &kRigorous, &bound);
            else bf16_margin(D, &kRigorous, &bound);
            MRF_TRY(launch_merge(Z, n, D, o->cone, K, S, ps, pi, nullptr, nullptr, o->tie_tol,
                                 o->certify, margin, idx_out, rho_out, X_out, D->vlist,
                                 D->nlist, D->err, D->counters, st, 2.f * bound + o->tie_tol));
        }
        if (o->certify) MRF_TRY(research_uncertified(D, Z, K, o, idx_out, rho_out, X_out, st));
        return MRF_OK;
    }
    if (o->mode == MRF_PROJ_BF16X3) {
        // exact form: split-BF16 correlations on the tensor cores, the top K rescored exactly,
        // each voxel certified against its own rigorous bound, the rest searched in FP32
        const float brs = rescore_bound(D->L);
        {
            ProfScope ps1(1, 1, st);
            MRF_TRY(launch_pack_queries_x3(Z, n, D, brs, D->zq3, D->zmarg, st));
        }
        const int S = bf16_choose_splits(D, n);
        MRF_TRY(ensure_part(D, n, S, K));
        float* ps = static_cast<float*>(D->part);
        int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(S) * n * K);
        {
            ProfScope ps2(2, 1, st);
            MRF_TRY(launch_x3_topk(D->zq3, n, D, o->cone, K, S, ps, pi, st));
        }
        if (o->certify) MRF_CUDA_TRY(cudaMemsetAsync(D->nlist, 0, sizeof(int32_t), st));
        {
            ProfScope ps4(4, 1, st);
            // rescore window: twice the largest kernel bound, plus tie_tol
            const float window = 2.f * x3_bound_worst(D) + o->tie_tol;
            const bool own = !(o->cert_margin > 0.f);
            MRF_TRY(launch_merge(Z, n, D, o->cone, K, S, ps, pi, nullptr, nullptr, o->tie_tol,
                                 o->certify, o->cert_margin, idx_out, rho_out, X_out, D->vlist,
                                 D->nlist, D->err, D->counters, st, window,
                                 own ? D->zmarg : nullptr));
        }
        if (o->certify) MRF_TRY(research_uncertified(D, Z, K, o, idx_out, rho_out, X_out, st));
        return MRF_OK;
    }
    if (o->mode == MRF_PROJ_TREE_TC) {
        // block balls of the tree's depth-first order pruned per voxel, voxel tiles sharing one
        // block list, the tiles searched on the tensor cores (split-BF16 operand when certifying)
        const bool split = ttc_has_split(D) && (o->certify || !ttc_has_bf16(D));
        const float brs = rescore_bound(D->L);
        TtcOut t;
        MRF_TRY(ttc_search(D, Z, n, o->cone, o->eps, split, K, brs, &t, st));
        if (o->certify) MRF_CUDA_TRY(cudaMemsetAsync(D->nlist, 0, sizeof(int32_t), st));
        float margin = o->cert_margin, window;
        const float* vm = nullptr;
        if (split) {
            window = 2.f * x3_bound_worst(D) + o->tie_tol;
            if (!(o->cert_margin > 0.f)) vm = D->zmarg;
        } else {
            bf16_margin(D, o, &margin);
            float bound;
            bf16_margin(D, &kRigorous, &bound);
            window = 2.f * bound + o->tie_tol;
        }
        {
            ProfScope ps4(4, 1, st);
            MRF_TRY(launch_merge(Z, n, D, o->cone, K, t.S, t.part_s, t.part_i, t.vorder, t.count,
                                 o->tie_tol, o->certify, margin, idx_out, rho_out, X_out,
                                 D->vlist, D->nlist, D->err, D->counters, st, window, vm));
        }
        if (o->certify) MRF_TRY(research_uncertified(D, Z, K, o, idx_out, rho_out, X_out, st));
        return MRF_OK;
    }
    if (o->mode == MRF_PROJ_COVERTREE) {
        MRF_TRY(ensure_part(D, n, 1, 8));
        float* ps = static_cast<float*>(D->part);
        int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(n) * 8);
        MRF_CUDA_TRY(cudaMemsetAsync(D->nlist, 0, 2 * sizeof(int32_t), st));
        {
            ProfScope ps7(7, 1, st);
            MRF_TRY(launch_ct_search(Z, n, D, o->cone, warm, o->eps, o->tree_route, ps, pi,
                                     D->vlist, D->nlist, st));
        }
        {
            ProfScope ps4(4, 1, st);
            MRF_TRY(launch_merge(Z, n, D, o->cone, 8, 1, ps, pi, nullptr, nullptr, o->tie_tol, 0,
                                 0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err,
                                 D->counters, st));
        }
        if (D->sync_free && D->bop && !o->certify)
            return exhaustive_on_list(D, Z, static_cast<int32_t>(n), o, idx_out, rho_out, X_out, st);
        int32_t cnt = 0;
        MRF_CUDA_TRY(cudaMemcpyAsync(&cnt, D->nlist, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        if (cnt > 0) MRF_TRY(exhaustive_on_list(D, Z, cnt, o, idx_out, rho_out, X_out, st));
        return MRF_OK;
    }
    if (o->mode == MRF_PROJ_LEARNED) {
        MRF_TRY(ensure_part(D, n, 1, 8));
        float* ps = static_cast<float*>(D->part);
        int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(n) * 8);
        MRF_CUDA_TRY(cudaMemsetAsync(D->nlist, 0, 2 * sizeof(int32_t), st));
        {
            ProfScope ps7(7, 4, st);
            MRF_TRY(learned_candidates(D, Z, n, o->cone, ps, pi, st));
        }
        {
            ProfScope ps4(4, 2, st);
            MRF_TRY(launch_merge(Z, n, D, o->cone, 8, 1, ps, pi, nullptr, nullptr, o->tie_tol, 0,
                                 0.f, idx_out, rho_out, X_out, nullptr, nullptr, D->err,
                                 D->counters, st));
            MRF_TRY(learned_flag(D, Z, n, idx_out, o->fallback_thr, o->learned_edge != 0,
                                 o->cone, D->vlist, D->nlist, st));
        }
        if (D->sync_free && D->bop && !o->certify)
            return exhaustive_on_list(D, Z, static_cast<int32_t>(n), o, idx_out, rho_out, X_out, st);
        int32_t cnt = 0;
        MRF_CUDA_TRY(cudaMemcpyAsync(&cnt, D->nlist, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        if (cnt > 0) MRF_TRY(exhaustive_on_list(D, Z, cnt, o, idx_out, rho_out, X_out, st));
        return MRF_OK;
    }
    return fail(MRF_EUNSUPPORTED, "projection mode not available in this build");
}
}  // namespace

// Projection with the dictionary's phase alignment applied when it has one: queries rotated by
// their v1 phase for the real cone (into the FFT workspace), densities mapped back to the atoms
// as given, and the voxel phase restored in X.
mrf_status project_core(mrf_dict* D, const float2* Z, int64_t n, const mrf_proj_opts* o,
                        const int32_t* warm, int32_t* idx_out, float2* rho_out, float2* X_out,
                        bool zq_ready, cudaStream_t st) {
    if (!D->aligned || n == 0)
        return project_impl(D, Z, n, o, warm, idx_out, rho_out, X_out, zq_ready, st);
    MRF_TRY(ensure_scratch(D, n));
    const bool realc = (o->cone == MRF_CONE_REAL_POS);
    const float2* Zs = Z;
    if (realc) {
        MRF_TRY(launch_align_queries(D, Z, n, D->wbuf, D->qph, st));
        Zs = D->wbuf;
        zq_ready = false;
    }
    MRF_TRY(project_impl(D, Zs, n, o, warm, idx_out, rho_out, X_out, zq_ready, st));
    return launch_align_post(D, n, idx_out, realc ? D->qph : nullptr, rho_out,
                             realc ? X_out : nullptr, st);
}

// Z = X - mu (A^H A X - AHY) for one slice: W is an n x L FFT workspace, zq (optional) receives
// the BF16 query operand of Z.
mrf_status gradient_to(const mrf_op* op, const float2* AHY, const float2* X, float mu, float2* Z,
                       float2* W, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st) {
    const int64_t n = static_cast<int64_t>(op->Ny) * op->Nx;
    if (grad_fused_supported(op->Ny)) {          // one pass: y-transforms, mask, combine
        ProfScope ps0(0, 1, st);
        return launch_grad_fused(op, AHY, X, mu, Z, zq, Kp, err, st);
    }
    if (grad_multi_supported(op->Ny)) {          // the same pass with mixed-radix transforms
        ProfScope ps0(0, 1, st);
        return launch_grad_mixed(op, AHY, X, mu, Z, zq, Kp, err, st);
    }
    cufftHandle hy;
    MRF_TRY(get_plan(0, op->Ny, op->Nx, op->L, st, &hy));
    ProfScope ps0(0, 2, st);
    MRF_TRY(fft_exec(hy, X, W, CUFFT_FORWARD));
    MRF_TRY(launch_mask_ky(W, op->mask, op->Ny, op->Nx, op->L, st));
    MRF_TRY(fft_exec(hy, W, W, CUFFT_INVERSE));
    MRF_TRY(launch_grad_combine(X, W, AHY, Z, n, op->L, mu, 1.0f / static_cast<float>(op->Ny), zq,
                                Kp, err, st));
    return MRF_OK;
}

namespace {

// Z = X - mu (A^H A X - AHY) into D->zbuf (and its BF16 operand when `want_zq`).
mrf_status gradient(mrf_dict* D, const mrf_op* op, const float2* AHY, const float2* X, float mu,
                    bool want_zq, cudaStream_t st) {
    return gradient_to(op, AHY, X, mu, D->zbuf, D->wbuf, want_zq ? D->zq : nullptr, D->Kp,
                       D->err, st);
}

double read_red(mrf_dict* D, int i, cudaStream_t st, mrf_status* s) {
    double v = 0.0;
    if (cudaMemcpyAsync(&v, D->red + i, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *s = fail(MRF_ECUDA, "reading a device reduction failed");
    }
    return v;
}

}  // namespace

// ================================================================================ C ABI
extern "C" {

const char* mrf_last_error(void) { return g_last_error.c_str(); }

const char* mrf_status_str(mrf_status s) {
    switch (s) {
        case MRF_OK: return "MRF_OK";
        case MRF_EINVAL: return "MRF_EINVAL";
        case MRF_ENOMEM: return "MRF_ENOMEM";
        case MRF_ECUDA: return "MRF_ECUDA";
        case MRF_ENONFINITE: return "MRF_ENONFINITE";
        case MRF_ETIMEOUT: return "MRF_ETIMEOUT";
        case MRF_EUNSUPPORTED: return "MRF_EUNSUPPORTED";
        case MRF_EINTERNAL: return "MRF_EINTERNAL";
    }
    return "MRF_UNKNOWN";
}

void mrf_default_index_opts(mrf_index_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->pack_bf16 = 1;
    o->tree_cone = MRF_CONE_COMPLEX;
    o->tree_dup_tol = 1e-5f;
}

void mrf_default_proj_opts(mrf_proj_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = MRF_PROJ_FP32_EXACT;
    o->cone = MRF_CONE_COMPLEX;
    o->topk = 0;
    o->certify = 1;
    o->tie_tol = 1e-5f;
    o->cert_margin = 0.f;
    o->eps = 0.f;
    o->fallback_thr = 0.98f;
    o->tree_route = 0.9f;
    o->learned_edge = 1;
}

void mrf_default_recon_opts(mrf_recon_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->iters = 10;
    o->mu = 1.f;
    o->zeta = 2.f;
    o->max_shrink = 30;
    mrf_default_proj_opts(&o->proj);
}

void mrf_dict_free(mrf_dict* D) {
    if (!D) return;
    if (D->ttc) ttc_free(D->ttc);
    if (D->tree) ct_free(D->tree);
    if (D->mlp) mlp_detach(D->mlp);
    void* ptrs[] = {D->atoms, D->inv_norm2, D->inv_norm, D->norm2, D->params, D->bop, D->zq, D->fop,
                    D->zq8, D->qs8, D->bop3, D->zq3, D->zmarg, D->v1, D->ealign, D->qph, D->zbuf,
                    D->wbuf, D->xprev, D->vlist, D->vlist2, D->nlist, D->part, D->err,
                    D->counters, D->red};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete D;
}

mrf_status mrf_build_dict_index(const void* atoms, int64_t d, int32_t L, const float* params,
                                int32_t P, const int32_t* grid_shape, int32_t grid_ndim,
                                const mrf_index_opts* opts, mrf_dict** out, void* stream) {
    if (!out) return fail(MRF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!atoms) return fail(MRF_EINVAL, "atoms is NULL");
    if (d < 1 || L < 1 || L > 4096) return fail(MRF_EINVAL, "need d >= 1 and 1 <= L <= 4096");
    if (d > INT32_MAX) return fail(MRF_EINVAL, "d exceeds the int32 index range");
    if (P < 0 || (P > 0 && !params)) return fail(MRF_EINVAL, "params / P mismatch");
    if (grid_ndim < 0 || (grid_ndim > 0 && !grid_shape)) return fail(MRF_EINVAL, "grid_shape");
    mrf_index_opts o;
    if (opts) o = *opts; else mrf_default_index_opts(&o);
    if (o.build_tree && o.tree_cone != MRF_CONE_COMPLEX && o.tree_cone != MRF_CONE_REAL_POS)
        return fail(MRF_EINVAL, "tree_cone must be a mrf_cone");
    if (o.build_tree && !(o.tree_dup_tol >= 0.f)) return fail(MRF_EINVAL, "tree_dup_tol < 0");
    if (o.tree_tc && !o.build_tree) return fail(MRF_EINVAL, "tree_tc needs build_tree");
    if (o.tree_tc && !o.pack_bf16 && !o.pack_bf16x3)
        return fail(MRF_EINVAL, "tree_tc needs pack_bf16 or pack_bf16x3");
    cudaStream_t st = S_(stream);
    mrf_dict* D = new mrf_dict();
    D->d = d;
    D->L = L;
    D->P = P;
    for (int i = 0; i < grid_ndim; ++i) D->grid_shape.push_back(grid_shape[i]);
    cudaGetDevice(&D->device);
    cudaDeviceGetAttribute(&D->num_sms, cudaDevAttrMultiProcessorCount, D->device);
    mrf_status s = MRF_OK;
    auto bail = [&](mrf_status e) { mrf_dict_free(D); return e; };
    if ((s = dalloc(&D->atoms, static_cast<size_t>(d * L))) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->inv_norm2, static_cast<size_t>(d))) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->inv_norm, static_cast<size_t>(d))) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->norm2, static_cast<size_t>(d))) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->err, 1)) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->counters, CNT_N)) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->red, 8)) != MRF_OK) return bail(s);
    if ((s = dalloc(&D->nlist, 2)) != MRF_OK) return bail(s);
    if (P > 0 && (s = dalloc(&D->params, static_cast<size_t>(d * P))) != MRF_OK) return bail(s);
    auto cuda_bail = [&](cudaError_t e, const char* what) {
        mrf_set_error(std::string(what) + ": " + cudaGetErrorString(e));
        mrf_dict_free(D);
        return MRF_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMemcpyAsync(D->atoms, atoms, sizeof(float2) * d * L, cudaMemcpyDefault, st)))
        return cuda_bail(e, "copy atoms");
    if (P > 0 && (e = cudaMemcpyAsync(D->params, params, sizeof(float) * d * P,
                                      cudaMemcpyDefault, st)))
        return cuda_bail(e, "copy params");
    if ((e = cudaMemsetAsync(D->err, 0, sizeof(uint32_t), st))) return cuda_bail(e, "memset");
    if ((e = cudaMemsetAsync(D->counters, 0, sizeof(unsigned long long) * CNT_N, st)))
        return cuda_bail(e, "memset");
    if ((s = launch_atom_norms(D, st)) != MRF_OK) return bail(s);
    if (o.phase_align && (s = phase_align_dictionary(D, st)) != MRF_OK) return bail(s);
    D->nblk = (d + 127) / 128;
    D->Kp = ((2 * L + 15) / 16) * 16;
    if (o.pack_bf16) {
        if ((s = dalloc(&D->bop, static_cast<size_t>(D->nblk * 256 * D->Kp))) != MRF_OK)
            return bail(s);
        if ((s = launch_pack_bop(D, st)) != MRF_OK) return bail(s);
    }
    if (o.pack_bf16x3) {
        D->Kp3 = 3 * D->Kp;
        if ((s = dalloc(&D->bop3, static_cast<size_t>(D->nblk * 256 * D->Kp3))) != MRF_OK)
            return bail(s);
        if ((s = launch_pack_bop3(D, st)) != MRF_OK) return bail(s);
    }
    if (o.pack_fp8) {
        D->Kp8 = ((2 * L + 31) / 32) * 32;
        if ((s = dalloc(&D->fop, static_cast<size_t>(D->nblk * 256 * D->Kp8))) != MRF_OK)
            return bail(s);
        // one power of two for the whole normalised dictionary: its largest magnitude m goes to
        // (224, 448]
        unsigned int mb = 0;
        unsigned int* dmb = reinterpret_cast<unsigned int*>(D->red);
        if ((e = cudaMemsetAsync(dmb, 0, sizeof(unsigned int), st))) return cuda_bail(e, "memset");
        if ((s = launch_atoms_absmax(D, dmb, st)) != MRF_OK) return bail(s);
        if ((e = cudaMemcpyAsync(&mb, dmb, sizeof(mb), cudaMemcpyDeviceToHost, st)))
            return cuda_bail(e, "read atom maximum");
        if ((e = cudaStreamSynchronize(st))) return cuda_bail(e, "atom maximum");
        float m;
        std::memcpy(&m, &mb, sizeof(m));
        float sg = 1.f;
        if (m > 0.f && std::isfinite(m)) {
            int ex = std::ilogb(448.f / m);
            ex = ex > 126 ? 126 : (ex < -126 ? -126 : ex);
            sg = std::ldexp(1.f, ex);
        }
        D->g8 = 1.f / sg;
        if ((s = launch_pack_fop(D, sg, st)) != MRF_OK) return bail(s);
    }
    uint32_t werr = 0;
    if ((e = cudaMemcpyAsync(&werr, D->err, sizeof(werr), cudaMemcpyDeviceToHost, st)))
        return cuda_bail(e, "read error word");
    if ((e = cudaStreamSynchronize(st))) return cuda_bail(e, "build");
    if (werr & MRF_DERR_NONFINITE) {
        mrf_set_error("an atom has a zero or non-finite norm");
        mrf_dict_free(D);
        return MRF_ENONFINITE;
    }
    if (o.build_tree) {
        s = ct_build_upload(D, o.tree_cone == MRF_CONE_COMPLEX ? 0 : 1, o.tree_dup_tol);
        if (s != MRF_OK) { mrf_dict_free(D); return s; }
        if (o.tree_tc) {
            s = ttc_build(D, st);
            if (s != MRF_OK) { mrf_dict_free(D); return s; }
        }
    }
    *out = D;
    return MRF_OK;
}

mrf_status mrf_tree_get_info(const mrf_dict* D, mrf_tree_info* info) {
    if (!D || !info) return fail(MRF_EINVAL, "dict and info are required");
    return ct_info(D, info);
}

mrf_status mrf_tree_blocks(const mrf_dict* D, int64_t* nblk, float* radius, int32_t* perm) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    return ttc_blocks(D, nblk, radius, perm);
}

mrf_status mrf_tree_export(const mrf_dict* D, int32_t* first_level, int32_t* parent,
                           int32_t* rep, int32_t* en_atom, int32_t* en_level, float* en_maxdist) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    return ct_export(D, first_level, parent, rep, en_atom, en_level, en_maxdist);
}

mrf_status mrf_dict_info(const mrf_dict* D, int64_t* d, int32_t* L, int32_t* P) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    if (d) *d = D->d;
    if (L) *L = D->L;
    if (P) *P = D->P;
    return MRF_OK;
}

mrf_status mrf_dict_reserve(mrf_dict* D, int64_t n_max) {
    if (!D || n_max < 0) return fail(MRF_EINVAL, "bad dict or n_max");
    MRF_TRY(ensure_scratch(D, n_max));
    return MRF_OK;
}

mrf_status mrf_dict_check(mrf_dict* D, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    cudaStream_t st = S_(stream);
    mrf_status s = read_stats(D, 0, nullptr, st);
    MRF_CUDA_TRY(cudaMemsetAsync(D->err, 0, sizeof(uint32_t), st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

mrf_status mrf_project(mrf_dict* D, const void* Z, int64_t n, const mrf_proj_opts* opts,
                       const int32_t* warm_idx, int32_t* idx_out, void* rho_out, void* X_out,
                       mrf_stats* stats, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    if (n < 0 || n > INT32_MAX) return fail(MRF_EINVAL, "n out of range");
    if (n > 0 && (!Z || !idx_out)) return fail(MRF_EINVAL, "Z and idx_out are required");
    mrf_proj_opts o;
    if (opts) o = *opts; else mrf_default_proj_opts(&o);
    MRF_TRY(check_proj_opts(D, &o));
    cudaStream_t st = S_(stream);
    if (stats) MRF_CUDA_TRY(cudaMemsetAsync(D->counters, 0, sizeof(unsigned long long) * CNT_N, st));
    MRF_TRY(project_core(D, static_cast<const float2*>(Z), n, &o, warm_idx, idx_out,
                         static_cast<float2*>(rho_out), static_cast<float2*>(X_out), false, st));
    if (stats) return read_stats(D, n, stats, st);
    return MRF_OK;
}

mrf_status mrf_search_candidates(mrf_dict* D, const void* Z, int64_t n,
                                 const mrf_proj_opts* opts, float* score_out, int32_t* idx_out,
                                 float* bound_out, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    if (n < 0 || n > INT32_MAX) return fail(MRF_EINVAL, "n out of range");
    mrf_proj_opts o;
    if (opts) o = *opts; else mrf_default_proj_opts(&o);
    MRF_TRY(check_proj_opts(D, &o));
    if (o.mode != MRF_PROJ_BF16 && o.mode != MRF_PROJ_FP8 && o.mode != MRF_PROJ_BF16X3)
        return fail(MRF_EINVAL, "candidate lists exist for the tensor-core modes only");
    if (n == 0) return MRF_OK;
    if (!Z || !score_out || !idx_out) return fail(MRF_EINVAL, "Z, score_out and idx_out are required");
    cudaStream_t st = S_(stream);
    const int K = topk_slots(&o);
    MRF_TRY(ensure_scratch(D, n));
    MRF_TRY(ensure_part(D, n, 1, K));
    float* ps = static_cast<float*>(D->part);
    int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(n) * K);
    const float2* z = static_cast<const float2*>(Z);
    if (o.mode == MRF_PROJ_BF16X3) {
        MRF_TRY(launch_pack_queries_x3(z, n, D, 0.f, D->zq3, bound_out ? bound_out : D->zmarg, st));
        MRF_TRY(launch_x3_topk(D->zq3, n, D, o.cone, K, 1, ps, pi, st));
    } else if (o.mode == MRF_PROJ_FP8) {
        MRF_TRY(launch_pack_queries_fp8(z, nullptr, n, D->L, D->Kp8, D->zq8, D->qs8, st));
        MRF_TRY(launch_fp8_topk(D->zq8, D->qs8, n, D, o.cone, K, 1, ps, pi, st));
        float b;
        fp8_margin(D, &kRigorous, &b);
        if (bound_out) MRF_TRY(launch_fill(bound_out, n, b, st));
    } else {
        MRF_TRY(launch_pack_queries(z, n, D->L, D->Kp, D->zq, st));
        MRF_TRY(launch_bf16_topk(D->zq, n, D, o.cone, K, 1, ps, pi, st));
        float b;
        bf16_margin(D, &kRigorous, &b);
        if (bound_out) MRF_TRY(launch_fill(bound_out, n, b, st));
    }
    MRF_CUDA_TRY(cudaMemcpyAsync(score_out, ps, sizeof(float) * n * K, cudaMemcpyDeviceToDevice, st));
    MRF_CUDA_TRY(cudaMemcpyAsync(idx_out, pi, sizeof(int32_t) * n * K, cudaMemcpyDeviceToDevice, st));
    return MRF_OK;
}

mrf_status mrf_forward(const mrf_op* op, const void* X, void* Y, void* stream) {
    MRF_TRY(check_op(op));
    if (!X || !Y) return fail(MRF_EINVAL, "X and Y are required");
    cudaStream_t st = S_(stream);
    cufftHandle h2;
    MRF_TRY(get_plan(1, op->Ny, op->Nx, op->L, st, &h2));
    MRF_TRY(fft_exec(h2, static_cast<const float2*>(X), static_cast<float2*>(Y), CUFFT_FORWARD));
    MRF_TRY(launch_mask_ky(static_cast<float2*>(Y), op->mask, op->Ny, op->Nx, op->L, st));
    const int64_t cnt = static_cast<int64_t>(op->Ny) * op->Nx * op->L;
    MRF_TRY(launch_scale(static_cast<float2*>(Y), cnt,
                         1.0f / std::sqrt(static_cast<float>(op->Ny) * op->Nx), st));
    return MRF_OK;
}

mrf_status mrf_adjoint(const mrf_op* op, const void* Y, void* AHY, void* stream) {
    MRF_TRY(check_op(op));
    if (!Y || !AHY) return fail(MRF_EINVAL, "Y and AHY are required");
    cudaStream_t st = S_(stream);
    const int64_t cnt = static_cast<int64_t>(op->Ny) * op->Nx * op->L;
    if (AHY != Y)
        MRF_CUDA_TRY(cudaMemcpyAsync(AHY, Y, sizeof(float2) * cnt, cudaMemcpyDeviceToDevice, st));
    MRF_TRY(launch_mask_ky(static_cast<float2*>(AHY), op->mask, op->Ny, op->Nx, op->L, st));
    cufftHandle h2;
    MRF_TRY(get_plan(1, op->Ny, op->Nx, op->L, st, &h2));
    MRF_TRY(fft_exec(h2, static_cast<float2*>(AHY), static_cast<float2*>(AHY), CUFFT_INVERSE));
    MRF_TRY(launch_scale(static_cast<float2*>(AHY), cnt,
                         1.0f / std::sqrt(static_cast<float>(op->Ny) * op->Nx), st));
    return MRF_OK;
}

mrf_status mrf_gradient(mrf_dict* D, const mrf_op* op, const void* AHY, const void* X,
                        float mu, void* Z, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    MRF_TRY(check_op(op));
    if (op->L != D->L) return fail(MRF_EINVAL, "op->L differs from the dictionary's L");
    if (!AHY || !X || !Z) return fail(MRF_EINVAL, "AHY, X and Z are required");
    if (!std::isfinite(mu)) return fail(MRF_EINVAL, "mu must be finite");
    cudaStream_t st = S_(stream);
    const int64_t n = static_cast<int64_t>(op->Ny) * op->Nx;
    MRF_TRY(ensure_scratch(D, n));
    MRF_TRY(gradient(D, op, static_cast<const float2*>(AHY), static_cast<const float2*>(X), mu,
                     false, st));
    MRF_CUDA_TRY(cudaMemcpyAsync(Z, D->zbuf, sizeof(float2) * n * op->L, cudaMemcpyDeviceToDevice,
                                 st));
    return MRF_OK;
}

mrf_status mrf_ipg_step(mrf_dict* D, const mrf_op* op, const void* AHY, void* X, float mu,
                        const mrf_proj_opts* opts, int32_t* idx_io, void* rho_out,
                        mrf_stats* stats, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    MRF_TRY(check_op(op));
    if (op->L != D->L) return fail(MRF_EINVAL, "op->L differs from the dictionary's L");
    if (!AHY || !X || !idx_io) return fail(MRF_EINVAL, "AHY, X and idx_io are required");
    if (!std::isfinite(mu)) return fail(MRF_EINVAL, "mu must be finite");
    mrf_proj_opts o;
    if (opts) o = *opts; else mrf_default_proj_opts(&o);
    MRF_TRY(check_proj_opts(D, &o));
    cudaStream_t st = S_(stream);
    const int64_t n = static_cast<int64_t>(op->Ny) * op->Nx;
    MRF_TRY(ensure_scratch(D, n));
    if (stats) MRF_CUDA_TRY(cudaMemsetAsync(D->counters, 0, sizeof(unsigned long long) * CNT_N, st));
    const bool zq = (o.mode == MRF_PROJ_BF16);
    MRF_TRY(gradient(D, op, static_cast<const float2*>(AHY), static_cast<const float2*>(X), mu,
                     zq, st));
    MRF_TRY(project_core(D, D->zbuf, n, &o, idx_io, idx_io, static_cast<float2*>(rho_out),
                         static_cast<float2*>(X), zq, st));
    if (stats) return read_stats(D, n, stats, st);
    return MRF_OK;
}

mrf_status mrf_lut(const mrf_dict* D, const int32_t* idx, int64_t n, float* params_out,
                   void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    if (D->P == 0) return fail(MRF_EINVAL, "dictionary has no parameter table");
    if (n > 0 && (!idx || !params_out)) return fail(MRF_EINVAL, "idx and params_out required");
    ProfScope ps6(6, 1, S_(stream));
    return launch_lut(idx, n, D->params, D->P, D->d, params_out, D->err, S_(stream));
}

mrf_status mrf_get_tune(const mrf_dict* D, mrf_tune* out) {
    if (!D || !out) return fail(MRF_EINVAL, "dict and out are required");
    *out = D->tune;
    return MRF_OK;
}

mrf_status mrf_set_tune(mrf_dict* D, const mrf_tune* in) {
    if (!D || !in) return fail(MRF_EINVAL, "dict and in are required");
    if (in->bf16_cluster != 0 && in->bf16_cluster != 1 && in->bf16_cluster != 2 &&
        in->bf16_cluster != 4)
        return fail(MRF_EINVAL, "bf16_cluster must be 0, 1, 2 or 4");
    if (in->bf16_live_tiles < 0 || in->bf16_splits < 0 || in->fp32_splits < 0 ||
        in->bf16_splits > 4096 || in->fp32_splits > 4096)
        return fail(MRF_EINVAL, "tuning values out of range");
    if (in->tree_list_cap != 0 && (in->tree_list_cap < 64 || in->tree_list_cap > 512))
        return fail(MRF_EINVAL, "tree_list_cap must be 0 or in 64..512");
    if (in->bf16_pair < 0 || in->bf16_pair > 2) return fail(MRF_EINVAL, "bf16_pair must be 0, 1 or 2");
    if (in->tree_order < 0 || in->tree_order > 2) return fail(MRF_EINVAL, "tree_order must be 0, 1 or 2");
    if (in->tree_tc_group < 0 || in->tree_tc_group > 64)
        return fail(MRF_EINVAL, "tree_tc_group must be in 0..64");
    if (in->tree_tc_chunks < 0 || in->tree_tc_chunks > 64)
        return fail(MRF_EINVAL, "tree_tc_chunks must be in 0..64");
    if (in->tree_tc_super < 0 || in->tree_tc_super > 256)
        return fail(MRF_EINVAL, "tree_tc_super must be in 0..256");
    // all values checked: none is applied when one is refused
    D->tune.tree_list_cap = in->tree_list_cap;
    D->tune.bf16_pair = in->bf16_pair;
    D->tune.tree_order = in->tree_order;
    D->tune.tree_tc_group = in->tree_tc_group;
    D->tune.tree_tc_chunks = in->tree_tc_chunks;
    D->tune.tree_tc_super = in->tree_tc_super;
    D->tune.bf16_cluster = in->bf16_cluster;
    D->tune.bf16_live_tiles = in->bf16_live_tiles;
    D->tune.bf16_splits = in->bf16_splits;
    D->tune.fp32_splits = in->fp32_splits;
    return MRF_OK;
}

mrf_status mrf_profile_enable(int32_t on) {
    prof_clear();
    g_prof_on = on != 0;
    return MRF_OK;
}

mrf_status mrf_profile_read(double* ms, int64_t* launches, int32_t n_stages) {
    if (n_stages < 0 || (n_stages > 0 && (!ms || !launches)))
        return fail(MRF_EINVAL, "ms/launches required");
    for (auto& e : g_prof_pending) {
        float t = 0.f;
        if (cudaEventSynchronize(e.b) != cudaSuccess ||
            cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) {
            cudaGetLastError();
            prof_clear();
            return fail(MRF_ECUDA, "reading profiler events failed");
        }
        g_prof_ms[e.stage] += t;
        g_prof_launch[e.stage] += e.launches;
    }
    for (int i = 0; i < n_stages && i < MRF_PROFILE_STAGES; ++i) {
        ms[i] = g_prof_ms[i];
        launches[i] = g_prof_launch[i];
    }
    prof_clear();
    return MRF_OK;
}

namespace {
mrf_status reconstruct_dev(mrf_dict* D, const mrf_op* op, const void* Y,
                           const mrf_recon_opts* ropts, void* X_out, int32_t* idx_out,
                           void* rho_out, float* params_out, mrf_stats* stats, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    MRF_TRY(check_op(op));
    if (op->L != D->L) return fail(MRF_EINVAL, "op->L differs from the dictionary's L");
    if (!Y || !X_out || !idx_out) return fail(MRF_EINVAL, "Y, X_out and idx_out are required");
    mrf_recon_opts r;
    if (ropts) r = *ropts; else mrf_default_recon_opts(&r);
    if (r.iters < 0 || !(r.mu > 0.f) || (r.adaptive && !(r.zeta > 1.f)) || r.max_shrink < 0 ||
        r.resume < 0 || r.resume > 1)
        return fail(MRF_EINVAL, "bad reconstruction options");
    MRF_TRY(check_proj_opts(D, &r.proj));
    if (params_out && D->P == 0) return fail(MRF_EINVAL, "dictionary has no parameter table");
    cudaStream_t st = S_(stream);
    const int64_t n = static_cast<int64_t>(op->Ny) * op->Nx;
    const int64_t cnt = n * op->L;
    MRF_TRY(ensure_scratch(D, n));
    if ((r.adaptive || r.kappa || r.tol > 0.f) && !D->xprev)
        MRF_TRY(dalloc(&D->xprev, static_cast<size_t>(cnt)));
    // scratch: AHY in a dedicated buffer (the gradient uses zbuf and wbuf)
    float2* AHY = nullptr;
    MRF_TRY(dalloc(&AHY, static_cast<size_t>(cnt)));
    float2* rho = static_cast<float2*>(rho_out);
    float2* rho_tmp = nullptr;
    if (!rho) {
        mrf_status s = dalloc(&rho_tmp, static_cast<size_t>(n));
        if (s != MRF_OK) { cudaFree(AHY); return s; }
        rho = rho_tmp;
    }
    float2* X = static_cast<float2*>(X_out);
    const bool zq = (r.proj.mode == MRF_PROJ_BF16);
    mrf_status s = MRF_OK;
    auto body = [&]() -> mrf_status {
        MRF_CUDA_TRY(cudaMemsetAsync(D->counters, 0, sizeof(unsigned long long) * CNT_N, st));
        MRF_TRY(mrf_adjoint(op, Y, AHY, stream));
        if (!r.resume) {
            MRF_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(float2) * cnt, st));
            MRF_CUDA_TRY(cudaMemsetAsync(idx_out, 0, sizeof(int32_t) * n, st));
        }
        double ynorm2 = -1.0, prev_obj = -1.0;
        float mu0 = r.mu;
        for (int k = 0; k < r.iters; ++k) {
            float mu_k = mu0;
            if (r.adaptive || r.kappa || r.tol > 0.f)
                MRF_CUDA_TRY(cudaMemcpyAsync(D->xprev, X, sizeof(float2) * cnt,
                                             cudaMemcpyDeviceToDevice, st));
            int shrinks_k = 0;
            for (int shrink = 0;; ++shrink) {
                shrinks_k = shrink;
                MRF_TRY(gradient(D, op, AHY, r.adaptive ? D->xprev : X, mu_k, zq, st));
                MRF_TRY(project_core(D, D->zbuf, n, &r.proj, idx_out, idx_out, rho, X, zq, st));
                if (!r.adaptive) break;
                // step rule (eq. steprule): accept when mu_k < ||dX||^2 / ||A dX||^2
                MRF_CUDA_TRY(cudaMemsetAsync(D->red, 0, sizeof(double) * 2, st));
                MRF_TRY(launch_sqdiff(X, D->xprev, cnt, D->red, st));
                MRF_CUDA_TRY(cudaMemcpyAsync(D->wbuf, X, sizeof(float2) * cnt,
                                             cudaMemcpyDeviceToDevice, st));
                MRF_TRY(launch_axpby(D->wbuf, D->xprev, cnt, 1.f, -1.f, st));
                MRF_TRY(mrf_forward(op, D->wbuf, D->zbuf, stream));
                MRF_TRY(launch_sqnorm(D->zbuf, cnt, D->red + 1, st));
                double num = read_red(D, 0, st, &s);
                double den = read_red(D, 1, st, &s);
                if (s != MRF_OK) return s;
                if (den == 0.0 || static_cast<double>(mu_k) < num / den || shrink >= r.max_shrink)
                    break;
                mu_k /= r.zeta;
            }
            if (r.mu_history) r.mu_history[k] = mu_k;
            if (r.shrink_history) r.shrink_history[k] = shrinks_k;
            if (r.kappa && k == 0 && !r.resume) {
                if (ynorm2 < 0.0) {
                    MRF_CUDA_TRY(cudaMemsetAsync(D->red + 2, 0, sizeof(double), st));
                    MRF_TRY(launch_sqnorm(static_cast<const float2*>(Y), cnt, D->red + 2, st));
                    ynorm2 = read_red(D, 2, st, &s);
                }
                MRF_TRY(mrf_forward(op, X, D->zbuf, stream));
                MRF_CUDA_TRY(cudaMemsetAsync(D->red + 3, 0, sizeof(double), st));
                MRF_TRY(launch_sqnorm(D->zbuf, cnt, D->red + 3, st));
                double ax = read_red(D, 3, st, &s);
                if (s != MRF_OK) return s;
                if (ax > 0.0) {
                    float kap = static_cast<float>(std::sqrt(ynorm2 / ax));
                    MRF_TRY(launch_scale(X, cnt, kap, st));
                    MRF_TRY(launch_scale(rho, n, kap, st));
                    mu0 *= kap;
                }
            }
            if (r.tol > 0.f) {
                // objective ||Y - A X||^2 (Y is zero off the sampled lines after masking)
                MRF_TRY(mrf_forward(op, X, D->zbuf, stream));
                MRF_CUDA_TRY(cudaMemcpyAsync(D->wbuf, Y, sizeof(float2) * cnt,
                                             cudaMemcpyDeviceToDevice, st));
                MRF_TRY(launch_mask_ky(D->wbuf, op->mask, op->Ny, op->Nx, op->L, st));
                MRF_CUDA_TRY(cudaMemsetAsync(D->red + 4, 0, sizeof(double), st));
                MRF_TRY(launch_sqdiff(D->wbuf, D->zbuf, cnt, D->red + 4, st));
                double obj = read_red(D, 4, st, &s);
                if (s != MRF_OK) return s;
                if (prev_obj > 0.0 && std::fabs(prev_obj - obj) / prev_obj < r.tol) break;
                prev_obj = obj;
            }
        }
        if (params_out) MRF_TRY(mrf_lut(D, idx_out, n, params_out, stream));
        return MRF_OK;
    };
    s = body();
    mrf_status s2 = read_stats(D, n, stats, st);
    cudaFree(AHY);
    if (rho_tmp) cudaFree(rho_tmp);
    if (s != MRF_OK) return s;
    return s2;
}

// Host memory (pinned or pageable) as opposed to memory a kernel of this device can address.
bool is_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}
}  // namespace

// Whole reconstruction; host buffers (pinned or pageable) among Y and the outputs are staged
// through device buffers allocated for the call, with every copy inside the call.
mrf_status mrf_reconstruct(mrf_dict* D, const mrf_op* op, const void* Y,
                           const mrf_recon_opts* ropts, void* X_out, int32_t* idx_out,
                           void* rho_out, float* params_out, mrf_stats* stats, void* stream) {
    if (!D) return fail(MRF_EINVAL, "dict is NULL");
    MRF_TRY(check_op(op));
    if (!Y || !X_out || !idx_out) return fail(MRF_EINVAL, "Y, X_out and idx_out are required");
    const bool hY = is_host_ptr(Y), hX = is_host_ptr(X_out), hI = is_host_ptr(idx_out);
    const bool hR = rho_out && is_host_ptr(rho_out);
    const bool hP = params_out && is_host_ptr(params_out);
    if (!hY && !hX && !hI && !hR && !hP)
        return reconstruct_dev(D, op, Y, ropts, X_out, idx_out, rho_out, params_out, stats, stream);
    cudaStream_t st = S_(stream);
    const int64_t n = static_cast<int64_t>(op->Ny) * op->Nx;
    const size_t cnt = static_cast<size_t>(n) * op->L;
    const bool resume = ropts && ropts->resume;
    float2 *dY = nullptr, *dX = nullptr, *dR = nullptr;
    int32_t* dI = nullptr;
    float* dP = nullptr;
    auto release = [&]() {
        void* ptrs[] = {dY, dX, dR, dI, dP};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    };
    mrf_status s = MRF_OK;
    auto run = [&]() -> mrf_status {
        if (hY) MRF_TRY(dalloc(&dY, cnt));
        if (hX) MRF_TRY(dalloc(&dX, cnt));
        if (hI) MRF_TRY(dalloc(&dI, static_cast<size_t>(n)));
        if (hR) MRF_TRY(dalloc(&dR, static_cast<size_t>(n)));
        if (hP) MRF_TRY(dalloc(&dP, static_cast<size_t>(n) * (D->P > 0 ? D->P : 1)));
        if (hY) MRF_CUDA_TRY(cudaMemcpyAsync(dY, Y, sizeof(float2) * cnt, cudaMemcpyHostToDevice, st));
        if (hX && resume)
            MRF_CUDA_TRY(cudaMemcpyAsync(dX, X_out, sizeof(float2) * cnt, cudaMemcpyHostToDevice, st));
        if (hI && resume)
            MRF_CUDA_TRY(cudaMemcpyAsync(dI, idx_out, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        MRF_TRY(reconstruct_dev(D, op, hY ? dY : Y, ropts, hX ? dX : X_out, hI ? dI : idx_out,
                                hR ? static_cast<void*>(dR) : rho_out, hP ? dP : params_out,
                                stats, stream));
        if (hX) MRF_CUDA_TRY(cudaMemcpyAsync(X_out, dX, sizeof(float2) * cnt, cudaMemcpyDeviceToHost, st));
        if (hI) MRF_CUDA_TRY(cudaMemcpyAsync(idx_out, dI, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        if (hR) MRF_CUDA_TRY(cudaMemcpyAsync(rho_out, dR, sizeof(float2) * n, cudaMemcpyDeviceToHost, st));
        if (hP)
            MRF_CUDA_TRY(cudaMemcpyAsync(params_out, dP, sizeof(float) * n * D->P,
                                         cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        return MRF_OK;
    };
    s = run();
    cudaStreamSynchronize(st);
    release();
    return s;
}

void mrf_debug_fail_alloc(int32_t k) { g_fail_alloc_after.store(k < 0 ? -1 : k); }

}  // extern "C"
