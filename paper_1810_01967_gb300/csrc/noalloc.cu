// Exhaustive FP32 projection whose working memory is a fixed, file-scope device array, so that a
// call allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// It exists for callers that are not allowed to allocate device memory after start-up, e.g.
// applications whose device memory is owned by their own pool or allocator, and real-time
// pipelines that forbid allocation once they are running.  It reuses the library's FP32 search
// and merge kernels unchanged; only where their scratch lives differs.
//
// The array (about 20 MB: candidates for 4096 voxels x 32 atom splits x 8, plus per-atom norms
// for up to 2^20 atoms, an error word and counters) is part of the library image, so every GPU
// that loads the library holds it until the process exits.  In host code the array's name is only
// a host-side stand-in; its device address is fetched once per device with
// cudaGetSymbolAddress, by the first call on that device, with that device current.
#include <mutex>

#include "mrf_internal.cuh"

namespace {

constexpr int64_t kMaxN = 4096;          // voxels per call
constexpr int64_t kMaxD = 1 << 20;       // atoms
constexpr int kMaxS = 32;                // atom splits of the FP32 search
constexpr int kK = 8;                    // candidates per voxel and split

constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t kPartBytes = align256(static_cast<size_t>(kMaxS) * kMaxN * kK * 8);
constexpr size_t kInvNormOff = kPartBytes;
constexpr size_t kNorm2Off = kInvNormOff + align256(kMaxD * sizeof(float));
constexpr size_t kErrOff = kNorm2Off + align256(kMaxD * sizeof(double));
constexpr size_t kCountOff = kErrOff + 256;
constexpr size_t kScratchBytes = kCountOff + align256(CNT_N * sizeof(unsigned long long));

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

mrf_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        mrf_set_error("device ordinal out of range for the static scratch table");
        return MRF_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            mrf_set_error(std::string("cudaGetSymbolAddress(static scratch): ") +
                          cudaGetErrorString(e));
            return MRF_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return MRF_OK;
}

}  // namespace

extern "C" mrf_status mrf_project_fp32_static(const void* atoms, int64_t d, int32_t L,
                                              const void* Z, int64_t n, int32_t cone,
                                              int32_t* idx_out, void* rho_out, void* X_out,
                                              void* stream) {
    if (!atoms) {
        mrf_set_error("atoms is NULL");
        return MRF_EINVAL;
    }
    if (d < 1 || d > kMaxD) {
        mrf_set_error("mrf_project_fp32_static: d must be in 1.." + std::to_string(kMaxD) +
                      " (the static scratch holds norms for at most that many atoms)");
        return MRF_EINVAL;
    }
    if (L < 1 || L > 4096) {
        mrf_set_error("mrf_project_fp32_static: L must be in 1..4096");
        return MRF_EINVAL;
    }
    if (n < 0 || n > kMaxN) {
        mrf_set_error("mrf_project_fp32_static: n must be in 0.." + std::to_string(kMaxN) +
                      " voxels per call (the static scratch is sized for that many)");
        return MRF_EINVAL;
    }
    if (cone != MRF_CONE_COMPLEX && cone != MRF_CONE_REAL_POS) {
        mrf_set_error("unknown cone");
        return MRF_EINVAL;
    }
    if (n > 0 && (!Z || !idx_out)) {
        mrf_set_error("Z and idx_out are required");
        return MRF_EINVAL;
    }
    if (n == 0) return MRF_OK;
    int dev = 0;
    MRF_CUDA_TRY(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    MRF_TRY(scratch_address(dev, &base));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // A host-side view of the dictionary pointing into the caller's atoms and the static array.
    mrf_dict view;
    view.d = d;
    view.L = L;
    view.device = dev;
    view.atoms = const_cast<float2*>(static_cast<const float2*>(atoms));
    view.inv_norm2 = reinterpret_cast<float*>(base + kInvNormOff);
    view.norm2 = reinterpret_cast<double*>(base + kNorm2Off);
    view.err = reinterpret_cast<uint32_t*>(base + kErrOff);
    view.counters = reinterpret_cast<unsigned long long*>(base + kCountOff);
    MRF_CUDA_TRY(cudaDeviceGetAttribute(&view.num_sms, cudaDevAttrMultiProcessorCount, dev));

    // the error word and counters keep the previous call's values: clear them first
    MRF_CUDA_TRY(cudaMemsetAsync(view.err, 0, sizeof(uint32_t), st));
    MRF_CUDA_TRY(cudaMemsetAsync(view.counters, 0, CNT_N * sizeof(unsigned long long), st));
    MRF_TRY(launch_atom_norms(&view, st));
    int S = fp32_choose_splits(n, d, view.num_sms);
    if (S > kMaxS) S = kMaxS;
    float* ps = reinterpret_cast<float*>(base);
    int32_t* pi = reinterpret_cast<int32_t*>(ps + static_cast<size_t>(S) * n * kK);
    MRF_TRY(launch_fp32_topk(static_cast<const float2*>(Z), nullptr, nullptr, n, &view, cone, kK,
                             S, ps, pi, st));
    MRF_TRY(launch_merge(static_cast<const float2*>(Z), n, &view, cone, kK, S, ps, pi, nullptr,
                         nullptr, 1e-5f, 0, 0.f, idx_out, static_cast<float2*>(rho_out),
                         static_cast<float2*>(X_out), nullptr, nullptr, view.err,
                         view.counters, st));
    uint32_t werr = 0;
    MRF_CUDA_TRY(cudaMemcpyAsync(&werr, view.err, sizeof(werr), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    if (werr & MRF_DERR_NONFINITE) {
        mrf_set_error("an atom has a zero or non-finite norm");
        return MRF_ENONFINITE;
    }
    if (werr) {
        mrf_set_error("device-side error word " + std::to_string(werr));
        return MRF_EINTERNAL;
    }
    return MRF_OK;
}
