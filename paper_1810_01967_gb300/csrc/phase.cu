// Phase alignment for the real positive cone (§4.3: the heuristic that extends the paper's
// real-density projection to complex data).
//
// v1 is the dominant eigenvector of sum_j D_j D_j^H (the first principal component).  Every
// atom is rotated so that v1^H D_j is real positive (alpha_j = angle(v1^H D_j), the stored atom
// becomes D_j e^{-i alpha_j}); at every projection with the real cone each query is rotated the
// same way (beta_v = angle(v1^H Z_v)), the real positive projection runs on the aligned
// vectors, and the voxel's phase is restored: X_v = gamma e^{i beta_v} D'_j, i.e. the density
// relative to the atom as given is gamma e^{i (beta_v - alpha_j)}.  With the complex cone the
// alignment changes nothing but the reference phase of rho, which is mapped back to the atom
// as given.
#include "mrf_internal.cuh"

namespace {

constexpr int kT = 256;

inline unsigned warps_grid(int64_t rows) {
    return static_cast<unsigned>((rows * 32 + kT - 1) / kT);
}

__device__ __forceinline__ float2 unit_phase(float re, float im) {
    const float a = sqrtf(re * re + im * im);
    return a > 0.f ? make_float2(re / a, im / a) : make_float2(1.f, 0.f);
}

// One warp per row: e = (v1^H r) / |v1^H r|; row <- row conj(e) into `out`; ph[row] = e.
// (R and out may be the same array: each lane rewrites only the entries it read, after the
// warp-wide reduction.)
__global__ void k_align_rows(const float2* R, int64_t n, int L, const float2* __restrict__ v1,
                             float2* out, float2* __restrict__ ph) {
    const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float2* row = R + r * L;
    float re = 0.f, im = 0.f;
    for (int t = lane; t < L; t += 32) {
        const float2 v = v1[t], a = row[t];
        re = fmaf(v.x, a.x, fmaf(v.y, a.y, re));     // conj(v) a
        im = fmaf(v.x, a.y, fmaf(-v.y, a.x, im));
    }
    for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const float2 e = unit_phase(re, im);
    float2* dst = out + r * L;
    for (int t = lane; t < L; t += 32) {
        const float2 a = row[t];
        dst[t] = make_float2(a.x * e.x + a.y * e.y, a.y * e.x - a.x * e.y);   // a conj(e)
    }
    if (lane == 0) ph[r] = e;
}

// rho_v <- rho_v eb_v conj(ea_j) (eb absent: 1); X_v <- X_v eb_v when eb is given.
__global__ void k_align_post(int64_t n, int L, const int32_t* __restrict__ idx,
                             const float2* __restrict__ ea, const float2* __restrict__ eb,
                             float2* __restrict__ rho, float2* __restrict__ X) {
    const int64_t v = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const float2 b = eb ? eb[v] : make_float2(1.f, 0.f);
    if (rho && lane == 0) {
        const float2 a = ea[idx[v]];
        const float2 r = rho[v];
        const float2 rb = make_float2(r.x * b.x - r.y * b.y, r.x * b.y + r.y * b.x);
        rho[v] = make_float2(rb.x * a.x + rb.y * a.y, rb.y * a.x - rb.x * a.y);   // rb conj(a)
    }
    if (X && eb) {
        float2* x = X + v * L;
        for (int t = lane; t < L; t += 32) {
            const float2 a = x[t];
            x[t] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
        }
    }
}

mrf_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mrf_set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

}  // namespace

mrf_status phase_align_dictionary(mrf_dict* D, cudaStream_t st) {
    if (cudaMalloc(&D->v1, sizeof(float2) * D->L) != cudaSuccess ||
        cudaMalloc(&D->ealign, sizeof(float2) * D->d) != cudaSuccess) {
        cudaGetLastError();
        mrf_set_error("phase alignment allocation failed");
        return MRF_ENOMEM;
    }
    MRF_TRY(mrf_svd_basis(D, 1, D->v1, nullptr, st));
    k_align_rows<<<warps_grid(D->d), kT, 0, st>>>(D->atoms, D->d, D->L, D->v1, D->atoms, D->ealign);
    MRF_TRY(check_launch("phase alignment of the atoms"));
    D->aligned = true;
    return MRF_OK;
}

mrf_status launch_align_queries(const mrf_dict* D, const float2* Z, int64_t n, float2* Zout,
                                float2* eb, cudaStream_t st) {
    if (n == 0) return MRF_OK;
    k_align_rows<<<warps_grid(n), kT, 0, st>>>(Z, n, D->L, D->v1, Zout, eb);
    return check_launch("phase alignment of the queries");
}

mrf_status launch_align_post(const mrf_dict* D, int64_t n, const int32_t* idx, const float2* eb,
                             float2* rho, float2* X, cudaStream_t st) {
    if (n == 0 || (!rho && !(X && eb))) return MRF_OK;
    k_align_post<<<warps_grid(n), kT, 0, st>>>(n, D->L, idx, D->ealign, eb, rho, X);
    return check_launch("phase restoration");
}
