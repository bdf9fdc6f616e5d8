// Elementwise and packing kernels around the projection: atom norms, BF16 and FP8 operand packing,
// the k-space line mask and the gradient-step combination of §3.2 eq. blip, the look-up table
// of Algorithm 2 and FP64 reductions used by the step rule (eq. steprule).
#include "mrf_internal.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void k_atom_norms(const float2* __restrict__ atoms, int64_t d, int L,
                             double* __restrict__ norm2, float* __restrict__ inv_norm2,
                             float* __restrict__ inv_norm, uint32_t* err) {
    int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (j >= d) return;
    const float2* a = atoms + j * L;
    double s = 0.0;
    for (int t = lane; t < L; t += 32) {
        float2 v = a[t];
        s += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        bool bad = !(s > 0.0) || !isfinite(s);
        if (bad) atomicOr(err, MRF_DERR_NONFINITE);
        norm2[j] = s;
        inv_norm2[j] = bad ? 0.f : static_cast<float>(1.0 / s);
        if (inv_norm) inv_norm[j] = bad ? 0.f : static_cast<float>(1.0 / sqrt(s));
    }
}

// Row r of block b: atom j = 128 b + (r mod 128); r < 128 holds (Re d, Im d) per frame,
// r >= 128 holds (-Im d, Re d), so that a query row (Re z, Im z) gives Re(d^H z) and Im(d^H z).
// Atom rows are normalised (D_j / ||D_j||, the FP64 norm) before rounding, so the kernels' scores
// need no per-atom weight.
// With `perm` (length nblk * 128) the operand slot p holds atom perm[p] (-1: an empty slot).
__global__ void k_pack_bop(const float2* __restrict__ atoms, const float* __restrict__ inv_norm,
                           int64_t d, int L, int Kp, int64_t nblk,
                           __nv_bfloat162* __restrict__ bop, const int32_t* __restrict__ perm) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t half = Kp / 2;
    int64_t total = nblk * 256 * half;
    if (i >= total) return;
    int64_t row = i / half;
    int t = static_cast<int>(i - row * half);
    int64_t b = row >> 8;
    int r = static_cast<int>(row & 255);
    int64_t j = b * 128 + (r & 127);
    if (perm) j = perm[j] < 0 ? d : perm[j];
    float2 v = make_float2(0.f, 0.f);
    if (j < d && t < L) {
        const float inv = inv_norm[j];
        v = atoms[j * L + t];
        v.x *= inv;
        v.y *= inv;
    }
    float x = (r < 128) ? v.x : -v.y;
    float y = (r < 128) ? v.y : v.x;
    bop[i] = __floats2bfloat162_rn(x, y);
}

__global__ void k_pack_queries(const float2* __restrict__ Z, int64_t n, int L, int Kp,
                               __nv_bfloat162* __restrict__ zq) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t half = Kp / 2;
    if (i >= n * half) return;
    int64_t v = i / half;
    int t = static_cast<int>(i - v * half);
    float2 z = (t < L) ? Z[v * L + t] : make_float2(0.f, 0.f);
    zq[i] = __floats2bfloat162_rn(z.x, z.y);
}

// Rows of the listed voxels; with `count` (device) only the first *count entries of the list
// are present and n is the list's capacity.
__global__ void k_pack_gather(const float2* __restrict__ Z, const int32_t* __restrict__ vlist,
                              const int32_t* __restrict__ count, int64_t n, int L, int Kp,
                              __nv_bfloat162* __restrict__ zq) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t half = Kp / 2;
    if (i >= n * half) return;
    int64_t k = i / half;
    if (count && k >= *count) return;
    int t = static_cast<int>(i - k * half);
    const int64_t v = vlist[k];
    float2 z = (t < L) ? Z[v * L + t] : make_float2(0.f, 0.f);
    zq[i] = __floats2bfloat162_rn(z.x, z.y);
}

// ----------------------------------------------------------------------------- FP8 (E4M3)
// Query rows are scaled by a power of two s chosen from the row's largest real or imaginary
// magnitude m so that s m lies in (224, 448] (448 is the largest finite E4M3 value); a zero row
// keeps s = 1.  Atoms use one such power of two for the whole (normalised) dictionary.  Each
// value is rounded to nearest with saturation.  The kernel multiplies the scores it keeps by
// the inverse factors, so FP8 scores are in the units of the BF16 ones.
__device__ __forceinline__ float e4m3_row_scale(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int e = ilogbf(448.f / m);
    e = e > 126 ? 126 : (e < -126 ? -126 : e);
    return ldexpf(1.f, e);
}

__device__ __forceinline__ uint16_t e4m3_pair(float x, float y) {
    const uint16_t lo = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
    const uint16_t hi = __nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
    return static_cast<uint16_t>(lo | (hi << 8));
}

__device__ __forceinline__ float warp_max(float x) {
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Largest real or imaginary magnitude of the normalised atoms (one warp per atom), as float
// bits in *m_bits (non-negative floats order like their bit patterns).
__global__ void k_atoms_absmax(const float2* __restrict__ atoms, const float* __restrict__ inv_norm,
                               int64_t d, int L, unsigned int* m_bits) {
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= d) return;
    const float inv = inv_norm[j];
    float m = 0.f;
    for (int t = lane; t < L; t += 32) {
        float2 v = atoms[j * L + t];
        m = fmaxf(m, fmaxf(fabsf(v.x * inv), fabsf(v.y * inv)));
    }
    m = warp_max(m);
    if (lane == 0 && isfinite(m)) atomicMax(m_bits, __float_as_uint(m));
}

// One warp per atom slot of the padded blocks: the two operand rows of the normalised atom (as
// in k_pack_bop) times the dictionary-wide power of two `s`, in E4M3.  With unit atoms the
// rows' norms are s >= 224 ... so every row keeps the relative accuracy of a per-row scale,
// and the kernel needs no per-atom weight.
__global__ void k_pack_fop(const float2* __restrict__ atoms, const float* __restrict__ inv_norm,
                           int64_t d, int L, int Kp8, int64_t nblk, float s,
                           uint16_t* __restrict__ fop) {
    const int64_t slot = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= nblk * 128) return;
    const int64_t b = slot >> 7;
    const int r = static_cast<int>(slot & 127);
    const int64_t j = slot;
    const bool real = j < d;
    const float inv = real ? inv_norm[j] : 0.f;
    const int half = Kp8 / 2;
    uint16_t* re_row = fop + (b * 256 + r) * half;
    uint16_t* im_row = fop + (b * 256 + 128 + r) * half;
    for (int t = lane; t < half; t += 32) {
        float2 v = make_float2(0.f, 0.f);
        if (real && t < L) {
            v = atoms[j * L + t];
            v.x = (v.x * inv) * s;
            v.y = (v.y * inv) * s;
        }
        re_row[t] = e4m3_pair(v.x, v.y);
        im_row[t] = e4m3_pair(-v.y, v.x);
    }
}

// One warp per voxel (listed voxels when vlist is given): the E4M3 query row and qs = 1 / s.
__global__ void k_pack_queries_fp8(const float2* __restrict__ Z, const int32_t* __restrict__ vlist,
                                   int64_t n, int L, int Kp8, uint16_t* __restrict__ zq8,
                                   float* __restrict__ qs) {
    const int64_t k = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= n) return;
    const int64_t v = vlist ? static_cast<int64_t>(vlist[k]) : k;
    const float2* z = Z + v * L;
    float m = 0.f;
    for (int t = lane; t < L; t += 32) {
        const float2 a = z[t];
        m = fmaxf(m, fmaxf(fabsf(a.x), fabsf(a.y)));
    }
    m = warp_max(m);
    const float s = e4m3_row_scale(m);
    const int half = Kp8 / 2;
    uint16_t* row = zq8 + k * half;
    for (int t = lane; t < half; t += 32) {
        const float2 a = (t < L) ? z[t] : make_float2(0.f, 0.f);
        row[t] = e4m3_pair(a.x * s, a.y * s);
    }
    if (lane == 0) qs[k] = 1.f / s;
}

__global__ void k_mask_ky(float2* __restrict__ W, const uint8_t* __restrict__ mask, int Ny,
                          int Nx, int L) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t total = static_cast<int64_t>(Ny) * Nx * L;
    if (i >= total) return;
    int t = static_cast<int>(i % L);
    int ky = static_cast<int>(i / (static_cast<int64_t>(Nx) * L));
    if (!mask[static_cast<int64_t>(t) * Ny + ky]) W[i] = make_float2(0.f, 0.f);
}

// Z = X - mu (g_scale G - AHY); optionally also the BF16 query operand of Z.
__global__ void k_grad_combine(const float2* __restrict__ X, const float2* __restrict__ G,
                               const float2* __restrict__ AHY, float2* __restrict__ Z,
                               int64_t n, int L, float mu, float gs,
                               __nv_bfloat162* __restrict__ zq, int Kp, uint32_t* err) {
    int64_t half = Kp / 2;
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * half) return;
    int64_t v = i / half;
    int t = static_cast<int>(i - v * half);
    float2 z = make_float2(0.f, 0.f);
    if (t < L) {
        int64_t o = v * L + t;
        float2 x = X[o], g = G[o], a = AHY[o];
        z.x = x.x - mu * (gs * g.x - a.x);
        z.y = x.y - mu * (gs * g.y - a.y);
        if (!isfinite(z.x) || !isfinite(z.y)) atomicOr(err, MRF_DERR_NONFINITE);
        Z[o] = z;
    }
    if (zq) zq[i] = __floats2bfloat162_rn(z.x, z.y);
}

__global__ void k_scale(float2* X, int64_t count, float s) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) { X[i].x *= s; X[i].y *= s; }
}

__global__ void k_axpby(float2* Y, const float2* X, int64_t count, float a, float b) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) {
        float2 y = Y[i], x = X[i];
        Y[i] = make_float2(a * y.x + b * x.x, a * y.y + b * x.y);
    }
}

__global__ void k_lut(const int32_t* __restrict__ idx, int64_t n, const float* __restrict__ prm,
                      int P, int64_t d, float* __restrict__ out, uint32_t* err) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * P) return;
    int64_t v = i / P;
    int p = static_cast<int>(i - v * P);
    int32_t j = idx[v];
    if (j < 0 || j >= d) {
        atomicOr(err, MRF_DERR_BOUNDS);
        out[i] = __int_as_float(0x7fc00000);
        return;
    }
    out[i] = prm[static_cast<int64_t>(j) * P + p];
}

__device__ __forceinline__ double block_sum(double s) {
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < kThreads / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

__global__ void k_sqnorm(const float2* __restrict__ X, int64_t count, double* out) {
    double s = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float2 v = X[i];
        s += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

__global__ void k_sqdiff(const float2* __restrict__ A, const float2* __restrict__ B,
                         int64_t count, double* out) {
    double s = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float2 a = A[i], b = B[i];
        double dx = static_cast<double>(a.x) - b.x, dy = static_cast<double>(a.y) - b.y;
        s += dx * dx + dy * dy;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

inline unsigned grid_for(int64_t work) {
    return static_cast<unsigned>((work + kThreads - 1) / kThreads);
}

}  // namespace

#define LAUNCH_CHECK()                                                                  \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) {                                                        \
            mrf_set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));     \
            return MRF_ECUDA;                                                           \
        }                                                                               \
    } while (0)

mrf_status launch_atom_norms(mrf_dict* D, cudaStream_t st) {
    k_atom_norms<<<grid_for(D->d * 32), kThreads, 0, st>>>(D->atoms, D->d, D->L, D->norm2,
                                                            D->inv_norm2, D->inv_norm, D->err);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_pack_bop(mrf_dict* D, cudaStream_t st) {
    return launch_pack_bop_perm(D, D->bop, nullptr, st);
}

mrf_status launch_pack_bop_perm(const mrf_dict* D, __nv_bfloat16* dst, const int32_t* perm,
                                cudaStream_t st) {
    int64_t total = D->nblk * 256 * (D->Kp / 2);
    k_pack_bop<<<grid_for(total), kThreads, 0, st>>>(D->atoms, D->inv_norm, D->d, D->L, D->Kp, D->nblk,
                                                      reinterpret_cast<__nv_bfloat162*>(dst), perm);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_atoms_absmax(const mrf_dict* D, unsigned int* m_bits, cudaStream_t st) {
    k_atoms_absmax<<<grid_for(D->d * 32), kThreads, 0, st>>>(D->atoms, D->inv_norm, D->d, D->L,
                                                              m_bits);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_pack_fop(mrf_dict* D, float s, cudaStream_t st) {
    const int64_t slots = D->nblk * 128;
    k_pack_fop<<<grid_for(slots * 32), kThreads, 0, st>>>(
        D->atoms, D->inv_norm, D->d, D->L, D->Kp8, D->nblk, s, reinterpret_cast<uint16_t*>(D->fop));
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_pack_queries_fp8(const float2* Z, const int32_t* vlist, int64_t n, int L,
                                   int Kp8, uint8_t* zq8, float* qs, cudaStream_t st) {
    if (n == 0) return MRF_OK;
    k_pack_queries_fp8<<<grid_for(n * 32), kThreads, 0, st>>>(
        Z, vlist, n, L, Kp8, reinterpret_cast<uint16_t*>(zq8), qs);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_pack_queries(const float2* Z, int64_t n, int L, int Kp, __nv_bfloat16* zq,
                               cudaStream_t st) {
    if (n == 0) return MRF_OK;
    k_pack_queries<<<grid_for(n * (Kp / 2)), kThreads, 0, st>>>(
        Z, n, L, Kp, reinterpret_cast<__nv_bfloat162*>(zq));
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_pack_gather(const float2* Z, const int32_t* vlist, int64_t n, int L, int Kp,
                              __nv_bfloat16* zq, cudaStream_t st, const int32_t* count) {
    if (n == 0) return MRF_OK;
    k_pack_gather<<<grid_for(n * (Kp / 2)), kThreads, 0, st>>>(
        Z, vlist, count, n, L, Kp, reinterpret_cast<__nv_bfloat162*>(zq));
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_mask_ky(float2* W, const uint8_t* mask, int Ny, int Nx, int L,
                          cudaStream_t st) {
    int64_t total = static_cast<int64_t>(Ny) * Nx * L;
    k_mask_ky<<<grid_for(total), kThreads, 0, st>>>(W, mask, Ny, Nx, L);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_grad_combine(const float2* X, const float2* G, const float2* AHY, float2* Z,
                               int64_t n, int L, float mu, float g_scale, __nv_bfloat16* zq,
                               int Kp, uint32_t* err, cudaStream_t st) {
    int kp = zq ? Kp : 2 * L;
    k_grad_combine<<<grid_for(n * (kp / 2)), kThreads, 0, st>>>(
        X, G, AHY, Z, n, L, mu, g_scale, reinterpret_cast<__nv_bfloat162*>(zq), kp, err);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_scale(float2* X, int64_t count, float s, cudaStream_t st) {
    k_scale<<<grid_for(count), kThreads, 0, st>>>(X, count, s);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_axpby(float2* Y, const float2* X, int64_t count, float a, float b,
                        cudaStream_t st) {
    k_axpby<<<grid_for(count), kThreads, 0, st>>>(Y, X, count, a, b);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_lut(const int32_t* idx, int64_t n, const float* params, int P, int64_t d,
                      float* out, uint32_t* err, cudaStream_t st) {
    if (n * P == 0) return MRF_OK;
    k_lut<<<grid_for(n * P), kThreads, 0, st>>>(idx, n, params, P, d, out, err);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_sqnorm(const float2* X, int64_t count, double* out, cudaStream_t st) {
    k_sqnorm<<<1024, kThreads, 0, st>>>(X, count, out);
    LAUNCH_CHECK();
    return MRF_OK;
}

mrf_status launch_sqdiff(const float2* A, const float2* B, int64_t count, double* out,
                         cudaStream_t st) {
    k_sqdiff<<<1024, kThreads, 0, st>>>(A, B, count, out);
    LAUNCH_CHECK();
    return MRF_OK;
}
