// Split-BF16 operands of the exact tensor-core matched filter (§3.2, eq. exactP) and the rigorous
// bound of its correlation error.
//
// Every FP32 value x is written as x = hi + lo + e with hi = bf16(x), lo = bf16(x - hi) (both
// round to nearest even; x - hi and (x - hi) - lo are exact in FP32), so |lo| <= u (1 + u) |x|
// and |e| <= u^2 |x| with u = 2^-8.  A query row is stored as three segments [lo | hi | hi] and
// an atom row as [hi | lo | hi] (each segment Kp elements), so the tensor cores' one MMA chain
// over Kp3 = 3 Kp accumulates z_lo d_hi + z_hi d_lo first (partial sums of size ~2u) and then
// z_hi d_hi; the dropped terms are z_lo d_lo and those of e.
//
// Error of the computed correlation c~ against c = d^H z (unit atom d), per voxel, in units of
// ||z|| (normalised correlation):
//   operand part (Cauchy-Schwarz on the stored residuals, rigorous):
//     |c_split - c| <= ||z_lo|| ||d_lo|| + ||z_hi + z_lo|| ||e_d|| + ||e_z|| ||d||
//     with max_j ||d_lo,j|| = A_l and max_j ||e_d,j|| = A_e measured at packing (FP64, rounded
//     up) and the query's own ||z_lo||, ||e_z|| measured here;
//   accumulation part (a model of the tensor core's FP32 accumulation, not a documented
//     property): each MMA instruction (16 exact products of BF16 values) updates the FP32
//     accumulator with one rounding of relative error at most 2^-23 (nearest or directed).  A
//     partial sum of the first 2 Kp / 16 instructions is at most
//       m_lo = ||z_lo|| ||d_hi|| + ||z_hi|| ||d_lo||,
//     of the last Kp / 16 at most m_hi = m_lo + ||z_hi|| ||d_hi||, so the accumulated error is at
//     most 2^-23 (2 Kp / 16 m_lo + Kp / 16 m_hi) in each of Re c and Im c (sqrt 2 of it in |c|);
//   epilogue: the score re^2 + im^2 with two FP32 roundings, at most 2^-23 in |c|.
// The margin written per voxel is that bound plus `extra` (the caller adds the bound of the
// FP32 rescore it compares against).  Rows with ||z|| below 2^-40 (where subnormal parts and
// the squares of the split residuals underflow) are not covered by the bound; a zero row gets
// margin 0.
#include <cstring>

#include "mrf_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l,
                                           float& hf, float& lf, float& e) {
    h = __float2bfloat16_rn(x);
    hf = __bfloat162float(h);
    const float r = x - hf;          // exact
    l = __float2bfloat16_rn(r);
    lf = __bfloat162float(l);
    e = r - lf;                      // exact
}

__device__ __forceinline__ double warp_sumd(double x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One warp per atom slot of the padded blocks: the real-part row (Re d, Im d) and the
// imaginary-part row (-Im d, Re d) of the normalised atom (FP32, as the BF16 operand rounds it),
// each as [hi | lo | hi]; and per atom the largest ||lo|| and ||d/||d|| - hi - lo|| (the exact
// unit atom in FP64) into `bits` (float bit patterns, rounded up; non-negative floats order like
// their bits).
// With `sel` (length nsel) operand slot p holds atom sel[p] for p < nsel (nothing where
// sel[p] < 0) and nothing after.
__global__ void k_pack_bop3(const float2* __restrict__ atoms, const float* __restrict__ inv_norm,
                            const double* __restrict__ norm2, int64_t d, int L, int Kp,
                            int64_t nblk, __nv_bfloat162* __restrict__ bop3,
                            unsigned int* __restrict__ bits, const int32_t* __restrict__ sel,
                            int64_t nsel) {
    const int64_t slot = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= nblk * 128) return;
    const int64_t b = slot >> 7;
    const int r = static_cast<int>(slot & 127);
    int64_t j = sel ? (slot < nsel ? static_cast<int64_t>(sel[slot]) : d) : slot;
    if (j < 0) j = d;                                   // empty slot of a selection
    const bool real = j < d;
    const float inv = real ? inv_norm[j] : 0.f;
    const double invd = real ? 1.0 / sqrt(norm2[j]) : 0.0;
    const int half = Kp / 2;
    __nv_bfloat162* re_row = bop3 + (b * 256 + r) * (3 * half);
    __nv_bfloat162* im_row = bop3 + (b * 256 + 128 + r) * (3 * half);
    double al = 0.0, ae = 0.0;
    for (int t = lane; t < half; t += 32) {
        float2 v = make_float2(0.f, 0.f);
        const bool in = real && t < L;
        if (in) v = atoms[j * L + t];
        __nv_bfloat16 hx, lx, hy, ly;
        float hxf, lxf, ex, hyf, lyf, ey;
        split_bf16(v.x * inv, hx, lx, hxf, lxf, ex);
        split_bf16(v.y * inv, hy, ly, hyf, lyf, ey);
        re_row[t] = __halves2bfloat162(hx, hy);
        re_row[half + t] = __halves2bfloat162(lx, ly);
        re_row[2 * half + t] = __halves2bfloat162(hx, hy);
        im_row[t] = __halves2bfloat162(__hneg(hy), hx);
        im_row[half + t] = __halves2bfloat162(__hneg(ly), lx);
        im_row[2 * half + t] = __halves2bfloat162(__hneg(hy), hx);
        if (in) {
            const double dx = static_cast<double>(v.x) * invd - hxf - lxf;
            const double dy = static_cast<double>(v.y) * invd - hyf - lyf;
            ae += dx * dx + dy * dy;
            al += static_cast<double>(lxf) * lxf + static_cast<double>(lyf) * lyf;
        }
    }
    al = warp_sumd(al);
    ae = warp_sumd(ae);
    if (lane == 0 && real) {
        atomicMax(bits, __float_as_uint(__double2float_ru(sqrt(al) * (1.0 + 1e-9))));
        atomicMax(bits + 1, __float_as_uint(__double2float_ru(sqrt(ae) * (1.0 + 1e-9))));
    }
}

struct BoundConsts {
    double Al, Ae;        // max ||d_lo||, max ||e_d|| over the atoms
    double n_lo, n_hi;    // MMA instructions of the small-product and the main segments
    float extra;
};

// One warp per voxel: the query row [lo | hi | hi] and the voxel's margin.
__global__ void k_pack_queries_x3(const float2* __restrict__ Z, int64_t n, int L, int Kp,
                                  BoundConsts bc, __nv_bfloat162* __restrict__ zq3,
                                  float* __restrict__ margin, const int32_t* __restrict__ vlist,
                                  float* __restrict__ znorm) {
    const int64_t v = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const int half = Kp / 2;
    const int64_t src = vlist ? static_cast<int64_t>(vlist[v]) : v;
    const float2* z = Z + src * L;
    __nv_bfloat162* row = zq3 + v * (3 * half);
    // squared norms in FP32 (each a sum of non-negative terms: relative error below
    // (L / 32 + 5) 2^-24, covered by the final (1 + 2^-10) inflation of the ratios below)
    float zz = 0.f, ll = 0.f, ee = 0.f, hh = 0.f;
    for (int t = lane; t < half; t += 32) {
        const float2 a = (t < L) ? z[t] : make_float2(0.f, 0.f);
        __nv_bfloat16 hx, lx, hy, ly;
        float hxf, lxf, ex, hyf, lyf, ey;
        split_bf16(a.x, hx, lx, hxf, lxf, ex);
        split_bf16(a.y, hy, ly, hyf, lyf, ey);
        row[t] = __halves2bfloat162(lx, ly);
        row[half + t] = __halves2bfloat162(hx, hy);
        row[2 * half + t] = __halves2bfloat162(hx, hy);
        zz = fmaf(a.x, a.x, fmaf(a.y, a.y, zz));
        ll = fmaf(lxf, lxf, fmaf(lyf, lyf, ll));
        ee = fmaf(ex, ex, fmaf(ey, ey, ee));
        hh = fmaf(hxf, hxf, fmaf(hyf, hyf, hh));
    }
    for (int o = 16; o; o >>= 1) {
        zz += __shfl_xor_sync(0xffffffffu, zz, o);
        ll += __shfl_xor_sync(0xffffffffu, ll, o);
        ee += __shfl_xor_sync(0xffffffffu, ee, o);
        hh += __shfl_xor_sync(0xffffffffu, hh, o);
    }
    if (lane == 0 && znorm) znorm[v] = sqrtf(zz);
    if (lane == 0 && margin) {
        float m = 0.f;
        if (zz > 0.f) {
            const double zn = sqrt(static_cast<double>(zz)) * (1.0 - 0x1p-10);
            const double up = 1.0 + 0x1p-10;
            const double zl = sqrt(static_cast<double>(ll)) * up / zn;
            const double ze = sqrt(static_cast<double>(ee)) * up / zn;
            const double zh = sqrt(static_cast<double>(hh)) * up / zn;
            const double dh = 1.0 + bc.Al + bc.Ae;            // bound on ||d_hi||
            const double e_op = zl * bc.Al + (1.0 + ze) * bc.Ae + ze;
            const double m_lo = zl * dh + zh * bc.Al;
            const double m_hi = m_lo + zh * dh;
            const double eps = 1.1920928955078125e-07;         // 2^-23
            const double e_acc = eps * (bc.n_lo * m_lo + bc.n_hi * m_hi);
            const double b = e_op + 1.4142135623730951 * e_acc + eps;
            m = __double2float_ru(b * (1.0 + 1e-6)) + bc.extra;
        }
        margin[src] = m;
    }
}

__global__ void k_fill(float* __restrict__ out, int64_t n, float v) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

inline unsigned grid_for(int64_t work) {
    return static_cast<unsigned>((work + kThreads - 1) / kThreads);
}

}  // namespace

mrf_status launch_pack_bop3(mrf_dict* D, cudaStream_t st) {
    unsigned int* bits = reinterpret_cast<unsigned int*>(D->red);
    MRF_CUDA_TRY(cudaMemsetAsync(bits, 0, 2 * sizeof(unsigned int), st));
    const int64_t slots = D->nblk * 128;
    k_pack_bop3<<<grid_for(slots * 32), kThreads, 0, st>>>(
        D->atoms, D->inv_norm, D->norm2, D->d, D->L, D->Kp3 / 3, D->nblk,
        reinterpret_cast<__nv_bfloat162*>(D->bop3), bits, nullptr, 0);
    MRF_CUDA_TRY(cudaGetLastError());
    unsigned int h[2] = {0u, 0u};
    MRF_CUDA_TRY(cudaMemcpyAsync(h, bits, sizeof(h), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    float al, ae;
    std::memcpy(&al, &h[0], sizeof(al));
    std::memcpy(&ae, &h[1], sizeof(ae));
    D->x3_al = al;
    D->x3_ae = ae;
    return MRF_OK;
}

mrf_status launch_pack_sel3(const mrf_dict* D, const int32_t* sel, int64_t nsel, int64_t nblk_out,
                            __nv_bfloat16* dst, float* al_out, float* ae_out, cudaStream_t st) {
    unsigned int* bits = reinterpret_cast<unsigned int*>(D->red);
    MRF_CUDA_TRY(cudaMemsetAsync(bits, 0, 2 * sizeof(unsigned int), st));
    k_pack_bop3<<<grid_for(nblk_out * 128 * 32), kThreads, 0, st>>>(
        D->atoms, D->inv_norm, D->norm2, D->d, D->L, D->Kp, nblk_out,
        reinterpret_cast<__nv_bfloat162*>(dst), bits, sel, nsel);
    MRF_CUDA_TRY(cudaGetLastError());
    unsigned int h[2] = {0u, 0u};
    MRF_CUDA_TRY(cudaMemcpyAsync(h, bits, sizeof(h), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(al_out, &h[0], sizeof(float));
    std::memcpy(ae_out, &h[1], sizeof(float));
    return MRF_OK;
}

mrf_status launch_pack_queries_x3(const float2* Z, int64_t n, const mrf_dict* D, float extra,
                                  __nv_bfloat16* zq3, float* margin, cudaStream_t st) {
    return launch_pack_queries_x3_with(Z, n, D->L, D->Kp3 / 3, D->x3_al, D->x3_ae, extra, zq3,
                                       margin, st);
}

mrf_status launch_pack_queries_x3_with(const float2* Z, int64_t n, int L, int Kp, float Al,
                                       float Ae, float extra, __nv_bfloat16* zq3, float* margin,
                                       cudaStream_t st, const int32_t* vlist, float* znorm) {
    if (n == 0) return MRF_OK;
    BoundConsts bc;
    bc.Al = Al;
    bc.Ae = Ae;
    bc.n_lo = 2.0 * Kp / 16.0;
    bc.n_hi = Kp / 16.0;
    bc.extra = extra;
    k_pack_queries_x3<<<grid_for(n * 32), kThreads, 0, st>>>(
        Z, n, L, Kp, bc, reinterpret_cast<__nv_bfloat162*>(zq3), margin, vlist, znorm);
    MRF_CUDA_TRY(cudaGetLastError());
    return MRF_OK;
}

mrf_status launch_fill(float* out, int64_t n, float v, cudaStream_t st) {
    if (n == 0) return MRF_OK;
    k_fill<<<grid_for(n), kThreads, 0, st>>>(out, n, v);
    MRF_CUDA_TRY(cudaGetLastError());
    return MRF_OK;
}
