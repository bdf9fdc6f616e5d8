// Candidate merge, exact rescore and density (§3.2, eqs. exactP / exactPs).
//
// One warp per voxel.  The S x K candidates of the exhaustive kernels are reduced to the K best
// by their kernel score; those of them that can still be the best given the kernel's error
// bound (`window`; all K when window < 0) are rescored exactly in FP32 from the complex64
// operands; if
// several lie within `tie_tol` (absolute, in normalised correlation |c| / (||d|| ||z||)) of the
// best, they are rescored with FP64-class accuracy (compensated FP32 sums, reduced in FP64) and
// the largest wins (ties to the smallest index).  The density is rho = D_j^H Z_v / ||D_j||^2
// with the same accumulation (real cone: gamma = max(Re(.), 0)), and
// X_v = rho D_j is written when requested.  A zero fingerprint gives j = 0, rho = 0.
// With `certify`, a voxel whose K-th kernel score is within `cert_margin` of the best exact
// score (same units) is appended to a fallback list (the low-precision ranking could have missed the best).
#include "mrf_internal.cuh"

namespace {

constexpr int WARPS = 8;

__device__ __forceinline__ float warp_sum(float x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sumd(double x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Compensated FP32 accumulation ("double-float"): a product a b is split exactly into
// p + e with an FMA (p = fl(a b), e = a b - p), p is added to the running sum `hi` with Knuth's
// two-sum and every rounding error goes to `lo`.  hi + lo carries the sum with an error of a
// few units of 2^-46 of the sum of |terms| -- the accuracy of FP64 accumulation for these
// sums -- at FP32 throughput: FP64 runs at 1/64 of the FP32 rate on this GPU.
// The _rn intrinsics keep the compiler from contracting these steps into FMAs, which would
// break the error-free transformations.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    lo = __fadd_rn(lo, __fadd_rn(err, e));
    hi = s;
}

// D_j^H z over the warp's frames in compensated FP32, reduced across the warp in FP64.
__device__ __forceinline__ void cdot_df(const float2* __restrict__ a, const float2* __restrict__ z,
                                        int L, int lane, double& re, double& im) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int t = lane; t < L; t += 32) {
        const float2 dv = a[t], zv = z[t];
        df_fma(rh, rl, dv.x, zv.x);
        df_fma(rh, rl, dv.y, zv.y);
        df_fma(ih, il, dv.x, zv.y);
        df_fma(ih, il, -dv.y, zv.x);
    }
    re = warp_sumd(static_cast<double>(rh) + static_cast<double>(rl));
    im = warp_sumd(static_cast<double>(ih) + static_cast<double>(il));
}

// (s, j) ordering: larger score first, then smaller index; j < 0 marks an empty slot.
__device__ __forceinline__ bool better(float sa, int32_t ja, float sb, int32_t jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    if (sa != sb) return sa > sb;
    return ja < jb;
}

template <int KT>
__global__ void __launch_bounds__(WARPS * 32, KT >= 32 ? 2 : 3)
k_merge(const float2* __restrict__ Z, int64_t n_in, const int32_t* __restrict__ vlist,
        const int32_t* __restrict__ nlist, const float2* __restrict__ atoms,
        const float* __restrict__ inv_norm2, const double* __restrict__ norm2, int64_t d,
        int L, int cone, int S, const float* __restrict__ part_s,
        const int32_t* __restrict__ part_i, float tie_tol, int certify, float cert_margin,
        float window, int32_t* __restrict__ idx_out, float2* __restrict__ rho_out,
        float2* __restrict__ X_out, int32_t* __restrict__ fb_list, int32_t* __restrict__ fb_n,
        uint32_t* err, unsigned long long* cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t n = vlist ? static_cast<int64_t>(*nlist) : n_in;
    const int64_t vl = static_cast<int64_t>(blockIdx.x) * WARPS + (threadIdx.x >> 5);
    if (vl >= n) return;
    const int64_t v = vlist ? static_cast<int64_t>(vlist[vl]) : vl;
    const float2* z = Z + v * L;

    // 1. lane-local top-KT over a strided share of the S*KT candidates, then KT warp rounds
    float ls[KT];
    int32_t li[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) { ls[q] = -INFINITY; li[q] = -1; }
    const int total = S * KT;
    for (int c = lane; c < total; c += 32) {
        const int s = c / KT, k = c - s * KT;
        const int64_t o = (static_cast<int64_t>(s) * n + vl) * KT + k;
        float sc = part_s[o];
        int32_t j = part_i[o];
        if (j < 0 || j >= d) continue;
        if (better(sc, j, ls[KT - 1], li[KT - 1])) {
            ls[KT - 1] = sc;
            li[KT - 1] = j;
#pragma unroll
            for (int q = KT - 1; q > 0; --q) {
                bool up = better(ls[q], li[q], ls[q - 1], li[q - 1]);
                float a = ls[q], b = ls[q - 1];
                int32_t ia = li[q], ib = li[q - 1];
                ls[q - 1] = up ? a : b; ls[q] = up ? b : a;
                li[q - 1] = up ? ia : ib; li[q] = up ? ib : ia;
            }
        }
    }
    float cs[KT];       // kernel scores of the warp's top-KT (uniform across lanes)
    int32_t cj[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        float bs = ls[0];
        int32_t bj = li[0];
        int bl = lane;
        for (int o = 16; o; o >>= 1) {
            float os = __shfl_xor_sync(0xffffffffu, bs, o);
            int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
            int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (better(os, oj, bs, bj) || (os == bs && oj == bj && ol < bl)) {
                bs = os; bj = oj; bl = ol;
            }
        }
        cs[q] = bs;
        cj[q] = bj;
        if (lane == bl) {
#pragma unroll
            for (int p = 0; p < KT - 1; ++p) { ls[p] = ls[p + 1]; li[p] = li[p + 1]; }
            ls[KT - 1] = -INFINITY;
            li[KT - 1] = -1;
        }
    }

    // 2. exact FP32 rescore of the candidates inside the window.  The candidates are sorted by
    //    kernel score; one whose kernel correlation lies more than `window` below the first's
    //    cannot be the exactly best (window = twice the kernel's error bound plus tie_tol), so
    //    only a prefix of nw candidates is rescored.  All of them are gathered together (one
    //    pass over the frames, up to KT independent loads in flight per lane).
    float zn2 = 0.f;
    for (int t = lane; t < L; t += 32) { float2 a = z[t]; zn2 += a.x * a.x + a.y * a.y; }
    zn2 = warp_sum(zn2);
    int nw = 0;
    {
        float lower = -INFINITY;
        if (window >= 0.f && cj[0] >= 0) {
            const float zn0 = sqrtf(zn2);
            if (cone == MRF_CONE_COMPLEX) {
                const float c = sqrtf(fmaxf(cs[0], 0.f)) - window * zn0;
                lower = c > 0.f ? c * c : -INFINITY;
            } else {
                lower = cs[0] - window * zn0;
            }
        }
#pragma unroll
        for (int q = 0; q < KT; ++q) nw += (cj[q] >= 0 && cs[q] >= lower) ? 1 : 0;
    }
    float er[KT], ei[KT];
    const float2* ap[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        er[q] = 0.f;
        ei[q] = 0.f;
        ap[q] = atoms + static_cast<int64_t>(q < nw ? cj[q] : 0) * L;
    }
    for (int t = lane; t < L; t += 32) {
        const float2 zv = z[t];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (q < nw) {
                const float2 dv = ap[q][t];
                er[q] = fmaf(dv.x, zv.x, fmaf(dv.y, zv.y, er[q]));
                ei[q] = fmaf(dv.x, zv.y, fmaf(-dv.y, zv.x, ei[q]));
            }
        }
    }
    float es[KT];
    int best = -1;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        es[q] = -INFINITY;
        if (q >= nw) continue;
        const float re = warp_sum(er[q]);
        const float im = warp_sum(ei[q]);
        const float w = inv_norm2[cj[q]];
        es[q] = (cone == MRF_CONE_COMPLEX) ? (re * re + im * im) * w : re * sqrtf(w);
        if (best < 0 || better(es[q], cj[q], es[best], cj[best])) best = q;
    }
    if (best < 0) {          // no candidate at all (cannot happen with d >= 1)
        if (lane == 0) atomicOr(err, MRF_DERR_BOUNDS);
        return;
    }

    // 3. extended-precision rescore of the near-ties.  Windows are absolute in normalised correlation
    //    |c| / (||d|| ||z||): rounding errors of the FP32 (and BF16) sums scale with ||z||, not
    //    with the correlation itself.
    const float eb = es[best];
    const float zn = sqrtf(zn2);
    auto floor_of = [&](float tol) -> float {     // lowest score still within `tol`
        if (cone == MRF_CONE_COMPLEX) {
            float c = sqrtf(fmaxf(eb, 0.f)) - tol * zn;
            return c > 0.f ? c * c : 0.f;
        }
        return eb - tol * zn;
    };
    const float thr = floor_of(tie_tol);
    int ntie = 0;
#pragma unroll
    for (int q = 0; q < KT; ++q) ntie += (cj[q] >= 0 && es[q] >= thr) ? 1 : 0;
    int32_t jstar = cj[best];
    double cre = 0.0, cim = 0.0;
    bool have64 = false;
    if (ntie > 1) {
        double bs64 = -INFINITY;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (cj[q] < 0 || es[q] < thr) continue;
            double re, im;
            cdot_df(atoms + static_cast<int64_t>(cj[q]) * L, z, L, lane, re, im);
            double nn = norm2[cj[q]];
            double s64 = (cone == MRF_CONE_COMPLEX) ? (re * re + im * im) / nn : re / sqrt(nn);
            if (s64 > bs64 || (s64 == bs64 && cj[q] < jstar)) {
                bs64 = s64;
                jstar = cj[q];
                cre = re;
                cim = im;
            }
        }
        have64 = true;
        if (lane == 0) atomicAdd(cnt + CNT_TIE_RESCORED, 1ULL);
        if (lane == 0 && cj[KT - 1] >= 0 && es[KT - 1] >= thr)
            atomicAdd(cnt + CNT_TIE_OVERFLOW, 1ULL);
    }
    // 4. certification of the low-precision ranking: the K-th kernel score must lie more than
    //    cert_margin (normalised correlation) below the best exact score
    if (certify && cj[KT - 1] >= 0 && zn2 > 0.f && cs[KT - 1] >= floor_of(cert_margin)) {
        if (lane == 0) {
            int pos = atomicAdd(fb_n, 1);
            fb_list[pos] = static_cast<int32_t>(v);
            atomicAdd(cnt + CNT_UNCERT, 1ULL);
        }
    }
    // 5. density with the same extended-precision accumulation
    if (!have64) {
        cdot_df(atoms + static_cast<int64_t>(jstar) * L, z, L, lane, cre, cim);
    }
    double nn = norm2[jstar];
    double rr = cre / nn, ri = cim / nn;
    if (cone != MRF_CONE_COMPLEX) { rr = rr > 0.0 ? rr : 0.0; ri = 0.0; }
    if (zn2 == 0.f) {
        jstar = 0; rr = 0.0; ri = 0.0;
        if (lane == 0) atomicAdd(cnt + CNT_ZERO, 1ULL);
    }
    const float2 rho = make_float2(static_cast<float>(rr), static_cast<float>(ri));
    if (lane == 0) {
        idx_out[v] = jstar;
        if (rho_out) rho_out[v] = rho;
    }
    if (X_out) {
        const float2* a = atoms + static_cast<int64_t>(jstar) * L;
        float2* x = X_out + v * L;
        for (int t = lane; t < L; t += 32) {
            float2 dv = a[t];
            x[t] = make_float2(rho.x * dv.x - rho.y * dv.y, rho.x * dv.y + rho.y * dv.x);
        }
    }
}

}  // namespace

mrf_status launch_merge(const float2* Z, int64_t n, const mrf_dict* D, int cone, int K, int S,
                        const float* part_s, const int32_t* part_i, const int32_t* vlist,
                        const int32_t* nlist, float tie_tol, int certify, float cert_margin,
                        int32_t* idx_out, float2* rho_out, float2* X_out, int32_t* fb_list,
                        int32_t* fb_n, uint32_t* err, unsigned long long* counters,
                        cudaStream_t st, float window) {
    if (n == 0) return MRF_OK;
    dim3 grid(static_cast<unsigned>((n + WARPS - 1) / WARPS));
    if (K == 8) {
        k_merge<8><<<grid, WARPS * 32, 0, st>>>(Z, n, vlist, nlist, D->atoms, D->inv_norm2,
                                                D->norm2, D->d, D->L, cone, S, part_s, part_i,
                                                tie_tol, certify, cert_margin, window, idx_out,
                                                rho_out, X_out, fb_list, fb_n, err, counters);
    } else if (K == 16) {
        k_merge<16><<<grid, WARPS * 32, 0, st>>>(Z, n, vlist, nlist, D->atoms, D->inv_norm2,
                                                 D->norm2, D->d, D->L, cone, S, part_s, part_i,
                                                 tie_tol, certify, cert_margin, window,
                                                 idx_out, rho_out, X_out, fb_list, fb_n, err,
                                                 counters);
    } else if (K == 32) {
        k_merge<32><<<grid, WARPS * 32, 0, st>>>(Z, n, vlist, nlist, D->atoms, D->inv_norm2,
                                                 D->norm2, D->d, D->L, cone, S, part_s, part_i,
                                                 tie_tol, certify, cert_margin, window,
                                                 idx_out, rho_out, X_out, fb_list, fb_n, err,
                                                 counters);
    } else {
        mrf_set_error("merge: K must be 8, 16 or 32");
        return MRF_EINVAL;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mrf_set_error(std::string("merge launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}
