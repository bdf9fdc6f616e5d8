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
// Candidates gathered per pass over the frames and resident blocks per SM: for K <= 16 four per
// pass at 64 registers (four blocks of 8 warps per SM, more gathers in flight), for K = 32 eight
// per pass at 80 (three blocks; 64 registers would spill its lists).
template <int KT> constexpr int merge_g() { return KT >= 32 ? 8 : 4; }
template <int KT, int NL> constexpr int merge_min_blocks() { return NL >= 32 ? 2 : (KT >= 32 ? 3 : 4); }

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

// Order-preserving map of a float's bits to an unsigned key (larger float, larger key; a valid
// score never maps to 0) and back.
__device__ __forceinline__ uint32_t ord_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_score(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <int KT, int NL>
__global__ void __launch_bounds__(WARPS * 32, (merge_min_blocks<KT, NL>()))
k_merge(const float2* __restrict__ Z, int64_t n_in, const int32_t* __restrict__ vlist,
        const int32_t* __restrict__ nlist, const float2* __restrict__ atoms,
        const float* __restrict__ inv_norm2, const double* __restrict__ norm2, int64_t d,
        int L, int cone, int S, const float* __restrict__ part_s,
        const int32_t* __restrict__ part_i, float tie_tol, int certify, float cert_margin,
        float window, const float* __restrict__ vmargin, int32_t* __restrict__ idx_out,
        float2* __restrict__ rho_out,
        float2* __restrict__ X_out, int32_t* __restrict__ fb_list, int32_t* __restrict__ fb_n,
        uint32_t* err, unsigned long long* cnt) {
    const int lane = threadIdx.x & 31;
    // with a list, *nlist voxels are present; the candidate lists keep the stride n_in (the
    // capacity the search was launched for)
    const int64_t n = vlist ? min(static_cast<int64_t>(*nlist), n_in) : n_in;
    const int64_t vl = static_cast<int64_t>(blockIdx.x) * WARPS + (threadIdx.x >> 5);
    if (vl >= n) return;
    const int64_t v = vlist ? static_cast<int64_t>(vlist[vl]) : vl;
    const float2* z = Z + v * L;

    // 1. lane-local sorted lists of NL over a strided share of the S*KT candidates (NL covers
    //    the lane's share), then KT warp rounds: the largest head by a warp max-reduction of
    //    the order-preserving bit pattern of its score, ties to the smallest atom by a
    //    min-reduction; its lane pops it
    float ls[NL];
    int32_t li[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) { ls[q] = -INFINITY; li[q] = -1; }
    const int total = S * KT;
    for (int c = lane; c < total; c += 32) {
        const int s = c / KT, k = c - s * KT;
        const int64_t o = (static_cast<int64_t>(s) * n_in + vl) * KT + k;
        float sc = part_s[o];
        int32_t j = part_i[o];
        if (j < 0 || j >= d || sc != sc) continue;
        if (better(sc, j, ls[NL - 1], li[NL - 1])) {
            // sorted insertion without a dependency chain: slot q keeps its entry, takes the
            // new one, or takes its upper neighbour's
            bool keep[NL];
#pragma unroll
            for (int q = 0; q < NL; ++q) keep[q] = !better(sc, j, ls[q], li[q]);
#pragma unroll
            for (int q = NL - 1; q > 0; --q) {
                ls[q] = keep[q] ? ls[q] : (keep[q - 1] ? sc : ls[q - 1]);
                li[q] = keep[q] ? li[q] : (keep[q - 1] ? j : li[q - 1]);
            }
            ls[0] = keep[0] ? ls[0] : sc;
            li[0] = keep[0] ? li[0] : j;
        }
    }
    // kernel scores and atoms of the warp's top-KT, sorted (uniform across the warp; kept in
    // shared memory to leave the registers to the gathers)
    __shared__ float s_cs[WARPS][KT];
    __shared__ int32_t s_cj[WARPS][KT];
    float* cs = s_cs[threadIdx.x >> 5];
    int32_t* cj = s_cj[threadIdx.x >> 5];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        const uint32_t hk = li[0] >= 0 ? ord_key(ls[0]) : 0u;     // 0: empty
        const uint32_t m = __reduce_max_sync(0xffffffffu, hk);
        const uint32_t jc = (li[0] >= 0 && hk == m) ? static_cast<uint32_t>(li[0]) : 0xffffffffu;
        const uint32_t jm = __reduce_min_sync(0xffffffffu, jc);
        if (lane == 0) {
            cs[q] = m ? key_score(m) : -INFINITY;
            cj[q] = m ? static_cast<int32_t>(jm) : -1;
        }
        if (m != 0 && jc == jm) {
#pragma unroll
            for (int p = 0; p < NL - 1; ++p) { ls[p] = ls[p + 1]; li[p] = li[p + 1]; }
            ls[NL - 1] = -INFINITY;
            li[NL - 1] = -1;
        }
    }
    __syncwarp();

    // 2. exact FP32 rescore.  All KT candidates are gathered in passes of G over the frames
    //    (G independent loads per lane and frame step, two frames per 16-byte load when the
    //    rows allow it; rows of empty slots alias the first candidate's row), and ||z||^2
    //    rides along with the first pass.  The candidates are sorted by kernel score; one
    //    whose kernel correlation lies more than `window` below the first's cannot be the
    //    exactly best (window = twice the kernel's error bound plus tie_tol), so only the
    //    prefix of nw candidates inside the window competes for the best.
    constexpr int G = KT < merge_g<KT>() ? KT : merge_g<KT>();
    float zn2 = 0.f;
    int nw = 0;
    __shared__ float s_es[WARPS][KT];      // exact scores (-inf outside the window)
    float* es = s_es[threadIdx.x >> 5];
    if (lane < KT) es[lane] = -INFINITY;
    __syncwarp();
    float bsc = -INFINITY;      // best exact score and its atom
    int32_t jstar = -1;
    {
        const int64_t row0 = cj[0] >= 0 ? cj[0] : 0;
        const bool vec2 = (L & 1) == 0 && (reinterpret_cast<uintptr_t>(Z) & 15) == 0 &&
                          (reinterpret_cast<uintptr_t>(atoms) & 15) == 0;
#pragma unroll
        for (int g0 = 0; g0 < KT; g0 += G) {
            const float2* ap[G];
            float ar[G], ai[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                ar[q] = 0.f;
                ai[q] = 0.f;
                ap[q] = atoms + (cj[g0 + q] >= 0 ? static_cast<int64_t>(cj[g0 + q]) : row0) * L;
            }
            float za = 0.f;
            int t0 = 0;
            if (vec2) {
                // frames t, t + 1 in one load (t even; every row starts on 16 bytes)
                for (int t = 2 * lane; t + 1 < L; t += 64) {
                    const float4 zv = *reinterpret_cast<const float4*>(z + t);
                    float4 dv[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) dv[q] = *reinterpret_cast<const float4*>(ap[q] + t);
                    if (g0 == 0)
                        za = fmaf(zv.x, zv.x, fmaf(zv.y, zv.y, fmaf(zv.z, zv.z, fmaf(zv.w, zv.w, za))));
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        ar[q] = fmaf(dv[q].x, zv.x, fmaf(dv[q].y, zv.y, ar[q]));
                        ai[q] = fmaf(dv[q].x, zv.y, fmaf(-dv[q].y, zv.x, ai[q]));
                        ar[q] = fmaf(dv[q].z, zv.z, fmaf(dv[q].w, zv.w, ar[q]));
                        ai[q] = fmaf(dv[q].z, zv.w, fmaf(-dv[q].w, zv.z, ai[q]));
                    }
                }
                t0 = L;
            }
            for (int t = t0 + lane; t < L; t += 32) {
                const float2 zv = z[t];
                float2 dv[G];
#pragma unroll
                for (int q = 0; q < G; ++q) dv[q] = ap[q][t];
                if (g0 == 0) za = fmaf(zv.x, zv.x, fmaf(zv.y, zv.y, za));
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    ar[q] = fmaf(dv[q].x, zv.x, fmaf(dv[q].y, zv.y, ar[q]));
                    ai[q] = fmaf(dv[q].x, zv.y, fmaf(-dv[q].y, zv.x, ai[q]));
                }
            }
            if (g0 == 0) {
                zn2 = warp_sum(za);
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
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int qq = g0 + q;
                if (qq >= nw) continue;
                const float re = warp_sum(ar[q]);
                const float im = warp_sum(ai[q]);
                const float w = inv_norm2[cj[qq]];
                const float e = (cone == MRF_CONE_COMPLEX) ? (re * re + im * im) * w : re * sqrtf(w);
                if (lane == 0) es[qq] = e;
                if (jstar < 0 || better(e, cj[qq], bsc, jstar)) { bsc = e; jstar = cj[qq]; }
            }
            if (g0 + G >= nw) break;     // the remaining candidates lie outside the window
        }
    }
    __syncwarp();
    if (jstar < 0) {         // no candidate at all (cannot happen with d >= 1)
        if (lane == 0) atomicOr(err, MRF_DERR_BOUNDS);
        return;
    }

    // 3. extended-precision rescore of the near-ties.  Windows are absolute in normalised correlation
    //    |c| / (||d|| ||z||): rounding errors of the FP32 (and BF16) sums scale with ||z||, not
    //    with the correlation itself.
    const float eb = bsc;
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
    //    cert_margin (normalised correlation; the voxel's own margin when vmargin is given)
    //    below the best exact score
    if (certify && cj[KT - 1] >= 0 && zn2 > 0.f &&
        cs[KT - 1] >= floor_of(vmargin ? vmargin[v] : cert_margin)) {
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
                        cudaStream_t st, float window, const float* vmargin) {
    if (n == 0) return MRF_OK;
    dim3 grid(static_cast<unsigned>((n + WARPS - 1) / WARPS));
    if (K != 8 && K != 16 && K != 32) {
        mrf_set_error("merge: K must be 8, 16 or 32");
        return MRF_EINVAL;
    }
    // candidates per lane, rounded up to the lane-list length of an instantiation
    const int64_t per = (static_cast<int64_t>(S) * K + 31) / 32;
    const int NL = per <= 4 ? 4 : (per <= 8 ? 8 : (per <= 16 ? 16 : 32));
    const int nl = NL < K ? NL : K;
#define MRF_MERGE_ARGS Z, n, vlist, nlist, D->atoms, D->inv_norm2, D->norm2, D->d, D->L, cone, S, \
        part_s, part_i, tie_tol, certify, cert_margin, window, vmargin, idx_out, rho_out, X_out,   \
        fb_list,                                                                                    \
        fb_n, err, counters
    if (K == 8) {
        if (nl == 4) k_merge<8, 4><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else k_merge<8, 8><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
    } else if (K == 16) {
        if (nl == 4) k_merge<16, 4><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else if (nl == 8) k_merge<16, 8><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else k_merge<16, 16><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
    } else {
        if (nl == 4) k_merge<32, 4><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else if (nl == 8) k_merge<32, 8><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else if (nl == 16) k_merge<32, 16><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
        else k_merge<32, 32><<<grid, WARPS * 32, 0, st>>>(MRF_MERGE_ARGS);
    }
#undef MRF_MERGE_ARGS
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mrf_set_error(std::string("merge launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}
