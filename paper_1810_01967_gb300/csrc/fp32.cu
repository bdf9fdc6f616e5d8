// Exhaustive FP32 matched filter (§3.2, eq. exactP): for every voxel v and atom j the score
//   complex cone:  s_vj = |D_j^H Z_v|^2 / ||D_j||^2
//   real cone:     s_vj = Re(D_j^H Z_v) / ||D_j||
// is computed with FP32 FFMA (SIMT), and only each voxel's running top-K (score, j) leaves the
// CTA: the n x d score matrix is never written to memory.
//
// CTA tile: 128 voxels x 64 atoms, frames staged through shared memory 16 at a time (register
// prefetch of the next chunk).  Thread (ty, tx), ty in [0,32), tx in [0,8), accumulates the
// 4 x 8 complex correlations of voxels {2ty, 2ty+1, 64+2ty, 65+2ty} and atoms
// {16q + 2tx + r}.  After a tile the scores go to shared memory and two threads per voxel
// fold them into per-thread sorted top-K lists; at the end the two lists are merged and
// written as the split's candidates.  Grid = (voxel tiles) x (atom splits).
#include "mrf_internal.cuh"

namespace {

constexpr int TM = 128;     // voxels per CTA tile
constexpr int TN = 64;      // atoms per CTA tile
constexpr int TK = 16;      // frames per shared-memory chunk
constexpr int NT = 256;     // threads
constexpr int SPAD = TN + 1;

template <int KT>
__device__ __forceinline__ void topk_insert(float (&ts)[KT], int32_t (&ti)[KT], float s,
                                            int32_t j) {
    if (s > ts[KT - 1]) {
        ts[KT - 1] = s;
        ti[KT - 1] = j;
#pragma unroll
        for (int q = KT - 1; q > 0; --q) {
            bool up = ts[q] > ts[q - 1];
            float a = ts[q], b = ts[q - 1];
            int32_t ia = ti[q], ib = ti[q - 1];
            ts[q - 1] = up ? a : b;
            ts[q] = up ? b : a;
            ti[q - 1] = up ? ia : ib;
            ti[q] = up ? ib : ia;
        }
    }
}

template <int KT>
__global__ void __launch_bounds__(NT, 2)
k_fp32_topk(const float2* __restrict__ Z, const int32_t* __restrict__ vlist,
            const int32_t* __restrict__ nlist, int64_t n_in,
            const float2* __restrict__ atoms, const float* __restrict__ inv_norm2, int64_t d,
            int L, int cone, int S, int tiles_per_split, float* __restrict__ part_s,
            int32_t* __restrict__ part_i) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* Zs = reinterpret_cast<float2*>(smem_raw);                 // [TK][TM]
    float2* Ds = Zs + TK * TM;                                          // [TK][TN]
    float* Ss = reinterpret_cast<float*>(Ds + TK * TN);                 // [TM][SPAD]

    const int64_t n = vlist ? static_cast<int64_t>(*nlist) : n_in;
    const int64_t Mt = (n_in + TM - 1) / TM;
    const int64_t mt = blockIdx.x % Mt;
    const int s = static_cast<int>(blockIdx.x / Mt);
    const int64_t m0 = mt * TM;
    if (m0 >= n) return;
    const int64_t n_atom_tiles = (d + TN - 1) / TN;
    const int64_t at0 = static_cast<int64_t>(s) * tiles_per_split;
    const int64_t at1 = min(at0 + tiles_per_split, n_atom_tiles);

    const int tid = threadIdx.x;
    const int tx = tid & 7, ty = tid >> 3;
    // loader roles
    const int zl_v = tid >> 1, zl_f = (tid & 1) * 8;
    const int dl_a = tid >> 2, dl_f = (tid & 3) * 4;
    int64_t zrow = -1;
    if (m0 + zl_v < n) zrow = vlist ? static_cast<int64_t>(vlist[m0 + zl_v]) : m0 + zl_v;
    // scan roles
    const int sv = tid >> 1, sh = tid & 1;

    float ts[KT];
    int32_t ti[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) { ts[q] = -INFINITY; ti[q] = -1; }

    const int nchunks = (L + TK - 1) / TK;
    float2 zreg[8], dreg[4];

    for (int64_t at = at0; at < at1; ++at) {
        const int64_t a0 = at * TN;
        const int64_t drow = a0 + dl_a;
        auto load_chunk = [&](int c) {
            const int t0 = c * TK;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int t = t0 + zl_f + i;
                zreg[i] = (zrow >= 0 && t < L) ? Z[zrow * L + t] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int t = t0 + dl_f + i;
                dreg[i] = (drow < d && t < L) ? atoms[drow * L + t] : make_float2(0.f, 0.f);
            }
        };
        float acc_re[4][8], acc_im[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) { acc_re[i][j] = 0.f; acc_im[i][j] = 0.f; }

        load_chunk(0);
        for (int c = 0; c < nchunks; ++c) {
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; ++i) Zs[(zl_f + i) * TM + zl_v] = zreg[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) Ds[(dl_f + i) * TN + dl_a] = dreg[i];
            __syncthreads();
            if (c + 1 < nchunks) load_chunk(c + 1);
#pragma unroll 4
            for (int k = 0; k < TK; ++k) {
                float4 za = *reinterpret_cast<const float4*>(&Zs[k * TM + 2 * ty]);
                float4 zb = *reinterpret_cast<const float4*>(&Zs[k * TM + 64 + 2 * ty]);
                float zx[4] = {za.x, za.z, zb.x, zb.z};
                float zy[4] = {za.y, za.w, zb.y, zb.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 dq = *reinterpret_cast<const float4*>(&Ds[k * TN + 16 * q + 2 * tx]);
                    float dx[2] = {dq.x, dq.z};
                    float dy[2] = {dq.y, dq.w};
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            // conj(d) z = (dx zx + dy zy) + i (dx zy - dy zx)
                            acc_re[i][2 * q + r] = fmaf(dx[r], zx[i], acc_re[i][2 * q + r]);
                            acc_re[i][2 * q + r] = fmaf(dy[r], zy[i], acc_re[i][2 * q + r]);
                            acc_im[i][2 * q + r] = fmaf(dx[r], zy[i], acc_im[i][2 * q + r]);
                            acc_im[i][2 * q + r] = fmaf(-dy[r], zx[i], acc_im[i][2 * q + r]);
                        }
                }
            }
        }
        // scores of this tile -> shared memory
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int la = 16 * q + 2 * tx + r;
                const int64_t j = a0 + la;
                float w = (j < d) ? inv_norm2[j] : 0.f;
                float rs = sqrtf(w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int lv = (i < 2) ? (2 * ty + i) : (64 + 2 * ty + i - 2);
                    float re = acc_re[i][2 * q + r], im = acc_im[i][2 * q + r];
                    float sc = (cone == MRF_CONE_COMPLEX) ? (re * re + im * im) * w : re * rs;
                    Ss[lv * SPAD + la] = (j < d) ? sc : -INFINITY;
                }
            }
        __syncthreads();
#pragma unroll 4
        for (int a = 0; a < 32; ++a) {
            const int la = sh * 32 + a;
            const int64_t j = a0 + la;
            if (j < d) topk_insert<KT>(ts, ti, Ss[sv * SPAD + la], static_cast<int32_t>(j));
        }
    }
    // merge the two half-lists of each voxel through shared memory
    __syncthreads();
    float* Ms = Ss;                                        // [TM][2][KT] scores
    int32_t* Mi = reinterpret_cast<int32_t*>(Ss + TM * 2 * KT);
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        Ms[(sv * 2 + sh) * KT + q] = ts[q];
        Mi[(sv * 2 + sh) * KT + q] = ti[q];
    }
    __syncthreads();
    if (sh == 0 && m0 + sv < n) {
        const float* as = Ms + sv * 2 * KT;
        const float* bs = as + KT;
        const int32_t* ai = Mi + sv * 2 * KT;
        const int32_t* bi = ai + KT;
        int pa = 0, pb = 0;
        const int64_t o = (static_cast<int64_t>(s) * n + (m0 + sv)) * KT;
        for (int q = 0; q < KT; ++q) {
            bool takea;
            if (pa >= KT) takea = false;
            else if (pb >= KT) takea = true;
            else if (as[pa] != bs[pb]) takea = as[pa] > bs[pb];
            else takea = (ai[pa] >= 0 && (bi[pb] < 0 || ai[pa] < bi[pb]));
            if (takea) { part_s[o + q] = as[pa]; part_i[o + q] = ai[pa]; ++pa; }
            else { part_s[o + q] = bs[pb]; part_i[o + q] = bi[pb]; ++pb; }
        }
    }
}

constexpr size_t smem_bytes() {
    return sizeof(float2) * (TK * TM + TK * TN) + sizeof(float) * TM * SPAD;
}

}  // namespace

int fp32_choose_splits(int64_t n, int64_t d, int num_sms) {
    // (callers apply mrf_tune.fp32_splits before falling back to this default)
    int64_t Mt = (n + TM - 1) / TM;
    int64_t tiles = (d + TN - 1) / TN;
    int64_t target = 4LL * num_sms;
    int64_t S = (target + Mt - 1) / Mt;
    if (S < 1) S = 1;
    if (S > tiles) S = tiles;
    if (S > 4096) S = 4096;
    return static_cast<int>(S);
}

mrf_status launch_fp32_topk(const float2* Z, const int32_t* vlist, const int32_t* nlist,
                            int64_t n, const mrf_dict* D, int cone, int K, int S,
                            float* part_s, int32_t* part_i, cudaStream_t st) {
    if (n == 0) return MRF_OK;
    int64_t Mt = (n + TM - 1) / TM;
    int64_t tiles = (D->d + TN - 1) / TN;
    int tps = static_cast<int>((tiles + S - 1) / S);
    dim3 grid(static_cast<unsigned>(Mt * S));
    size_t sm = smem_bytes();
    static_assert(smem_bytes() >= sizeof(float) * TM * 2 * 16 * 2, "merge scratch fits");
    if (K == 8) {
        cudaFuncSetAttribute(k_fp32_topk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm));
        k_fp32_topk<8><<<grid, NT, sm, st>>>(Z, vlist, nlist, n, D->atoms, D->inv_norm2, D->d,
                                             D->L, cone, S, tps, part_s, part_i);
    } else if (K == 16) {
        cudaFuncSetAttribute(k_fp32_topk<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm));
        k_fp32_topk<16><<<grid, NT, sm, st>>>(Z, vlist, nlist, n, D->atoms, D->inv_norm2, D->d,
                                              D->L, cone, S, tps, part_s, part_i);
    } else {
        mrf_set_error("fp32 kernel: K must be 8 or 16");
        return MRF_EINVAL;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mrf_set_error(std::string("fp32 kernel launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}
