// Dense products on the 5th-generation tensor cores -- the learned proposal's network layers and
// the cover-tree search's query-to-centre correlations:
//   out[m][n] = act(sum_k A[m][k] W[k][n] + bias[n]),  A [M][Kp] BF16, W given transposed as
//   Wt [N][Kp] BF16 (both K-major), FP32 accumulation in tensor memory, bias (optional) and the
//   activation (GELU or identity) in FP32.
//
// Persistent CTAs, one per SM, walk the 128-row x BN-column output tiles (BN <= 256, a multiple
// of 16 dividing N; tiles column by column, so the CTAs running together share one or two BN-row
// slices of W while the A rows of all of M stay in L2 -- W can be far larger than L2, as with
// the tree search's block centres): warp 0 streams 128-byte K slices of the A tile and of the BN weight rows with TMA
// into a 4-stage ring (128-byte swizzle), warp 1 issues tcgen05.mma kind::f16 128 x BN x 16 (four
// per stage) into one of two 256-column TMEM accumulators, and warps 2..5 drain the other one
// row by row (TMEM lanes 32 (w mod 4) ...), fusing bias + GELU and writing the FP32 activations
// and/or their BF16 copy (the next layer's A operand) while the next tile is multiplied.  Every
// mbarrier wait is bounded; on expiry the CTA raises MRF_DERR_TIMEOUT, waits (bounded) for the
// loads and products it issued and exits.
#include <cuda.h>
#include <string>

#include "mrf_internal.cuh"
#include "ptx.cuh"
#include "tma_host.h"

namespace {

constexpr int TM = 128;                  // rows per tile
constexpr int TK = 64;                   // BF16 elements per 128-byte stage row
constexpr int TSTAGES = 4;
constexpr int TBN_MAX = 256;
constexpr int T_A_BYTES = TM * 128;      // 16 KB
constexpr int T_B_BYTES = TBN_MAX * 128; // 32 KB (a BN-row tile uses BN x 128 bytes of it)
constexpr int T_STAGE = T_A_BYTES + T_B_BYTES;
constexpr int T_THREADS = 192;
constexpr int T_TMEM_COLS = 512;         // two accumulators of up to 256 columns

struct DenseShared {
    uint64_t full[TSTAGES];
    uint64_t empty[TSTAGES];
    uint64_t tfull[2];                   // accumulator ready (MMA commit)
    uint64_t tempty[2];                  // accumulator drained (128 epilogue threads)
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

constexpr size_t kDenseSmem = TSTAGES * T_STAGE + sizeof(DenseShared) + 1024;

__device__ __forceinline__ float gelu(float v) {
    return 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
}

__global__ void __launch_bounds__(T_THREADS, 1)
k_tc_dense_gelu(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                int M, int N, int Kp, int BN, int tiles_m, int tiles, uint32_t idesc,
                const float* __restrict__ bias, int act, float* __restrict__ out,
                __nv_bfloat16* __restrict__ outb, uint32_t* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    DenseShared* sh = reinterpret_cast<DenseShared*>(base + TSTAGES * T_STAGE);
    volatile int* abort_flag = &sh->abort;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nk = (Kp + TK - 1) / TK;
    const uint32_t b_bytes = static_cast<uint32_t>(BN) * 128u;

    if (threadIdx.x == 0) {
        for (int i = 0; i < TSTAGES; ++i) {
            mrfk::mbar_init(&sh->full[i], 1);
            mrfk::mbar_init(&sh->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mrfk::mbar_init(&sh->tfull[i], 1);
            mrfk::mbar_init(&sh->tempty[i], 128);
        }
        mrfk::mbar_init(&sh->drain, 1);
        sh->abort = 0;
        mrfk::fence_mbar_init();
    }
    if (warp == 1) {
        mrfk::tmem_alloc(&sh->tmem_base, T_TMEM_COLS);
        mrfk::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        mrfk::tma_prefetch_desc(&tmA);
        mrfk::tma_prefetch_desc(&tmB);
    }
    mrfk::tc_fence_before();
    __syncthreads();
    mrfk::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    auto fail = [&]() {
        atomicOr(err, MRF_DERR_TIMEOUT);
        *abort_flag = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool used[TSTAGES] = {};
            uint32_t last[TSTAGES] = {};
            for (int t = blockIdx.x; t < tiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (t % tiles_m) * TM;
                const int n0 = (t / tiles_m) * BN;
                for (int kc = 0; kc < nk; ++kc) {
                    if (!mrfk::mbar_wait(&sh->empty[stage], phase ^ 1u)) { fail(); break; }
                    unsigned char* sa = base + stage * T_STAGE;
                    mrfk::mbar_arrive_expect_tx(&sh->full[stage], T_A_BYTES + b_bytes);
                    mrfk::tma_load_2d(sa, &tmA, &sh->full[stage], kc * TK, m0);
                    mrfk::tma_load_2d(sa + T_A_BYTES, &tmB, &sh->full[stage], kc * TK, n0);
                    used[stage] = true;
                    last[stage] = phase;
                    if (++stage == TSTAGES) { stage = 0; phase ^= 1u; }
                }
            }
            // Before the CTA may leave: every fill of its slots has landed, and the products
            // reading them have released them.
            for (int i = 0; i < TSTAGES; ++i) {
                if (!used[i]) continue;
                if (*abort_flag) mrfk::mbar_wait(&sh->full[i], last[i]);
                if (!mrfk::mbar_wait(&sh->empty[i], last[i])) atomicOr(err, MRF_DERR_TIMEOUT);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t aphase = 0;
            bool any = false;
            for (int t = blockIdx.x; t < tiles && !*abort_flag; t += gridDim.x) {
                if (!mrfk::mbar_wait(&sh->tempty[acc], aphase ^ 1u)) { fail(); break; }
                mrfk::tc_fence_after();
                const uint32_t dt = tmem + static_cast<uint32_t>(acc * TBN_MAX);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc) {
                    if (!mrfk::mbar_wait(&sh->full[stage], phase)) { fail(); ok = false; break; }
                    mrfk::tc_fence_after();
                    const uint32_t sa = mrfk::smem_u32(base + stage * T_STAGE);
                    const uint32_t sb = sa + T_A_BYTES;
#pragma unroll
                    for (int k = 0; k < TK / 16; ++k)
                        mrfk::mma_bf16(dt, mrfk::sdesc_k_sw128(sa + k * 32),
                                       mrfk::sdesc_k_sw128(sb + k * 32), idesc,
                                       (kc > 0 || k > 0) ? 1u : 0u);
                    mrfk::mma_commit(&sh->empty[stage]);
                    any = true;
                    if (++stage == TSTAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mrfk::mma_commit(&sh->tfull[acc]);
                if (++acc == 2) { acc = 0; aphase ^= 1u; }
            }
            if (any) {
                // every product issued by this thread completes before TMEM is released
                mrfk::mma_commit(&sh->drain);
                if (!mrfk::mbar_wait(&sh->drain, 0)) atomicOr(err, MRF_DERR_TIMEOUT);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (4 warps)
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        int acc = 0;
        uint32_t aphase = 0;
        for (int t = blockIdx.x; t < tiles && !*abort_flag; t += gridDim.x) {
            const int m = (t % tiles_m) * TM + row;
            const int n0 = (t / tiles_m) * BN;
            if (!mrfk::mbar_wait(&sh->tfull[acc], aphase)) { fail(); break; }
            mrfk::tc_fence_after();
            const uint32_t tb = tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                static_cast<uint32_t>(acc * TBN_MAX);
            for (int c = 0; c * 32 < BN; ++c) {
                uint32_t r[32];
                __syncwarp();
                mrfk::tmem_ld32(tb + c * 32, r);
                mrfk::tmem_ld_wait();
                if (m >= M) continue;
                const int nb = n0 + c * 32;
                const int cnt = BN - c * 32 < 32 ? BN - c * 32 : 32;
                float g[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float v =
                        i < cnt ? __uint_as_float(r[i]) + (bias ? bias[nb + i] : 0.f) : 0.f;
                    g[i] = act ? gelu(v) : v;
                }
                const int64_t o = static_cast<int64_t>(m) * N + nb;
                if (cnt == 32) {           // 16-byte stores (N and nb are multiples of 16)
                    if (out) {
                        float4* d = reinterpret_cast<float4*>(out + o);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            d[i] = make_float4(g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
                    }
                    if (outb) {
                        uint4* d = reinterpret_cast<uint4*>(outb + o);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            __nv_bfloat162 h[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                h[q] = __floats2bfloat162_rn(g[8 * i + 2 * q], g[8 * i + 2 * q + 1]);
                            d[i] = *reinterpret_cast<uint4*>(h);
                        }
                    }
                } else {
                    for (int i = 0; i < cnt; ++i) {
                        if (out) out[o + i] = g[i];
                        if (outb) outb[o + i] = __float2bfloat16_rn(g[i]);
                    }
                }
            }
            mrfk::tc_fence_before();
            mrfk::mbar_arrive(&sh->tempty[acc]);
            if (++acc == 2) { acc = 0; aphase ^= 1u; }
        }
    }
    mrfk::tc_fence_before();
    __syncthreads();
    mrfk::tc_fence_after();
    if (warp == 1) mrfk::tmem_dealloc(tmem, T_TMEM_COLS);
}

}  // namespace

int dense_tile_n(int N) {
    if (N <= 0 || N % 16) return 0;
    int bn = N < TBN_MAX ? N : TBN_MAX;
    while (bn > 16 && N % bn) bn -= 16;
    return bn;
}

mrf_status launch_dense_gelu(const __nv_bfloat16* A, int M, int Kp, const __nv_bfloat16* Wt,
                             int N, const float* bias, float* out, __nv_bfloat16* outb,
                             uint32_t* err, cudaStream_t st) {
    return launch_dense(A, M, Kp, Wt, N, bias, 1, out, outb, err, st);
}

mrf_status launch_dense(const __nv_bfloat16* A, int M, int Kp, const __nv_bfloat16* Wt, int N,
                        const float* bias, int act, float* out, __nv_bfloat16* outb,
                        uint32_t* err, cudaStream_t st) {
    if (M == 0) return MRF_OK;
    const int BN = dense_tile_n(N);
    if (BN == 0 || Kp <= 0 || (Kp * 2) % 16) {
        mrf_set_error("dense layer: N must be a multiple of 16 and the row pitch of 16 bytes");
        return MRF_EINVAL;
    }
    CUtensorMap ta, tb;
    MRF_TRY(tma_map_k128(&ta, A, M, Kp, TM, false));
    MRF_TRY(tma_map_k128(&tb, Wt, N, Kp, BN, false));
    const uint32_t idesc = mrfk::idesc_bf16(TM, static_cast<uint32_t>(BN));
    const int tiles_m = (M + TM - 1) / TM;
    const int64_t tiles64 = static_cast<int64_t>(tiles_m) * (N / BN);
    if (tiles64 > INT32_MAX) {
        mrf_set_error("dense layer: more than 2^31 - 1 output tiles");
        return MRF_EINVAL;
    }
    const int tiles = static_cast<int>(tiles64);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_dense_gelu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kDenseSmem));
    if (e == cudaSuccess) {
        const int grid = sms < tiles ? sms : tiles;          // one persistent CTA per SM
        k_tc_dense_gelu<<<grid, T_THREADS, kDenseSmem, st>>>(ta, tb, M, N, Kp, BN, tiles_m,
                                                             tiles, idesc, bias, act, out, outb,
                                                             err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("dense layer launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}
