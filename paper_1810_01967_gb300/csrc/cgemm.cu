// Small batched complex products of the subspace-compressed iteration (§3.3, eqs. CS1,
// gradupdate, gradcompression): compression X conj(V_s) and expansion Xc V_s^T of fingerprint
// rows, the per-line operators H_ky = V_s^H diag(mask[., ky]) V_s, and their application to the
// compressed k-space rows of every phase-encode line.  All are
//   Out[b][r][j] = sum_k In[b][r][k] m_b(k) op(M[b][k][j])
// over row-major operands, FP32 complex with FP32 accumulation.  The shapes are thin (s <= L,
// 20..200 compressed frames) and the operands of one batch fit L2, so a shared-memory tiled
// SIMT product is enough: 32 x 32 outputs per CTA of 16 x 16 threads, each thread 2 x 2
// outputs, K in steps of 16.
#include "mrf_internal.cuh"

namespace {

constexpr int TM = 32, TN = 32, TK = 16;

template <bool CONJ, bool MASKED>
__global__ void __launch_bounds__(256)
k_cgemm(const float2* __restrict__ In, int64_t in_ld, int64_t in_bs,
        const float2* __restrict__ M, int64_t m_ld, int64_t m_bs,
        float2* __restrict__ Out, int64_t out_ld, int64_t out_bs, int R, int K, int J,
        const uint8_t* __restrict__ kmask, int64_t kmask_ld, int64_t kmask_bs) {
    __shared__ float2 sA[TM][TK + 1];
    __shared__ float2 sB[TK][TN + 1];
    const int64_t b = blockIdx.z;
    const int r0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const float2* A = In + b * in_bs;
    const float2* B = M + b * m_bs;
    const uint8_t* mk = MASKED ? kmask + b * kmask_bs : nullptr;
    float2 acc[2][2] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f)},
                        {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {       // In tile [32][16]
            const int rr = e / TK, kk = e - rr * TK;
            const int r = r0 + rr, k = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (r < R && k < K) {
                v = A[static_cast<int64_t>(r) * in_ld + k];
                if (MASKED && !mk[static_cast<int64_t>(k) * kmask_ld]) v = make_float2(0.f, 0.f);
            }
            sA[rr][kk] = v;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {       // M tile [16][32]
            const int kk = e / TN, jj = e - kk * TN;
            const int k = k0 + kk, j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (k < K && j < J) {
                v = B[static_cast<int64_t>(k) * m_ld + j];
                if (CONJ) v.y = -v.y;
            }
            sB[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            const float2 a0 = sA[ty][kk], a1 = sA[ty + 16][kk];
            const float2 b0 = sB[kk][tx], b1 = sB[kk][tx + 16];
            acc[0][0].x = fmaf(a0.x, b0.x, fmaf(-a0.y, b0.y, acc[0][0].x));
            acc[0][0].y = fmaf(a0.x, b0.y, fmaf(a0.y, b0.x, acc[0][0].y));
            acc[0][1].x = fmaf(a0.x, b1.x, fmaf(-a0.y, b1.y, acc[0][1].x));
            acc[0][1].y = fmaf(a0.x, b1.y, fmaf(a0.y, b1.x, acc[0][1].y));
            acc[1][0].x = fmaf(a1.x, b0.x, fmaf(-a1.y, b0.y, acc[1][0].x));
            acc[1][0].y = fmaf(a1.x, b0.y, fmaf(a1.y, b0.x, acc[1][0].y));
            acc[1][1].x = fmaf(a1.x, b1.x, fmaf(-a1.y, b1.y, acc[1][1].x));
            acc[1][1].y = fmaf(a1.x, b1.y, fmaf(a1.y, b1.x, acc[1][1].y));
        }
        __syncthreads();
    }
    float2* C = Out + b * out_bs;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < R && c < J) C[static_cast<int64_t>(r) * out_ld + c] = acc[i][j];
        }
}

__global__ void k_cdot_re(const float2* __restrict__ a, const float2* __restrict__ b,
                          int64_t count, double* out) {
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 x = a[i], y = b[i];
        s += static_cast<double>(x.x) * y.x + static_cast<double>(x.y) * y.y;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

}  // namespace

mrf_status launch_cgemm(const float2* In, int64_t in_ld, int64_t in_bs, const float2* M,
                        int64_t m_ld, int64_t m_bs, bool conj_m, float2* Out, int64_t out_ld,
                        int64_t out_bs, int R, int K, int J, int batches, const uint8_t* kmask,
                        int64_t kmask_ld, int64_t kmask_bs, cudaStream_t st) {
    if (R <= 0 || J <= 0 || batches <= 0) return MRF_OK;
    if (batches > 65535) {
        mrf_set_error("complex product: more than 65535 batches");
        return MRF_EINVAL;
    }
    const dim3 grid(static_cast<unsigned>((J + TN - 1) / TN), static_cast<unsigned>((R + TM - 1) / TM),
                    static_cast<unsigned>(batches));
#define MRF_CG_ARGS In, in_ld, in_bs, M, m_ld, m_bs, Out, out_ld, out_bs, R, K, J, kmask, kmask_ld, kmask_bs
    if (kmask) {
        if (conj_m) k_cgemm<true, true><<<grid, 256, 0, st>>>(MRF_CG_ARGS);
        else k_cgemm<false, true><<<grid, 256, 0, st>>>(MRF_CG_ARGS);
    } else {
        if (conj_m) k_cgemm<true, false><<<grid, 256, 0, st>>>(MRF_CG_ARGS);
        else k_cgemm<false, false><<<grid, 256, 0, st>>>(MRF_CG_ARGS);
    }
#undef MRF_CG_ARGS
    MRF_CUDA_TRY(cudaGetLastError());
    return MRF_OK;
}

mrf_status launch_cdot_re(const float2* a, const float2* b, int64_t count, double* out,
                          cudaStream_t st) {
    if (count == 0) return MRF_OK;
    k_cdot_re<<<1024, 256, 0, st>>>(a, b, count, out);
    MRF_CUDA_TRY(cudaGetLastError());
    return MRF_OK;
}
