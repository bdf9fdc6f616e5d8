// The gradient step of §3.2 eq. blip in one pass for power-of-two Ny:
//   Z = X - mu (A^H A X - A^H Y),   A^H A = F_y^H P_t F_y per frame (F_x cancels for line masks).
//
// A CTA owns 16 consecutive columns c = x L + t of the [Ny][Nx][L] image (stride Nx L between
// phase-encode rows, so each row of the tile is one coalesced 128-byte load; 32 KB of shared
// memory, so six CTAs share an SM and hide the passes' latency -- 0.65 ms per 256 x 256 x 1000
// step against 0.90 ms with 32-column tiles and 0.81 ms with 8).  It transforms the
// tile along y in shared memory (decimation in time on bit-reversed input, natural-order
// k-space, two radix-2 stages per shared-memory pass), zeroes the lines that frame t did not
// sample, transforms back (decimation in frequency, conjugate twiddles, bit-reversed result),
// and combines with X and A^H Y while
// writing Z and the BF16 query operand.  One read of X, X again for the combine (L2), A^H Y,
// and the writes of Z and the operand: instead of two cuFFT passes, a mask pass and a combine
// pass over the whole image.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "mrf_internal.cuh"

namespace {

constexpr int NT = 256;         // threads per CTA
constexpr int kTileLog = 4;     // log2 of the columns per CTA

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Forward transform along y of the TC columns of the tile s ([Ny][TC], bit-reversed rows on
// entry, natural-order k-space on exit): decimation in time, two radix-2 stages per pass (a
// quadruple {i, i + h, i + 2h, i + 3h} closes under the stages h and 2h), a last single stage
// when log2 Ny is odd.  Ends with a barrier.
template <int LTC>
__device__ __forceinline__ void tile_fft_fwd(float2* s, const float2* w, int Ny, int logNy,
                                             int tid, int jt) {
    constexpr int TC = 1 << LTC;
    const int nbf = (Ny / 2) * TC;
    const int nq = (Ny / 4) * TC;
    for (int lh = 0; lh < logNy;) {
        const int h = 1 << lh;
        if (lh + 1 < logNy) {
            for (int q = tid; q < nq; q += NT) {
                const int b = q >> LTC;
                const int g = b >> lh, p = b & (h - 1);
                const int i = (((g << (lh + 2)) + p) << LTC) + jt, hs = h << LTC;
                const float2 a0 = s[i], a1 = s[i + hs], a2 = s[i + 2 * hs], a3 = s[i + 3 * hs];
                const float2 w1 = w[p << (logNy - 1 - lh)];
                const float2 wa = w[p << (logNy - 2 - lh)], wb = w[(p + h) << (logNy - 2 - lh)];
                const float2 t1 = cmul(a1, w1), t3 = cmul(a3, w1);
                const float2 b0 = make_float2(a0.x + t1.x, a0.y + t1.y);
                const float2 b1 = make_float2(a0.x - t1.x, a0.y - t1.y);
                const float2 b2 = make_float2(a2.x + t3.x, a2.y + t3.y);
                const float2 b3 = make_float2(a2.x - t3.x, a2.y - t3.y);
                const float2 u2 = cmul(b2, wa), u3 = cmul(b3, wb);
                s[i] = make_float2(b0.x + u2.x, b0.y + u2.y);
                s[i + 2 * hs] = make_float2(b0.x - u2.x, b0.y - u2.y);
                s[i + hs] = make_float2(b1.x + u3.x, b1.y + u3.y);
                s[i + 3 * hs] = make_float2(b1.x - u3.x, b1.y - u3.y);
            }
            lh += 2;
        } else {
            for (int q = tid; q < nbf; q += NT) {
                const int b = q >> LTC;
                const int g = b >> lh, p = b & (h - 1);
                const int i0 = (((g << (lh + 1)) + p) << LTC) + jt, i1 = i0 + (h << LTC);
                const float2 u = s[i0], v = cmul(s[i1], w[p << (logNy - 1 - lh)]);
                s[i0] = make_float2(u.x + v.x, u.y + v.y);
                s[i1] = make_float2(u.x - v.x, u.y - v.y);
            }
            lh += 1;
        }
        __syncthreads();
    }
}

// Inverse transform along y (natural-order rows on entry, bit-reversed rows on exit, no 1/Ny):
// decimation in frequency with conjugate twiddles, stages 2q and q in one pass on the quadruple
// {i, i + q, i + 2q, i + 3q}.  Ends with a barrier.
template <int LTC>
__device__ __forceinline__ void tile_fft_inv(float2* s, const float2* w, int Ny, int logNy,
                                             int tid, int jt) {
    constexpr int TC = 1 << LTC;
    const int nbf = (Ny / 2) * TC;
    const int nq = (Ny / 4) * TC;
    for (int lh = logNy - 1; lh >= 0;) {
        if (lh >= 1) {
            const int qq = 1 << (lh - 1);
            for (int q = tid; q < nq; q += NT) {
                const int b = q >> LTC;
                const int g = b >> (lh - 1), p0 = b & (qq - 1);
                const int i = (((g << (lh + 1)) + p0) << LTC) + jt, qst = qq << LTC;
                const float2 a0 = s[i], a1 = s[i + qst], a2 = s[i + 2 * qst], a3 = s[i + 3 * qst];
                const float2 ta = w[p0 << (logNy - 1 - lh)], tb = w[(p0 + qq) << (logNy - 1 - lh)];
                const float2 tc = w[p0 << (logNy - lh)];
                const float2 wa = make_float2(ta.x, -ta.y), wb = make_float2(tb.x, -tb.y);
                const float2 wc = make_float2(tc.x, -tc.y);
                const float2 b0 = make_float2(a0.x + a2.x, a0.y + a2.y);
                const float2 b2 = cmul(make_float2(a0.x - a2.x, a0.y - a2.y), wa);
                const float2 b1 = make_float2(a1.x + a3.x, a1.y + a3.y);
                const float2 b3 = cmul(make_float2(a1.x - a3.x, a1.y - a3.y), wb);
                s[i] = make_float2(b0.x + b1.x, b0.y + b1.y);
                s[i + qst] = cmul(make_float2(b0.x - b1.x, b0.y - b1.y), wc);
                s[i + 2 * qst] = make_float2(b2.x + b3.x, b2.y + b3.y);
                s[i + 3 * qst] = cmul(make_float2(b2.x - b3.x, b2.y - b3.y), wc);
            }
            lh -= 2;
        } else {
            for (int q = tid; q < nbf; q += NT) {       // h = 1: twiddle 1
                const int b = q >> LTC;
                const int i0 = (b << (LTC + 1)) + jt, i1 = i0 + TC;
                const float2 u = s[i0], v = s[i1];
                s[i0] = make_float2(u.x + v.x, u.y + v.y);
                s[i1] = make_float2(u.x - v.x, u.y - v.y);
            }
            lh -= 1;
        }
        __syncthreads();
    }
}

// Z = X - mu (G / Ny - AHY) for the tile's columns, G = the tile (bit-reversed rows) read back
// in natural order; also the BF16 query operand of Z when zq is given.
template <int LTC>
__device__ __forceinline__ void tile_combine(const float2* s, const float2* __restrict__ X,
                                             const float2* __restrict__ AHY, int Ny, int logNy,
                                             int Nx, int L, float mu, float2* __restrict__ Z,
                                             __nv_bfloat162* __restrict__ zq, int Kp,
                                             uint32_t* err, int tid, int jt, int64_t ct,
                                             bool live) {
    constexpr int TC = 1 << LTC;
    const int64_t NxL = static_cast<int64_t>(Nx) * L;
    const float gs = 1.0f / static_cast<float>(Ny);
    const int half = Kp / 2;
    if (!live) return;
    const int tcol = static_cast<int>(ct % L);
    const int64_t xcol = ct / L;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        const int r = static_cast<int>(__brev(static_cast<unsigned>(ky)) >> (32 - logNy));
        const float2 gv = s[(r << LTC) + jt];
        const int64_t o = static_cast<int64_t>(ky) * NxL + ct;
        const float2 x = X[o], a = AHY[o];
        float2 z;
        z.x = x.x - mu * (gs * gv.x - a.x);
        z.y = x.y - mu * (gs * gv.y - a.y);
        if (!isfinite(z.x) || !isfinite(z.y)) atomicOr(err, MRF_DERR_NONFINITE);
        Z[o] = z;
        if (zq) {
            const int64_t v = static_cast<int64_t>(ky) * Nx + xcol;
            zq[v * half + tcol] = __floats2bfloat162_rn(z.x, z.y);
            if (tcol == L - 1)
                for (int tt = L; tt < half; ++tt) zq[v * half + tt] = __floats2bfloat162_rn(0.f, 0.f);
        }
    }
}

// tw[k] = exp(-2 pi i k / Ny), k < Ny / 2.  A CTA owns TC = 2^LTC columns.
template <int LTC>
__global__ void __launch_bounds__(NT)
k_grad_pow2(const float2* __restrict__ X, const float2* __restrict__ AHY,
            const uint8_t* __restrict__ mask, const float2* __restrict__ tw, int Ny, int logNy,
            int Nx, int L, float mu, float2* __restrict__ Z, __nv_bfloat162* __restrict__ zq,
            int Kp, uint32_t* err) {
    constexpr int TC = 1 << LTC;
    extern __shared__ float2 sbuf[];            // [Ny][TC] tile, then [Ny / 2] twiddles
    float2* s = sbuf;
    float2* w = sbuf + Ny * TC;
    const int tid = threadIdx.x;
    const int64_t NxL = static_cast<int64_t>(Nx) * L;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * TC;
    for (int k = tid; k < Ny / 2; k += NT) w[k] = tw[k];
    // every index a thread touches has column j = tid mod TC (NT is a multiple of TC)
    const int jt = tid & (TC - 1);
    const int64_t ct = c0 + jt;
    const bool live = ct < NxL;
    const int tcol = live ? static_cast<int>(ct % L) : 0;      // frame of the column
    const int64_t xcol = live ? ct / L : 0;                     // x of the column
    // load X bit-reversed along y
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        const int r = static_cast<int>(__brev(static_cast<unsigned>(ky)) >> (32 - logNy));
        s[(r << LTC) + jt] = live ? X[static_cast<int64_t>(ky) * NxL + ct] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    tile_fft_fwd<LTC>(s, w, Ny, logNy, tid, jt);
    // keep the sampled lines of each column's frame
    const uint8_t* mrow = mask + static_cast<int64_t>(tcol) * Ny;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        if (!live || !mrow[ky]) s[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    tile_fft_inv<LTC>(s, w, Ny, logNy, tid, jt);
    tile_combine<LTC>(s, X, AHY, Ny, logNy, Nx, L, mu, Z, zq, Kp, err, tid, jt, ct, live);
}

// The two halves of the one-pass kernel around an operator that mixes the columns of one
// phase-encode line (the compressed gradient of §3.3, eq. gradcompression, where the per-frame
// masks become an s x s product per line): the forward y-transform of every column into W
// (natural-order k-space, no scaling), and the inverse y-transform of W2 followed by the same
// combine as above.
template <int LTC>
__global__ void __launch_bounds__(NT)
k_yfft_fwd(const float2* __restrict__ X, const float2* __restrict__ tw, int Ny, int logNy,
           int64_t NxL, float2* __restrict__ W) {
    constexpr int TC = 1 << LTC;
    extern __shared__ float2 sbuf[];
    float2* s = sbuf;
    float2* w = sbuf + Ny * TC;
    const int tid = threadIdx.x;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * TC;
    for (int k = tid; k < Ny / 2; k += NT) w[k] = tw[k];
    const int jt = tid & (TC - 1);
    const int64_t ct = c0 + jt;
    const bool live = ct < NxL;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        const int r = static_cast<int>(__brev(static_cast<unsigned>(ky)) >> (32 - logNy));
        s[(r << LTC) + jt] = live ? X[static_cast<int64_t>(ky) * NxL + ct] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    tile_fft_fwd<LTC>(s, w, Ny, logNy, tid, jt);
    if (!live) return;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        W[static_cast<int64_t>(ky) * NxL + ct] = s[i];
    }
}

template <int LTC>
__global__ void __launch_bounds__(NT)
k_yfft_inv_combine(const float2* __restrict__ W2, const float2* __restrict__ X,
                   const float2* __restrict__ AHY, const float2* __restrict__ tw, int Ny,
                   int logNy, int Nx, int L, float mu, float2* __restrict__ Z,
                   __nv_bfloat162* __restrict__ zq, int Kp, uint32_t* err) {
    constexpr int TC = 1 << LTC;
    extern __shared__ float2 sbuf[];
    float2* s = sbuf;
    float2* w = sbuf + Ny * TC;
    const int tid = threadIdx.x;
    const int64_t NxL = static_cast<int64_t>(Nx) * L;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * TC;
    for (int k = tid; k < Ny / 2; k += NT) w[k] = tw[k];
    const int jt = tid & (TC - 1);
    const int64_t ct = c0 + jt;
    const bool live = ct < NxL;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        s[i] = live ? W2[static_cast<int64_t>(ky) * NxL + ct] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    tile_fft_inv<LTC>(s, w, Ny, logNy, tid, jt);
    tile_combine<LTC>(s, X, AHY, Ny, logNy, Nx, L, mu, Z, zq, Kp, err, tid, jt, ct, live);
}

std::mutex g_tw_mu;
std::map<std::pair<int, int>, float2*> g_tw;     // (device, Ny) -> twiddles

mrf_status twiddles(int Ny, const float2** out) {
    int dev = 0;
    MRF_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto key = std::make_pair(dev, Ny);
    auto it = g_tw.find(key);
    if (it != g_tw.end()) { *out = it->second; return MRF_OK; }
    std::vector<float2> h(Ny / 2);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < Ny / 2; ++k) {
        const double a = two_pi * k / Ny;
        h[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(-std::sin(a)));
    }
    float2* d = nullptr;
    MRF_CUDA_TRY(cudaMalloc(&d, sizeof(float2) * h.size()));
    MRF_CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
    g_tw[key] = d;
    *out = d;
    return MRF_OK;
}

}  // namespace

bool grad_fused_supported(int Ny) {
    return Ny >= 2 && Ny <= 512 && (Ny & (Ny - 1)) == 0;
}

mrf_status launch_grad_fused(const mrf_op* op, const float2* AHY, const float2* X, float mu,
                             float2* Z, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st) {
    const int Ny = op->Ny;
    int logNy = 0;
    while ((1 << logNy) < Ny) ++logNy;
    const float2* tw = nullptr;
    MRF_TRY(twiddles(Ny, &tw));
    const int64_t cols = static_cast<int64_t>(op->Nx) * op->L;
    constexpr int LTC = kTileLog;
    constexpr int TC = 1 << LTC;
    const size_t sm = sizeof(float2) * (static_cast<size_t>(Ny) * TC + Ny / 2);
    cudaError_t e = cudaFuncSetAttribute(k_grad_pow2<LTC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess) {
        k_grad_pow2<LTC><<<static_cast<unsigned>((cols + TC - 1) / TC), NT, sm, st>>>(
            X, AHY, op->mask, tw, Ny, logNy, op->Nx, op->L, mu, Z,
            reinterpret_cast<__nv_bfloat162*>(zq), zq ? Kp : 2 * op->L, err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("fused gradient launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

namespace {
int log2_of(int Ny) {
    int l = 0;
    while ((1 << l) < Ny) ++l;
    return l;
}
}  // namespace

mrf_status launch_yfft_fwd(const float2* X, int Ny, int Nx, int C, float2* W, cudaStream_t st) {
    const int logNy = log2_of(Ny);
    const float2* tw = nullptr;
    MRF_TRY(twiddles(Ny, &tw));
    const int64_t cols = static_cast<int64_t>(Nx) * C;
    constexpr int LTC = kTileLog;
    constexpr int TC = 1 << LTC;
    const size_t sm = sizeof(float2) * (static_cast<size_t>(Ny) * TC + Ny / 2);
    cudaError_t e = cudaFuncSetAttribute(k_yfft_fwd<LTC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess) {
        k_yfft_fwd<LTC><<<static_cast<unsigned>((cols + TC - 1) / TC), NT, sm, st>>>(
            X, tw, Ny, logNy, cols, W);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("forward y-transform launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

mrf_status launch_yfft_inv_combine(const float2* W2, const float2* X, const float2* AHY, int Ny,
                                   int Nx, int C, float mu, float2* Z, __nv_bfloat16* zq, int Kp,
                                   uint32_t* err, cudaStream_t st) {
    const int logNy = log2_of(Ny);
    const float2* tw = nullptr;
    MRF_TRY(twiddles(Ny, &tw));
    const int64_t cols = static_cast<int64_t>(Nx) * C;
    constexpr int LTC = kTileLog;
    constexpr int TC = 1 << LTC;
    const size_t sm = sizeof(float2) * (static_cast<size_t>(Ny) * TC + Ny / 2);
    cudaError_t e = cudaFuncSetAttribute(k_yfft_inv_combine<LTC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess) {
        k_yfft_inv_combine<LTC><<<static_cast<unsigned>((cols + TC - 1) / TC), NT, sm, st>>>(
            W2, X, AHY, tw, Ny, logNy, Nx, C, mu, Z, reinterpret_cast<__nv_bfloat162*>(zq),
            zq ? Kp : 2 * C, err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("inverse y-transform launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}
