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

// ------------------------------------------------------------------ any Ny with factors 2, 3, 5
// The same gradient step for Ny = 2^a 3^b 5^c (up to kMultiMaxNy), and for many slices of
// different sizes in one launch (the stacked slices of a batch): a CTA owns TC columns of one
// slice, found from its tile index in the slices' descriptor table.  The y-transforms are
// Stockham autosort passes of radix 4, 2, 3 and 5 between two shared-memory buffers (natural
// order in and out), with a full-length twiddle table exp(-2 pi i m / Ny).
namespace {

constexpr int kMultiMaxNy = 512;
constexpr float kC3 = 0.86602540378443864676f;          // sin(2 pi / 3)
constexpr float kC51 = 0.30901699437494742410f;         // cos(2 pi / 5)
constexpr float kC52 = -0.80901699437494742410f;        // cos(4 pi / 5)
constexpr float kS51 = 0.95105651629515357212f;         // sin(2 pi / 5)
constexpr float kS52 = 0.58778525229247312917f;         // sin(4 pi / 5)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// s i z for the sign s = +1 / -1
__device__ __forceinline__ float2 cmul_si(float2 z, float s) { return make_float2(-s * z.y, s * z.x); }

// In-place DFT of size R (2, 3, 4, 5) with kernel exp(s 2 pi i r k / R).
__device__ __forceinline__ void small_dft(float2 (&v)[5], int R, float s) {
    if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = cmul_si(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if (R == 3) {
        const float2 u = cadd(v[1], v[2]), w = cmul_si(csub(v[1], v[2]), s * kC3);
        const float2 m = csub(v[0], cscale(u, 0.5f));
        v[0] = cadd(v[0], u);
        v[1] = cadd(m, w);
        v[2] = csub(m, w);
    } else {   // R == 5
        const float2 b1 = cadd(v[1], v[4]), b2 = cadd(v[2], v[3]);
        const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        const float2 a0 = v[0];
        const float2 p1 = cadd(a0, cadd(cscale(b1, kC51), cscale(b2, kC52)));
        const float2 p2 = cadd(a0, cadd(cscale(b1, kC52), cscale(b2, kC51)));
        const float2 q1 = cmul_si(cadd(cscale(d1, kS51), cscale(d2, kS52)), s);
        const float2 q2 = cmul_si(csub(cscale(d1, kS52), cscale(d2, kS51)), s);
        v[0] = cadd(a0, cadd(b1, b2));
        v[1] = cadd(p1, q1);
        v[4] = csub(p1, q1);
        v[2] = cadd(p2, q2);
        v[3] = csub(p2, q2);
    }
}

// Stockham y-transform of the TC columns of `a` ([Ny][TC], natural order); the result is in
// the returned buffer (a or b).  s = -1 forward, +1 inverse (unscaled).  Ends with a barrier.
template <int LTC>
__device__ float2* tile_fft_mixed(float2* a, float2* b, const float2* tw, int Ny, float s,
                                  int tid, int jt) {
    constexpr int TC = 1 << LTC;
    int rem = Ny, Ns = 1;
    while (rem > 1) {
        const int R = (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : (rem % 3 == 0) ? 3 : 5;
        const int NR = Ny / R;
        const int step = Ny / (Ns * R);          // twiddle index stride for k * r
        for (int q = tid; q < NR * TC; q += NT) {
            const int j = q >> LTC;
            const int k = j % Ns;
            float2 v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) v[r] = a[((j + r * NR) << LTC) + jt];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < 5; ++r)
                    if (r < R) {
                        float2 w = tw[(k * r * step) % Ny];      // exp(-2 pi i m / Ny)
                        if (s > 0.f) w.y = -w.y;                   // inverse: conjugate
                        v[r] = cmul(v[r], w);
                    }
            }
            small_dft(v, R, s);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) b[((base + r * Ns) << LTC) + jt] = v[r];
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
        rem /= R;
    }
    return a;
}


// Per-slice descriptor of a multi-slice launch (slices stacked voxel-major: slice i's voxels
// start at row voff of the stacked [n][L] arrays).
struct SliceDesc {
    int64_t voff;          // first stacked voxel of the slice
    int64_t tile0;         // first CTA tile of the slice
    int32_t Ny, Nx;
    const uint8_t* mask;   // [L][Ny]
    const float2* tw;      // [Ny] exp(-2 pi i m / Ny)
};

// One CTA: TC consecutive columns c = x L + t of one slice.  Dynamic shared memory: two
// [maxNy][TC] buffers and the twiddles.
template <int LTC>
__global__ void __launch_bounds__(NT)
k_grad_multi(const SliceDesc* __restrict__ descs, SliceDesc one, int nslices, int maxNy,
             const float2* __restrict__ X, const float2* __restrict__ AHY, int L, float mu,
             float2* __restrict__ Z, __nv_bfloat162* __restrict__ zq, int Kp, uint32_t* err) {
    constexpr int TC = 1 << LTC;
    extern __shared__ float2 sbuf[];
    __shared__ int s_slice;
    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    if (tid == 0) {
        int lo = 0, hi = nslices - 1;             // last slice whose tile0 <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
        }
        s_slice = lo;
    }
    __syncthreads();
    const SliceDesc sd = (nslices == 1 && descs == nullptr) ? one : descs[s_slice];
    const int Ny = sd.Ny, Nx = sd.Nx;
    float2* bufA = sbuf;
    float2* bufB = sbuf + static_cast<int64_t>(maxNy) * TC;
    float2* w = sbuf + 2 * static_cast<int64_t>(maxNy) * TC;
    for (int k = tid; k < Ny; k += NT) w[k] = sd.tw[k];
    const int64_t NxL = static_cast<int64_t>(Nx) * L;
    const int jt = tid & (TC - 1);
    const int64_t ct = (tile - sd.tile0) * TC + jt;
    const bool live = ct < NxL;
    const int tcol = live ? static_cast<int>(ct % L) : 0;
    const int64_t xcol = live ? ct / L : 0;
    const float2* Xs = X + sd.voff * L;
    const float2* As = AHY + sd.voff * L;
    float2* Zs = Z + sd.voff * L;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        bufA[i] = live ? Xs[static_cast<int64_t>(ky) * NxL + ct] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* kf = tile_fft_mixed<LTC>(bufA, bufB, w, Ny, -1.f, tid, jt);
    const uint8_t* mrow = sd.mask + static_cast<int64_t>(tcol) * Ny;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        if (!live || !mrow[ky]) kf[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* other = (kf == bufA) ? bufB : bufA;
    const float2* g = tile_fft_mixed<LTC>(kf, other, w, Ny, 1.f, tid, jt);
    if (!live) return;
    const float gs = 1.0f / static_cast<float>(Ny);
    const int half = Kp / 2;
    for (int i = tid; i < Ny * TC; i += NT) {
        const int ky = i >> LTC;
        const float2 gv = g[i];
        const int64_t o = static_cast<int64_t>(ky) * NxL + ct;
        const float2 x = Xs[o], a = As[o];
        float2 z;
        z.x = x.x - mu * (gs * gv.x - a.x);
        z.y = x.y - mu * (gs * gv.y - a.y);
        if (!isfinite(z.x) || !isfinite(z.y)) atomicOr(err, MRF_DERR_NONFINITE);
        Zs[o] = z;
        if (zq) {
            const int64_t v = sd.voff + static_cast<int64_t>(ky) * Nx + xcol;
            zq[v * half + tcol] = __floats2bfloat162_rn(z.x, z.y);
            if (tcol == L - 1)
                for (int tt = L; tt < half; ++tt) zq[v * half + tt] = __floats2bfloat162_rn(0.f, 0.f);
        }
    }
}

std::mutex g_twf_mu;
std::map<std::pair<int, int>, float2*> g_twf;    // (device, Ny) -> full-length twiddles

mrf_status twiddles_full(int Ny, const float2** out) {
    int dev = 0;
    MRF_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_twf_mu);
    auto key = std::make_pair(dev, Ny);
    auto it = g_twf.find(key);
    if (it != g_twf.end()) { *out = it->second; return MRF_OK; }
    std::vector<float2> h(Ny);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < Ny; ++k) {
        const double a = two_pi * k / Ny;
        h[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(-std::sin(a)));
    }
    float2* d = nullptr;
    MRF_CUDA_TRY(cudaMalloc(&d, sizeof(float2) * h.size()));
    MRF_CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
    g_twf[key] = d;
    *out = d;
    return MRF_OK;
}

size_t multi_smem(int maxNy) {
    constexpr int TC = 1 << kTileLog;
    return sizeof(float2) * (2 * static_cast<size_t>(maxNy) * TC + maxNy);
}

mrf_status launch_multi(const SliceDesc* descs, SliceDesc one, int nslices, int64_t tiles,
                        int maxNy, const float2* X, const float2* AHY, int L, float mu, float2* Z,
                        __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st) {
    constexpr int LTC = kTileLog;
    const size_t sm = multi_smem(maxNy);
    cudaError_t e = cudaFuncSetAttribute(k_grad_multi<LTC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess) {
        k_grad_multi<LTC><<<static_cast<unsigned>(tiles), NT, sm, st>>>(
            descs, one, nslices, maxNy, X, AHY, L, mu, Z, reinterpret_cast<__nv_bfloat162*>(zq),
            zq ? Kp : 2 * L, err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("multi-slice gradient launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

}  // namespace

bool grad_multi_supported(int Ny) {
    if (Ny < 2 || Ny > kMultiMaxNy) return false;
    int r = Ny;
    for (int f : {2, 3, 5})
        while (r % f == 0) r /= f;
    return r == 1;
}

mrf_status launch_grad_mixed(const mrf_op* op, const float2* AHY, const float2* X, float mu,
                             float2* Z, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st) {
    SliceDesc one{};
    one.voff = 0;
    one.tile0 = 0;
    one.Ny = op->Ny;
    one.Nx = op->Nx;
    one.mask = op->mask;
    MRF_TRY(twiddles_full(op->Ny, &one.tw));
    constexpr int TC = 1 << kTileLog;
    const int64_t tiles = (static_cast<int64_t>(op->Nx) * op->L + TC - 1) / TC;
    return launch_multi(nullptr, one, 1, tiles, op->Ny, X, AHY, op->L, mu, Z, zq, Kp, err, st);
}

// The batch's slices in one launch: builds the descriptor table (device memory owned by the
// caller through *table, reused while the slices stay the same).
mrf_status grad_multi_table(const mrf_op* ops, const int64_t* voff, int nslices, void** table,
                            int64_t* tiles, int* maxNy, cudaStream_t st) {
    constexpr int TC = 1 << kTileLog;
    std::vector<SliceDesc> h(nslices);
    int64_t t = 0;
    int mx = 0;
    for (int i = 0; i < nslices; ++i) {
        if (!grad_multi_supported(ops[i].Ny)) {
            mrf_set_error("multi-slice gradient: Ny must be 2^a 3^b 5^c, at most 512");
            return MRF_EUNSUPPORTED;
        }
        h[i].voff = voff[i];
        h[i].tile0 = t;
        h[i].Ny = ops[i].Ny;
        h[i].Nx = ops[i].Nx;
        h[i].mask = ops[i].mask;
        MRF_TRY(twiddles_full(ops[i].Ny, &h[i].tw));
        t += (static_cast<int64_t>(ops[i].Nx) * ops[i].L + TC - 1) / TC;
        mx = ops[i].Ny > mx ? ops[i].Ny : mx;
    }
    if (!*table) MRF_CUDA_TRY(cudaMalloc(table, sizeof(SliceDesc) * nslices));
    MRF_CUDA_TRY(cudaMemcpyAsync(*table, h.data(), sizeof(SliceDesc) * nslices,
                                 cudaMemcpyHostToDevice, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    *tiles = t;
    *maxNy = mx;
    return MRF_OK;
}

mrf_status launch_grad_multi(const void* table, int nslices, int64_t tiles, int maxNy,
                             const float2* X, const float2* AHY, int L, float mu, float2* Z,
                             __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st) {
    return launch_multi(static_cast<const SliceDesc*>(table), SliceDesc{}, nslices, tiles, maxNy,
                        X, AHY, L, mu, Z, zq, Kp, err, st);
}
