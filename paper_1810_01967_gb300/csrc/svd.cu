// Temporal subspace compression (§3.3, eqs. CS1, gradupdate, gradcompression; option of §4.3
// and §6).
//
// V_s (L x s) spans the s dominant eigenvectors of the frame Gram matrix
// M = sum_j D_j D_j^H.  Fingerprints are rows, so compression is X -> X conj(V_s) and expansion
// Xc -> Xc V_s^T (the library's batched complex product, cgemm.cu).  The compressed gradient of
// eq. gradcompression runs the y-transforms on s compressed frames; the per-frame line masks do
// not commute with V_s, so between the transforms each k-space row is multiplied by the s x s
// matrix H_ky = V_s^H diag(mask[., ky]) V_s of its phase-encode line (decompress, mask,
// compress in one step; one batched product over the Ny lines).  For power-of-two Ny the
// transforms are the two halves of the fused gradient kernel (forward transform; inverse
// transform with the combine and the BF16 packing), otherwise cuFFT with the combine kernel.
// The step rule of eq. steprule in the compressed domain (§4.3) needs ||A(dXc V_s^T)||^2, which
// is sum over k-space rows of Re(K^H H_ky K) / Ny with K the unscaled y-transform of dXc.  The
// projection is the ordinary one on a dictionary index built from the compressed atoms
// D conj(V_s).
//
// The basis comes from subspace iteration on M in FP64 (M from Hermitian rank-k updates of
// the atoms converted to FP64 with cuBLAS, shifted CholeskyQR3 orthonormalisation) followed by
// Rayleigh-Ritz with a cyclic Jacobi eigensolver on the host: a one-time set-up, outside the
// iterations.  Any orthonormal basis of the same subspace gives identical
// reconstructions (only V_s V_s^H enters), so the Ritz step only selects the dominant s
// directions among the iterated ones.
#include <cublas_v2.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <random>
#include <vector>

#include "mrf_internal.cuh"

mrf_status get_plan(int kind, int Ny, int Nx, int L, cudaStream_t st, cufftHandle* out);
mrf_status fft_exec(cufftHandle h, const float2* in, float2* out, int dir);

struct mrf_svd_op {
    int32_t L = 0, s = 0;
    bool has_op = false;
    mrf_op op = {};
    float2* V = nullptr;    // [L][s]
    float2* VT = nullptr;   // V transposed, [s][L]
    float2* H = nullptr;    // [Ny] blocks of s x s; block ky holds H_ky[b][a] at b + a s
    float2* w2 = nullptr;   // [cap][s] workspace of the gradient
    int64_t cap = 0;
};

namespace {

using cd = std::complex<double>;

mrf_status sfail(mrf_status s, const std::string& m) {
    mrf_set_error(m);
    return s;
}

#define BLAS_TRY(expr)                                                                  \
    do {                                                                                \
        cublasStatus_t b_ = (expr);                                                     \
        if (b_ != CUBLAS_STATUS_SUCCESS)                                                \
            return sfail(MRF_ECUDA, std::string(#expr) + ": cuBLAS status " +           \
                                        std::to_string(static_cast<int>(b_)));          \
    } while (0)

constexpr int kT = 256;

inline unsigned blocks(int64_t work) {
    return static_cast<unsigned>(std::min<int64_t>((work + kT - 1) / kT, 1 << 20));
}

// VT[a][t] = V[t][a]
__global__ void k_transpose(const float2* __restrict__ V, int L, int s, float2* __restrict__ VT) {
    const int64_t n = static_cast<int64_t>(L) * s;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int a = static_cast<int>(i / L), t = static_cast<int>(i - static_cast<int64_t>(a) * L);
        VT[i] = V[static_cast<int64_t>(t) * s + a];
    }
}

// D = A - B
__global__ void k_sub(const float2* __restrict__ A, const float2* __restrict__ B, int64_t n,
                      float2* __restrict__ D) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        D[i] = make_float2(A[i].x - B[i].x, A[i].y - B[i].y);
}

__global__ void k_f2d(const float2* __restrict__ a, int64_t n, double2* __restrict__ b) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[i] = make_double2(a[i].x, a[i].y);
}

// ------------------------------------------------------------------ host linear algebra
// Cholesky A = R^H R of an m x m Hermitian positive definite matrix (column-major, upper
// triangle used); returns false when a pivot is not positive.
bool cholesky_upper(std::vector<cd>& A, int m) {
    for (int j = 0; j < m; ++j) {
        double dj = A[j + j * m].real();
        for (int k = 0; k < j; ++k) dj -= std::norm(A[k + j * m]);
        if (!(dj > 0.0)) return false;
        const double rjj = std::sqrt(dj);
        A[j + j * m] = rjj;
        for (int i = j + 1; i < m; ++i) {
            cd v = A[j + i * m];
            for (int k = 0; k < j; ++k) v -= std::conj(A[k + j * m]) * A[k + i * m];
            A[j + i * m] = v / rjj;
        }
    }
    for (int j = 0; j < m; ++j)
        for (int i = j + 1; i < m; ++i) A[i + j * m] = 0.0;
    return true;
}

// Cyclic Jacobi for an m x m Hermitian matrix (column-major): on return the diagonal of A holds
// the eigenvalues and the columns of U the eigenvectors.  Each rotation first turns the
// pivot's phase into the basis (diag(1, e^{-i phi})), then applies the real symmetric Jacobi
// rotation that annihilates the now real off-diagonal pair.
void jacobi_hermitian(std::vector<cd>& A, std::vector<cd>& U, int m) {
    U.assign(static_cast<size_t>(m) * m, 0.0);
    for (int i = 0; i < m; ++i) U[i + i * m] = 1.0;
    auto at = [&](int r, int c) -> cd& { return A[r + static_cast<size_t>(c) * m]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int c = 0; c < m; ++c)
            for (int r = 0; r < m; ++r)
                (r == c ? diag : off) += std::norm(at(r, c));
        if (off <= 1e-30 * std::max(diag, 1e-300)) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const cd apq = at(p, q);
                const double g = std::abs(apq);
                if (g <= 1e-300) continue;
                const cd ph = apq / g;                        // e^{i phi}
                const double app = at(p, p).real(), aqq = at(q, q).real();
                const double tau = (aqq - app) / (2.0 * g);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                // U2 = diag(1, conj(ph)) [[cs, sn], [-sn, cs]]
                const cd u00 = cs, u01 = sn, u10 = -std::conj(ph) * sn, u11 = std::conj(ph) * cs;
                for (int k = 0; k < m; ++k) {          // A <- A U2
                    const cd x = at(k, p), y = at(k, q);
                    at(k, p) = x * u00 + y * u10;
                    at(k, q) = x * u01 + y * u11;
                }
                for (int k = 0; k < m; ++k) {          // A <- U2^H A
                    const cd x = at(p, k), y = at(q, k);
                    at(p, k) = std::conj(u00) * x + std::conj(u10) * y;
                    at(q, k) = std::conj(u01) * x + std::conj(u11) * y;
                }
                at(p, q) = 0.0;
                at(q, p) = 0.0;
                at(p, p) = at(p, p).real();
                at(q, q) = at(q, q).real();
                for (int k = 0; k < m; ++k) {          // U <- U U2
                    const cd x = U[k + static_cast<size_t>(p) * m], y = U[k + static_cast<size_t>(q) * m];
                    U[k + static_cast<size_t>(p) * m] = x * u00 + y * u10;
                    U[k + static_cast<size_t>(q) * m] = x * u01 + y * u11;
                }
            }
    }
}

// CholQR: Q <- Q R^{-1} with Q^H Q + shift I = R^H R (device, column-major L x m, FP64).  With
// `shifted` the diagonal gets the shift of shifted CholeskyQR (11 (L m + m (m + 1)) u ||G||,
// u = 2^-53, ||G|| bounded by its trace), which keeps the factorisation defined when Q is
// numerically rank deficient; two plain passes after it restore orthogonality.
mrf_status cholqr(cublasHandle_t h, cuDoubleComplex* Q, int L, int m, cuDoubleComplex* G,
                  cudaStream_t st, bool shifted = false) {
    const double one = 1.0, zero = 0.0;
    BLAS_TRY(cublasZherk(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_C, m, L, &one, Q, L, &zero, G, m));
    std::vector<cd> hg(static_cast<size_t>(m) * m);
    MRF_CUDA_TRY(cudaMemcpyAsync(hg.data(), G, hg.size() * sizeof(cd), cudaMemcpyDeviceToHost, st));
    MRF_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < m; ++j)             // fill the lower triangle (unused by the factorisation)
        for (int i = j + 1; i < m; ++i) hg[i + j * m] = std::conj(hg[j + i * m]);
    if (shifted) {
        double tr = 0.0;
        for (int j = 0; j < m; ++j) tr += hg[j + j * m].real();
        const double sh = 11.0 * (static_cast<double>(L) * m + static_cast<double>(m) * (m + 1)) *
                          std::ldexp(1.0, -53) * tr;
        for (int j = 0; j < m; ++j) hg[j + j * m] += sh;
    }
    if (!cholesky_upper(hg, m)) return sfail(MRF_EINTERNAL, "subspace iteration lost rank");
    MRF_CUDA_TRY(cudaMemcpyAsync(G, hg.data(), hg.size() * sizeof(cd), cudaMemcpyHostToDevice, st));
    const cuDoubleComplex alpha = make_cuDoubleComplex(1.0, 0.0);
    BLAS_TRY(cublasZtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                         CUBLAS_DIAG_NON_UNIT, L, m, &alpha, G, m, Q, L));
    return MRF_OK;
}

mrf_status ensure_w2(mrf_svd_op* so, int64_t n) {
    if (n <= so->cap) return MRF_OK;
    if (so->w2) cudaFree(so->w2);
    so->w2 = nullptr;
    so->cap = 0;
    if (cudaMalloc(&so->w2, sizeof(float2) * n * so->s) != cudaSuccess) {
        cudaGetLastError();
        return sfail(MRF_ENOMEM, "svd workspace allocation failed");
    }
    so->cap = n;
    return MRF_OK;
}

// Xc = X conj(V) for rows of length L -> s.
mrf_status compress_rows(const mrf_svd_op* so, const float2* X, int64_t n, float2* Xc,
                         cudaStream_t st) {
    return launch_cgemm(X, so->L, 0, so->V, so->s, 0, true, Xc, so->s, 0, static_cast<int>(n),
                        so->L, so->s, 1, nullptr, 0, 0, st);
}

// X = Xc V^T for rows of length s -> L.
mrf_status expand_rows(const mrf_svd_op* so, const float2* Xc, int64_t n, float2* X,
                       cudaStream_t st) {
    return launch_cgemm(Xc, so->s, 0, so->VT, so->L, 0, false, X, so->L, 0, static_cast<int>(n),
                        so->s, so->L, 1, nullptr, 0, 0, st);
}

// K (unscaled y-transform, natural order) of the compressed image Xc [Ny][Nx][s].
mrf_status yfft_c(mrf_svd_op* so, const float2* Xc, float2* K, cudaStream_t st) {
    const mrf_op& op = so->op;
    if (grad_fused_supported(op.Ny)) return launch_yfft_fwd(Xc, op.Ny, op.Nx, so->s, K, st);
    cufftHandle hy;
    MRF_TRY(get_plan(0, op.Ny, op.Nx, so->s, st, &hy));
    return fft_exec(hy, Xc, K, CUFFT_FORWARD);
}

// W2 = H_ky applied to every k-space row of line ky: W2[ky][kx][b] = sum_a H_ky[b][a] W[ky][kx][a].
mrf_status apply_h(mrf_svd_op* so, const float2* W, float2* W2, cudaStream_t st) {
    const mrf_op& op = so->op;
    const int s = so->s;
    return launch_cgemm(W, s, static_cast<int64_t>(op.Nx) * s, so->H, s,
                        static_cast<int64_t>(s) * s, false, W2, s,
                        static_cast<int64_t>(op.Nx) * s, op.Nx, s, s, op.Ny, nullptr, 0, 0, st);
}

// Zc = Xc - mu (compress(A^H A expand(Xc)) - AHYc) into D->zbuf (and the BF16 operand).
mrf_status gradient_c(mrf_dict* D, mrf_svd_op* so, const float2* AHYc, const float2* Xc,
                      float mu, bool want_zq, cudaStream_t st) {
    const mrf_op& op = so->op;
    const int s = so->s;
    const int64_t n = static_cast<int64_t>(op.Ny) * op.Nx;
    MRF_TRY(ensure_w2(so, n));
    ProfScope ps0(0, 3, st);
    MRF_TRY(yfft_c(so, Xc, D->wbuf, st));
    MRF_TRY(apply_h(so, D->wbuf, so->w2, st));
    __nv_bfloat16* zq = want_zq ? D->zq : nullptr;
    if (grad_fused_supported(op.Ny))
        return launch_yfft_inv_combine(so->w2, Xc, AHYc, op.Ny, op.Nx, s, mu, D->zbuf, zq, D->Kp,
                                       D->err, st);
    cufftHandle hy;
    MRF_TRY(get_plan(0, op.Ny, op.Nx, s, st, &hy));
    MRF_TRY(fft_exec(hy, so->w2, so->w2, CUFFT_INVERSE));
    return launch_grad_combine(Xc, so->w2, AHYc, D->zbuf, n, s, mu,
                               1.0f / static_cast<float>(op.Ny), zq, D->Kp, D->err, st);
}

// *out += ||A(expand(Dc))||^2 = sum of Re(K^H H_ky K) / Ny over the k-space rows, K the
// unscaled y-transform of Dc; uses D->zbuf and so->w2 as workspace (Dc may be D->wbuf).
mrf_status normal_quad(mrf_dict* D, mrf_svd_op* so, const float2* Dc, double* out,
                       cudaStream_t st) {
    const int64_t cnt = static_cast<int64_t>(so->op.Ny) * so->op.Nx * so->s;
    MRF_TRY(ensure_w2(so, static_cast<int64_t>(so->op.Ny) * so->op.Nx));
    MRF_TRY(yfft_c(so, Dc, D->zbuf, st));
    MRF_TRY(apply_h(so, D->zbuf, so->w2, st));
    return launch_cdot_re(D->zbuf, so->w2, cnt, out, st);
}

double read_dev(const double* p, cudaStream_t st, mrf_status* s) {
    double v = 0.0;
    if (cudaMemcpyAsync(&v, p, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        *s = sfail(MRF_ECUDA, "reading a device reduction failed");
    return v;
}

}  // namespace

extern "C" {

mrf_status mrf_svd_basis(const mrf_dict* D, int32_t s, void* V_out, double* eig_out,
                         void* stream) {
    if (!D || !V_out) return sfail(MRF_EINVAL, "dict and V_out are required");
    const int L = D->L;
    if (s < 1 || s > L) return sfail(MRF_EINVAL, "need 1 <= s <= L");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int m = std::min(L, s + std::max(10, s / 5));   // oversampled block
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return sfail(MRF_ECUDA, "cublasCreate failed");
    float2* Mf = nullptr;
    double2 *M = nullptr, *Q = nullptr, *Y = nullptr, *G = nullptr;
    auto cleanup = [&]() {
        cublasDestroy(h);
        void* ptrs[] = {Mf, M, Q, Y, G};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    auto run = [&]() -> mrf_status {
        BLAS_TRY(cublasSetStream(h, st));
        const size_t LL = static_cast<size_t>(L) * L;
        if (cudaMalloc(&M, LL * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&Q, static_cast<size_t>(L) * m * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&Y, static_cast<size_t>(L) * m * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&G, static_cast<size_t>(m) * m * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return sfail(MRF_ENOMEM, "svd basis allocation failed");
        }
        // M (column-major, upper triangle) = A_cm A_cm^H in FP64, A_cm = atoms as an L x d
        // matrix: M[t][t'] = sum_j D_j[t] conj(D_j[t']); chunks of atoms converted to FP64
        // (an FP32 Gram matrix would leave the small eigenvalues below its rounding noise)
        const int64_t chunk = std::max<int64_t>(1, (int64_t{1} << 26) / L);
        double2* Ad = reinterpret_cast<double2*>(Mf);
        Mf = nullptr;
        if (cudaMalloc(&Ad, sizeof(double2) * chunk * L) != cudaSuccess) {
            cudaGetLastError();
            return sfail(MRF_ENOMEM, "svd basis allocation failed");
        }
        Mf = reinterpret_cast<float2*>(Ad);       // freed by the cleanup
        for (int64_t j0 = 0; j0 < D->d; j0 += chunk) {
            const int64_t nj = std::min(chunk, D->d - j0);
            k_f2d<<<blocks(nj * L), kT, 0, st>>>(D->atoms + j0 * L, nj * L, Ad);
            MRF_CUDA_TRY(cudaGetLastError());
            const double one = 1.0, beta = (j0 == 0) ? 0.0 : 1.0;
            BLAS_TRY(cublasZherk(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, L, static_cast<int>(nj),
                                 &one, reinterpret_cast<const cuDoubleComplex*>(Ad), L, &beta,
                                 reinterpret_cast<cuDoubleComplex*>(M), L));
        }
        // seeded start block
        std::vector<cd> hq(static_cast<size_t>(L) * m);
        std::mt19937_64 rng(0x5eedULL + static_cast<uint64_t>(L) * 131 + s);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (auto& v : hq) v = cd(nd(rng), nd(rng));
        MRF_CUDA_TRY(cudaMemcpyAsync(Q, hq.data(), hq.size() * sizeof(cd), cudaMemcpyHostToDevice, st));
        auto* Qz = reinterpret_cast<cuDoubleComplex*>(Q);
        auto* Yz = reinterpret_cast<cuDoubleComplex*>(Y);
        auto* Mz = reinterpret_cast<cuDoubleComplex*>(M);
        auto* Gz = reinterpret_cast<cuDoubleComplex*>(G);
        auto orthonormalise = [&]() -> mrf_status {     // shifted CholeskyQR3
            MRF_TRY(cholqr(h, Qz, L, m, Gz, st, true));
            MRF_TRY(cholqr(h, Qz, L, m, Gz, st));
            return cholqr(h, Qz, L, m, Gz, st);
        };
        MRF_TRY(orthonormalise());
        const cuDoubleComplex z1 = make_cuDoubleComplex(1.0, 0.0), z0 = make_cuDoubleComplex(0.0, 0.0);
        const int iters = (m == L) ? 0 : 40;      // the whole space needs no iteration
        for (int it = 0; it < iters; ++it) {
            BLAS_TRY(cublasZhemm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, L, m, &z1, Mz, L,
                                 Qz, L, &z0, Yz, L));
            std::swap(Qz, Yz);
            MRF_TRY(orthonormalise());
        }
        // Rayleigh-Ritz: T = Q^H M Q (m x m), eigenvectors W, V_s = Q W[:, top s]
        BLAS_TRY(cublasZhemm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, L, m, &z1, Mz, L, Qz, L,
                             &z0, Yz, L));
        BLAS_TRY(cublasZgemm(h, CUBLAS_OP_C, CUBLAS_OP_N, m, m, L, &z1, Qz, L, Yz, L, &z0, Gz, m));
        std::vector<cd> T(static_cast<size_t>(m) * m), W;
        MRF_CUDA_TRY(cudaMemcpyAsync(T.data(), Gz, T.size() * sizeof(cd), cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaMemcpyAsync(hq.data(), Qz, hq.size() * sizeof(cd), cudaMemcpyDeviceToHost, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int j = 0; j < m; ++j)                  // exact Hermitian symmetry
            for (int i = j + 1; i < m; ++i) {
                const cd a = 0.5 * (T[i + j * m] + std::conj(T[j + i * m]));
                T[i + j * m] = a;
                T[j + i * m] = std::conj(a);
            }
        jacobi_hermitian(T, W, m);
        std::vector<int> ord(m);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int a, int b) {
            return T[a + a * m].real() > T[b + b * m].real();
        });
        // V[t][k] = sum_i Q[t][i] W[i][ord[k]], phase: largest-magnitude entry real positive
        std::vector<float2> hv(static_cast<size_t>(L) * s);
        for (int k = 0; k < s; ++k) {
            const int c = ord[k];
            std::vector<cd> col(L, 0.0);
            for (int i = 0; i < m; ++i) {
                const cd w = W[i + static_cast<size_t>(c) * m];
                for (int t = 0; t < L; ++t) col[t] += hq[t + static_cast<size_t>(i) * L] * w;
            }
            int big = 0;
            for (int t = 1; t < L; ++t)
                if (std::abs(col[t]) > std::abs(col[big])) big = t;
            const cd ph = std::abs(col[big]) > 0 ? std::conj(col[big]) / std::abs(col[big]) : cd(1.0);
            double nrm = 0.0;
            for (int t = 0; t < L; ++t) nrm += std::norm(col[t]);
            nrm = std::sqrt(nrm);
            for (int t = 0; t < L; ++t) {
                const cd v = col[t] * ph / nrm;
                hv[static_cast<size_t>(t) * s + k] = make_float2(static_cast<float>(v.real()),
                                                                 static_cast<float>(v.imag()));
            }
            if (eig_out) eig_out[k] = T[c + static_cast<size_t>(c) * m].real();
        }
        MRF_CUDA_TRY(cudaMemcpyAsync(V_out, hv.data(), hv.size() * sizeof(float2),
                                     cudaMemcpyDefault, st));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        return MRF_OK;
    };
    const mrf_status r = run();
    cleanup();
    return r;
}

void mrf_svd_op_free(mrf_svd_op* so) {
    if (!so) return;
    void* ptrs[] = {so->V, so->VT, so->H, so->w2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete so;
}

mrf_status mrf_svd_op_create(const mrf_op* op, const void* V, int32_t L, int32_t s,
                             mrf_svd_op** out, void* stream) {
    if (!out || !V) return sfail(MRF_EINVAL, "V and out are required");
    *out = nullptr;
    if (op) {
        MRF_TRY(check_op_public(op));
        if (op->L != L) return sfail(MRF_EINVAL, "op->L differs from L");
        if (op->Ny > 65535) return sfail(MRF_EINVAL, "Ny above 65535 phase-encode lines");
    }
    if (L < 1 || s < 1 || s > L) return sfail(MRF_EINVAL, "need 1 <= s <= L");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mrf_svd_op* so = new mrf_svd_op();
    so->L = L;
    so->s = s;
    auto bail = [&](mrf_status e, const std::string& m) {
        mrf_svd_op_free(so);
        return sfail(e, m);
    };
    const size_t Ls = static_cast<size_t>(L) * s;
    if (cudaMalloc(&so->V, Ls * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&so->VT, Ls * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return bail(MRF_ENOMEM, "svd op allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(so->V, V, Ls * sizeof(float2), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return bail(MRF_ECUDA, std::string("copy V: ") + cudaGetErrorString(e));
    k_transpose<<<blocks(static_cast<int64_t>(Ls)), kT, 0, st>>>(so->V, L, s, so->VT);
    if (op) {
        so->has_op = true;
        so->op = *op;
        const int Ny = op->Ny;
        if (cudaMalloc(&so->H, sizeof(float2) * Ny * s * s) != cudaSuccess) {
            cudaGetLastError();
            return bail(MRF_ENOMEM, "svd op allocation failed");
        }
        // block ky, element (a, b) at a s + b: sum_t V[t][a] mask[t][ky] conj(V[t][b]) =
        // H_ky[b][a] (row b of H_ky is what line ky's compressed row a contributes to)
        mrf_status r = launch_cgemm(so->VT, L, 0, so->V, s, 0, true, so->H, s,
                                    static_cast<int64_t>(s) * s, s, L, s, Ny, op->mask, Ny, 1, st);
        if (r != MRF_OK) {
            mrf_svd_op_free(so);
            return r;
        }
    }
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(MRF_ECUDA, std::string("svd op: ") + cudaGetErrorString(e));
    *out = so;
    return MRF_OK;
}

mrf_status mrf_svd_compress(const mrf_svd_op* so, const void* X, int64_t n, void* Xc,
                            void* stream) {
    if (!so || n < 0 || (n > 0 && (!X || !Xc))) return sfail(MRF_EINVAL, "bad compress arguments");
    if (n > INT32_MAX) return sfail(MRF_EINVAL, "too many rows");
    return compress_rows(so, static_cast<const float2*>(X), n, static_cast<float2*>(Xc),
                         reinterpret_cast<cudaStream_t>(stream));
}

mrf_status mrf_svd_expand(const mrf_svd_op* so, const void* Xc, int64_t n, void* X,
                          void* stream) {
    if (!so || n < 0 || (n > 0 && (!X || !Xc))) return sfail(MRF_EINVAL, "bad expand arguments");
    if (n > INT32_MAX) return sfail(MRF_EINVAL, "too many rows");
    return expand_rows(so, static_cast<const float2*>(Xc), n, static_cast<float2*>(X),
                       reinterpret_cast<cudaStream_t>(stream));
}

mrf_status mrf_svd_gradient(mrf_dict* Dc, mrf_svd_op* so, const void* AHYc, const void* Xc,
                            float mu, void* Zc, void* stream) {
    if (!Dc || !so || !AHYc || !Xc || !Zc) return sfail(MRF_EINVAL, "missing argument");
    if (!so->has_op) return sfail(MRF_EINVAL, "the svd op was created without a sampling op");
    if (Dc->L != so->s) return sfail(MRF_EINVAL, "dictionary length differs from s");
    if (!std::isfinite(mu)) return sfail(MRF_EINVAL, "mu must be finite");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = static_cast<int64_t>(so->op.Ny) * so->op.Nx;
    MRF_TRY(dict_ensure_scratch(Dc, n));
    MRF_TRY(gradient_c(Dc, so, static_cast<const float2*>(AHYc), static_cast<const float2*>(Xc),
                       mu, false, st));
    MRF_CUDA_TRY(cudaMemcpyAsync(Zc, Dc->zbuf, sizeof(float2) * n * so->s,
                                 cudaMemcpyDeviceToDevice, st));
    return MRF_OK;
}

mrf_status mrf_svd_ipg_step(mrf_dict* Dc, mrf_svd_op* so, const void* AHYc, void* Xc, float mu,
                            const mrf_proj_opts* opts, int32_t* idx_io, void* rho_out,
                            void* stream) {
    if (!Dc || !so || !AHYc || !Xc || !idx_io) return sfail(MRF_EINVAL, "missing argument");
    if (!so->has_op) return sfail(MRF_EINVAL, "the svd op was created without a sampling op");
    if (Dc->L != so->s) return sfail(MRF_EINVAL, "dictionary length differs from s");
    if (!std::isfinite(mu)) return sfail(MRF_EINVAL, "mu must be finite");
    mrf_proj_opts o;
    if (opts) o = *opts; else mrf_default_proj_opts(&o);
    MRF_TRY(check_proj_public(Dc, &o));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = static_cast<int64_t>(so->op.Ny) * so->op.Nx;
    MRF_TRY(dict_ensure_scratch(Dc, n));
    const bool zq = (o.mode == MRF_PROJ_BF16);
    MRF_TRY(gradient_c(Dc, so, static_cast<const float2*>(AHYc), static_cast<const float2*>(Xc),
                       mu, zq, st));
    return project_core(Dc, Dc->zbuf, n, &o, idx_io, idx_io, static_cast<float2*>(rho_out),
                        static_cast<float2*>(Xc), zq, st);
}

mrf_status mrf_svd_reconstruct(mrf_dict* Dc, mrf_svd_op* so, const void* Y,
                               const mrf_recon_opts* ropts, void* Xc_out, void* X_out,
                               int32_t* idx_out, void* rho_out, float* params_out,
                               void* stream) {
    if (!Dc || !so || !Y || !Xc_out || !idx_out) return sfail(MRF_EINVAL, "missing argument");
    if (!so->has_op) return sfail(MRF_EINVAL, "the svd op was created without a sampling op");
    if (Dc->L != so->s) return sfail(MRF_EINVAL, "dictionary length differs from s");
    mrf_recon_opts r;
    if (ropts) r = *ropts; else mrf_default_recon_opts(&r);
    if (r.iters < 0 || !(r.mu > 0.f) || (r.adaptive && !(r.zeta > 1.f)) || r.max_shrink < 0)
        return sfail(MRF_EINVAL, "bad reconstruction options");
    if (r.tol > 0.f || r.resume)
        return sfail(MRF_EUNSUPPORTED, "tol and resume are not available for compressed iterations");
    MRF_TRY(check_proj_public(Dc, &r.proj));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = static_cast<int64_t>(so->op.Ny) * so->op.Nx;
    const int64_t cnt = n * so->s;
    MRF_TRY(dict_ensure_scratch(Dc, n));
    float2* AHY = nullptr;
    float2* AHYc = nullptr;
    float2* Xp = nullptr;
    float2* rho_tmp = nullptr;
    double* red = nullptr;
    auto run = [&]() -> mrf_status {
        if (cudaMalloc(&AHY, sizeof(float2) * n * so->L) != cudaSuccess ||
            cudaMalloc(&AHYc, sizeof(float2) * cnt) != cudaSuccess ||
            cudaMalloc(&red, sizeof(double) * 4) != cudaSuccess ||
            ((r.adaptive || r.kappa) && cudaMalloc(&Xp, sizeof(float2) * cnt) != cudaSuccess) ||
            (!rho_out && cudaMalloc(&rho_tmp, sizeof(float2) * n) != cudaSuccess)) {
            cudaGetLastError();
            return sfail(MRF_ENOMEM, "svd reconstruction allocation failed");
        }
        float2* Xc = static_cast<float2*>(Xc_out);
        float2* rho = rho_out ? static_cast<float2*>(rho_out) : rho_tmp;
        MRF_TRY(mrf_adjoint(&so->op, Y, AHY, stream));
        MRF_TRY(compress_rows(so, AHY, n, AHYc, st));
        MRF_CUDA_TRY(cudaMemsetAsync(Xc, 0, sizeof(float2) * cnt, st));
        MRF_CUDA_TRY(cudaMemsetAsync(idx_out, 0, sizeof(int32_t) * n, st));
        const bool zq = (r.proj.mode == MRF_PROJ_BF16);
        float mu0 = r.mu;
        mrf_status rs = MRF_OK;
        for (int32_t k = 0; k < r.iters; ++k) {
            float mu_k = mu0;
            int shrinks_k = 0;
            if (r.adaptive || r.kappa)
                MRF_CUDA_TRY(cudaMemcpyAsync(Xp, Xc, sizeof(float2) * cnt,
                                             cudaMemcpyDeviceToDevice, st));
            for (int shrink = 0;; ++shrink) {
                shrinks_k = shrink;
                MRF_TRY(gradient_c(Dc, so, AHYc, r.adaptive ? Xp : Xc, mu_k, zq, st));
                MRF_TRY(project_core(Dc, Dc->zbuf, n, &r.proj, idx_out, idx_out, rho, Xc, zq, st));
                if (!r.adaptive) break;
                // compressed step rule (§4.3): mu_k < ||dXc||^2 / ||A(expand(dXc))||^2
                MRF_CUDA_TRY(cudaMemsetAsync(red, 0, sizeof(double) * 2, st));
                k_sub<<<blocks(cnt), kT, 0, st>>>(Xc, Xp, cnt, Dc->wbuf);
                MRF_CUDA_TRY(cudaGetLastError());
                MRF_TRY(launch_sqnorm(Dc->wbuf, cnt, red, st));
                MRF_TRY(normal_quad(Dc, so, Dc->wbuf, red + 1, st));
                const double num = read_dev(red, st, &rs);
                const double den = read_dev(red + 1, st, &rs) / so->op.Ny;
                if (rs != MRF_OK) return rs;
                if (den <= 0.0 || static_cast<double>(mu_k) < num / den || shrink >= r.max_shrink)
                    break;
                mu_k /= r.zeta;
            }
            if (r.mu_history) r.mu_history[k] = mu_k;
            if (r.shrink_history) r.shrink_history[k] = shrinks_k;
            if (r.kappa && k == 0) {
                // kappa = ||Y|| / ||A(X^1)||, X^1 and rho scaled, mu scaled alike
                MRF_CUDA_TRY(cudaMemsetAsync(red + 2, 0, sizeof(double) * 2, st));
                MRF_TRY(launch_sqnorm(static_cast<const float2*>(Y), n * so->L, red + 2, st));
                MRF_TRY(normal_quad(Dc, so, Xc, red + 3, st));
                const double yy = read_dev(red + 2, st, &rs);
                const double ax = read_dev(red + 3, st, &rs) / so->op.Ny;
                if (rs != MRF_OK) return rs;
                if (ax > 0.0) {
                    const float kap = static_cast<float>(std::sqrt(yy / ax));
                    MRF_TRY(launch_scale(Xc, cnt, kap, st));
                    MRF_TRY(launch_scale(rho, n, kap, st));
                    mu0 *= kap;
                }
            }
        }
        if (X_out) MRF_TRY(expand_rows(so, Xc, n, static_cast<float2*>(X_out), st));
        if (params_out && Dc->P > 0) MRF_TRY(mrf_lut(Dc, idx_out, n, params_out, stream));
        MRF_CUDA_TRY(cudaStreamSynchronize(st));
        return MRF_OK;
    };
    const mrf_status rr = run();
    void* ptrs[] = {AHY, AHYc, Xp, rho_tmp, red};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (rr != MRF_OK) return rr;
    return mrf_dict_check(Dc, stream);
}

}  // extern "C"
