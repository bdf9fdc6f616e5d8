// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "../../include/mrf.h"

// Device error word bits (OR-ed by kernels, read by mrf_dict_check / stats calls).
enum : uint32_t {
    MRF_DERR_NONFINITE = 1u << 0,
    MRF_DERR_TIMEOUT = 1u << 1,
    MRF_DERR_BOUNDS = 1u << 2,
};

// Device counters (indices into mrf_dict::counters).
enum {
    CNT_ZERO = 0,
    CNT_TIE_RESCORED = 1,
    CNT_TIE_OVERFLOW = 2,
    CNT_UNCERT = 3,
    CNT_FALLBACK = 4,
    CNT_DIST = 5,
    CNT_N = 8
};

struct CoverTreeDev;   // flattened cover tree (covertree.cu)
struct TreeTC;         // block balls and depth-first operands of the tensor-core tree search

struct mrf_dict {
    int64_t d = 0;
    int32_t L = 0, P = 0;
    int device = 0;
    std::vector<int32_t> grid_shape;
    float2* atoms = nullptr;        // [d][L] complex64 as given
    float* inv_norm2 = nullptr;     // [d] 1 / ||D_j||^2 (from an FP64 sum)
    float* inv_norm = nullptr;      // [d] 1 / ||D_j|| (same sum; operand normalisation)
    double* norm2 = nullptr;        // [d] ||D_j||^2 in FP64
    float* params = nullptr;        // [d][P]
    // BF16 tensor-core operand of the normalised atoms D_j / ||D_j||: blocks of 128 atoms, 256
    // rows each (128 real-part rows, then 128 imaginary-part rows), row length Kp = 2L rounded
    // up to 16, interleaved (re, im).
    __nv_bfloat16* bop = nullptr;
    int64_t nblk = 0;
    int32_t Kp = 0;
    // FP8 E4M3 operand: the same blocks and rows of normalised atoms, row length Kp8 = 2L
    // rounded up to 32, all scaled by one power of two 1 / g8
    uint8_t* fop = nullptr;
    float g8 = 1.f;
    int32_t Kp8 = 0;
    // Split-BF16 operand of the exact tensor-core form: the same blocks and rows, each row three
    // segments of Kp elements, [hi | lo | hi] of the normalised atom (hi = bf16(d), lo =
    // bf16(d - hi)), against query rows [lo | hi | hi], so one MMA chain over Kp3 = 3 Kp sums
    // z_lo d_hi + z_hi d_lo (the small products first) + z_hi d_hi.  x3_al / x3_ae: the largest
    // ||lo|| and ||D_j/||D_j|| - hi - lo|| over the atoms (FP64, rounded up).
    __nv_bfloat16* bop3 = nullptr;
    int32_t Kp3 = 0;
    float x3_al = 0.f, x3_ae = 0.f;
    // scratch (grown on demand, or reserved up front)
    int64_t cap_n = 0;
    __nv_bfloat16* zq = nullptr;    // [cap_n][Kp]
    uint8_t* zq8 = nullptr;         // [cap_n][Kp8] FP8 queries (with the FP8 operand)
    __nv_bfloat16* zq3 = nullptr;   // [cap_n][Kp3] split-BF16 queries (with the split operand)
    float* zmarg = nullptr;         // [cap_n] per-voxel certification margin of the split form
    float* qs8 = nullptr;           // [cap_n] 1 / s of each FP8 query row
    float2* zbuf = nullptr;         // [cap_n][L] gradient-step output Z
    float2* wbuf = nullptr;         // [cap_n][L] FFT workspace
    float2* xprev = nullptr;        // [cap_n][L] previous iterate (step rule)
    int32_t* vlist = nullptr;       // [cap_n] compacted voxel list (fallback)
    int32_t* nlist = nullptr;       // [2] lengths of vlist and vlist2
    int32_t* vlist2 = nullptr;      // [cap_n] second-level list (certification of a fallback)
    size_t part_bytes = 0;
    void* part = nullptr;           // partial top-k candidates (scores then indices)
    uint32_t* err = nullptr;        // device error word
    unsigned long long* counters = nullptr;   // [CNT_N]
    double* red = nullptr;          // [8] reductions (norms for the step rule / kappa)
    CoverTreeDev* tree = nullptr;
    TreeTC* ttc = nullptr;           // tensor-core tree search (treetc.cu)
    mrf_mlp* mlp = nullptr;          // attached learned proposal (not owned)
    // phase alignment (real positive cone on complex data): atoms stored as D_j e^{-i alpha_j}
    bool aligned = false;
    float2* v1 = nullptr;            // [L] dominant eigenvector of sum_j D_j D_j^H
    float2* ealign = nullptr;        // [d] e^{i alpha_j}
    float2* qph = nullptr;           // [cap_n] e^{i beta_v} of the last aligned queries
    int num_sms = 148;
    // no host synchronisation inside a projection (set while a batch iteration is captured into
    // a graph): the cover-tree and learned fallbacks take their voxel count from the device
    bool sync_free = false;
    mrf_tune tune = {};              // requested geometry (0 = default) and last launches
};

// thread-local error text
void mrf_set_error(const std::string& msg);

// Epoch of the device buffers a captured iteration may reference: bumped whenever such a buffer
// (dictionary scratch, candidate partials, learned-proposal and tree workspaces) is freed to be
// reallocated.  A CUDA graph captured at one epoch is replayed only at that epoch.
uint64_t scratch_epoch();
void scratch_epoch_bump();

#define MRF_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            mrf_set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));          \
            return MRF_ECUDA;                                                           \
        }                                                                               \
    } while (0)

#define MRF_TRY(expr)                                                                   \
    do {                                                                                \
        mrf_status s_ = (expr);                                                         \
        if (s_ != MRF_OK) return s_;                                                    \
    } while (0)

// Records an event pair around a stage on `st` while the stage profiler is enabled (abi.cu).
struct ProfScope {
    ProfScope(int stage, int launches, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
    bool on;
    cudaStream_t st;
    int stage_ = 0, launches_ = 0;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// ----- host helpers shared across translation units (abi.cu)
mrf_status project_core(mrf_dict* D, const float2* Z, int64_t n, const mrf_proj_opts* o,
                        const int32_t* warm, int32_t* idx_out, float2* rho_out, float2* X_out,
                        bool zq_ready, cudaStream_t st);
mrf_status gradient_to(const mrf_op* op, const float2* AHY, const float2* X, float mu, float2* Z,
                       float2* W, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st);
mrf_status dict_ensure_scratch(mrf_dict* D, int64_t n);
bool profiler_suspend();
void profiler_resume(bool was);
mrf_status check_op_public(const mrf_op* op);
mrf_status check_proj_public(const mrf_dict* D, const mrf_proj_opts* o);

// ----- kernels (launch wrappers); all asynchronous on `st`
// prep.cu
mrf_status launch_atom_norms(mrf_dict* D, cudaStream_t st);
mrf_status launch_pack_bop(mrf_dict* D, cudaStream_t st);
mrf_status launch_pack_queries(const float2* Z, int64_t n, int L, int Kp, __nv_bfloat16* zq,
                               cudaStream_t st);
mrf_status launch_atoms_absmax(const mrf_dict* D, unsigned int* m_bits, cudaStream_t st);
mrf_status launch_pack_fop(mrf_dict* D, float s, cudaStream_t st);
mrf_status launch_pack_queries_fp8(const float2* Z, const int32_t* vlist, int64_t n, int L,
                                   int Kp8, uint8_t* zq8, float* qs, cudaStream_t st);
mrf_status launch_pack_gather(const float2* Z, const int32_t* vlist, int64_t n, int L, int Kp,
                              __nv_bfloat16* zq, cudaStream_t st,
                              const int32_t* count = nullptr);
mrf_status launch_mask_ky(float2* W, const uint8_t* mask, int Ny, int Nx, int L,
                          cudaStream_t st);
// split-BF16 operand of the atoms (D->bop3) and the split statistics D->x3_al / D->x3_ae
// (synchronises `st` to read them)
mrf_status launch_pack_bop3(mrf_dict* D, cudaStream_t st);
// split-BF16 query rows [lo | hi | hi] and, per voxel, the rigorous error bound of the split
// form's correlations (normalised-correlation units) plus `extra` (the rescore's bound)
mrf_status launch_pack_queries_x3(const float2* Z, int64_t n, const mrf_dict* D, float extra,
                                  __nv_bfloat16* zq3, float* margin, cudaStream_t st);
mrf_status launch_fill(float* out, int64_t n, float v, cudaStream_t st);
// split-BF16 operand of the atoms sel[0 .. nsel) in nblk_out blocks of 128 (row length 3 Kp;
// sel[p] < 0 leaves slot p empty), with their split statistics (host floats); the query split
// with explicit statistics and Kp: with vlist, row i holds voxel vlist[i] and its margin goes
// to margin[vlist[i]]; znorm (optional) receives the FP32 norm of each row's voxel
mrf_status launch_pack_sel3(const mrf_dict* D, const int32_t* sel, int64_t nsel, int64_t nblk_out,
                            __nv_bfloat16* dst, float* al_out, float* ae_out, cudaStream_t st);
mrf_status launch_pack_queries_x3_with(const float2* Z, int64_t n, int L, int Kp, float Al,
                                       float Ae, float extra, __nv_bfloat16* zq3, float* margin,
                                       cudaStream_t st, const int32_t* vlist = nullptr,
                                       float* znorm = nullptr);
// the BF16 operand with atom perm[p] in slot p (perm of length nblk * 128, -1 = empty)
mrf_status launch_pack_bop_perm(const mrf_dict* D, __nv_bfloat16* dst, const int32_t* perm,
                                cudaStream_t st);
mrf_status launch_grad_combine(const float2* X, const float2* G, const float2* AHY, float2* Z,
                               int64_t n, int L, float mu, float g_scale, __nv_bfloat16* zq,
                               int Kp, uint32_t* err, cudaStream_t st);
mrf_status launch_scale(float2* X, int64_t count, float s, cudaStream_t st);
mrf_status launch_lut(const int32_t* idx, int64_t n, const float* params, int P, int64_t d,
                      float* out, uint32_t* err, cudaStream_t st);
mrf_status launch_sqnorm(const float2* X, int64_t count, double* out, cudaStream_t st);
mrf_status launch_sqdiff(const float2* A, const float2* B, int64_t count, double* out,
                         cudaStream_t st);
mrf_status launch_axpby(float2* Y, const float2* X, int64_t count, float a, float b,
                        cudaStream_t st);
// fp32.cu
mrf_status launch_fp32_topk(const float2* Z, const int32_t* vlist, const int32_t* nlist,
                            int64_t n, const mrf_dict* D, int cone, int K, int S,
                            float* part_s, int32_t* part_i, cudaStream_t st);
int fp32_choose_splits(int64_t n, int64_t d, int num_sms);
// bf16.cu
// count (device, may be NULL): voxels actually present when the rows were listed on the device;
// n is then the capacity the launch is sized for
mrf_status launch_bf16_topk(const __nv_bfloat16* zq, int64_t n, mrf_dict* D, int cone, int K,
                            int S, float* part_s, int32_t* part_i, cudaStream_t st,
                            const int32_t* count = nullptr);
int bf16_choose_splits(const mrf_dict* D, int64_t n);
mrf_status launch_fp8_topk(const uint8_t* zq8, const float* qs, int64_t n, mrf_dict* D, int cone,
                           int K, int S, float* part_s, int32_t* part_i, cudaStream_t st);
mrf_status launch_x3_topk(const __nv_bfloat16* zq3, int64_t n, mrf_dict* D, int cone, int K,
                          int S, float* part_s, int32_t* part_i, cudaStream_t st);
mrf_status launch_bf16_topk_list(const __nv_bfloat16* zq, int64_t n, mrf_dict* D,
                                 const __nv_bfloat16* op, int Kp, int cone, int K, int group,
                                 int chunk, int sg, bool pair, const int32_t* tfirst,
                                 const int32_t* blist, const int32_t* uoff, const int32_t* perm,
                                 float* part_s, int32_t* part_i, cudaStream_t st);
// covertree.cu
mrf_status ct_build_upload(mrf_dict* D, int metric, double dup_tol);
void ct_free(CoverTreeDev* t);
mrf_status launch_ct_search(const float2* Z, int64_t n, const mrf_dict* D, int cone,
                            const int32_t* warm, float eps, float route, float* part_s,
                            int32_t* part_i, int32_t* fb_list, int32_t* fb_n, cudaStream_t st);
mrf_status ct_info(const mrf_dict* D, mrf_tree_info* info);
mrf_status ct_dfs_order(const mrf_dict* D, std::vector<int32_t>* out);
int ct_metric(const mrf_dict* D);
mrf_status ct_export(const mrf_dict* D, int32_t* first_level, int32_t* parent, int32_t* rep,
                     int32_t* en_atom, int32_t* en_level, float* en_maxdist);
// treetc.cu
struct TtcOut {
    int S = 0;                   // candidate lists per voxel row
    const float* part_s = nullptr;
    const int32_t* part_i = nullptr;   // [S][n][K] atom indices (-1 empty)
    const int32_t* vorder = nullptr;   // [n] voxel of each row
    const int32_t* count = nullptr;    // device int = n (the merge's list length)
    int64_t tiles = 0;
};
mrf_status ttc_build(mrf_dict* D, cudaStream_t st);
void ttc_free(TreeTC* t);
bool ttc_has_split(const mrf_dict* D);
bool ttc_has_bf16(const mrf_dict* D);
mrf_status ttc_search(mrf_dict* D, const float2* Z, int64_t n, int cone, float eps, bool split,
                      int K, float extra, TtcOut* out, cudaStream_t st);
mrf_status ttc_blocks(const mrf_dict* D, int64_t* nblk, float* radius_host, int32_t* perm_host);
// gradfft.cu
bool grad_fused_supported(int Ny);
mrf_status launch_grad_fused(const mrf_op* op, const float2* AHY, const float2* X, float mu,
                             float2* Z, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st);
// any Ny = 2^a 3^b 5^c up to 512 (mixed-radix y-transforms): one slice, or the stacked slices
// of a batch in one launch from a descriptor table (grad_multi_table builds it in *table)
bool grad_multi_supported(int Ny);
mrf_status launch_grad_mixed(const mrf_op* op, const float2* AHY, const float2* X, float mu,
                             float2* Z, __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st);
mrf_status grad_multi_table(const mrf_op* ops, const int64_t* voff, int nslices, void** table,
                            int64_t* tiles, int* maxNy, cudaStream_t st);
mrf_status launch_grad_multi(const void* table, int nslices, int64_t tiles, int maxNy,
                             const float2* X, const float2* AHY, int L, float mu, float2* Z,
                             __nv_bfloat16* zq, int Kp, uint32_t* err, cudaStream_t st);
// the halves of the fused kernel for an image of C columns per x (power-of-two Ny): W = the
// unscaled y-DFT of X; Z = X - mu (F_y^-1 W2 (unscaled, then / Ny) - AHY) (+ BF16 operand)
mrf_status launch_yfft_fwd(const float2* X, int Ny, int Nx, int C, float2* W, cudaStream_t st);
mrf_status launch_yfft_inv_combine(const float2* W2, const float2* X, const float2* AHY, int Ny,
                                   int Nx, int C, float mu, float2* Z, __nv_bfloat16* zq, int Kp,
                                   uint32_t* err, cudaStream_t st);
// cgemm.cu: batched complex FP32 product Out[b][r][j] = sum_k In[b][r][k] m_b(k) op(M[b][k][j])
// (row-major; op = conj when conj_m; m_b(k) = kmask[b * kmask_bs + k * kmask_ld] != 0 when a
// mask is given, else 1)
mrf_status launch_cgemm(const float2* In, int64_t in_ld, int64_t in_bs, const float2* M,
                        int64_t m_ld, int64_t m_bs, bool conj_m, float2* Out, int64_t out_ld,
                        int64_t out_bs, int R, int K, int J, int batches, const uint8_t* kmask,
                        int64_t kmask_ld, int64_t kmask_bs, cudaStream_t st);
// Re sum_i conj(a_i) b_i accumulated in FP64 into *out (added)
mrf_status launch_cdot_re(const float2* a, const float2* b, int64_t count, double* out,
                          cudaStream_t st);
// phase.cu
mrf_status phase_align_dictionary(mrf_dict* D, cudaStream_t st);
mrf_status launch_align_queries(const mrf_dict* D, const float2* Z, int64_t n, float2* Zout,
                                float2* eb, cudaStream_t st);
mrf_status launch_align_post(const mrf_dict* D, int64_t n, const int32_t* idx, const float2* eb,
                             float2* rho, float2* X, cudaStream_t st);
// tcgemm.cu: out/outb [M][N] = gelu(A [M][Kp] Wt^T + bias), BF16 operands (K-major, 16-byte row
// pitch), FP32 accumulation on the tensor cores; N a multiple of 16; either output may be NULL
mrf_status launch_dense_gelu(const __nv_bfloat16* A, int M, int Kp, const __nv_bfloat16* Wt,
                             int N, const float* bias, float* out, __nv_bfloat16* outb,
                             uint32_t* err, cudaStream_t st);
int dense_tile_n(int N);
// the same product with act = 0 (identity) or 1 (GELU); bias may be NULL
mrf_status launch_dense(const __nv_bfloat16* A, int M, int Kp, const __nv_bfloat16* Wt, int N,
                        const float* bias, int act, float* out, __nv_bfloat16* outb,
                        uint32_t* err, cudaStream_t st);
// mlp.cu
void mlp_detach(mrf_mlp* M);
mrf_status learned_candidates(mrf_dict* D, const float2* Z, int64_t n, int cone, float* part_s,
                              int32_t* part_i, cudaStream_t st);
mrf_status learned_flag(mrf_dict* D, const float2* Z, int64_t n, const int32_t* idx, float thr,
                        bool edge, int cone, int32_t* list, int32_t* cnt_list, cudaStream_t st);
// merge.cu
mrf_status launch_merge(const float2* Z, int64_t n, const mrf_dict* D, int cone, int K, int S,
                        const float* part_s, const int32_t* part_i, const int32_t* vlist,
                        const int32_t* nlist, float tie_tol, int certify, float cert_margin,
                        int32_t* idx_out, float2* rho_out, float2* X_out, int32_t* fb_list,
                        int32_t* fb_n, uint32_t* err, unsigned long long* counters,
                        cudaStream_t st, float window = -1.f,    // window < 0: rescore all K
                        const float* vmargin = nullptr);  // per-voxel cert_margin when given
