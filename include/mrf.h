/*
 * mrf.h -- C ABI of the GB300 matched-filtering reconstruction library (libmrf.so).
 *
 * The library solves the per-voxel cone-constrained least-squares problem of MRF
 * reconstruction (arXiv 1810.01967, §3.2, eq. CS) by projected gradient iterations (BLIP,
 * §3.2 eq. blip; CoverBLIP, Algorithm 2): a gradient step Z = X - mu A^H(A X - Y) followed by
 * the matched-filtering projection of every voxel's fingerprint Z_v onto the cone of the
 * dictionary (eqs. exactP / exactPs).
 *
 * Conventions
 *   - complex numbers are interleaved float2 (complex64), row-major, indices 0-based;
 *   - the image X is [n][L] with voxel v = y * Nx + x and the frame t contiguous (row v is the
 *     fingerprint X_v of §3, eq. CS footnote);
 *   - k-space Y is [Ny][Nx][L] (ky, kx, t) in DFT order (DC at index 0), entries of lines that
 *     were not sampled are ignored (treated as zero);
 *   - masks are uint8 [L][Ny]: mask[t][ky] = 1 when phase-encode line ky is in Omega_t;
 *   - the Fourier transform F is the unitary 2-D DFT of each frame, one coil (S = identity);
 *   - "device" pointers are CUDA global memory of the current device, owned by the caller;
 *     the library never frees caller memory.  The library owns only an mrf_dict and its
 *     scratch buffers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.  One mrf_dict must not be used by
 *     two calls in flight at the same time (its scratch buffers are shared).
 *   - Errors: no C++ exception crosses this boundary.  Every call returns an mrf_status; the
 *     message of the last failure on the calling thread is returned by mrf_last_error().
 *     Argument errors are detected on the host before any launch.  Device-side conditions
 *     (non-finite input, an exhausted wait bound) set an error word in the dict that calls
 *     which synchronise (stats != NULL, mrf_reconstruct, mrf_dict_check) report.
 */
#ifndef MRF_H
#define MRF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mrf_status {
    MRF_OK = 0,
    MRF_EINVAL = 1,        /* bad argument (null pointer, size, mode) */
    MRF_ENOMEM = 2,        /* device or host allocation failed */
    MRF_ECUDA = 3,         /* a CUDA runtime / driver / cuFFT call failed */
    MRF_ENONFINITE = 4,    /* NaN or Inf found in an input */
    MRF_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    MRF_EUNSUPPORTED = 6,  /* feature not built for this dictionary / device */
    MRF_EINTERNAL = 7
} mrf_status;

/* How the projection (the nearest-neighbour search of eq. exactP) is computed. */
typedef enum mrf_proj_mode {
    MRF_PROJ_FP32_EXACT = 0,  /* exhaustive, FP32 SIMT correlations; near-ties rescored with
                                 compensated FP32 sums (FP64-class accuracy) */
    MRF_PROJ_BF16 = 1,        /* exhaustive, BF16 tensor cores (tcgen05), top-K rescored
                                 exactly in FP32, near-ties in extended precision */
    MRF_PROJ_FP8 = 2,         /* exhaustive, FP8 e4m3 tensor cores, rescored as BF16 */
    MRF_PROJ_COVERTREE = 3,   /* cover-tree (1+eps)-ANNS, Algorithm 1 (§4.1) */
    MRF_PROJ_LEARNED = 4,     /* MLP proposal + exact neighbourhood rescore + fallback */
    MRF_PROJ_BF16X3 = 5,      /* exact exhaustive projection on the tensor cores: split-BF16
                                 operands (x = hi + lo, three products per pair in one FP32
                                 accumulation), top-K (default 32) rescored exactly, every voxel
                                 certified against its own error bound (see cert_margin) and
                                 the uncertified ones searched in FP32; needs
                                 mrf_index_opts.pack_bf16x3 */
    MRF_PROJ_TREE_TC = 6      /* query-batched cover-tree search on the tensor cores (§4.1
                                 Algorithm 1 and Def. eNN, with the query grouping of §7): the
                                 tree's depth-first order cut into 128-atom blocks with exact
                                 enclosing balls; per voxel the blocks that can hold an atom
                                 closer than r_v / (1 + eps) (r_v: the nearest block centre's
                                 distance, bounded from the split-BF16 centre correlations);
                                 voxels grouped into 128-voxel tiles by nearest centre, each
                                 tile's union of blocks searched on the tensor cores and the
                                 top K rescored exactly.  With `certify` (and the split-BF16
                                 operand) the result is certified as for MRF_PROJ_BF16X3: the
                                 exact nearest atom for eps = 0, a (1 + eps)-approximate one
                                 otherwise; without, the BF16 operand ranks the candidates.
                                 Needs mrf_index_opts.tree_tc and a tree whose metric matches
                                 the cone */
} mrf_proj_mode;

/* The cone of eq. model/conedef.  COMPLEX: X_v = rho D_j, rho complex, j maximises
 * |D_j^H Z_v| / ||D_j||.  REAL_POS: the paper's gamma > 0, j minimises ||Z_v - D_j/||D_j|| ||
 * and gamma = max(Re(D_j^H Z_v) / ||D_j||^2, 0) (eqs. exactP / exactPs). */
typedef enum mrf_cone { MRF_CONE_COMPLEX = 0, MRF_CONE_REAL_POS = 1 } mrf_cone;

typedef struct mrf_dict mrf_dict;   /* opaque; owned by the library */

typedef struct mrf_index_opts {
    int32_t pack_bf16;     /* build the BF16 tensor-core operand (default 1) */
    int32_t pack_fp8;      /* build the FP8 e4m3 operand (default 0) */
    int32_t build_tree;    /* build the cover tree on the host (default 0), §4.1 */
    int32_t tree_cone;     /* metric of the tree: MRF_CONE_COMPLEX = phase-quotient distance
                              min_phi ||x - e^{i phi} y|| (default), MRF_CONE_REAL_POS =
                              Euclidean distance of the unit atoms */
    float   tree_dup_tol;  /* atoms within this distance of an earlier node are represented by
                              it (default 1e-5) */
    int32_t phase_align;   /* §4.3 phase alignment (default 0): atoms are stored rotated so that
                              v1^H D_j is real positive (v1 = dominant eigenvector of
                              sum_j D_j D_j^H); projections with MRF_CONE_REAL_POS rotate each
                              query the same way, project with the real positive density and
                              restore the query's phase, so rho = gamma e^{i(beta_v - alpha_j)}.
                              Densities are always reported relative to the atoms as given. */
    int32_t pack_bf16x3;   /* build the split-BF16 operand of MRF_PROJ_BF16X3 (default 0):
                              3 x the BF16 operand's memory (2.4 GB for 100k atoms at L = 1000) */
    int32_t tree_tc;       /* with build_tree: the block balls of MRF_PROJ_TREE_TC and copies of
                              the BF16 / split-BF16 operands (those packed) in the tree's
                              depth-first order (default 0) */
} mrf_index_opts;

typedef struct mrf_proj_opts {
    int32_t mode;          /* mrf_proj_mode (default MRF_PROJ_FP32_EXACT) */
    int32_t cone;          /* mrf_cone (default MRF_CONE_COMPLEX) */
    int32_t topk;          /* candidates kept per voxel by the exhaustive kernels, 1..32
                              (rounded up to 8, 16 or 32; FP32 at most 16); 0 = mode default
                              (8 for FP32, 16 for BF16, 32 for FP8, whose coarser scores need
                              the longer list to hold the best atom, and 32 for BF16X3, whose
                              flat background voxels have many atoms inside their bound) */
    int32_t certify;       /* BF16/FP8/BF16X3: recompute voxels whose k-th candidate is within
                              cert_margin of the best with the FP32 exact kernel (default 1) */
    float   tie_tol;       /* candidates whose normalised correlation |D_j^H Z_v| /
                              (||D_j|| ||Z_v||) is within this absolute distance of the best
                              are rescored with FP64-class accuracy: compensated FP32
                              sums reduced in FP64 (default 1e-5) */
    float   cert_margin;   /* margin of `certify`, same units; <= 0 selects the rigorous
                              bound of the BF16 correlation error, 2^-7 + 2^-16 (operand
                              rounding) + 2L 2^-24 (FP32 accumulation), or for FP8
                              2 u8 + u8^2 + 2L 2^-13 with u8 = 2^-4 + sqrt(2L) 2^-10 / 224
                              (E4M3 rounding of rows scaled into (224, 448]; 13-bit partial
                              sums assumed); for MRF_PROJ_BF16X3 each voxel's own bound
                              (operand part rigorous from the stored split residuals:
                              ||z_lo|| A_l + ||z_hi + z_lo|| A_e + ||e_z||, with A_l, A_e the
                              largest residual norms of the atoms; accumulation part from a
                              model of one FP32 rounding per MMA instruction, the small
                              products summed first) plus the FP32 rescore's bound
                              (default 0) */
    float   eps;           /* cover tree (1+eps) approximation (default 0) */
    float   fallback_thr;  /* learned proposal: normalised correlation threshold (0.98) */
    float   tree_route;    /* cover tree: a voxel whose candidate list exceeds 64 entries while
                              its best distance to z/||z|| is above this goes to the exhaustive
                              search, where Algorithm 1 cannot prune; so does a warm-started
                              voxel whose warm atom is already farther than this, before the
                              traversal (default 0.9; >= 2 disables routing) */
    int32_t learned_edge;  /* learned proposal: also send a voxel to the exhaustive search when
                              the best atom of its neighbourhood lies on the neighbourhood's
                              edge with grid cells beyond it (a better atom may lie outside);
                              an accepted proposal is then a local maximum of the correlation
                              over its grid neighbours (default 1) */
    int32_t reserved[6];
} mrf_proj_opts;

/* Filled by calls given a non-NULL pointer; such calls synchronise `stream` before return. */
typedef struct mrf_stats {
    int64_t n_voxels;         /* voxels projected */
    int64_t n_zero;           /* zero queries (idx 0, rho 0) */
    int64_t n_tie_rescored;   /* voxels whose leading candidates were rescored with
                                 FP64-class accuracy (compensated FP32, FP64 reduction) */
    int64_t n_tie_overflow;   /* voxels whose k-th candidate was still within tie_tol */
    int64_t n_uncertified;    /* BF16/FP8 voxels sent to the FP32 exact kernel */
    int64_t n_fallback;       /* learned proposal voxels sent to the exhaustive search */
    int64_t n_dist_evals;     /* cover tree: distance evaluations */
    int32_t device_error;     /* raw device error word (0 = none) */
    int32_t reserved;
} mrf_stats;

/* Cartesian single-coil sampling operator A = P_Omega F (§3, eq. forward). */
typedef struct mrf_op {
    int32_t Ny, Nx, L;
    const uint8_t* mask;   /* device, [L][Ny] */
} mrf_op;

typedef struct mrf_recon_opts {
    int32_t iters;         /* iterations (default 10) */
    float   mu;            /* initial step size (default 1) */
    int32_t adaptive;      /* step rule of eq. steprule / Algorithm 2 (default 0) */
    float   zeta;          /* shrink factor of the step rule (default 2) */
    int32_t kappa;         /* rescale the first iterate by ||Y|| / ||A X^1|| (default 0) */
    float   tol;           /* stop when the objective's relative progress < tol (0 = off) */
    int32_t max_shrink;    /* bound on step-rule shrinks per iteration (default 30) */
    int32_t resume;        /* 1: continue from the iterate in X_out and the warm-start atoms in
                              idx_out (a saved checkpoint: the iterate is fully described by X,
                              or by idx and rho) instead of X^0 = 0; the kappa rescale of the
                              first iterate is skipped and the step rule restarts from mu
                              (default 0) */
    float*   mu_history;   /* host float [iters] or NULL: the step size each iteration accepted
                              (after the step rule's shrinks, before the kappa rescale) */
    int32_t* shrink_history;  /* host int32 [iters] or NULL: the step rule's divisions by zeta
                              in each iteration (Prop. stepbound bounds them) */
    mrf_proj_opts proj;
} mrf_recon_opts;

void mrf_default_index_opts(mrf_index_opts* o);
void mrf_default_proj_opts(mrf_proj_opts* o);
void mrf_default_recon_opts(mrf_recon_opts* o);

/*
 * Build the dictionary index (§3.1 eq. fingerprints; §4.3 "cover tree built for the normalized
 * fingerprint dictionary").
 *   atoms      complex64 [d][L], host or device memory (detected); copied.  Atoms need not be
 *              normalised: the projection divides by the norm of each stored atom.
 *   params     host float32 [d][P] (e.g. T1, T2, B0), copied; the look-up table of Algorithm 2.
 *              May be NULL when P == 0.
 *   grid_shape host int32 [grid_ndim] or NULL: the parameter grid (used by the learned
 *              proposal's neighbourhood); d must not exceed its number of cells.
 *   out        receives the new dict; free it with mrf_dict_free.
 * Synchronises `stream` before returning.  Errors: MRF_EINVAL (d < 1, L < 1, L > 4096,
 * null atoms/out), MRF_ENOMEM, MRF_ECUDA, MRF_ENONFINITE (an atom with zero or non-finite
 * norm).
 */
mrf_status mrf_build_dict_index(const void* atoms, int64_t d, int32_t L,
                                const float* params, int32_t P,
                                const int32_t* grid_shape, int32_t grid_ndim,
                                const mrf_index_opts* opts, mrf_dict** out, void* stream);

void mrf_dict_free(mrf_dict* dict);

/* d, L, P of a dict (any pointer may be NULL). */
mrf_status mrf_dict_info(const mrf_dict* dict, int64_t* d, int32_t* L, int32_t* P);

/* Cover tree built by mrf_build_dict_index (levels r_i = sigma 2^-i, §4.1). */
typedef struct mrf_tree_info {
    int64_t nodes;            /* distinct atoms in the tree */
    int64_t explicit_nodes;   /* (node, level) pairs with children other than the node itself */
    int32_t levels;           /* i_max */
    int32_t metric;           /* mrf_cone the tree was built for */
    double  sigma;            /* maximal distance from the root, the level-0 radius */
    double  build_ms;         /* host construction + upload time */
    int64_t device_bytes;     /* device memory of the flattened tree */
} mrf_tree_info;

mrf_status mrf_tree_get_info(const mrf_dict* dict, mrf_tree_info* info);

/* Copy the tree structure to host arrays (any may be NULL): per atom [d] the level at which it
 * first appears (-1 for a duplicate), its parent atom at the level above (-1 for the root and
 * duplicates) and its representative node; per explicit node [explicit_nodes] its atom, its level
 * i (its new children first appear at i + 1) and its maxdist, the largest distance from the node
 * to its subtree (§4.1, eq. maxdistbound). */
mrf_status mrf_tree_export(const mrf_dict* dict, int32_t* first_level, int32_t* parent,
                           int32_t* rep, int32_t* en_atom, int32_t* en_level, float* en_maxdist);

/* Blocks of MRF_PROJ_TREE_TC (any output may be NULL): their number, each block's radius
 * (host float [nblk]: an upper bound on the tree-metric distance from the block's first atom to
 * each of its atoms) and the depth-first order (host int32 [nblk * 128]: the atom at each
 * position, -1 past the last atom).  MRF_EUNSUPPORTED without mrf_index_opts.tree_tc. */
mrf_status mrf_tree_blocks(const mrf_dict* dict, int64_t* nblk, float* radius, int32_t* perm);

/* Build the cover tree of host atoms on the host alone (no GPU; offline use and tests), with
 * the construction mrf_build_dict_index uses.  atoms: host complex64 [d][L]; cone: the metric.
 * Outputs as mrf_tree_export, with the explicit-node arrays sized d (there are at most d - 1
 * explicit nodes); *n_explicit, *sigma and *levels receive the counts and the root radius. */
mrf_status mrf_tree_build_host(const void* atoms, int64_t d, int32_t L, int32_t cone,
                               float dup_tol, int32_t* first_level, int32_t* parent,
                               int32_t* rep, int32_t* en_atom, int32_t* en_level,
                               float* en_maxdist, int64_t* n_explicit, double* sigma,
                               int32_t* levels);

/* Pre-allocate scratch for up to n_max voxels (so later calls allocate nothing). */
mrf_status mrf_dict_reserve(mrf_dict* dict, int64_t n_max);

/* Synchronise `stream`, read and clear the device error word; returns the matching status. */
mrf_status mrf_dict_check(mrf_dict* dict, void* stream);

/*
 * Matched-filtering projection of n fingerprints (§3.2, eqs. exactP / exactPs; with
 * MRF_PROJ_COVERTREE, the (1+eps)-ANNS of Algorithm 1 on Z_v / ||Z_v|| warm-started at
 * warm_idx (§4.3, eq. ANN1), then the exact rescore of the 8 best atoms it visited; voxels
 * routed away by `tree_route` (a warm atom, or a long candidate list, still farther than it) or
 * whose candidate list would exceed its capacity (mrf_tune.tree_list_cap) are projected by the
 * exhaustive search instead: BF16 tensor cores (certified as `certify` says) when the
 * dictionary has the BF16 operand, else FP32).
 *   Z         device complex64 [n][L]
 *   warm_idx  device int32 [n] or NULL: previous atoms, the warm start of the tree search
 *   idx_out   device int32 [n]: j*_v
 *   rho_out   device complex64 [n]: rho_v = D_j*^H Z_v / ||D_j*||^2 (complex cone) or
 *             gamma_v (real cone, imaginary part 0); compensated FP32 sums (exact products,
 *             two-sum accumulation) reduced in FP64, an error of a few units of 2^-46
 *   X_out     device complex64 [n][L] or NULL: X_v = rho_v D_j*
 * A zero fingerprint gives j* = 0, rho = 0.  Exact ties go to the smallest index.
 */
mrf_status mrf_project(mrf_dict* dict, const void* Z, int64_t n, const mrf_proj_opts* opts,
                       const int32_t* warm_idx, int32_t* idx_out, void* rho_out, void* X_out,
                       mrf_stats* stats, void* stream);

/*
 * Candidate lists of the tensor-core matched filter, before any rescore (diagnostics and the
 * error-bound tests): for modes MRF_PROJ_BF16, MRF_PROJ_FP8 and MRF_PROJ_BF16X3 the kernel's K
 * best atoms of each voxel (K = the mode's topk) with one atom split, in descending kernel
 * score, ties to the smallest index.  Queries are used as given (no phase alignment).
 *   Z          device complex64 [n][L]
 *   score_out  device float32 [n][K]: |c~|^2 (complex cone) or Re c~ (real cone), c~ the
 *              kernel's correlation of the voxel with the normalised atom D_j / ||D_j||
 *   idx_out    device int32 [n][K]: the atoms (-1 for slots past d)
 *   bound_out  device float32 [n] or NULL: the bound of |c~ - c| / ||Z_v|| the library uses
 *              for that mode (the voxel's own bound for MRF_PROJ_BF16X3)
 * Errors: MRF_EINVAL (other modes, null outputs), MRF_EUNSUPPORTED (operand not packed).
 */
mrf_status mrf_search_candidates(mrf_dict* dict, const void* Z, int64_t n,
                                 const mrf_proj_opts* opts, float* score_out, int32_t* idx_out,
                                 float* bound_out, void* stream);

/* A(X) = P_Omega F X: X device complex64 [n][L] -> Y device complex64 [Ny][Nx][L] (lines
 * outside Omega_t are written as zero). */
mrf_status mrf_forward(const mrf_op* op, const void* X, void* Y, void* stream);

/* A^H(Y) = F^H P_Omega^H Y: Y device [Ny][Nx][L] -> AHY device [n][L]. */
mrf_status mrf_adjoint(const mrf_op* op, const void* Y, void* AHY, void* stream);

/* Gradient step alone (§3.2, eq. blip; Algorithm 2 "gradient update"):
 * Z = X - mu (A^H A X - AHY), all device complex64 [n][L]; X and Z may not alias. */
mrf_status mrf_gradient(mrf_dict* dict, const mrf_op* op, const void* AHY, const void* X,
                        float mu, void* Z, void* stream);

/*
 * One BLIP iteration (§3.2, eq. blip): Z = X - mu (A^H A X - AHY), then the projection; X is
 * overwritten by rho_v D_j*.
 *   AHY     device complex64 [n][L]: A^H Y (mrf_adjoint)
 *   X       device complex64 [n][L], in/out
 *   idx_io  device int32 [n]: in = the previous atoms (warm start), out = the new atoms
 *   rho_out device complex64 [n] or NULL
 */
mrf_status mrf_ipg_step(mrf_dict* dict, const mrf_op* op, const void* AHY, void* X, float mu,
                        const mrf_proj_opts* opts, int32_t* idx_io, void* rho_out,
                        mrf_stats* stats, void* stream);

/*
 * Whole reconstruction (Algorithm 2): A^H Y once, X^0 = 0 (or the iterate in X_out with
 * mrf_recon_opts.resume), `iters` iterations with the options' step rule and kappa rescale,
 * then the look-up table.  Synchronises `stream`.
 *   Y          complex64 [Ny][Nx][L]
 *   X_out      complex64 [n][L]
 *   idx_out    int32 [n]
 *   rho_out    complex64 [n] or NULL
 *   params_out float32 [n][P] or NULL
 * Each of these may be device memory or host memory (pinned or pageable; detected).  Host
 * buffers are staged through device buffers that the call allocates and frees: Y (and, with
 * `resume`, X_out and idx_out) is copied in at the start and the outputs are copied back
 * before the call returns, so every transfer lies inside the call.  op->mask stays device
 * memory.
 */
mrf_status mrf_reconstruct(mrf_dict* dict, const mrf_op* op, const void* Y,
                           const mrf_recon_opts* opts, void* X_out, int32_t* idx_out,
                           void* rho_out, float* params_out, mrf_stats* stats, void* stream);

/*
 * Exhaustive FP32 projection that allocates no device memory (the paper has no counterpart:
 * this is a deployment variant of mrf_project's FP32 mode).  For callers that must not
 * allocate once running -- applications whose device memory belongs to their own pool or
 * allocator, or real-time pipelines that forbid cudaMalloc/cudaFree after start-up.  The caller
 * passes the dictionary and every input and output; the working memory is one file-scope device
 * array of about 20 MB that every GPU loading the library holds until the process exits.
 *   atoms    device complex64 [d][L], 1 <= d <= 1,048,576, 1 <= L <= 4096 (zero atoms rejected)
 *   Z        device complex64 [n][L], 0 <= n <= 4096 voxels per call
 *   cone     mrf_cone
 *   idx_out  device int32 [n]; rho_out device complex64 [n] or NULL; X_out device [n][L] or NULL
 * The atoms are used as given: no phase alignment is applied (with MRF_CONE_REAL_POS the real
 * positive rule runs on the atoms and queries as they are).  Results equal mrf_project's FP32
 * mode on a dictionary built from the same atoms without phase_align (top-8 candidates,
 * near-tie rescore and density in compensated FP32 reduced in FP64).  Larger sizes return
 * MRF_EINVAL with a message, before any launch.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the one array, so
 * calls that overlap on the GPU (other streams, other threads) race; serialise them.  The call
 * synchronises `stream` before returning.
 */
mrf_status mrf_project_fp32_static(const void* atoms, int64_t d, int32_t L, const void* Z,
                                   int64_t n, int32_t cone, int32_t* idx_out, void* rho_out,
                                   void* X_out, void* stream);

/*
 * Learned proposal (the build's learned form of the projection; the paper keeps learned
 * matching out of its comparisons, §2).  A network x (2L) -> hidden -> hidden -> 3 with GELU
 * maps the canonical fingerprint -- z/||z|| rotated by exp(-i angle(v1^H z)), v1 the
 * dictionary's dominant right singular vector -- to standardised (log T1, log T2, B0).  The
 * nearest grid cell's (2 radius + 1)^k neighbourhood of valid atoms is rescored exactly, and a
 * voxel whose best normalised correlation stays below mrf_proj_opts.fallback_thr, or (with
 * mrf_proj_opts.learned_edge) whose best atom lies on the neighbourhood's edge, is projected
 * by the exhaustive search.  Training and inference run on this library's kernels.
 */
typedef struct mrf_mlp mrf_mlp;

typedef struct mrf_mlp_opts {
    int32_t  hidden;        /* hidden width, a multiple of 16 in 16..4096 (default 512) */
    int32_t  radius;        /* neighbourhood radius per grid dimension (default 2: 5x5x5) */
    int64_t  residue_pool;  /* capacity of the aliasing-residue pool, fingerprints (262144) */
    uint64_t seed;          /* initialisation and sampling seed (default 5000) */
    int32_t  reserved[8];
} mrf_mlp_opts;

typedef struct mrf_train_opts {
    int32_t steps;          /* Adam steps */
    int32_t batch;          /* fingerprints per step, <= 65536 */
    float   lr;             /* Adam learning rate (beta1 0.9, beta2 0.999, eps 1e-8) */
    float   snr_lo, snr_hi; /* noise SNR range, dB */
    float   p_residue;      /* probability that a sample carries a residue from the pool */
    int32_t reserved[6];
} mrf_train_opts;

void mrf_default_mlp_opts(mrf_mlp_opts* o);

/* Create a model for `dict` (built with params (T1, T2[, B0]) and grid_shape (n1, n2[, nB0]) in
 * that order).  grid_axes: host float32, the axis values concatenated (n1 T1 values, n2 T2
 * values[, nB0 B0 values]), each ascending; cell_atom: host int32 [n1 n2 (nB0)], the atom of each
 * grid cell or -1.  Initialises the weights (He normal, seed), the target standardisation from
 * the dictionary's parameters, and v1 by power iteration.  Synchronises `stream`. */
mrf_status mrf_mlp_create(mrf_dict* dict, const float* grid_axes, const int32_t* cell_atom,
                          const mrf_mlp_opts* opts, mrf_mlp** out, void* stream);
void mrf_mlp_free(mrf_mlp* mlp);

/* Append aliasing residues (Z_v - X0_v) / ||X0_v|| of voxels with X0_v != 0 to the pool (Z: an
 * IPG query, X0: the ground-truth image; device complex64 [n][L]); reservoir sampling once full. */
mrf_status mrf_mlp_add_residues(mrf_mlp* mlp, const void* Z, const void* X0, int64_t n,
                                void* stream);

/* `steps` Adam steps on batches synthesised on the GPU: a random atom, a complex scale of
 * modulus U[0.5, 1], a pool residue with probability p_residue, complex Gaussian noise at an SNR
 * drawn from [snr_lo, snr_hi] dB.  loss_history: host float [steps] or NULL (if given, the
 * call synchronises every step). */
mrf_status mrf_mlp_train(mrf_mlp* mlp, const mrf_train_opts* opts, float* loss_history,
                         void* stream);

/* Read (set = 0) or write (set = 1) all parameters as one host float32 array in the order
 * W1 [2L][H], b1 [H], W2 [H][H], b2 [H], W3 [H][3], b3 [3]; *count receives its length. */
mrf_status mrf_mlp_params(mrf_mlp* mlp, float* host_params, int32_t set, int64_t* count);

/* Forward pass on X (device float32 [B][2L]) into Y_out ([B][3], host or device, may be NULL);
 * with targets T ([B][3]) also the MSE loss (host double) and the gradient of every parameter
 * (grads_out, same layout as mrf_mlp_params, host or device).  Synchronises `stream`. */
mrf_status mrf_mlp_grad(mrf_mlp* mlp, const float* X, const float* T, int64_t B, float* Y_out,
                        float* grads_out, double* loss_out, void* stream);

/* Inference as the learned projection runs it: weights and activations rounded to BF16, the two
 * hidden layers on the tensor cores with FP32 accumulation and bias + GELU in FP32, the output
 * layer in FP32.  X device float32 [B][2L] (canonical inputs), Y_out device float32 [B][3]
 * (standardised targets).  Asynchronous on `stream`; device errors are reported by the
 * dictionary's next checked call (mrf_dict_check). */
mrf_status mrf_mlp_infer(mrf_mlp* mlp, const float* X, int64_t B, float* Y_out, void* stream);

/* Canonical network inputs of Z (device complex64 [n][L]) into X (device float32 [n][2L]); also
 * copies v1 (host complex64 [L]) and the target means and standard deviations (host float [6])
 * when those pointers are not NULL.  Synchronises `stream`. */
mrf_status mrf_mlp_canonical(mrf_mlp* mlp, const void* Z, int64_t n, float* X, float* v1_host,
                             float* tstats_host, void* stream);

/* Use `mlp` for MRF_PROJ_LEARNED projections of `dict` (NULL detaches). */
mrf_status mrf_dict_attach_mlp(mrf_dict* dict, mrf_mlp* mlp);

/*
 * Batches of slices (the batching form: many slices of different sizes through whole BLIP
 * iterations).  The slices share the dictionary; all of them stay resident, stacked voxel-major,
 * and each iteration is every slice's gradient step followed by one projection of all stacked
 * voxels (one persistent launch of the search).  With use_graph the iteration is captured once
 * into a CUDA graph and replayed (projections without host synchronisation only, certify = 0:
 * FP32, BF16, FP8, the tensor-core tree search, and -- when the dictionary has the BF16
 * operand -- the cover-tree and learned forms, whose exhaustive fallback then reads its voxel
 * count on the device).  The masks of
 * `ops` are read at every iteration and must stay alive.
 */
typedef struct mrf_batch mrf_batch;

/* n_slices operators (their L must be the dictionary's).  Allocates the stacked buffers and the
 * dictionary's scratch for the total voxel count. */
mrf_status mrf_batch_create(mrf_dict* dict, int32_t n_slices, const mrf_op* ops,
                            mrf_batch** out);
void mrf_batch_free(mrf_batch* batch);

/* A^H Y of every slice (Y: host array of n_slices device pointers to complex64 [Ny][Nx][L])
 * into the batch; X = 0 and the warm-start atoms = 0. */
mrf_status mrf_batch_load(mrf_batch* batch, const void* const* Y, void* stream);

/* `iters` iterations (step mu, projection `opts`) over all slices, asynchronous on `stream`. */
mrf_status mrf_batch_run(mrf_batch* batch, int32_t iters, float mu, const mrf_proj_opts* opts,
                         int32_t use_graph, void* stream);

/* Device pointers to slice s's rows of the stacked image, atoms and densities; its voxel count
 * and offset (any output may be NULL). */
mrf_status mrf_batch_slice(mrf_batch* batch, int32_t s, void** X, int32_t** idx, void** rho,
                           int64_t* n, int64_t* offset);

/* Look-up table of all stacked voxels: params_out device float32 [sum n_s][P]. */
mrf_status mrf_batch_lut(mrf_batch* batch, float* params_out, void* stream);

/*
 * Temporal subspace compression (§3.3, eqs. CS1, gradupdate and gradcompression; the option of
 * §4.3 and §6).  V_s (device complex64 [L][s], row t = frame t) spans the s dominant eigenvectors
 * of the frame Gram matrix sum_j D_j D_j^H.  A fingerprint row x compresses to x conj(V_s)
 * (= V_s^H x) and a compressed row expands to xc V_s^T.  BLIP then runs on compressed images
 * [n][s] against a dictionary index built from the compressed atoms (mrf_svd_compress of the
 * atoms, then mrf_build_dict_index); only V_s V_s^H enters the results, so any orthonormal
 * basis of the same subspace gives the same reconstruction.
 */
typedef struct mrf_svd_op mrf_svd_op;

/* V_out (device complex64 [L][s]) = the s dominant eigenvectors of sum_j D_j D_j^H, each with
 * its largest-magnitude entry real positive; eig_out (host, may be NULL) = their eigenvalues,
 * largest first.  Subspace iteration in FP64 with Rayleigh-Ritz; synchronous. */
mrf_status mrf_svd_basis(const mrf_dict* dict, int32_t s, void* V_out, double* eig_out,
                         void* stream);

/* Compression operator for V (host or device complex64 [L][s], copied).  With a sampling op
 * (op->L == L) it also holds, per phase-encode line ky, the s x s matrix
 * V_s^H diag(mask[., ky]) V_s of the compressed normal operator; op may be NULL for
 * compression only.  The op's mask must stay alive. */
mrf_status mrf_svd_op_create(const mrf_op* op, const void* V, int32_t L, int32_t s,
                             mrf_svd_op** out, void* stream);
void mrf_svd_op_free(mrf_svd_op* so);

/* Xc [n][s] = X [n][L] conj(V_s) and X [n][L] = Xc V_s^T (device complex64, row-major). */
mrf_status mrf_svd_compress(const mrf_svd_op* so, const void* X, int64_t n, void* Xc,
                            void* stream);
mrf_status mrf_svd_expand(const mrf_svd_op* so, const void* Xc, int64_t n, void* X,
                          void* stream);

/* The compressed gradient step alone (eq. gradupdate / gradcompression):
 * Zc = Xc - mu (compress(A^H A expand(Xc)) - AHYc), all device complex64 [n][s]; the same
 * kernels as mrf_svd_ipg_step's gradient (for power-of-two Ny the two halves of the fused
 * y-transform kernel around the per-line s x s product, else cuFFT). */
mrf_status mrf_svd_gradient(mrf_dict* dict_c, mrf_svd_op* so, const void* AHYc, const void* Xc,
                            float mu, void* Zc, void* stream);

/* One compressed iteration (eq. gradupdate + projection onto cone(D conj(V_s))): dict_c is the
 * index of the compressed atoms (its L must be s), AHYc = compress(A^H Y), Xc [n][s] in/out,
 * idx_io the warm start / result.  Same projection options as mrf_project. */
mrf_status mrf_svd_ipg_step(mrf_dict* dict_c, mrf_svd_op* so, const void* AHYc, void* Xc,
                            float mu, const mrf_proj_opts* opts, int32_t* idx_io,
                            void* rho_out, void* stream);

/* Whole compressed BLIP from Xc = 0 (Algorithm 2 in C^s): A^H Y, compression, opts->iters
 * iterations with opts->mu and, when opts->adaptive, the step rule of eq. steprule in the
 * compressed form of §4.3, mu_k < ||Xc^{k+1} - Xc^k||^2 / ||A((Xc^{k+1} - Xc^k) V_s^T)||^2
 * (shrinks by opts->zeta, at most opts->max_shrink), the kappa rescale of the first iterate
 * (opts->kappa), the histories of opts->mu_history / shrink_history, then optionally the
 * expanded image X_out [n][L] and the look-up table params_out [n][P].  opts->tol and
 * opts->resume are not available here (MRF_EUNSUPPORTED).  Y device [Ny][Nx][L].
 * Synchronous; reports device errors. */
mrf_status mrf_svd_reconstruct(mrf_dict* dict_c, mrf_svd_op* so, const void* Y,
                               const mrf_recon_opts* opts, void* Xc_out, void* X_out,
                               int32_t* idx_out, void* rho_out, float* params_out,
                               void* stream);

/* Look-up table Theta_v = params[idx_v] (Algorithm 2, last step): device int32 [n] ->
 * device float32 [n][P]. */
mrf_status mrf_lut(const mrf_dict* dict, const int32_t* idx, int64_t n, float* params_out,
                   void* stream);

/*
 * Launch-geometry tuning of the exhaustive kernels (read by the project's autotuner).  Zero
 * fields select the library's defaults.  The `last_*` fields report the geometry of the most
 * recent launch on this dictionary.
 */
typedef struct mrf_tune {
    int32_t bf16_cluster;      /* CTAs per cluster co-scheduled on the same atom blocks, each
                                  loading its own copy (no multicast): 1, 2, 4; default 1 */
    int32_t bf16_live_tiles;   /* voxel tiles (128 rows) kept live per super-group, >= 1 */
    int32_t bf16_splits;       /* atom splits of the BF16 search, >= 1 */
    int32_t fp32_splits;       /* atom splits of the FP32 search, >= 1 */
    int32_t last_bf16_ctas;    /* out: CTAs of the last BF16 search launch */
    int32_t last_bf16_cluster; /* out: its cluster size */
    int32_t last_bf16_splits;  /* out: its atom splits */
    int32_t last_fp32_splits;  /* out: atom splits of the last FP32 search launch */
    int32_t tree_list_cap;     /* cover-tree candidate list capacity per voxel, 64..512; 0 = the
                                  longest list with which four CTAs of four queries stay
                                  resident per SM (256 for L <= 768, 192 at L = 1000, 64 from
                                  L = 1480): shorter lists fit more warps per SM, longer lists
                                  route fewer voxels to the exhaustive search */
    int32_t bf16_pair;         /* 1: the tensor-core search on CTA pairs (2-SM MMA, M = 256,
                                  each CTA staging half of every atom block) instead of single
                                  CTAs or clusters (bf16_cluster is then ignored); 2: single
                                  CTAs or clusters; 0 = the library's default (single CTAs for
                                  the exhaustive forms and the tree search's split operand,
                                  CTA pairs for the tree search's BF16 operand) */
    int32_t tree_order;        /* cover-tree queries of a warm-started search: 1 = processed in
                                  the order of their warm-start atom's tree position, so that
                                  queries of one subtree run side by side and share cached tree
                                  nodes and atoms (results are the same either way); 2 = voxel
                                  order; 0 = the library's default */
    int32_t tree_tc_group;     /* MRF_PROJ_TREE_TC: consecutive 128-voxel tiles that share one
                                  block list (the union of their voxels' lists), 1..64: larger
                                  groups search more blocks per voxel but stream each block
                                  once for the whole group, as the exhaustive search does;
                                  0 = the library's default (2 for the BF16 operand, 4 for the
                                  split-BF16 one) */
    int32_t tree_tc_chunks;    /* MRF_PROJ_TREE_TC: chunks a full block list is cut into, the
                                  work units of the persistent search and the candidate lists
                                  per voxel, 1..64; 0 = the library's default (32) */
    int32_t tree_tc_super;     /* MRF_PROJ_TREE_TC: neighbouring block lists whose work units
                                  run chunk round by chunk round together (so the CTAs share
                                  the blocks their lists have in common through L2), 1..256;
                                  0 = the library's default (1) */
    int32_t reserved[2];
} mrf_tune;

mrf_status mrf_get_tune(const mrf_dict* dict, mrf_tune* out);
mrf_status mrf_set_tune(mrf_dict* dict, const mrf_tune* in);

/*
 * Stage profiler (tracing aid; the paper reports search and total times, Tables 2-3).  While
 * enabled, every call records a CUDA event pair on its own stream around each stage and counts
 * the library's kernel launches.  mrf_profile_read synchronises on the recorded events, adds
 * their elapsed times into ms[stage] and launches[stage] for stage < n_stages, and clears
 * them.  Stages: 0 gradient step (cuFFT + mask + combine; cuFFT's kernels are timed here but
 * not counted as launches), 1 query packing (BF16 or FP8), 2 tensor-core search (BF16 or
 * FP8), 3 FP32 search,
 * 4 merge / rescore / density, 5 fallback to the exhaustive search (certification, cover-tree
 * routing or overflow, learned-proposal fallback), 6 look-up table, 7 proposal search (cover
 * tree traversal, learned network + neighbourhood rescore, or the tensor-core tree search's
 * centre product, bounds, voxel sort and tile lists; its block-list search counts as stage 2).  Enabling or disabling clears the tables.  Not thread-safe.
 */
#define MRF_PROFILE_STAGES 8
mrf_status mrf_profile_enable(int32_t on);
mrf_status mrf_profile_read(double* ms, int64_t* launches, int32_t n_stages);

/*
 * Failure injection, for tests of the error paths (no GPU fault is ever provoked).
 * mrf_debug_fail_alloc(k): the library's device allocations (dictionary index, scratch, the
 * reconstruction's buffers) succeed k more times, then one is refused with MRF_ENOMEM and
 * injection turns itself off; k < 0 turns it off.  Process-wide.
 * mrf_selftest_wait_timeout: one thread waits on an mbarrier that nothing arrives on, with the
 * library's bounded wait cut to timeout_ns (1 ns .. 1 s); the wait gives up, the kernel raises
 * the device error word and the call returns MRF_ETIMEOUT -- the path every persistent kernel of
 * the library takes when a bound expires.  Synchronises `stream`.
 */
void mrf_debug_fail_alloc(int32_t k);
mrf_status mrf_selftest_wait_timeout(int64_t timeout_ns, void* stream);

const char* mrf_status_str(mrf_status s);
const char* mrf_last_error(void);   /* thread-local message of the last failure */

#ifdef __cplusplus
}
#endif
#endif /* MRF_H */
