// Query-batched cover-tree search on the tensor cores (§4.1 Algorithm 1 and Def. eNN; the
// closing remark of §7 on grouping queries that fall in the same part of the tree).
//
// The tree is used the way a dual-tree search uses its reference side: its depth-first order
// cuts the dictionary into 128-atom blocks whose atoms lie close together in the tree metric
// (each subtree is contiguous), and every block b gets a ball -- centre c_b = its first atom,
// radius R_b = max_{j in b} delta(c_b, j), exact in FP64 and rounded up.  Per projection:
//   1. every voxel's correlations with all block centres: one dense split-BF16 product on the
//      tensor cores (queries [lo | hi | hi] x centres [hi | lo | hi]), with the voxel's rigorous
//      error bound b_v;
//   2. per voxel, lower and upper bounds delta_lo / delta_hi of delta(z^, c_b) from those
//      correlations (directed rounding), r_v = min_b delta_hi (the nearest centre is an atom, so
//      the nearest atom is at most r_v away), and the blocks that can still hold an atom closer
//      than r_v / (1 + eps): delta_lo(b) - R_b <= r_v / (1 + eps) (triangle inequality), plus
//      the nearest centre's block;
//   3. voxels sorted by radius class (r_v in steps of 0.1), then by nearest centre, so a
//      128-voxel tile holds voxels of one region of the tree with lists of similar reach; a few
//      consecutive tiles share one block list, the union of their voxels' lists (the query
//      batch shares one candidate set);
//   4. the tensor-core search kernel in block-list mode scans each group's list in chunks of
//      equal length over the depth-first operand (BF16 on CTA pairs of 256 voxels, or
//      split-BF16 on single CTAs for certified results) and keeps each voxel's top K per chunk;
//      the merge rescoring and certification follow in the caller.
// A block is dropped only when none of its atoms can be closer than r_v / (1 + eps), so the best
// atom over the searched blocks is a (1 + eps)-approximate nearest neighbour (Def. eNN), and the
// exact one for eps = 0.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include <cub/cub.cuh>

#include "mrf_internal.cuh"

struct TreeTC {
    int metric = 0;              // tree metric: 0 phase-quotient (complex cone), 1 Euclidean
    int64_t nblk = 0;            // blocks of the depth-first operands (= the dictionary's)
    int64_t words = 0;           // 32-bit words of one block mask
    int32_t* perm = nullptr;     // [nblk * 128] atom at each depth-first position, -1 = empty
    __nv_bfloat16* op = nullptr;    // BF16 operand in depth-first order (with the BF16 operand)
    __nv_bfloat16* op3 = nullptr;   // split-BF16 operand in depth-first order (with the split one)
    float op3_al = 0.f, op3_ae = 0.f;
    int64_t ncb = 0, ncbblk = 0; // centres (one per block), centre operand blocks
    int32_t* cidx = nullptr;     // [ncb] centre atoms
    __nv_bfloat16* cop3 = nullptr;  // [ncbblk * 256][3 Kp] split-BF16 operand of the centres
    float c_al = 0.f, c_ae = 0.f;
    float* radius = nullptr;     // [nblk] R_b, rounded up
    double build_ms = 0.0;
    // per-projection scratch (grown on demand)
    int64_t cap = 0, crows = 0, tiles_cap = 0, blist_cap = 0;
    __nv_bfloat16* zc3 = nullptr;   // [crows][3 Kp] queries of the centre product
    float* cs = nullptr;         // [crows][ncbblk * 256] centre correlations (re, im rows)
    float* znorm = nullptr;      // [crows]
    float* cmarg = nullptr;      // [crows] bound of the centre correlations
    uint32_t* keep = nullptr;    // [cap][words] per-voxel block masks
    int32_t* key = nullptr;      // [cap] nearest centre
    int32_t* val = nullptr;      // [cap] voxel
    int32_t* skey = nullptr;
    int32_t* vorder = nullptr;   // [cap] voxels in tile order
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    uint32_t* tmask = nullptr;   // [tiles][words]
    uint32_t* gmask = nullptr;   // [tiles][words] (groups of tiles; at most one per tile)
    int32_t* tcnt = nullptr;     // [tiles + 1] group list lengths
    int32_t* tfirst = nullptr;   // [tiles + 1] group list offsets
    int32_t* sgmax = nullptr;    // [tiles + 1] chunk rounds of each super-group
    int32_t* ucnt = nullptr;     // [tiles + 1] super-group work units
    int32_t* uoff = nullptr;     // [tiles + 1] first work unit of each super-group
    int32_t* blist = nullptr;    // [blist_cap]
    int32_t* misc = nullptr;     // [4]: total blocks, longest tile list, voxel count
    void* part = nullptr;        // candidates [S][cap][K] scores then indices
    size_t part_bytes = 0;
};

namespace {

constexpr int kThreads = 256;
constexpr int kGroupBf16 = 2;     // default tiles per block list (BF16 operand)
constexpr int kGroupSplit = 4;    // the same for the split-BF16 operand (3x the MMA per block)
constexpr int kChunks = 32;       // chunks (candidate slots) a full block list is cut into
constexpr int kRadiusBins = 16;   // radius classes of the voxel sort (r_v in steps of 0.1)
constexpr int kSuper = 1;         // groups per super-group

inline unsigned grid_for(int64_t work) {
    return static_cast<unsigned>((work + kThreads - 1) / kThreads);
}

template <class T>
mrf_status talloc(T** p, size_t count) {
    if (*p) {
        cudaFree(*p);
        scratch_epoch_bump();
        *p = nullptr;
    }
    if (count == 0) return MRF_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        mrf_set_error(std::string("cudaMalloc(tree search): ") + cudaGetErrorString(e));
        return MRF_ENOMEM;
    }
    return MRF_OK;
}

// R_b = max over the block's atoms j of delta(c_b, j), c_b the block's first atom: one warp per
// depth-first position, the unit correlation u_c^H u_j accumulated in FP64 from the stored
// atoms and their FP64 norms; delta^2 = 2 - 2 |.| (phase-quotient metric) or 2 - 2 Re(.)
// (Euclidean).  The FP64 cancellation in 2 - 2 c costs at most ~1e-13 in delta^2, so
// delta (1 + 1e-6) + 1e-6 bounds the exact distance from above; maxima via the order of
// non-negative float bit patterns.
__global__ void k_block_radius(const float2* __restrict__ atoms, const double* __restrict__ norm2,
                               const int32_t* __restrict__ perm, int64_t npos, int L, int metric,
                               unsigned int* __restrict__ rbits) {
    const int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= npos) return;
    const int32_t j = perm[p];
    const int64_t b = p >> 7;
    const int32_t c = perm[b << 7];
    if (j < 0 || c < 0 || j == c) return;
    const float2* u = atoms + static_cast<int64_t>(c) * L;
    const float2* w = atoms + static_cast<int64_t>(j) * L;
    double re = 0.0, im = 0.0;
    for (int t = lane; t < L; t += 32) {
        const float2 a = u[t], z = w[t];
        re += static_cast<double>(a.x) * z.x + static_cast<double>(a.y) * z.y;
        im += static_cast<double>(a.x) * z.y - static_cast<double>(a.y) * z.x;
    }
    for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane != 0) return;
    const double s = 1.0 / sqrt(norm2[c] * norm2[j]);
    const double cr = (metric == 0) ? sqrt(re * re + im * im) * s : re * s;
    const double d2 = fmax(0.0, 2.0 - 2.0 * cr);
    const float r = __double2float_ru(sqrt(d2) * (1.0 + 1e-6) + 1e-6);
    atomicMax(rbits + b, __float_as_uint(r));
}

}  // namespace

namespace {

// One warp per voxel of a row chunk: bounds on delta(z^, c_b) for every centre from the split-BF16
// correlations cs (row v: for centre b, Re at (b / 128) 256 + b % 128, Im 128 further), the
// voxel's correlation bound bz (normalised units) and the relative bound kappa of its FP32
// norm; every step rounded away from the side it bounds (delta^2 = 2 - 2 c for unit vectors).
// Writes the voxel's block mask, its sort key (radius class, then nearest centre in the low
// cbits bits) and its index.
__global__ void k_tree_bounds(const float* __restrict__ cs, int64_t ld, int64_t rows,
                              int64_t row0, const float* __restrict__ znorm,
                              const float* __restrict__ cmarg, float kappa,
                              const float* __restrict__ radius, int64_t ncb, int64_t words,
                              int metric, float inv1e, int cbits, uint32_t* __restrict__ keep,
                              int32_t* __restrict__ key, int32_t* __restrict__ val) {
    const int64_t v = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= rows) return;
    const int64_t g = row0 + v;
    uint32_t* km = keep + g * words;
    const float zn = znorm[v];
    if (!(zn > 0.f) || !(zn < INFINITY)) {
        // zero (or non-finite) query: the merge assigns atom 0 (or flags the voxel); one block
        for (int64_t w = lane; w < words; w += 32) km[w] = (w == 0) ? 1u : 0u;
        if (lane == 0) {
            key[g] = (kRadiusBins - 1) << cbits;
            val[g] = static_cast<int32_t>(g);
        }
        return;
    }
    const float zlo = __fmul_rd(zn, 1.f - kappa), zhi = __fmul_ru(zn, 1.f + kappa);
    const float rlo = __frcp_ru(zlo), rhi = __frcp_rd(zhi);   // >= 1 / ||z||, <= 1 / ||z||
    const float bz = cmarg[v];
    const float* row = cs + v * ld;
    const bool cplx = (metric == 0);
    // Pass 1: the centre with the largest lower bound of c = |u^H z^| (or Re u^H z^): the lower
    // bound is a non-decreasing function of |c~|^2 rounded down (of Re c~), so the arg max of
    // that plain quantity is the centre of r_v = min_b delta_hi (ties: the first centre).
    float sbest = -INFINITY;
    int64_t bbest = ncb;
    for (int64_t b = lane; b < ncb; b += 32) {
        const int64_t col = (b >> 7) * 256 + (b & 127);
        const float re = row[col];
        const float sv = cplx ? __fmaf_rd(re, re, __fmul_rd(row[col + 128], row[col + 128])) : re;
        if (sv > sbest) { sbest = sv; bbest = b; }
    }
    for (int o = 16; o; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, sbest, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bbest, o);
        if (os > sbest || (os == sbest && oi < bbest)) { sbest = os; bbest = oi; }
    }
    if (bbest >= ncb) bbest = 0;   // non-finite correlations: the merge flags the voxel
    float clo;
    if (cplx) clo = __fmul_rd(__fsqrt_rd(fmaxf(sbest, 0.f)), rhi);
    else clo = sbest >= 0.f ? __fmul_rd(sbest, rhi) : __fmul_rd(sbest, rlo);
    clo = fmaxf(__fsub_rd(clo, bz), cplx ? 0.f : -1.f);
    const float best = __fsqrt_ru(fmaxf(0.f, __fmaf_ru(-2.f, clo, 2.f)));   // r_v
    const float thr = __fmul_ru(best, inv1e);
    // Pass 2: block b can be dropped when even the upper bound of c is below the correlation
    // 1 - (thr + R_b)^2 / 2 of distance thr + R_b (rounded down); for the complex cone the test
    // runs on |c~|^2 rounded up against ((bound - b_v) ||z||)^2 rounded down: no square root
    // or division per centre.
    for (int64_t w = 0; w < words; ++w) {
        const int64_t b = w * 32 + lane;
        bool k = false;
        if (b < ncb) {
            const int64_t col = (b >> 7) * 256 + (b & 127);
            const float re = row[col];
            const float q = __fadd_ru(thr, radius[b]);
            const float rhs = __fmaf_rd(-0.5f, __fmul_ru(q, q), 1.f);
            bool drop;
            if (cplx) {
                const float im = row[col + 128];
                const float m2 = __fmaf_ru(re, re, __fmul_ru(im, im));
                const float t = __fmul_rd(__fsub_rd(rhs, bz), zlo);
                drop = t > 0.f && m2 < __fmul_rd(t, t);
            } else {
                const float ub = __fadd_ru(re >= 0.f ? __fmul_ru(re, rlo) : __fmul_ru(re, rhi), bz);
                drop = ub < rhs;
            }
            k = (b == bbest) || !drop;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, k);
        if (lane == 0) km[w] = m;
    }
    if (lane == 0) {
        // sort key: the voxel's radius class (r_v in steps of 0.1), then its nearest centre --
        // the voxels of a tile then share both their region of the tree and the reach of their
        // block lists, so the tile's union stays close to each voxel's own list
        const int32_t rb =
            static_cast<int32_t>(fminf(best * 10.f, static_cast<float>(kRadiusBins - 1)));
        key[g] = (rb << cbits) | static_cast<int32_t>(bbest);
        val[g] = static_cast<int32_t>(g);
    }
}

// One CTA per 128-voxel tile (voxels vorder[128 g ...]): the union of their block masks.  The
// threads split the (word, row) pairs, OR-ing into shared memory (words x 4 bytes, dynamic).
__global__ void k_tile_union(const uint32_t* __restrict__ keep, int64_t words,
                             const int32_t* __restrict__ vorder, int64_t n,
                             uint32_t* __restrict__ tmask) {
    extern __shared__ uint32_t sm[];
    const int64_t g = blockIdx.x;
    const int64_t i0 = g * 128;
    const int rows = static_cast<int>(n - i0 < 128 ? n - i0 : 128);
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) sm[w] = 0u;
    __syncthreads();
    const int64_t rp = words >= blockDim.x ? 1 : blockDim.x / words;   // row parts
    for (int64_t i = threadIdx.x; i < rp * words; i += blockDim.x) {
        const int64_t w = i % words, part = i / words;
        uint32_t m = 0;
        for (int64_t r = part; r < rows; r += rp)
            m |= keep[static_cast<int64_t>(vorder[i0 + r]) * words + w];
        if (m) atomicOr(&sm[w], m);
    }
    __syncthreads();
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) tmask[g * words + w] = sm[w];
}

// One CTA per group of `group` consecutive tiles: the union of their masks (the group's block
// list), its length, its super-group's chunk rounds (the longest list of the super-group in
// chunks of `chunk` blocks), the running total and maximum, and the voxel-atom pairs the
// search will evaluate (distance-evaluation counter); block 0 also stores the voxel count for
// the merge.
__global__ void k_group_union(const uint32_t* __restrict__ tmask, int64_t words, int64_t ntiles,
                              int group, int chunk, int sg, int64_t n, uint32_t* __restrict__ gmask,
                              int32_t* __restrict__ gcnt, int32_t* __restrict__ sgmax,
                              int32_t* __restrict__ misc, unsigned long long* counters) {
    __shared__ int red[kThreads / 32];
    const int64_t k = blockIdx.x;
    const int64_t t0 = k * group;
    const int64_t t1 = t0 + group < ntiles ? t0 + group : ntiles;
    int cnt = 0;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
        uint32_t m = 0;
        for (int64_t t = t0; t < t1; ++t) m |= tmask[t * words + w];
        gmask[k * words + w] = m;
        cnt += __popc(m);
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0 && k == 0) misc[2] = static_cast<int32_t>(n);   // the merge's count
    if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) c += red[i];
        gcnt[k] = c;
        atomicMax(sgmax + k / sg, (c + chunk - 1) / chunk);    // chunk rounds of the super-group
        atomicAdd(misc, c);
        atomicMax(misc + 1, c);
        const int64_t v0 = t0 * 128, v1 = t1 * 128 < n ? t1 * 128 : n;
        atomicAdd(counters + CNT_DIST, static_cast<unsigned long long>(c) * 128ull *
                                           static_cast<unsigned long long>(v1 - v0));
    }
}

// Work units of each super-group of sg groups: chunk rounds x groups x unit slots per group.
__global__ void k_sg_units(const int32_t* __restrict__ sgmax, int64_t nsg, int64_t ngroups,
                           int sg, int ppg, int32_t* __restrict__ ucnt) {
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= nsg) return;
    const int64_t ng = ngroups - q * sg < sg ? ngroups - q * sg : sg;
    ucnt[q] = sgmax[q] * static_cast<int32_t>(ng) * ppg;
}

// One warp per group: the set bits of its mask, in increasing block order, written to
// blist[tfirst[g] ...].
__global__ void k_tile_list(const uint32_t* __restrict__ tmask, int64_t words, int64_t ntiles,
                            const int32_t* __restrict__ tfirst, int32_t* __restrict__ blist) {
    const int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ntiles) return;
    int64_t off = tfirst[g];
    for (int64_t base = 0; base < words; base += 32) {
        const int64_t w = base + lane;
        uint32_t m = (w < words) ? tmask[g * words + w] : 0u;
        const int c = __popc(m);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int64_t pos = off + incl - c;
        while (m) {
            const int bit = __ffs(m) - 1;
            blist[pos++] = static_cast<int32_t>(w * 32 + bit);
            m &= m - 1;
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
}

}  // namespace

void ttc_free(TreeTC* t) {
    if (!t) return;
    void* ptrs[] = {t->perm, t->op,   t->op3,   t->cidx,  t->cop3, t->radius, t->zc3,
                    t->cs,   t->znorm, t->cmarg, t->keep, t->key,  t->val,    t->skey,
                    t->vorder, t->tmp, t->tmask, t->gmask, t->tcnt, t->tfirst, t->sgmax,
                    t->ucnt, t->uoff, t->blist, t->misc, t->part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete t;
}

// Depth-first operands, centres and block balls of the dictionary's cover tree.
mrf_status ttc_build(mrf_dict* D, cudaStream_t st) {
    if (!D->tree) {
        mrf_set_error("the tensor-core tree search needs the cover tree (build_tree)");
        return MRF_EINVAL;
    }
    if (!D->bop && !D->bop3) {
        mrf_set_error("the tensor-core tree search needs the BF16 or the split-BF16 operand");
        return MRF_EINVAL;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int32_t> order;
    MRF_TRY(ct_dfs_order(D, &order));
    TreeTC* t = new TreeTC();
    auto bail = [&](mrf_status s) {
        ttc_free(t);
        return s;
    };
    t->metric = ct_metric(D);
    t->nblk = D->nblk;
    t->words = (t->nblk + 31) / 32;
    if (t->words * 4 > 48 * 1024) {        // block masks are OR-ed in shared memory
        delete t;
        mrf_set_error("tree search: more than 1.5M blocks of 128 atoms");
        return MRF_EUNSUPPORTED;
    }
    const int64_t npos = t->nblk * 128;
    std::vector<int32_t> perm(static_cast<size_t>(npos), -1);
    std::copy(order.begin(), order.end(), perm.begin());
    mrf_status s;
    if ((s = talloc(&t->perm, static_cast<size_t>(npos))) != MRF_OK) return bail(s);
    cudaError_t e = cudaMemcpyAsync(t->perm, perm.data(), npos * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        mrf_set_error(std::string("tree search upload: ") + cudaGetErrorString(e));
        return bail(MRF_ECUDA);
    }
    const int64_t Kp = D->Kp, Kp3 = 3 * D->Kp;
    if (D->bop) {
        if ((s = talloc(&t->op, static_cast<size_t>(t->nblk * 256 * Kp))) != MRF_OK) return bail(s);
        if ((s = launch_pack_bop_perm(D, t->op, t->perm, st)) != MRF_OK) return bail(s);
    }
    if (D->bop3) {
        if ((s = talloc(&t->op3, static_cast<size_t>(t->nblk * 256 * Kp3))) != MRF_OK) return bail(s);
        if ((s = launch_pack_sel3(D, t->perm, npos, t->nblk, t->op3, &t->op3_al, &t->op3_ae, st)) !=
            MRF_OK)
            return bail(s);
    }
    t->ncb = t->nblk;
    t->ncbblk = (t->ncb + 127) / 128;
    std::vector<int32_t> cidx(static_cast<size_t>(t->ncb));
    for (int64_t b = 0; b < t->ncb; ++b) cidx[b] = perm[b * 128];
    if ((s = talloc(&t->cidx, static_cast<size_t>(t->ncb))) != MRF_OK) return bail(s);
    e = cudaMemcpyAsync(t->cidx, cidx.data(), t->ncb * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        mrf_set_error(std::string("tree search upload: ") + cudaGetErrorString(e));
        return bail(MRF_ECUDA);
    }
    if ((s = talloc(&t->cop3, static_cast<size_t>(t->ncbblk * 256 * Kp3))) != MRF_OK) return bail(s);
    if ((s = launch_pack_sel3(D, t->cidx, t->ncb, t->ncbblk, t->cop3, &t->c_al, &t->c_ae, st)) !=
        MRF_OK)
        return bail(s);
    if ((s = talloc(&t->radius, static_cast<size_t>(t->nblk))) != MRF_OK) return bail(s);
    e = cudaMemsetAsync(t->radius, 0, t->nblk * sizeof(float), st);
    if (e == cudaSuccess) {
        k_block_radius<<<grid_for(npos * 32), kThreads, 0, st>>>(
            D->atoms, D->norm2, t->perm, npos, D->L, t->metric,
            reinterpret_cast<unsigned int*>(t->radius));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        mrf_set_error(std::string("tree search balls: ") + cudaGetErrorString(e));
        return bail(MRF_ECUDA);
    }
    t->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
    D->ttc = t;
    return MRF_OK;
}

bool ttc_has_split(const mrf_dict* D) { return D->ttc && D->ttc->op3; }
bool ttc_has_bf16(const mrf_dict* D) { return D->ttc && D->ttc->op; }

mrf_status ttc_blocks(const mrf_dict* D, int64_t* nblk, float* radius_host, int32_t* perm_host) {
    const TreeTC* t = D->ttc;
    if (!t) {
        mrf_set_error("dictionary built without the tensor-core tree search (tree_tc)");
        return MRF_EUNSUPPORTED;
    }
    if (nblk) *nblk = t->nblk;
    if (radius_host)
        MRF_CUDA_TRY(cudaMemcpy(radius_host, t->radius, t->nblk * sizeof(float),
                                cudaMemcpyDeviceToHost));
    if (perm_host)
        MRF_CUDA_TRY(cudaMemcpy(perm_host, t->perm, t->nblk * 128 * sizeof(int32_t),
                                cudaMemcpyDeviceToHost));
    return MRF_OK;
}

namespace {

// per-projection scratch for n voxels
mrf_status ttc_scratch(TreeTC* t, const mrf_dict* D, int64_t n) {
    if (n <= t->cap) return MRF_OK;
    t->cap = 0;
    const int64_t Kp3 = 3 * D->Kp;
    const int64_t ld = t->ncbblk * 256;
    // centre product in row chunks of at most ~512 MB of rows and correlations
    const int64_t per_row = ld * 4 + Kp3 * 2;
    int64_t crows = ((int64_t{1} << 29) / per_row) / 128 * 128;
    crows = std::max<int64_t>(crows, 128);
    crows = std::min<int64_t>(crows, (n + 127) / 128 * 128);
    t->crows = crows;
    const int64_t tiles = (n + 127) / 128;
    MRF_TRY(talloc(&t->zc3, static_cast<size_t>(crows * Kp3)));
    MRF_TRY(talloc(&t->cs, static_cast<size_t>(crows * ld)));
    MRF_TRY(talloc(&t->znorm, static_cast<size_t>(crows)));
    MRF_TRY(talloc(&t->cmarg, static_cast<size_t>(crows)));
    MRF_TRY(talloc(&t->keep, static_cast<size_t>(n * t->words)));
    MRF_TRY(talloc(&t->key, static_cast<size_t>(n)));
    MRF_TRY(talloc(&t->val, static_cast<size_t>(n)));
    MRF_TRY(talloc(&t->skey, static_cast<size_t>(n)));
    MRF_TRY(talloc(&t->vorder, static_cast<size_t>(n)));
    MRF_TRY(talloc(&t->tmask, static_cast<size_t>(tiles * t->words)));
    MRF_TRY(talloc(&t->gmask, static_cast<size_t>(tiles * t->words)));
    MRF_TRY(talloc(&t->tcnt, static_cast<size_t>(tiles + 1)));
    MRF_TRY(talloc(&t->tfirst, static_cast<size_t>(tiles + 1)));
    MRF_TRY(talloc(&t->sgmax, static_cast<size_t>(tiles + 1)));
    MRF_TRY(talloc(&t->ucnt, static_cast<size_t>(tiles + 1)));
    MRF_TRY(talloc(&t->uoff, static_cast<size_t>(tiles + 1)));
    MRF_TRY(talloc(&t->blist, static_cast<size_t>(tiles * t->nblk)));
    MRF_TRY(talloc(&t->misc, 4));
    size_t b1 = 0, b2 = 0;
    MRF_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, b1, t->key, t->skey, t->val, t->vorder,
                                                 static_cast<int>(n)));
    MRF_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, b2, t->tcnt, t->tfirst,
                                               static_cast<int>(tiles + 1)));
    t->tmp_bytes = std::max(b1, b2);
    unsigned char* tmp = nullptr;
    MRF_TRY(talloc(&tmp, t->tmp_bytes));
    if (t->tmp) cudaFree(t->tmp);
    t->tmp = tmp;
    t->tiles_cap = tiles;
    t->blist_cap = tiles * t->nblk;
    t->cap = n;
    return MRF_OK;
}

mrf_status ttc_part(TreeTC* t, size_t need) {
    if (need <= t->part_bytes) return MRF_OK;
    unsigned char* p = static_cast<unsigned char*>(t->part);
    t->part = nullptr;
    t->part_bytes = 0;
    MRF_TRY(talloc(&p, need));
    t->part = p;
    t->part_bytes = need;
    return MRF_OK;
}

}  // namespace

// Steps 1-4 of the tree search for Z [n][L] (device): fills `out` with the candidate lists
// ([S][n][K] scores then atom indices, rows in tile order), the tile order itself (voxel of each
// row) and a device count of the rows (= n) for the merge.
// split: search the split-BF16 operand (rows packed with the per-voxel bound plus `extra` into
// D->zmarg, indexed by voxel); else the BF16 operand (rows in D->zq).  Asynchronous on `st`.
mrf_status ttc_search(mrf_dict* D, const float2* Z, int64_t n, int cone, float eps, bool split,
                      int K, float extra, TtcOut* out, cudaStream_t st) {
    TreeTC* t = D->ttc;
    if (!t) {
        mrf_set_error("dictionary built without the tensor-core tree search (tree_tc)");
        return MRF_EUNSUPPORTED;
    }
    if (split ? !t->op3 : !t->op) {
        mrf_set_error(split ? "tree search: no split-BF16 operand (pack_bf16x3)"
                            : "tree search: no BF16 operand (pack_bf16)");
        return MRF_EUNSUPPORTED;
    }
    if (n > INT32_MAX) {
        mrf_set_error("tree search: more than 2^31 - 1 voxels");
        return MRF_EINVAL;
    }
    MRF_TRY(ttc_scratch(t, D, n));
    const int L = D->L;
    const int Kp = D->Kp;
    const int64_t ld = t->ncbblk * 256;
    // relative bound of the FP32 norm: (2 ceil(Kp / 64) + 5) roundings of a sum of non-negative
    // terms, a correctly rounded square root, with room
    const int m = 2 * ((Kp / 2 + 31) / 32) + 5;
    const float kappa = static_cast<float>((m + 8) * std::ldexp(1.0, -24));
    const float inv1e = std::nextafter(static_cast<float>(1.0 / (1.0 + static_cast<double>(eps))),
                                       2.f);
    int cbits = 1;
    while ((int64_t{1} << cbits) <= t->ncb) ++cbits;
    for (int64_t r0 = 0; r0 < n; r0 += t->crows) {
        {
            ProfScope ps(7, 3, st);   // query split, centre product, bounds
            const int64_t rows = std::min<int64_t>(t->crows, n - r0);
            MRF_TRY(launch_pack_queries_x3_with(Z + r0 * L, rows, L, Kp, t->c_al, t->c_ae,
                                                std::ldexp(1.f, -22), t->zc3, t->cmarg, st,
                                                nullptr, t->znorm));
            MRF_TRY(launch_dense(t->zc3, static_cast<int>(rows), 3 * Kp, t->cop3,
                                 static_cast<int>(ld), nullptr, 0, t->cs, nullptr, D->err, st));
            k_tree_bounds<<<grid_for(rows * 32), kThreads, 0, st>>>(
                t->cs, ld, rows, r0, t->znorm, t->cmarg, kappa, t->radius, t->ncb, t->words,
                t->metric, inv1e, cbits, t->keep, t->key, t->val);
            MRF_CUDA_TRY(cudaGetLastError());
        }
    }
    const int64_t tiles = (n + 127) / 128;
    // tiles sharing one block list: the units of a group stream the same blocks of a split
    // together, so L2 serves the repeats (with one list per tile they drift apart and stream
    // from DRAM); a few tiles keep most of the per-voxel pruning
    // tile shape: CTA pairs (256 voxels, each CTA staging half of every block, a 6-stage ring)
    // for the BF16 operand, whose lists stream from DRAM; single CTAs for the split operand,
    // where the three-times-longer blocks already give each load more products to cover it
    const bool pair = D->tune.bf16_pair == 1 || (D->tune.bf16_pair == 0 && !split);
    int group = D->tune.tree_tc_group > 0 ? D->tune.tree_tc_group
                                          : (split ? kGroupSplit : kGroupBf16);
    if (pair && (group % 2)) ++group;          // a CTA pair takes two tiles of one group
    const int64_t groups = (tiles + group - 1) / group;
    const int tpu = pair ? 2 : 1;
    // super-groups: neighbouring groups whose units run chunk round by chunk round together
    const int sg = D->tune.tree_tc_super > 0 ? D->tune.tree_tc_super : kSuper;
    const int64_t nsg = (groups + sg - 1) / sg;
    // a group's list in chunks of equal length (a fixed fraction of the dictionary), the work
    // units of the persistent search: equal units keep its CTAs balanced whatever the lists'
    // lengths
    const int nch = D->tune.tree_tc_chunks > 0 ? D->tune.tree_tc_chunks : kChunks;
    const int chunk = static_cast<int>((t->nblk + nch - 1) / nch);
    const int S = static_cast<int>((t->nblk + chunk - 1) / chunk);
    {
        // sort (histogram, bin scan, two digit passes), row packing, two unions, two scans (two
        // launches each), lists
        ProfScope ps(7, 12, st);
        size_t tb = t->tmp_bytes;
        MRF_CUDA_TRY(cub::DeviceRadixSort::SortPairs(t->tmp, tb, t->key, t->skey, t->val,
                                                     t->vorder, static_cast<int>(n), 0,
                                                     cbits + 4, st));
        if (split)
            MRF_TRY(launch_pack_queries_x3_with(Z, n, L, Kp, t->op3_al, t->op3_ae, extra, D->zq3,
                                                D->zmarg, st, t->vorder, nullptr));
        else
            MRF_TRY(launch_pack_gather(Z, t->vorder, n, L, Kp, D->zq, st));
        MRF_CUDA_TRY(cudaMemsetAsync(t->misc, 0, 4 * sizeof(int32_t), st));
        MRF_CUDA_TRY(cudaMemsetAsync(t->tcnt + groups, 0, sizeof(int32_t), st));
        MRF_CUDA_TRY(cudaMemsetAsync(t->sgmax, 0, (nsg + 1) * sizeof(int32_t), st));
        MRF_CUDA_TRY(cudaMemsetAsync(t->ucnt + nsg, 0, sizeof(int32_t), st));
        k_tile_union<<<static_cast<unsigned>(tiles), kThreads, t->words * sizeof(uint32_t), st>>>(
            t->keep, t->words, t->vorder, n, t->tmask);
        MRF_CUDA_TRY(cudaGetLastError());
        k_group_union<<<static_cast<unsigned>(groups), kThreads, 0, st>>>(
            t->tmask, t->words, tiles, group, chunk, sg, n, t->gmask, t->tcnt, t->sgmax, t->misc,
            D->counters);
        MRF_CUDA_TRY(cudaGetLastError());
        k_sg_units<<<grid_for(nsg), kThreads, 0, st>>>(t->sgmax, nsg, groups, sg,
                                                       (group + tpu - 1) / tpu, t->ucnt);
        MRF_CUDA_TRY(cudaGetLastError());
        tb = t->tmp_bytes;
        MRF_CUDA_TRY(cub::DeviceScan::ExclusiveSum(t->tmp, tb, t->tcnt, t->tfirst,
                                                   static_cast<int>(groups + 1), st));
        tb = t->tmp_bytes;
        MRF_CUDA_TRY(cub::DeviceScan::ExclusiveSum(t->tmp, tb, t->ucnt, t->uoff,
                                                   static_cast<int>(nsg + 1), st));
        k_tile_list<<<grid_for(groups * 32), kThreads, 0, st>>>(t->gmask, t->words, groups,
                                                                t->tfirst, t->blist);
        MRF_CUDA_TRY(cudaGetLastError());
    }
    const size_t pn = static_cast<size_t>(S) * n * K;
    MRF_TRY(ttc_part(t, pn * (sizeof(float) + sizeof(int32_t))));
    float* ps = static_cast<float*>(t->part);
    int32_t* pi = reinterpret_cast<int32_t*>(ps + pn);
    // slots of chunks a group does not have are not written: they read as empty (index -1,
    // NaN score)
    MRF_CUDA_TRY(cudaMemsetAsync(t->part, 0xff, pn * (sizeof(float) + sizeof(int32_t)), st));
    {
        ProfScope ps2(2, 1, st);
        MRF_TRY(launch_bf16_topk_list(split ? D->zq3 : D->zq, n, D, split ? t->op3 : t->op,
                                      split ? 3 * Kp : Kp, cone, K, group, chunk, sg, pair,
                                      t->tfirst, t->blist, t->uoff, t->perm, ps, pi, st));
    }
    out->S = S;
    out->part_s = ps;
    out->part_i = pi;
    out->vorder = t->vorder;
    out->count = t->misc + 2;
    out->tiles = tiles;
    return MRF_OK;
}
