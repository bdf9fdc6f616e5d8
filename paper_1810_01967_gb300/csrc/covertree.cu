// Cover-tree (1+eps)-approximate nearest-neighbour projection on the GPU (§4.1 Algorithm 1;
// §4.3 eq. ANN1 and Algorithm 2: the search runs on Z_v / ||Z_v||, warm-started at the previous
// atom).
//
// One warp per voxel; the children a level adds are evaluated eight at a time (one pass over
// the frames with eight independent accumulations per lane).  The tree lives flat in HBM: unit atoms in BFS order (the children of a
// node at a level are contiguous rows), and per node a CSR list of its "explicit" levels -- the
// levels at which it has children other than itself -- with the children's position range and
// the exact maxdist of the node at that level.  The candidate sets Q_i of Algorithm 1 are two
// ping-pong lists in shared memory (position, distance, cursor into the node's explicit levels,
// maxdist at the next level).  Per level: expand (self child carried, new children evaluated),
// update (q_c, dist_min), refine with dist <= dist_min + maxdist.  A voxel whose list has grown
// past 64 entries while dist_min still exceeds `route` -- a far query, for which the refinement
// keeps almost the whole net -- or whose list would exceed its capacity is handed to the
// exhaustive search; so is, before any traversal, a warm-started voxel whose warm atom is
// already farther than `route`.  The 8 best atoms seen go to the merge
// kernel, which rescores them exactly and computes the density.
//
// Query batching (the paper's closing remark on inter-voxel correlation in a query batch):
// warm-started queries are taken in the order of their warm atom's position in the tree, so
// the warps of a CTA and of neighbouring CTAs traverse the same subtrees and find the nodes'
// atoms in L1/L2; each query still runs its own Algorithm 1, so results do not change.
//
// Distances: d(u, z) = min_phi ||z^ - e^{i phi} u|| for the complex cone (Euclidean for the real
// cone), both unit vectors.  The first pass computes c = u^H z^ in FP32; when c is close to 1
// (d < 0.2) a second pass evaluates ||z^ - w u|| with w = c / |c| directly, which keeps the
// relative accuracy of small distances that 2 - 2|c| loses to cancellation.
#include <algorithm>
#include <chrono>
#include <initializer_list>

#include <cub/cub.cuh>

#include "mrf_internal.cuh"
#include "covertree_host.h"

struct CoverTreeDev {
    CtTree host;                 // host copy (export, info)
    float2* tatoms = nullptr;    // [nt][L]
    int32_t* rep = nullptr;      // [d]
    int32_t* pos = nullptr;      // [d]
    int32_t* order = nullptr;    // [nt]
    int32_t* node_first = nullptr;   // [nt + 1]
    int32_t* en_level = nullptr;
    int32_t* en_cb = nullptr;
    int32_t* en_ce = nullptr;
    float* en_maxdist = nullptr;
    int64_t nt = 0, ne = 0;
    double build_ms = 0.0;
    // query ordering scratch (grown on demand): sort keys and voxel indices, in and out
    int32_t* okey = nullptr;
    int32_t* oval = nullptr;
    void* otmp = nullptr;
    size_t otmp_bytes = 0;
    int64_t ocap = 0;
};

namespace {

constexpr int CAP = 256;          // longest default candidate list per warp (mrf_tune.tree_list_cap
                                  // overrides); shorter lists when L is long, see default_cap
constexpr int WARPS = 4;          // warps (queries) per CTA
constexpr int TOPC = 8;           // candidates handed to the merge
constexpr int kRouteList = 64;    // list size from which far queries are routed away
constexpr int kBatch = 8;         // candidate distances evaluated together
constexpr int kDefaultOrder = 1;  // mrf_tune.tree_order when 0: warm-started queries in tree order

struct TreeArgs {
    const float2* tatoms;
    const int32_t* rep;
    const int32_t* pos;
    const int32_t* order;
    const int32_t* node_first;
    const int32_t* en_level;
    const int32_t* en_cb;
    const int32_t* en_ce;
    const float* en_maxdist;
    int64_t d;
    int imax;
    float sigma;
    int metric;
};

struct Entry {
    int32_t pos;
    float dist;
    int32_t cur;
    float md;
};

__device__ __forceinline__ float warp_sum(float x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Distance from the unit query q (shared memory) to the unit atom at `p`; also returns the
// correlation used to rank candidates (|u^H z^| or Re(u^H z^)).
__device__ __forceinline__ float tree_dist(const TreeArgs& T, const float2* q, int L, int32_t p,
                                           int lane, float* corr) {
    const float2* u = T.tatoms + static_cast<int64_t>(p) * L;
    float re = 0.f, im = 0.f;
    for (int t = lane; t < L; t += 32) {
        const float2 a = u[t], z = q[t];
        re = fmaf(a.x, z.x, fmaf(a.y, z.y, re));
        im = fmaf(a.x, z.y, fmaf(-a.y, z.x, im));
    }
    re = warp_sum(re);
    im = warp_sum(im);
    float c, wr, wi;
    if (T.metric == 0) {
        c = sqrtf(re * re + im * im);
        wr = c > 0.f ? re / c : 1.f;
        wi = c > 0.f ? im / c : 0.f;
    } else {
        c = re;
        wr = 1.f;
        wi = 0.f;
    }
    *corr = c;
    float d2 = fmaxf(0.f, 2.f - 2.f * c);
    if (d2 < 0.04f) {   // accurate small distances: ||z^ - w u||^2
        float s = 0.f;
        for (int t = lane; t < L; t += 32) {
            const float2 a = u[t], z = q[t];
            const float xr = z.x - (wr * a.x - wi * a.y);
            const float xi = z.y - (wr * a.y + wi * a.x);
            s = fmaf(xr, xr, fmaf(xi, xi, s));
        }
        d2 = warp_sum(s);
    }
    return sqrtf(d2);
}

// The same distances for up to B candidates at once: one pass over the frames with B
// independent accumulations per lane (B unconditional loads in flight; slots past nb alias the
// first candidate's row), then one accurate second pass shared by the close candidates.  nb
// (<= B) is uniform across the warp.
template <int B>
__device__ __forceinline__ void tree_dist_batch(const TreeArgs& T, const float2* q, int L,
                                                const int32_t (&pos)[B], int nb, int lane,
                                                float (&dist)[B], float (&corr)[B]) {
    float re[B], im[B];
    const float2* u[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        re[b] = 0.f;
        im[b] = 0.f;
        u[b] = T.tatoms + static_cast<int64_t>(b < nb ? pos[b] : pos[0]) * L;
    }
#pragma unroll 2
    for (int t = lane; t < L; t += 32) {
        const float2 z = q[t];
        float2 a[B];
#pragma unroll
        for (int b = 0; b < B; ++b) a[b] = u[b][t];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            re[b] = fmaf(a[b].x, z.x, fmaf(a[b].y, z.y, re[b]));
            im[b] = fmaf(a[b].x, z.y, fmaf(-a[b].y, z.x, im[b]));
        }
    }
    float wr[B], wi[B];
    unsigned close = 0;          // candidates that need the accurate distance (warp-uniform)
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const float r = warp_sum(re[b]);
        const float m = warp_sum(im[b]);
        float c;
        if (T.metric == 0) {
            c = sqrtf(r * r + m * m);
            wr[b] = c > 0.f ? r / c : 1.f;
            wi[b] = c > 0.f ? m / c : 0.f;
        } else {
            c = r;
            wr[b] = 1.f;
            wi[b] = 0.f;
        }
        corr[b] = c;
        const float d2 = fmaxf(0.f, 2.f - 2.f * c);
        dist[b] = d2;
        if (b < nb && d2 < 0.04f) close |= 1u << b;
    }
    if (close) {                 // accurate small distances: ||z^ - w u||^2
        float sacc[B];
#pragma unroll
        for (int b = 0; b < B; ++b) sacc[b] = 0.f;
#pragma unroll 2
        for (int t = lane; t < L; t += 32) {
            const float2 z = q[t];
            float2 a[B];
#pragma unroll
            for (int b = 0; b < B; ++b) a[b] = u[b][t];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float xr = z.x - (wr[b] * a[b].x - wi[b] * a[b].y);
                const float xi = z.y - (wr[b] * a[b].y + wi[b] * a[b].x);
                sacc[b] = fmaf(xr, xr, fmaf(xi, xi, sacc[b]));
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float s2 = warp_sum(sacc[b]);
            if (close & (1u << b)) dist[b] = s2;
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) dist[b] = sqrtf(dist[b]);
}

__device__ __forceinline__ void top_insert(float (&cs)[TOPC], int32_t (&ci)[TOPC], float c,
                                           int32_t a) {
    if (c > cs[TOPC - 1]) {
        cs[TOPC - 1] = c;
        ci[TOPC - 1] = a;
#pragma unroll
        for (int k = TOPC - 1; k > 0; --k) {
            const bool up = cs[k] > cs[k - 1];
            const float x = cs[k], y = cs[k - 1];
            const int32_t ix = ci[k], iy = ci[k - 1];
            cs[k - 1] = up ? x : y;
            cs[k] = up ? y : x;
            ci[k - 1] = up ? ix : iy;
            ci[k] = up ? iy : ix;
        }
    }
}

// Sort keys of the query ordering: the tree position of each query's warm-start atom (queries
// without a valid one last, key = `none`, one past the last position), and the identity
// permutation to be sorted along.
__global__ void k_order_keys(const int32_t* __restrict__ warm, int64_t n, TreeArgs T,
                             int32_t none, int32_t* __restrict__ key, int32_t* __restrict__ val) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t a = warm[k];
    key[k] = (a >= 0 && a < T.d) ? T.pos[T.rep[a]] : none;
    val[k] = static_cast<int32_t>(k);
}

// One warp per query; warp k of the grid takes voxel order[k] (voxel k without an order).
__global__ void __launch_bounds__(WARPS * 32)
k_ct_search(const float2* __restrict__ Z, int64_t n, int L, TreeArgs T, int cap,
            const int32_t* __restrict__ warm, const int32_t* __restrict__ order, float eps,
            float route, float* __restrict__ part_s,
            int32_t* __restrict__ part_i, int32_t* __restrict__ fb_list,
            int32_t* __restrict__ fb_n, unsigned long long* cnt) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t kq = static_cast<int64_t>(blockIdx.x) * WARPS + w;
    const size_t per_warp = static_cast<size_t>(L) * sizeof(float2) + 2 * cap * sizeof(Entry);
    unsigned char* mine = smem + per_warp * w;
    float2* q = reinterpret_cast<float2*>(mine);
    Entry* QA = reinterpret_cast<Entry*>(mine + static_cast<size_t>(L) * sizeof(float2));
    Entry* QB = QA + cap;
    if (kq >= n) return;
    const int64_t v = order ? static_cast<int64_t>(order[kq]) : kq;
    // unit query
    const float2* z = Z + v * L;
    float s = 0.f;
    for (int t = lane; t < L; t += 32) { const float2 a = z[t]; s = fmaf(a.x, a.x, fmaf(a.y, a.y, s)); }
    s = warp_sum(s);
    float cs[TOPC];
    int32_t ci[TOPC];
#pragma unroll
    for (int k = 0; k < TOPC; ++k) { cs[k] = -INFINITY; ci[k] = -1; }
    if (s == 0.f) {   // zero query: any candidate; the merge returns (0, 0)
        if (lane < TOPC) {
            part_s[v * TOPC + lane] = lane == 0 ? 0.f : -INFINITY;
            part_i[v * TOPC + lane] = lane == 0 ? 0 : -1;
        }
        return;
    }
    const float inv = rsqrtf(s);
    for (int t = lane; t < L; t += 32) { const float2 a = z[t]; q[t] = make_float2(a.x * inv, a.y * inv); }
    __syncwarp();
    unsigned long long evals = 0;
    float corr;
    // initialisation: the root (position 0) and the warm start are evaluated
    const float droot = tree_dist(T, q, L, 0, lane, &corr);
    ++evals;
    top_insert(cs, ci, corr, T.order[0]);
    float dmin = droot;
    if (warm) {
        const int32_t a = warm[v];
        if (a >= 0 && a < T.d) {
            const int32_t p = T.pos[T.rep[a]];
            if (p > 0) {
                const float dw = tree_dist(T, q, L, p, lane, &corr);
                ++evals;
                top_insert(cs, ci, corr, T.order[p]);
                dmin = fminf(dmin, dw);
            }
        }
    }
    bool overflow = false;
    // a warm-started query whose warm atom is already farther than `route` goes to the
    // exhaustive search before the traversal (unless the stop rule would end the search at the
    // first level): such a query would be routed after building its lists anyway
    if (warm && dmin > route && (eps == 0.f || T.sigma * 2.f * (1.f + 1.f / eps) > dmin)) {
        const int32_t a = warm[v];
        if (a >= 0 && a < T.d) overflow = true;
    }
    Entry* Q = QA;
    Entry* N = QB;
    int nq = overflow ? 0 : 1;
    if (lane == 0) {
        const int32_t c0 = T.node_first[0];
        Q[0] = {0, droot, c0, (c0 < T.node_first[1]) ? T.en_maxdist[c0] : 0.f};
    }
    __syncwarp();
    const float inv_eps = eps > 0.f ? 1.f / eps : 0.f;
    for (int i = 0; i < T.imax && nq > 0; ++i) {
        if (eps > 0.f && T.sigma * exp2f(static_cast<float>(1 - i)) * (1.f + inv_eps) <= dmin) break;
        // expand: new children enter the list with their distance pending (< 0), the parents
        // carry theirs
        int nn = 0;
        for (int e = 0; e < nq && !overflow; ++e) {
            const Entry E = Q[e];
            int32_t cur = E.cur;
            const int32_t cend = T.node_first[E.pos + 1];
            if (cur < cend && T.en_level[cur] == i) {
                const int32_t cb = T.en_cb[cur], ce = T.en_ce[cur];
                for (int32_t c = cb; c < ce; ++c) {
                    if (nn >= cap) { overflow = true; break; }
                    const int32_t cc = T.node_first[c];
                    const float mdc = (cc < T.node_first[c + 1]) ? T.en_maxdist[cc] : 0.f;
                    if (lane == 0) N[nn] = {c, -1.f, cc, mdc};
                    ++nn;
                }
                ++cur;
            }
            if (overflow) break;
            if (nn >= cap) { overflow = true; break; }
            if (lane == 0) N[nn] = {E.pos, E.dist, cur, (cur < cend) ? T.en_maxdist[cur] : 0.f};
            ++nn;
        }
        __syncwarp();
        if (overflow) break;
        // distances of the new children, kBatch at a time
        for (int e0 = 0; e0 < nn;) {
            int32_t pos[kBatch], slot[kBatch];
            int nb = 0;
            while (e0 < nn && nb < kBatch) {
                if (N[e0].dist < 0.f) { slot[nb] = e0; pos[nb] = N[e0].pos; ++nb; }
                ++e0;
            }
            if (nb == 0) break;
            float db[kBatch], cb[kBatch];
            tree_dist_batch<kBatch>(T, q, L, pos, nb, lane, db, cb);
            evals += nb;
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                if (b < nb) {
                    top_insert(cs, ci, cb[b], T.order[pos[b]]);
                    if (lane == 0) N[slot[b]].dist = db[b];
                }
            }
        }
        __syncwarp();
        // nearest new candidate
        float bmin = INFINITY;
        for (int e = lane; e < nn; e += 32) bmin = fminf(bmin, N[e].dist);
        for (int o = 16; o; o >>= 1) bmin = fminf(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
        if (bmin < dmin) dmin = bmin;
        // far query: the list has grown and the nearest atom is still far -- the refinement
        // below would keep most of the net, so the exhaustive search takes this voxel
        // (with eps > 0 the stop rule of Algorithm 1 ends far searches itself: route only when it
        // will not fire at the next level)
        if (nn > kRouteList && dmin > route &&
            (eps == 0.f || T.sigma * exp2f(static_cast<float>(-i)) * (1.f + inv_eps) > dmin)) {
            overflow = true;
            break;
        }
        // refine: keep candidates that can still hold the nearest neighbour
        const float slack = 1e-5f + 1e-5f * dmin;
        int m = 0;
        for (int e0 = 0; e0 < nn; e0 += 32) {
            const int e = e0 + lane;
            Entry E;
            bool keep = false;
            if (e < nn) {
                E = N[e];
                keep = E.dist <= dmin + E.md + slack;
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (keep) Q[m + __popc(b & ((1u << lane) - 1u))] = E;
            m += __popc(b);
        }
        __syncwarp();
        nq = m;
        if (nq == 0) break;
    }
    if (overflow) {
        if (lane == 0) {
            const int p = atomicAdd(fb_n, 1);
            fb_list[p] = static_cast<int32_t>(v);
            atomicAdd(cnt + CNT_FALLBACK, 1ULL);
        }
    }
    if (lane == 0) atomicAdd(cnt + CNT_DIST, evals);
    if (lane < TOPC) {
        float sv = cs[0];
        int32_t iv = ci[0];
#pragma unroll
        for (int k = 1; k < TOPC; ++k)
            if (lane == k) { sv = cs[k]; iv = ci[k]; }
        part_s[v * TOPC + lane] = sv;
        part_i[v * TOPC + lane] = iv;
    }
}

// Default list capacity: the longest list (a multiple of 16, 64 .. CAP) with which four CTAs of
// WARPS queries fit in an SM's shared memory (224 KB after the per-block reservations), each
// query holding its unit query (L x 8 bytes) and two lists of 16-byte entries.  Residency
// decides the search's speed (it is latency-bound), the capacity how many voxels overflow to
// the exhaustive search: on the 256 x 256 x 1000 slice 192 entries (16 warps per SM) beat 256
// (12 warps) by 10 % over a whole CoverBLIP reconstruction despite 8 % more routed voxels.
int default_cap(int L) {
    const int per_warp = (229376 / 4) / WARPS;
    int cap = (per_warp - L * static_cast<int>(sizeof(float2))) / (2 * static_cast<int>(sizeof(Entry)));
    cap = (cap / 16) * 16;
    return cap < 64 ? 64 : (cap > CAP ? CAP : cap);
}

template <typename T>
mrf_status up(T** dst, const std::vector<T>& src) {
    if (src.empty()) { *dst = nullptr; return MRF_OK; }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mrf_set_error(std::string("cover tree upload: ") + cudaGetErrorString(e));
        return MRF_ENOMEM;
    }
    return MRF_OK;
}

}  // namespace

void ct_free(CoverTreeDev* t) {
    if (!t) return;
    void* ptrs[] = {t->tatoms, t->rep, t->pos, t->order, t->node_first, t->en_level,
                    t->en_cb, t->en_ce, t->en_maxdist, t->okey, t->oval, t->otmp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete t;
}

mrf_status ct_build_upload(mrf_dict* D, int metric, double dup_tol) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::complex<float>> host(static_cast<size_t>(D->d) * D->L);
    MRF_CUDA_TRY(cudaMemcpy(host.data(), D->atoms, host.size() * sizeof(float2),
                            cudaMemcpyDeviceToHost));
    CoverTreeDev* t = new CoverTreeDev();
    CtParams P;
    P.atoms = host.data();
    P.d = D->d;
    P.L = D->L;
    P.metric = metric;
    P.dup_tol = dup_tol;
    int rc = ct_build(P, &t->host);
    if (rc != 0) {
        delete t;
        mrf_set_error("cover tree construction failed (code " + std::to_string(rc) + ")");
        return MRF_EINTERNAL;
    }
    CtTree& h = t->host;
    t->nt = static_cast<int64_t>(h.order.size());
    t->ne = static_cast<int64_t>(h.en_level.size());
    std::vector<float2> ta(h.unit_atoms.size());
    for (size_t k = 0; k < ta.size(); ++k) ta[k] = make_float2(h.unit_atoms[k].real(), h.unit_atoms[k].imag());
    std::vector<int32_t> nf(h.node_first.begin(), h.node_first.end());
    mrf_status s = MRF_OK;
    if ((s = up(&t->tatoms, ta)) == MRF_OK && (s = up(&t->rep, h.rep)) == MRF_OK &&
        (s = up(&t->pos, h.pos)) == MRF_OK && (s = up(&t->order, h.order)) == MRF_OK &&
        (s = up(&t->node_first, nf)) == MRF_OK && (s = up(&t->en_level, h.en_level)) == MRF_OK &&
        (s = up(&t->en_cb, h.en_cb)) == MRF_OK && (s = up(&t->en_ce, h.en_ce)) == MRF_OK &&
        (s = up(&t->en_maxdist, h.en_maxdist)) == MRF_OK) {
        h.unit_atoms.clear();
        h.unit_atoms.shrink_to_fit();
        t->build_ms = std::chrono::duration<double, std::milli>(
                          std::chrono::steady_clock::now() - t0).count();
        if (D->tree) ct_free(D->tree);
        D->tree = t;
        return MRF_OK;
    }
    ct_free(t);
    return s;
}

mrf_status launch_ct_search(const float2* Z, int64_t n, const mrf_dict* D, int cone,
                            const int32_t* warm, float eps, float route, float* part_s,
                            int32_t* part_i, int32_t* fb_list, int32_t* fb_n, cudaStream_t st) {
    const CoverTreeDev* t = D->tree;
    if (!t) {
        mrf_set_error("dictionary built without a cover tree (mrf_index_opts.build_tree = 0)");
        return MRF_EUNSUPPORTED;
    }
    if ((cone == MRF_CONE_COMPLEX) != (t->host.metric == 0)) {
        mrf_set_error("the cover tree was built for the other cone (mrf_index_opts.tree_cone)");
        return MRF_EINVAL;
    }
    if (n == 0) return MRF_OK;
    TreeArgs T;
    T.tatoms = t->tatoms;
    T.rep = t->rep;
    T.pos = t->pos;
    T.order = t->order;
    T.node_first = t->node_first;
    T.en_level = t->en_level;
    T.en_cb = t->en_cb;
    T.en_ce = t->en_ce;
    T.en_maxdist = t->en_maxdist;
    T.d = D->d;
    T.imax = t->host.imax;
    T.sigma = static_cast<float>(t->host.sigma);
    T.metric = t->host.metric;
    const int cap = D->tune.tree_list_cap > 0 ? D->tune.tree_list_cap : default_cap(D->L);
    const size_t per_warp = static_cast<size_t>(D->L) * sizeof(float2) + 2 * cap * sizeof(Entry);
    const size_t sm = per_warp * WARPS;
    // query order: warm-started queries sorted by their warm atom's tree position
    const int32_t* order = nullptr;
    const int tord = D->tune.tree_order ? D->tune.tree_order : kDefaultOrder;
    if (warm && tord == 1 && n > 1) {
        CoverTreeDev* tm = D->tree;
        if (n > tm->ocap) {
            size_t need = 0;
            if (cub::DeviceRadixSort::SortPairs(nullptr, need, tm->okey, tm->okey, tm->oval,
                                                tm->oval, static_cast<int>(n)) != cudaSuccess) {
                mrf_set_error("query order: sort workspace query failed");
                return MRF_ECUDA;
            }
            for (void** p : {reinterpret_cast<void**>(&tm->okey), reinterpret_cast<void**>(&tm->oval),
                             &tm->otmp}) {
                if (*p) {
                    cudaFree(*p);
                    scratch_epoch_bump();
                }
                *p = nullptr;
            }
            tm->ocap = 0;
            MRF_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&tm->okey), sizeof(int32_t) * 2 * n));
            MRF_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&tm->oval), sizeof(int32_t) * 2 * n));
            MRF_CUDA_TRY(cudaMalloc(&tm->otmp, need));
            tm->otmp_bytes = need;
            tm->ocap = n;
        }
        int32_t* kin = tm->okey;
        int32_t* kout = tm->okey + n;
        int32_t* vin = tm->oval;
        int32_t* vout = tm->oval + n;
        const int32_t none = static_cast<int32_t>(tm->nt);
        k_order_keys<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(warm, n, T, none,
                                                                            kin, vin);
        MRF_CUDA_TRY(cudaGetLastError());
        size_t bytes = tm->otmp_bytes;
        int end_bit = 1;            // keys lie in [0, nt]
        while (end_bit < 31 && (int64_t{1} << end_bit) <= tm->nt) ++end_bit;
        if (cub::DeviceRadixSort::SortPairs(tm->otmp, bytes, kin, kout, vin, vout,
                                            static_cast<int>(n), 0, end_bit, st) != cudaSuccess) {
            mrf_set_error("query order: sort failed");
            return MRF_ECUDA;
        }
        order = vout;
    }
    cudaError_t e = cudaFuncSetAttribute(k_ct_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess) {
        k_ct_search<<<static_cast<unsigned>((n + WARPS - 1) / WARPS), WARPS * 32, sm, st>>>(
            Z, n, D->L, T, cap, warm, order, eps, route, part_s, part_i, fb_list, fb_n,
            D->counters);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("cover tree search launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

mrf_status ct_info(const mrf_dict* D, mrf_tree_info* info) {
    const CoverTreeDev* t = D->tree;
    if (!t) {
        mrf_set_error("dictionary has no cover tree");
        return MRF_EUNSUPPORTED;
    }
    info->nodes = t->nt;
    info->explicit_nodes = t->ne;
    info->levels = t->host.imax;
    info->metric = t->host.metric;
    info->sigma = t->host.sigma;
    info->build_ms = t->build_ms;
    info->device_bytes = t->nt * D->L * static_cast<int64_t>(sizeof(float2)) +
                         (3 * D->d + 2 * t->nt + 1) * static_cast<int64_t>(sizeof(int32_t)) +
                         t->ne * static_cast<int64_t>(3 * sizeof(int32_t) + sizeof(float));
    return MRF_OK;
}

mrf_status ct_export(const mrf_dict* D, int32_t* first_level, int32_t* parent, int32_t* rep,
                     int32_t* en_atom, int32_t* en_level, float* en_maxdist) {
    const CoverTreeDev* t = D->tree;
    if (!t) {
        mrf_set_error("dictionary has no cover tree");
        return MRF_EUNSUPPORTED;
    }
    const CtTree& h = t->host;
    for (int64_t a = 0; a < D->d; ++a) {
        if (first_level) first_level[a] = h.first_level[a];
        if (parent) parent[a] = h.parent[a];
        if (rep) rep[a] = h.rep[a];
    }
    for (int64_t e = 0; e < t->ne; ++e) {
        if (en_atom) en_atom[e] = h.en_parent[e];
        if (en_level) en_level[e] = h.en_level[e];
        if (en_maxdist) en_maxdist[e] = h.en_maxdist[e];
    }
    return MRF_OK;
}

extern "C" mrf_status mrf_tree_build_host(const void* atoms, int64_t d, int32_t L, int32_t cone,
                                          float dup_tol, int32_t* first_level, int32_t* parent,
                                          int32_t* rep, int32_t* en_atom, int32_t* en_level,
                                          float* en_maxdist, int64_t* n_explicit, double* sigma,
                                          int32_t* levels) {
    if (!atoms || d < 1 || L < 1 || L > 4096 || d > INT32_MAX) {
        mrf_set_error("mrf_tree_build_host: need atoms, 1 <= d, 1 <= L <= 4096");
        return MRF_EINVAL;
    }
    if ((cone != MRF_CONE_COMPLEX && cone != MRF_CONE_REAL_POS) || !(dup_tol >= 0.f)) {
        mrf_set_error("mrf_tree_build_host: bad cone or dup_tol");
        return MRF_EINVAL;
    }
    CtParams P;
    P.atoms = static_cast<const std::complex<float>*>(atoms);
    P.d = d;
    P.L = L;
    P.metric = cone == MRF_CONE_COMPLEX ? 0 : 1;
    P.dup_tol = dup_tol;
    CtTree T;
    if (ct_build(P, &T) != 0) {
        mrf_set_error("cover tree construction failed");
        return MRF_EINTERNAL;
    }
    for (int64_t a = 0; a < d; ++a) {
        if (first_level) first_level[a] = T.first_level[a];
        if (parent) parent[a] = T.parent[a];
        if (rep) rep[a] = T.rep[a];
    }
    const int64_t ne = static_cast<int64_t>(T.en_level.size());
    for (int64_t e = 0; e < ne; ++e) {
        if (en_atom) en_atom[e] = T.en_parent[e];
        if (en_level) en_level[e] = T.en_level[e];
        if (en_maxdist) en_maxdist[e] = T.en_maxdist[e];
    }
    if (n_explicit) *n_explicit = ne;
    if (sigma) *sigma = T.sigma;
    if (levels) *levels = T.imax;
    return MRF_OK;
}

// Depth-first (pre-order) order of the tree's atoms: a node, then its children (the atoms whose
// parent it is, by the level they first appear at, then by index), each subtree contiguous;
// duplicates, which are not tree nodes, right after their representative.  Consecutive positions are close
// in the tree metric, so 128-atom blocks of this order have small enclosing balls.
mrf_status ct_dfs_order(const mrf_dict* D, std::vector<int32_t>* out) {
    const CoverTreeDev* t = D->tree;
    if (!t) {
        mrf_set_error("dictionary built without a cover tree");
        return MRF_EUNSUPPORTED;
    }
    const CtTree& h = t->host;
    const int64_t d = D->d;
    std::vector<std::vector<int32_t>> kids(static_cast<size_t>(d));
    int32_t root = -1;
    for (int64_t j = 0; j < d; ++j) {
        if (h.first_level[j] < 0) continue;
        if (h.parent[j] < 0) root = static_cast<int32_t>(j);
        else kids[h.parent[j]].push_back(static_cast<int32_t>(j));
    }
    if (root < 0) {
        mrf_set_error("cover tree without a root");
        return MRF_EINTERNAL;
    }
    for (auto& k : kids)
        std::sort(k.begin(), k.end(), [&](int32_t a, int32_t b) {
            return h.first_level[a] != h.first_level[b] ? h.first_level[a] < h.first_level[b] : a < b;
        });
    // duplicates (atoms represented by an earlier node) follow their representative
    std::vector<std::vector<int32_t>> dups(static_cast<size_t>(d));
    for (int64_t j = 0; j < d; ++j)
        if (h.first_level[j] < 0 && h.rep[j] >= 0 && h.rep[j] != j)
            dups[h.rep[j]].push_back(static_cast<int32_t>(j));
    out->clear();
    out->reserve(static_cast<size_t>(d));
    std::vector<int32_t> stack{root};
    while (!stack.empty()) {
        const int32_t u = stack.back();
        stack.pop_back();
        out->push_back(u);
        for (int32_t j : dups[u]) out->push_back(j);
        for (auto it = kids[u].rbegin(); it != kids[u].rend(); ++it) stack.push_back(*it);
    }
    if (static_cast<int64_t>(out->size()) != d) {
        mrf_set_error("cover tree depth-first order does not cover the dictionary");
        return MRF_EINTERNAL;
    }
    return MRF_OK;
}

int ct_metric(const mrf_dict* D) { return D->tree ? D->tree->host.metric : -1; }
