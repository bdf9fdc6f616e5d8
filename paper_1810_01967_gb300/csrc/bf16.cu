// Exhaustive matched filter on the 5th-generation tensor cores (§3.2, eq. exactP): BF16 or FP8
// (E4M3) inputs with FP32 accumulation in tensor memory.
//
// The complex correlation D_j^H Z_v is a real GEMM: query row v = (Re z_0, Im z_0, Re z_1, ...)
// (K = 2L, padded to Kp), and per block of 128 atoms 256 operand rows: 128 rows
// (Re d_t, Im d_t)_t giving Re(D^H z) and 128 rows (-Im d_t, Re d_t)_t giving Im(D^H z).  One
// UMMA of shape M = 128 voxels x N = 256 columns therefore yields, for every voxel row, the real
// parts of 128 atoms in columns [0,128) and their imaginary parts in columns [128,256) of the
// same TMEM lane, so the epilogue thread that owns the row forms |c|^2 / ||D_j||^2 without any
// data exchange and keeps a sorted top-K in registers.  Scores never reach global memory.
//
// Clusters of C CTAs (default C = 1) work on C consecutive voxel tiles against the same atom
// blocks at the same time; every CTA loads its own copy of each atom block with a plain TMA
// tile load (no multicast), so the second and later reads of a block are L2 hits.  Persistent
// clusters walk work units (atom split s, voxel-tile group g); the unit order keeps a few dozen
// voxel tiles live at a time (super-groups of PG groups, all splits) so the query tiles being
// re-read stay resident in L2 while the atom blocks stream.
// Warp roles: warp 0 = TMA producer, warp 1 = TMEM owner and MMA issuer, warps 2..5 = epilogue
// (TMEM lanes 32 (w mod 4) ...).  4-stage shared-memory ring (48 KB per stage: A 128 rows and
// B 256 rows of 128 bytes = 64 BF16 or 128 E4M3 elements, 128-byte swizzle), double-buffered
// 2 x 256-column FP32 accumulator.  The FP8 form uses kind::f8f6f4 (K = 32 per instruction
// instead of 16, the same 32 bytes), per-row power-of-two scales folded into the atom weights
// and into a per-query factor applied to the K scores a voxel keeps.
// Every mbarrier wait is bounded; on expiry the CTA raises MRF_DERR_TIMEOUT, drains what it
// issued and exits.
#include <cuda.h>
#include "mrf_internal.cuh"
#include "ptx.cuh"
#include "tma_host.h"

namespace {

constexpr int BM = 128;
constexpr int BN = 256;          // 128 atoms x (re, im)
constexpr int BKB = 128;         // bytes per stage row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BKB;
constexpr int B_BYTES = BN * BKB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NTHREADS = 192;
constexpr uint32_t IDESC = mrfk::idesc_bf16(BM, BN);
constexpr uint32_t IDESC8 = mrfk::idesc_e4m3(BM, BN);

struct Shared {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort;
};

// Work-unit schedule shared by all roles.  Cluster unit uc -> (split s, group g); the voxel
// tile of CTA `rank` is g * C + rank.
struct Sched {
    int64_t NG;      // voxel-tile groups (ceil(Mt / C))
    int64_t S;       // atom splits
    int64_t PG;      // groups per super-group
    __device__ __forceinline__ void map(int64_t uc, int64_t& s, int64_t& g) const {
        const int64_t per_sg = PG * S;
        const int64_t sg = uc / per_sg;
        const int64_t l = uc - sg * per_sg;
        const int64_t g0 = sg * PG;
        const int64_t pe = min(PG, NG - g0);
        s = l / pe;
        g = g0 + (l - s * pe);
    }
};

// Block lists of the cover-tree search: the tiles of group k (tiles [k group, (k + 1) group))
// share the ascending block list blist[tfirst[k] .. tfirst[k + 1]), cut into chunks of `chunk`
// blocks.  Groups are gathered into super-groups of `sg` consecutive groups (similar lists:
// voxels are sorted by where they lie in the tree); super-group q owns the work units
// [uoff[q], uoff[q + 1]), numbered chunk by chunk -- chunk c of every group of q, then chunk c
// + 1 -- and within a chunk group by group, tile (or tile pair) by tile, so the CTAs running
// together scan the same part of neighbouring lists and L2 serves the blocks they share.  A
// super-group has as many chunk rounds as its longest list; units past a shorter list, or past
// a short last group's tiles, are empty.  *units = uoff[nsg]; perm maps operand positions to
// atoms.
struct ListArgs {
    const int32_t* tfirst;
    const int32_t* blist;
    const int32_t* perm;
    const int32_t* uoff;
    const int32_t* units;
    int group, chunk, sg;
    int tpu;                     // voxel tiles per unit: 1 (single CTA) or 2 (CTA pair)
    int64_t ngroups, nsg, ntiles;
};

// The work unit uc: tile g (tile pair g with CTA pairs), candidate slot s (its chunk),
// positions [b0, b1) of the group's list starting at lb (LIST); or the exhaustive schedule's
// unit: split s, tile group g, block range [b0, b1).  False when the unit has no block.
template <bool LIST>
__device__ __forceinline__ bool unit_of(const Sched& sc, const ListArgs& la, int64_t uc, int bps,
                                        int64_t nblk, int64_t& s, int64_t& g, int64_t& b0,
                                        int64_t& b1, int64_t& lb) {
    if (LIST) {
        int64_t lo = 0, hi = la.nsg;                     // last q with uoff[q] <= uc
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (la.uoff[mid] <= uc) lo = mid;
            else hi = mid;
        }
        const int64_t k0 = lo * la.sg;                    // first group of the super-group
        const int64_t ng = min(static_cast<int64_t>(la.sg), la.ngroups - k0);
        const int64_t ppg = (la.group + la.tpu - 1) / la.tpu;   // unit slots per group
        const int64_t l = uc - la.uoff[lo];
        const int64_t per = ng * ppg;                     // units per chunk round
        s = l / per;
        const int64_t r = l - s * per;
        const int64_t k = k0 + r / ppg;
        const int64_t pi = r - (r / ppg) * ppg;
        const int64_t t0 = k * la.group;
        const int64_t gsz = min(static_cast<int64_t>(la.group), la.ntiles - t0);
        g = t0 / la.tpu + pi;                             // tile (or tile pair) index
        if (pi * la.tpu >= gsz) { b0 = b1 = lb = 0; return false; }
        lb = la.tfirst[k];
        const int64_t cnt = la.tfirst[k + 1] - lb;
        b0 = s * la.chunk;
        b1 = min(b0 + la.chunk, cnt);
    } else {
        sc.map(uc, s, g);
        lb = 0;
        b0 = s * bps;
        b1 = min(b0 + bps, nblk);
    }
    return b0 < b1;
}

// Insert (s, j) into the descending list ts (ties keep the earlier entry first).  Every slot
// decides on its own from one comparison with s -- stay, take s, or take its upper neighbour
// -- so the KT steps carry no dependency chain: one warp per SM sub-partition runs this and
// nothing else would hide the latency of a compare-exchange bubble.
template <int KT>
__device__ __forceinline__ void topk_insert(float (&ts)[KT], int32_t (&ti)[KT], float s,
                                            int32_t j) {
    if (s > ts[KT - 1]) {
        bool ge[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) ge[q] = ts[q] >= s;
#pragma unroll
        for (int q = KT - 1; q > 0; --q) {
            ts[q] = ge[q] ? ts[q] : (ge[q - 1] ? s : ts[q - 1]);
            ti[q] = ge[q] ? ti[q] : (ge[q - 1] ? j : ti[q - 1]);
        }
        ts[0] = ge[0] ? ts[0] : s;
        ti[0] = ge[0] ? ti[0] : j;
    }
}

// One 128-atom block of the accumulator (TMEM columns tb .. tb + 255: real parts, then
// imaginary parts) into the thread's running top-KT: per 32-atom chunk the scores of the
// normalised atoms, their maximum against the K-th best, and only when it is beaten the slow
// path through the thread's shared-memory column `col` (stride BM floats).
template <int KT>
__device__ __forceinline__ void epilogue_block(uint32_t tb, int cone, int64_t b, int64_t d,
                                               float* col, float (&ts)[KT], int32_t (&ti)[KT]) {
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        uint32_t re[32], im[32];
        __syncwarp();
        mrfk::tmem_ld32(tb + c * 32, re);
        mrfk::tmem_ld32(tb + 128 + c * 32, im);
        mrfk::tmem_ld_wait();
        float mx = -INFINITY;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float x = __uint_as_float(re[i]);
            const float y = __uint_as_float(im[i]);
            const float v = (cone == MRF_CONE_COMPLEX) ? fmaf(x, x, y * y) : x;
            re[i] = __float_as_uint(v);
            mx = fmaxf(mx, v);
        }
        if (mx > ts[KT - 1]) {
            const float thr = ts[KT - 1];
            uint32_t hits = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float v = __uint_as_float(re[i]);
                col[i * BM] = v;
                hits |= (v > thr) ? (1u << i) : 0u;
            }
            const int64_t jb = b * 128 + c * 32;
            while (hits) {
                const int i = __ffs(hits) - 1;
                hits &= hits - 1;
                const int64_t j = jb + i;
                if (j < d) topk_insert<KT>(ts, ti, col[i * BM], static_cast<int32_t>(j));
            }
        }
    }
}

// F8: E4M3 operands (kind::f8f6f4); the K kept scores of voxel v are multiplied by
// (qs[v] gsc)^2 (complex cone) or qs[v] gsc (real cone), qs = 1 / (the query row's scale) and
// gsc = 1 / (the dictionary's scale).  BF16: scores are used as computed.
// LIST: the block-list mode of the cover-tree search -- unit (group, chunk s, voxel tile g) scans
// chunk s of the group's block list of an operand in the tree's depth-first order, and
// the kept candidates are mapped back to atom indices through la.perm.
template <int KT, int C, bool F8, bool LIST = false>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_topk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          int64_t n, int64_t d, int64_t nblk, int Kp, int cone, Sched sc, int blocks_per_split,
          float gsc, const float* __restrict__ qs, const int32_t* __restrict__ count,
          float* __restrict__ part_s, int32_t* __restrict__ part_i, uint32_t* err,
          ListArgs la) {
    constexpr int EK = F8 ? 128 : 64;     // elements per stage row
    constexpr int KPER = F8 ? 32 : 16;    // elements per MMA instruction (32 bytes either way)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    Shared* sh = reinterpret_cast<Shared*>(base + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = (C > 1) ? mrfk::cluster_ctarank() : 0u;
    const int64_t cluster = blockIdx.x / C;
    const int64_t nclusters = gridDim.x / C;
    const int64_t units = LIST ? static_cast<int64_t>(*la.units) : sc.NG * sc.S;
    // with a device-side voxel count (lists built on the device) the tiles past it are skipped
    const int64_t nact = count ? min(static_cast<int64_t>(*count), n) : n;
    const int nk = (Kp + EK - 1) / EK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
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
        mrfk::tmem_alloc(&sh->tmem_base, 512);
        mrfk::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        mrfk::tma_prefetch_desc(&tmA);
        mrfk::tma_prefetch_desc(&tmB);
    }
    mrfk::tc_fence_before();
    if (C > 1) mrfk::cluster_sync(); else __syncthreads();
    mrfk::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    auto fail = [&]() {
        atomicOr(err, MRF_DERR_TIMEOUT);
        sh->abort = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t slot_phase[STAGES];
            bool slot_used[STAGES];
            for (int i = 0; i < STAGES; ++i) { slot_used[i] = false; slot_phase[i] = 0; }
            for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
                int64_t s, g, b0, b1, lb;
                const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
                if (g * C * BM >= nact) continue;     // the cluster's tiles are all past the count
                const int64_t m = g * C + rank;
                if (!has) continue;
                for (int64_t q = b0; q < b1 && !sh->abort; ++q) {
                    const int64_t b = LIST ? static_cast<int64_t>(la.blist[lb + q]) : q;
                    for (int kc = 0; kc < nk; ++kc) {
                        if (!mrfk::mbar_wait(&sh->empty[stage], phase ^ 1u)) { fail(); break; }
                        unsigned char* sa = base + stage * STAGE_BYTES;
                        mrfk::mbar_arrive_expect_tx(&sh->full[stage], STAGE_BYTES);
                        mrfk::tma_load_2d(sa, &tmA, &sh->full[stage], kc * EK,
                                          static_cast<int32_t>(m * BM));
                        mrfk::tma_load_2d(sa + A_BYTES, &tmB, &sh->full[stage], kc * EK,
                                          static_cast<int32_t>(b * BN));
                        slot_used[stage] = true;
                        slot_phase[stage] = phase;
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            // Before the CTA may leave: every fill of its slots has landed, and its MMAs have
            // released them.
            for (int i = 0; i < STAGES; ++i) {
                if (!slot_used[i]) continue;
                if (sh->abort) mrfk::mbar_wait(&sh->full[i], slot_phase[i]);
                if (!mrfk::mbar_wait(&sh->empty[i], slot_phase[i])) atomicOr(err, MRF_DERR_TIMEOUT);
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
            for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
                int64_t s, g, b0, b1, lb;
                const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
                if (g * C * BM >= nact) continue;     // the cluster's tiles are all past the count
                if (!has) continue;
                for (int64_t q = b0; q < b1 && !sh->abort; ++q) {
                    if (!mrfk::mbar_wait(&sh->tempty[acc], aphase ^ 1u)) { fail(); break; }
                    mrfk::tc_fence_after();
                    const uint32_t dt = tmem + static_cast<uint32_t>(acc * BN);
                    bool ok = true;
                    for (int kc = 0; kc < nk; ++kc) {
                        if (!mrfk::mbar_wait(&sh->full[stage], phase)) { fail(); ok = false; break; }
                        mrfk::tc_fence_after();
                        const uint32_t sa = mrfk::smem_u32(base + stage * STAGE_BYTES);
                        const uint32_t sb = sa + A_BYTES;
                        const int rem = Kp - kc * EK;
                        const int nmma = rem >= EK ? EK / KPER : rem / KPER;
                        for (int k = 0; k < nmma; ++k) {
                            const uint64_t da = mrfk::sdesc_k_sw128(sa + k * 32);
                            const uint64_t db = mrfk::sdesc_k_sw128(sb + k * 32);
                            if (F8)
                                mrfk::mma_f8(dt, da, db, IDESC8, (kc > 0 || k > 0) ? 1u : 0u);
                            else
                                mrfk::mma_bf16(dt, da, db, IDESC, (kc > 0 || k > 0) ? 1u : 0u);
                        }
                        mrfk::mma_commit(&sh->empty[stage]);
                        any = true;
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mrfk::mma_commit(&sh->tfull[acc]);
                    if (++acc == 2) { acc = 0; aphase ^= 1u; }
                }
            }
            if (any) {
                // all MMAs issued by this thread complete before TMEM is released
                mrfk::mma_commit(&sh->drain);
                if (!mrfk::mbar_wait(&sh->drain, 0)) atomicOr(err, MRF_DERR_TIMEOUT);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (4 warps)
        // Per 32-atom chunk: scores |c|^2 (complex cone) or Re c (real cone) of the normalised
        // atoms, their maximum against the thread's K-th best, and only when it is beaten the
        // slow path: the chunk's scores go to this thread's column of shared memory and the
        // beating atoms are inserted one by one (one copy of the insertion code).
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
        float* col = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES + sizeof(Shared)) + row;
        int acc = 0;
        uint32_t aphase = 0;
        for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
            int64_t s, g, b0, b1, lb;
            const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
            if (g * C * BM >= nact) continue;     // the cluster's tiles are all past the count
            const int64_t m = g * C + rank;
            if (!has) continue;
            float ts[KT];
            int32_t ti[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) { ts[q] = -INFINITY; ti[q] = -1; }
            bool ok = true;
            for (int64_t qb = b0; qb < b1; ++qb) {
                const int64_t b = LIST ? static_cast<int64_t>(la.blist[lb + qb]) : qb;
                if (!mrfk::mbar_wait(&sh->tfull[acc], aphase)) { fail(); ok = false; break; }
                mrfk::tc_fence_after();
                const uint32_t tb = tmem + lane_base + static_cast<uint32_t>(acc * BN);
                epilogue_block<KT>(tb, cone, b, d, col, ts, ti);
                mrfk::tc_fence_before();
                mrfk::mbar_arrive(&sh->tempty[acc]);
                if (++acc == 2) { acc = 0; aphase ^= 1u; }
            }
            if (!ok) break;
            const int64_t v = m * BM + row;
            if (v < n) {
                if (F8) {
                    const float q = qs[v] * gsc;
                    const float f = (cone == MRF_CONE_COMPLEX) ? q * q : q;
#pragma unroll
                    for (int q2 = 0; q2 < KT; ++q2) ts[q2] *= f;
                }
                const int64_t o = (s * n + v) * KT;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    part_s[o + q] = ts[q];
                    part_i[o + q] = (LIST && ti[q] >= 0) ? la.perm[ti[q]] : ti[q];
                }
            }
        }
    }
    mrfk::tc_fence_before();
    __syncthreads();
    if (C > 1) mrfk::cluster_sync();
    mrfk::tc_fence_after();
    if (warp == 1) mrfk::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------- CTA-pair kernel
// The same search with the 2-SM MMA (cta_group::2): a cluster of two CTAs on one TPC computes
// a 256-voxel x 256-column tile per instruction; each CTA stages its own 128 query rows and one
// half of the atom block (CTA 0 the 128 real-part rows, CTA 1 the 128 imaginary-part rows), so
// a stage is 32 KB instead of 48 KB and six stages fit.  Both CTAs' loads report to CTA 0's
// `full` barrier; the even CTA issues every MMA and its commits arrive in both CTAs; both
// epilogues report a drained accumulator to CTA 0.  Each CTA's tensor memory holds its own
// 128 rows x 256 columns, so the epilogue is unchanged.
constexpr int P_STAGES = 6;
constexpr int P_A_BYTES = BM * BKB;
constexpr int P_B_BYTES = 128 * BKB;
constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;
constexpr uint32_t IDESC_P = mrfk::idesc_bf16(2 * BM, BN);
constexpr uint32_t IDESC8_P = mrfk::idesc_e4m3(2 * BM, BN);

struct SharedP {
    uint64_t full[P_STAGES];    // CTA 0: both CTAs' halves of the stage landed
    uint64_t empty[P_STAGES];   // both CTAs: the pair's MMAs finished reading the stage
    uint64_t tfull[2];          // both CTAs: accumulator ready
    uint64_t tempty[2];         // CTA 0: drained by the 4 + 4 epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort;
};

template <int KT, bool F8, bool LIST = false>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_topk_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int64_t n, int64_t d, int64_t nblk, int Kp, int cone, Sched sc,
               int blocks_per_split, float gsc, const float* __restrict__ qs,
               const int32_t* __restrict__ count, float* __restrict__ part_s,
               int32_t* __restrict__ part_i, uint32_t* err, ListArgs la) {
    constexpr int EK = F8 ? 128 : 64;
    constexpr int KPER = F8 ? 32 : 16;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    SharedP* sh = reinterpret_cast<SharedP*>(base + P_STAGES * P_STAGE_BYTES);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = mrfk::cluster_ctarank();      // 0 = issues the MMAs
    const int64_t cluster = blockIdx.x / 2;
    const int64_t nclusters = gridDim.x / 2;
    const int64_t units = LIST ? static_cast<int64_t>(*la.units) : sc.NG * sc.S;
    const int64_t nact = count ? min(static_cast<int64_t>(*count), n) : n;
    const int nk = (Kp + EK - 1) / EK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < P_STAGES; ++i) {
            mrfk::mbar_init(&sh->full[i], 1);
            mrfk::mbar_init(&sh->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mrfk::mbar_init(&sh->tfull[i], 1);
            mrfk::mbar_init(&sh->tempty[i], 8);
        }
        mrfk::mbar_init(&sh->drain, 1);
        sh->abort = 0;
        mrfk::fence_mbar_init();
    }
    if (warp == 1) {
        mrfk::tmem_alloc_pair(&sh->tmem_base, 512);
        mrfk::tmem_relinquish_pair();
    }
    if (warp == 0 && lane == 0) {
        mrfk::tma_prefetch_desc(&tmA);
        mrfk::tma_prefetch_desc(&tmB);
    }
    mrfk::tc_fence_before();
    mrfk::cluster_sync();
    mrfk::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    auto fail = [&]() {
        atomicOr(err, MRF_DERR_TIMEOUT);
        sh->abort = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            const uint32_t full0 = mrfk::mapa_shared(mrfk::smem_u32(&sh->full[0]), 0);
            int stage = 0;
            uint32_t phase = 0;
            uint32_t slot_phase[P_STAGES];
            bool slot_used[P_STAGES];
            for (int i = 0; i < P_STAGES; ++i) { slot_used[i] = false; slot_phase[i] = 0; }
            for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
                int64_t s, g, b0, b1, lb;
                const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
                if (g * 2 * BM >= nact) continue;     // the cluster's tiles are all past the count
                const int64_t m = g * 2 + rank;
                if (!has) continue;
                for (int64_t q = b0; q < b1 && !sh->abort; ++q) {
                    const int64_t b = LIST ? static_cast<int64_t>(la.blist[lb + q]) : q;
                    for (int kc = 0; kc < nk; ++kc) {
                        if (!mrfk::mbar_wait(&sh->empty[stage], phase ^ 1u)) { fail(); break; }
                        unsigned char* sa = base + stage * P_STAGE_BYTES;
                        const uint32_t fb = full0 + static_cast<uint32_t>(stage * sizeof(uint64_t));
                        if (rank == 0) mrfk::mbar_arrive_expect_tx(&sh->full[stage], 2 * P_STAGE_BYTES);
                        mrfk::tma_load_2d_pair(sa, &tmA, fb, kc * EK, static_cast<int32_t>(m * BM));
                        mrfk::tma_load_2d_pair(sa + P_A_BYTES, &tmB, fb, kc * EK,
                                               static_cast<int32_t>(b * BN + rank * 128));
                        slot_used[stage] = true;
                        slot_phase[stage] = phase;
                        if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            // before leaving: the pair's last MMAs released every slot this CTA filled (their
            // commit arrivals target this CTA, and they imply that its loads had landed)
            for (int i = 0; i < P_STAGES; ++i) {
                if (!slot_used[i]) continue;
                if (rank == 0 && sh->abort) mrfk::mbar_wait(&sh->full[i], slot_phase[i]);
                if (!mrfk::mbar_wait(&sh->empty[i], slot_phase[i])) atomicOr(err, MRF_DERR_TIMEOUT);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // -------------------------------------------------------- CTA 0: MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t aphase = 0;
            bool any = false;
            for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
                int64_t s, g, b0, b1, lb;
                const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
                if (g * 2 * BM >= nact) continue;     // the cluster's tiles are all past the count
                if (!has) continue;
                for (int64_t q = b0; q < b1 && !sh->abort; ++q) {
                    if (!mrfk::mbar_wait_cluster(&sh->tempty[acc], aphase ^ 1u)) { fail(); break; }
                    mrfk::tc_fence_after();
                    const uint32_t dt = tmem + static_cast<uint32_t>(acc * BN);
                    bool ok = true;
                    for (int kc = 0; kc < nk; ++kc) {
                        if (!mrfk::mbar_wait(&sh->full[stage], phase)) { fail(); ok = false; break; }
                        mrfk::tc_fence_after();
                        const uint32_t sa = mrfk::smem_u32(base + stage * P_STAGE_BYTES);
                        const uint32_t sb = sa + P_A_BYTES;
                        const int rem = Kp - kc * EK;
                        const int nmma = rem >= EK ? EK / KPER : rem / KPER;
                        for (int k = 0; k < nmma; ++k) {
                            const uint64_t da = mrfk::sdesc_k_sw128(sa + k * 32);
                            const uint64_t db = mrfk::sdesc_k_sw128(sb + k * 32);
                            if (F8)
                                mrfk::mma_f8_pair(dt, da, db, IDESC8_P, (kc > 0 || k > 0) ? 1u : 0u);
                            else
                                mrfk::mma_bf16_pair(dt, da, db, IDESC_P, (kc > 0 || k > 0) ? 1u : 0u);
                        }
                        mrfk::mma_commit_pair_mc(&sh->empty[stage], 3);
                        any = true;
                        if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mrfk::mma_commit_pair_mc(&sh->tfull[acc], 3);
                    if (++acc == 2) { acc = 0; aphase ^= 1u; }
                }
            }
            if (any) {
                mrfk::mma_commit_pair_mc(&sh->drain, 1);
                if (!mrfk::mbar_wait(&sh->drain, 0)) atomicOr(err, MRF_DERR_TIMEOUT);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (both CTAs)
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
        float* col = reinterpret_cast<float*>(base + P_STAGES * P_STAGE_BYTES + sizeof(SharedP)) + row;
        const uint32_t remote_tempty0 = mrfk::mapa_shared(mrfk::smem_u32(&sh->tempty[0]), 0);
        int acc = 0;
        uint32_t aphase = 0;
        for (int64_t uc = cluster; uc < units && !sh->abort; uc += nclusters) {
            int64_t s, g, b0, b1, lb;
            const bool has = unit_of<LIST>(sc, la, uc, blocks_per_split, nblk, s, g, b0, b1, lb);
            if (g * 2 * BM >= nact) continue;     // the cluster's tiles are all past the count
            const int64_t m = g * 2 + rank;
            if (!has) continue;
            float ts[KT];
            int32_t ti[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) { ts[q] = -INFINITY; ti[q] = -1; }
            bool ok = true;
            for (int64_t qb = b0; qb < b1; ++qb) {
                const int64_t b = LIST ? static_cast<int64_t>(la.blist[lb + qb]) : qb;
                if (!mrfk::mbar_wait(&sh->tfull[acc], aphase)) { fail(); ok = false; break; }
                mrfk::tc_fence_after();
                const uint32_t tb = tmem + lane_base + static_cast<uint32_t>(acc * BN);
                epilogue_block<KT>(tb, cone, b, d, col, ts, ti);
                mrfk::tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mrfk::mbar_arrive_cluster(remote_tempty0 +
                                              static_cast<uint32_t>(acc * sizeof(uint64_t)));
                if (++acc == 2) { acc = 0; aphase ^= 1u; }
            }
            if (!ok) break;
            const int64_t v = m * BM + row;
            if (v < n) {
                if (F8) {
                    const float q = qs[v] * gsc;
                    const float f = (cone == MRF_CONE_COMPLEX) ? q * q : q;
#pragma unroll
                    for (int q2 = 0; q2 < KT; ++q2) ts[q2] *= f;
                }
                const int64_t o = (s * n + v) * KT;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    part_s[o + q] = ts[q];
                    part_i[o + q] = (LIST && ti[q] >= 0) ? la.perm[ti[q]] : ti[q];
                }
            }
        }
    }
    mrfk::tc_fence_before();
    __syncthreads();
    mrfk::cluster_sync();
    mrfk::tc_fence_after();
    if (warp == 1) mrfk::tmem_dealloc_pair(tmem, 512);
}

constexpr size_t kSmemP = P_STAGES * P_STAGE_BYTES + sizeof(SharedP) + 32 * BM * sizeof(float) + 1024;

// ring + barriers + the epilogue's score columns (32 x 128 floats) + alignment slack
constexpr size_t kSmem = STAGES * STAGE_BYTES + sizeof(Shared) + 32 * BM * sizeof(float) + 1024;

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

}  // namespace

// Tensor map over a row-major [rows][Kp] operand of 2-byte (BF16) or 1-byte (E4M3) elements;
// boxes of 128 bytes x box_rows rows with the 128-byte swizzle the UMMA descriptors expect.
mrf_status tma_map_k128(CUtensorMap* m, const void* ptr, int64_t rows, int Kp, int box_rows,
                        bool f8) {
    EncodeFn enc = get_encode();
    if (!enc) {
        mrf_set_error("cuTensorMapEncodeTiled is unavailable");
        return MRF_ECUDA;
    }
    const int esz = f8 ? 1 : 2;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(Kp), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(Kp) * esz};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BKB / esz), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void*>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        mrf_set_error("cuTensorMapEncodeTiled failed: " + std::to_string(static_cast<int>(r)));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

namespace {

template <int KT, int C, bool F8>
mrf_status launch_t(const CUtensorMap& ta, const CUtensorMap& tb, int64_t n, const mrf_dict* D,
                    int Kp, int cone, Sched sc, int bps, int nclusters, float gsc, const float* qs,
                    const int32_t* count, float* part_s, int32_t* part_i, cudaStream_t st) {
    auto kern = k_tc_topk<KT, C, F8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmem));
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(nclusters * C));
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, ta, tb, n, D->d, D->nblk, Kp, cone,
                               sc, bps, gsc, qs, count, part_s, part_i, D->err, ListArgs{});
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("tensor-core search launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

template <int KT, bool F8>
mrf_status launch_pair(const CUtensorMap& ta, const CUtensorMap& tb, int64_t n, const mrf_dict* D,
                       int Kp, int cone, Sched sc, int bps, int nclusters, float gsc,
                       const float* qs, const int32_t* count, float* part_s, int32_t* part_i,
                       cudaStream_t st) {
    auto kern = k_tc_topk_pair<KT, F8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemP));
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(nclusters * 2));
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = kSmemP;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, ta, tb, n, D->d, D->nblk, Kp, cone,
                               sc, bps, gsc, qs, count, part_s, part_i, D->err, ListArgs{});
    }
    if (e != cudaSuccess) {
        mrf_set_error(std::string("tensor-core search (CTA pairs) launch: ") + cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    return MRF_OK;
}

template <int KT>
int max_pairs(cudaStream_t st) {
    auto kern = k_tc_topk_pair<KT, false>;   // same resources for both element types
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmemP)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = kSmemP;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

// Co-resident clusters of size C (persistent grid), from the occupancy calculator.
template <int KT, int C>
int max_clusters(cudaStream_t st) {
    auto kern = k_tc_topk<KT, C, false>;   // same resources for both element types
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

// Pick the atom split S minimising the makespan ceil(units / G) * (ceil(nblk / S) + h) of the
// static schedule (units = NG * S, G co-resident clusters), where h = 2 blocks models the cost of
// starting a unit (pipeline refill on a new query tile, the candidates written per unit and
// read again by the merge).  S * 16 candidates per voxel are kept below 1024.
int choose_splits(int64_t NG, int64_t nblk, int64_t G) {
    int best = 1;
    double best_t = 1e300;
    for (int64_t S = 1; S <= nblk && S <= 64; ++S) {
        int64_t units = NG * S;
        int64_t g = units < G ? units : G;
        int64_t waves = (units + g - 1) / g;
        int64_t per = (nblk + S - 1) / S;
        double t = static_cast<double>(waves) * (per + 2) + 1e-3 * S;
        if (t < best_t) { best_t = t; best = static_cast<int>(S); }
    }
    return best;
}

constexpr int kDefaultCluster = 1;     // CTAs co-scheduled on the same atom blocks
constexpr int64_t kDefaultLive = 32;   // voxel tiles kept live per super-group (~16 MB, L=1000)
constexpr int64_t kDefaultLiveX3 = 8;  // the same for the split-BF16 form

int cluster_of(const mrf_dict* D) {
    int c = D->tune.bf16_cluster;
    return (c == 1 || c == 2 || c == 4) ? c : kDefaultCluster;
}

template <int KT>
int max_clusters_any(int C, cudaStream_t st) {
    switch (C) {
        case 1: return max_clusters<KT, 1>(st);
        case 2: return max_clusters<KT, 2>(st);
        default: return max_clusters<KT, 4>(st);
    }
}

}  // namespace

int bf16_choose_splits(const mrf_dict* D, int64_t n) {
    if (D->tune.bf16_splits > 0) return static_cast<int>(D->tune.bf16_splits);
    const int C = D->tune.bf16_pair == 1 ? 2 : cluster_of(D);
    const int64_t Mt = (n + BM - 1) / BM;
    const int64_t NG = (Mt + C - 1) / C;
    return choose_splits(NG, D->nblk, D->num_sms / C);
}

namespace {

template <int KT, bool F8>
mrf_status launch_c(int C, const CUtensorMap& ta, const CUtensorMap& tb, int64_t n,
                    const mrf_dict* D, int Kp, int cone, Sched sc, int bps, int nc, float wts,
                    const float* qs, const int32_t* count, float* part_s, int32_t* part_i,
                    cudaStream_t st) {
    switch (C) {
        case 1: return launch_t<KT, 1, F8>(ta, tb, n, D, Kp, cone, sc, bps, nc, wts, qs, count, part_s, part_i, st);
        case 2: return launch_t<KT, 2, F8>(ta, tb, n, D, Kp, cone, sc, bps, nc, wts, qs, count, part_s, part_i, st);
        default: return launch_t<KT, 4, F8>(ta, tb, n, D, Kp, cone, sc, bps, nc, wts, qs, count, part_s, part_i, st);
    }
}

// Operand forms of the tensor-core search.
enum Form { FORM_BF16 = 0, FORM_FP8 = 1, FORM_X3 = 2 };

// Shared launch path of every operand form: operand maps, schedule, persistent grid.  The split
// form runs the BF16 kernel over its three-segment rows (Kp3 = 3 Kp).
mrf_status launch_tc(int form, const void* zq, const float* qs, int64_t n, mrf_dict* D, int cone,
                     int K, int S, float* part_s, int32_t* part_i, const int32_t* count,
                     cudaStream_t st) {
    if (n == 0) return MRF_OK;
    const bool f8 = (form == FORM_FP8);
    const void* op = f8 ? static_cast<const void*>(D->fop)
                        : (form == FORM_X3 ? static_cast<const void*>(D->bop3)
                                           : static_cast<const void*>(D->bop));
    if (!op) {
        mrf_set_error(f8 ? "FP8 operand was not packed (mrf_index_opts.pack_fp8 = 0)"
                         : (form == FORM_X3
                                ? "split-BF16 operand was not packed (mrf_index_opts.pack_bf16x3 = 0)"
                                : "BF16 operand was not packed (mrf_index_opts.pack_bf16 = 0)"));
        return MRF_EUNSUPPORTED;
    }
    if (K != 8 && K != 16 && K != 32) {
        mrf_set_error("tensor-core search: K must be 8, 16 or 32");
        return MRF_EINVAL;
    }
    const bool pair = D->tune.bf16_pair == 1;
    const int C = pair ? 2 : cluster_of(D);
    const int Kp = f8 ? D->Kp8 : (form == FORM_X3 ? D->Kp3 : D->Kp);
    CUtensorMap ta, tb;
    MRF_TRY(tma_map_k128(&ta, zq, n, Kp, BM, f8));
    MRF_TRY(tma_map_k128(&tb, op, D->nblk * 256, Kp, pair ? BN / 2 : BN, f8));
    const int64_t Mt = (n + BM - 1) / BM;
    // the split form's 128-atom blocks are three times longer (3 MB at L = 1000): fewer live
    // voxel tiles keep the CTAs that stream the same atoms close enough for L2 to serve them
    const int64_t live = D->tune.bf16_live_tiles > 0
                             ? D->tune.bf16_live_tiles
                             : (form == FORM_X3 ? kDefaultLiveX3 : kDefaultLive);
    Sched sc;
    sc.NG = (Mt + C - 1) / C;
    sc.S = S;
    sc.PG = (live + C - 1) / C;
    const int bps = static_cast<int>((D->nblk + S - 1) / S);
    const int64_t units = sc.NG * sc.S;
    int nc = pair ? ((K == 8) ? max_pairs<8>(st) : (K == 16) ? max_pairs<16>(st) : max_pairs<32>(st))
                  : ((K == 8) ? max_clusters_any<8>(C, st)
                              : (K == 16) ? max_clusters_any<16>(C, st) : max_clusters_any<32>(C, st));
    if (nc <= 0) {
        mrf_set_error("tensor-core search: no cluster of the requested size fits on this device");
        return MRF_EUNSUPPORTED;
    }
    if (nc > units) nc = static_cast<int>(units);
    D->tune.last_bf16_ctas = nc * C;
    D->tune.last_bf16_cluster = C;
    D->tune.last_bf16_splits = S;
    const float wts = f8 ? D->g8 : 1.f;
#define MRF_TC_ARGS ta, tb, n, D, Kp, cone, sc, bps, nc, wts, qs, count, part_s, part_i, st
    if (pair) {
        if (f8)
            return K == 8 ? launch_pair<8, true>(MRF_TC_ARGS)
                 : K == 16 ? launch_pair<16, true>(MRF_TC_ARGS) : launch_pair<32, true>(MRF_TC_ARGS);
        return K == 8 ? launch_pair<8, false>(MRF_TC_ARGS)
             : K == 16 ? launch_pair<16, false>(MRF_TC_ARGS) : launch_pair<32, false>(MRF_TC_ARGS);
    }
    if (f8)
        return K == 8 ? launch_c<8, true>(C, MRF_TC_ARGS)
             : K == 16 ? launch_c<16, true>(C, MRF_TC_ARGS) : launch_c<32, true>(C, MRF_TC_ARGS);
    return K == 8 ? launch_c<8, false>(C, MRF_TC_ARGS)
         : K == 16 ? launch_c<16, false>(C, MRF_TC_ARGS) : launch_c<32, false>(C, MRF_TC_ARGS);
#undef MRF_TC_ARGS
}

}  // namespace

mrf_status launch_bf16_topk(const __nv_bfloat16* zq, int64_t n, mrf_dict* D, int cone, int K,
                            int S, float* part_s, int32_t* part_i, cudaStream_t st,
                            const int32_t* count) {
    return launch_tc(FORM_BF16, zq, nullptr, n, D, cone, K, S, part_s, part_i, count, st);
}

mrf_status launch_fp8_topk(const uint8_t* zq8, const float* qs, int64_t n, mrf_dict* D, int cone,
                           int K, int S, float* part_s, int32_t* part_i, cudaStream_t st) {
    return launch_tc(FORM_FP8, zq8, qs, n, D, cone, K, S, part_s, part_i, nullptr, st);
}

mrf_status launch_x3_topk(const __nv_bfloat16* zq3, int64_t n, mrf_dict* D, int cone, int K,
                          int S, float* part_s, int32_t* part_i, cudaStream_t st) {
    return launch_tc(FORM_X3, zq3, nullptr, n, D, cone, K, S, part_s, part_i, nullptr, st);
}

// Block-list search of the cover-tree form: queries zq [n][Kp] (grouped into 128-row tiles),
// the depth-first operand op ([nblk * 256][Kp]; BF16 layout, or the split form with Kp = 3 x
// the BF16 row length), the block lists of the tile groups (see ListArgs: tfirst, blist, uoff
// per super-group of `sg` groups, *units = uoff[super-groups], all on the device), chunks of
// `chunk` blocks, at most S per group;
// candidates [S][n][K] (slot = chunk) with atom indices perm[position]; slots of chunks a group
// does not have are not written.  Persistent grid of single CTAs, or of CTA pairs (256 voxels
// per unit, each CTA staging half of every block; `group` must then be even); the unit count
// is read on the device.
mrf_status launch_bf16_topk_list(const __nv_bfloat16* zq, int64_t n, mrf_dict* D,
                                 const __nv_bfloat16* op, int Kp, int cone, int K, int group,
                                 int chunk, int sg, bool pair, const int32_t* tfirst,
                                 const int32_t* blist, const int32_t* uoff, const int32_t* perm,
                                 float* part_s, int32_t* part_i, cudaStream_t st) {
    if (n == 0) return MRF_OK;
    if (K != 8 && K != 16 && K != 32) {
        mrf_set_error("tree search: K must be 8, 16 or 32");
        return MRF_EINVAL;
    }
    if (pair && (group % 2)) {
        mrf_set_error("tree search: CTA pairs need an even number of tiles per block list");
        return MRF_EINVAL;
    }
    CUtensorMap ta, tb;
    MRF_TRY(tma_map_k128(&ta, zq, n, Kp, BM, false));
    MRF_TRY(tma_map_k128(&tb, op, D->nblk * 256, Kp, pair ? BN / 2 : BN, false));
    const int64_t Mt = (n + BM - 1) / BM;
    ListArgs la;
    la.tfirst = tfirst;
    la.blist = blist;
    la.perm = perm;
    la.uoff = uoff;
    la.group = group;
    la.chunk = chunk;
    la.tpu = pair ? 2 : 1;
    la.ntiles = Mt;
    la.sg = sg;
    la.ngroups = (Mt + group - 1) / group;
    la.nsg = (la.ngroups + sg - 1) / sg;
    la.units = uoff + la.nsg;
    Sched sc{pair ? (Mt + 1) / 2 : Mt, 1, 1};
    if (pair) {
        const int nc = (K == 8) ? max_pairs<8>(st) : (K == 16) ? max_pairs<16>(st)
                                                               : max_pairs<32>(st);
        if (nc <= 0) {
            mrf_set_error("tree search: no CTA pair fits on this device");
            return MRF_EUNSUPPORTED;
        }
        auto go = [&](auto kern) -> mrf_status {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kSmemP));
            if (e == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(static_cast<unsigned>(nc * 2));
                cfg.blockDim = dim3(NTHREADS);
                cfg.dynamicSmemBytes = kSmemP;
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 2;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, kern, ta, tb, n, D->d, D->nblk, Kp, cone, sc, 0, 1.f,
                                       static_cast<const float*>(nullptr),
                                       static_cast<const int32_t*>(nullptr), part_s, part_i,
                                       D->err, la);
            }
            if (e != cudaSuccess) {
                mrf_set_error(std::string("tree block-list search (CTA pairs) launch: ") +
                              cudaGetErrorString(e));
                return MRF_ECUDA;
            }
            return MRF_OK;
        };
        if (K == 8) return go(k_tc_topk_pair<8, false, true>);
        if (K == 16) return go(k_tc_topk_pair<16, false, true>);
        return go(k_tc_topk_pair<32, false, true>);
    }
    int nc = (K == 8) ? max_clusters<8, 1>(st) : (K == 16) ? max_clusters<16, 1>(st)
                                                           : max_clusters<32, 1>(st);
    if (nc <= 0) {
        mrf_set_error("tree search: the kernel does not fit on this device");
        return MRF_EUNSUPPORTED;
    }
    auto go = [&](auto kern) -> mrf_status {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kSmem));
        if (e == cudaSuccess) {
            kern<<<static_cast<unsigned>(nc), NTHREADS, kSmem, st>>>(
                ta, tb, n, D->d, D->nblk, Kp, cone, sc, 0, 1.f, nullptr, nullptr, part_s,
                part_i, D->err, la);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            mrf_set_error(std::string("tree block-list search launch: ") + cudaGetErrorString(e));
            return MRF_ECUDA;
        }
        return MRF_OK;
    };
    if (K == 8) return go(k_tc_topk<8, 1, false, true>);
    if (K == 16) return go(k_tc_topk<16, 1, false, true>);
    return go(k_tc_topk<32, 1, false, true>);
}
