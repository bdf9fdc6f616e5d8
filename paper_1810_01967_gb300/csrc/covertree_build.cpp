// Host construction of the cover tree of the normalised dictionary (§4.1; §4.3 "cover tree
// structure built for the normalized fingerprint dictionary").
//
// Levels i = 0, 1, ... have radii r_i = sigma 2^-i, sigma = max_j delta(root, u_j), root = atom 0.
// Each net S_{i+1} is S_i plus a maximal r_{i+1}-separated set of the remaining atoms, chosen
// greedily in index order (the lexicographically first maximal independent set), so:
//   nesting     S_i is a subset of S_{i+1};
//   separation  nodes of S_{i+1} are pairwise farther than r_{i+1} (old nodes are r_i apart);
//   covering    every atom is within r_{i+1} of S_{i+1} (maximality), so a new node's nearest
//               node of S_i -- its parent -- is within r_i.
// The construction is level-synchronous: every remaining atom keeps its nearest node of the
// current net ("cell"), and every node keeps its neighbours within 4 r_i, which contain all nodes
// that a query of radius r_{i+1} around an atom of its cell can reach (and, refined, the
// neighbours at the next level).  Distance work is split over threads; the triangle inequality
// skips whole cells.  maxdist (the largest distance from a node to its subtree) is exact.
// Atoms closer than `dup_tol` to an earlier atom are duplicates, represented by that atom.
// Distances above 0.25 are evaluated with FP32 sums, so the invariants hold up to a relative
// rounding of about 1e-7 (the search's pruning slack is 1e-5).
// Neighbour lists keep at most `max_neighbours` nearest nodes.  A truncated list can only miss a
// conflict between far-apart cells, which adds a node (separation may then fail there); covering
// and the exact maxdist -- what Algorithm 1's (1+eps) guarantee rests on -- always hold, because
// an atom stays out of a net only after a node covering it has been found, and its cell search
// examines that node's cell.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <complex>
#include <cstdint>
#include <functional>
#include <thread>
#include <vector>

#include "covertree_host.h"

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
}

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
    unsigned hw = std::thread::hardware_concurrency();
    int64_t T = hw ? static_cast<int64_t>(hw) : 4;
    if (n < 2048 || T <= 1) {
        body(0, n);
        return;
    }
    if (T > 64) T = 64;
    std::vector<std::thread> th;
    std::atomic<int64_t> next(0);
    const int64_t chunk = std::max<int64_t>(256, n / (T * 16));
    for (int64_t t = 0; t < T; ++t)
        th.emplace_back([&]() {
            for (;;) {
                int64_t a = next.fetch_add(chunk);
                if (a >= n) break;
                body(a, std::min(n, a + chunk));
            }
        });
    for (auto& x : th) x.join();
}

struct Builder {
    const CtParams& P;
    int64_t d;
    int L;
    std::vector<std::complex<float>> U;   // unit atoms (normalised in FP64, stored FP32)
    std::vector<double> nrm2;             // exact squared norms of the stored unit atoms

    explicit Builder(const CtParams& p) : P(p), d(p.d), L(p.L) {}

    // Correlation in FP32 with 8 independent partial sums (vectorisable); pairs closer than
    // 0.25 are recomputed with FP64 sums, which keeps small distances accurate (the cancellation
    // in ||a||^2 + ||b||^2 - 2|c| costs FP32 about 1e-7 / distance).
    double dist(int64_t a, int64_t b) const {
        const float* x = reinterpret_cast<const float*>(&U[static_cast<size_t>(a) * L]);
        const float* y = reinterpret_cast<const float*>(&U[static_cast<size_t>(b) * L]);
        float fr[8] = {0, 0, 0, 0, 0, 0, 0, 0}, fi[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int t = 0;
        for (; t + 8 <= L; t += 8)
            for (int k = 0; k < 8; ++k) {
                const float xr = x[2 * (t + k)], xi = x[2 * (t + k) + 1];
                const float yr = y[2 * (t + k)], yi = y[2 * (t + k) + 1];
                fr[k] += xr * yr + xi * yi;
                fi[k] += xr * yi - xi * yr;
            }
        for (; t < L; ++t) {
            const float xr = x[2 * t], xi = x[2 * t + 1], yr = y[2 * t], yi = y[2 * t + 1];
            fr[0] += xr * yr + xi * yi;
            fi[0] += xr * yi - xi * yr;
        }
        double R = 0.0, I = 0.0;
        for (int k = 0; k < 8; ++k) { R += fr[k]; I += fi[k]; }
        double c = (P.metric == 0) ? std::sqrt(R * R + I * I) : R;
        double d2 = nrm2[a] + nrm2[b] - 2.0 * c;
        if (d2 > 0.0625) return std::sqrt(d2);
        double re[8] = {0, 0, 0, 0, 0, 0, 0, 0}, im[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        t = 0;
        for (; t + 8 <= L; t += 8)
            for (int k = 0; k < 8; ++k) {
                const double xr = x[2 * (t + k)], xi = x[2 * (t + k) + 1];
                const double yr = y[2 * (t + k)], yi = y[2 * (t + k) + 1];
                re[k] += xr * yr + xi * yi;
                im[k] += xr * yi - xi * yr;
            }
        for (; t < L; ++t) {
            const double xr = x[2 * t], xi = x[2 * t + 1], yr = y[2 * t], yi = y[2 * t + 1];
            re[0] += xr * yr + xi * yi;
            im[0] += xr * yi - xi * yr;
        }
        R = ((re[0] + re[1]) + (re[2] + re[3])) + ((re[4] + re[5]) + (re[6] + re[7]));
        I = ((im[0] + im[1]) + (im[2] + im[3])) + ((im[4] + im[5]) + (im[6] + im[7]));
        c = (P.metric == 0) ? std::sqrt(R * R + I * I) : R;
        return std::sqrt(std::max(0.0, nrm2[a] + nrm2[b] - 2.0 * c));
    }
};

struct Nb {
    int32_t node;
    float dist;
};

}  // namespace

int ct_build(const CtParams& P, CtTree* out) {
    Builder B(P);
    const int64_t d = P.d;
    const int L = P.L;
    if (d < 1 || L < 1) return 1;
    // unit atoms
    B.U.resize(static_cast<size_t>(d) * L);
    B.nrm2.resize(d);
    parallel_for(d, [&](int64_t a0, int64_t a1) {
        for (int64_t a = a0; a < a1; ++a) {
            const std::complex<float>* x = P.atoms + static_cast<size_t>(a) * L;
            double s = 0.0;
            for (int t = 0; t < L; ++t) s += static_cast<double>(std::norm(x[t]));
            const double inv = s > 0.0 ? 1.0 / std::sqrt(s) : 0.0;
            double s2 = 0.0;
            for (int t = 0; t < L; ++t) {
                std::complex<float> u(static_cast<float>(x[t].real() * inv),
                                      static_cast<float>(x[t].imag() * inv));
                B.U[static_cast<size_t>(a) * L + t] = u;
                s2 += static_cast<double>(u.real()) * u.real() +
                      static_cast<double>(u.imag()) * u.imag();
            }
            B.nrm2[a] = s2;
        }
    });
    out->d = d;
    out->L = L;
    out->metric = P.metric;
    out->rep.assign(d, -1);
    out->first_level.assign(d, -1);
    out->parent.assign(d, -1);
    // cells: nearest net node of every remaining atom
    std::vector<int32_t> cell(d, 0);
    std::vector<double> dcell(d, 0.0);
    const int32_t root = 0;
    parallel_for(d, [&](int64_t a0, int64_t a1) {
        for (int64_t a = a0; a < a1; ++a) dcell[a] = (a == root) ? 0.0 : B.dist(root, a);
    });
    out->rep[root] = root;
    out->first_level[root] = 0;
    double sigma = 0.0;
    for (int64_t a = 0; a < d; ++a) sigma = std::max(sigma, dcell[a]);
    // distances above 0.25 come from FP32 sums (relative error ~1e-7): widen the root's radius
    // so that covering holds for every atom in exact arithmetic too
    sigma *= 1.0 + 1e-6;
    out->sigma = sigma;
    std::vector<int32_t> remaining;
    remaining.reserve(d);
    for (int64_t a = 1; a < d; ++a) {
        if (dcell[a] <= P.dup_tol) out->rep[a] = root;   // duplicate of the root
        else remaining.push_back(static_cast<int32_t>(a));
    }
    // neighbour lists of the current net (node -> nodes within 4 r_i, with distances)
    std::vector<int32_t> net = {root};
    std::vector<std::vector<Nb>> nbr(d);
    nbr[root].push_back({root, 0.f});
    std::vector<std::vector<int32_t>> newkids(d);   // new nodes per cell at this level
    int level = 0;
    while (!remaining.empty() && sigma > 0.0) {
        if (level >= 60) return 2;
        const double ri = sigma * std::ldexp(1.0, -level);   // current covering radius
        const double r = ri * 0.5;                           // next level's radius
        const auto t_level = Clock::now();
        // ---- 1. greedy maximal r-separated selection in index order (remaining is sorted)
        for (int32_t p : net) newkids[p].clear();
        std::vector<char> covered(remaining.size(), 0);
        std::vector<int32_t> selected;
        const int64_t R = static_cast<int64_t>(remaining.size());
        const int64_t CH = 4096;
        std::vector<int64_t> stamp_of(d, -1);   // chunk in which a cell first got a new node
        std::vector<size_t> start_of(d, 0);     // its newkids size at that moment
        for (int64_t c0 = 0; c0 < R; c0 += CH) {
            const int64_t c1 = std::min(R, c0 + CH);
            // (a) against new nodes selected in earlier chunks, in neighbouring cells (parallel).
            //     A new node y of cell p2 is skipped when |d(x,p2) - d(p2,y)| > r.
            parallel_for(c1 - c0, [&](int64_t k0, int64_t k1) {
                for (int64_t k = c0 + k0; k < c0 + k1; ++k) {
                    const int32_t x = remaining[k];
                    if (dcell[x] <= r) { covered[k] = 1; continue; }   // an old node covers x
                    const int32_t p = cell[x];
                    bool cov = false;
                    for (const Nb& nb : nbr[p]) {   // sorted by distance from p
                        if (nb.dist - dcell[x] - ri > r) break;
                        const std::vector<int32_t>& ys = newkids[nb.node];
                        if (ys.empty()) continue;
                        const double dx2 = (nb.node == p) ? dcell[x] : B.dist(x, nb.node);
                        for (int32_t y : ys)
                            if (std::fabs(dx2 - dcell[y]) <= r && B.dist(x, y) <= r) {
                                cov = true;
                                break;
                            }
                        if (cov) break;
                    }
                    covered[k] = cov ? 1 : 0;
                }
            });
            // (b) in index order, against the nodes selected earlier in this chunk
            for (int64_t k = c0; k < c1; ++k) {
                if (covered[k]) continue;
                const int32_t x = remaining[k];
                const int32_t p = cell[x];
                bool cov = false;
                for (const Nb& nb : nbr[p]) {
                    if (nb.dist - dcell[x] - ri > r) break;
                    if (stamp_of[nb.node] != c0) continue;
                    const std::vector<int32_t>& ys = newkids[nb.node];
                    const double dx2 = (nb.node == p) ? dcell[x] : B.dist(x, nb.node);
                    for (size_t q = start_of[nb.node]; q < ys.size(); ++q)
                        if (std::fabs(dx2 - dcell[ys[q]]) <= r && B.dist(x, ys[q]) <= r) {
                            cov = true;
                            break;
                        }
                    if (cov) break;
                }
                if (cov) { covered[k] = 1; continue; }
                if (stamp_of[p] != c0) { stamp_of[p] = c0; start_of[p] = newkids[p].size(); }
                newkids[p].push_back(x);
                selected.push_back(x);
            }
        }
        const double t1 = ms_since(t_level);
        // ---- 2. new nodes: parent = nearest node of S_i (their cell), first level = level+1
        for (int32_t x : selected) {
            out->first_level[x] = level + 1;
            out->parent[x] = cell[x];
            out->rep[x] = x;
        }
        // ---- 3. neighbour lists of S_{i+1} (radius 4 r) from the refinement of the old lists
        std::vector<int32_t> net2 = net;
        net2.insert(net2.end(), selected.begin(), selected.end());
        std::vector<std::vector<Nb>> nb2(net2.size());
        parallel_for(static_cast<int64_t>(net2.size()), [&](int64_t q0, int64_t q1) {
            for (int64_t qi = q0; qi < q1; ++qi) {
                const int32_t q = net2[qi];
                const int32_t p = (out->first_level[q] == level + 1) ? out->parent[q] : q;
                const double dqp = (p == q) ? 0.0 : dcell[q];
                std::vector<Nb>& lst = nb2[qi];
                for (const Nb& nb : nbr[p]) {
                    const int32_t p2 = nb.node;
                    // candidates: p2 itself and its new children (within ri of p2)
                    const std::vector<int32_t>& ks = newkids[p2];
                    if (nb.dist - dqp > 4.0 * r + (ks.empty() ? 0.0 : ri)) continue;
                    const double dq2 = (p2 == q) ? 0.0 : (p2 == p ? dqp : B.dist(q, p2));
                    if (dq2 <= 4.0 * r) lst.push_back({p2, static_cast<float>(dq2)});
                    for (int32_t c : ks) {
                        if (std::fabs(dq2 - dcell[c]) > 4.0 * r) continue;
                        const double dd = (c == q) ? 0.0 : B.dist(q, c);
                        if (dd <= 4.0 * r) lst.push_back({c, static_cast<float>(dd)});
                    }
                }
            }
        });
        const double t3 = ms_since(t_level);
        // ---- 4. new cells of the atoms still outside the net: nearest node of S_{i+1}
        std::vector<int32_t> rem2;
        rem2.reserve(remaining.size());
        for (size_t k = 0; k < remaining.size(); ++k)
            if (out->first_level[remaining[k]] < 0) rem2.push_back(remaining[k]);
        std::vector<int32_t> cell2(rem2.size());
        std::vector<double> dcell2(rem2.size());
        parallel_for(static_cast<int64_t>(rem2.size()), [&](int64_t k0, int64_t k1) {
            for (int64_t k = k0; k < k1; ++k) {
                const int32_t x = rem2[k];
                const int32_t p = cell[x];
                int32_t best = p;
                double bd = dcell[x];
                for (const Nb& nb : nbr[p]) {
                    const int32_t p2 = nb.node;
                    const std::vector<int32_t>& ks = newkids[p2];
                    const double lb = nb.dist - dcell[x];   // lower bound on d(x, p2)
                    if (lb > bd + ri) break;                // sorted: no later cell can win
                    if (lb > bd && ks.empty()) continue;
                    const double dx2 = (p2 == p) ? dcell[x] : B.dist(x, p2);
                    if (p2 != p && (dx2 < bd || (dx2 == bd && p2 < best))) { bd = dx2; best = p2; }
                    for (int32_t c : ks) {
                        if (std::fabs(dx2 - dcell[c]) > bd) continue;
                        const double dd = B.dist(x, c);
                        if (dd < bd || (dd == bd && c < best)) { bd = dd; best = c; }
                    }
                }
                cell2[k] = best;
                dcell2[k] = bd;
            }
        });
        // duplicates: closer than dup_tol to their nearest node
        std::vector<int32_t> rem3;
        rem3.reserve(rem2.size());
        for (size_t k = 0; k < rem2.size(); ++k) {
            const int32_t x = rem2[k];
            cell[x] = cell2[k];
            dcell[x] = dcell2[k];
            if (dcell2[k] <= P.dup_tol) out->rep[x] = cell2[k];
            else rem3.push_back(x);
        }
        if (P.verbose)
            std::fprintf(stderr, "[cover tree] level %d: %zu new nodes, %zu remaining, "
                         "select %.0f ms, neighbours %.0f ms, cells %.0f ms\n", level + 1,
                         selected.size(), rem3.size(), t1, t3 - t1, ms_since(t_level) - t3);
        remaining.swap(rem3);
        parallel_for(static_cast<int64_t>(net2.size()), [&](int64_t q0, int64_t q1) {
            for (int64_t qi = q0; qi < q1; ++qi) {
                std::vector<Nb>& l = nb2[qi];
                auto cmp = [](const Nb& a, const Nb& b) {
                    return a.dist != b.dist ? a.dist < b.dist : a.node < b.node;
                };
                if (static_cast<int>(l.size()) > P.max_neighbours) {
                    std::partial_sort(l.begin(), l.begin() + P.max_neighbours, l.end(), cmp);
                    l.resize(P.max_neighbours);
                } else {
                    std::sort(l.begin(), l.end(), cmp);
                }
            }
        });
        for (size_t qi = 0; qi < net2.size(); ++qi) nbr[net2[qi]].swap(nb2[qi]);
        for (int32_t x : selected) { cell[x] = x; dcell[x] = 0.0; }
        net.swap(net2);
        ++level;
    }
    out->imax = level;
    // representatives of duplicates point at tree nodes (resolve chains)
    for (int64_t a = 0; a < d; ++a) {
        int32_t r = out->rep[a];
        while (r >= 0 && out->rep[r] != r) r = out->rep[r];
        out->rep[a] = r;
    }
    // ---- explicit nodes (parent, level) with their children, BFS positions, exact maxdist
    std::vector<std::vector<int32_t>> kids_by_level(level + 1);
    for (int64_t a = 0; a < d; ++a)
        if (out->rep[a] == a && a != root) kids_by_level[out->first_level[a]].push_back(a);
    out->pos.assign(d, -1);
    out->order.clear();
    out->order.push_back(root);
    out->pos[root] = 0;
    out->node_first.clear();
    out->en_level.clear();
    out->en_cb.clear();
    out->en_ce.clear();
    out->en_parent.clear();
    for (int lv = 1; lv <= level; ++lv) {
        std::vector<int32_t>& ks = kids_by_level[lv];
        std::sort(ks.begin(), ks.end(), [&](int32_t x, int32_t y) {
            const int32_t px = out->pos[out->parent[x]], py = out->pos[out->parent[y]];
            return px != py ? px < py : x < y;
        });
        size_t k = 0;
        while (k < ks.size()) {
            const int32_t p = out->parent[ks[k]];
            size_t e = k;
            while (e < ks.size() && out->parent[ks[e]] == p) ++e;
            out->en_parent.push_back(p);
            out->en_level.push_back(lv - 1);
            out->en_cb.push_back(static_cast<int32_t>(out->order.size()));
            for (size_t q = k; q < e; ++q) {
                out->pos[ks[q]] = static_cast<int32_t>(out->order.size());
                out->order.push_back(ks[q]);
            }
            out->en_ce.push_back(static_cast<int32_t>(out->order.size()));
            k = e;
        }
    }
    const int64_t nt = static_cast<int64_t>(out->order.size());
    const int64_t ne = static_cast<int64_t>(out->en_parent.size());
    // explicit nodes sorted by (parent position, level) -> per-node CSR
    std::vector<int64_t> eo(ne);
    for (int64_t e = 0; e < ne; ++e) eo[e] = e;
    std::sort(eo.begin(), eo.end(), [&](int64_t a, int64_t b) {
        const int32_t pa = out->pos[out->en_parent[a]], pb = out->pos[out->en_parent[b]];
        return pa != pb ? pa < pb : out->en_level[a] < out->en_level[b];
    });
    std::vector<int32_t> lvl(ne), cb(ne), ce(ne), par(ne);
    for (int64_t e = 0; e < ne; ++e) {
        lvl[e] = out->en_level[eo[e]];
        cb[e] = out->en_cb[eo[e]];
        ce[e] = out->en_ce[eo[e]];
        par[e] = out->en_parent[eo[e]];
    }
    out->en_level.swap(lvl);
    out->en_cb.swap(cb);
    out->en_ce.swap(ce);
    out->en_parent.swap(par);
    out->node_first.assign(nt + 1, 0);
    for (int64_t e = 0; e < ne; ++e) out->node_first[out->pos[out->en_parent[e]] + 1]++;
    for (int64_t q = 0; q < nt; ++q) out->node_first[q + 1] += out->node_first[q];
    const auto t_md = Clock::now();
    // subtree member ranges: a node's subtree is itself plus its children's subtrees.  Members
    // are gathered into one array by a post-order walk (positions only increase downwards).
    out->en_maxdist.assign(ne, 0.f);
    std::vector<std::vector<int32_t>> sub(nt);   // subtree members (positions) per node
    for (int64_t q = nt - 1; q >= 0; --q) {
        std::vector<int32_t>& s = sub[q];
        s.push_back(static_cast<int32_t>(q));
        for (int32_t e = out->node_first[q]; e < out->node_first[q + 1]; ++e)
            for (int32_t c = out->en_cb[e]; c < out->en_ce[e]; ++c) {
                s.insert(s.end(), sub[c].begin(), sub[c].end());
            }
    }
    // maxdist(q, level of explicit node e) = max over children of e and of q's deeper explicit
    // nodes, of the distance from q to every member of those children's subtrees
    parallel_for(nt, [&](int64_t q0, int64_t q1) {
        for (int64_t q = q0; q < q1; ++q) {
            const int32_t a = out->order[q];
            double run = 0.0;
            for (int32_t e = out->node_first[q + 1] - 1; e >= out->node_first[q]; --e) {
                for (int32_t c = out->en_cb[e]; c < out->en_ce[e]; ++c)
                    for (int32_t m : sub[c]) run = std::max(run, B.dist(a, out->order[m]));
                // round up so the stored bound never undercuts the exact maximum
                out->en_maxdist[e] = std::nextafter(static_cast<float>(run), INFINITY);
            }
        }
    });
    if (P.verbose) std::fprintf(stderr, "[cover tree] maxdist %.0f ms\n", ms_since(t_md));
    // unit atoms in BFS order for the device
    out->unit_atoms.resize(static_cast<size_t>(nt) * L);
    for (int64_t q = 0; q < nt; ++q)
        std::copy(&B.U[static_cast<size_t>(out->order[q]) * L],
                  &B.U[static_cast<size_t>(out->order[q]) * L] + L,
                  &out->unit_atoms[static_cast<size_t>(q) * L]);
    return 0;
}
