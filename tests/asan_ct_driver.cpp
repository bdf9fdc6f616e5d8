// Drives the host cover-tree builder (paper_1810_01967_gb300/csrc/covertree_build.cpp) under
// AddressSanitizer and UndefinedBehaviorSanitizer: seeded random atoms with exact and near
// duplicates, both metrics, from one atom to a few hundred; checks that every index of the flat
// layout stays in range.  Exit status 0 = clean.
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "covertree_host.h"

static int check(const CtTree& T, int64_t d) {
    const int64_t nt = static_cast<int64_t>(T.order.size());
    if (nt < 1 || nt > d) return 1;
    if (static_cast<int64_t>(T.node_first.size()) != nt + 1) return 2;
    const int64_t ne = static_cast<int64_t>(T.en_level.size());
    for (int64_t p = 0; p < nt; ++p) {
        if (T.node_first[p] > T.node_first[p + 1] || T.node_first[p + 1] > ne) return 3;
        if (T.order[p] < 0 || T.order[p] >= d) return 4;
    }
    for (int64_t e = 0; e < ne; ++e) {
        if (T.en_cb[e] < 0 || T.en_cb[e] > T.en_ce[e] || T.en_ce[e] > nt) return 5;
        if (!(T.en_maxdist[e] >= 0.f)) return 6;
    }
    for (int64_t j = 0; j < d; ++j) {
        if (T.rep[j] < 0 || T.rep[j] >= d) return 7;
        if (T.pos[T.rep[j]] < 0 || T.pos[T.rep[j]] >= nt) return 8;
    }
    if (static_cast<int64_t>(T.unit_atoms.size()) != nt * T.L) return 9;
    return 0;
}

int main() {
    std::mt19937_64 g(1810);
    std::normal_distribution<float> nd(0.f, 1.f);
    const int64_t ds[] = {1, 2, 3, 129, 300};
    const int Ls[] = {1, 7, 16};
    int failures = 0;
    for (int metric = 0; metric < 2; ++metric)
        for (int64_t d : ds)
            for (int L : Ls) {
                std::vector<std::complex<float>> a(static_cast<size_t>(d) * L);
                for (auto& x : a) x = {nd(g), nd(g)};
                if (d > 2) {           // an exact duplicate and a near duplicate
                    for (int t = 0; t < L; ++t) {
                        a[static_cast<size_t>(d - 1) * L + t] = a[t];
                        a[static_cast<size_t>(d - 2) * L + t] = a[L + t] * 1.0000001f;
                    }
                }
                CtParams P;
                P.atoms = a.data();
                P.d = d;
                P.L = L;
                P.metric = metric;
                CtTree T;
                const int rc = ct_build(P, &T);
                const int bad = rc ? 100 + rc : check(T, d);
                if (bad) {
                    std::printf("metric %d d %lld L %d: failure %d\n", metric,
                                static_cast<long long>(d), L, bad);
                    ++failures;
                }
            }
    std::printf(failures ? "FAILED\n" : "ok\n");
    return failures ? 1 : 0;
}
