// Host-side cover tree representation shared by the builder (covertree_build.cpp) and the
// device upload / search (covertree.cu).
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

struct CtParams {
    const std::complex<float>* atoms = nullptr;   // host [d][L]
    int64_t d = 0;
    int L = 0;
    int metric = 0;          // 0 phase-quotient (complex cone), 1 euclidean (real cone)
    double dup_tol = 1e-5;   // atoms this close to an earlier node are duplicates
    int max_neighbours = 64; // neighbour-list cap per node (see covertree_build.cpp)
    int verbose = 0;         // per-level timing on stderr
};

struct CtTree {
    int64_t d = 0;
    int L = 0;
    int metric = 0;
    double sigma = 0.0;      // covering radius of the root (level 0)
    int imax = 0;            // deepest level (all distinct atoms are nodes there)
    // per atom (index = atom id)
    std::vector<int32_t> rep;          // representative tree node (itself unless duplicate)
    std::vector<int32_t> first_level;  // level at which the atom first appears (-1 duplicate)
    std::vector<int32_t> parent;       // parent atom at first_level - 1 (-1 root / duplicate)
    std::vector<int32_t> pos;          // BFS position (-1 duplicate)
    // per BFS position
    std::vector<int32_t> order;        // atom at each position (root at 0)
    std::vector<int32_t> node_first;   // [nt + 1] CSR of the explicit nodes of each position
    // explicit nodes (node at a level where it has new children), sorted by (position, level)
    std::vector<int32_t> en_parent;    // atom
    std::vector<int32_t> en_level;     // level i: the children first appear at i + 1
    std::vector<int32_t> en_cb, en_ce; // children occupy positions [cb, ce)
    std::vector<float> en_maxdist;     // max distance from the node to its subtree at level i
    std::vector<std::complex<float>> unit_atoms;   // [nt][L] unit atoms in BFS order
};

// Returns 0 on success.
int ct_build(const CtParams& params, CtTree* out);
