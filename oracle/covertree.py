"""Textbook cover tree and its (1+eps)-approximate nearest-neighbour search (§4.1, Algorithm 1).

TEST INFRASTRUCTURE (see the package docstring): never imported by the product path.

Metric.  The complex cone identifies a fingerprint with all its phase rotations, so the tree is
built on the unit atoms u_j = D_j / ||D_j|| (float64) with the phase-quotient distance
    delta(x, y) = min_phi ||x - e^{i phi} y|| = sqrt(||x||^2 + ||y||^2 - 2 |x^H y|),
a metric on C^L / U(1) (U(1) acts by isometries).  For a unit query z^ its nearest atom is
argmax_j |D_j^H z| / ||D_j||, i.e. the exact complex-cone projection.  ``metric="euclid"``
uses ||x - y|| (the paper's real-positive setting).

Construction (from the three invariants of §4.1; the paper relies on existing code for it):
  S_0 = {root}, root = atom 0, sigma = max_j delta(root, u_j).
  S_{i+1} = S_i plus, scanning the remaining atoms in index order, every atom farther than
  sigma 2^-(i+1) from all nodes already in S_{i+1} (a maximal separated net, so every atom is
  within sigma 2^-i of S_i, which gives covering).  A new node's parent is its nearest node in
  S_i (ties to the smaller index); an old node is its own parent (nesting).  Exact duplicates
  (delta = 0 up to float64 rounding) never separate: each is represented by its smallest index.
  i_max is the first level whose net holds every distinct atom.
  maxdist(q, i) is the exact largest distance from q to the atoms of its subtree.

Search (Algorithm 1): candidate sets Q_i per level, the current best q_c (warm start or the
root), and the refinement Q_{i+1} = {q in children(Q_i): delta(p,q) <= dist_min + maxdist(q)}.
The loop runs while i < i_max and sigma 2^(-i+1) (1 + 1/eps) > dist_min (eps = 0: always).  The
root's distance is evaluated at initialisation, so every candidate's distance is known -- the
(1+eps) bound of Definition eNN follows from the covering radius of the candidates' subtrees.
"""
from __future__ import annotations

import numpy as np


def unit_atoms(D) -> np.ndarray:
    D = np.asarray(D, np.complex128)
    return D / np.linalg.norm(D, axis=1)[:, None]


def pair_dist(A, B, metric="phase", chunk=8) -> np.ndarray:
    """delta between rows of A and rows of B, float64 [len(A), len(B)].

    Evaluated as the norm of the difference with the optimal phase applied,
    ||a - u b|| with u = (b^H a) / |b^H a| (u = 1 for the Euclidean metric), which keeps full
    relative accuracy for nearby points (the expanded form loses it to cancellation).
    """
    A = np.asarray(A, np.complex128)
    B = np.asarray(B, np.complex128)
    g = A @ B.conj().T
    if metric == "phase":
        mag = np.abs(g)
        u = np.where(mag > 0, g / np.where(mag > 0, mag, 1.0), 1.0)
    else:
        u = np.ones_like(g)
    out = np.empty(g.shape)
    for a in range(0, A.shape[0], chunk):
        diff = A[a:a + chunk, None, :] - u[a:a + chunk, :, None] * B[None, :, :]
        out[a:a + chunk] = np.sqrt(np.sum(diff.real ** 2 + diff.imag ** 2, axis=2))
    return out


DUP_TOL = 1e-12        # delta this small is zero up to float64 rounding


class CoverTree:
    def __init__(self, D, metric: str = "phase"):
        self.metric = metric
        self.U = unit_atoms(D)
        d = self.U.shape[0]
        G = pair_dist(self.U, self.U, metric)           # full distance table (tiny d only)
        G = 0.5 * (G + G.T)
        np.fill_diagonal(G, 0.0)
        self.G = G
        # duplicates: represented by their smallest index
        rep = np.arange(d)
        for j in range(d):
            if rep[j] != j:
                continue
            dup = np.flatnonzero(G[j] <= DUP_TOL)
            dup = dup[dup > j]
            rep[dup] = j
        self.rep = rep
        distinct = np.flatnonzero(rep == np.arange(d))
        self.root = 0
        self.sigma = float(G[0, distinct].max())
        levels = [[0]]
        parent = [{0: None}]
        in_net = np.zeros(d, bool)
        in_net[0] = True
        i = 0
        while not in_net[distinct].all():
            r = self.sigma * 2.0 ** (-(i + 1))
            net = list(levels[i])
            par = {q: q for q in levels[i]}
            for p in distinct:
                if in_net[p]:
                    continue
                if np.all(G[p, net] > r):
                    net.append(p)
                    in_net[p] = True
                    prev = np.asarray(levels[i])
                    dd = G[p, prev]
                    par[p] = int(prev[np.flatnonzero(dd == dd.min())[0]])
            levels.append(net)
            parent.append(par)
            i += 1
            if self.sigma == 0.0:
                break
        self.levels = levels                 # levels[i] = S_i (atom ids)
        self.parent = parent                 # parent[i+1][q] = parent of q at level i
        self.imax = len(levels) - 1
        self.children = []                   # children[i][p] = nodes of S_{i+1} under p
        for i in range(self.imax):
            ch = {p: [] for p in levels[i]}
            for q, p in parent[i + 1].items():
                ch[p].append(q)
            self.children.append(ch)
        # exact maxdist(q, i) over the subtree of node (q, i)
        self.desc = [None] * (self.imax + 1)
        self.desc[self.imax] = {q: [q] for q in levels[self.imax]}
        for i in range(self.imax - 1, -1, -1):
            self.desc[i] = {p: [a for c in self.children[i][p] for a in self.desc[i + 1][c]]
                            for p in levels[i]}
        self.maxdist = [{q: float(G[q, self.desc[i][q]].max()) for q in levels[i]}
                        for i in range(self.imax + 1)]

    # -- invariants of §4.1 ---------------------------------------------------------------------
    def check_invariants(self) -> None:
        G, s = self.G, self.sigma
        for i in range(self.imax):
            assert set(self.levels[i]) <= set(self.levels[i + 1]), "nesting"
            for q, p in self.parent[i + 1].items():
                assert p in self.levels[i]
                assert G[p, q] <= s * 2.0 ** (-i) * (1 + 1e-12), "covering"
        for i in range(self.imax + 1):
            net = np.asarray(self.levels[i])
            if len(net) > 1:
                sub = G[np.ix_(net, net)] + np.eye(len(net)) * 1e300
                assert sub.min() > s * 2.0 ** (-i), "separation"
        for i in range(self.imax + 1):
            for q in self.levels[i]:
                assert self.maxdist[i][q] < s * 2.0 ** (-i + 1) or self.maxdist[i][q] == 0.0, \
                    "maxdist bound (eq. maxdistbound)"
        distinct = np.flatnonzero(self.rep == np.arange(len(self.rep)))
        assert set(self.levels[self.imax]) == set(distinct.tolist())

    # -- Algorithm 1 ------------------------------------------------------------------------------
    def search(self, p, eps: float, warm: int | None = None) -> tuple[int, int]:
        """(1+eps)-ANNS of the unit query p; returns (atom index, distance evaluations)."""
        p = np.asarray(p, np.complex128)

        def dist(q):
            return float(pair_dist(p[None, :], self.U[[q]], self.metric)[0, 0])

        evals = 0
        known = {}
        qc = self.root if warm is None else int(self.rep[warm])
        known[qc] = dist(qc)
        evals += 1
        if self.root not in known:
            known[self.root] = dist(self.root)
            evals += 1
        dmin = known[qc]
        if known[self.root] < dmin:
            qc, dmin = self.root, known[self.root]
        Q = [self.root]
        i = 0
        while i < self.imax and (eps == 0.0 or
                                 self.sigma * 2.0 ** (-i + 1) * (1.0 + 1.0 / eps) > dmin):
            cand = [c for q in Q for c in self.children[i][q]]
            if not cand:
                break
            dd = {}
            for c in cand:
                if c not in known:
                    known[c] = dist(c)
                    evals += 1
                dd[c] = known[c]
            qs = min(cand, key=lambda c: (dd[c], c))
            if dd[qs] < dmin:
                dmin, qc = dd[qs], qs
            Q = [c for c in cand if dd[c] <= dmin + self.maxdist[i + 1][c]]
            i += 1
        return int(qc), evals

    def brute(self, p) -> tuple[int, float]:
        """Exact nearest atom by exhaustive search (ties to the smallest index)."""
        dd = pair_dist(np.asarray(p)[None, :], self.U, self.metric)[0]
        j = int(np.argmin(dd))
        return j, float(dd[j])

    def dist_to(self, p, j) -> float:
        return float(pair_dist(np.asarray(p)[None, :], self.U[[j]], self.metric)[0, 0])
