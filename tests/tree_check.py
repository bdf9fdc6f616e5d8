"""Checks of an exported cover tree against the three invariants of §4.1 and the definition of
maxdist, with distances evaluated by the oracle (float64).  Tolerance 1e-6 relative: the builder
evaluates distances above 0.25 with FP32 sums."""
import numpy as np

from oracle import covertree as ct


def check_tree(A, T, cone="complex", dup_tol=1e-5, rel=1e-6):
    metric = "phase" if cone == "complex" else "euclid"
    U = ct.unit_atoms(np.asarray(A, np.complex64).astype(np.complex128))
    U = U.astype(np.complex64).astype(np.complex128)        # the builder's stored unit atoms
    G = ct.pair_dist(U, U, metric)
    G = 0.5 * (G + G.T)
    np.fill_diagonal(G, 0.0)
    s = T["sigma"]
    fl, par, rep = T["first_level"], T["parent"], T["rep"]
    nodes = np.flatnonzero(fl >= 0)
    dup = np.flatnonzero(fl < 0)
    assert np.all(rep[nodes] == nodes)
    assert np.all(G[dup, rep[dup]] <= dup_tol * (1 + rel) + 1e-9), "duplicates"
    assert fl[0] == 0 and par[0] == -1
    for q in nodes[nodes != 0]:
        assert fl[par[q]] < fl[q], "nesting: a parent appears above its child"
        assert G[q, par[q]] <= s * 2.0 ** (-(fl[q] - 1)) * (1 + rel), ("covering", q)
    for i in range(int(T["levels"]) + 1):
        net = nodes[fl[nodes] <= i]
        if len(net) > 1:
            sub = G[np.ix_(net, net)] + np.eye(len(net)) * 1e9
            assert sub.min() > s * 2.0 ** (-i) * (1 - rel), ("separation", i)
    children = {}
    for q in nodes[nodes != 0]:
        children.setdefault(int(par[q]), []).append(int(q))

    def desc(a, lvl):
        out = []
        for c in children.get(a, []):
            if fl[c] > lvl:
                out.append(c)
                out += desc(c, fl[c])
        return out

    for a, i, m in zip(T["en_atom"], T["en_level"], T["en_maxdist"]):
        D = desc(int(a), int(i))
        assert D, "explicit node without children"
        true = G[a, D].max()
        assert true * (1 - rel) - 1e-7 <= m <= true * (1 + 1e-5) + 1e-7, ("maxdist", a, i)
        assert true < s * 2.0 ** (-i + 1) * (1 + rel), "maxdist bound (eq. maxdistbound)"
    return len(nodes), len(dup)
