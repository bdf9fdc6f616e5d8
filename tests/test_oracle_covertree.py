"""Pins of the oracle cover tree (§4.1): the three invariants and the maxdist bound, exactness of
eps = 0 against brute force, the (1+eps) guarantee of Definition eNN, warm-start
non-expansiveness (§4.3) and the metric axioms of the phase-quotient distance."""
import numpy as np
import pytest

import mrfgen
from oracle import covertree as ct
from oracle import mrf_oracle as mo


def _rand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


@pytest.fixture(scope="module")
def small_dic():
    d = mrfgen.make_dictionary(1, L=32, t1t2=300)
    return d["atoms"]


def _queries(D, g, n=60, noise=0.3):
    j = g.integers(0, D.shape[0], n)
    Z = np.asarray(D, np.complex128)[j] * np.exp(1j * g.uniform(0, 6.3, n))[:, None]
    Z = Z + noise * _rand(g, n, D.shape[1]) / np.sqrt(D.shape[1])
    return Z / np.linalg.norm(Z, axis=1)[:, None]


def test_metric_axioms():
    g = np.random.Generator(np.random.PCG64(31))
    P = _rand(g, 200, 6)
    P /= np.linalg.norm(P, axis=1)[:, None]
    Dm = ct.pair_dist(P, P)
    assert np.allclose(Dm, Dm.T)
    assert np.all(np.diag(Dm) < 1e-7)
    for a, b, c in g.integers(0, 200, (3000, 3)):
        assert Dm[a, c] <= Dm[a, b] + Dm[b, c] + 1e-12
    # phase quotient: rotations are at distance zero, and delta = min over phi by scanning phi
    assert ct.pair_dist(P[:1], P[:1] * np.exp(1.3j))[0, 0] < 1e-7
    phi = np.linspace(0, 2 * np.pi, 20001)
    scan = np.min(np.linalg.norm(P[0][None, :] - np.exp(1j * phi)[:, None] * P[1][None, :],
                                 axis=1))
    assert abs(scan - Dm[0, 1]) < 1e-6


@pytest.mark.parametrize("which", ["random", "epg", "dups"])
def test_invariants(which, small_dic):
    g = np.random.Generator(np.random.PCG64(32))
    if which == "random":
        D = _rand(g, 150, 4)
    elif which == "epg":
        D = small_dic
    else:
        D = _rand(g, 40, 3)
        D = np.concatenate([D, D[:10] * np.exp(0.7j), D[5:8]])
    tree = ct.CoverTree(D)
    tree.check_invariants()
    if which == "dups":
        assert tree.rep[40] == 0 and tree.rep[50] == 5


def test_eps0_equals_brute_force(small_dic):
    tree = ct.CoverTree(small_dic)
    g = np.random.Generator(np.random.PCG64(33))
    for p in _queries(small_dic, g):
        j, _ = tree.search(p, 0.0)
        jb, db = tree.brute(p)
        assert abs(tree.dist_to(p, j) - db) <= 1e-12


@pytest.mark.parametrize("eps", [0.2, 0.5, 1.0])
def test_eps_guarantee_and_warm_start(eps, small_dic):
    tree = ct.CoverTree(small_dic)
    g = np.random.Generator(np.random.PCG64(34))
    Q = _queries(small_dic, g, noise=0.6)
    for p in Q:
        _, db = tree.brute(p)
        j, _ = tree.search(p, eps)
        assert tree.dist_to(p, j) <= (1 + eps) * db + 1e-12
        warm = int(g.integers(0, small_dic.shape[0]))
        jw, _ = tree.search(p, eps, warm=warm)
        assert tree.dist_to(p, jw) <= tree.dist_to(p, warm) + 1e-12
        assert tree.dist_to(p, jw) <= (1 + eps) * db + 1e-12


def test_tree_nn_is_complex_cone_projection(small_dic):
    """The phase-quotient nearest atom of z/||z|| is the exact complex-cone projection."""
    tree = ct.CoverTree(small_dic)
    g = np.random.Generator(np.random.PCG64(35))
    Q = _queries(small_dic, g) * 2.5
    ref = mo.project(Q, small_dic)
    for v, p in enumerate(Q):
        j, _ = tree.search(p / np.linalg.norm(p), 0.0)
        sj = mo.correlation(p[None], small_dic, np.array([j]))[0]
        assert sj >= ref["s1"][v] * (1 - 1e-12)


def test_search_cost_below_brute_force(small_dic):
    tree = ct.CoverTree(small_dic)
    g = np.random.Generator(np.random.PCG64(36))
    Q = _queries(small_dic, g, noise=0.05)
    evals = [tree.search(p, 0.5)[1] for p in Q]
    assert np.mean(evals) < 0.5 * small_dic.shape[0]


def test_unit_atoms_keep_direction_and_phase():
    """u_j = D_j / ||D_j||: unit rows, and D_j is a positive multiple of u_j."""
    g = np.random.Generator(np.random.PCG64(51))
    D = (g.standard_normal((6, 9)) + 1j * g.standard_normal((6, 9))) * g.uniform(0.1, 5, (6, 1))
    U = ct.unit_atoms(D)
    np.testing.assert_allclose(np.linalg.norm(U, axis=1), 1.0, atol=1e-14)
    ratio = D / U
    np.testing.assert_allclose(ratio.imag, 0.0, atol=1e-12)
    assert np.all(ratio.real > 0)
    np.testing.assert_allclose(ratio.real, np.linalg.norm(D, axis=1)[:, None] * np.ones((1, 9)))
