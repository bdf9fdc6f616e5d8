"""Pins of the oracle's exact projection (§3.2, eqs. exactP / exactPs) against facts that do not
come from the oracle itself: a hand-derived fixture, per-pair least squares, an explicit loop,
the atom-times-scalar identity, tie and zero-query rules."""
import json
import os

import numpy as np
import pytest

from oracle import mrf_oracle as mo

GOLD = os.path.join(os.path.dirname(__file__), "golden", "projection_small.json")


def _c(a):
    a = np.asarray(a, np.float64)
    return a[..., 0] + 1j * a[..., 1]


def _rand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_golden_small(cone):
    gold = json.load(open(GOLD))
    D, Z = _c(gold["atoms"]), _c(gold["queries"])
    r = mo.project(Z, D, cone)
    assert r["idx"].tolist() == gold[cone]["idx"]
    np.testing.assert_allclose(r["rho"], _c(gold[cone]["rho"]), atol=1e-15)


def test_least_squares_per_pair():
    """min_rho ||z - rho d|| solved by numpy's least-squares routine for every (voxel, atom)."""
    g = np.random.Generator(np.random.PCG64(11))
    D = _rand(g, 9, 6) * g.uniform(0.3, 3.0, (9, 1))
    Z = _rand(g, 7, 6)
    r = mo.project(Z, D)
    for v in range(Z.shape[0]):
        best = None
        for j in range(D.shape[0]):
            sol, res, *_ = np.linalg.lstsq(D[j][:, None], Z[v], rcond=None)
            resid = float(np.linalg.norm(Z[v] - D[j] * sol[0]))
            if best is None or resid < best[0]:
                best = (resid, j, sol[0])
        assert r["idx"][v] == best[1]
        assert abs(r["rho"][v] - best[2]) < 1e-12


def test_explicit_loop_real_pos():
    """Paper's rule: j* = argmin_j ||z - D_j/||D_j|| ||, gamma = max(Re<z,D_j*>/||D_j*||^2, 0)."""
    g = np.random.Generator(np.random.PCG64(12))
    D = _rand(g, 8, 5) * g.uniform(0.5, 2.0, (8, 1))
    Z = _rand(g, 6, 5)
    r = mo.project(Z, D, "real_pos")
    for v in range(Z.shape[0]):
        dist = [sum(abs(Z[v][t] - D[j][t] / np.sqrt(sum(abs(x) ** 2 for x in D[j]))) ** 2
                    for t in range(5)) for j in range(8)]
        j = int(np.argmin(dist))
        inner = sum(np.conj(D[j][t]) * Z[v][t] for t in range(5))
        gam = max(inner.real / sum(abs(x) ** 2 for x in D[j]), 0.0)
        assert r["idx"][v] == j
        assert abs(r["rho"][v] - gam) < 1e-12


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_atom_times_scalar(cone):
    """z = rho D_j projects back to exactly (j, rho) (cone membership, eq. conedef)."""
    import mrfgen
    dic = mrfgen.make_dictionary(1)
    D = dic["atoms"]
    g = np.random.Generator(np.random.PCG64(13))
    js = g.choice(D.shape[0], 40, replace=False)
    rho = g.uniform(0.2, 2.0, 40) * (np.exp(1j * g.uniform(0, 2 * np.pi, 40))
                                     if cone == "complex" else 1.0)
    Z = rho[:, None] * D[js].astype(np.complex128)
    r = mo.project(Z, D, cone)
    assert np.array_equal(r["idx"], js)
    np.testing.assert_allclose(r["rho"], rho, rtol=1e-12, atol=1e-12)


def test_planted_conjugation_error_is_caught():
    """Planting the wrong conjugation side (D^T z instead of D^H z) breaks the scalar pin."""
    g = np.random.Generator(np.random.PCG64(14))
    D = _rand(g, 12, 10)
    js = np.arange(12)
    rho = np.exp(1j * g.uniform(0, 2 * np.pi, 12))
    Z = rho[:, None] * D[js]
    bad = mo.project(Z, np.conj(D))          # the oracle run with the mistake planted
    ok = np.array_equal(bad["idx"], js) and np.allclose(bad["rho"], rho, atol=1e-9)
    assert not ok


def test_ties_and_zero_query():
    D = np.array([[1, 0], [1, 0], [0, 1]], np.complex128)
    Z = np.array([[2, 0], [0, 0], [0, 3j]], np.complex128)
    r = mo.project(Z, D)
    assert r["idx"].tolist() == [0, 0, 2]
    np.testing.assert_allclose(r["rho"], [2, 0, 3j])


def test_phase_and_scale_invariance_of_argmax():
    g = np.random.Generator(np.random.PCG64(15))
    D = _rand(g, 30, 8)
    Z = _rand(g, 20, 8)
    a = mo.project(Z, D)
    b = mo.project(Z * 3.7 * np.exp(1j * 0.9), D)
    assert np.array_equal(a["idx"], b["idx"])
    np.testing.assert_allclose(b["rho"], a["rho"] * 3.7 * np.exp(1j * 0.9), rtol=1e-12)


def test_residual_is_minimal_against_perturbations():
    """The returned rho D_j* is no farther from z than any atom with any perturbed scalar."""
    g = np.random.Generator(np.random.PCG64(16))
    D = _rand(g, 15, 7)
    Z = _rand(g, 10, 7)
    r = mo.project(Z, D)
    for v in range(10):
        best = np.linalg.norm(Z[v] - r["rho"][v] * D[r["idx"][v]])
        for j in range(15):
            opt = np.vdot(D[j], Z[v]) / np.vdot(D[j], D[j])
            for _ in range(20):
                rho = opt + (g.standard_normal() + 1j * g.standard_normal()) * 0.3
                assert np.linalg.norm(Z[v] - rho * D[j]) >= best - 1e-12
