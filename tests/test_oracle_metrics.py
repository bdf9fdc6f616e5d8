"""Pins of the oracle's per-pair density and correlation (§3.2, eq. exactPs) and of its accuracy
metric (§6, evaluation metrics) against facts that do not come from those functions: the
hand-derived pairs of the golden fixture (one of them shows the conjugation side), numpy's
least-squares routine per voxel (complex cone) and the clipped real least-squares solution
(real positive cone), explicit loops over the frames, and a hand-computed accuracy.  Each pin
is also run on a planted mistake (wrong conjugation side, a dropped normalisation) to show
that it catches it."""
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


# planted mistakes (the oracle's formulas with one error each), to show the pins catch them
def _density_conj_wrong(Z, D, idx, cone="complex"):
    d = np.asarray(D, np.complex128)[idx]
    c = np.sum(d * np.conj(Z), axis=1) / np.sum(np.abs(d) ** 2, axis=1)     # z^H d
    return c if cone == "complex" else np.maximum(c.real, 0.0).astype(np.complex128)


def _density_unnormalised(Z, D, idx, cone="complex"):
    d = np.asarray(D, np.complex128)[idx]
    c = np.sum(np.conj(d) * Z, axis=1)                                        # no / ||d||^2
    return c if cone == "complex" else np.maximum(c.real, 0.0).astype(np.complex128)


def _corr_conj_wrong(Z, D, idx, cone="complex"):
    d = np.asarray(D, np.complex128)[idx]
    c = np.sum(d * Z, axis=1)                                                 # d^T z
    den = np.sqrt(np.sum(np.abs(d) ** 2, axis=1) * np.sum(np.abs(Z) ** 2, axis=1))
    return (np.abs(c) if cone == "complex" else c.real) / den


def _corr_unnormalised(Z, D, idx, cone="complex"):
    d = np.asarray(D, np.complex128)[idx]
    c = np.sum(np.conj(d) * Z, axis=1)
    den = np.sqrt(np.sum(np.abs(d) ** 2, axis=1))                             # no ||z||
    return (np.abs(c) if cone == "complex" else c.real) / den


def _gold_pairs():
    gold = json.load(open(GOLD))
    pr = gold["pairs"]
    D, Q = _c(gold["atoms"]), _c(gold["queries"])
    Z = Q[np.asarray(pr["query"])]
    idx = np.asarray(pr["atom"])
    return pr, D, Z, idx


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_golden_pairs(cone):
    pr, D, Z, idx = _gold_pairs()
    np.testing.assert_allclose(mo.density(Z, D, idx, cone), _c(pr[cone]["rho"]), atol=1e-15)
    np.testing.assert_allclose(mo.correlation(Z, D, idx, cone), pr[cone]["corr"], atol=1e-15)


def test_golden_pairs_catch_planted_mistakes():
    pr, D, Z, idx = _gold_pairs()
    for wrong in (_density_conj_wrong, _density_unnormalised):
        assert not np.allclose(wrong(Z, D, idx), _c(pr["complex"]["rho"]), atol=1e-9)
    for wrong in (_corr_conj_wrong, _corr_unnormalised):
        assert not np.allclose(wrong(Z, D, idx), pr["complex"]["corr"], atol=1e-9)
    assert not np.allclose(_corr_unnormalised(Z, D, idx, "real_pos"), pr["real_pos"]["corr"],
                           atol=1e-9)


def _density_lstsq(Z, D, idx, cone):
    """Per voxel: argmin_rho ||z - rho d|| by numpy's least squares; the real positive cone
    solves the real problem over [Re; Im] and clips at zero (exact for one nonnegative
    coefficient: the objective is a convex parabola in gamma)."""
    out = np.zeros(len(idx), np.complex128)
    for v, j in enumerate(idx):
        d, z = D[j], Z[v]
        if cone == "complex":
            sol, *_ = np.linalg.lstsq(d[:, None], z, rcond=None)
            out[v] = sol[0]
        else:
            A = np.concatenate([d.real, d.imag])[:, None]
            b = np.concatenate([z.real, z.imag])
            sol, *_ = np.linalg.lstsq(A, b, rcond=None)
            out[v] = max(sol[0], 0.0)
    return out


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_density_is_least_squares(cone):
    g = np.random.Generator(np.random.PCG64(21))
    D = _rand(g, 11, 9) * g.uniform(0.3, 3.0, (11, 1))
    Z = _rand(g, 40, 9)
    idx = g.integers(0, 11, 40)
    ref = _density_lstsq(Z, D, idx, cone)
    np.testing.assert_allclose(mo.density(Z, D, idx, cone), ref, rtol=1e-12, atol=1e-13)
    if cone == "real_pos":
        assert np.any(ref == 0.0) and np.any(ref.real > 0.0)   # both branches of the clip
    # the conjugation side leaves Re(.) unchanged, so only the complex cone can show it
    planted = (_density_conj_wrong, _density_unnormalised) if cone == "complex" \
        else (_density_unnormalised,)
    for wrong in planted:
        assert not np.allclose(wrong(Z, D, idx, cone), ref, rtol=1e-6, atol=1e-9)


def _corr_loop(Z, D, idx, cone):
    out = []
    for v, j in enumerate(idx):
        re = im = dd = zz = 0.0
        for t in range(D.shape[1]):
            a, b = D[j][t], Z[v][t]
            # conj(a) b = (a.re b.re + a.im b.im) + i (a.re b.im - a.im b.re)
            re += a.real * b.real + a.imag * b.imag
            im += a.real * b.imag - a.imag * b.real
            dd += a.real ** 2 + a.imag ** 2
            zz += b.real ** 2 + b.imag ** 2
        num = (re * re + im * im) ** 0.5 if cone == "complex" else re
        out.append(num / (dd * zz) ** 0.5)
    return np.array(out)


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_correlation_explicit_loop(cone):
    g = np.random.Generator(np.random.PCG64(22))
    D = _rand(g, 10, 7) * g.uniform(0.5, 2.0, (10, 1))
    Z = _rand(g, 30, 7) * g.uniform(0.1, 5.0, (30, 1))
    idx = g.integers(0, 10, 30)
    ref = _corr_loop(Z, D, idx, cone)
    np.testing.assert_allclose(mo.correlation(Z, D, idx, cone), ref, rtol=1e-12, atol=1e-14)
    assert np.all(np.abs(ref) <= 1.0 + 1e-12)                          # Cauchy-Schwarz
    for wrong in (_corr_conj_wrong, _corr_unnormalised):
        assert not np.allclose(wrong(Z, D, idx, cone), ref, rtol=1e-6, atol=1e-9)


def test_correlation_is_the_projection_score():
    """The best atom's correlation is the oracle projection's s1 and bounds every other atom."""
    g = np.random.Generator(np.random.PCG64(23))
    D = _rand(g, 25, 6)
    Z = _rand(g, 12, 6)
    r = mo.project(Z, D)
    np.testing.assert_allclose(mo.correlation(Z, D, r["idx"]), r["s1"], rtol=1e-13)
    for j in range(25):
        assert np.all(mo.correlation(Z, D, np.full(12, j)) <= r["s1"] + 1e-13)


def test_accuracy_hand_computed():
    truth = np.array([100.0, 200.0, 400.0, 800.0])
    mask = np.array([True, True, True, False])
    est = np.array([110.0, 180.0, 400.0, 0.0])        # 10 %, 10 %, 0 %; the 4th is masked out
    assert mo.accuracy(est, truth, mask) == pytest.approx(1.0 - 0.2 / 3, abs=1e-15)
    assert mo.accuracy(truth, truth, mask) == 1.0
    # over-estimates count like under-estimates (absolute relative error)
    assert mo.accuracy(np.array([90.0, 220.0, 400.0, 1.0]), truth, mask) == \
        pytest.approx(1.0 - 0.2 / 3, abs=1e-15)
    # the error is relative to the truth, not to the estimate
    assert mo.accuracy(np.array([200.0]), np.array([100.0]), np.array([True])) == \
        pytest.approx(0.0, abs=1e-15)
