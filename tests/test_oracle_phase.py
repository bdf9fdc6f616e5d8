"""Pins of the phase-aligned projection oracle (§4.3): any complex multiple of an atom is
recovered exactly (index and complex density), real positive atoms and queries reduce it to the
plain real positive projection, and the aligned score never exceeds the complex-cone score."""
import numpy as np

from oracle import mrf_oracle as mo
from oracle import phase


def _dictionary(seed, d=60, L=32, real=False):
    g = np.random.Generator(np.random.PCG64(seed))
    base = np.abs(g.standard_normal((d, L))) + 0.1          # positive profiles
    if real:
        A = base.astype(np.complex128)
    else:
        A = base * np.exp(1j * (g.uniform(0, 2 * np.pi, (d, 1)) + 0.3 * g.standard_normal((d, L))))
    return A / np.linalg.norm(A, axis=1, keepdims=True), g


def test_complex_multiples_of_atoms_are_recovered():
    A, g = _dictionary(1)
    js = g.integers(0, A.shape[0], 200)
    c = g.uniform(0.2, 3.0, 200) * np.exp(1j * g.uniform(0, 2 * np.pi, 200))
    Z = c[:, None] * A[js]
    r = phase.project_phase_aligned(Z, A)
    assert np.array_equal(r["idx"], js)
    np.testing.assert_allclose(r["rho"], c, rtol=1e-12)


def test_real_positive_data_reduces_to_the_real_cone():
    A, g = _dictionary(2, real=True)
    Z = np.abs(g.standard_normal((100, A.shape[1]))) + 0.05
    r = phase.project_phase_aligned(Z, A)
    ref = mo.project(Z, A, "real_pos")
    assert np.array_equal(r["idx"], ref["idx"])
    np.testing.assert_allclose(r["rho"], ref["rho"], rtol=1e-12)
    assert np.allclose(r["ea"], 1.0) and np.allclose(r["eb"], 1.0)


def test_aligned_score_is_bounded_by_the_complex_score():
    A, g = _dictionary(3)
    Z = g.standard_normal((150, A.shape[1])) + 1j * g.standard_normal((150, A.shape[1]))
    r = phase.project_phase_aligned(Z, A)
    c = mo.project(Z, A, "complex")
    assert np.all(r["s1"] <= c["s1"] + 1e-12)


def test_unit_phase_values():
    """e^{i theta} of r e^{i theta} for r > 0, and 1 for a zero value (no phase to remove)."""
    th = np.array([0.0, 0.5, -2.0, np.pi])
    r = np.array([3.0, 1e-20, 7.0, 0.25])
    np.testing.assert_allclose(phase.unit_phase(r * np.exp(1j * th)), np.exp(1j * th), atol=1e-15)
    assert phase.unit_phase(np.array([0j]))[0] == 1.0
