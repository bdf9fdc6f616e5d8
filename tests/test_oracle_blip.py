"""Pins of the oracle's forward model, gradient step and BLIP iteration (§3, eq. forward;
§3.2, eq. blip; Algorithm 2 and the step rule eq. steprule; Theorem inexactmonotone)."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo


def _rand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_dft_matches_explicit_matrix():
    """F is the unitary 2-D DFT: compare with an explicitly built DFT matrix (brute force)."""
    g = np.random.Generator(np.random.PCG64(21))
    Ny, Nx, L = 6, 5, 3
    X = _rand(g, Ny * Nx, L)
    masks = np.ones((L, Ny), np.uint8)
    Y = mo.forward(X, masks, Ny, Nx)
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(Ny), np.arange(Ny)) / Ny) / np.sqrt(Ny)
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(Nx), np.arange(Nx)) / Nx) / np.sqrt(Nx)
    for t in range(L):
        img = X[:, t].reshape(Ny, Nx)
        np.testing.assert_allclose(Y[:, :, t], Fy @ img @ Fx.T, atol=1e-12)


def test_adjoint_identity():
    g = np.random.Generator(np.random.PCG64(22))
    Ny, Nx, L = 16, 12, 7
    masks = mrfgen.line_masks(Ny, L, 4.0, 5)
    X = _rand(g, Ny * Nx, L)
    Y = _rand(g, Ny, Nx, L)
    lhs = np.vdot(Y, mo.forward(X, masks, Ny, Nx))
    rhs = np.vdot(mo.adjoint(Y, masks, Ny, Nx), X)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_full_sampling_is_unitary_and_y_only_identity():
    """Full masks: A^H A = I.  Line masks: A^H A = F_y^H P_t F_y per frame (F_x cancels)."""
    g = np.random.Generator(np.random.PCG64(23))
    Ny, Nx, L = 8, 6, 5
    X = _rand(g, Ny * Nx, L)
    full = np.ones((L, Ny), np.uint8)
    np.testing.assert_allclose(mo.adjoint(mo.forward(X, full, Ny, Nx), full, Ny, Nx), X,
                               atol=1e-12)
    m = mrfgen.line_masks(Ny, L, 2.0, 9)
    aha = mo.adjoint(mo.forward(X, m, Ny, Nx), m, Ny, Nx).reshape(Ny, Nx, L)
    ky = np.fft.fft(X.reshape(Ny, Nx, L), axis=0, norm="ortho") * m.T[:, None, :]
    np.testing.assert_allclose(np.fft.ifft(ky, axis=0, norm="ortho"), aha, atol=1e-12)


@pytest.fixture(scope="module")
def dic1():
    return mrfgen.make_dictionary(1)


def test_noiseless_full_sampling_exact_recovery(dic1):
    """Noiseless, fully sampled, on-grid phantom: one iteration recovers the truth exactly."""
    p = mrfgen.make_problem(1, dic=dic1, snap=True, full_sampling=True, noiseless=True)
    r = mo.blip(p["Y"], p["masks"], dic1["atoms"], p["Ny"], p["Nx"], iters=1)
    fg = p["phantom"]["labels"] >= 0
    assert np.array_equal(r["idx"][fg], p["truth_idx"][fg])
    np.testing.assert_allclose(r["rho"][fg], p["phantom"]["rho"][fg], rtol=1e-6)
    est = mo.lut(r["idx"], dic1["params"])
    np.testing.assert_array_equal(est[fg, 0], p["phantom"]["T1"][fg].astype(np.float32))
    np.testing.assert_array_equal(est[fg, 1], p["phantom"]["T2"][fg].astype(np.float32))
    assert np.all(np.abs(r["rho"][~fg]) < 1e-6)   # Y is stored in complex64


def test_tm_is_first_iteration(dic1):
    """Template matching = the first BLIP iteration from X^0 = 0 (§3.2, Table algs)."""
    p = mrfgen.make_problem(1, dic=dic1)
    r = mo.blip(p["Y"], p["masks"], dic1["atoms"], p["Ny"], p["Nx"], iters=1, mu=1.0)
    tm = mo.project(mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]), dic1["atoms"])
    assert np.array_equal(r["idx"], tm["idx"])
    np.testing.assert_allclose(r["rho"], tm["rho"], rtol=1e-12, atol=1e-15)


def test_adaptive_step_monotone_fidelity_and_bound(dic1):
    """With the step rule, ||Y - A X^k|| is non-increasing (Theorem inexactmonotone) and each
    iteration shrinks at most ceil(log_zeta(beta mu)) + 1 times with beta <= ||A||^2 = 1
    (Proposition stepbound)."""
    p = mrfgen.make_problem(1, dic=dic1)
    mu = p["Ny"] / p["masks"].sum(1).mean()
    r = mo.blip(p["Y"], p["masks"], dic1["atoms"], p["Ny"], p["Nx"], iters=8, mu=mu,
                adaptive=True, history=True)
    f = np.asarray(r["history"]["fidelity"])
    assert np.all(np.diff(f) <= 1e-12)
    assert max(r["history"]["shrinks"]) <= int(np.ceil(np.log2(mu))) + 1


def test_iterations_improve_on_tm(dic1):
    p = mrfgen.make_problem(1, dic=dic1)
    fg = p["phantom"]["labels"] >= 0
    accs = []
    for it in (1, 10):
        r = mo.blip(p["Y"], p["masks"], dic1["atoms"], p["Ny"], p["Nx"], iters=it)
        est = mo.lut(r["idx"], dic1["params"])
        accs.append(mo.accuracy(est[:, 0], p["phantom"]["T1"], fg))
    assert accs[1] > accs[0]
    assert accs[1] > 0.85


def _objective(X, Y, masks, Ny, Nx):
    """f(X) = 1/2 ||A(X) - Y||^2, the data-fidelity term whose gradient step eq. blip takes."""
    R = mo.forward(X, masks, Ny, Nx) - Y
    return 0.5 * float(np.sum(np.abs(R) ** 2))


def test_gradient_step_is_the_fidelity_gradient():
    """(X - Z) / mu is the gradient of f at X, checked by central differences along random
    complex directions (partial line masks): 2 eps Re<grad, E> = f(X + eps E) - f(X - eps E)
    exactly for a quadratic."""
    g = np.random.Generator(np.random.PCG64(31))
    Ny, Nx, L, mu = 8, 6, 5, 0.7
    masks = (g.random((L, Ny)) < 0.5).astype(np.uint8)
    X, X0 = _rand(g, Ny * Nx, L), _rand(g, Ny * Nx, L)
    Y = mo.forward(X0, masks, Ny, Nx) + 0.1 * _rand(g, Ny, Nx, L) * masks.T[:, None, :]
    grad = (X - mo.gradient_step(X, Y, masks, Ny, Nx, mu)) / mu
    eps = 1e-3
    for _ in range(4):
        E = _rand(g, Ny * Nx, L)
        fd = (_objective(X + eps * E, Y, masks, Ny, Nx)
              - _objective(X - eps * E, Y, masks, Ny, Nx)) / (2 * eps)
        assert abs(fd - float(np.real(np.vdot(grad, E)))) <= 1e-9 * max(1.0, abs(fd))


def test_gradient_step_special_cases():
    """Full sampling (A^H A = I): Z = (1 - mu) X + mu X0 for Y = A X0.  No sampled line
    (A = 0, Y = 0): Z = X."""
    g = np.random.Generator(np.random.PCG64(32))
    Ny, Nx, L, mu = 8, 4, 3, 0.3
    X, X0 = _rand(g, Ny * Nx, L), _rand(g, Ny * Nx, L)
    full = np.ones((L, Ny), np.uint8)
    Z = mo.gradient_step(X, mo.forward(X0, full, Ny, Nx), full, Ny, Nx, mu)
    np.testing.assert_allclose(Z, (1 - mu) * X + mu * X0, atol=1e-12)
    none = np.zeros((L, Ny), np.uint8)
    Z = mo.gradient_step(X, np.zeros((Ny, Nx, L), complex), none, Ny, Nx, mu)
    np.testing.assert_allclose(Z, X, atol=0)


def test_rescale_reproduces_complex_multiples_of_atoms():
    """Projection then rescale (eq. exactPs) maps rho D_k back to itself for any complex rho."""
    g = np.random.Generator(np.random.PCG64(33))
    D = _rand(g, 40, 12)
    k = g.integers(0, 40, 9)
    rho = _rand(g, 9)
    Z = rho[:, None] * D[k]
    r = mo.project(Z, D)
    np.testing.assert_array_equal(r["idx"], k)
    np.testing.assert_allclose(mo.rescale(r["idx"], r["rho"], D), Z, atol=1e-12)


def test_nmse_values():
    g = np.random.Generator(np.random.PCG64(34))
    X0 = _rand(g, 10, 4)
    assert mo.nmse(X0, X0) == 0.0
    assert mo.nmse(2 * X0, X0) == pytest.approx(1.0)
    assert mo.nmse(np.zeros_like(X0), X0) == pytest.approx(1.0)
