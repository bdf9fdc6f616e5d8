"""Pins of the oracle network: central finite differences of every parameter gradient, the
closed form of Adam's first step, tabulated GELU values, invariances of the canonical input."""
import numpy as np
import pytest

from oracle import mlp


def test_gelu_values_and_derivative():
    # x * Phi(x) with Phi(1) = 0.8413447460685429 (standard normal CDF)
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) < 1e-15
    x = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_gradients_by_finite_differences():
    g = np.random.Generator(np.random.PCG64(41))
    p = mlp.init(10, n_hidden=7, n_out=3, seed=3)
    for k in p:
        if k.startswith("b"):
            p[k] = g.normal(0, 0.3, p[k].shape)
    x = g.normal(size=(5, 10))
    t = g.normal(size=(5, 3))
    y, cache = mlp.forward(p, x)
    loss, dy = mlp.mse(y, t)
    grads = mlp.backward(p, cache, dy)
    h = 1e-6
    for k in p:
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            ix = it.multi_index
            old = p[k][ix]
            p[k][ix] = old + h
            lp, _ = mlp.mse(mlp.forward(p, x)[0], t)
            p[k][ix] = old - h
            lm, _ = mlp.mse(mlp.forward(p, x)[0], t)
            p[k][ix] = old
            assert abs((lp - lm) / (2 * h) - grads[k][ix]) < 1e-7, (k, ix)


def test_adam_first_step_closed_form():
    """First Adam step: m^ = g, v^ = g^2, so each weight moves by -lr g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    gr = {"w": np.array([0.3, -0.01, 0.0])}
    st = {}
    mlp.adam(p, gr, st, lr=0.1)
    expect = np.array([1.0, -2.0, 0.5]) - 0.1 * gr["w"] / (np.abs(gr["w"]) + 1e-8)
    np.testing.assert_allclose(p["w"], expect, rtol=1e-12)


def test_canonical_input_invariances():
    g = np.random.Generator(np.random.PCG64(42))
    D = g.normal(size=(50, 8)) + 1j * g.normal(size=(50, 8))
    v1 = mlp.dominant_vector(D)
    w, V = np.linalg.eigh(D.conj().T @ D)
    assert abs(abs(np.vdot(V[:, -1], v1)) - 1) < 1e-10
    Z = g.normal(size=(6, 8)) + 1j * g.normal(size=(6, 8))
    a = mlp.canonicalise(Z, v1)
    b = mlp.canonicalise(Z * 4.2 * np.exp(2.1j), v1)
    np.testing.assert_allclose(a, b, atol=1e-12)
    np.testing.assert_allclose(np.sum(a * a, axis=1), 1.0, rtol=1e-12)
