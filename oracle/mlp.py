"""Float64 oracle of the learned proposal network (fingerprint -> (log T1, log T2, B0)).

TEST INFRASTRUCTURE (see the package docstring): never imported by the product path.

Network: x in R^{2L} -> h1 = x W1 + b1 -> a1 = gelu(h1) -> h2 = a1 W2 + b2 -> a2 = gelu(h2)
-> y = a2 W3 + b3 in R^3, with gelu(x) = x Phi(x) (Phi the standard normal CDF).  Loss: mean
squared error over batch and outputs.  Optimiser: Adam with bias correction.
Input canonicalisation for the complex cone: z^ = z / ||z||, rotated by exp(-i angle(v1^H z^))
with v1 the dictionary's dominant right singular vector, laid out [Re t0, Im t0, Re t1, ...].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def init(n_in: int, n_hidden: int = 512, n_out: int = 3, seed: int = 5000) -> dict:
    g = np.random.Generator(np.random.PCG64(seed))
    p = {}
    dims = [(n_in, n_hidden), (n_hidden, n_hidden), (n_hidden, n_out)]
    for k, (a, b) in enumerate(dims, 1):
        p[f"W{k}"] = g.normal(0.0, np.sqrt(2.0 / a), size=(a, b))
        p[f"b{k}"] = np.zeros(b)
    return p


def forward(p: dict, x: np.ndarray):
    h1 = x @ p["W1"] + p["b1"]
    a1 = gelu(h1)
    h2 = a1 @ p["W2"] + p["b2"]
    a2 = gelu(h2)
    y = a2 @ p["W3"] + p["b3"]
    return y, (x, h1, a1, h2, a2)


def mse(y, t):
    r = y - t
    return float(np.mean(r * r)), 2.0 * r / r.size


def backward(p: dict, cache, dy) -> dict:
    x, h1, a1, h2, a2 = cache
    g = {"W3": a2.T @ dy, "b3": dy.sum(0)}
    da2 = dy @ p["W3"].T
    dh2 = da2 * gelu_grad(h2)
    g["W2"] = a1.T @ dh2
    g["b2"] = dh2.sum(0)
    da1 = dh2 @ p["W2"].T
    dh1 = da1 * gelu_grad(h1)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(0)
    return g


def adam(p: dict, g: dict, state: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """One Adam step in place; ``state`` holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m *= b1
        m += (1 - b1) * g[k]
        v *= b2
        v += (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)


def dominant_vector(D) -> np.ndarray:
    """v1: unit eigenvector of D^H D with the largest eigenvalue, phase fixed so that its
    largest-magnitude entry is real and positive."""
    D = np.asarray(D, np.complex128)
    w, V = np.linalg.eigh(D.conj().T @ D)
    v = V[:, -1]
    k = int(np.argmax(np.abs(v)))
    return v * np.exp(-1j * np.angle(v[k]))


def canonicalise(Z, v1) -> np.ndarray:
    """[n, 2L] real network input of the complex queries Z [n, L]."""
    Z = np.asarray(Z, np.complex128)
    nz = np.linalg.norm(Z, axis=1)
    u = Z / np.where(nz == 0, 1.0, nz)[:, None]
    ph = np.angle(u @ np.conj(v1))
    u = u * np.exp(-1j * ph)[:, None]
    out = np.empty((Z.shape[0], 2 * Z.shape[1]))
    out[:, 0::2] = u.real
    out[:, 1::2] = u.imag
    return out
