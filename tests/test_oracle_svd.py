"""Pins of the subspace-compressed BLIP oracle (§3.3): with the full basis (s = L, V unitary)
the compressed iteration is the uncompressed one after the change of variable X = Xc V^T, so
it reproduces BLIP exactly; the basis is orthonormal, ordered, and solves the eigenproblem of
the frame Gram matrix; compression keeps the energy the eigenvalues predict; a dictionary that
is exactly rank s is reconstructed identically with s components."""
import numpy as np

import mrfgen
from oracle import mrf_oracle as mo
from oracle import svd


def small_problem():
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic, N=16)
    return dic, p


def test_basis_is_the_gram_eigenbasis():
    dic, _ = small_problem()
    A = dic["atoms"].astype(np.complex128)
    V, w = svd.svd_basis(A, 12)
    assert np.allclose(V.conj().T @ V, np.eye(12), atol=1e-10)
    assert np.all(np.diff(w) <= 1e-9)
    M = A.T @ A.conj()
    assert np.allclose(M @ V, V * w[None, :], atol=1e-8 * w[0])
    # energy kept by compression = sum of the kept eigenvalues
    kept = np.sum(np.abs(svd.compress(A, V)) ** 2)
    assert abs(kept - w.sum()) <= 1e-9 * w.sum()
    # largest-magnitude entry of each column real positive
    k = np.argmax(np.abs(V), axis=0)
    ph = V[k, np.arange(12)]
    assert np.allclose(ph.imag, 0) and np.all(ph.real > 0)


def test_full_basis_reproduces_blip():
    dic, p = small_problem()
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    V, _ = svd.svd_basis(dic["atoms"], L)
    r = svd.blip_svd(p["Y"], p["masks"], dic["atoms"], V, Ny, Nx, iters=3)
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=3)
    assert np.array_equal(r["idx"], ref["idx"])
    np.testing.assert_allclose(r["X"], ref["X"], rtol=0, atol=1e-9 * np.abs(ref["X"]).max())


def test_exactly_low_rank_dictionary():
    """Atoms built from s orthonormal frame patterns: s components lose nothing, so compressed
    and uncompressed BLIP agree."""
    g = np.random.Generator(np.random.PCG64(3))
    L, s, d, Ny, Nx = 24, 5, 40, 8, 8
    B, _ = np.linalg.qr(g.standard_normal((L, s)) + 1j * g.standard_normal((L, s)))
    coef = g.standard_normal((d, s)) + 1j * g.standard_normal((d, s))
    A = coef @ B.T
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    js = g.integers(0, d, Ny * Nx)
    X0 = A[js] * (0.5 + g.random(Ny * Nx))[:, None]
    masks = (g.random((L, Ny)) < 0.5).astype(np.uint8)
    masks[:, 0] = 1
    Y = mo.forward(X0, masks, Ny, Nx)
    V, w = svd.svd_basis(A, s)
    assert w[-1] > 1e-6
    r = svd.blip_svd(Y, masks, A, V, Ny, Nx, iters=4)
    ref = mo.blip(Y, masks, A, Ny, Nx, iters=4)
    assert np.array_equal(r["idx"], ref["idx"])
    np.testing.assert_allclose(r["X"], ref["X"], atol=1e-9 * np.abs(ref["X"]).max())
