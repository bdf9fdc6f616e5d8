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


def _rand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_expand_inverts_compress():
    """With orthonormal columns (V^H V = I) compress(expand(Xc)) = Xc for any s; with the full
    basis (V unitary) expand(compress(X)) = X as well."""
    g = np.random.Generator(np.random.PCG64(41))
    L = 9
    Q, _ = np.linalg.qr(_rand(g, L, L))
    Xc = _rand(g, 7, 4)
    np.testing.assert_allclose(svd.compress(svd.expand(Xc, Q[:, :4]), Q[:, :4]), Xc, atol=1e-12)
    X = _rand(g, 7, L)
    np.testing.assert_allclose(svd.expand(svd.compress(X, Q), Q), X, atol=1e-12)


def test_compressed_step_is_the_compressed_fidelity_gradient():
    """eq. gradupdate: (Xc - Zc) / mu is the gradient of f_c(Xc) = 1/2 ||A(V_s Xc) - Y||^2,
    checked by central differences along random complex directions (partial masks)."""
    g = np.random.Generator(np.random.PCG64(42))
    Ny, Nx, L, s, mu = 8, 4, 6, 3, 0.9
    Q, _ = np.linalg.qr(_rand(g, L, L))
    V = Q[:, :s]
    masks = (g.random((L, Ny)) < 0.5).astype(np.uint8)
    Y = mo.forward(_rand(g, Ny * Nx, L), masks, Ny, Nx)
    Xc = _rand(g, Ny * Nx, s)

    def f(Xc_):
        R = mo.forward(svd.expand(Xc_, V), masks, Ny, Nx) - Y
        return 0.5 * float(np.sum(np.abs(R) ** 2))

    grad = (Xc - svd.gradient_step_c(Xc, Y, masks, Ny, Nx, mu, V)) / mu
    eps = 1e-3
    for _ in range(4):
        E = _rand(g, Ny * Nx, s)
        fd = (f(Xc + eps * E) - f(Xc - eps * E)) / (2 * eps)
        assert abs(fd - float(np.real(np.vdot(grad, E)))) <= 1e-9 * max(1.0, abs(fd))


def test_full_basis_step_rule_and_kappa_reproduce_blip():
    """With the full basis the compressed step rule of §4.3 is eq. steprule itself (expansion is
    unitary, so ||dXc|| = ||dX|| and A(expand(dXc)) = A(dX)): adaptive compressed BLIP takes
    the same steps, shrinks and iterates as the oracle's adaptive BLIP, and its kappa rescale
    the same factor."""
    dic, p = small_problem()
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    V, _ = svd.svd_basis(dic["atoms"], L)
    mu = float(Ny / p["masks"].sum(1).mean())
    r = svd.blip_svd(p["Y"], p["masks"], dic["atoms"], V, Ny, Nx, iters=4, mu=mu, adaptive=True,
                     history=True)
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=4, mu=mu, adaptive=True,
                  history=True)
    assert r["history"]["shrinks"] == ref["history"]["shrinks"]
    np.testing.assert_allclose(r["history"]["mu"], ref["history"]["mu"], rtol=1e-12)
    assert max(r["history"]["shrinks"]) > 0          # the rule did shrink
    assert np.array_equal(r["idx"], ref["idx"])
    np.testing.assert_allclose(r["X"], ref["X"], rtol=0, atol=1e-9 * np.abs(ref["X"]).max())
    rk = svd.blip_svd(p["Y"], p["masks"], dic["atoms"], V, Ny, Nx, iters=3, kappa=True)
    refk = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=3, kappa=True)
    assert np.array_equal(rk["idx"], refk["idx"])
    np.testing.assert_allclose(rk["X"], refk["X"], rtol=0, atol=1e-9 * np.abs(refk["X"]).max())


def test_compressed_step_rule_monotone_fidelity():
    """With s < L the accepted steps meet the compressed rule and the fidelity
    ||Y - A(expand(Xc^k))|| does not increase (Thm. inexactmonotone with the compressed
    projection, which is a projection onto a cone inside the compressed subspace)."""
    dic, p = small_problem()
    Ny, Nx = p["Ny"], p["Nx"]
    V, _ = svd.svd_basis(dic["atoms"], 12)
    mu = float(Ny / p["masks"].sum(1).mean())
    fid = []
    for k in range(1, 6):
        r = svd.blip_svd(p["Y"], p["masks"], dic["atoms"], V, Ny, Nx, iters=k, mu=mu,
                         adaptive=True, history=True)
        fid.append(np.linalg.norm(p["Y"] - mo.forward(r["X"], p["masks"], Ny, Nx)))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(fid, fid[1:])), fid
    assert all(1.0 / 2.0 <= m <= mu for m in r["history"]["mu"])
