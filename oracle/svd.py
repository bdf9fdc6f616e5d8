"""Float64 oracle of BLIP with temporal subspace compression (§3.3, eqs. CS1, gradupdate and
gradcompression; the option of §4.3 and §6).

TEST INFRASTRUCTURE: never imported by the product path.

V holds the s dominant eigenvectors of the dictionary's frame Gram matrix
sum_j D_j D_j^H = V Sigma V^H (L x L).  Storing fingerprints as rows (X_v is row v of X), the
compressed proxy of a fingerprint x is V_s^H x, i.e. row-wise ``compress(X) = X conj(V_s)``, and
a compressed image expands back to frames as ``expand(Xc) = Xc V_s^T``.  The iteration is
eq. gradupdate, Zc = Xc - mu compress(A^H(A(expand(Xc)) - Y)), followed by the projection of
each row onto the cone of the compressed atoms Dc = compress(D) (eq. exactP in C^s).
"""
from __future__ import annotations

import numpy as np

from . import mrf_oracle as mo

C128 = np.complex128


def svd_basis(D: np.ndarray, s: int) -> tuple[np.ndarray, np.ndarray]:
    """(V_s [L, s], eigenvalues [s]) of sum_j D_j D_j^H, largest first; each column's phase is
    fixed so its largest-magnitude entry is real and positive."""
    A = np.asarray(D, C128)
    M = A.T @ A.conj()                      # M[t, t'] = sum_j D_j[t] conj(D_j[t'])
    w, V = np.linalg.eigh(M)
    order = np.argsort(w)[::-1][:s]
    V = V[:, order]
    k = np.argmax(np.abs(V), axis=0)
    ph = V[k, np.arange(V.shape[1])]
    V = V * (np.abs(ph) / ph)[None, :]
    return V, w[order]


def compress(X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Rows x -> V_s^H x."""
    return np.asarray(X, C128) @ np.asarray(V, C128).conj()


def expand(Xc: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Rows xc -> V_s xc."""
    return np.asarray(Xc, C128) @ np.asarray(V, C128).T


def gradient_step_c(Xc, Y, masks, Ny, Nx, mu, V) -> np.ndarray:
    """eq. gradupdate: Zc = Xc - mu compress(A^H(A(expand(Xc)) - Y))."""
    X = expand(Xc, V)
    R = mo.forward(X, masks, Ny, Nx) - np.asarray(Y, C128)
    return np.asarray(Xc, C128) - mu * compress(mo.adjoint(R, masks, Ny, Nx), V)


def blip_svd(Y, masks, D, V, Ny, Nx, iters, mu=1.0, cone="complex", adaptive=False, zeta=2.0,
             kappa=False, max_shrink=60, history=False) -> dict:
    """BLIP in the compressed domain from Xc = 0: returns the compressed image Xc [n, s], the
    atoms idx, the densities rho and the expanded image X = expand(Xc).

    With ``adaptive`` each iteration starts from ``mu`` and divides it by ``zeta`` while
    mu_k >= ||Xc^{k+1} - Xc^k||^2 / ||A(expand(Xc^{k+1} - Xc^k))||^2 (the compressed form of
    eq. steprule, §4.3), recomputing the iteration each time.  With ``kappa`` the first iterate
    is rescaled by kappa = ||Y|| / ||A(expand(Xc^1))|| and mu by kappa (§4.3)."""
    Dc = compress(D, V)
    n, s = Ny * Nx, V.shape[1]
    Xc = np.zeros((n, s), C128)
    idx = np.zeros(n, np.int64)
    rho = np.zeros(n, C128)
    mu0 = float(mu)
    hist = {"mu": [], "shrinks": []}
    for k in range(iters):
        mu_k = mu0
        shrinks = 0
        while True:
            Zc = gradient_step_c(Xc, Y, masks, Ny, Nx, mu_k, V)
            r = mo.project(Zc, Dc, cone)
            Xn = r["rho"][:, None] * Dc[r["idx"]]
            if not adaptive:
                break
            dXc = Xn - Xc
            num = np.sum(np.abs(dXc) ** 2)
            den = np.sum(np.abs(mo.forward(expand(dXc, V), masks, Ny, Nx)) ** 2)
            if den == 0.0 or mu_k < num / den or shrinks >= max_shrink:
                break
            mu_k /= zeta
            shrinks += 1
        idx, rho = r["idx"], r["rho"]
        if kappa and k == 0:
            kap = np.linalg.norm(Y) / max(np.linalg.norm(mo.forward(expand(Xn, V), masks, Ny, Nx)),
                                         1e-300)
            Xn = kap * Xn
            rho = kap * rho
            mu0 *= kap
        Xc = Xn
        hist["mu"].append(mu_k)
        hist["shrinks"].append(shrinks)
    out = {"Xc": Xc, "idx": idx, "rho": rho, "X": expand(Xc, V)}
    if history:
        out["history"] = hist
    return out
