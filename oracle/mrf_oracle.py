"""Float64 oracle of the BLIP iteration and its exact matched-filtering projection.

TEST INFRASTRUCTURE (see the package docstring): never imported by the product path.

Notation follows §3: X is the [n, L] MRF image (row v = voxel fingerprint X_v, column t = frame
X_t, voxel v = y * Nx + x), D the [d, L] dictionary, Y the k-space [Ny, Nx, L] (ky, kx, t) in
DFT order with zeros where a line was not sampled, masks the [L, Ny] 0/1 line sets Omega_t.
"""
from __future__ import annotations

import numpy as np

C128 = np.complex128


# ---------------------------------------------------------------------------------------------
# Forward model and its adjoint (§3, eq. forward with one coil: A = P_Omega F)
# ---------------------------------------------------------------------------------------------
def forward(X: np.ndarray, masks: np.ndarray, Ny: int, Nx: int) -> np.ndarray:
    """A(X) = P_Omega F X: unitary 2-D DFT of every frame, then keep the lines of Omega_t."""
    L = X.shape[1]
    img = np.asarray(X, C128).reshape(Ny, Nx, L)
    k = np.fft.fft2(img, axes=(0, 1), norm="ortho")
    return k * masks.T.astype(np.float64)[:, None, :]


def adjoint(Y: np.ndarray, masks: np.ndarray, Ny: int, Nx: int) -> np.ndarray:
    """A^H(Y) = F^H P_Omega^H Y (zero-filled lines, inverse unitary DFT), as [n, L]."""
    L = Y.shape[2]
    k = np.asarray(Y, C128) * masks.T.astype(np.float64)[:, None, :]
    return np.fft.ifft2(k, axes=(0, 1), norm="ortho").reshape(Ny * Nx, L)


def gradient_step(X, Y, masks, Ny, Nx, mu) -> np.ndarray:
    """Z = X - mu A^H(A(X) - Y)  (§3.2, eq. blip, the argument of the projection)."""
    X = np.asarray(X, C128)
    return X - mu * adjoint(forward(X, masks, Ny, Nx) - Y, masks, Ny, Nx)


# ---------------------------------------------------------------------------------------------
# Exact projection onto the cone of fingerprints (§3.2, eqs. exactP / exactPs)
# ---------------------------------------------------------------------------------------------
def project(Z: np.ndarray, D: np.ndarray, cone: str = "complex", chunk: int = 256) -> dict:
    """Per-voxel Euclidean projection onto cone(D) by exhaustive search.

    complex cone {rho D_j : rho in C}:   residual_j = ||z||^2 - |D_j^H z|^2 / ||D_j||^2,
        j* = argmin_j residual_j, rho = D_j*^H z / ||D_j*||^2.
    real_pos cone (the paper's gamma > 0, eq. exactP):  j* = argmin_j ||z - D_j / ||D_j|| ||,
        gamma = max(Re(D_j*^H z) / ||D_j*||^2, 0).
    Ties go to the smallest j; a zero query gives j* = 0, rho = 0.
    Also returns, per voxel, the best and second-best normalised correlation
    |D_j^H z| / (||D_j|| ||z||) (for real_pos: Re(D_j^H z) / (||D_j|| ||z||)) so callers can tell
    near-ties apart.
    """
    Z = np.asarray(Z, C128)
    D = np.asarray(D, C128)
    n = Z.shape[0]
    dn2 = np.sum(D.real ** 2 + D.imag ** 2, axis=1)
    dn = np.sqrt(dn2)
    idx = np.zeros(n, np.int64)
    rho = np.zeros(n, C128)
    s1 = np.zeros(n)
    s2 = np.zeros(n)
    DH = D.conj().T                              # D^H, formed once for all chunks
    for a in range(0, n, chunk):
        z = Z[a:a + chunk]
        zn2 = np.sum(z.real ** 2 + z.imag ** 2, axis=1)
        c = z @ DH                               # c[v, j] = D_j^H z_v
        if cone == "complex":
            resid = zn2[:, None] - (c.real ** 2 + c.imag ** 2) / dn2[None, :]
            score = np.abs(c) / dn[None, :]
        elif cone == "real_pos":
            resid = zn2[:, None] + 1.0 - 2.0 * c.real / dn[None, :]
            score = c.real / dn[None, :]
        else:
            raise ValueError(cone)
        j = np.argmin(resid, axis=1)
        r = np.arange(z.shape[0])
        cj = c[r, j]
        if cone == "complex":
            rh = cj / dn2[j]
        else:
            rh = np.maximum(cj.real / dn2[j], 0.0).astype(C128)
        zero = zn2 == 0.0
        j[zero] = 0
        rh[zero] = 0.0
        znrm = np.where(zero, 1.0, np.sqrt(zn2))
        # the two largest scores of each row (a partial selection: the same values as a sort)
        if score.shape[1] > 1:
            top = -np.partition(-score, 1, axis=1)[:, :2]
            first, second = top[:, 0], top[:, 1]
        else:
            first, second = score[:, 0], np.full(score.shape[0], -np.inf)
        idx[a:a + chunk] = j
        rho[a:a + chunk] = rh
        s1[a:a + chunk] = first / znrm
        s2[a:a + chunk] = second / znrm
    return {"idx": idx, "rho": rho, "s1": s1, "s2": s2}


def correlation(Z: np.ndarray, D: np.ndarray, idx: np.ndarray, cone: str = "complex"):
    """Normalised correlation of each voxel with the atom idx[v] (same measure as s1)."""
    Z = np.asarray(Z, C128)
    d = np.asarray(D, C128)[idx]
    c = np.sum(np.conj(d) * Z, axis=1)
    den = np.sqrt(np.sum(np.abs(d) ** 2, axis=1) * np.sum(np.abs(Z) ** 2, axis=1))
    den = np.where(den == 0, 1.0, den)
    return (np.abs(c) if cone == "complex" else c.real) / den


def density(Z: np.ndarray, D: np.ndarray, idx: np.ndarray, cone: str = "complex"):
    """rho_v = D_j^H Z_v / ||D_j||^2 (complex cone) or max(Re(.), 0) (real_pos), j = idx[v]."""
    Z = np.asarray(Z, C128)
    d = np.asarray(D, C128)[idx]
    c = np.sum(np.conj(d) * Z, axis=1) / np.sum(np.abs(d) ** 2, axis=1)
    return c if cone == "complex" else np.maximum(c.real, 0.0).astype(C128)


def rescale(idx, rho, D) -> np.ndarray:
    """X_v = rho_v D_j*  (§3.2, eq. exactPs; Algorithm 2, rescaling)."""
    return rho[:, None] * np.asarray(D, C128)[idx]


def lut(idx, params) -> np.ndarray:
    """Theta_v = look-up-table(D_j*) (Algorithm 2, final step)."""
    return np.asarray(params)[idx]


# ---------------------------------------------------------------------------------------------
# BLIP / CoverBLIP iteration (§3.2 eq. blip; Algorithm 2 with the step rule eq. steprule)
# ---------------------------------------------------------------------------------------------
def blip(Y, masks, D, Ny, Nx, iters, mu=1.0, cone="complex", adaptive=False, zeta=2.0,
         kappa=False, tol=None, project_fn=None, X_init=None, idx_init=None,
         max_shrink=60, history=False) -> dict:
    """Iterate X^{k+1} = P_C(X^k - mu_k A^H(A X^k - Y)) from X^0 = 0.

    ``project_fn(Z, warm_idx) -> (idx, rho)`` replaces the exact projection (CoverBLIP passes
    the (1+eps)-ANNS here, warm-started at the previous atoms).  With ``adaptive`` every
    iteration starts from ``mu`` and divides it by ``zeta`` while
    mu_k >= ||X^{k+1} - X^k||^2 / ||A(X^{k+1} - X^k)||^2, recomputing the iteration each time.
    With ``kappa`` the first iterate is rescaled by kappa = ||Y|| / ||A(X^1)|| and mu by kappa.
    ``tol`` stops when the objective's relative progress falls below it (§6, cost paragraph).
    """
    n, L = Ny * Nx, Y.shape[2]
    X = np.zeros((n, L), C128) if X_init is None else np.asarray(X_init, C128).copy()
    idx = np.zeros(n, np.int64) if idx_init is None else np.asarray(idx_init).copy()
    rho = np.zeros(n, C128)
    if project_fn is None:
        def project_fn(Z, warm):
            r = project(Z, D, cone)
            return r["idx"], r["rho"]
    mu0 = float(mu)
    hist = {"fidelity": [], "mu": [], "shrinks": []}
    prev_obj = None
    Dc = np.asarray(D, C128)
    for k in range(iters):
        mu_k = mu0
        shrinks = 0
        while True:
            Z = gradient_step(X, Y, masks, Ny, Nx, mu_k)
            j, r = project_fn(Z, idx)
            Xn = r[:, None] * Dc[j]
            if not adaptive:
                break
            dX = Xn - X
            den = np.sum(np.abs(forward(dX, masks, Ny, Nx)) ** 2)
            num = np.sum(np.abs(dX) ** 2)
            if den == 0.0 or mu_k < num / den or shrinks >= max_shrink:
                break
            mu_k /= zeta
            shrinks += 1
        if kappa and k == 0:
            kap = np.linalg.norm(Y) / max(np.linalg.norm(forward(Xn, masks, Ny, Nx)), 1e-300)
            Xn = kap * Xn
            r = kap * r
            mu0 *= kap
        X, idx, rho = Xn, np.asarray(j), np.asarray(r)
        obj = float(np.sum(np.abs(Y - forward(X, masks, Ny, Nx)) ** 2))
        hist["fidelity"].append(np.sqrt(obj) / max(np.linalg.norm(Y), 1e-300))
        hist["mu"].append(mu_k)
        hist["shrinks"].append(shrinks)
        if tol is not None and prev_obj is not None and prev_obj > 0 \
                and abs(prev_obj - obj) / prev_obj < tol:
            break
        prev_obj = obj
    out = {"X": X, "idx": idx, "rho": rho}
    if history:
        out["history"] = hist
    return out


# ---------------------------------------------------------------------------------------------
# Evaluation metrics (§6, evaluation metrics)
# ---------------------------------------------------------------------------------------------
def nmse(Xhat, X0) -> float:
    """||Xhat - X0|| / ||X0||."""
    X0 = np.asarray(X0, C128)
    return float(np.linalg.norm(np.asarray(Xhat, C128) - X0) / np.linalg.norm(X0))


def accuracy(est, truth, mask) -> float:
    """1 - mean over the mask of |est - truth| / truth (T1 and T2 accuracy)."""
    e, t = np.asarray(est, np.float64)[mask], np.asarray(truth, np.float64)[mask]
    return float(1.0 - np.mean(np.abs(e - t) / t))
