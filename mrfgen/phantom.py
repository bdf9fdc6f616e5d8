"""Ellipse phantoms, Cartesian phase-encode line masks and the simulated acquisition.

The acquisition follows the data model of §3, eq. forward, for one coil (S = identity):
Y_t = P_{Omega_t} F X_t + xi, with F the unitary 2-D DFT of each frame and Omega_t a set of
phase-encode (ky) lines per frame.  Image layout: X is [n, L] with voxel v = y * Nx + x
(row-major, y outer) and the frame index t contiguous.  k-space layout: Y is [Ny, Nx, L]
(ky, kx, t) in DFT order (DC at index 0), zero where a line was not sampled.
"""
from __future__ import annotations

import numpy as np

from .sequence import rng


def _ellipse_mask(N, cy, cx, ay, ax, ang):
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    yy, xx = y - cy, x - cx
    c, s = np.cos(ang), np.sin(ang)
    u = xx * c + yy * s
    w = -xx * s + yy * c
    return (u / ax) ** 2 + (w / ay) ** 2 <= 1.0


def _smooth_field(g, N, lo, hi):
    y, x = np.mgrid[0:N, 0:N].astype(np.float64) / N
    f = np.zeros((N, N))
    for _ in range(4):
        cy, cx = g.uniform(0.0, 1.0, 2)
        sig = g.uniform(0.15, 0.5)
        amp = g.uniform(-1.0, 1.0)
        f += amp * np.exp(-((y - cy) ** 2 + (x - cx) ** 2) / (2 * sig * sig))
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    return lo + (hi - lo) * f


def ellipse_phantom(N: int, seed: int, b0: str | None = None, smooth_b1: bool = False,
                    n_ellipses: int = 6) -> dict:
    """Six ellipses painted in order on a zero background (later ones overwrite).

    Ellipse 0 is large (semi-axes U[0.35,0.45] N, centre U[0.45,0.55] N); the others have
    centres U[0.25,0.75] N and semi-axes U[0.05,0.25] N; angles U[0, pi).  Per ellipse:
    T1 ~ U[300,2500] ms, T2 ~ U[30,300] ms, rho ~ U[0.5,1] exp(i U[0,2pi)); with b0="ellipse"
    also B0 ~ U[-50,50] Hz.  b0="smooth" / smooth_b1 give fields made of 4 seeded Gaussians,
    rescaled to [-50,50] Hz and [0.6,1.4].  Returns flat [n] maps (n = N*N, y outer).
    """
    g = rng(seed)
    lab = np.full((N, N), -1, np.int32)
    tissues = []
    for e in range(n_ellipses):
        if e == 0:
            cy, cx = g.uniform(0.45, 0.55, 2) * N
            ay, ax = g.uniform(0.35, 0.45, 2) * N
        else:
            cy, cx = g.uniform(0.25, 0.75, 2) * N
            ay, ax = g.uniform(0.05, 0.25, 2) * N
        ang = g.uniform(0.0, np.pi)
        t1 = g.uniform(300.0, 2500.0)
        t2 = g.uniform(30.0, 300.0)
        rho = g.uniform(0.5, 1.0) * np.exp(1j * g.uniform(0.0, 2 * np.pi))
        b0v = g.uniform(-50.0, 50.0) if b0 == "ellipse" else 0.0
        tissues.append((t1, t2, rho, b0v))
        lab[_ellipse_mask(N, cy, cx, ay, ax, ang)] = e
    n = N * N
    lab = lab.reshape(n)
    T1, T2, B0 = np.zeros(n), np.zeros(n), np.zeros(n)
    B1 = np.ones(n)
    rho = np.zeros(n, np.complex128)
    for e, (t1, t2, r, b) in enumerate(tissues):
        sel = lab == e
        T1[sel], T2[sel], rho[sel], B0[sel] = t1, t2, r, b
    if b0 == "smooth":
        B0 = _smooth_field(g, N, -50.0, 50.0).reshape(n) * (lab >= 0)
    if smooth_b1:
        B1 = np.where(lab >= 0, _smooth_field(g, N, 0.6, 1.4).reshape(n), 1.0)
    return {"N": N, "labels": lab, "T1": T1, "T2": T2, "B0": B0, "B1": B1, "rho": rho}


def line_masks(Ny: int, L: int, R: float, seed: int) -> np.ndarray:
    """Variable-density ky-line masks, uint8 [L, Ny] in DFT order.

    Per frame the central max(2, Ny // 32) lines are always kept; the others are drawn without
    replacement with probability proportional to (1 - |c - Ny/2| / (Ny/2))^2 + 0.05 (c the
    centred line index) until round(Ny / R) lines are kept.
    """
    g = rng(seed)
    m = max(int(round(Ny / R)), 1)
    nc = min(max(2, Ny // 32), m)
    c = np.arange(Ny)
    central = np.arange(Ny // 2 - nc // 2, Ny // 2 - nc // 2 + nc)
    rest = np.setdiff1d(c, central)
    p = (1.0 - np.abs(rest - Ny / 2) / (Ny / 2)) ** 2 + 0.05
    p = p / p.sum()
    out = np.zeros((L, Ny), np.uint8)
    for t in range(L):
        pick = g.choice(rest, size=m - nc, replace=False, p=p) if m > nc else np.array([], int)
        lines = np.concatenate([central, pick]).astype(np.int64)
        out[t, (lines - Ny // 2) % Ny] = 1
    return out


def epi_masks(Ny: int, L: int, R: int) -> np.ndarray:
    """Multi-shot EPI pattern of §6.1: every R-th line, shifted by one line per frame."""
    out = np.zeros((L, Ny), np.uint8)
    for t in range(L):
        out[t, (t + R * np.arange(Ny // R)) % Ny] = 1
    return out


def ground_truth(ph: dict, fingerprint) -> np.ndarray:
    """X0 [n, L] complex64 with X0_v = rho_v * b_v / ||b_v||, where ``fingerprint(T1, T2, B0,
    B1)`` returns unnormalised complex128 responses [k, L] for parameter vectors of length k."""
    n = ph["labels"].shape[0]
    fg = np.flatnonzero(ph["labels"] >= 0)
    keys = np.stack([ph["T1"][fg], ph["T2"][fg], ph["B0"][fg], ph["B1"][fg]], 1)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    sig = fingerprint(uniq[:, 0], uniq[:, 1], uniq[:, 2], uniq[:, 3])
    sig = sig / np.sqrt(np.sum(np.abs(sig) ** 2, axis=1))[:, None]
    X0 = np.zeros((n, sig.shape[1]), np.complex64)
    X0[fg] = (ph["rho"][fg, None] * sig[inv.reshape(-1)]).astype(np.complex64)
    return X0


def acquire(X0: np.ndarray, masks: np.ndarray, Ny: int, Nx: int, snr_db: float | None,
            seed: int, chunk: int = 64) -> np.ndarray:
    """Y = P_Omega F X0 + xi as complex64 [Ny, Nx, L] (eq. forward, one coil).

    xi is circular complex Gaussian on the sampled entries with per-component variance
    ||Y_clean||^2 / (2 N_s 10^(snr/10)), N_s the number of sampled entries; snr_db=None is
    noiseless.
    """
    L = X0.shape[1]
    Y = np.zeros((Ny, Nx, L), np.complex64)
    img = X0.reshape(Ny, Nx, L)
    for s in range(0, L, chunk):
        k = np.fft.fft2(img[:, :, s:s + chunk].astype(np.complex128), axes=(0, 1), norm="ortho")
        k *= masks[s:s + chunk].T[:, None, :]
        Y[:, :, s:s + chunk] = k
    if snr_db is not None:
        g = rng(seed)
        ns = int(masks.sum()) * Nx
        e = float(np.sum(np.abs(Y.astype(np.complex128)) ** 2))
        sd = np.sqrt(e / (2.0 * ns * 10.0 ** (snr_db / 10.0)))
        samp = np.broadcast_to(masks.T[:, None, :].astype(bool), Y.shape)
        noise = sd * (g.standard_normal(ns) + 1j * g.standard_normal(ns))
        Y[samp] += noise.astype(np.complex64)
    return Y
