"""Discrete-time Bloch responses B(Theta; TR, TE, alpha) (§3.1, eq. fingerprints).

Two simulators, both vectorised over atoms and run in float64:

* :func:`epg_fisp` -- inversion-recovery FISP (unbalanced gradient, one dephasing cycle per TR)
  by the extended-phase-graph recursion, exact (no state truncation: L + 1 states).  In ideal
  FISP a uniform off-resonance only multiplies the echo by the constant phase exp(i 2 pi B0 TE)
  (the spoiled ensemble is invariant to a shift of the per-TR precession), so B0 is not a
  parameter of this simulator.
* :func:`bssfp` -- inversion-recovery balanced SSFP, the sequence of the paper's own
  experiments (§6), one isochromat per atom, alternating RF phase, off-resonance B0 precession.

Magnetisation convention: M+ = Mx + i My; an RF pulse of angle a about x maps
(My, Mz) -> (My cos a - Mz sin a, My sin a + Mz cos a); relaxation over tau multiplies the
transverse part by exp(-tau/T2) and relaxes Mz towards 1 with exp(-tau/T1).
"""
from __future__ import annotations

import numpy as np

from .sequence import TR_MS, TE_MS


def _as1d(x, d):
    a = np.asarray(x, np.float64)
    return np.broadcast_to(a, (d,)).astype(np.float64) if a.ndim == 0 else a.astype(np.float64)


def epg_fisp(T1, T2, alpha_deg, B1=1.0, TR=TR_MS, TE=TE_MS) -> np.ndarray:
    """IR-FISP echoes F+_0 at TE for every frame; complex128 [d, L] (not normalised).

    Per frame: RF(alpha_t * B1) -> relax over TE -> read F+_0 -> relax over TR - TE ->
    gradient dephasing by one configuration.  Starts from Mz = -1 (inversion, no TI delay).
    """
    T1 = np.atleast_1d(np.asarray(T1, np.float64))
    d = T1.shape[0]
    T2 = _as1d(T2, d)
    B1 = _as1d(B1, d)
    alpha = np.deg2rad(np.asarray(alpha_deg, np.float64))
    L = alpha.shape[0]
    K = L + 1
    Fp = np.zeros((d, K), np.complex128)
    Fm = np.zeros((d, K), np.complex128)
    Z = np.zeros((d, K), np.complex128)
    Z[:, 0] = -1.0
    e1a, e2a = np.exp(-TE / T1)[:, None], np.exp(-TE / T2)[:, None]
    e1b, e2b = np.exp(-(TR - TE) / T1)[:, None], np.exp(-(TR - TE) / T2)[:, None]
    out = np.empty((d, L), np.complex128)
    for t in range(L):
        a = (alpha[t] * B1)[:, None]
        c2, s2, sa, ca = np.cos(a / 2) ** 2, np.sin(a / 2) ** 2, np.sin(a), np.cos(a)
        fp = c2 * Fp + s2 * Fm - 1j * sa * Z
        fm = s2 * Fp + c2 * Fm + 1j * sa * Z
        z = -0.5j * sa * Fp + 0.5j * sa * Fm + ca * Z
        fp *= e2a
        fm *= e2a
        z *= e1a
        z[:, 0] += 1.0 - e1a[:, 0]
        out[:, t] = fp[:, 0]
        fp *= e2b
        fm *= e2b
        z *= e1b
        z[:, 0] += 1.0 - e1b[:, 0]
        Fp[:, 1:] = fp[:, :-1]
        Fm[:, :-1] = fm[:, 1:]
        Fm[:, -1] = 0.0
        Fp[:, 0] = np.conj(Fm[:, 0])
        Z = z
    return out


def isochromat_fisp(T1, T2, alpha_deg, B1=1.0, TR=TR_MS, TE=TE_MS, n_iso=None) -> np.ndarray:
    """Direct Bloch rotation of n_iso isochromats dephased uniformly over one cycle per TR.

    The ensemble mean of M+ at TE equals the exact EPG echo once n_iso > 2 L (no aliasing of
    configuration orders); used to check :func:`epg_fisp`.  Scalar T1/T2, complex128 [L].
    """
    alpha = np.deg2rad(np.asarray(alpha_deg, np.float64))
    L = alpha.shape[0]
    m = n_iso or (2 * L + 8)
    theta = 2 * np.pi * np.arange(m) / m
    mx, my, mz = np.zeros(m), np.zeros(m), -np.ones(m)
    out = np.empty(L, np.complex128)
    e1a, e2a = np.exp(-TE / T1), np.exp(-TE / T2)
    e1b, e2b = np.exp(-(TR - TE) / T1), np.exp(-(TR - TE) / T2)
    for t in range(L):
        a = alpha[t] * B1
        my, mz = my * np.cos(a) - mz * np.sin(a), my * np.sin(a) + mz * np.cos(a)
        mx, my, mz = mx * e2a, my * e2a, mz * e1a + (1 - e1a)
        out[t] = np.mean(mx + 1j * my)
        mx, my, mz = mx * e2b, my * e2b, mz * e1b + (1 - e1b)
        c, s = np.cos(theta), np.sin(theta)
        mx, my = mx * c - my * s, mx * s + my * c
    return out


def bssfp(T1, T2, B0, alpha_deg, B1=1.0, TR=TR_MS, TE=TE_MS) -> np.ndarray:
    """IR-bSSFP signal at TE, one isochromat per atom; complex128 [d, L] (not normalised).

    RF phase alternates (+x, -x) and the readout is demodulated by (-1)^t.  B0 in Hz precesses
    M+ by exp(i 2 pi B0 tau) over each free interval tau.
    """
    T1 = np.atleast_1d(np.asarray(T1, np.float64))
    d = T1.shape[0]
    T2, B0, B1 = _as1d(T2, d), _as1d(B0, d), _as1d(B1, d)
    alpha = np.deg2rad(np.asarray(alpha_deg, np.float64))
    L = alpha.shape[0]
    e1a, e2a = np.exp(-TE / T1), np.exp(-TE / T2)
    e1b, e2b = np.exp(-(TR - TE) / T1), np.exp(-(TR - TE) / T2)
    pa, pb = 2 * np.pi * B0 * TE * 1e-3, 2 * np.pi * B0 * (TR - TE) * 1e-3
    ca_, sa_ = np.cos(pa), np.sin(pa)
    cb_, sb_ = np.cos(pb), np.sin(pb)
    mx, my, mz = np.zeros(d), np.zeros(d), -np.ones(d)
    out = np.empty((d, L), np.complex128)
    for t in range(L):
        a = alpha[t] * B1 * (1.0 if t % 2 == 0 else -1.0)
        ca, sa = np.cos(a), np.sin(a)
        my, mz = my * ca - mz * sa, my * sa + mz * ca
        mx, my = e2a * (mx * ca_ - my * sa_), e2a * (mx * sa_ + my * ca_)
        mz = mz * e1a + (1 - e1a)
        out[:, t] = (mx + 1j * my) * (1.0 if t % 2 == 0 else -1.0)
        mx, my = e2b * (mx * cb_ - my * sb_), e2b * (mx * sb_ + my * cb_)
        mz = mz * e1b + (1 - e1b)
    return out


def simulate_dictionary(params: np.ndarray, names, alpha_deg, seq: str,
                        chunk: int = 32768) -> np.ndarray:
    """Unit-norm atoms, complex64 [d, L]: simulated in float64, normalised in float64, cast.

    ``seq`` is "fisp" (columns T1, T2[, B1]) or "bssfp" (columns T1, T2[, B1], B0).
    """
    params = np.asarray(params, np.float64)
    col = {n: i for i, n in enumerate(names)}
    d, L = params.shape[0], len(alpha_deg)
    out = np.empty((d, L), np.complex64)
    for s in range(0, d, chunk):
        p = params[s:s + chunk]
        b1 = p[:, col["B1"]] if "B1" in col else 1.0
        if seq == "fisp":
            sig = epg_fisp(p[:, col["T1"]], p[:, col["T2"]], alpha_deg, B1=b1)
        elif seq == "bssfp":
            b0 = p[:, col["B0"]] if "B0" in col else 0.0
            sig = bssfp(p[:, col["T1"]], p[:, col["T2"]], b0, alpha_deg, B1=b1)
        else:
            raise ValueError(seq)
        nrm = np.sqrt(np.sum(sig.real ** 2 + sig.imag ** 2, axis=1))
        out[s:s + chunk] = (sig / nrm[:, None]).astype(np.complex64)
    return out
