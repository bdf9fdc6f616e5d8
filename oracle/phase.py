"""Float64 oracle of the phase-aligned real positive projection (§4.3, the heuristic that
extends the real-density projection of eqs. exactP / exactPs to complex data).

TEST INFRASTRUCTURE: never imported by the product path.

v1 is the dictionary's first principal component (dominant eigenvector of sum_j D_j D_j^H).
Atoms and queries are rotated so that their component along v1 is real positive
(alpha_j = angle(v1^H D_j), beta_v = angle(v1^H Z_v)); the real positive cone projection runs
on the aligned vectors; the voxel's phase is then put back, so the density relative to the atom
as given is rho_v = gamma_v e^{i (beta_v - alpha_j)} and X_v = rho_v D_j.
"""
from __future__ import annotations

import numpy as np

from . import mrf_oracle as mo
from . import svd

C128 = np.complex128


def unit_phase(c: np.ndarray) -> np.ndarray:
    a = np.abs(c)
    return np.where(a > 0, c / np.where(a > 0, a, 1.0), 1.0 + 0j)


def project_phase_aligned(Z: np.ndarray, D: np.ndarray, v1: np.ndarray | None = None) -> dict:
    """idx, rho (relative to the atoms as given), the aligned real scores s1 (best) and the
    alignment phases of the queries and atoms."""
    Dc = np.asarray(D, C128)
    if v1 is None:
        V, _ = svd.svd_basis(Dc, 1)
        v1 = V[:, 0]
    v1 = np.asarray(v1, C128)
    ea = unit_phase(Dc @ v1.conj())              # e^{i alpha_j}, v1^H D_j = sum_t conj(v1) D_j
    eb = unit_phase(np.asarray(Z, C128) @ v1.conj())
    Da = Dc * ea.conj()[:, None]
    Za = np.asarray(Z, C128) * eb.conj()[:, None]
    r = mo.project(Za, Da, "real_pos")
    rho = r["rho"] * eb * ea[r["idx"]].conj()
    zero = np.sum(np.abs(np.asarray(Z, C128)) ** 2, axis=1) == 0
    rho[zero] = 0
    return {"idx": r["idx"], "rho": rho, "s1": r["s1"], "s2": r["s2"], "ea": ea, "eb": eb,
            "v1": v1}
