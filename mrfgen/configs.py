"""The five synthetic workloads and their seed scheme.

Seeds: flip train 1810 + L; phantom 2000 + 100 c + i; mask 3000 + 100 c + i;
noise 4000 + 100 c + i (c = workload number 1..5, i = slice index).

1  32x32 phantom, L=100, ~2000 atoms over (T1, T2), IR-FISP, R=8 variable-density lines,
   40 dB, 10 iterations, mu = 1.
2  256x256, L=1000, ~100k atoms over (T1, T2, B0 in -50:2:50 Hz), IR-bSSFP, R=16, 20 iterations.
3  256x256, L=500, ~1M atoms over (T1, T2, B1 in 0.6:0.1:1.4, B0), smooth B0/B1 fields.
4  the learned proposal, trained and run on workload 2's dictionary and phantom.
5  64 slices with N drawn from {128, 192, 256, 320}, L=1000, workload 2's dictionary,
   R drawn from [8, 24].
"""
from __future__ import annotations

import numpy as np

from .sequence import flip_train, param_grid, rng
from .bloch import simulate_dictionary, epg_fisp, bssfp
from .phantom import ellipse_phantom, line_masks, ground_truth, acquire

B0_AXIS = np.arange(-50.0, 50.0 + 1e-9, 2.0)
B1_AXIS = np.round(np.arange(0.6, 1.4 + 1e-9, 0.1), 10)

CONFIGS = {
    1: dict(N=32, L=100, t1t2=2000, b0=False, b1=False, seq="fisp", R=8.0, snr=40.0, iters=10,
            phantom_b0=None, smooth_b1=False),
    2: dict(N=256, L=1000, t1t2=1961, b0=True, b1=False, seq="bssfp", R=16.0, snr=40.0,
            iters=20, phantom_b0="ellipse", smooth_b1=False),
    3: dict(N=256, L=500, t1t2=2179, b0=True, b1=True, seq="bssfp", R=16.0, snr=40.0,
            iters=20, phantom_b0="smooth", smooth_b1=True),
    4: dict(N=256, L=1000, t1t2=1961, b0=True, b1=False, seq="bssfp", R=16.0, snr=40.0,
            iters=20, phantom_b0="ellipse", smooth_b1=False),
    5: dict(N=None, L=1000, t1t2=1961, b0=True, b1=False, seq="bssfp", R=None, snr=40.0,
            iters=20, phantom_b0="ellipse", smooth_b1=False, slices=64,
            sizes=(128, 192, 256, 320), R_range=(8.0, 24.0)),
}


def config(cfg: int, **over) -> dict:
    c = dict(CONFIGS[cfg])
    c.update(over)
    c["cfg"] = cfg
    return c


def make_dictionary(cfg: int, **over) -> dict:
    """Dictionary of workload ``cfg``: atoms complex64 [d, L] (unit norm), params float32 [d, P]."""
    c = config(cfg, **over)
    grid = param_grid(c["t1t2"], b0_hz=B0_AXIS if c["b0"] else None,
                      b1=B1_AXIS if c["b1"] else None)
    alpha = flip_train(c["L"])
    atoms = simulate_dictionary(grid["params"], grid["names"], alpha, c["seq"])
    grid.update(atoms=atoms, alpha=alpha, seq=c["seq"], L=c["L"])
    return grid


def _fingerprint_fn(seq, alpha):
    if seq == "fisp":
        return lambda t1, t2, b0, b1: epg_fisp(t1, t2, alpha, B1=b1)
    return lambda t1, t2, b0, b1: bssfp(t1, t2, b0, alpha, B1=b1)


def _snap(ph: dict, dic: dict) -> np.ndarray:
    """Snap every foreground voxel to its nearest valid grid cell; returns atom index [n]."""
    names = dic["names"]
    maps = {"T1": ph["T1"], "T2": ph["T2"], "B0": ph["B0"], "B1": ph["B1"]}
    n = ph["labels"].shape[0]
    idx = np.zeros(n, np.int64)
    fg = ph["labels"] >= 0
    cell = []
    for name, ax in zip(names, dic["axes"]):
        v = maps[name][fg]
        key = np.log(v) if name in ("T1", "T2") else v
        grid = np.log(ax) if name in ("T1", "T2") else ax
        cell.append(np.abs(key[:, None] - grid[None, :]).argmin(1))
    a = dic["cell_atom"][tuple(cell)]
    if np.any(a < 0):
        raise ValueError("snapped cell invalid (T2 >= T1)")
    idx[fg] = a
    return idx


def slice_geometry(cfg: int, i: int = 0, **over) -> tuple[int, float]:
    """(N, R) of slice i: fixed for workloads 1-4; for workload 5 a seeded draw of the matrix
    size from `sizes` and of the acceleration from `R_range`."""
    c = config(cfg, **over)
    N, R = c["N"], c["R"]
    if cfg == 5 and N is None:
        g = rng(2000 + 100 * cfg + i + 77)
        N = int(g.choice(np.asarray(c["sizes"])))
        R = float(g.uniform(*c["R_range"]))
    return N, R


def make_problem(cfg: int, i: int = 0, dic: dict | None = None, snap: bool = False,
                 full_sampling: bool = False, noiseless: bool = False, **over) -> dict:
    """Phantom, masks, ground truth X0 and k-space Y for slice ``i`` of workload ``cfg``.

    With ``snap`` the phantom's parameters are moved to grid values and X0_v = rho_v * D_j
    uses the stored atom (requires ``dic``); ``full_sampling`` keeps every line.
    """
    c = config(cfg, **over)
    L = c["L"]
    N, R = slice_geometry(cfg, i, **over)
    ph = ellipse_phantom(N, 2000 + 100 * cfg + i, b0=c["phantom_b0"], smooth_b1=c["smooth_b1"])
    masks = (np.ones((L, N), np.uint8) if full_sampling
             else line_masks(N, L, R, 3000 + 100 * cfg + i))
    alpha = flip_train(L)
    truth_idx = None
    if snap:
        truth_idx = _snap(ph, dic)
        X0 = (ph["rho"][:, None] * dic["atoms"][truth_idx].astype(np.complex128))
        X0[ph["labels"] < 0] = 0
        X0 = X0.astype(np.complex64)
        p = dic["params"][truth_idx]
        for k, name in enumerate(dic["names"]):
            ph[name] = np.where(ph["labels"] >= 0, p[:, k].astype(np.float64), ph[name])
    else:
        X0 = ground_truth(ph, _fingerprint_fn(c["seq"], alpha))
    snr = None if noiseless else c["snr"]
    Y = acquire(X0, masks, N, N, snr, 4000 + 100 * cfg + i)
    return {"cfg": cfg, "slice": i, "Ny": N, "Nx": N, "L": L, "R": R, "masks": masks,
            "Y": Y, "X0": X0, "phantom": ph, "truth_idx": truth_idx, "iters": c["iters"],
            "alpha": alpha}
