"""Excitation sequence and the discretised parameter grid of the dictionary.

The paper simulates an inversion-recovery sequence of L frames with a pseudo-random flip-angle
pattern, TR = 10 ms and TE = TR/2 (§6.1), and discretises (T1, T2, B0) on a grid whose cells with
T2 >= T1 are dropped (§3.1, eq. fingerprints).  The workloads here use a smooth-plus-noise flip
train alpha_t = 10 + 50|sin(pi t / 50)| + N(0, 1) degrees and log-spaced T1/T2 axes.
"""
from __future__ import annotations

import numpy as np

TR_MS = 10.0
TE_MS = 5.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def flip_train(L: int, seed: int | None = None) -> np.ndarray:
    """Flip angles in degrees, shape [L], float64 (seed defaults to 1810 + L)."""
    g = rng(1810 + L if seed is None else seed)
    t = np.arange(L, dtype=np.float64)
    return 10.0 + 50.0 * np.abs(np.sin(np.pi * t / 50.0)) + g.normal(0.0, 1.0, size=L)


def _log_axis(lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


def _valid_count(n1: int, n2: int, t1r, t2r) -> int:
    t1 = _log_axis(*t1r, n1)
    t2 = _log_axis(*t2r, n2)
    return int(np.searchsorted(t2, t1, side="left").sum())


def choose_t1t2(target: int, t1r=(100.0, 4000.0), t2r=(10.0, 600.0)) -> tuple[int, int]:
    """Smallest-error (n1, n2) whose count of valid (T2 < T1) cells is closest to ``target``."""
    best = None
    for n1 in range(8, 400):
        for n2 in range(max(4, n1 - 24), n1 + 25):
            c = _valid_count(n1, n2, t1r, t2r)
            key = (abs(c - target), abs(n1 - n2), n1)
            if best is None or key < best[0]:
                best = (key, n1, n2)
        if best[0][0] == 0 and n1 > best[1] + 30:
            break
    return best[1], best[2]


def param_grid(t1t2_target: int, b0_hz=None, b1=None,
               t1r=(100.0, 4000.0), t2r=(10.0, 600.0)) -> dict:
    """Dictionary parameter grid.

    Atoms are enumerated with T1 outermost, then T2, then B1, then B0 innermost; cells with
    T2 >= T1 are skipped.  Returns
      params      float32 [d, P]  columns (T1 ms, T2 ms[, B1][, B0 Hz])
      names       column names
      grid_shape  (n1, n2[, nB1][, nB0])
      cell_atom   int32 array of grid_shape: atom index of each cell, -1 where invalid
      axes        list of the per-axis value arrays
    """
    n1, n2 = choose_t1t2(t1t2_target, t1r, t2r)
    t1 = _log_axis(*t1r, n1)
    t2 = _log_axis(*t2r, n2)
    axes = [t1, t2]
    names = ["T1", "T2"]
    if b1 is not None:
        axes.append(np.asarray(b1, np.float64))
        names.append("B1")
    if b0_hz is not None:
        axes.append(np.asarray(b0_hz, np.float64))
        names.append("B0")
    shape = tuple(len(a) for a in axes)
    mesh = np.meshgrid(*axes, indexing="ij")
    valid = mesh[1] < mesh[0]
    cell_atom = np.full(shape, -1, np.int32)
    cell_atom[valid] = np.arange(int(valid.sum()), dtype=np.int32)
    params = np.stack([m[valid] for m in mesh], axis=1).astype(np.float32)
    return {"params": params, "names": names, "grid_shape": shape,
            "cell_atom": cell_atom, "axes": axes}
