"""Launch-geometry autotuner for the tensor-core search (mrf_get_tune / mrf_set_tune).

The search kernel's geometry has four knobs: the MMA tile shape (bf16_pair = 0: 128 voxels x
256 atom rows per CTA; 1: 256 voxels x 256 rows on a CTA pair, each CTA staging half of every
atom block, so the pair reads each block once for twice the voxels), the cluster size C (CTAs
co-scheduled on the same atom blocks, each loading its own copy with plain TMA tile loads;
single CTAs only), the number of voxel tiles kept live per super-group (how many query tiles
the persistent clusters sweep together, i.e. the L2 working set), and the atom split S (work
units per voxel tile; 0 lets the library pick it from its makespan model).  For the
tensor-core tree search (mode "tree_tc") the grid is its own schedule instead: the tile shape of
the block-list search (CTA pairs or single CTAs), the voxel tiles that share one block list and
the chunks a list is cut into (`TREE_GRID`); the approximation factor of the timed projections
is passed with `proj`, e.g. {"eps": 0.5}, since the lists depend on it.  `tune` times
mrf_project on the caller's queries for each combination with CUDA events on the current
stream, keeps the fastest, applies it to the dictionary and records it in a JSON cache keyed by
device, dictionary size, frame count, voxel count and precision, so later processes can apply
the cached choice without timing again.  Every timed call is an ordinary projection; nothing
here changes numerical results (the candidate sets may differ between splits, the certified
answers do not).
"""
from __future__ import annotations

import itertools
import json
import os

from . import Dictionary, proj_opts, project

DEFAULT_GRID = {"bf16_pair": (0, 1), "bf16_cluster": (1, 2, 4),
                "bf16_live_tiles": (16, 32, 64), "bf16_splits": (0,)}
TREE_GRID = {"bf16_pair": (1, 2), "tree_tc_group": (2, 4, 8), "tree_tc_chunks": (16, 32)}


def _key(D: Dictionary, n: int, mode: str) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    return f"{dev}|d={D.d}|L={D.L}|n={n}|{mode}"


def load_cache(path: str) -> dict:
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def apply_cached(D: Dictionary, n: int, mode: str, path: str) -> dict | None:
    """Apply a cached geometry for (device, D, n, mode); returns it or None."""
    hit = load_cache(path).get(_key(D, n, mode))
    if hit:
        D.set_tune(**hit["tune"])
    return hit


def tune(D: Dictionary, Z, mode: str = "bf16", grid: dict | None = None, reps: int = 3,
         cache: str | None = None, proj: dict | None = None) -> dict:
    """Time every geometry of `grid` on the device queries Z ([n][L] complex64) and keep the
    fastest (uncertified projections of `mode`, with the extra projection options `proj`).
    Returns {"tune": best settings, "ms": its time, "table": all timings}."""
    import torch
    if grid is None:
        grid = TREE_GRID if mode == "tree_tc" else DEFAULT_GRID
    grid = dict(grid)
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device=Z.device)
    o = proj_opts(mode=mode, certify=False, **(proj or {}))
    stream = torch.cuda.current_stream()
    names = list(grid)
    table = []
    best = None
    for values in itertools.product(*(grid[k] for k in names)):
        setting = dict(zip(names, values))
        if setting.get("bf16_pair", 0) == 1 and setting.get("bf16_cluster", 1) != 1:
            continue                               # the pair form ignores the cluster size
        D.set_tune(**setting)
        project(D, Z, idx, opts=o)                 # warm-up (and first-use set-up)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            project(D, Z, idx, opts=o)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        got = D.get_tune()
        table.append({"tune": setting, "ms": ms, "splits_used": got["last_bf16_splits"],
                      "ctas": got["last_bf16_ctas"]})
        if best is None or ms < best["ms"]:
            best = table[-1]
    D.set_tune(**best["tune"])
    out = {"tune": best["tune"], "ms": best["ms"], "table": table}
    if cache:
        data = load_cache(cache)
        data[_key(D, n, mode)] = {"tune": best["tune"], "ms": best["ms"]}
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return out
