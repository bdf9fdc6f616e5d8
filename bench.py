"""Benchmark: BLIP iterations with the exhaustive BF16 tensor-core matched filter.

Workload (per GPU): a 256 x 256 ellipse phantom, L = 1000 frames, an IR-bSSFP dictionary of
100,011 atoms over (T1, T2, B0 in -50:2:50 Hz), 1/16 variable-density Cartesian lines, 40 dB.
One step = one BLIP iteration through the C ABI (mrf_ipg_step: y-FFTs + mask + gradient
combine + BF16 query packing + tcgen05 search with fused top-K + FP32/FP64 rescore + density
+ X update) followed by the look-up table (mrf_lut).  Metric: voxel-atom matches per second,
n * d per step.  Inputs (dictionary operand 800 MB, image 524 MB) are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank reconstructs its own slice with its own copy of the dictionary
(no data exchange; weak scaling); the timed region is bracketed by barriers and the max over
ranks is reported.  ``--impl reference`` times the float64 CPU oracle on a bounded voxel sample
of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("voxel·atom matches/s and recon s/slice at fixed T1/T2 error; "
          "learned/BF16 vs FP32 exact")
UNIT = "voxel·atom matches/s"
WORKLOAD = "blip-bf16-exhaustive 256x256 L=1000 d=100011 (T1,T2,B0) IR-bSSFP R=16 40dB"


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """x of the slowest rank (max over the process group; x itself for one process)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_slices(n_slices: int, rank: int, world: int) -> list[int]:
    """Slices of this rank: dealt round-robin, so every slice goes to exactly one rank."""
    return list(range(rank, n_slices, world))


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "_source": "fallback"}


def kernel_digest() -> str:
    src = os.path.join(ROOT, "paper_1810_01967_gb300", "csrc", "bf16.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def traffic_per_launch(n: int, d: int, mode: str = "bf16") -> float | None:
    """DRAM bytes per launch of the search kernel (BF16 or FP8 operands) from the committed ncu
    summary, scaled to this workload by the number of voxel-atom pairs; None if the kernel
    changed since."""
    p = os.path.join(ROOT, "profiles", f"{mode}_search_traffic.json")
    if not os.path.exists(p):
        return None
    t = json.load(open(p))
    if t.get("kernel_sha256_16") != kernel_digest():
        return None
    return float(t["dram_bytes_per_pair"]) * n * d


def t_accuracy(est, truth, mask) -> float:
    """T1 / T2 accuracy as the paper reports it: 1 - mean over the object voxels (mask) of the
    relative error |est - truth| / truth."""
    e, t = np.asarray(est, np.float64)[mask], np.asarray(truth, np.float64)[mask]
    return float(1.0 - np.mean(np.abs(e - t) / t))


def oracle_baseline(Zs: np.ndarray, atoms: np.ndarray, target_s: float = 12.0,
                    gpu_idx=None) -> dict:
    """Time the oracle's exhaustive projection on a voxel sample (about target_s seconds).
    gpu_idx(Z) -> atom indices, if given, projects the timed voxels on the GPU as well and the
    result carries the share of voxels where both sides pick the same atom."""
    from oracle import mrf_oracle as mo
    d = atoms.shape[0]
    t0 = time.perf_counter()
    mo.project(Zs[:32], atoms)
    t32 = time.perf_counter() - t0
    m = int(min(len(Zs), max(32, 32 * target_s / max(t32, 1e-3))))
    m = max(32, (m // 32) * 32)
    t0 = time.perf_counter()
    ref = mo.project(Zs[:m], atoms)
    dt = time.perf_counter() - t0
    out = {"value": m * d / dt, "unit": UNIT, "cores": cores(), "kind": "oracle",
           "sample": f"{m} voxels x {d} atoms x L={atoms.shape[1]}, float64 exhaustive "
                     f"projection (numpy complex128), {dt:.1f} s"}
    if gpu_idx is not None:
        try:
            out["gpu_agreement_on_sample"] = float(np.mean(gpu_idx(Zs[:m]) == ref["idx"]))
        except Exception as e:             # an auxiliary figure: report, do not abort the bench
            out["gpu_agreement_error"] = f"{type(e).__name__}: {e}"[:200]
    return out


def oracle_baseline_1thread(Zs: np.ndarray, atoms: np.ndarray, target_s: float = 6.0) -> dict:
    """The same oracle timing with one thread (BLAS pinned to one thread in a child process)."""
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        np.save(os.path.join(tmp, "z.npy"), Zs)
        np.save(os.path.join(tmp, "a.npy"), atoms)
        code = (
            "import sys, time, json, numpy as np\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "from oracle import mrf_oracle as mo\n"
            f"Z = np.load({os.path.join(tmp, 'z.npy')!r}); A = np.load({os.path.join(tmp, 'a.npy')!r})\n"
            "t0 = time.perf_counter(); mo.project(Z[:4], A); t4 = time.perf_counter() - t0\n"
            f"m = int(min(len(Z), max(4, 4 * {target_s} / max(t4, 1e-3))))\n"
            "t0 = time.perf_counter(); mo.project(Z[:m], A); dt = time.perf_counter() - t0\n"
            "print(json.dumps({'m': m, 'dt': dt}))\n")
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                   MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    o = json.loads(r.stdout.strip().splitlines()[-1])
    d = atoms.shape[0]
    return {"value": o["m"] * d / o["dt"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{o['m']} voxels x {d} atoms, one BLAS thread, {o['dt']:.1f} s"}


def small_workload_full(mrf, dev) -> dict:
    """The small workload (32², L = 100, 2,001 atoms, 10 iterations) reconstructed whole by the
    float64 oracle on the host and by the library (BF16 and FP32) on the GPU."""
    import torch
    import mrfgen
    from oracle import mrf_oracle as mo
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, d, iters = Ny * Nx, dic["atoms"].shape[0], p["iters"]
    t0 = time.perf_counter()
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=iters)
    cpu_s = time.perf_counter() - t0
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, torch.from_numpy(p["masks"]).to(dev))
    Yd = torch.from_numpy(p["Y"]).to(dev)
    out = {"oracle_s": cpu_s, "oracle_cores": cores(), "n": n, "d": d, "L": L, "iters": iters}
    for mode in ("bf16", "fp32"):
        X = torch.empty((n, L), dtype=torch.complex64, device=dev)
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        ro = mrf.recon_opts(iters=iters, mode=mode)
        mrf.reconstruct(D, op, Yd, X, idx, opts=ro)                  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mrf.reconstruct(D, op, Yd, X, idx, opts=ro)
        torch.cuda.synchronize()
        out[f"gpu_{mode}_s"] = time.perf_counter() - t0
        out[f"gpu_{mode}_agreement_with_oracle"] = float(np.mean(idx.cpu().numpy() == ref["idx"]))
    D.close()
    return out


def make_workload(slice_idx: int):
    import mrfgen
    dic = mrfgen.make_dictionary(2)
    p = mrfgen.make_problem(2, i=slice_idx, dic=dic)
    return dic, p


def train_learned(mrf, D, dic, dev, phantoms: int = 64, steps: int = 2000):
    """Learned proposal for the workload's dictionary: aliasing residues from 4 IPG iterates of
    `phantoms` seeded 96x96 training phantoms, then `steps` Adam steps of 1024 synthetic
    fingerprints (2M at the defaults).  Returns (model, seconds of GPU training)."""
    import torch
    import mrfgen
    M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=512)
    for k in range(phantoms):
        pk = mrfgen.make_problem(2, i=1000 + k, dic=dic, N=96)
        Ny, Nx, L = pk["Ny"], pk["Nx"], pk["L"]
        n = Ny * Nx
        opk = mrf.make_op(Ny, Nx, L, torch.from_numpy(pk["masks"]).to(dev))
        AHY = torch.empty((n, L), dtype=torch.complex64, device=dev)
        mrf.adjoint(opk, torch.from_numpy(pk["Y"]).to(dev), AHY)
        X0 = torch.from_numpy(pk["X0"]).to(dev)
        X = torch.zeros((n, L), dtype=torch.complex64, device=dev)
        idx = torch.zeros(n, dtype=torch.int32, device=dev)
        Zk = torch.empty_like(X)
        for _ in range(4):
            mrf.gradient(D, opk, AHY, X, 1.0, Zk)
            M.add_residues(Zk, X0)
            mrf.ipg_step(D, opk, AHY, X, 1.0, idx, opts=mrf.proj_opts(mode="bf16", certify=False))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = M.train(steps=steps, batch=1024, lr=1e-3, history=True)
    torch.cuda.synchronize()
    return M, time.perf_counter() - t0, hist


def reconstruction_quality(mrf, D, op, p, dic, dev, stream, iters: int, fp32: bool = True,
                           forms: bool = True, keep: bool = False):
    """Whole reconstructions (iters BLIP / CoverBLIP iterations) of the slice with every form of
    the projection -- BF16 exhaustive, FP32 exhaustive (the plain comparator), cover tree
    (eps = 0.4, CoverBLIP) and the learned proposal (threshold 0.98) -- reporting time per slice,
    matches/s, T1/T2 accuracy against the phantom (mask rho != 0), B0 error, atom agreement with
    FP32 and the search work.  With `keep` the second dictionary (cover tree, FP8 operand,
    trained learned model attached) is returned open with the results, for the caller to reuse
    and close."""
    import torch
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, d = Ny * Nx, dic["atoms"].shape[0]
    ph = p["phantom"]
    fg = ph["labels"] >= 0
    Yd = torch.from_numpy(p["Y"]).to(dev)
    out, idxs = {}, {}
    runs = [("bf16", {}), ("fp8", {})]
    if fp32:
        runs.append(("fp32", {}))
    D2 = None
    if forms:
        # a second dictionary with the cover tree and the learned model; the caller's D stays
        # open (its owner closes it)
        t0 = time.perf_counter()
        D2 = mrf.build_dict_index(dic["atoms"], dic["params"], grid_shape=dic["grid_shape"],
                                  build_tree=True, pack_fp8=True, tree_tc=True)
        out["tree_build_s"] = time.perf_counter() - t0
        M, tsec, hist = train_learned(mrf, D2, dic, dev)
        mrf.attach_mlp(D2, M)
        out["learned_train"] = {"gpu_s": tsec, "fingerprints": 2000 * 1024,
                                "loss_first": float(hist[:20].mean()),
                                "loss_last": float(hist[-100:].mean())}
        D = D2
        runs += [("covertree", {"eps": 0.4}), ("tree_tc", {"eps": 0.4}),
                 ("learned", {"fallback_thr": 0.98})]
    for mode, kw in runs:
        X = torch.empty((n, L), dtype=torch.complex64, device=dev)
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device=dev)
        ro = mrf.recon_opts(iters=iters, mode=mode, certify=False, **kw)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = mrf.reconstruct(D, op, Yd, X, idx, None, prm, opts=ro, stats=True)
        b.record(stream)
        torch.cuda.synchronize()
        s = a.elapsed_time(b) / 1e3
        pr = prm.cpu().numpy()
        idxs[mode] = idx.cpu().numpy()
        out[mode] = {"s_per_slice": s, "iters": iters, "matches_per_s": n * d * iters / s,
                     "T1_acc": t_accuracy(pr[:, 0], ph["T1"], fg),
                     "T2_acc": t_accuracy(pr[:, 1], ph["T2"], fg),
                     "B0_mae_hz": float(np.mean(np.abs(pr[fg, 2] - ph["B0"][fg]))),
                     "exhaustive_fallback_voxel_iters": st["n_fallback"],
                     "tree_distance_evals": st["n_dist_evals"], **kw}
    if forms:
        # temporal subspace compression (§3.3): BF16 BLIP on s-dimensional proxies
        A_dev = torch.from_numpy(dic["atoms"]).to(dev)
        energy = float(np.sum(np.abs(dic["atoms"].astype(np.complex128)) ** 2))
        for s in (50, 200):
            t0 = time.perf_counter()
            V, eig = mrf.svd_basis(D, s)
            basis_s = time.perf_counter() - t0
            so = mrf.SvdOp(V, op)
            Ac = torch.empty((d, s), dtype=torch.complex64, device=dev)
            so.compress(A_dev, Ac)
            Dc = mrf.build_dict_index(Ac, dic["params"])
            Xc = torch.empty((n, s), dtype=torch.complex64, device=dev)
            idx = torch.empty(n, dtype=torch.int32, device=dev)
            prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device=dev)
            o = mrf.proj_opts(mode="bf16", certify=False)
            so.reconstruct(Dc, Yd, 1, Xc, idx, opts=o)        # warm-up (plans, scratch)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            so.reconstruct(Dc, Yd, iters, Xc, idx, None, None, prm, opts=o)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1e3
            pr = prm.cpu().numpy()
            key = f"bf16_svd{s}"
            idxs[key] = idx.cpu().numpy()
            out[key] = {"s_per_slice": sec, "iters": iters, "s": s,
                        "matches_per_s": n * d * iters / sec,
                        "T1_acc": t_accuracy(pr[:, 0], ph["T1"], fg),
                        "T2_acc": t_accuracy(pr[:, 1], ph["T2"], fg),
                        "B0_mae_hz": float(np.mean(np.abs(pr[fg, 2] - ph["B0"][fg]))),
                        "energy_kept": float(eig.sum() / energy), "basis_s": basis_s}
            so.close()
            Dc.close()
        del A_dev
        # the paper's real positive density with the phase alignment of §4.3
        Da = mrf.build_dict_index(dic["atoms"], dic["params"], phase_align=True)
        X = torch.empty((n, L), dtype=torch.complex64, device=dev)
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device=dev)
        ro = mrf.recon_opts(iters=iters, mode="bf16", certify=False, cone="real_pos")
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mrf.reconstruct(Da, op, Yd, X, idx, None, prm, opts=ro)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        pr = prm.cpu().numpy()
        idxs["bf16_aligned_real"] = idx.cpu().numpy()
        out["bf16_aligned_real"] = {"s_per_slice": sec, "iters": iters,
                                    "matches_per_s": n * d * iters / sec,
                                    "T1_acc": t_accuracy(pr[:, 0], ph["T1"], fg),
                                    "T2_acc": t_accuracy(pr[:, 1], ph["T2"], fg),
                                    "B0_mae_hz": float(np.mean(np.abs(pr[fg, 2] - ph["B0"][fg])))}
        Da.close()
    if D2 is not None and not keep:
        D2.close()
        D2 = None
    for mode in idxs:
        if "fp32" in idxs:
            out[mode]["atom_agreement_vs_fp32"] = float(np.mean(idxs[mode] == idxs["fp32"]))
    return (out, D2) if keep else out


def peaks_sustained() -> tuple[float, str]:
    pk = measured_peaks()
    return (float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))),
            pk["_source"] + " sustained bf16")


def exact_tc_leg(mrf, D, op, AHY, n, d, L, stream, peak, steps: int = 5) -> dict:
    """The exact tensor-core form (split-BF16, certified) on the same slice: `steps` BLIP
    iterations from X = 0 timed with CUDA events, then the same steps with the stage profiler
    for the search kernel's duration and the voxels certification sent to the FP32 search.
    Roofline: 8 L flop per pair against a third of the sustained BF16 peak (three products)."""
    import torch
    X = torch.zeros((n, L), dtype=torch.complex64, device=AHY.device)
    idx = torch.zeros(n, dtype=torch.int32, device=AHY.device)
    rho = torch.empty(n, dtype=torch.complex64, device=AHY.device)
    o = mrf.proj_opts(mode="bf16x3", certify=True)
    mrf.ipg_step(D, op, AHY, X, 1.0, idx, rho, opts=o)          # warm-up (scratch, maps)
    X.zero_()
    idx.zero_()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        mrf.ipg_step(D, op, AHY, X, 1.0, idx, rho, opts=o)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    X.zero_()
    idx.zero_()
    mrf.profile_enable(True)
    unc = []
    for _ in range(steps):
        st = mrf.ipg_step(D, op, AHY, X, 1.0, idx, rho, opts=o, stats=True)
        unc.append(int(st["n_uncertified"]))
    torch.cuda.synchronize()
    prof = mrf.profile_read()
    mrf.profile_enable(False)
    sm, sl = prof["search_tc"]
    fl = 8.0 * L * n * d
    ach = fl * sl / (sm / 1e3) / 1e12 if sm else 0.0
    pk, src = peak
    return {"matches_per_s": n * d / (ms / 1e3), "ms_per_iteration": ms, "iterations": steps,
            "uncertified_voxels_per_iteration": unc,
            "uncertified_fraction_max": max(unc) / n if unc else None,
            "stage_ms_per_iteration": {k: v[0] / steps for k, v in prof.items()},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": pk / 3.0,
                         "unit": "TFLOP/s", "frac": ach / (pk / 3.0), "kernel": "k_tc_topk (split)",
                         "traffic": traffic_per_launch(n, d, "bf16x3"),
                         "peak_source": src + " / 3 (three BF16 products per pair)",
                         "flops_per_launch": fl}}


def run_profile_case(args) -> None:
    """Projection only (mrf_project) on N voxels of the workload's slice: the small case for
    kernel-level ncu captures (about 2 GB on the device).  Exhaustive modes project the first
    N rows of A^H Y (so does the tensor-core tree search, eps 0.5, uncertified: its
    block-list kernel over the depth-first BF16 operand); the cover tree (eps 0.4) projects the
    phantom's object fingerprints with
    the slice's noise level, i.e. queries near the dictionary, where the tree search does its
    work instead of routing far queries to the exhaustive search.  Two more cases time single
    stages: `gradient` runs whole IPG steps (mrf_ipg_step, fixed mu = 1) of the full N x N x L
    slice against the first 4,096 atoms, so the fused gradient kernel runs at full size with a
    small dictionary (N voxels ignored), `mlp` runs the learned proposal's BF16 tensor-core
    inference of N fingerprints (random network: the timing does not depend on the weights),
    and `learned` the whole learned projection of the first N rows of A^H Y with that network
    (inference, neighbourhood rescore, exhaustive fallback)."""
    import torch
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    b.build()
    dic, p = make_workload(0)
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = args.profile_case
    if args.mode in ("gradient", "mlp", "learned"):
        run_stage_case(args, mrf, dic, p)
        return
    tree = args.mode == "covertree"
    ttc = args.mode == "tree_tc"
    D = mrf.build_dict_index(dic["atoms"], dic["params"], pack_fp8=(args.mode == "fp8"),
                             build_tree=tree or ttc, tree_tc=ttc,
                             pack_bf16x3=(args.mode == "bf16x3"))
    if tree:
        fg = np.flatnonzero(p["phantom"]["labels"] >= 0)
        g = np.random.Generator(np.random.PCG64(123))
        X0 = p["X0"][fg[g.integers(0, fg.size, n)]].astype(np.complex128)
        sig = 0.01 * np.linalg.norm(X0, axis=1, keepdims=True) / np.sqrt(2 * L)
        X0 += sig * (g.standard_normal(X0.shape) + 1j * g.standard_normal(X0.shape))
        Z = torch.from_numpy(X0.astype(np.complex64)).cuda()
    else:
        mask = torch.from_numpy(p["masks"]).cuda()
        op = mrf.make_op(Ny, Nx, L, mask)
        AHY = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
        mrf.adjoint(op, torch.from_numpy(p["Y"]).cuda(), AHY)
        Z = AHY[:n].contiguous()
        del AHY
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    o = mrf.proj_opts(mode=args.mode, certify=(args.mode == "bf16x3"),
                      eps=0.4 if tree else (0.5 if ttc else 0.0))
    mrf.profile_enable(True)
    st = None
    for i in range(args.steps):
        st = mrf.project(D, Z, idx, rho, opts=o, stats=(i == args.steps - 1))
    prof = mrf.profile_read()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n, "d": int(dic["atoms"].shape[0]), "L": L,
                      "stage_ms": {k: v[0] for k, v in prof.items()},
                      "stage_launches": {k: v[1] for k, v in prof.items()},
                      "stats_last_step": st}))


def run_stage_case(args, mrf, dic, p) -> None:
    import torch
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    mrf.profile_enable(True)
    if args.mode == "gradient":
        D = mrf.build_dict_index(np.ascontiguousarray(dic["atoms"][:4096]), None)
        op = mrf.make_op(Ny, Nx, L, torch.from_numpy(p["masks"]).cuda())
        AHY = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
        mrf.adjoint(op, torch.from_numpy(p["Y"]).cuda(), AHY)
        X = AHY.clone()
        idx = torch.zeros(Ny * Nx, dtype=torch.int32, device="cuda")
        o = mrf.proj_opts(mode="bf16", certify=False)

        def call():
            mrf.ipg_step(D, op, AHY, X, 1.0, idx, opts=o)
        n = Ny * Nx
    elif args.mode == "learned":
        D = mrf.build_dict_index(dic["atoms"], dic["params"], grid_shape=dic["grid_shape"])
        M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=512, residue_pool=4096)
        mrf.attach_mlp(D, M)
        n = args.profile_case
        op = mrf.make_op(Ny, Nx, L, torch.from_numpy(p["masks"]).cuda())
        AHY = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
        mrf.adjoint(op, torch.from_numpy(p["Y"]).cuda(), AHY)
        Z = AHY[:n].contiguous()
        del AHY
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        rho = torch.empty(n, dtype=torch.complex64, device="cuda")
        o = mrf.proj_opts(mode="learned", certify=False, fallback_thr=0.98)

        def call():
            mrf.project(D, Z, idx, rho, opts=o)
    else:
        D = mrf.build_dict_index(dic["atoms"], dic["params"], grid_shape=dic["grid_shape"],
                                 pack_bf16=False)
        M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=512, residue_pool=4096)
        n = args.profile_case
        g = torch.Generator(device="cuda").manual_seed(7)
        Xin = torch.randn((n, 2 * L), generator=g, device="cuda", dtype=torch.float32)
        Y = torch.empty((n, 3), dtype=torch.float32, device="cuda")

        def call():
            M.infer(Xin, Y)
    call()                                   # first call: plans and scratch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    prof = mrf.profile_read()
    print(json.dumps({"profile_case": n, "mode": args.mode, "L": L,
                      "ms_per_call": e0.elapsed_time(e1) / args.steps,
                      "stage_ms": {k: v[0] for k, v in prof.items()},
                      "stage_launches": {k: v[1] for k, v in prof.items()}}))


SLICES_WORKLOAD = ("64 slices of {128,192,256,320}^2 (seeded draw), L=1000, d=100011 shared "
                   "(T1,T2,B0) IR-bSSFP, R in [8,24], 20 BLIP iterations")


def slices_inputs(dic, dev, rank: int = 0, world: int = 1):
    """The 64-slice workload's seeded geometry (matrix size and acceleration per slice), this
    rank's slices, and one generated slice per matrix size (masks and k-space on the device),
    reused by every slice of that size."""
    import torch
    import mrfgen
    geo = [mrfgen.slice_geometry(5, i) for i in range(64)]
    mine = rank_slices(64, rank, world)
    first = {}
    for i in mine:
        first.setdefault(geo[i][0], i)
    probs = {N: mrfgen.make_problem(5, i, dic=dic) for N, i in first.items()}
    masks = {N: torch.from_numpy(p["masks"]).to(dev) for N, p in probs.items()}
    Ys = {N: torch.from_numpy(p["Y"]).to(dev) for N, p in probs.items()}
    return geo, mine, masks, Ys


def slices_leg(mrf, D, dic, dev, stream, masks, Ys, geo, mine, forms, group, iters, world,
               autotune_on, both=True, model=None):
    """The batching form's measurement on the 64-slice workload (all slices submitted at t = 0):
    per form, one batch of all slices (latency = the makespan, when `both`) and groups of
    `group` slices, shortest first (latency = its group's completion).  `model` (an MLP already
    attached to D) skips the learned form's training.  Returns (per-form results, training
    seconds, autotuned geometries)."""
    import torch
    import torch.distributed as dist

    def sync():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    L = dic["atoms"].shape[1]
    first = {}
    for i in mine:
        first.setdefault(geo[i][0], i)
    out = {}
    mlp_s = None
    tuned = {}
    Zt = None
    if autotune_on:
        # the largest slice's A^H Y: the autotuner times the search geometries on it, once per
        # element type (the learned form's fallback searches in BF16)
        from paper_1810_01967_gb300 import autotune
        Nb = max(first)
        opb = mrf.make_op(Nb, Nb, L, masks[Nb])
        Zt = torch.empty((Nb * Nb, L), dtype=torch.complex64, device=dev)
        mrf.adjoint(opb, Ys[Nb], Zt)
    for mode, graph in forms:
        if Zt is not None:
            tmode = "fp8" if mode == "fp8" else "bf16"
            if tmode not in tuned:
                tuned[tmode] = autotune.tune(D, Zt, tmode, reps=2)
            else:
                D.set_tune(**tuned[tmode]["tune"])
        kw = {}
        if mode == "learned":
            if model is None:
                M, mlp_s, _ = train_learned(mrf, D, dic, dev)
                mrf.attach_mlp(D, M)
            kw = {"fallback_thr": 0.98}
        if mode == "tree_tc":
            kw = {"eps": 0.4}
        o = mrf.proj_opts(mode=mode, certify=False, **kw)
        # --- all slices in one batch
        t_all = None
        if both:
            ops = [mrf.make_op(geo[i][0], geo[i][0], L, masks[geo[i][0]]) for i in mine]
            B = mrf.Batch(D, ops)
            B.load([Ys[geo[i][0]] for i in mine])
            B.run(2, 1.0, o, use_graph=graph)        # warm-up: plans, scratch, graph capture
            sync()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.load([Ys[geo[i][0]] for i in mine])
            B.run(iters, 1.0, o, use_graph=graph)
            e.record(stream)
            sync()
            t_all = max_over_ranks(a.elapsed_time(e) / 1e3, world, dev)
            B.close()
            del B
        # --- groups of `group` slices, shortest first
        order = sorted(mine, key=lambda i: (geo[i][0], i))
        groups = [order[k:k + group] for k in range(0, len(order), group)]
        # warm up the largest group first: it sizes the dictionary's scratch, so no later
        # warm-up reallocates buffers that an earlier group's captured graph references
        Bs = [None] * len(groups)
        for k in reversed(range(len(groups))):
            gi = groups[k]
            og = [mrf.make_op(geo[i][0], geo[i][0], L, masks[geo[i][0]]) for i in gi]
            Bg = mrf.Batch(D, og)
            Bg.load([Ys[geo[i][0]] for i in gi])
            Bg.run(2, 1.0, o, use_graph=graph)
            Bs[k] = Bg
        sync()
        a = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ends = []
        for gi, Bg in zip(groups, Bs):
            Bg.load([Ys[geo[i][0]] for i in gi])
            Bg.run(iters, 1.0, o, use_graph=graph)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            ends.append(ev)
        sync()
        lat = []
        for gi, ev in zip(groups, ends):
            lat += [a.elapsed_time(ev) / 1e3] * len(gi)
        t_grp = max_over_ranks(max(lat), world, dev)
        for Bg in Bs:
            Bg.close()
        del Bs
        lat_all = lat
        if world > 1:
            g = [None] * world
            dist.all_gather_object(g, lat)
            lat_all = [x for part in g for x in part]
        one = None if t_all is None else {"s": t_all, "slices_per_s": 64 / t_all,
                                          "p50_s": t_all, "p99_s": t_all}
        out[mode] = {"graph": graph, "one_batch": one,
                     "groups": {"group": group, "s": t_grp, "slices_per_s": 64 / t_grp,
                                "p50_s": float(np.percentile(lat_all, 50)),
                                "p99_s": float(np.percentile(lat_all, 99))}, **kw}
    return out, mlp_s, tuned


def run_slices(args) -> None:
    """The batching form on the 64-slice workload: every slice's 20 BLIP iterations through
    mrf_batch.  Two schedules, all slices submitted at t = 0: one batch of all slices (one
    projection launch per iteration covers every slice; latency = the makespan), and groups of
    `--group` slices, shortest first (per-slice latency = its group's completion).  Forms: BF16,
    FP8 and the learned proposal with exhaustive fallback, each iteration replayed as a CUDA
    graph (the fallback reads its voxel count on the device).  Inputs: one seeded slice per matrix size
    is generated (k-space, masks), and the 64 slices of the seeded draw use the generated slice
    of their size.  Under torchrun the slices are dealt to ranks round-robin."""
    import torch
    import torch.distributed as dist
    import mrfgen
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    if rank == 0 or world == 1:
        b.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    dic = mrfgen.make_dictionary(5)
    atoms, params = dic["atoms"], dic["params"]
    d, L = atoms.shape
    geo, mine, masks, Ys = slices_inputs(dic, dev, rank, world)
    D = mrf.build_dict_index(atoms, params, grid_shape=dic["grid_shape"], pack_fp8=True)
    iters = args.iters
    forms = [("bf16", True), ("fp8", True)]
    if not args.no_forms:
        forms.append(("learned", True))

    def sync():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    out, mlp_s, tuned = slices_leg(mrf, D, dic, dev, stream, masks, Ys, geo, mine, forms,
                                   args.group, iters, world, not args.no_autotune, both=True)
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    best = out["bf16"]["one_batch"]
    line = {"metric": "slices/s (64 uneven slices, 20 BLIP iterations each)",
            "value": best["slices_per_s"], "unit": "slices/s", "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * best["s"], "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": SLICES_WORKLOAD, "voxels": int(sum(geo[i][0] ** 2 for i in range(64))),
                       "inputs": "one generated slice per matrix size, reused by the slices of that size"},
            "forms": out, "learned_train_gpu_s": mlp_s,
            "autotune": {m: {"tune": t["tune"], "ms": t["ms"]} for m, t in tuned.items()} or None}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


TREE_WORKLOAD = ("256x256, L=500, d=999,702 (T1,T2,B1,B0) IR-bSSFP, smooth B0/B1 fields, R=16, "
                 "20 iterations: CoverBLIP eps in {0, 0.2, 0.5, 1.0} vs BF16 brute force, "
                 "and both searches on temporally compressed fingerprints")


def tree_leg(mrf, dev, stream, iters: int, tree_svd=()) -> dict:
    """The cover-tree workload: the million-atom dictionary, the tree built on the host, then
    whole reconstructions of one slice with the BF16 tensor-core brute force and with CoverBLIP
    (Algorithm 2, warm-started searches) at eps in {0, 0.2, 0.5, 1.0}, plus one cold tree
    projection of A^H Y per eps for the search kernel's own rate (distance evaluations, unique
    bytes), and for each s of `tree_svd` both searches on temporally compressed fingerprints."""
    import torch
    import mrfgen

    class _A:
        pass

    args = _A()
    args.iters, args.tree_svd = iters, list(tree_svd)
    t0 = time.perf_counter()
    dic = mrfgen.make_dictionary(3)
    p = mrfgen.make_problem(3, dic=dic)
    gen_s = time.perf_counter() - t0
    atoms, params = dic["atoms"], dic["params"]
    d, L = atoms.shape
    Ny, Nx = p["Ny"], p["Nx"]
    n = Ny * Nx
    t0 = time.perf_counter()
    D = mrf.build_dict_index(atoms, params, build_tree=True, tree_tc=True)
    build_s = time.perf_counter() - t0
    info = D.tree_info()
    op = mrf.make_op(Ny, Nx, L, torch.from_numpy(p["masks"]).to(dev))
    Yd = torch.from_numpy(p["Y"]).to(dev)
    ph = p["phantom"]
    fg = ph["labels"] >= 0
    AHY = torch.empty((n, L), dtype=torch.complex64, device=dev)
    mrf.adjoint(op, Yd, AHY)
    runs = ([("bf16", {})] + [("covertree", {"eps": e}) for e in (0.0, 0.2, 0.5, 1.0)]
            + [("tree_tc", {"eps": e}) for e in (0.0, 0.2, 0.5, 1.0)])
    out = {}
    ref_idx = None
    for mode, kw in runs:
        X = torch.empty((n, L), dtype=torch.complex64, device=dev)
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        prm = torch.empty((n, params.shape[1]), dtype=torch.float32, device=dev)
        ro = mrf.recon_opts(iters=args.iters, mode=mode, certify=False, **kw)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = mrf.reconstruct(D, op, Yd, X, idx, None, prm, opts=ro, stats=True)
        e.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(e) / 1e3
        pr = prm.cpu().numpy()
        gi = idx.cpu().numpy()
        if mode == "bf16":
            ref_idx = gi
        r = {"s_per_slice": sec, "matches_per_s_bruteforce_equiv": n * d * args.iters / sec,
             "T1_acc": t_accuracy(pr[:, 0], ph["T1"], fg),
             "T2_acc": t_accuracy(pr[:, 1], ph["T2"], fg),
             "atom_agreement_vs_bf16": float(np.mean(gi == ref_idx)),
             "distance_evals": st["n_dist_evals"],
             "exhaustive_voxel_iters": st["n_fallback"], **kw}
        if mode == "tree_tc":
            # one cold projection of A^H Y: centre bounds and tile lists, then the block-list
            # search on the tensor cores
            ii = torch.empty(n, dtype=torch.int32, device=dev)
            mrf.profile_enable(True)
            s2 = mrf.project(D, AHY, ii, opts=mrf.proj_opts(mode="tree_tc", eps=kw["eps"],
                                                           certify=False), stats=True)
            prof = mrf.profile_read()
            mrf.profile_enable(False)
            sms = prof["search_tc"][0]
            ach = 8.0 * L * s2["n_dist_evals"] / (sms / 1e3) / 1e12 if sms else None
            sus, sus_src = peaks_sustained()
            r["first_projection"] = {
                "bounds_lists_ms": prof["search_proposal"][0], "search_ms": sms,
                "merge_ms": prof["merge"][0],
                "pairs_fraction_of_bruteforce": s2["n_dist_evals"] / (d * n),
                # the block-list kernel's rate on the pairs it searched (8 L flop per pair)
                "search_roofline": {"bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
                                    "peak": sus, "peak_source": sus_src,
                                    "frac": (ach / sus) if ach else None}}
        if mode == "covertree":
            # one cold projection of A^H Y: the tree search kernel's own rate
            ii = torch.empty(n, dtype=torch.int32, device=dev)
            mrf.profile_enable(True)
            s2 = mrf.project(D, AHY, ii, opts=mrf.proj_opts(mode="covertree", eps=kw["eps"],
                                                           certify=False), stats=True)
            prof = mrf.profile_read()
            mrf.profile_enable(False)
            ms = prof["search_proposal"][0]
            r["first_projection"] = {
                "tree_ms": ms, "fallback_ms": prof["fallback"][0], "merge_ms": prof["merge"][0],
                "evals_per_voxel": s2["n_dist_evals"] / n,
                "bruteforce_ratio": d * n / max(s2["n_dist_evals"], 1),
                "routed_voxels": s2["n_fallback"],
                "unique_GBps": s2["n_dist_evals"] * L * 8 / (ms / 1e3) / 1e9 if ms else None}
        out[f"{mode}" + (f"_eps{kw['eps']}" if kw else "")] = r
    # the temporal compression option for both searches (§3.3, §6): basis, compressed atoms,
    # a tree built on them, then compressed reconstructions (basis and tree build reported
    # apart from the per-slice time)
    if args.tree_svd:
        A_dev = torch.from_numpy(atoms).to(dev)
        for s in args.tree_svd:
            t0 = time.perf_counter()
            V, eig = mrf.svd_basis(D, s)
            basis_s = time.perf_counter() - t0
            so = mrf.SvdOp(V, op)
            Ac = torch.empty((d, s), dtype=torch.complex64, device=dev)
            so.compress(A_dev, Ac)
            t0 = time.perf_counter()
            Dc = mrf.build_dict_index(Ac, params, build_tree=True)
            tree_s = time.perf_counter() - t0
            AHYc = torch.empty((n, s), dtype=torch.complex64, device=dev)
            so.compress(AHY, AHYc)
            Xc = torch.empty((n, s), dtype=torch.complex64, device=dev)
            idx = torch.empty(n, dtype=torch.int32, device=dev)
            prm = torch.empty((n, params.shape[1]), dtype=torch.float32, device=dev)
            for mode, kw in [("bf16", {})] + [("covertree", {"eps": e}) for e in (0.0, 0.5)]:
                o = mrf.proj_opts(mode=mode, certify=False, **kw)
                so.reconstruct(Dc, Yd, 1, Xc, idx, opts=o)        # warm-up (plans, scratch)
                mrf.profile_enable(True)
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                so.reconstruct(Dc, Yd, args.iters, Xc, idx, None, None, prm, opts=o)
                e.record(stream)
                torch.cuda.synchronize()
                prof = mrf.profile_read()
                mrf.profile_enable(False)
                sec = a.elapsed_time(e) / 1e3
                pr = prm.cpu().numpy()
                gi = idx.cpu().numpy()
                r = {"s_per_slice": sec, "s": s, "energy_kept": float(eig.sum() / d),
                     "basis_s": basis_s, "tree_build_s": tree_s,
                     "matches_per_s_bruteforce_equiv": n * d * args.iters / sec,
                     "T1_acc": t_accuracy(pr[:, 0], ph["T1"], fg),
                     "T2_acc": t_accuracy(pr[:, 1], ph["T2"], fg),
                     "atom_agreement_vs_bf16": float(np.mean(gi == ref_idx)),
                     "stage_ms": {k: v[0] for k, v in prof.items() if v[1]}, **kw}
                if mode == "covertree":
                    ii = torch.empty(n, dtype=torch.int32, device=dev)
                    s2 = mrf.project(Dc, AHYc, ii, opts=o, stats=True)
                    r["first_projection"] = {"evals_per_voxel": s2["n_dist_evals"] / n,
                                             "bruteforce_ratio": d * n / max(s2["n_dist_evals"], 1),
                                             "routed_voxels": s2["n_fallback"]}
                out[f"{mode}_svd{s}" + (f"_eps{kw['eps']}" if kw else "")] = r
            so.close()
            Dc.close()
            del Ac, AHYc, Xc
        del A_dev
    D.close()
    return {"n_voxels": n, "L": L, "d": d, "tree": {"build_s_host": build_s, **info},
            "generate_s": gen_s, "forms": out}


def run_tree(args) -> None:
    import torch
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    b.build()
    r = tree_leg(mrf, torch.device("cuda", 0), torch.cuda.current_stream(), args.iters,
                 args.tree_svd)
    out = r["forms"]
    # the line's value: the tensor-core tree search at eps 0.5 (CoverBLIP's approximate search
    # on the tensor cores); every form, the SIMT cover tree included, is in "forms"
    line = {"metric": "recon s/slice at fixed T1/T2 error (cover tree vs brute force)",
            "value": out["tree_tc_eps0.5"]["s_per_slice"], "unit": "s/slice", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * out["tree_tc_eps0.5"]["s_per_slice"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": TREE_WORKLOAD, "n_voxels": r["n_voxels"], "L": r["L"],
                       "d": r["d"]},
            "tree": r["tree"], "generate_s": r["generate_s"], "forms": out}
    print(json.dumps(line), flush=True)


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import mrf_oracle as mo
    dic, p = make_workload(0)
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"])
    g = np.random.Generator(np.random.PCG64(77))
    sample = Z[g.permutation(Z.shape[0])[:64]]
    atoms = dic["atoms"]
    d = atoms.shape[0]
    for _ in range(args.warmup):
        mo.project(sample[:8], atoms)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mo.project(sample, atoms)
    dt = time.perf_counter() - t0
    value = sample.shape[0] * d * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_voxels": int(Z.shape[0]), "L": int(atoms.shape[1]),
                       "d": int(d), "step": "exhaustive float64 projection of a voxel sample",
                       "projection": "oracle", "sample_voxels": int(sample.shape[0])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle",
                             "sample": f"{sample.shape[0]} voxels x {d} atoms per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    if rank == 0 or world == 1:
        b.build()
    if world > 1:
        dist.barrier()
    mrf.lib()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    dic, p = make_workload(rank)
    atoms, params = dic["atoms"], dic["params"]
    d, L = atoms.shape
    Ny, Nx = p["Ny"], p["Nx"]
    n = Ny * Nx
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    D = mrf.build_dict_index(atoms, params, pack_fp8=True, pack_bf16x3=True)
    D.reserve(n)
    mask = torch.from_numpy(p["masks"]).to(dev)
    op = mrf.make_op(Ny, Nx, L, mask)
    Yd = torch.from_numpy(p["Y"]).to(dev)
    AHY = torch.empty((n, L), dtype=torch.complex64, device=dev)
    mrf.adjoint(op, Yd, AHY)
    del Yd
    X = torch.zeros((n, L), dtype=torch.complex64, device=dev)
    idx = torch.zeros(n, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.complex64, device=dev)
    prm = torch.empty((n, params.shape[1]), dtype=torch.float32, device=dev)
    exact = args.mode == "bf16x3"        # the exact tensor-core form runs certified
    opts = mrf.proj_opts(mode=args.mode, certify=exact)
    tuned = None
    if args.autotune and args.mode in ("bf16", "fp8"):
        from paper_1810_01967_gb300 import autotune
        tuned = autotune.tune(D, AHY, args.mode,
                              grid={"bf16_cluster": (1, 2, 4), "bf16_live_tiles": (16, 32, 64, 128),
                                    "bf16_splits": (0,)}, reps=2)

    def step(Xb, AHYb, idxb, rhob, prmb):
        mrf.ipg_step(D, op, AHYb, Xb, 1.0, idxb, rhob, opts=opts)
        mrf.lut(D, idxb, prmb)

    for _ in range(args.warmup):
        step(X, AHY, idx, rho, prm)
    barrier()
    # ------------------------------------------------------------- timed region (device)
    # No instrumentation inside: the stage profiler runs in a separate pass below.
    clk = ClockSampler(local)
    clk.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(X, AHY, idx, rho, prm)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    ms_max = max_over_ranks(ms, world, dev)
    D.check()
    # ------------------------------------------------------------- stage split (profiled pass)
    # The same K steps again with the library's stage profiler on: CUDA events on the stream
    # every stage is launched on give each stage's time and launch count (the search kernel's
    # average duration for the roofline).
    mrf.profile_enable(True)
    for _ in range(args.steps):
        step(X, AHY, idx, rho, prm)
    barrier()
    prof = mrf.profile_read()
    mrf.profile_enable(False)
    # ------------------------------------------------------------- end to end (host buffers)
    # One call of the public API, mrf_reconstruct, from host k-space to host outputs: the
    # library copies Y in, computes A^H Y, runs K iterations of the timed step's form and the
    # look-up table, and copies X, the atoms, the densities and the parameter maps back, all
    # inside the call (pinned host buffers).
    Yh = torch.from_numpy(p["Y"]).pin_memory()
    Xh = torch.empty((n, L), dtype=torch.complex64).pin_memory()
    idx_h = torch.empty(n, dtype=torch.int32).pin_memory()
    rho_h = torch.empty(n, dtype=torch.complex64).pin_memory()
    prm_h = torch.empty((n, params.shape[1]), dtype=torch.float32).pin_memory()
    e2e_steps = max(1, args.steps)
    ro_warm = mrf.recon_opts(iters=1, mode=args.mode, certify=opts.certify != 0)
    ro = mrf.recon_opts(iters=e2e_steps, mode=args.mode, certify=opts.certify != 0)
    mrf.reconstruct(D, op, Yh, Xh, idx_h, rho_h, prm_h, opts=ro_warm)
    barrier()
    t0 = time.perf_counter()
    mrf.reconstruct(D, op, Yh, Xh, idx_h, rho_h, prm_h, opts=ro)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    h2d = Yh.numel() * 8
    d2h = n * L * 8 + n * 4 + n * 8 + n * params.shape[1] * 4
    del Yh, Xh
    # ------------------------------------------------------------- exact tensor-core leg
    exact_leg = None
    if rank == 0 and not exact and not args.no_exact:
        exact_leg = exact_tc_leg(mrf, D, op, AHY, n, d, L, stream, peaks_sustained(),
                                 steps=min(args.steps, 5))
    # ------------------------------------------------------------- FP32 exact comparator
    fp32_rate = None
    if args.fp32_sample > 0 and rank == 0:
        m = min(args.fp32_sample, n)
        Zs = AHY[:m].contiguous()
        ii = torch.empty(m, dtype=torch.int32, device=dev)
        rr = torch.empty(m, dtype=torch.complex64, device=dev)
        mrf.project(D, Zs, ii, rr, opts=mrf.proj_opts(mode="fp32"))
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        mrf.project(D, Zs, ii, rr, opts=mrf.proj_opts(mode="fp32"))
        f1.record(stream)
        barrier()
        fp32_rate = m * d / (f0.elapsed_time(f1) / 1e3)
    # ------------------------------------------------------------- quality (rank 0)
    quality = None
    D2 = None
    if rank == 0 and not args.no_quality:
        quality, D2 = reconstruction_quality(mrf, D, op, p, dic, dev, stream, args.iters,
                                             fp32=not args.no_fp32, forms=not args.no_forms,
                                             keep=True)
    # ------------------------------------------------------------- batching form (rank 0)
    # the 64-slice workload (its dictionary is this one): BF16 and, with the quality leg's
    # trained network and tree, the learned form and the tensor-core tree search (eps 0.4),
    # each under CUDA-graph replay, groups of 8 slices
    slices = None
    if rank == 0 and not args.no_slices:
        geo, mine, smasks, sYs = slices_inputs(dic, dev)
        forms = [("bf16", True)] + ([("learned", True), ("tree_tc", True)]
                                    if D2 is not None else [])
        Ds = D2 if D2 is not None else D
        sout, _, stuned = slices_leg(mrf, Ds, dic, dev, stream, smasks, sYs, geo, mine, forms,
                                     8, args.iters, 1, True, both=False,
                                     model=True if D2 is not None else None)
        slices = {"workload": SLICES_WORKLOAD, "forms": sout,
                  "autotune": {m: {"tune": t["tune"], "ms": t["ms"]} for m, t in stuned.items()}}
        del smasks, sYs
    if D2 is not None:
        D2.close()
    # ------------------------------------------------------------- cover tree, 1M atoms (rank 0)
    tree = None
    if rank == 0 and not args.no_tree:
        tree = tree_leg(mrf, dev, stream, args.iters)
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    # ------------------------------------------------------------- report
    peaks = measured_peaks()
    value = world * n * d * args.steps / (ms_max / 1e3)
    tc = args.mode in ("bf16", "fp8", "bf16x3")
    search_ms, search_launches = prof["search_tc"] if tc else prof["search_fp32"]
    flops_per_launch = 8.0 * L * n * d
    achieved = flops_per_launch * search_launches / (search_ms / 1e3) / 1e12 if search_ms else 0.0
    if tc:
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        src = peaks["_source"] + " sustained bf16"
        if args.mode == "fp8":
            peak, src = 2.0 * peak, src + " x 2 (nominal fp8 / bf16 dense ratio, 4.5 / 2.25)"
        if args.mode == "bf16x3":
            peak, src = peak / 3.0, src + " / 3 (three BF16 products per voxel-atom pair)"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_per_launch(n, d, args.mode),
                "kernel": "k_tc_topk", "peak_source": src, "flops_per_launch": flops_per_launch}
    else:
        # FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 flop (FFMA) x 2070 MHz maximum SM clock
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_fp32_topk",
                "peak_source": "152 SMs x 128 lanes x 2 flop x 2.07 GHz"}
    launches = int(sum(v[1] for v in prof.values()))
    cpu = cpu1 = None
    if not args.no_cpu and world == 1:
        # the CPU baseline leg: the float64 oracle timed on the host cores on a bounded sample
        # of the slice's voxels (its answers on that sample also give the GPU form's agreement
        # with it), on one thread, and on the small workload's whole reconstruction
        from oracle import mrf_oracle as mo
        Zh = mo.adjoint(p["Y"], p["masks"], Ny, Nx)
        g = np.random.Generator(np.random.PCG64(77))
        sample = Zh[g.permutation(n)[:4096]]

        def gpu_idx(Zs):
            Zd = torch.from_numpy(np.ascontiguousarray(Zs, dtype=np.complex64)).to(dev)
            ii = torch.empty(Zd.shape[0], dtype=torch.int32, device=dev)
            mrf.project(D, Zd, ii, opts=opts)
            torch.cuda.synchronize()
            return ii.cpu().numpy()
        cpu = oracle_baseline(sample, atoms, gpu_idx=gpu_idx)
        cpu1 = oracle_baseline_1thread(sample[:256], atoms)
        cpu["small_workload_full"] = small_workload_full(mrf, dev)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "fp8": "fp8_e4m3", "fp32": "f32",
                      "bf16x3": "bf16x3 (split bf16, f32 accumulate)"}[args.mode],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_voxels": n, "L": L, "d": d,
                       "step": "one BLIP iteration (ipg_step) + look-up table",
                       "projection": args.mode,
                       "topk": {"fp32": 8, "bf16": 16, "fp8": 32, "bf16x3": 32}[args.mode],
                       "certify": exact,
                       "l2": "inputs larger than L2 (BF16 dictionary operand 800 MB)"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * n * d * e2e_steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                    "call": f"mrf_reconstruct from pinned host buffers, {e2e_steps} iterations "
                            f"per call (Y in, X / atoms / densities / parameter maps out)",
                    "h2d_bytes_per_call": h2d, "d2h_bytes_per_call": d2h,
                    "s_per_call": e2e_s},
            "gpu_launches": launches, "clocks": clocks,
            "extra": {"recon_s_per_slice_20_iters": 20 * ms_max / args.steps / 1e3,
                      "quality": quality,
                      "stage_ms": {k: v[0] for k, v in prof.items()},
                      "stage_launches": {k: v[1] for k, v in prof.items()},
                      "cpu_baseline_1thread": cpu1,
                      "autotune": tuned,
                      "fp32_exact_matches_per_s": fp32_rate,
                      "exact_tc": exact_leg,
                      "slices64": slices,
                      "tree1m_eps_sweep": tree,
                      "fp32_sample_voxels": args.fp32_sample}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the 25 s FP32 reconstruction")
    ap.add_argument("--no-forms", action="store_true", help="skip the cover tree and learned forms")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="bf16",
                    choices=["bf16", "fp8", "fp32", "bf16x3", "covertree", "tree_tc", "gradient",
                             "mlp", "learned"],
                    help="projection of the timed step (covertree, tree_tc, gradient, mlp, "
                         "learned: --profile-case only)")
    ap.add_argument("--autotune", action="store_true",
                    help="time the search geometries on the workload first and use the fastest "
                         "(always on for the slices64 workload, whose batching form picks its "
                         "geometry with the autotuner)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="slices64: keep the library's default search geometry")
    ap.add_argument("--fp32-sample", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-slices", action="store_true",
                    help="skip the 64-slice batching leg of the default run")
    ap.add_argument("--no-tree", action="store_true",
                    help="skip the million-atom cover-tree leg of the default run")
    ap.add_argument("--no-exact", action="store_true",
                    help="skip the exact tensor-core (split-BF16) leg of the default run")
    ap.add_argument("--workload", default="slice", choices=["slice", "slices64", "tree1m"],
                    help="slice: the BLIP-iteration bench; slices64: the batching form; "
                         "tree1m: the cover tree on the million-atom dictionary")
    ap.add_argument("--group", type=int, default=8, help="slices per group (slices64)")
    ap.add_argument("--tree-svd", type=int, nargs="*", default=[20, 100],
                    help="compressed dimensions s for the tree1m workload's compressed forms")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="projection-only small case with N voxels (for ncu captures)")
    args = ap.parse_args()
    if args.mode in ("covertree", "tree_tc", "gradient", "mlp", "learned") and args.profile_case <= 0:
        ap.error(f"--mode {args.mode} needs --profile-case")
    if args.profile_case > 0:
        run_profile_case(args)
    elif args.workload == "slices64" and args.impl == "ours":
        run_slices(args)
    elif args.workload == "tree1m" and args.impl == "ours":
        run_tree(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
