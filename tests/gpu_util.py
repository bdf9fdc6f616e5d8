"""Shared helpers of the GPU parity tests: device copies and the oracle comparison rules.

Comparison rules (tolerances of the parity bar):
  * atom index: identical to the oracle's, except where the oracle scores the GPU's atom within
    TIE_REL = 1e-6 (relative, normalised correlation) of its own best -- a near-tie, where either
    index is accepted;
  * density rho and image X: within RHO_REL = 1e-4 relative error of the oracle's values for the
    accepted atom (float64 evaluation of the same formula).
"""
import numpy as np

from oracle import mrf_oracle as mo

TIE_REL = 1e-6
RHO_REL = 1e-4


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def check_projection(Z, D, g_idx, g_rho, cone="complex", g_X=None, tie=TIE_REL, rho_rel=RHO_REL,
                     ref=None):
    """Assert the parity rules; returns (exact agreement rate, number of near-tie mismatches)."""
    Z = np.asarray(Z, np.complex128)
    ref = ref if ref is not None else mo.project(Z, D, cone)
    g_idx = np.asarray(g_idx, np.int64)
    assert g_idx.min() >= 0 and g_idx.max() < D.shape[0]
    s_g = mo.correlation(Z, D, g_idx, cone)
    s1 = ref["s1"]
    zero = np.sum(np.abs(Z) ** 2, axis=1) == 0
    mism = (g_idx != ref["idx"]) & ~zero
    near = s_g >= s1 - tie * np.abs(s1)
    bad = np.flatnonzero(mism & ~near)
    assert bad.size == 0, (f"{bad.size} atom mismatches beyond the near-tie rule, e.g. v={bad[:5]}"
                           f" gpu={g_idx[bad[:5]]} ref={ref['idx'][bad[:5]]}"
                           f" s_gpu={s_g[bad[:5]]} s_ref={s1[bad[:5]]}")
    assert np.all(g_idx[zero] == 0)
    rho_ref = mo.density(Z, D, g_idx, cone)
    rho_ref[zero] = 0
    err = np.abs(np.asarray(g_rho, np.complex128) - rho_ref)
    scale = np.maximum(np.abs(rho_ref), 1e-30)
    worst = np.max(np.where(zero, err, err / scale)) if err.size else 0.0
    assert worst <= rho_rel, f"rho relative error {worst:.3e}"
    if g_X is not None:
        Xr = rho_ref[:, None] * np.asarray(D, np.complex128)[g_idx]
        num = np.linalg.norm(np.asarray(g_X, np.complex128) - Xr, axis=1)
        den = np.maximum(np.linalg.norm(Xr, axis=1), 1e-30)
        wx = np.max(np.where(zero, num, num / den))
        assert wx <= rho_rel, f"X relative error {wx:.3e}"
    return float(np.mean(~mism)), int(np.sum(mism))


def bf16_bound(L):
    """Rigorous bound of the BF16 kernel's correlation error (normalised correlation): operand
    rounding 2u + u^2 with u = 2^-8, plus FP32 accumulation of 2L products."""
    return 2.0 ** -7 + 2.0 ** -16 + 2 * L * 2.0 ** -24


def check_bound_rule(Z, D, g_idx, g_rho, bound, cone="complex", g_X=None, rho_rel=RHO_REL,
                     ref=None):
    """Uncertified tensor-core forms: the answer is the exact best of the candidates the kernel
    kept, so its normalised correlation lies within twice the kernel's error bound of the
    oracle's best, and rho / X are the exact density of the returned atom.  Returns the exact
    agreement rate (a report, not a bar)."""
    Z = np.asarray(Z, np.complex128)
    ref = ref if ref is not None else mo.project(Z, D, cone)
    g_idx = np.asarray(g_idx, np.int64)
    assert g_idx.min() >= 0 and g_idx.max() < D.shape[0]
    zero = np.sum(np.abs(Z) ** 2, axis=1) == 0
    s_g = mo.correlation(Z, D, g_idx, cone)
    bad = np.flatnonzero(~zero & (s_g < ref["s1"] - 2.0 * bound))
    assert bad.size == 0, f"{bad.size} answers beyond twice the kernel bound, e.g. v={bad[:5]}"
    assert np.all(g_idx[zero] == 0)
    rho_ref = mo.density(Z, D, g_idx, cone)
    rho_ref[zero] = 0
    err = np.abs(np.asarray(g_rho, np.complex128) - rho_ref)
    scale = np.maximum(np.abs(rho_ref), 1e-30)
    worst = np.max(np.where(zero, err, err / scale)) if err.size else 0.0
    assert worst <= rho_rel, f"rho relative error {worst:.3e}"
    if g_X is not None:
        Xr = rho_ref[:, None] * np.asarray(D, np.complex128)[g_idx]
        num = np.linalg.norm(np.asarray(g_X, np.complex128) - Xr, axis=1)
        den = np.maximum(np.linalg.norm(Xr, axis=1), 1e-30)
        assert np.max(np.where(zero, num, num / den)) <= rho_rel
    return float(np.mean((g_idx == ref["idx"]) | zero))


def iterate_checked(mrf, D, op, AHY, atoms, iters, opts, cone="complex", rule="exact",
                    bound=None, sample=None, mu=1.0, X=None, idx=None, check=None):
    """BLIP iterations through the C ABI, one gradient step (mrf_gradient) and one projection
    (mrf_project, warm-started at the previous atoms) at a time -- the two halves of
    mrf_ipg_step.  After every projection the oracle projects the GPU's own Z (the voxels of
    `sample`, all when None) and the answers are compared by `rule`: "exact" (check_projection)
    or "bound" (check_bound_rule with `bound`); `check(Z, idx, rho, X)` replaces both when
    given.  Returns the device X, idx, rho and the per-iteration exact agreement rates."""
    import torch
    n, L = AHY.shape
    X = torch.zeros((n, L), dtype=torch.complex64, device="cuda") if X is None else X
    idx = torch.zeros(n, dtype=torch.int32, device="cuda") if idx is None else idx
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Z = torch.empty_like(X)
    rates = []
    for _ in range(iters):
        mrf.gradient(D, op, AHY, X, mu, Z)
        mrf.project(D, Z, idx, rho, X, warm_idx=idx, opts=opts)
        torch.cuda.synchronize()
        ti = None if sample is None else torch.as_tensor(sample, device="cuda")
        Zs = (Z if ti is None else Z[ti]).cpu().numpy()
        gi = (idx if ti is None else idx[ti]).cpu().numpy()
        gr = (rho if ti is None else rho[ti]).cpu().numpy()
        gx = (X if ti is None else X[ti]).cpu().numpy()
        if check is not None:
            rates.append(check(Zs, gi, gr, gx))
        elif rule == "exact":
            rates.append(check_projection(Zs, atoms, gi, gr, cone=cone, g_X=gx)[0])
        else:
            rates.append(check_bound_rule(Zs, atoms, gi, gr, bound, cone=cone, g_X=gx))
    return X, idx, rho, rates
