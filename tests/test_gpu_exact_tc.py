"""GPU parity of the exact tensor-core projection (MRF_PROJ_BF16X3: split-BF16 operands, three
products per pair in one FP32 accumulation, per-voxel certification, FP32 re-search of the
uncertified voxels) against the float64 oracle through the C ABI (§3.2, eqs. exactP /
exactPs): aliased fingerprints of the small workload, atoms times scalars with zero rows, odd
frame counts, one atom, one voxel, ragged tiles, both cones; and the error bound itself -- the
kernel's raw candidate scores (mrf_search_candidates) against float64 correlations, on the
small workload and on an adversarial case whose products are all positive (monotone partial
sums, where rounding errors of the accumulation cannot cancel)."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mrf():
    import paper_1810_01967_gb300 as m
    from paper_1810_01967_gb300 import build as b
    b.build()
    return m


@pytest.fixture(scope="module")
def cfg1():
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"])
    return dic, p, Z.astype(np.complex64)


def run(mrf, D, Z, cone="complex", certify=True, X=True):
    n = Z.shape[0]
    Zd = to_dev(Z)
    idx = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Xo = torch.empty_like(Zd) if X else None
    st = mrf.project(D, Zd, idx, rho, Xo,
                     opts=mrf.proj_opts(mode="bf16x3", cone=cone, certify=certify), stats=True)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), rho.cpu().numpy(), None if Xo is None else Xo.cpu().numpy(), st


def candidates(mrf, D, Z, mode="bf16x3", cone="complex"):
    n = Z.shape[0]
    K = 32 if mode in ("bf16x3", "fp8") else 16
    Zd = to_dev(Z)
    sc = torch.empty((n, K), dtype=torch.float32, device="cuda")
    ix = torch.empty((n, K), dtype=torch.int32, device="cuda")
    bd = torch.empty(n, dtype=torch.float32, device="cuda")
    mrf.search_candidates(D, Zd, sc, ix, bd, opts=mrf.proj_opts(mode=mode, cone=cone))
    torch.cuda.synchronize()
    return sc.cpu().numpy(), ix.cpu().numpy(), bd.cpu().numpy()


def check_bound(Z, A, sc, ix, bd, cone):
    """Every kept candidate's kernel correlation lies within the voxel's bound (times ||z||) of
    its float64 value; returns the largest observed error relative to the bound."""
    Z = np.asarray(Z, np.complex128)
    A = np.asarray(A, np.complex128)
    zn = np.linalg.norm(Z, axis=1)
    worst = 0.0
    for k in range(ix.shape[1]):
        j = ix[:, k]
        ok = j >= 0
        if not ok.any():
            continue
        c = np.sum(np.conj(A[j[ok]]) * Z[ok], axis=1) / np.linalg.norm(A[j[ok]], axis=1)
        if cone == "complex":
            got, ref = np.sqrt(np.maximum(sc[ok, k], 0.0)), np.abs(c)
        else:
            got, ref = sc[ok, k], c.real
        err = np.abs(got - ref)
        lim = bd[ok] * zn[ok]
        assert np.all(err <= lim), (f"kernel error {err.max():.3e} beyond its bound "
                                    f"{lim[np.argmax(err - lim)]:.3e}")
        worst = max(worst, float(np.max(err / np.maximum(lim, 1e-300))))
    return worst


@pytest.mark.parametrize("n", [1024, 1000, 1])
@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_aliased_fingerprints(mrf, cfg1, n, cone):
    dic, p, Z = cfg1
    D = mrf.build_dict_index(dic["atoms"], dic["params"], pack_bf16x3=True)
    Zs = Z[:n]
    idx, rho, X, st = run(mrf, D, Zs, cone=cone)
    agree, ties = check_projection(Zs, dic["atoms"], idx, rho, cone=cone, g_X=X)
    assert st["device_error"] == 0
    print(f"bf16x3 {cone} n={n}: agreement {agree:.5f}, near-tie swaps {ties}, "
          f"uncertified {st['n_uncertified']}")


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_atoms_times_scalars_and_zero_rows(mrf, cfg1, cone):
    A = cfg1[0]["atoms"]
    g = np.random.Generator(np.random.PCG64(301))
    n = 517
    js = g.integers(0, A.shape[0], n)
    rho = g.uniform(0.3, 2.0, n) * (np.exp(1j * g.uniform(0, 2 * np.pi, n))
                                    if cone == "complex" else 1.0)
    Z = (rho[:, None] * A[js].astype(np.complex128)).astype(np.complex64)
    Z[::37] = 0
    D = mrf.build_dict_index(A, pack_bf16x3=True)
    idx, r, X, st = run(mrf, D, Z, cone=cone)
    check_projection(Z, A, idx, r, cone=cone, g_X=X)
    zero = np.zeros(n, bool)
    zero[::37] = True
    assert np.all(idx[zero] == 0) and np.all(r[zero] == 0)
    assert st["n_zero"] == zero.sum()


@pytest.mark.parametrize("L,d,n", [(37, 5, 70), (100, 1, 3), (8, 300, 129), (1000, 257, 300)])
def test_odd_sizes(mrf, L, d, n):
    g = np.random.Generator(np.random.PCG64(302 + L))
    A = (g.standard_normal((d, L)) + 1j * g.standard_normal((d, L))).astype(np.complex64)
    A *= g.uniform(0.2, 3.0, (d, 1)).astype(np.float32)
    Z = (g.standard_normal((n, L)) + 1j * g.standard_normal((n, L))).astype(np.complex64)
    D = mrf.build_dict_index(A, pack_bf16x3=True)
    for cone in ("complex", "real_pos"):
        idx, r, X, st = run(mrf, D, Z, cone=cone)
        check_projection(Z, A, idx, r, cone=cone, g_X=X)


def test_empty_input_and_missing_operand(mrf, cfg1):
    A = cfg1[0]["atoms"]
    D = mrf.build_dict_index(A, pack_bf16x3=True)
    run(mrf, D, np.zeros((0, A.shape[1]), np.complex64))
    D2 = mrf.build_dict_index(A)                       # no split operand packed
    with pytest.raises(mrf.MRFError, match="split-BF16"):
        run(mrf, D2, cfg1[2][:4])


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_kernel_scores_within_their_bound(mrf, cfg1, cone):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, pack_bf16x3=True)
    sc, ix, bd = candidates(mrf, D, Z, "bf16x3", cone)
    assert np.all(bd > 0) and np.all(bd < 1e-3)
    worst = check_bound(Z, A, sc, ix, bd, cone)
    # the plain BF16 kernel against its own (much wider) rigorous bound
    sc1, ix1, bd1 = candidates(mrf, D, Z, "bf16", cone)
    worst1 = check_bound(Z, A, sc1, ix1, bd1, cone)
    print(f"{cone}: split-BF16 bound {np.median(bd):.2e} (median), largest error / bound "
          f"{worst:.3f}; BF16 bound {bd1[0]:.2e}, largest error / bound {worst1:.3f}")


def test_kernel_scores_within_their_bound_monotone_sums(mrf):
    """All products positive: atoms with 256 entries 1/32 (unit atoms 1/16, exact in BF16, so
    the operand terms vanish) against queries with positive real and imaginary parts, L = 1024;
    every partial sum of the accumulation grows, the case where per-instruction roundings add
    up instead of cancelling."""
    g = np.random.Generator(np.random.PCG64(303))
    L, d, n = 1024, 300, 256
    A = np.zeros((d, L), np.complex64)
    for j in range(d):
        A[j, g.choice(L, 256, replace=False)] = 1.0 / 32.0
    Z = (g.uniform(0.5, 1.5, (n, L)) + 1j * g.uniform(0.5, 1.5, (n, L))).astype(np.complex64)
    Z *= g.uniform(0.1, 10.0, (n, 1)).astype(np.float32)
    D = mrf.build_dict_index(A, pack_bf16x3=True)
    sc, ix, bd = candidates(mrf, D, Z, "bf16x3", "complex")
    worst = check_bound(Z, A, sc, ix, bd, "complex")
    print(f"monotone sums: bound {np.median(bd):.2e}, largest error / bound {worst:.3f}")
    idx, r, X, st = run(mrf, D, Z)
    check_projection(Z, A, idx, r, g_X=X)
