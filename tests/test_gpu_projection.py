"""GPU parity of the matched-filtering projection (mrf_project) against the FP64 oracle, through
the C ABI, for the FP32 SIMT kernel and the BF16 and FP8 tcgen05 kernels: realistic aliased fingerprints,
several tiles plus ragged tails, edge cases (zero rows, single voxel, tiny dictionaries, odd L,
duplicate atoms) and both cone readings."""
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


def run(mrf, D, Z, mode, cone="complex", X=True, topk=0, certify=True):
    n = Z.shape[0]
    Zd = to_dev(Z)
    idx = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Xo = torch.empty_like(Zd) if X else None
    st = mrf.project(D, Zd, idx, rho, Xo,
                     opts=mrf.proj_opts(mode=mode, cone=cone, topk=topk, certify=certify),
                     stats=True)
    torch.cuda.synchronize()
    return (idx.cpu().numpy(), rho.cpu().numpy(), None if Xo is None else Xo.cpu().numpy(), st)


@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("n", [1000, 1024, 1])
def test_aliased_fingerprints(mrf, cfg1, mode, n):
    dic, p, Z = cfg1
    D = mrf.build_dict_index(dic["atoms"], dic["params"], pack_fp8=(mode == "fp8"))
    Zs = Z[:n]
    idx, rho, X, st = run(mrf, D, Zs, mode)
    agree, ties = check_projection(Zs, dic["atoms"], idx, rho, g_X=X)
    assert st["device_error"] == 0
    print(f"{mode} n={n}: agreement {agree:.5f}, near-tie swaps {ties}, stats {st}")


@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_atoms_times_scalars_and_zero_rows(mrf, cfg1, mode, cone):
    dic = cfg1[0]
    A = dic["atoms"]
    g = np.random.Generator(np.random.PCG64(101))
    n = 517
    js = g.integers(0, A.shape[0], n)
    rho = g.uniform(0.3, 2.0, n) * (np.exp(1j * g.uniform(0, 2 * np.pi, n))
                                    if cone == "complex" else 1.0)
    Z = (rho[:, None] * A[js].astype(np.complex128)).astype(np.complex64)
    Z[::37] = 0
    D = mrf.build_dict_index(A, dic["params"], pack_fp8=(mode == "fp8"))
    idx, r, X, st = run(mrf, D, Z, mode, cone=cone)
    check_projection(Z, A, idx, r, cone=cone, g_X=X)
    zero = np.zeros(n, bool)
    zero[::37] = True
    assert np.all(idx[zero] == 0) and np.all(r[zero] == 0)
    assert st["n_zero"] == zero.sum()


@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("L,d,n", [(37, 5, 70), (100, 1, 3), (8, 300, 129), (1000, 257, 300)])
def test_odd_shapes(mrf, mode, L, d, n):
    g = np.random.Generator(np.random.PCG64(L * 1000 + d))
    A = (g.standard_normal((d, L)) + 1j * g.standard_normal((d, L))).astype(np.complex64)
    A *= g.uniform(0.5, 2.0, (d, 1)).astype(np.float32)
    Z = (g.standard_normal((n, L)) + 1j * g.standard_normal((n, L))).astype(np.complex64)
    D = mrf.build_dict_index(A, pack_fp8=(mode == "fp8"))
    idx, r, X, _ = run(mrf, D, Z, mode)
    check_projection(Z, A, idx, r, g_X=X)


@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp8"])
def test_duplicate_atoms_tie_to_smallest_index(mrf, mode):
    g = np.random.Generator(np.random.PCG64(7))
    B = (g.standard_normal((40, 64)) + 1j * g.standard_normal((40, 64))).astype(np.complex64)
    A = np.concatenate([B, B, B[:10]])
    js = g.integers(0, 40, 200)
    Z = (A[js] * np.complex64(1.5 - 0.5j)).astype(np.complex64)
    D = mrf.build_dict_index(A, pack_fp8=(mode == "fp8"))
    idx, r, X, _ = run(mrf, D, Z, mode)
    assert np.array_equal(idx, js)
    np.testing.assert_allclose(r, 1.5 - 0.5j, rtol=1e-5)


@pytest.mark.parametrize("topk", [4, 8, 16])
def test_topk_and_uncertified_bf16(mrf, cfg1, topk):
    """Without certification the BF16 form is top-K + exact rescore: report its agreement and
    check that every miss is within the rigorous BF16 correlation error bound of the best."""
    dic, p, Z = cfg1
    D = mrf.build_dict_index(dic["atoms"])
    idx, r, X, st = run(mrf, D, Z, "bf16", topk=topk, certify=False)
    ref = mo.project(Z, dic["atoms"])
    agree = float(np.mean(idx == ref["idx"]))
    sg = mo.correlation(Z, dic["atoms"], idx)
    bound = 2.0 ** -7 + 2.0 ** -16 + 2 * Z.shape[1] * 2.0 ** -24   # BF16: u = 2^-8
    assert np.all(sg >= ref["s1"] - 2 * bound)
    assert agree > {4: 0.9, 8: 0.97, 16: 0.98}[topk], agree
    print(f"bf16 top-{topk} uncertified agreement {agree:.5f}")
    idx, r, X, st = run(mrf, D, Z, "fp32", topk=topk)
    check_projection(Z, dic["atoms"], idx, r, g_X=X)


@pytest.mark.parametrize("cone,K", [("complex", 16), ("real_pos", 16), ("complex", 32)])
def test_fp8_search_matches_e4m3_emulation(mrf, cfg1, cone, K):
    """The FP8 kernel ranks by the correlations of the E4M3-quantised operands (rows scaled by
    powers of two).  Uncertified, the answer is the exactly best atom among the 16 best by that
    ranking: compare with a float64 evaluation of the quantised products (fp8_emul), allowing
    for near-ties at the 16th place within the FP32 accumulation error, and check the rigorous
    bound on every miss."""
    from fp8_emul import fp8_scores
    dic, p, Z = cfg1
    A = dic["atoms"]
    Zs = Z[:600]
    D = mrf.build_dict_index(A, pack_fp8=True)
    idx, r, X, st = run(mrf, D, Zs, "fp8", cone=cone, topk=K, certify=False)
    S8 = fp8_scores(Zs, A, cone)
    Zc, Ac = Zs.astype(np.complex128), A.astype(np.complex128)
    C = Zc @ Ac.conj().T
    den = np.linalg.norm(Zc, axis=1)[:, None] * np.linalg.norm(Ac, axis=1)[None, :]
    ex = (np.abs(C) if cone == "complex" else C.real) / np.maximum(den, 1e-300)
    srt = -np.sort(-S8, axis=1)
    kth = srt[:, K - 1]
    tol = 1e-4 * np.maximum(np.abs(srt[:, 0]), 1e-30)    # FP32 accumulation, generous
    sure = S8 >= (kth + tol)[:, None]                     # in the top K for any rounding
    maybe = S8 >= (kth - tol)[:, None]                    # possibly in the top K
    lo = np.max(np.where(sure, ex, -np.inf), axis=1)
    hi = np.max(np.where(maybe, ex, -np.inf), axis=1)
    got = ex[np.arange(len(idx)), idx]
    ok = (got >= lo - 1e-6) & (got <= hi + 1e-6) & maybe[np.arange(len(idx)), idx]
    assert np.all(ok), np.flatnonzero(~ok)[:10]
    ref = mo.project(Zs, A, cone)
    agree = float(np.mean(idx == ref["idx"]))
    print(f"fp8 uncertified ({cone}, top-{K}) agreement with the exact projection {agree:.4f}")
    rr = mo.density(Zs, A, idx, cone)
    assert np.max(np.abs(r - rr) / np.maximum(np.abs(rr), 1e-30)) <= 1e-4


@pytest.mark.parametrize("mode,K", [("bf16", 16), ("fp8", 32)])
@pytest.mark.parametrize("S", [1, 3, 8, 32, 64])
def test_atom_splits_and_merge_lane_lists(mrf, cfg1, mode, K, S):
    """The search split into S atom ranges (more splits than the 16 atom blocks leave empty
    ranges) and the merge's lane lists sized for S x K candidates per voxel (4 up to 32 per
    lane): the same projection for every split."""
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, pack_fp8=(mode == "fp8"))
    D.set_tune(bf16_splits=S)
    Zs = Z[:777]
    L = A.shape[1]
    # uncertified: the exact best of the kept candidates, within twice the kernel's bound
    idx, rho, X, st = run(mrf, D, Zs, mode, topk=K, certify=False)
    assert D.get_tune()["last_bf16_splits"] == S
    assert st["device_error"] == 0
    if mode == "bf16":
        bound = 2.0 ** -7 + 2.0 ** -16 + 2 * L * 2.0 ** -24
    else:
        u8 = 2.0 ** -4 + np.sqrt(2 * L) * 2.0 ** -10 / 224
        bound = 2 * u8 + u8 * u8 + 2 * L * 2.0 ** -13
    ref = mo.project(Zs, A)
    sg = mo.correlation(Zs, A, idx)
    assert np.all(sg >= ref["s1"] - 2 * bound)
    assert np.mean(idx == ref["idx"]) >= (0.97 if mode == "bf16" else 0.6)
    rr = mo.density(Zs, A, idx)
    assert np.max(np.abs(rho - rr) / np.maximum(np.abs(rr), 1e-30)) <= 1e-4
    # certified: the exact projection
    idx, rho, X, st = run(mrf, D, Zs, mode, topk=K, certify=True)
    check_projection(Zs, A, idx, rho, g_X=X, ref=ref)


def test_empty_projection_is_a_no_op(mrf, cfg1):
    dic = cfg1[0]
    D = mrf.build_dict_index(dic["atoms"])
    Z = torch.empty((0, dic["atoms"].shape[1]), dtype=torch.complex64, device="cuda")
    idx = torch.empty(0, dtype=torch.int32, device="cuda")
    mrf.project(D, Z, idx)


def test_bad_arguments_raise(mrf, cfg1):
    dic = cfg1[0]
    D = mrf.build_dict_index(dic["atoms"], pack_bf16=False)
    Z = to_dev(np.zeros((4, dic["atoms"].shape[1]), np.complex64))
    idx = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(mrf.MRFError):
        mrf.project(D, Z, idx, opts=mrf.proj_opts(mode="bf16"))
    with pytest.raises(mrf.MRFError):
        mrf.project(D, Z, idx, opts=mrf.proj_opts(topk=40))
    bad = dic["atoms"][:3].copy()
    bad[1] = 0
    with pytest.raises(mrf.MRFError):
        mrf.build_dict_index(bad)
