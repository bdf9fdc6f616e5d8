"""GPU parity of the query-batched tensor-core tree search (MRF_PROJ_TREE_TC) against the
float64 oracle through the C ABI: the block balls enclose their atoms (oracle distances, §4.1);
eps = 0 with certification is the exact projection of §3.2 (eqs. exactP / exactPs) for both
cones, ragged sizes, zero rows, duplicates and a one-atom dictionary; eps > 0 meets the (1+eps)
bound of Definition eNN; the uncertified BF16 form meets the BF16 error-bound rule; and every
iteration of a reconstruction projects the GPU's own Z as the oracle does (Algorithm 2)."""
import numpy as np
import pytest

import mrfgen
from oracle import covertree as ct
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection, check_bound_rule, bf16_bound, iterate_checked

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
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]).astype(np.complex64)
    return dic, p, Z


@pytest.fixture(scope="module")
def dicts(mrf, cfg1):
    A = cfg1[0]["atoms"]
    return {cone: mrf.build_dict_index(A, cfg1[0]["params"], build_tree=True, tree_cone=cone,
                                       tree_tc=True, pack_bf16x3=True)
            for cone in ("complex", "real_pos")}


def run(mrf, D, Z, eps, cone="complex", certify=True):
    n = Z.shape[0]
    idx = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Xo = torch.empty((n, Z.shape[1]), dtype=torch.complex64, device="cuda")
    st = mrf.project(D, to_dev(Z), idx, rho, Xo, stats=True,
                     opts=mrf.proj_opts(mode="tree_tc", eps=eps, cone=cone, certify=certify))
    torch.cuda.synchronize()
    assert st["device_error"] == 0
    return idx.cpu().numpy(), rho.cpu().numpy(), Xo.cpu().numpy(), st


def unit_dist(Z, A, idx, cone="complex"):
    """Oracle distance between z/||z|| and the unit atom idx (phase-quotient or Euclidean)."""
    metric = "phase" if cone == "complex" else "euclid"
    U = ct.unit_atoms(np.asarray(A, np.complex128))
    Zn = Z.astype(np.complex128) / np.linalg.norm(Z, axis=1)[:, None]
    return np.array([ct.pair_dist(Zn[v:v + 1], U[idx[v]:idx[v] + 1], metric)[0, 0]
                     for v in range(Z.shape[0])])


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_blocks_enclose_their_atoms(mrf, cfg1, dicts, cone):
    A = cfg1[0]["atoms"]
    d = A.shape[0]
    B = dicts[cone].tree_blocks()
    nb, perm, rad = B["nblk"], B["perm"], B["radius"]
    assert nb == (d + 127) // 128 and perm.shape == (nb * 128,)
    assert np.array_equal(np.sort(perm[:d]), np.arange(d)) and np.all(perm[d:] == -1)
    U = ct.unit_atoms(A.astype(np.complex128))
    metric = "phase" if cone == "complex" else "euclid"
    slack = []
    for b in range(nb):
        js = perm[b * 128:(b + 1) * 128]
        js = js[js >= 0]
        dist = ct.pair_dist(U[js[:1]], U[js], metric)[0]
        assert rad[b] >= dist.max(), (b, rad[b], dist.max())
        slack.append(rad[b] - dist.max())
    assert max(slack) < 1e-5
    # depth-first blocks are tighter than blocks of the atoms in index order
    idx_rad = [ct.pair_dist(U[b * 128:b * 128 + 1], U[b * 128:(b + 1) * 128], metric)[0].max()
               for b in range(nb)]
    print(f"{cone}: median block radius {np.median(rad):.3f} (index order "
          f"{np.median(idx_rad):.3f})")


@pytest.mark.parametrize("n", [1024, 1000, 1])
@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_eps0_is_the_exact_projection(mrf, cfg1, dicts, n, cone):
    dic, p, Z = cfg1
    Zs = Z[:n]
    idx, rho, X, st = run(mrf, dicts[cone], Zs, 0.0, cone=cone)
    agree, ties = check_projection(Zs, dic["atoms"], idx, rho, cone=cone, g_X=X)
    nb = (dic["atoms"].shape[0] + 127) // 128
    tiles = (n + 127) // 128
    assert 0 < st["n_dist_evals"] <= tiles * 128 * nb * 128
    print(f"{cone} n={n}: agreement {agree:.5f}, ties {ties}, uncertified "
          f"{st['n_uncertified']}, pairs {st['n_dist_evals']} of "
          f"{n * dic['atoms'].shape[0]} brute force")


@pytest.mark.parametrize("eps", [0.2, 0.5, 1.0])
def test_eps_bound(mrf, cfg1, dicts, eps):
    dic, p, Z = cfg1
    A = dic["atoms"]
    ref = mo.project(Z, A)
    idx, rho, X, st = run(mrf, dicts["complex"], Z, eps)
    dg = unit_dist(Z, A, idx)
    dn = unit_dist(Z, A, ref["idx"])
    assert np.all(dg <= (1 + eps) * dn + 1e-6), np.max(dg - (1 + eps) * dn)
    rr = mo.density(Z, A, idx)
    assert np.max(np.abs(rho - rr) / np.abs(rr)) <= 1e-4
    print(f"eps={eps}: exact agreement {np.mean(idx == ref['idx']):.4f}, pairs "
          f"{st['n_dist_evals']} ({st['n_dist_evals'] / (Z.shape[0] * A.shape[0]):.3f} of "
          f"brute force)")


def test_bf16_form_meets_the_bound_rule(mrf, cfg1, dicts):
    """Without certification the depth-first BF16 operand ranks the candidates: at eps = 0 the
    searched blocks hold the nearest atom, so the answer is within twice the BF16 bound."""
    dic, p, Z = cfg1
    idx, rho, X, st = run(mrf, dicts["complex"], Z, 0.0, certify=False)
    rate = check_bound_rule(Z, dic["atoms"], idx, rho, bf16_bound(dic["atoms"].shape[1]),
                            g_X=X)
    assert st["n_uncertified"] == 0
    print(f"BF16 tree form: exact agreement {rate:.4f}")


@pytest.mark.parametrize("L,d,n", [(37, 300, 129), (100, 1, 5), (64, 1000, 300)])
def test_odd_sizes_zero_rows_duplicates(mrf, L, d, n):
    g = np.random.Generator(np.random.PCG64(500 + L + d))
    A = (g.standard_normal((d, L)) + 1j * g.standard_normal((d, L))).astype(np.complex64)
    if d > 10:
        A[d // 2:d // 2 + 5] = A[:5] * np.complex64(np.exp(0.7j))     # duplicates (phase)
    A *= g.uniform(0.3, 3.0, (d, 1)).astype(np.float32)
    js = g.integers(0, d, n)
    Z = (A[js] * (g.uniform(0.5, 2, n) * np.exp(1j * g.uniform(0, 6.3, n)))[:, None])
    Z = (Z + 0.3 * (g.standard_normal((n, L)) + 1j * g.standard_normal((n, L)))
         * np.linalg.norm(A[js], axis=1)[:, None] / np.sqrt(L)).astype(np.complex64)
    Z[::17] = 0
    D = mrf.build_dict_index(A, build_tree=True, tree_tc=True, pack_bf16x3=True)
    idx, rho, X, st = run(mrf, D, Z, 0.0)
    check_projection(Z, A, idx, rho, g_X=X)
    assert st["n_zero"] == len(range(0, n, 17))


def test_empty_input_and_missing_index(mrf, cfg1):
    A = cfg1[0]["atoms"]
    D = mrf.build_dict_index(A, build_tree=True, tree_tc=True)
    run(mrf, D, np.zeros((0, A.shape[1]), np.complex64), 0.0)
    D2 = mrf.build_dict_index(A, build_tree=True)
    with pytest.raises(mrf.MRFError, match="tree_tc"):
        run(mrf, D2, cfg1[2][:4], 0.0)
    with pytest.raises(mrf.MRFError, match="metric"):
        run(mrf, D, cfg1[2][:4], 0.0, cone="real_pos")


@pytest.mark.parametrize("eps", [0.0, 0.4])
def test_every_iteration_follows_the_oracle(mrf, cfg1, dicts, eps):
    dic, p, _ = cfg1
    A = dic["atoms"]
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    opts = mrf.proj_opts(mode="tree_tc", eps=eps)

    def eps_rule(Zs, gi, gr, gx):
        ref = mo.project(Zs, A)
        nz = np.linalg.norm(Zs, axis=1) > 0
        dg = unit_dist(Zs[nz], A, gi[nz])
        dn = unit_dist(Zs[nz], A, ref["idx"][nz])
        assert np.all(dg <= (1 + eps) * dn + 1e-6), np.max(dg - (1 + eps) * dn)
        rr = mo.density(Zs[nz], A, gi[nz])
        assert np.max(np.abs(gr[nz] - rr) / np.abs(rr)) <= 1e-4
        return float(np.mean(gi == ref["idx"]))

    X, idx, rho, rates = iterate_checked(mrf, dicts["complex"], op, AHY, A, p["iters"], opts,
                                         check=None if eps == 0.0 else eps_rule)
    print(f"eps={eps}: per-iteration exact agreement {np.round(rates, 4)}")


@pytest.mark.parametrize("group,chunks,pair,sup", [(1, 1, 2, 1), (3, 7, 2, 5), (64, 64, 2, 1),
                                                   (2, 32, 2, 16), (2, 32, 1, 16), (3, 7, 1, 3),
                                                   (64, 1, 1, 2), (0, 0, 0, 0)])
def test_schedule_knobs_keep_the_exact_result(mrf, cfg1, dicts, group, chunks, pair, sup):
    """Tiles per block list, chunks per list, lists per super-group and the tile shape (single
    CTAs, or CTA pairs of 256 voxels: an odd group is rounded up) change the work schedule and
    the candidate slots, never the answer: eps = 0 stays the exact projection (ragged voxel
    count, a short last group and super-group)."""
    dic, p, Z = cfg1
    D = dicts["complex"]
    D.set_tune(tree_tc_group=group, tree_tc_chunks=chunks, bf16_pair=pair, tree_tc_super=sup)
    try:
        for certify in (True, False):
            idx, rho, X, st = run(mrf, D, Z[:999], 0.0, certify=certify)
            if certify:
                check_projection(Z[:999], dic["atoms"], idx, rho, g_X=X)
            else:
                check_bound_rule(Z[:999], dic["atoms"], idx, rho,
                                 bf16_bound(dic["atoms"].shape[1]), g_X=X)
    finally:
        D.set_tune(tree_tc_group=0, tree_tc_chunks=0, bf16_pair=0, tree_tc_super=0)
