"""GPU parity of the cover-tree projection (MRF_PROJ_COVERTREE: Algorithm 1 per voxel, warm start,
exact rescore of the visited candidates) against the float64 oracle: the uploaded tree satisfies
the invariants of §4.1, eps = 0 equals the exhaustive projection, eps > 0 meets the (1+eps)
bound of Definition eNN, warm starts are non-expansive (§4.3), the search costs fewer distance
evaluations than brute force, the query order of warm-started searches does not change any
result, and CoverBLIP reconstructions match BLIP at eps = 0."""
import numpy as np
import pytest

import mrfgen
from oracle import covertree as ct
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection
from tree_check import check_tree

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


def run(mrf, D, Z, eps, warm=None, cone="complex"):
    n = Z.shape[0]
    idx = torch.full((n,), -3, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Xo = torch.empty((n, Z.shape[1]), dtype=torch.complex64, device="cuda")
    w = None if warm is None else to_dev(warm.astype(np.int32))
    st = mrf.project(D, to_dev(Z), idx, rho, Xo, warm_idx=w,
                     opts=mrf.proj_opts(mode="covertree", eps=eps, cone=cone), stats=True)
    return idx.cpu().numpy(), rho.cpu().numpy(), Xo.cpu().numpy(), st


def unit_dist(Z, A, idx, cone="complex"):
    """Oracle distance between z/||z|| and the unit atom idx (phase-quotient or Euclidean)."""
    metric = "phase" if cone == "complex" else "euclid"
    U = ct.unit_atoms(np.asarray(A, np.complex128))
    Zn = Z.astype(np.complex128) / np.linalg.norm(Z, axis=1)[:, None]
    return np.array([ct.pair_dist(Zn[v:v + 1], U[idx[v]:idx[v] + 1], metric)[0, 0]
                     for v in range(Z.shape[0])])


def test_uploaded_tree_invariants(mrf, cfg1):
    dic = cfg1[0]
    D = mrf.build_dict_index(dic["atoms"], build_tree=True)
    T = D.tree_export()
    check_tree(dic["atoms"], T)
    info = D.tree_info()
    assert info["nodes"] == dic["atoms"].shape[0] and info["levels"] == T["levels"]


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_eps0_equals_exhaustive(mrf, cfg1, cone):
    dic, p, Z = cfg1
    D = mrf.build_dict_index(dic["atoms"], build_tree=True, tree_cone=cone)
    idx, rho, X, st = run(mrf, D, Z, 0.0, cone=cone)
    check_projection(Z, dic["atoms"], idx, rho, cone=cone, g_X=X)
    assert st["n_dist_evals"] > 0


@pytest.mark.parametrize("eps", [0.2, 0.5, 1.0])
def test_eps_bound_and_warm_start(mrf, cfg1, eps):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, build_tree=True)
    ref = mo.project(Z, A)
    g = np.random.Generator(np.random.PCG64(int(eps * 10)))
    warm = g.integers(0, A.shape[0], Z.shape[0])
    for w in (None, warm):
        idx, rho, X, st = run(mrf, D, Z, eps, warm=w)
        dg = unit_dist(Z, A, idx)
        dnn = unit_dist(Z, A, ref["idx"])
        assert np.all(dg <= (1 + eps) * dnn + 1e-5), np.max(dg - (1 + eps) * dnn)
        if w is not None:
            assert np.all(dg <= unit_dist(Z, A, w) + 1e-6)   # non-expansive warm start
        # density of the returned atom is exact
        rr = mo.density(Z, A, idx)
        assert np.max(np.abs(rho - rr) / np.abs(rr)) <= 1e-4
        assert st["n_dist_evals"] < Z.shape[0] * A.shape[0] / 2


@pytest.mark.parametrize("eps", [0.0, 0.5])
def test_query_order_does_not_change_results(mrf, cfg1, eps):
    """Warm-started queries run in the order of their warm atom's tree position (mrf_tune
    tree_order = 1, the default) or in voxel order (2): each query runs its own Algorithm 1, so
    indices, densities and the number of distance evaluations are identical."""
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, build_tree=True)
    g = np.random.Generator(np.random.PCG64(11))
    warm = g.integers(-1, A.shape[0], Z.shape[0])      # includes invalid warm starts (-1)
    out = {}
    for order in (1, 2):
        D.set_tune(tree_order=order)
        out[order] = run(mrf, D, Z, eps, warm=warm)
    assert D.get_tune()["tree_order"] == 2
    assert np.array_equal(out[1][0], out[2][0])
    assert np.array_equal(out[1][1], out[2][1])
    assert out[1][3]["n_dist_evals"] == out[2][3]["n_dist_evals"]
    assert out[1][3]["n_fallback"] == out[2][3]["n_fallback"]
    if eps == 0.0:
        check_projection(Z, A, out[1][0], out[1][1], g_X=out[1][2])


def test_warm_start_at_the_answer_is_cheap(mrf, cfg1):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, build_tree=True)
    idx0, _, _, st0 = run(mrf, D, Z, 0.4)
    idx1, _, _, st1 = run(mrf, D, Z, 0.4, warm=idx0)
    assert st1["n_dist_evals"] <= st0["n_dist_evals"]
    assert np.all(unit_dist(Z, A, idx1) <= unit_dist(Z, A, idx0) + 1e-6)


def test_duplicates_and_zero_queries(mrf):
    g = np.random.Generator(np.random.PCG64(71))
    B = (g.standard_normal((50, 32)) + 1j * g.standard_normal((50, 32))).astype(np.complex64)
    A = np.concatenate([B, B[:10] * np.complex64(np.exp(0.3j))]).astype(np.complex64)
    js = g.integers(0, 50, 100)
    Z = (A[js] * np.complex64(2 - 1j)).astype(np.complex64)
    Z[::9] = 0
    D = mrf.build_dict_index(A, build_tree=True)
    idx, rho, X, st = run(mrf, D, Z, 0.0)
    check_projection(Z, A, idx, rho, g_X=X)
    assert st["n_zero"] == len(range(0, 100, 9))


@pytest.mark.parametrize("eps", [0.0, 0.4])
def test_coverblip_reconstruction(mrf, cfg1, eps):
    dic, p, _ = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    D = mrf.build_dict_index(dic["atoms"], dic["params"], build_tree=True)
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    out = {}
    for mode in ("fp32", "covertree"):
        X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
        st = mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx, None, prm,
                             opts=mrf.recon_opts(iters=p["iters"], mode=mode, eps=eps),
                             stats=True)
        out[mode] = (idx.cpu().numpy(), X.cpu().numpy(), prm.cpu().numpy(), st)
    fg = p["phantom"]["labels"] >= 0
    agree = np.mean(out["fp32"][0] == out["covertree"][0])
    acc = {m: mo.accuracy(out[m][2][:, 0], p["phantom"]["T1"], fg) for m in out}
    print(f"eps={eps}: agreement with exhaustive {agree:.4f}, T1 acc {acc}, "
          f"dist evals {out['covertree'][3]['n_dist_evals']}")
    if eps == 0.0:
        assert agree >= 0.995
    assert acc["covertree"] >= acc["fp32"] - 0.02
