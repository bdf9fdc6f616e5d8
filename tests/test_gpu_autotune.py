"""The launch-geometry autotuner and every geometry it explores: each tile shape, cluster size,
live-tile count and atom split gives the oracle's projection (certified BF16 and FP8), the fastest setting
is applied to the dictionary and cached, and the cache is applied again without timing."""
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
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]).astype(np.complex64)
    return dic, Z


@pytest.mark.parametrize("mode", ["bf16", "fp8"])
def test_every_geometry_is_exact(mrf, cfg1, mode):
    dic, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, pack_fp8=True)
    ref = mo.project(Z, A)
    Zd = to_dev(Z)
    n = Z.shape[0]
    for C in (1, 2, 4):
        for live in (1, 8, 64):
            for S in (0, 1, 5, 16):
                D.set_tune(bf16_cluster=C, bf16_live_tiles=live, bf16_splits=S)
                idx = torch.empty(n, dtype=torch.int32, device="cuda")
                rho = torch.empty(n, dtype=torch.complex64, device="cuda")
                mrf.project(D, Zd, idx, rho, opts=mrf.proj_opts(mode=mode, certify=True))
                t = D.get_tune()
                assert t["last_bf16_cluster"] == C
                if S:
                    assert t["last_bf16_splits"] == S
                check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy(), ref=ref)


def test_tune_applies_and_caches(mrf, cfg1, tmp_path):
    from paper_1810_01967_gb300 import autotune
    dic, Z = cfg1
    D = mrf.build_dict_index(dic["atoms"])
    Zd = to_dev(np.tile(Z, (4, 1)))
    cache = str(tmp_path / "tune.json")
    grid = {"bf16_cluster": (1, 2), "bf16_live_tiles": (8, 32), "bf16_splits": (0, 4)}
    res = autotune.tune(D, Zd, "bf16", grid=grid, reps=2, cache=cache)
    assert len(res["table"]) == 8
    assert res["ms"] == min(r["ms"] for r in res["table"])
    t = D.get_tune()
    for k, v in res["tune"].items():
        assert t[k] == v
    D2 = mrf.build_dict_index(dic["atoms"])
    hit = autotune.apply_cached(D2, Zd.shape[0], "bf16", cache)
    assert hit is not None and hit["tune"] == res["tune"]
    t2 = D2.get_tune()
    for k, v in res["tune"].items():
        assert t2[k] == v


def test_default_grid_explores_both_tile_shapes(mrf, cfg1):
    """The default grid times the single-CTA tile (128 voxels) with every cluster size and the
    CTA-pair tile (256 voxels; cluster size ignored, so timed once per live-tile count), and
    the projection under the chosen geometry is still the oracle's."""
    from paper_1810_01967_gb300 import autotune
    dic, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A)
    Zd = to_dev(np.tile(Z, (4, 1)))
    res = autotune.tune(D, Zd, "bf16", reps=1)
    shapes = [(r["tune"]["bf16_pair"], r["tune"]["bf16_cluster"]) for r in res["table"]]
    assert len(res["table"]) == 12
    assert (1, 1) in shapes and (1, 2) not in shapes and (0, 4) in shapes
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.project(D, to_dev(Z), idx, rho, opts=mrf.proj_opts(mode="bf16", certify=True))
    check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy())
    print("autotuned:", res["tune"], f"{res['ms']:.3f} ms")


def test_tree_search_grid(mrf, cfg1):
    """The tensor-core tree search's schedule grid (tile shape, tiles per block list, chunks per
    list) is timed at eps = 0.5 and the chosen schedule still gives the oracle's projection at
    eps = 0 with certification."""
    from paper_1810_01967_gb300 import autotune
    dic, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, build_tree=True, tree_tc=True, pack_bf16x3=True)
    res = autotune.tune(D, to_dev(np.tile(Z, (4, 1))), "tree_tc", reps=1, proj={"eps": 0.5})
    assert len(res["table"]) == 12
    assert set(res["tune"]) == {"bf16_pair", "tree_tc_group", "tree_tc_chunks"}
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.project(D, to_dev(Z), idx, rho, opts=mrf.proj_opts(mode="tree_tc", eps=0.0))
    check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy())
    print("tree search autotuned:", res["tune"], f"{res['ms']:.3f} ms")


@pytest.mark.parametrize("mode", ["bf16", "fp8"])
def test_cta_pair_kernel_is_exact(mrf, cfg1, mode):
    """The 2-SM (CTA pair) variant of the search under several schedules: certified results
    equal the oracle's, uncertified ones stay within the rigorous bound."""
    dic, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, pack_fp8=True)
    ref = mo.project(Z, A)
    Zd = to_dev(Z)
    n = Z.shape[0]
    for live in (1, 8, 64):
        for S in (0, 1, 5):
            D.set_tune(bf16_pair=1, bf16_live_tiles=live, bf16_splits=S)
            idx = torch.empty(n, dtype=torch.int32, device="cuda")
            rho = torch.empty(n, dtype=torch.complex64, device="cuda")
            mrf.project(D, Zd, idx, rho, opts=mrf.proj_opts(mode=mode, certify=True))
            t = D.get_tune()
            assert t["last_bf16_cluster"] == 2
            check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy(), ref=ref)
    # uncertified BF16 on the pair kernel: top-16 + exact rescore within 2 x the BF16 bound
    if mode == "bf16":
        D.set_tune(bf16_pair=1, bf16_live_tiles=0, bf16_splits=0)
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        mrf.project(D, Zd, idx, opts=mrf.proj_opts(mode="bf16", certify=False))
        gi = idx.cpu().numpy()
        bound = 2.0 ** -7 + 2.0 ** -16 + 2 * Z.shape[1] * 2.0 ** -24
        assert np.all(mo.correlation(Z, A, gi) >= ref["s1"] - 2 * bound)
        assert np.mean(gi == ref["idx"]) > 0.98
