"""Edge cases across the forms: a batch with a tiny slice among larger ones, extreme subspace
compression (s = 1) and FP8 on compressed atoms, the phase-aligned real cone through the cover
tree (Euclidean tree on the aligned atoms) and through the FP8 kernel, all against the float64
oracle."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from oracle import phase as oph
from oracle import svd as osvd
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
    return dic, p, Z


def test_batch_with_a_tiny_slice(mrf, cfg1):
    dic = cfg1[0]
    probs = [mrfgen.make_problem(1, i, dic=dic, N=N) for i, N in enumerate((8, 32))]
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    ops = [mrf.make_op(p["Ny"], p["Nx"], p["L"], to_dev(p["masks"])) for p in probs]
    B = mrf.Batch(D, ops)
    B.load([to_dev(p["Y"]) for p in probs])
    B.run(3, 1.0, mrf.proj_opts(mode="fp32", certify=False), use_graph=True)
    torch.cuda.synchronize()
    for s, p in enumerate(probs):
        ref = mo.blip(p["Y"], p["masks"], dic["atoms"], p["Ny"], p["Nx"], iters=3)
        v = B.views(s)
        agree = float(np.mean(v["idx"].cpu().numpy() == ref["idx"]))
        assert v["n"] == p["Ny"] * p["Nx"] and agree >= 0.99, (s, agree)


@pytest.mark.parametrize("s,mode", [(1, "fp32"), (12, "fp8")])
def test_extreme_compression_and_fp8_on_compressed_atoms(mrf, cfg1, s, mode):
    dic, p, Z = cfg1
    Vo, _ = osvd.svd_basis(dic["atoms"], s)
    V64 = Vo.astype(np.complex64)
    Ac = osvd.compress(dic["atoms"], V64).astype(np.complex64)
    Zc = osvd.compress(Z, V64).astype(np.complex64)
    D = mrf.build_dict_index(Ac, pack_fp8=(mode == "fp8"))
    n = Zc.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.project(D, to_dev(Zc), idx, rho, opts=mrf.proj_opts(mode=mode, certify=True))
    check_projection(Zc, Ac, idx.cpu().numpy(), rho.cpu().numpy())


def test_phase_aligned_real_cone_through_the_tree_and_fp8(mrf, cfg1):
    dic, p, Z = cfg1
    A = dic["atoms"]
    ref = oph.project_phase_aligned(Z, A)
    n = Z.shape[0]
    Za = Z.astype(np.complex128) * ref["eb"].conj()[:, None]
    Aa = A.astype(np.complex128) * ref["ea"].conj()[:, None]
    # the Euclidean cover tree on the aligned atoms, eps = 0: the aligned real projection
    D = mrf.build_dict_index(A, phase_align=True, pack_fp8=True, build_tree=True,
                             tree_cone="real_pos")
    for opts in (mrf.proj_opts(mode="covertree", cone="real_pos", eps=0.0),
                 mrf.proj_opts(mode="fp8", cone="real_pos", certify=True)):
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        mrf.project(D, to_dev(Z), idx, opts=opts)
        gi = idx.cpu().numpy()
        sg = mo.correlation(Za, Aa, gi, "real_pos")
        ok = (gi == ref["idx"]) | (sg >= ref["s1"] - 2e-6 * np.abs(ref["s1"]))
        assert np.all(ok), (opts.mode, np.flatnonzero(~ok)[:10])
