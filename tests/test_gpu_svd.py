"""GPU parity of the subspace-compressed BLIP (§3.3: eqs. CS1, gradupdate, gradcompression)
against the float64 oracle (oracle/svd.py): the basis spans the dominant eigenvectors of the
frame Gram matrix, compression and expansion, one compressed iteration from a common iterate,
whole compressed reconstructions in FP32 and BF16, the full basis reproducing BLIP, and the
cover tree built on the compressed atoms (CoverBLIP in C^s)."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
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
    return dic, p


@pytest.mark.parametrize("s", [10, 25])
def test_basis_matches_oracle(mrf, cfg1, s):
    dic, _ = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A)
    V, eig = mrf.svd_basis(D, s)
    Vg = V.cpu().numpy().astype(np.complex128)
    Vo, wo = osvd.svd_basis(A, s)
    assert np.max(np.abs(Vg.conj().T @ Vg - np.eye(s))) < 1e-5
    # FP64 Gram matrix: eigenvalues to rounding of the largest
    np.testing.assert_allclose(eig, wo, rtol=1e-6, atol=1e-9 * wo[0])
    # same subspace: the principal cosines are all ~1
    cos = np.linalg.svd(Vo.conj().T @ Vg, compute_uv=False)
    assert cos.min() > 0.9999, cos.min()
    # energy kept by the GPU basis equals the oracle's optimum
    kg = np.sum(np.abs(osvd.compress(A, Vg)) ** 2)
    assert abs(kg - wo.sum()) <= 2e-4 * wo.sum()


def test_compress_expand(mrf, cfg1):
    dic, p = cfg1
    L = p["L"]
    Vo, _ = osvd.svd_basis(dic["atoms"], 16)
    V = to_dev(Vo.astype(np.complex64))
    so = mrf.SvdOp(V)
    g = np.random.Generator(np.random.PCG64(5))
    X = (g.standard_normal((333, L)) + 1j * g.standard_normal((333, L))).astype(np.complex64)
    Xc = torch.empty((333, 16), dtype=torch.complex64, device="cuda")
    so.compress(to_dev(X), Xc)
    ref = osvd.compress(X, Vo.astype(np.complex64))
    np.testing.assert_allclose(Xc.cpu().numpy(), ref, atol=1e-5 * np.abs(ref).max())
    Xe = torch.empty((333, L), dtype=torch.complex64, device="cuda")
    so.expand(Xc, Xe)
    refe = osvd.expand(Xc.cpu().numpy(), Vo.astype(np.complex64))
    np.testing.assert_allclose(Xe.cpu().numpy(), refe, atol=1e-5 * np.abs(refe).max())


def _setup(mrf, dic, p, s):
    Vo, _ = osvd.svd_basis(dic["atoms"], s)
    V64 = Vo.astype(np.complex64)
    Vd = to_dev(V64)
    op = mrf.make_op(p["Ny"], p["Nx"], p["L"], to_dev(p["masks"]))
    so = mrf.SvdOp(Vd, op)
    Ac = osvd.compress(dic["atoms"], V64).astype(np.complex64)
    Dc = mrf.build_dict_index(Ac, dic["params"])
    return V64, so, Dc, Ac


def test_one_compressed_iteration(mrf, cfg1):
    dic, p = cfg1
    Ny, Nx = p["Ny"], p["Nx"]
    n, s = Ny * Nx, 20
    V64, so, Dc, Ac = _setup(mrf, dic, p, s)
    r1 = osvd.blip_svd(p["Y"], p["masks"], dic["atoms"], V64, Ny, Nx, iters=1)
    Xc1 = r1["Xc"].astype(np.complex64)
    # oracle's second gradient step from the same (rounded) iterate
    Zc = osvd.gradient_step_c(Xc1, p["Y"], p["masks"], Ny, Nx, 1.0, V64)
    AHYc = to_dev(osvd.compress(mo.adjoint(p["Y"], p["masks"], Ny, Nx), V64).astype(np.complex64))
    Xd = to_dev(Xc1)
    idx = to_dev(r1["idx"].astype(np.int32))
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    so.ipg_step(Dc, AHYc, Xd, 1.0, idx, rho, opts=mrf.proj_opts(mode="fp32"))
    torch.cuda.synchronize()
    agree, ties = check_projection(Zc, Ac, idx.cpu().numpy(), rho.cpu().numpy(),
                                   g_X=Xd.cpu().numpy(), tie=1e-5)
    print(f"compressed step: agreement {agree:.5f} ({ties} near-tie swaps)")


def iterate_c(mrf, so, Dc, AHYc, Ac, iters, opts, check):
    """Compressed BLIP iterations through the C ABI, one compressed gradient step
    (mrf_svd_gradient) and one projection (mrf_project, warm-started) at a time; after every
    projection `check(Zc, idx, rho, Xc)` compares the answers on the GPU's own Zc with the
    oracle's.  Returns the device Xc, idx, rho."""
    n, s = AHYc.shape
    Xc = torch.zeros((n, s), dtype=torch.complex64, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Zc = torch.empty_like(Xc)
    for _ in range(iters):
        so.gradient(Dc, AHYc, Xc, 1.0, Zc)
        mrf.project(Dc, Zc, idx, rho, Xc, warm_idx=idx, opts=opts)
        torch.cuda.synchronize()
        check(Zc.cpu().numpy(), idx.cpu().numpy(), rho.cpu().numpy(), Xc.cpu().numpy())
    return Xc, idx, rho


def _ahyc(so, p):
    n, L = p["Ny"] * p["Nx"], p["L"]
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf_mod = __import__("paper_1810_01967_gb300")
    op = mrf_mod.make_op(p["Ny"], p["Nx"], L, to_dev(p["masks"]))
    mrf_mod.adjoint(op, to_dev(p["Y"]), AHY)
    AHYc = torch.empty((n, so.s), dtype=torch.complex64, device="cuda")
    so.compress(AHY, AHYc)
    return AHYc


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_compressed_reconstruction(mrf, cfg1, mode):
    """Compressed BLIP (s = 20): every iteration's projection of the GPU's own compressed Z
    follows the oracle's exact projection onto the compressed atoms (FP32 and certified BF16),
    the single-call mrf_svd_reconstruct reproduces the checked run bit for bit, and the look-up
    table returns the atoms' parameters.  The compressed gradient step itself is compared with
    the oracle's (eq. gradupdate) on the GPU's iterates; the end state against the oracle's
    compressed BLIP is a report."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, s, iters = Ny * Nx, 20, p["iters"]
    V64, so, Dc, Ac = _setup(mrf, dic, p, s)
    AHYc = _ahyc(so, p)
    opts = mrf.proj_opts(mode=mode, certify=True)
    state = {"X": np.zeros((n, s), np.complex64)}

    def check(Zc, gi, gr, gx):
        Zr = osvd.gradient_step_c(state["X"], p["Y"], p["masks"], Ny, Nx, 1.0, V64)
        scale = np.sqrt(np.mean(np.sum(np.abs(Zr) ** 2, axis=1)))
        assert np.max(np.linalg.norm(Zc - Zr, axis=1)) < 2e-5 * scale
        check_projection(Zc, Ac, gi, gr, g_X=gx)
        state["X"] = gx

    Xi, ii, ri = iterate_c(mrf, so, Dc, AHYc, Ac, iters, opts, check)
    Xc = torch.empty((n, s), dtype=torch.complex64, device="cuda")
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
    so.reconstruct(Dc, to_dev(p["Y"]), iters, Xc, idx, X, None, prm, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(idx, ii) and torch.equal(Xc, Xi)
    gi = idx.cpu().numpy()
    assert np.array_equal(prm.cpu().numpy(), dic["params"][gi])
    Xe = osvd.expand(Xc.cpu().numpy(), V64)
    np.testing.assert_allclose(X.cpu().numpy(), Xe, rtol=0, atol=1e-5 * np.abs(Xe).max())
    ref = osvd.blip_svd(p["Y"], p["masks"], dic["atoms"], V64, Ny, Nx, iters=iters)
    print(f"svd s={s} {mode}: end state vs the oracle's compressed BLIP "
          f"{np.mean(gi == ref['idx']):.5f}")


def test_compressed_step_rule_and_kappa(mrf, cfg1):
    """The compressed step rule (§4.3) and kappa rescale on the GPU: the accepted steps and
    shrinks equal the oracle's compressed BLIP with the same options (within Prop. stepbound's
    count), every adaptive iteration's projection of the GPU's own compressed Z (the gradient
    at the accepted step) follows the oracle's exact projection, the fidelity
    ||Y - A(expand(Xc^k))|| does not increase, and kappa equals the oracle's formula on the
    GPU's own first iterate."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, s, iters = Ny * Nx, 20, 6
    V64, so, Dc, Ac = _setup(mrf, dic, p, s)
    AHYc = _ahyc(so, p)
    mu = float(Ny / p["masks"].sum(1).mean())
    ref = osvd.blip_svd(p["Y"], p["masks"], dic["atoms"], V64, Ny, Nx, iters=iters, mu=mu,
                        adaptive=True, history=True)
    Xc = torch.empty((n, s), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    Zc = torch.empty_like(Xc)
    prev = torch.zeros((n, s), dtype=torch.complex64, device="cuda")
    fid = [np.linalg.norm(p["Y"])]
    for k in range(1, iters + 1):
        mh, sh = np.zeros(k, np.float32), np.zeros(k, np.int32)
        so.reconstruct(Dc, to_dev(p["Y"]), k, Xc, idx, None, rho, mu=mu, adaptive=True,
                       opts=mrf.proj_opts(mode="fp32"), mu_history=mh, shrink_history=sh)
        so.gradient(Dc, AHYc, prev, float(mh[-1]), Zc)
        torch.cuda.synchronize()
        check_projection(Zc.cpu().numpy(), Ac, idx.cpu().numpy(), rho.cpu().numpy(),
                         g_X=Xc.cpu().numpy())
        Xk = osvd.expand(Xc.cpu().numpy(), V64)
        fid.append(np.linalg.norm(p["Y"] - mo.forward(Xk, p["masks"], Ny, Nx)))
        prev.copy_(Xc)
    np.testing.assert_allclose(mh, ref["history"]["mu"], rtol=1e-6)
    assert list(sh) == list(ref["history"]["shrinks"])
    assert max(sh) <= int(np.ceil(np.log(mu) / np.log(2.0))) + 1
    assert all(b <= a * (1 + 1e-6) for a, b in zip(fid, fid[1:])), fid
    # kappa on the GPU's own first iterate
    X1 = torch.empty((n, s), dtype=torch.complex64, device="cuda")
    X1k = torch.empty((n, s), dtype=torch.complex64, device="cuda")
    so.reconstruct(Dc, to_dev(p["Y"]), 1, X1, idx, opts=mrf.proj_opts(mode="fp32"))
    so.reconstruct(Dc, to_dev(p["Y"]), 1, X1k, idx, kappa=True, opts=mrf.proj_opts(mode="fp32"))
    torch.cuda.synchronize()
    x1 = X1.cpu().numpy().astype(np.complex128)
    kap = np.linalg.norm(p["Y"]) / np.linalg.norm(mo.forward(osvd.expand(x1, V64), p["masks"],
                                                              Ny, Nx))
    x1k = X1k.cpu().numpy()
    np.testing.assert_allclose(x1k, kap * x1, rtol=2e-6, atol=1e-6 * np.abs(x1k).max())
    print(f"compressed step rule: mu_k {mh.tolist()}, shrinks {sh.tolist()}, "
          f"fidelity {[round(f, 4) for f in fid]}, kappa {kap:.5f}")


def test_full_basis_reproduces_blip(mrf, cfg1):
    """The full basis (s = L): every compressed iteration follows the oracle's exact projection
    of the GPU's own Zc, and the expanded iterates stay those of BLIP (the compressed form is
    BLIP after the unitary change of variable X = Xc V^T)."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, iters = Ny * Nx, 4
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    V, _ = mrf.svd_basis(D, L)
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    so = mrf.SvdOp(V, op)
    Ac_d = torch.empty((dic["atoms"].shape[0], L), dtype=torch.complex64, device="cuda")
    mrf.SvdOp(V).compress(to_dev(dic["atoms"]), Ac_d)
    Ac = Ac_d.cpu().numpy()
    Dc = mrf.build_dict_index(Ac_d, dic["params"])
    AHYc = _ahyc(so, p)
    Xi, ii, _ = iterate_c(mrf, so, Dc, AHYc, Ac, iters, mrf.proj_opts(mode="fp32"),
                          lambda Zc, gi, gr, gx: check_projection(Zc, Ac, gi, gr, g_X=gx))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    so.expand(Xi, X)
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=iters)
    agree = float(np.mean(ii.cpu().numpy() == ref["idx"]))
    relX = np.linalg.norm(X.cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"])
    print(f"full basis: agreement with BLIP {agree:.5f} relX {relX:.2e}")


@pytest.mark.parametrize("eps", [0.0, 0.5])
def test_compressed_cover_tree(mrf, cfg1, eps):
    """CoverBLIP in the compressed domain (the paper's temporal compression option for every
    search, §4.3 and §6): the tree is built on the compressed atoms; eps = 0 reproduces the
    compressed exhaustive projection, eps > 0 meets the (1+eps) bound of Definition eNN in C^s,
    and whole compressed reconstructions match the oracle's compressed BLIP at eps = 0."""
    from oracle import covertree as ct
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, s, iters = Ny * Nx, 20, p["iters"]
    V64, so, _, Ac = _setup(mrf, dic, p, s)
    Dc = mrf.build_dict_index(Ac, dic["params"], build_tree=True)
    # one projection of the compressed first iterate
    Zc = osvd.compress(mo.adjoint(p["Y"], p["masks"], Ny, Nx), V64).astype(np.complex64)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    st = mrf.project(Dc, to_dev(Zc), idx, rho, stats=True,
                     opts=mrf.proj_opts(mode="covertree", eps=eps))
    gi = idx.cpu().numpy()
    if eps == 0.0:
        check_projection(Zc, Ac, gi, rho.cpu().numpy())
    else:
        U = ct.unit_atoms(Ac.astype(np.complex128))
        Zn = Zc.astype(np.complex128) / np.linalg.norm(Zc, axis=1)[:, None]
        ref = mo.project(Zc, Ac)
        dg = np.array([ct.pair_dist(Zn[v:v + 1], U[gi[v]:gi[v] + 1], "phase")[0, 0]
                       for v in range(n)])
        dn = np.array([ct.pair_dist(Zn[v:v + 1], U[ref["idx"][v]:ref["idx"][v] + 1], "phase")[0, 0]
                       for v in range(n)])
        assert np.all(dg <= (1 + eps) * dn + 1e-5), np.max(dg - (1 + eps) * dn)
    assert 0 < st["n_dist_evals"] < n * Ac.shape[0] / 2
    # whole compressed reconstruction
    Xc = torch.empty((n, s), dtype=torch.complex64, device="cuda")
    prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
    so.reconstruct(Dc, to_dev(p["Y"]), iters, Xc, idx, None, None, prm,
                   opts=mrf.proj_opts(mode="covertree", eps=eps))
    gi = idx.cpu().numpy()
    ref = osvd.blip_svd(p["Y"], p["masks"], dic["atoms"], V64, Ny, Nx, iters=iters)
    agree = float(np.mean(gi == ref["idx"]))
    print(f"compressed CoverBLIP eps={eps}: agreement with the oracle's compressed BLIP {agree:.4f}")
    fg = p["phantom"]["labels"] >= 0
    acc = mo.accuracy(dic["params"][gi, 0], p["phantom"]["T1"], fg)
    acc_ref = mo.accuracy(dic["params"][ref["idx"], 0], p["phantom"]["T1"], fg)
    print(f"  T1 accuracy {acc:.4f} (oracle's compressed BLIP {acc_ref:.4f})")
    assert acc >= acc_ref - 0.02
    assert np.array_equal(prm.cpu().numpy(), dic["params"][gi])
    # every iteration: eps = 0 is the exact compressed projection, eps > 0 meets the (1+eps)
    # bound of Definition eNN in C^s, on the GPU's own compressed Z
    U = ct.unit_atoms(Ac.astype(np.complex128))

    def check(Zc, gi, gr, gx):
        if eps == 0.0:
            check_projection(Zc, Ac, gi, gr, g_X=gx)
            return
        Zn = Zc.astype(np.complex128) / np.maximum(np.linalg.norm(Zc, axis=1), 1e-30)[:, None]
        ref = mo.project(Zc, Ac)
        live = np.linalg.norm(Zc, axis=1) > 0
        for v in np.flatnonzero(live):
            dg = ct.pair_dist(Zn[v:v + 1], U[gi[v]:gi[v] + 1], "phase")[0, 0]
            dn = ct.pair_dist(Zn[v:v + 1], U[ref["idx"][v]:ref["idx"][v] + 1], "phase")[0, 0]
            assert dg <= (1 + eps) * dn + 1e-5, (v, dg, dn)

    iterate_c(mrf, so, Dc, _ahyc(so, p), Ac, iters,
              mrf.proj_opts(mode="covertree", eps=eps), check)
