"""GPU parity of the sampling operator, one BLIP iteration and whole reconstructions (workload 1:
32x32 phantom, L = 100, ~2000 atoms) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection, iterate_checked, bf16_bound

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
    return dic, mrfgen.make_problem(1, dic=dic)


def test_forward_adjoint(mrf, cfg1):
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    g = np.random.Generator(np.random.PCG64(5))
    X = (g.standard_normal((Ny * Nx, L)) + 1j * g.standard_normal((Ny * Nx, L))).astype(np.complex64)
    mask = to_dev(p["masks"])
    op = mrf.make_op(Ny, Nx, L, mask)
    Yd = torch.empty((Ny, Nx, L), dtype=torch.complex64, device="cuda")
    mrf.forward(op, to_dev(X), Yd)
    Yr = mo.forward(X, p["masks"], Ny, Nx)
    assert np.linalg.norm(Yd.cpu().numpy() - Yr) / np.linalg.norm(Yr) < 1e-5
    A = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), A)
    Ar = mo.adjoint(p["Y"], p["masks"], Ny, Nx)
    assert np.linalg.norm(A.cpu().numpy() - Ar) / np.linalg.norm(Ar) < 1e-5


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_one_iteration_from_a_phantom_iterate(mrf, cfg1, mode):
    """mrf_ipg_step on a non-trivial X: compare Z-projection with the oracle's step."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    ref1 = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=1)
    X1 = ref1["X"].astype(np.complex64)
    mu = 1.0
    Zr = mo.gradient_step(X1, p["Y"], p["masks"], Ny, Nx, mu)
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    Xd = to_dev(X1)
    idx = to_dev(ref1["idx"].astype(np.int32))
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.ipg_step(D, op, AHY, Xd, mu, idx, rho, opts=mrf.proj_opts(mode=mode))
    torch.cuda.synchronize()
    # the GPU's Z differs from the FP64 one by FP32 rounding (~1e-7 relative): widen the
    # near-tie window accordingly and check rho against the oracle's Z
    agree, ties = check_projection(Zr, dic["atoms"], idx.cpu().numpy(), rho.cpu().numpy(),
                                   g_X=Xd.cpu().numpy(), tie=1e-5)
    print(f"{mode}: one-step agreement {agree:.5f} ({ties} near-tie swaps)")


@pytest.mark.parametrize("mode,cone,certify", [
    ("fp32", "complex", True), ("bf16", "complex", True), ("bf16x3", "complex", True),
    ("fp32", "real_pos", True), ("bf16", "real_pos", True), ("bf16", "complex", False)])
def test_reconstruct_workload1(mrf, cfg1, mode, cone, certify):
    """Whole BLIP reconstructions, both readings of the cone (the paper's real positive gamma
    and the complex density): every iteration's projection of the GPU's own Z follows the
    oracle (exact rule for the exact and certified forms, the kernel-bound rule for uncertified
    BF16), the single-call mrf_reconstruct reproduces the iteration-by-iteration run bit for
    bit, and the look-up table returns the atoms' parameters.  The agreement with the oracle's
    own whole reconstruction is printed as a report."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    iters = p["iters"]
    A = dic["atoms"]
    D = mrf.build_dict_index(A, dic["params"], pack_bf16x3=(mode == "bf16x3"))
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    po = mrf.proj_opts(mode=mode, cone=cone, certify=certify)
    rule = "exact" if (certify or mode in ("fp32", "bf16x3")) else "bound"
    Xi, ii, ri, rates = iterate_checked(mrf, D, op, AHY, A, iters, po, cone=cone, rule=rule,
                                        bound=bf16_bound(L))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx, rho, prm,
                    opts=mrf.recon_opts(iters=iters, mode=mode, cone=cone, certify=certify))
    torch.cuda.synchronize()
    assert torch.equal(idx, ii) and torch.equal(X, Xi) and torch.equal(rho, ri)
    gi = idx.cpu().numpy()
    assert np.array_equal(prm.cpu().numpy(), dic["params"][gi])
    ref = mo.blip(p["Y"], p["masks"], A, Ny, Nx, iters=iters, cone=cone)
    agree = float(np.mean(gi == ref["idx"]))
    relX = np.linalg.norm(X.cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"])
    fg = p["phantom"]["labels"] >= 0
    t1g = mo.accuracy(prm.cpu().numpy()[:, 0], p["phantom"]["T1"], fg)
    t1r = mo.accuracy(mo.lut(ref["idx"], dic["params"])[:, 0], p["phantom"]["T1"], fg)
    print(f"{mode} {cone} certify={certify}: per-iteration agreement with the oracle's "
          f"projection of the GPU's Z {min(rates):.5f}..{max(rates):.5f}; end state vs the "
          f"oracle's reconstruction {agree:.5f}, relX {relX:.2e}, T1 acc gpu {t1g:.4f} "
          f"oracle {t1r:.4f}")


def test_noiseless_full_sampling_exact(mrf, cfg1):
    dic, _ = cfg1
    p = mrfgen.make_problem(1, dic=dic, snap=True, full_sampling=True, noiseless=True)
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx, rho, opts=mrf.recon_opts(iters=1, mode="bf16"))
    fg = p["phantom"]["labels"] >= 0
    assert np.array_equal(idx.cpu().numpy()[fg], p["truth_idx"][fg])
    np.testing.assert_allclose(rho.cpu().numpy()[fg], p["phantom"]["rho"][fg], rtol=1e-5)


def _fidelity(X, p):
    """||Y - A X|| by the oracle's forward model (Y zero off the sampled lines)."""
    Ny, Nx = p["Ny"], p["Nx"]
    Yk = p["Y"] * p["masks"].T.astype(np.float64)[:, None, :]
    return float(np.linalg.norm(Yk - mo.forward(X, p["masks"], Ny, Nx)))


def test_step_rule_guarantees(mrf, cfg1):
    """The adaptive step rule (eq. steprule, Algorithm 2) on the GPU, FP32 exact projection,
    mu = n/m: every accepted step satisfies the rule (checked with the oracle's forward model on
    the GPU's own iterates), it lies in Prop. stepbound's interval [(zeta beta)^-1, mu] with
    beta = 1 (unitary F and line masks: ||A dX|| <= ||dX||) after at most
    ceil(log_zeta(mu beta)) + 1 sub-iterations, the fidelity ||Y - A X^k|| does not increase
    (Thm. inexactmonotone), and the accepted steps equal the oracle's adaptive BLIP."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, iters, zeta = Ny * Nx, 8, 2.0
    mu = float(Ny / p["masks"].sum(1).mean())
    A = dic["atoms"]
    D = mrf.build_dict_index(A, dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    mus = np.zeros(iters, np.float32)
    shr = np.zeros(iters, np.int32)
    Xs = [np.zeros((n, L), np.complex64)]
    for k in range(iters):            # one iteration per call (the rule restarts from mu)
        mh, sh = np.zeros(1, np.float32), np.zeros(1, np.int32)
        mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx,
                        opts=mrf.recon_opts(iters=1, mu=mu, adaptive=True, zeta=zeta,
                                            resume=(k > 0), mode="fp32", mu_history=mh,
                                            shrink_history=sh))
        torch.cuda.synchronize()
        mus[k], shr[k] = mh[0], sh[0]
        Xs.append(X.cpu().numpy())
    bound = int(np.ceil(np.log(mu * 1.0) / np.log(zeta))) + 1
    fid = [_fidelity(x, p) for x in Xs]
    for k in range(iters):
        dX = Xs[k + 1].astype(np.complex128) - Xs[k]
        num = np.sum(np.abs(dX) ** 2)
        den = np.sum(np.abs(mo.forward(dX, p["masks"], Ny, Nx)) ** 2)
        assert den == 0 or mus[k] < num / den * (1 + 1e-5), (k, mus[k], num / den)
        assert 1.0 / zeta <= mus[k] <= mu and shr[k] <= bound, (k, mus[k], shr[k], bound)
        assert fid[k + 1] <= fid[k] * (1 + 1e-6), (k, fid[k], fid[k + 1])
    ref = mo.blip(p["Y"], p["masks"], A, Ny, Nx, iters=iters, mu=mu, adaptive=True, zeta=zeta,
                  history=True)
    np.testing.assert_allclose(mus, ref["history"]["mu"], rtol=1e-6)
    assert list(shr) == list(ref["history"]["shrinks"])
    print(f"step rule: mu_k {mus.tolist()}, shrinks {shr.tolist()} (bound {bound}), "
          f"fidelity {[round(f, 5) for f in fid]}")


def test_kappa_rescale_matches_oracle(mrf, cfg1):
    """The kappa rescale of the first iterate (X^1 <- kappa X^1, mu <- kappa mu with
    kappa = ||Y|| / ||A X^1||, the step rule's initialisation option): kappa from the GPU's own
    first iterate equals the oracle's formula on it, and a 4-iteration kappa-rescaled FP32
    reconstruction matches oracle.blip(kappa=True) element by element (indices exact except
    near-ties, images within 1e-4 per voxel)."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    A = dic["atoms"]
    D = mrf.build_dict_index(A, dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    X1 = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    X1k = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X1, idx, opts=mrf.recon_opts(iters=1, mode="fp32"))
    mrf.reconstruct(D, op, to_dev(p["Y"]), X1k, idx,
                    opts=mrf.recon_opts(iters=1, kappa=True, mode="fp32"))
    torch.cuda.synchronize()
    x1, x1k = X1.cpu().numpy().astype(np.complex128), X1k.cpu().numpy().astype(np.complex128)
    Yk = p["Y"] * p["masks"].T.astype(np.float64)[:, None, :]
    kap = np.linalg.norm(Yk) / np.linalg.norm(mo.forward(x1, p["masks"], Ny, Nx))
    np.testing.assert_allclose(x1k, kap * x1, rtol=2e-6, atol=1e-6 * np.abs(x1k).max())
    iters = 4
    ref = mo.blip(p["Y"], p["masks"], A, Ny, Nx, iters=iters, kappa=True)
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx, rho,
                    opts=mrf.recon_opts(iters=iters, kappa=True, mode="fp32"))
    torch.cuda.synchronize()
    gi, gx = idx.cpu().numpy(), X.cpu().numpy()
    same = gi == ref["idx"]
    assert same.mean() >= 0.999, same.mean()
    # row errors relative to the image's RMS row norm: the FP32 transforms' rounding is bounded
    # relative to the whole transform, so weak background rows carry larger relative errors
    num = np.linalg.norm(gx[same] - ref["X"][same], axis=1)
    rms = np.sqrt(np.mean(np.sum(np.abs(ref["X"]) ** 2, axis=1)))
    assert np.max(num / rms) < 1e-5, np.max(num / rms)
    print(f"kappa {kap:.6f}: atoms equal to the oracle's {same.mean():.5f}, "
          f"largest row error / RMS row norm {np.max(num / rms):.2e}")


@pytest.mark.parametrize("N", [16, 24, 32, 64, 40, 48, 60, 96, 192, 28])
def test_gradient_step_both_paths(mrf, cfg1, N):
    """Z = X - mu A^H(A X - Y) against the oracle for power-of-two Ny (the one-pass kernel:
    radix-2 y-transforms, mask and combine in shared memory), Ny = 2^a 3^b 5^c (the same pass
    with mixed-radix Stockham transforms: 24, 40, 48, 60, 96, 192) and other Ny (cuFFT path:
    28)."""
    dic, _ = cfg1
    p = mrfgen.make_problem(1, dic=dic, N=N)
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    g = np.random.Generator(np.random.PCG64(N))
    X = (g.standard_normal((n, L)) + 1j * g.standard_normal((n, L))).astype(np.complex64)
    D = mrf.build_dict_index(dic["atoms"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    Z = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.gradient(D, op, AHY, to_dev(X), 0.7, Z)
    ref = mo.gradient_step(X, p["Y"], p["masks"], Ny, Nx, 0.7)
    err = np.linalg.norm(Z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 2e-6, err
