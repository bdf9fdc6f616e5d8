"""GPU parity of the sampling operator, one BLIP iteration and whole reconstructions (workload 1:
32x32 phantom, L = 100, ~2000 atoms) against the FP64 oracle, through the C ABI."""
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


@pytest.mark.parametrize("mode,cone", [("fp32", "complex"), ("bf16", "complex"),
                                       ("fp32", "real_pos"), ("bf16", "real_pos")])
def test_reconstruct_workload1(mrf, cfg1, mode, cone):
    """Whole BLIP reconstructions against the oracle's, for both readings of the cone (the
    paper's real positive gamma and the complex density)."""
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    iters = p["iters"]
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=iters, cone=cone)
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    prm = torch.empty((n, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
    st = mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx, rho, prm,
                         opts=mrf.recon_opts(iters=iters, mode=mode, cone=cone), stats=True)
    gi = idx.cpu().numpy()
    agree = float(np.mean(gi == ref["idx"]))
    relX = np.linalg.norm(X.cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"])
    fg = p["phantom"]["labels"] >= 0
    t1g = mo.accuracy(prm.cpu().numpy()[:, 0], p["phantom"]["T1"], fg)
    t1r = mo.accuracy(mo.lut(ref["idx"], dic["params"])[:, 0], p["phantom"]["T1"], fg)
    print(f"{mode} {cone}: agreement {agree:.5f} relX {relX:.2e} T1 acc gpu {t1g:.4f} "
          f"oracle {t1r:.4f}")
    assert agree >= 0.995
    assert relX < 1e-3
    assert abs(t1g - t1r) < 2e-3
    assert np.array_equal(prm.cpu().numpy(), dic["params"][gi])


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


def test_adaptive_step_and_kappa(mrf, cfg1):
    dic, p = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    mu = float(Ny / p["masks"].sum(1).mean())
    ref = mo.blip(p["Y"], p["masks"], dic["atoms"], Ny, Nx, iters=4, mu=mu, adaptive=True,
                  history=True)
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx,
                    opts=mrf.recon_opts(iters=4, mu=mu, adaptive=True, mode="fp32"))
    agree = float(np.mean(idx.cpu().numpy() == ref["idx"]))
    assert agree > 0.99, agree
    # kappa rescale runs and keeps the image finite
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx,
                    opts=mrf.recon_opts(iters=2, kappa=True, mode="fp32"))
    assert torch.isfinite(torch.view_as_real(X)).all()


@pytest.mark.parametrize("N", [16, 24, 32, 64, 40])
def test_gradient_step_both_paths(mrf, cfg1, N):
    """Z = X - mu A^H(A X - Y) against the oracle for power-of-two Ny (the one-pass kernel:
    y-transforms, mask and combine in shared memory) and other Ny (cuFFT path)."""
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
