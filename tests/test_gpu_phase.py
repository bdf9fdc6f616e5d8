"""GPU parity of the phase-aligned real positive projection (§4.3) against the float64 oracle
(oracle/phase.py): single projections in FP32 and certified BF16, the complex cone unchanged by
alignment (densities still relative to the atoms as given), and whole reconstructions."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from oracle import phase as oph
from gpu_util import to_dev, check_projection, iterate_checked

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


def aligned_scores(Z, A, idx, ref):
    """Aligned real score of atom idx[v] for voxel v, with the oracle's phases."""
    Za = Z.astype(np.complex128) * ref["eb"].conj()[:, None]
    Da = A.astype(np.complex128)[idx] * ref["ea"][idx].conj()[:, None]
    c = np.sum(Da.conj() * Za, axis=1).real
    den = np.linalg.norm(Da, axis=1) * np.linalg.norm(Za, axis=1)
    return c / np.where(den == 0, 1, den)


def run(mrf, D, Z, mode, cone):
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    X = torch.empty((n, Z.shape[1]), dtype=torch.complex64, device="cuda")
    mrf.project(D, to_dev(Z), idx, rho, X, opts=mrf.proj_opts(mode=mode, cone=cone))
    return idx.cpu().numpy(), rho.cpu().numpy(), X.cpu().numpy()


def check_aligned(Z, A, gi, gr, gX, v1=None, tie=2e-6):
    """The phase-aligned real positive projection against the oracle's: the atom (exact except
    aligned near-ties), the density gamma e^{i(beta - alpha)} relative to the atom as given and
    X = rho D_j, within 1e-4.  Returns the exact agreement rate."""
    ref = oph.project_phase_aligned(Z, A, v1)
    sg = aligned_scores(Z, A, gi, ref)
    ok = (gi == ref["idx"]) | (sg >= ref["s1"] - tie * np.abs(ref["s1"]))
    assert np.all(ok), np.flatnonzero(~ok)[:10]
    Ad = A.astype(np.complex128)[gi]
    gam = np.maximum(sg * np.linalg.norm(Z, axis=1) / np.linalg.norm(Ad, axis=1), 0.0)
    rr = gam * ref["eb"] * ref["ea"][gi].conj()
    err = np.abs(gr - rr) / np.maximum(np.abs(rr), 1e-30)
    assert np.max(np.where(np.abs(rr) > 0, err, np.abs(gr))) < 1e-4
    Xr = rr[:, None] * Ad
    assert np.max(np.linalg.norm(gX - Xr, axis=1) /
                  np.maximum(np.linalg.norm(Xr, axis=1), 1e-30)) < 1e-4
    return float(np.mean(gi == ref["idx"]))


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_aligned_projection_matches_oracle(mrf, cfg1, mode):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, phase_align=True)
    gi, gr, gX = run(mrf, D, Z, mode, "real_pos")
    agree = check_aligned(Z, A, gi, gr, gX)
    print(f"{mode}: aligned agreement {agree:.5f}")


def test_complex_cone_unchanged_by_alignment(mrf, cfg1):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = mrf.build_dict_index(A, phase_align=True)
    gi, gr, gX = run(mrf, D, Z, "bf16", "complex")
    check_projection(Z, A, gi, gr, g_X=gX)


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_aligned_reconstruction(mrf, cfg1, mode):
    """Whole aligned reconstructions: every iteration's projection of the GPU's own Z follows
    the oracle's phase-aligned projection (the certified forms), and the single-call
    mrf_reconstruct reproduces the iteration-by-iteration run bit for bit.  The agreement with
    the oracle's own aligned BLIP is printed as a report."""
    dic, p, _ = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n, iters = Ny * Nx, p["iters"]
    A = dic["atoms"]
    V1 = oph.project_phase_aligned(np.zeros((1, L)), A)["v1"]
    D = mrf.build_dict_index(A, dic["params"], phase_align=True)
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    po = mrf.proj_opts(mode=mode, cone="real_pos")
    Xi, ii, _, rates = iterate_checked(
        mrf, D, op, AHY, A, iters, po, cone="real_pos",
        check=lambda Z, gi, gr, gx: check_aligned(Z, A, gi, gr, gx, V1))
    X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    mrf.reconstruct(D, op, to_dev(p["Y"]), X, idx,
                    opts=mrf.recon_opts(iters=iters, mode=mode, cone="real_pos"))
    torch.cuda.synchronize()
    assert torch.equal(idx, ii) and torch.equal(X, Xi)

    def pf(Zv, warm):
        r = oph.project_phase_aligned(Zv, A, V1)
        return r["idx"], r["rho"]

    ref = mo.blip(p["Y"], p["masks"], A, Ny, Nx, iters=iters, project_fn=pf)
    agree = float(np.mean(idx.cpu().numpy() == ref["idx"]))
    relX = np.linalg.norm(X.cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"])
    print(f"aligned recon {mode}: per-iteration agreement {min(rates):.5f}..{max(rates):.5f}; "
          f"end state vs the oracle's aligned BLIP {agree:.5f}, relX {relX:.2e}")
