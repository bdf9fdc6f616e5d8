"""GPU parity of the tensor-core tree search at the million-atom size (workload 3: 999,702 atoms,
L = 500, the 256 x 256 slice's first iterate A^H Y), in the configuration bench.py times: every
voxel is projected, and a seeded sample of 128 voxels (96 object, 32 background) is checked
against the float64 oracle -- the exact rule at eps = 0 with certification (§3.2, eqs.
exactP / exactPs), and Definition eNN's (1 + eps) bound at eps = 0.5 with the BF16 operand
(up to the BF16 kernel's ranking bound)."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection, bf16_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mrf():
    import paper_1810_01967_gb300 as m
    from paper_1810_01967_gb300 import build as b
    b.build()
    return m


@pytest.fixture(scope="module")
def w3(mrf):
    dic = mrfgen.make_dictionary(3)
    p = mrfgen.make_problem(3, dic=dic)
    A = dic["atoms"]
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    D = mrf.build_dict_index(A, dic["params"], build_tree=True, tree_tc=True, pack_bf16x3=True)
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((Ny * Nx, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(3000))
    fg = np.flatnonzero(p["phantom"]["labels"] >= 0)
    bg = np.flatnonzero(p["phantom"]["labels"] < 0)
    s = np.sort(np.concatenate([g.choice(fg, 96, replace=False), g.choice(bg, 32, replace=False)]))
    Zs = AHY.cpu().numpy()[s]
    ref = mo.project(Zs, A, chunk=32)
    return {"A": A, "D": D, "AHY": AHY, "s": s, "Zs": Zs, "ref": ref, "L": L}


def _run(mrf, w, eps, certify):
    n = w["AHY"].shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    st = mrf.project(w["D"], w["AHY"], idx, rho, stats=True,
                     opts=mrf.proj_opts(mode="tree_tc", eps=eps, certify=certify))
    torch.cuda.synchronize()
    assert st["device_error"] == 0
    return idx.cpu().numpy()[w["s"]], rho.cpu().numpy()[w["s"]], st


def _unit_dist(Zs, A, idx):
    """Oracle phase-quotient distance between z/||z|| and the unit atom idx (float64)."""
    U = A[idx].astype(np.complex128)
    U /= np.linalg.norm(U, axis=1)[:, None]
    Zn = Zs.astype(np.complex128) / np.linalg.norm(Zs, axis=1)[:, None]
    return np.sqrt(np.maximum(2 - 2 * np.abs(np.sum(np.conj(U) * Zn, axis=1)), 0))


def test_eps0_certified_is_exact(mrf, w3):
    gi, gr, st = _run(mrf, w3, 0.0, True)
    agree, ties = check_projection(w3["Zs"], w3["A"], gi, gr, ref=w3["ref"])
    n, d = w3["AHY"].shape[0], w3["A"].shape[0]
    print(f"1M atoms, tree search eps 0 certified: sampled agreement {agree:.4f} ({ties} "
          f"near-ties), {st['n_uncertified']} voxels re-searched, pairs "
          f"{st['n_dist_evals'] / (n * d):.3f} of brute force")


def test_eps_half_meets_the_bound(mrf, w3):
    eps = 0.5
    gi, gr, st = _run(mrf, w3, eps, False)
    dg = _unit_dist(w3["Zs"], w3["A"], gi)
    dn = _unit_dist(w3["Zs"], w3["A"], w3["ref"]["idx"])
    lim = ((1 + eps) * dn) ** 2 + 4 * bf16_bound(w3["L"]) + 1e-12
    assert np.all(dg ** 2 <= lim), float(np.max(dg ** 2 - lim))
    rr = mo.density(w3["Zs"], w3["A"], gi)
    assert np.max(np.abs(gr - rr) / np.abs(rr)) <= 1e-4
    print(f"1M atoms, tree search eps {eps}: exact agreement "
          f"{np.mean(gi == w3['ref']['idx']):.4f}, worst distance ratio "
          f"{np.max(dg / np.maximum(dn, 1e-12)):.3f}")
