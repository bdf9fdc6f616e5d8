"""Failure detection without a GPU fault, and checkpoint / resume:
  * a bounded device-side wait that nothing satisfies gives up, the kernel raises the device
    error word and the call returns MRF_ETIMEOUT; the context stays usable;
  * device allocations refused on purpose (mrf_debug_fail_alloc) make the dictionary build, the
    scratch growth of a projection and a reconstruction fail with MRF_ENOMEM, and the library
    works normally afterwards;
  * a reconstruction resumed from a saved iterate (mrf_recon_opts.resume) equals the
    uninterrupted one bit for bit."""
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
    return dic, p, Z


def _project_ok(mrf, D, Z, A, mode="bf16"):
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    mrf.project(D, to_dev(Z), idx, rho, opts=mrf.proj_opts(mode=mode))
    check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy())


def test_bounded_wait_times_out(mrf, cfg1):
    from paper_1810_01967_gb300 import MRFError, _lib
    dic, p, Z = cfg1
    for ns in (1, 1_000_000):
        with pytest.raises(MRFError) as e:
            mrf.selftest_wait_timeout(ns)
        assert e.value.status == _lib.MRF_ETIMEOUT
    with pytest.raises(MRFError):
        mrf.selftest_wait_timeout(0)            # argument check
    # the context is intact
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    _project_ok(mrf, D, Z[:300], dic["atoms"])


def test_injected_allocation_failures(mrf, cfg1):
    from paper_1810_01967_gb300 import MRFError, _lib
    dic, p, Z = cfg1
    A = dic["atoms"]
    failed = 0
    try:
        # the dictionary build: each of its allocations refused in turn
        for k in range(64):
            mrf.debug_fail_alloc(k)
            try:
                D = mrf.build_dict_index(A, dic["params"], pack_fp8=True)
            except MRFError as e:
                assert e.status == _lib.MRF_ENOMEM
                failed += 1
                continue
            finally:
                mrf.debug_fail_alloc(-1)
            break
        assert failed >= 5, failed
        _project_ok(mrf, D, Z, A)
        # scratch growth inside a projection of more voxels than before
        D2 = mrf.build_dict_index(A, dic["params"])
        _project_ok(mrf, D2, Z[:10], A)
        mrf.debug_fail_alloc(0)
        n = Z.shape[0]
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        with pytest.raises(MRFError) as e:
            mrf.project(D2, to_dev(Z), idx, opts=mrf.proj_opts(mode="bf16"))
        assert e.value.status == _lib.MRF_ENOMEM
        mrf.debug_fail_alloc(-1)
        _project_ok(mrf, D2, Z, A)
        # a reconstruction's own buffers
        Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
        op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
        X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
        mrf.debug_fail_alloc(0)
        with pytest.raises(MRFError) as e:
            mrf.reconstruct(D2, op, to_dev(p["Y"]), X, idx,
                            opts=mrf.recon_opts(iters=2, mode="bf16"))
        assert e.value.status == _lib.MRF_ENOMEM
        mrf.debug_fail_alloc(-1)
        mrf.reconstruct(D2, op, to_dev(p["Y"]), X, idx, opts=mrf.recon_opts(iters=2, mode="bf16"))
        ref = mo.blip(p["Y"], p["masks"], A, Ny, Nx, iters=2)
        assert np.mean(idx.cpu().numpy() == ref["idx"]) >= 0.99
    finally:
        mrf.debug_fail_alloc(-1)


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_resume_equals_uninterrupted(mrf, cfg1, mode):
    dic, p, _ = cfg1
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    D = mrf.build_dict_index(dic["atoms"], dic["params"])
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    Y = to_dev(p["Y"])
    out = {}
    for split in (None, 3):
        X = torch.empty((n, L), dtype=torch.complex64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        if split is None:
            mrf.reconstruct(D, op, Y, X, idx, opts=mrf.recon_opts(iters=6, mode=mode))
        else:
            mrf.reconstruct(D, op, Y, X, idx, opts=mrf.recon_opts(iters=split, mode=mode))
            # checkpoint: the iterate and the atoms, saved to the host and restored
            Xh, ih = X.cpu(), idx.cpu()
            X2, idx2 = Xh.cuda(), ih.cuda()
            mrf.reconstruct(D, op, Y, X2, idx2,
                            opts=mrf.recon_opts(iters=6 - split, mode=mode, resume=True))
            X, idx = X2, idx2
        torch.cuda.synchronize()
        out[split] = (X.cpu().numpy(), idx.cpu().numpy())
    assert np.array_equal(out[None][1], out[3][1])
    assert np.array_equal(out[None][0], out[3][0])
