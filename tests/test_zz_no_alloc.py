"""The projection entry point that allocates no device memory (mrf_project_fp32_static).

It serves callers that may not allocate once running (their device memory belongs to their own
pool, or their pipeline forbids cudaMalloc after start-up).  Checked through the C ABI against
the float64 oracle's exact projection (both cones) and against mrf_project's FP32 mode on the
same inputs, twice in a row (the shared static scratch keeps the previous call's contents); a
call made while every library allocation is refused, and with the device's free memory
unchanged across it, shows that it allocates nothing; sizes past the static scratch are
rejected.  This file is collected last on purpose."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from gpu_util import check_projection

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    b.build()
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    Z1 = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]).astype(np.complex64)[:1000]
    g = np.random.Generator(np.random.PCG64(8))
    Z2 = (Z1[::-1] * np.complex64(0.3 + 0.7j)
          + (0.01 * (g.standard_normal(Z1.shape) + 1j * g.standard_normal(Z1.shape)))
          .astype(np.complex64)).astype(np.complex64)
    return mrf, dic["atoms"], [Z1, np.ascontiguousarray(Z2)]


def _static(mrf, Ad, d, L, Zd, cone, stream):
    n = Zd.shape[0]
    i_s = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    r_s = torch.empty(n, dtype=torch.complex64, device="cuda")
    X_s = torch.empty_like(Zd)
    st = mrf.lib().mrf_project_fp32_static(Ad.data_ptr(), d, L, Zd.data_ptr(), n, cone,
                                           i_s.data_ptr(), r_s.data_ptr(), X_s.data_ptr(), stream)
    assert st == 0, mrf.lib().mrf_last_error()
    torch.cuda.synchronize()
    return i_s, r_s, X_s


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_static_scratch_projection_matches_oracle_and_mrf_project(setup, cone):
    mrf, atoms, Zs = setup
    d, L = atoms.shape
    c = {"complex": 0, "real_pos": 1}[cone]
    Ad = torch.from_numpy(atoms).cuda()
    D = mrf.build_dict_index(atoms)
    stream = torch.cuda.current_stream().cuda_stream
    for Z in Zs:                                    # two calls in a row on the shared scratch
        n = Z.shape[0]
        Zd = torch.from_numpy(Z).cuda()
        i_s, r_s, X_s = _static(mrf, Ad, d, L, Zd, c, stream)
        gi, gr, gx = i_s.cpu().numpy(), r_s.cpu().numpy(), X_s.cpu().numpy()
        # the float64 oracle: indices exact except near-ties, rho and X within 1e-4
        check_projection(Z, atoms, gi, gr, cone=cone, g_X=gx)
        # the existing entry point's FP32 mode on the same inputs
        i_ref = torch.empty(n, dtype=torch.int32, device="cuda")
        r_ref = torch.empty(n, dtype=torch.complex64, device="cuda")
        X_ref = torch.empty_like(Zd)
        mrf.project(D, Zd, i_ref, r_ref, X_ref, opts=mrf.proj_opts(mode="fp32", cone=cone))
        torch.cuda.synchronize()
        assert torch.equal(i_s, i_ref)
        rr = r_ref.cpu().numpy()
        assert np.max(np.abs(gr - rr) / np.maximum(np.abs(rr), 1e-30)) <= 1e-4
        xr = X_ref.cpu().numpy()
        assert np.linalg.norm(gx - xr) <= 1e-4 * np.linalg.norm(xr)
    D.close()


def test_static_scratch_allocates_nothing(setup):
    mrf, atoms, Zs = setup
    d, L = atoms.shape
    Ad = torch.from_numpy(atoms).cuda()
    Zd = torch.from_numpy(Zs[0]).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    ref = _static(mrf, Ad, d, L, Zd, 0, stream)          # loads the kernels, looks up the array
    free0, _ = torch.cuda.mem_get_info()
    try:
        mrf.debug_fail_alloc(0)                 # the library's next device allocation fails
        got = _static(mrf, Ad, d, L, Zd, 0, stream)
        mrf.debug_fail_alloc(0)
        got2 = _static(mrf, Ad, d, L, Zd, 0, stream)
    finally:
        mrf.debug_fail_alloc(-1)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    for a, b in zip(got, got2):
        assert torch.equal(a, b)


def test_static_scratch_rejects_sizes_past_its_limit(setup):
    mrf, atoms, _ = setup
    d, L = atoms.shape
    L_ = mrf.lib()
    Ad = torch.from_numpy(atoms).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    big = torch.zeros((4097, L), dtype=torch.complex64, device="cuda")
    ib = torch.empty(4097, dtype=torch.int32, device="cuda")
    st = L_.mrf_project_fp32_static(Ad.data_ptr(), d, L, big.data_ptr(), 4097, 0,
                                    ib.data_ptr(), None, None, stream)
    assert st == 1 and b"4096" in L_.mrf_last_error()
