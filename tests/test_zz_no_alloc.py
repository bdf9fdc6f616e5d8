"""The projection entry point that allocates no device memory (mrf_project_fp32_static).

It serves callers that may not allocate once running (their device memory belongs to their own
pool, or their pipeline forbids cudaMalloc after start-up).  Checked through the C ABI against
mrf_project's FP32 mode on the same inputs, twice in a row (the shared static scratch keeps the
previous call's contents), plus the size limit.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_scratch_projection_matches_mrf_project():
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300 import build as b
    b.build()
    L_ = mrf.lib()
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    atoms = dic["atoms"]
    d, L = atoms.shape
    Z1 = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]).astype(np.complex64)[:1000]
    g = np.random.Generator(np.random.PCG64(8))
    Z2 = (Z1[::-1] * np.complex64(0.3 + 0.7j)
          + (0.01 * (g.standard_normal(Z1.shape) + 1j * g.standard_normal(Z1.shape)))
          .astype(np.complex64)).astype(np.complex64)
    Ad = torch.from_numpy(atoms).cuda()
    D = mrf.build_dict_index(atoms)
    stream = torch.cuda.current_stream().cuda_stream
    for Z in (Z1, np.ascontiguousarray(Z2)):
        n = Z.shape[0]
        Zd = torch.from_numpy(Z).cuda()
        i_ref = torch.empty(n, dtype=torch.int32, device="cuda")
        r_ref = torch.empty(n, dtype=torch.complex64, device="cuda")
        X_ref = torch.empty_like(Zd)
        mrf.project(D, Zd, i_ref, r_ref, X_ref, opts=mrf.proj_opts(mode="fp32"))
        i_s = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        r_s = torch.empty(n, dtype=torch.complex64, device="cuda")
        X_s = torch.empty_like(Zd)
        st = L_.mrf_project_fp32_static(Ad.data_ptr(), d, L, Zd.data_ptr(), n, 0,
                                        i_s.data_ptr(), r_s.data_ptr(), X_s.data_ptr(), stream)
        assert st == 0, L_.mrf_last_error()
        torch.cuda.synchronize()
        assert torch.equal(i_s, i_ref)
        rr, rs = r_ref.cpu().numpy(), r_s.cpu().numpy()
        assert np.max(np.abs(rs - rr) / np.maximum(np.abs(rr), 1e-30)) <= 1e-4
        xr, xs = X_ref.cpu().numpy(), X_s.cpu().numpy()
        assert np.linalg.norm(xs - xr) <= 1e-4 * np.linalg.norm(xr)
    # sizes beyond the static scratch are rejected before any launch
    big = torch.zeros((4097, L), dtype=torch.complex64, device="cuda")
    ib = torch.empty(4097, dtype=torch.int32, device="cuda")
    st = L_.mrf_project_fp32_static(Ad.data_ptr(), d, L, big.data_ptr(), 4097, 0,
                                    ib.data_ptr(), None, None, stream)
    assert st == 1 and b"4096" in L_.mrf_last_error()
