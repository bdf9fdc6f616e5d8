"""Host-only checks of the C ABI: the library builds and loads, exports every function that
include/mrf.h declares, and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1810_01967_gb300 import build as b
    b.build()
    import paper_1810_01967_gb300 as mrf
    return mrf.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrf_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_header(L):
    from paper_1810_01967_gb300._lib import SIGNATURES
    assert set(declared_functions()) == set(SIGNATURES)


def test_struct_sizes_match_header():
    from paper_1810_01967_gb300._lib import ProjOpts, ReconOpts, Stats, Op, IndexOpts
    assert C.sizeof(IndexOpts) == 32
    assert C.sizeof(ProjOpts) == 64
    assert C.sizeof(Stats) == 64
    assert C.sizeof(Op) == 24
    assert C.sizeof(ReconOpts) == 48 + 64


def test_host_argument_errors(L):
    import paper_1810_01967_gb300 as mrf
    from paper_1810_01967_gb300._lib import MRF_EINVAL
    h = C.c_void_p()
    assert L.mrf_build_dict_index(None, 10, 4, None, 0, None, 0, None, C.byref(h), None) \
        == MRF_EINVAL
    assert b"atoms" in L.mrf_last_error()
    assert L.mrf_project(None, None, 5, None, None, None, None, None, None, None) == MRF_EINVAL
    assert L.mrf_forward(None, None, None, None) == MRF_EINVAL
    op = mrf.Op(0, 4, 4, 1)
    assert L.mrf_adjoint(C.byref(op), 1, 1, None) == MRF_EINVAL
    assert L.mrf_dict_info(None, None, None, None) == MRF_EINVAL
    assert L.mrf_status_str(MRF_EINVAL) == b"MRF_EINVAL"
    assert L.mrf_batch_create(None, 2, None, C.byref(h)) == MRF_EINVAL
    assert L.mrf_batch_run(None, 1, 1.0, None, 0, None) == MRF_EINVAL
    assert L.mrf_batch_slice(None, 0, None, None, None, None, None) == MRF_EINVAL
    L.mrf_batch_free(None)
    o = mrf.proj_opts()
    assert o.topk == 0 and o.mode == 0 and abs(o.tie_tol - 1e-5) < 1e-12
    # the tensor-core tree search's index options are checked before any device work
    import numpy as np
    from paper_1810_01967_gb300._lib import IndexOpts
    atoms = np.ones((4, 8), np.complex64)
    io = IndexOpts()
    L.mrf_default_index_opts(C.byref(io))
    io.tree_tc = 1
    assert L.mrf_build_dict_index(atoms.ctypes.data, 4, 8, None, 0, None, 0, C.byref(io),
                                  C.byref(h), None) == MRF_EINVAL
    assert b"build_tree" in L.mrf_last_error()
    io.build_tree, io.pack_bf16, io.pack_bf16x3 = 1, 0, 0
    assert L.mrf_build_dict_index(atoms.ctypes.data, 4, 8, None, 0, None, 0, C.byref(io),
                                  C.byref(h), None) == MRF_EINVAL
    assert b"pack_bf16" in L.mrf_last_error()
    assert L.mrf_tree_blocks(None, None, None, None) == MRF_EINVAL
