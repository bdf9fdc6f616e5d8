"""ctypes binding of libmrf.so (include/mrf.h): argument marshalling only.

Every computation happens inside the library's CUDA kernels.  Tensors are passed as raw
pointers (``tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream`` handles.  The
library is required: importing this module without a built ``_build/libmrf.so`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmrf.so")

MRF_OK, MRF_EINVAL, MRF_ENOMEM, MRF_ECUDA, MRF_ENONFINITE, MRF_ETIMEOUT, \
    MRF_EUNSUPPORTED, MRF_EINTERNAL = range(8)
MODES = {"fp32": 0, "bf16": 1, "fp8": 2, "covertree": 3, "learned": 4, "bf16x3": 5,
         "tree_tc": 6}
CONES = {"complex": 0, "real_pos": 1}


class IndexOpts(C.Structure):
    _fields_ = [("pack_bf16", C.c_int32), ("pack_fp8", C.c_int32), ("build_tree", C.c_int32),
                ("tree_cone", C.c_int32), ("tree_dup_tol", C.c_float),
                ("phase_align", C.c_int32), ("pack_bf16x3", C.c_int32),
                ("tree_tc", C.c_int32)]


class TreeInfo(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("explicit_nodes", C.c_int64), ("levels", C.c_int32),
                ("metric", C.c_int32), ("sigma", C.c_double), ("build_ms", C.c_double),
                ("device_bytes", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProjOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("cone", C.c_int32), ("topk", C.c_int32),
                ("certify", C.c_int32), ("tie_tol", C.c_float), ("cert_margin", C.c_float),
                ("eps", C.c_float), ("fallback_thr", C.c_float), ("tree_route", C.c_float),
                ("learned_edge", C.c_int32), ("reserved", C.c_int32 * 6)]


class Stats(C.Structure):
    _fields_ = [("n_voxels", C.c_int64), ("n_zero", C.c_int64), ("n_tie_rescored", C.c_int64),
                ("n_tie_overflow", C.c_int64), ("n_uncertified", C.c_int64),
                ("n_fallback", C.c_int64), ("n_dist_evals", C.c_int64),
                ("device_error", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Op(C.Structure):
    _fields_ = [("Ny", C.c_int32), ("Nx", C.c_int32), ("L", C.c_int32), ("mask", C.c_void_p)]


class ReconOpts(C.Structure):
    _fields_ = [("iters", C.c_int32), ("mu", C.c_float), ("adaptive", C.c_int32),
                ("zeta", C.c_float), ("kappa", C.c_int32), ("tol", C.c_float),
                ("max_shrink", C.c_int32), ("resume", C.c_int32),
                ("mu_history", C.POINTER(C.c_float)), ("shrink_history", C.POINTER(C.c_int32)),
                ("proj", ProjOpts)]


class Tune(C.Structure):
    _fields_ = [("bf16_cluster", C.c_int32), ("bf16_live_tiles", C.c_int32),
                ("bf16_splits", C.c_int32), ("fp32_splits", C.c_int32),
                ("last_bf16_ctas", C.c_int32), ("last_bf16_cluster", C.c_int32),
                ("last_bf16_splits", C.c_int32), ("last_fp32_splits", C.c_int32),
                ("tree_list_cap", C.c_int32), ("bf16_pair", C.c_int32),
                ("tree_order", C.c_int32), ("tree_tc_group", C.c_int32),
                ("tree_tc_chunks", C.c_int32), ("tree_tc_super", C.c_int32),
                ("reserved", C.c_int32 * 2)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class MlpOpts(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("radius", C.c_int32), ("residue_pool", C.c_int64),
                ("seed", C.c_uint64), ("reserved", C.c_int32 * 8)]


class TrainOpts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("snr_lo", C.c_float), ("snr_hi", C.c_float), ("p_residue", C.c_float),
                ("reserved", C.c_int32 * 6)]


SIGNATURES = {
    "mrf_default_index_opts": (None, [C.POINTER(IndexOpts)]),
    "mrf_default_proj_opts": (None, [C.POINTER(ProjOpts)]),
    "mrf_default_recon_opts": (None, [C.POINTER(ReconOpts)]),
    "mrf_build_dict_index": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int32,
                                       C.c_void_p, C.c_int32, C.POINTER(IndexOpts),
                                       C.POINTER(C.c_void_p), C.c_void_p]),
    "mrf_dict_free": (None, [C.c_void_p]),
    "mrf_dict_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)]),
    "mrf_dict_reserve": (C.c_int, [C.c_void_p, C.c_int64]),
    "mrf_tree_build_host": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_float,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "mrf_tree_get_info": (C.c_int, [C.c_void_p, C.POINTER(TreeInfo)]),
    "mrf_tree_blocks": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p]),
    "mrf_tree_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "mrf_dict_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mrf_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(ProjOpts),
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(Stats), C.c_void_p]),
    "mrf_search_candidates": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(ProjOpts),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_forward": (C.c_int, [C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_adjoint": (C.c_int, [C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_gradient": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_float,
                               C.c_void_p, C.c_void_p]),
    "mrf_ipg_step": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_float,
                               C.POINTER(ProjOpts), C.c_void_p, C.c_void_p, C.POINTER(Stats),
                               C.c_void_p]),
    "mrf_reconstruct": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.POINTER(ReconOpts),
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(Stats), C.c_void_p]),
    "mrf_lut": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mrf_project_fp32_static": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                          C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    "mrf_get_tune": (C.c_int, [C.c_void_p, C.POINTER(Tune)]),
    "mrf_set_tune": (C.c_int, [C.c_void_p, C.POINTER(Tune)]),
    "mrf_profile_enable": (C.c_int, [C.c_int32]),
    "mrf_profile_read": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "mrf_default_mlp_opts": (None, [C.POINTER(MlpOpts)]),
    "mrf_mlp_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(MlpOpts),
                                 C.POINTER(C.c_void_p), C.c_void_p]),
    "mrf_mlp_free": (None, [C.c_void_p]),
    "mrf_mlp_add_residues": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                       C.c_void_p]),
    "mrf_mlp_train": (C.c_int, [C.c_void_p, C.POINTER(TrainOpts), C.c_void_p, C.c_void_p]),
    "mrf_mlp_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "mrf_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_mlp_canonical": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "mrf_mlp_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mrf_dict_attach_mlp": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mrf_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "mrf_batch_free": (None, [C.c_void_p]),
    "mrf_batch_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_batch_run": (C.c_int, [C.c_void_p, C.c_int32, C.c_float, C.POINTER(ProjOpts), C.c_int32,
                                C.c_void_p]),
    "mrf_batch_slice": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mrf_batch_lut": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_svd_basis": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_svd_op_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_void_p), C.c_void_p]),
    "mrf_svd_op_free": (None, [C.c_void_p]),
    "mrf_svd_compress": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mrf_svd_expand": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mrf_svd_ipg_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                   C.POINTER(ProjOpts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrf_svd_reconstruct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(ReconOpts),
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "mrf_svd_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                   C.c_void_p, C.c_void_p]),
    "mrf_debug_fail_alloc": (None, [C.c_int32]),
    "mrf_selftest_wait_timeout": (C.c_int, [C.c_int64, C.c_void_p]),
    "mrf_status_str": (C.c_char_p, [C.c_int]),
    "mrf_last_error": (C.c_char_p, []),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmrf.so not built ({path}); run "
                          "`python -m paper_1810_01967_gb300.build` (needs nvcc)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


class MRFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status
