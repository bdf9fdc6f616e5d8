"""GB300 matched-filtering MRF reconstruction (BLIP / CoverBLIP, arXiv 1810.01967).

Thin Python layer over the C ABI of ``libmrf.so`` (see include/mrf.h).  Functions keep the C
names without the ``mrf_`` prefix and only marshal arguments: torch CUDA tensors become device
pointers, numpy arrays host pointers, the current torch stream the call's stream.  There is no
CPU fallback: every function raises when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import (MODES, CONES, MRFError, ProjOpts, ReconOpts, IndexOpts, Stats, Op, Tune,
                   TreeInfo)

_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


def _check(status: int) -> None:
    if status != 0:
        L = lib()
        raise MRFError(status, f"{L.mrf_status_str(status).decode()}: "
                               f"{L.mrf_last_error().decode()}")


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libmrf must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libmrf must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} to libmrf")


def _stream(stream) -> int | None:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def proj_opts(mode: str = "fp32", cone: str = "complex", topk: int = 0, certify: bool = True,
              tie_tol: float = 1e-5, cert_margin: float = 0.0, eps: float = 0.0,
              fallback_thr: float = 0.98, tree_route: float = 0.9,
              learned_edge: bool = True) -> ProjOpts:
    o = ProjOpts()
    lib().mrf_default_proj_opts(C.byref(o))
    o.mode, o.cone, o.topk, o.certify = MODES[mode], CONES[cone], topk, int(certify)
    o.tie_tol, o.cert_margin, o.eps, o.fallback_thr = tie_tol, cert_margin, eps, fallback_thr
    o.tree_route = tree_route
    o.learned_edge = int(learned_edge)
    return o


def recon_opts(iters: int = 10, mu: float = 1.0, adaptive: bool = False, zeta: float = 2.0,
               kappa: bool = False, tol: float = 0.0, max_shrink: int = 30,
               resume: bool = False, mu_history=None, shrink_history=None,
               **proj) -> ReconOpts:
    """mu_history / shrink_history: host numpy float32 / int32 arrays of at least `iters`
    entries that receive each iteration's accepted step size and shrink count (kept alive by
    the returned options)."""
    r = ReconOpts()
    lib().mrf_default_recon_opts(C.byref(r))
    r.iters, r.mu, r.adaptive, r.zeta = iters, mu, int(adaptive), zeta
    r.kappa, r.tol, r.max_shrink, r.resume = int(kappa), tol, max_shrink, int(resume)
    for name, arr, ct in (("mu_history", mu_history, C.c_float),
                          ("shrink_history", shrink_history, C.c_int32)):
        if arr is not None:
            if arr.size < iters or not arr.flags["C_CONTIGUOUS"] or arr.itemsize != 4:
                raise ValueError(f"{name} must be a contiguous 4-byte array of >= iters entries")
            setattr(r, name, arr.ctypes.data_as(C.POINTER(ct)))
    r._keep = (mu_history, shrink_history)
    r.proj = proj_opts(**proj)
    return r


def make_op(Ny: int, Nx: int, L: int, mask) -> Op:
    """mrf_op for the device mask tensor [L][Ny] uint8 (the Op keeps the tensor alive)."""
    op = Op(Ny, Nx, L, _ptr(mask))
    op._mask_ref = mask
    return op


class Dictionary:
    """An mrf_dict: the dictionary copied to the GPU plus its packed operands."""

    def __init__(self, atoms, params=None, grid_shape=None, pack_bf16: bool = True,
                 build_tree: bool = False, tree_cone: str = "complex",
                 tree_dup_tol: float = 1e-5, stream=None, pack_fp8: bool = False,
                 phase_align: bool = False, pack_bf16x3: bool = False, tree_tc: bool = False):
        import numpy as np
        d, L = atoms.shape
        o = IndexOpts()
        lib().mrf_default_index_opts(C.byref(o))
        o.pack_bf16 = int(pack_bf16)
        o.pack_fp8 = int(pack_fp8)
        o.phase_align = int(phase_align)
        o.pack_bf16x3 = int(pack_bf16x3)
        o.build_tree = int(build_tree)
        o.tree_tc = int(tree_tc)
        o.tree_cone = CONES[tree_cone]
        o.tree_dup_tol = tree_dup_tol
        P = 0 if params is None else int(params.shape[1])
        gs = None
        if grid_shape is not None:
            gs = np.ascontiguousarray(np.asarray(grid_shape, np.int32))
        h = C.c_void_p()
        self._keep = (atoms, params, gs)
        _check(lib().mrf_build_dict_index(_ptr(atoms), d, L, _ptr(params), P, _ptr(gs),
                                          0 if gs is None else len(gs), C.byref(o),
                                          C.byref(h), _stream(stream)))
        self.handle = h
        self.d, self.L, self.P = int(d), int(L), P
        self._keep = None

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().mrf_dict_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, n_max: int) -> None:
        _check(lib().mrf_dict_reserve(self.handle, n_max))

    def check(self, stream=None) -> None:
        _check(lib().mrf_dict_check(self.handle, _stream(stream)))

    def tree_info(self) -> dict:
        t = TreeInfo()
        _check(lib().mrf_tree_get_info(self.handle, C.byref(t)))
        return t.as_dict()

    def tree_export(self) -> dict:
        """Host copy of the cover tree (see mrf_tree_export)."""
        import numpy as np
        info = self.tree_info()
        d, ne = self.d, info["explicit_nodes"]
        out = {"first_level": np.empty(d, np.int32), "parent": np.empty(d, np.int32),
               "rep": np.empty(d, np.int32), "en_atom": np.empty(ne, np.int32),
               "en_level": np.empty(ne, np.int32), "en_maxdist": np.empty(ne, np.float32)}
        _check(lib().mrf_tree_export(self.handle, *[_ptr(out[k]) for k in
                                                    ("first_level", "parent", "rep", "en_atom",
                                                     "en_level", "en_maxdist")]))
        out.update(info)
        return out

    def tree_blocks(self) -> dict:
        """Blocks of the tensor-core tree search (see mrf_tree_blocks): radius [nblk] and the
        depth-first order perm [nblk * 128] (-1 past the last atom)."""
        import numpy as np
        nb = C.c_int64()
        _check(lib().mrf_tree_blocks(self.handle, C.byref(nb), None, None))
        radius = np.empty(nb.value, np.float32)
        perm = np.empty(nb.value * 128, np.int32)
        _check(lib().mrf_tree_blocks(self.handle, C.byref(nb), _ptr(radius), _ptr(perm)))
        return {"nblk": nb.value, "radius": radius, "perm": perm}

    def get_tune(self) -> dict:
        t = Tune()
        _check(lib().mrf_get_tune(self.handle, C.byref(t)))
        return t.as_dict()

    def set_tune(self, **kw) -> None:
        t = Tune()
        _check(lib().mrf_get_tune(self.handle, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(lib().mrf_set_tune(self.handle, C.byref(t)))


def build_dict_index(atoms, params=None, grid_shape=None, pack_bf16=True, build_tree=False,
                     tree_cone="complex", tree_dup_tol=1e-5, stream=None, pack_fp8=False,
                     phase_align=False, pack_bf16x3=False, tree_tc=False):
    return Dictionary(atoms, params, grid_shape, pack_bf16, build_tree, tree_cone, tree_dup_tol,
                      stream, pack_fp8, phase_align, pack_bf16x3, tree_tc)


def tree_build_host(atoms, cone: str = "complex", dup_tol: float = 1e-5) -> dict:
    """Cover tree of host atoms built on the host alone (mrf_tree_build_host)."""
    import numpy as np
    atoms = np.ascontiguousarray(atoms, dtype=np.complex64)
    d, L = atoms.shape
    out = {k: np.empty(d, np.int32) for k in ("first_level", "parent", "rep", "en_atom",
                                              "en_level")}
    out["en_maxdist"] = np.empty(d, np.float32)
    ne, sig, lev = C.c_int64(), C.c_double(), C.c_int32()
    _check(lib().mrf_tree_build_host(_ptr(atoms), d, L, CONES[cone], dup_tol,
                                     *[_ptr(out[k]) for k in ("first_level", "parent", "rep",
                                                              "en_atom", "en_level",
                                                              "en_maxdist")],
                                     C.byref(ne), C.byref(sig), C.byref(lev)))
    for k in ("en_atom", "en_level", "en_maxdist"):
        out[k] = out[k][:ne.value]
    out.update(explicit_nodes=ne.value, sigma=sig.value, levels=lev.value)
    return out


def project(D: Dictionary, Z, idx_out, rho_out=None, X_out=None, warm_idx=None, opts=None,
            stats: bool = False, stream=None):
    n = Z.shape[0]
    o = opts or proj_opts()
    st = Stats() if stats else None
    _check(lib().mrf_project(D.handle, _ptr(Z), n, C.byref(o), _ptr(warm_idx), _ptr(idx_out),
                             _ptr(rho_out), _ptr(X_out), C.byref(st) if st else None,
                             _stream(stream)))
    return st.as_dict() if st else None


def search_candidates(D: Dictionary, Z, score_out, idx_out, bound_out=None, opts=None,
                      stream=None) -> None:
    """The tensor-core kernel's K best atoms per voxel before any rescore
    (mrf_search_candidates): score_out float32 [n][K], idx_out int32 [n][K], bound_out float32
    [n] or None."""
    o = opts or proj_opts(mode="bf16")
    _check(lib().mrf_search_candidates(D.handle, _ptr(Z), Z.shape[0], C.byref(o), _ptr(score_out),
                                       _ptr(idx_out), _ptr(bound_out), _stream(stream)))


def forward(op: Op, X, Y, stream=None) -> None:
    _check(lib().mrf_forward(C.byref(op), _ptr(X), _ptr(Y), _stream(stream)))


def adjoint(op: Op, Y, AHY, stream=None) -> None:
    _check(lib().mrf_adjoint(C.byref(op), _ptr(Y), _ptr(AHY), _stream(stream)))


def gradient(D: Dictionary, op: Op, AHY, X, mu: float, Z_out, stream=None) -> None:
    _check(lib().mrf_gradient(D.handle, C.byref(op), _ptr(AHY), _ptr(X), mu, _ptr(Z_out),
                              _stream(stream)))


def ipg_step(D: Dictionary, op: Op, AHY, X, mu: float, idx_io, rho_out=None, opts=None,
             stats: bool = False, stream=None):
    o = opts or proj_opts()
    st = Stats() if stats else None
    _check(lib().mrf_ipg_step(D.handle, C.byref(op), _ptr(AHY), _ptr(X), mu, C.byref(o),
                              _ptr(idx_io), _ptr(rho_out), C.byref(st) if st else None,
                              _stream(stream)))
    return st.as_dict() if st else None


def reconstruct(D: Dictionary, op: Op, Y, X_out, idx_out, rho_out=None, params_out=None,
                opts=None, stats: bool = False, stream=None):
    r = opts or recon_opts()
    st = Stats() if stats else None
    _check(lib().mrf_reconstruct(D.handle, C.byref(op), _ptr(Y), C.byref(r), _ptr(X_out),
                                 _ptr(idx_out), _ptr(rho_out), _ptr(params_out),
                                 C.byref(st) if st else None, _stream(stream)))
    return st.as_dict() if st else None


def lut(D: Dictionary, idx, params_out, stream=None) -> None:
    _check(lib().mrf_lut(D.handle, _ptr(idx), idx.shape[0], _ptr(params_out), _stream(stream)))


class MLP:
    """Learned proposal model (mrf_mlp) bound to a Dictionary."""

    def __init__(self, D: Dictionary, grid_axes, cell_atom, hidden: int = 512, radius: int = 2,
                 residue_pool: int = 262144, seed: int = 5000, stream=None):
        import numpy as np
        o = _lib.MlpOpts()
        lib().mrf_default_mlp_opts(C.byref(o))
        o.hidden, o.radius, o.residue_pool, o.seed = hidden, radius, residue_pool, seed
        ax = np.ascontiguousarray(np.concatenate([np.asarray(a, np.float32) for a in grid_axes]))
        ca = np.ascontiguousarray(np.asarray(cell_atom, np.int32).ravel())
        h = C.c_void_p()
        _check(lib().mrf_mlp_create(D.handle, _ptr(ax), _ptr(ca), C.byref(o), C.byref(h),
                                    _stream(stream)))
        self.handle, self.dict = h, D
        self.hidden, self.L = hidden, D.L

    def close(self):
        if getattr(self, "handle", None):
            lib().mrf_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_residues(self, Z, X0, stream=None):
        _check(lib().mrf_mlp_add_residues(self.handle, _ptr(Z), _ptr(X0), Z.shape[0],
                                          _stream(stream)))

    def train(self, steps: int, batch: int = 1024, lr: float = 1e-3, snr=(30.0, 50.0),
              p_residue: float = 0.5, history: bool = False, stream=None):
        import numpy as np
        o = _lib.TrainOpts(steps, batch, lr, snr[0], snr[1], p_residue)
        h = np.zeros(steps, np.float32) if history else None
        _check(lib().mrf_mlp_train(self.handle, C.byref(o), _ptr(h), _stream(stream)))
        return h

    def params(self, values=None):
        """Get (values None) or set all parameters as one float32 host array."""
        import numpy as np
        n = C.c_int64()
        _check(lib().mrf_mlp_params(self.handle, None, 0, C.byref(n)))
        if values is None:
            out = np.empty(n.value, np.float32)
            _check(lib().mrf_mlp_params(self.handle, _ptr(out), 0, C.byref(n)))
            return out
        v = np.ascontiguousarray(values, np.float32)
        assert v.size == n.value
        _check(lib().mrf_mlp_params(self.handle, _ptr(v), 1, C.byref(n)))

    def grad(self, X, T=None, stream=None):
        """(Y, loss, grads) for device float32 inputs X [B][2L] and targets T [B][3]."""
        import numpy as np
        import torch
        for t in (X, T):
            if t is not None and t.dtype != torch.float32:
                raise TypeError("MLP.grad expects float32 tensors")
        if X.shape[1] != 2 * self.L:
            raise ValueError("X must be [B][2L]")
        B = X.shape[0]
        Y = np.empty((B, 3), np.float32)
        n = C.c_int64()
        _check(lib().mrf_mlp_params(self.handle, None, 0, C.byref(n)))
        g = np.empty(n.value, np.float32) if T is not None else None
        loss = C.c_double()
        _check(lib().mrf_mlp_grad(self.handle, _ptr(X), _ptr(T), B, _ptr(Y), _ptr(g),
                                  C.byref(loss) if T is not None else None, _stream(stream)))
        return Y, (loss.value if T is not None else None), g

    def infer(self, X, Y_out, stream=None) -> None:
        """BF16 tensor-core inference (the learned projection's path): X [B][2L] float32,
        Y_out [B][3] float32, both on the GPU."""
        if X.shape[1] != 2 * self.L or Y_out.shape[0] != X.shape[0]:
            raise ValueError("X must be [B][2L] and Y_out [B][3]")
        _check(lib().mrf_mlp_infer(self.handle, _ptr(X), X.shape[0], _ptr(Y_out),
                                   _stream(stream)))

    def canonical(self, Z, X_out, stream=None):
        import numpy as np
        v1 = np.empty(self.L, np.complex64)
        ts = np.empty(6, np.float32)
        _check(lib().mrf_mlp_canonical(self.handle, _ptr(Z), Z.shape[0], _ptr(X_out), _ptr(v1),
                                       _ptr(ts), _stream(stream)))
        return v1, ts


class Batch:
    """Slices of different sizes reconstructed together (mrf_batch)."""

    def __init__(self, D: Dictionary, ops):
        arr = (Op * len(ops))(*ops)
        h = C.c_void_p()
        _check(lib().mrf_batch_create(D.handle, len(ops), arr, C.byref(h)))
        self.handle, self.dict, self._ops = h, D, list(ops)

    def close(self):
        if getattr(self, "handle", None):
            lib().mrf_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, Ys, stream=None):
        ptrs = (C.c_void_p * len(Ys))(*[_ptr(y) for y in Ys])
        self._Ys = list(Ys)
        _check(lib().mrf_batch_load(self.handle, ptrs, _stream(stream)))

    def run(self, iters: int, mu: float = 1.0, opts=None, use_graph: bool = False, stream=None):
        o = opts or proj_opts()
        _check(lib().mrf_batch_run(self.handle, iters, mu, C.byref(o), int(use_graph),
                                   _stream(stream)))

    def slice(self, s: int) -> dict:
        X, idx, rho = C.c_void_p(), C.c_void_p(), C.c_void_p()
        n, off = C.c_int64(), C.c_int64()
        _check(lib().mrf_batch_slice(self.handle, s, C.byref(X), C.byref(idx), C.byref(rho),
                                     C.byref(n), C.byref(off)))
        return {"X": X.value, "idx": idx.value, "rho": rho.value, "n": n.value,
                "offset": off.value}

    def views(self, s: int) -> dict:
        """Zero-copy torch views of slice s's rows: X complex64 [n, L], idx int32 [n],
        rho complex64 [n] (valid while the batch lives)."""
        import torch
        v = self.slice(s)
        n, L = v["n"], self._ops[0].L

        class _Dev:
            def __init__(self, ptr, shape, typestr):
                self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                                 "typestr": typestr, "version": 2}

        X = torch.as_tensor(_Dev(v["X"], (n, 2 * L), "<f4"), device="cuda")
        rho = torch.as_tensor(_Dev(v["rho"], (n, 2), "<f4"), device="cuda")
        idx = torch.as_tensor(_Dev(v["idx"], (n,), "<i4"), device="cuda")
        return {"X": X.view(torch.complex64), "idx": idx, "rho": rho.view(torch.complex64)[:, 0],
                "n": n, "offset": v["offset"]}

    def lut(self, params_out, stream=None):
        _check(lib().mrf_batch_lut(self.handle, _ptr(params_out), _stream(stream)))


def svd_basis(D: Dictionary, s: int, stream=None):
    """(V [L, s] complex64 on the GPU, eigenvalues [s] float64) of sum_j D_j D_j^H."""
    import numpy as np
    import torch
    V = torch.empty((D.L, s), dtype=torch.complex64, device="cuda")
    eig = np.empty(s, np.float64)
    _check(lib().mrf_svd_basis(D.handle, s, _ptr(V), eig.ctypes.data, _stream(stream)))
    return V, eig


class SvdOp:
    """Temporal compression with basis V [L, s] (mrf_svd_op); `op` adds the compressed normal
    operator of that sampling pattern."""

    def __init__(self, V, op: Op | None = None, stream=None):
        L, s = V.shape
        h = C.c_void_p()
        _check(lib().mrf_svd_op_create(None if op is None else C.byref(op), _ptr(V), L, s,
                                       C.byref(h), _stream(stream)))
        self.handle, self.L, self.s, self._op, self._V = h, L, s, op, V

    def close(self):
        if getattr(self, "handle", None):
            lib().mrf_svd_op_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compress(self, X, Xc, stream=None):
        _check(lib().mrf_svd_compress(self.handle, _ptr(X), X.shape[0], _ptr(Xc), _stream(stream)))

    def expand(self, Xc, X, stream=None):
        _check(lib().mrf_svd_expand(self.handle, _ptr(Xc), Xc.shape[0], _ptr(X), _stream(stream)))

    def ipg_step(self, Dc: Dictionary, AHYc, Xc, mu: float, idx_io, rho_out=None, opts=None,
                 stream=None):
        o = opts or proj_opts()
        _check(lib().mrf_svd_ipg_step(Dc.handle, self.handle, _ptr(AHYc), _ptr(Xc), mu, C.byref(o),
                                      _ptr(idx_io), _ptr(rho_out), _stream(stream)))

    def gradient(self, Dc: Dictionary, AHYc, Xc, mu: float, Zc_out, stream=None):
        _check(lib().mrf_svd_gradient(Dc.handle, self.handle, _ptr(AHYc), _ptr(Xc), mu,
                                      _ptr(Zc_out), _stream(stream)))

    def reconstruct(self, Dc: Dictionary, Y, iters: int, Xc_out, idx_out, X_out=None,
                    rho_out=None, params_out=None, mu: float = 1.0, opts=None, stream=None,
                    adaptive: bool = False, zeta: float = 2.0, kappa: bool = False,
                    max_shrink: int = 30, mu_history=None, shrink_history=None):
        """Compressed BLIP (mrf_svd_reconstruct); `opts` are the projection options."""
        r = recon_opts(iters=iters, mu=mu, adaptive=adaptive, zeta=zeta, kappa=kappa,
                       max_shrink=max_shrink, mu_history=mu_history,
                       shrink_history=shrink_history)
        if opts is not None:
            r.proj = opts
        _check(lib().mrf_svd_reconstruct(Dc.handle, self.handle, _ptr(Y), C.byref(r),
                                         _ptr(Xc_out), _ptr(X_out), _ptr(idx_out), _ptr(rho_out),
                                         _ptr(params_out), _stream(stream)))


def attach_mlp(D: Dictionary, mlp) -> None:
    _check(lib().mrf_dict_attach_mlp(D.handle, None if mlp is None else mlp.handle))
    D._mlp = mlp


PROFILE_STAGES = ["gradient", "pack_queries", "search_tc", "search_fp32", "merge", "fallback",
                  "lut", "search_proposal"]


def profile_enable(on: bool = True) -> None:
    _check(lib().mrf_profile_enable(int(on)))


def profile_read() -> dict:
    """{stage: (milliseconds, launches)} accumulated since the last read (synchronises)."""
    n = len(PROFILE_STAGES)
    ms = (C.c_double * n)()
    ln = (C.c_int64 * n)()
    _check(lib().mrf_profile_read(ms, ln, n))
    return {name: (ms[i], ln[i]) for i, name in enumerate(PROFILE_STAGES)}


def debug_fail_alloc(k: int) -> None:
    """Fault injection: the library's device allocations succeed k more times, then one fails
    with MRF_ENOMEM (k < 0: off)."""
    lib().mrf_debug_fail_alloc(k)


def selftest_wait_timeout(timeout_ns: int = 1_000_000, stream=None) -> None:
    """Runs the bounded-wait self-test; raises MRFError (status MRF_ETIMEOUT) as it should."""
    _check(lib().mrf_selftest_wait_timeout(timeout_ns, _stream(stream)))
