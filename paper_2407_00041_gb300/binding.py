"""ctypes binding of the C ABI in ``include/dd_wilson.h``.

Argument marshalling only: every computation runs in ``libddwilson.so``.
PyTorch supplies device memory and streams.  The functions keep the C names
(``dd_apply``, ``dd_solve`` ...); the small classes below own the handles.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

DD_OK = 0
DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA, DD_ERR_SINGULAR = -1, -2, -3, -4
DD_ERR_NOT_CONVERGED, DD_ERR_TIMEOUT, DD_ERR_UNSUPPORTED = -5, -6, -7
DD_PREC_F64, DD_PREC_F32, DD_PREC_F16 = 1, 2, 4
DD_PREC_DF64 = 8  # FP64-accurate arithmetic in FP32 pairs
DD_OP_D, DD_OP_DH, DD_OP_DHAT, DD_OP_DHAT_H, DD_OP_SC = 0, 1, 2, 3, 4
DD_LAYOUT_CANONICAL, DD_LAYOUT_CANONICAL_HOST, DD_LAYOUT_NATIVE, DD_LAYOUT_NATIVE_PAIRED = 0, 1, 2, 3
DD_LAYOUT_CANONICAL_C64, DD_LAYOUT_CANONICAL_HOST_C64 = 4, 5  # complex64 canonical fields

DD_PRECOND_NONE, DD_PRECOND_NORMAL, DD_PRECOND_CGNR, DD_PRECOND_SAP, DD_PRECOND_AMG = 0, 1, 2, 3, 4
DD_PRECOND_CGNR16 = 5  # CGNR with FP16-stored CG vectors (inner_prec F16)
PREC = {"f64": DD_PREC_F64, "f32": DD_PREC_F32, "f16": DD_PREC_F16, "df64": DD_PREC_DF64}
OPS = {"D": DD_OP_D, "DH": DD_OP_DH, "DHAT": DD_OP_DHAT, "DHAT_H": DD_OP_DHAT_H, "SC": DD_OP_SC}


class DDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.dd_error_string(status).decode()} "
                         f"({_lib.dd_last_error_detail().decode()})")


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("inner_prec", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("even_odd", ctypes.c_int), ("verbose", ctypes.c_int), ("precond", ctypes.c_int),
                ("gs_passes", ctypes.c_int), ("rhs_batch", ctypes.c_int), ("precond_iters", ctypes.c_int),
                ("sap_block", ctypes.c_int * 4), ("sap_cycles", ctypes.c_int), ("sap_mr_steps", ctypes.c_int),
                ("amg", ctypes.c_void_p), ("refine_prec", ctypes.c_int)]


class AmgParams(ctypes.Structure):
    _fields_ = [("aggregate", ctypes.c_int * 4), ("n_tv", ctypes.c_int), ("setup_iters", ctypes.c_int),
                ("init_sap_iters", ctypes.c_int), ("sap_block", ctypes.c_int * 4), ("sap_cycles", ctypes.c_int),
                ("sap_mr_steps", ctypes.c_int), ("coarse_tol", ctypes.c_double), ("coarse_restart", ctypes.c_int),
                ("coarse_max_restarts", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("inner_iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("applies_inner", ctypes.c_int), ("applies_fp64", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes)
_P, _I, _D, _L, _U, _S = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint,
                          ctypes.c_size_t)
SIGNATURES = {
    "dd_error_string": (ctypes.c_char_p, [_I]),
    "dd_last_error_detail": (ctypes.c_char_p, []),
    "dd_version": (_I, []),
    "dd_lattice_create": (_I, [_P, _I, _P]),
    "dd_lattice_destroy": (_I, [_P]),
    "dd_lattice_volume": (_L, [_P]),
    "dd_gauge_create": (_I, [_P, _P, _I, _U, _P]),
    "dd_gauge_generate": (_I, [_P, ctypes.c_uint64, _D, _U, _P]),
    "dd_gauge_destroy": (_I, [_P]),
    "dd_gauge_download": (_I, [_P, _P, _I]),
    "dd_clover_create": (_I, [_P, _D, _D, _U, _P]),
    "dd_clover_destroy": (_I, [_P]),
    "dd_clover_download": (_I, [_P, _P]),
    "dd_field_bytes": (_S, [_P, _I, _I, _I]),
    "dd_pack": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "dd_unpack": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "dd_pack_paired": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "dd_unpack_paired": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "dd_apply": (_I, [_P, _I, _I, _P, _P, _I, _I, _P]),
    "dd_solve_params_default": (None, [_P]),
    "dd_solve": (_I, [_P, _P, _P, _P, _I, _I, _P, _P]),
    "dd_force": (_I, [_P, _I, _P, _P, _I, _I, _P, _P, _P]),
    "dd_sap": (_I, [_P, _I, _P, _I, _I, _P, _P, _I, _I, _P]),
    "dd_amg_params_default": (None, [_P]),
    "dd_amg_create": (_I, [_P, _I, _P, _P, _P]),
    "dd_amg_destroy": (_I, [_P]),
    "dd_amg_info": (_I, [_P, _P, _P, _P, _P]),
    "dd_amg_coarse_download": (_I, [_P, _P]),
    "dd_amg_apply": (_I, [_P, _P, _P, _I, _I, _P]),
    "dd_batch_create": (_I, [_P, _I, _I, _P, _P]),
    "dd_batch_destroy": (_I, [_P]),
    "dd_batch_set_layout": (_I, [_P, _I]),
    "dd_apply_batched": (_I, [_P, _P, _P, _P]),
    "dd_batch_tune": (_I, [_P, _P, _P, _P, _P]),
    "dd_apply_batched_graph": (_I, [_P, _P, _P, _P]),
    "dd_dot": (_I, [_P, _P, _L, _I, _P, _P]),
    "dd_probe_flops": (_I, [_I, _P, _P]),
    "dd_device_status": (_I, [_P]),
    "dd_gauge_stored_rows": (_I, [_P, _I]),
    "dd_gauge_link_reals": (_I, [_P, _I]),
    "dd_gauge_compress_links": (_I, [_P, _I, _I]),
    "dd_dot_noalloc": (_I, [_P, _P, _L, _I, _P, _P]),
    "dd_decomp_create": (_I, [_P, _P, _P]),
    "dd_decomp_destroy": (_I, [_P]),
    "dd_decomp_info": (_I, [_P, _I, _P, _P, _P, _P]),
    "dd_decomp_scatter": (_I, [_P, _I, _I, _P, _I, _P]),
    "dd_decomp_gather": (_I, [_P, _I, _I, _P, _I, _P]),
    "dd_decomp_apply": (_I, [_P, _I, _I, _I, _P]),
    "dd_decomp_dot": (_I, [_P, _I, _I, _I, _P, _P]),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load ``libddwilson.so`` (building it in-tree first when it is missing or
    stale).  Raises when the library cannot be built or loaded: there is no
    CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status, where):
    if status != DD_OK:
        raise DDError(status, where)
    return status


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _ptr(t):
    return t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data


class Lattice:
    def __init__(self, dims, t_bc=-1):
        lib = load()
        self.dims = tuple(int(d) for d in dims)
        arr = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        check(lib.dd_lattice_create(arr, t_bc, ctypes.byref(h)), "dd_lattice_create")
        self.h, self.t_bc = h, t_bc
        self.V = int(lib.dd_lattice_volume(h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dd_lattice_destroy(self.h)
            self.h = None


class Gauge:
    """Links U as complex128 [V, 4, 3, 3] (numpy on the host or a torch tensor)."""

    def __init__(self, lattice, U, precisions=DD_PREC_F64 | DD_PREC_F32 | DD_PREC_F16):
        lib = load()
        self.lattice = lattice
        loc = 1 if (hasattr(U, "is_cuda") and U.is_cuda) else 0
        if hasattr(U, "contiguous"):
            U = U.contiguous()
        else:
            import numpy as np
            U = np.ascontiguousarray(U, dtype=np.complex128)
        h = ctypes.c_void_p()
        check(lib.dd_gauge_create(lattice.h, _ptr(U), loc, precisions, ctypes.byref(h)), "dd_gauge_create")
        self.h = h

    @classmethod
    def generate(cls, lattice, seed=20240700, eps=0.3, precisions=DD_PREC_F64 | DD_PREC_F32 | DD_PREC_F16):
        """Links exp(i eps H) drawn on the device by ``dd_gauge_generate``."""
        lib = load()
        self = cls.__new__(cls)
        self.lattice = lattice
        h = ctypes.c_void_p()
        check(lib.dd_gauge_generate(lattice.h, int(seed), float(eps), precisions, ctypes.byref(h)),
              "dd_gauge_generate")
        self.h = h
        return self

    def download(self, out=None):
        """The FP64 links as complex128 [V, 4, 3, 3] (numpy, or into a torch tensor on the device)."""
        import numpy as np
        if out is None:
            out = np.empty((self.lattice.V, 4, 3, 3), dtype=np.complex128)
            check(_lib.dd_gauge_download(self.h, out.ctypes.data, 0), "dd_gauge_download")
        else:
            check(_lib.dd_gauge_download(self.h, _ptr(out), 1 if out.is_cuda else 0), "dd_gauge_download")
        return out

    def link_reals(self, prec=DD_PREC_F32):
        """Reals per link read by single-RHS applies in `prec` (18, 12 or 8)."""
        r = _lib.dd_gauge_link_reals(self.h, prec)
        check(min(r, 0), "dd_gauge_link_reals")
        return r

    def compress_links(self, reals, prec=DD_PREC_F32):
        """Compressed link copy of `prec` with 18 (none), 12 or (FP32) 8 reals per link."""
        check(_lib.dd_gauge_compress_links(self.h, prec, reals), "dd_gauge_compress_links")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dd_gauge_destroy(self.h)
            self.h = None


class Operator:
    """Wilson-clover operator handle (dd_clover)."""

    def __init__(self, gauge, m0, csw, precisions=DD_PREC_F64 | DD_PREC_F32 | DD_PREC_F16):
        lib = load()
        self.gauge, self.lattice = gauge, gauge.lattice
        self.m0, self.csw = m0, csw
        h = ctypes.c_void_p()
        check(lib.dd_clover_create(gauge.h, m0, csw, precisions, ctypes.byref(h)), "dd_clover_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dd_clover_destroy(self.h)
            self.h = None

    # -- fields
    def field_bytes(self, prec, subset=0, nrhs=1):
        return int(_lib.dd_field_bytes(self.h, prec, subset, nrhs))

    def pack(self, prec, subset, canon, native, nrhs, stream=None):
        check(_lib.dd_pack(self.h, prec, subset, _ptr(canon), _ptr(native), nrhs, _stream(stream)), "dd_pack")

    def unpack(self, prec, subset, native, canon, nrhs, stream=None):
        check(_lib.dd_unpack(self.h, prec, subset, _ptr(native), _ptr(canon), nrhs, _stream(stream)), "dd_unpack")

    def pack_paired(self, prec, subset, canon, paired, nrhs, stream=None):
        check(_lib.dd_pack_paired(self.h, prec, subset, _ptr(canon), _ptr(paired), nrhs, _stream(stream)),
              "dd_pack_paired")

    def unpack_paired(self, prec, subset, paired, canon, nrhs, stream=None):
        check(_lib.dd_unpack_paired(self.h, prec, subset, _ptr(paired), _ptr(canon), nrhs, _stream(stream)),
              "dd_unpack_paired")

    # -- operators
    def apply(self, which, prec, inp, out, nrhs, layout=DD_LAYOUT_CANONICAL, stream=None):
        s = 0 if layout == DD_LAYOUT_CANONICAL_HOST and stream is None else _stream(stream)
        check(_lib.dd_apply(self.h, which, prec, _ptr(inp), _ptr(out), nrhs, layout, s), "dd_apply")

    def solve(self, b, x, nrhs, layout=DD_LAYOUT_CANONICAL, stream=None, **kw):
        p = SolveParams()
        _lib.dd_solve_params_default(ctypes.byref(p))
        for k, v in kw.items():
            if k == "sap_block":
                v = (ctypes.c_int * 4)(*v)
            if k == "amg":
                v = v.h if isinstance(v, Amg) else v
            setattr(p, k, v)
        st = Stats()
        s = 0 if layout == DD_LAYOUT_CANONICAL_HOST and stream is None else _stream(stream)
        status = _lib.dd_solve(self.h, ctypes.byref(p), _ptr(b), _ptr(x), nrhs, layout, s, ctypes.byref(st))
        if status not in (DD_OK, DD_ERR_NOT_CONVERGED):
            check(status, "dd_solve")
        return status, st.as_dict()

    def sap(self, prec, block, cycles, mr_steps, v, z, nrhs, layout=DD_LAYOUT_CANONICAL, stream=None):
        blk = (ctypes.c_int * 4)(*block)
        s = 0 if layout == DD_LAYOUT_CANONICAL_HOST and stream is None else _stream(stream)
        check(_lib.dd_sap(self.h, prec, blk, cycles, mr_steps, _ptr(v), _ptr(z), nrhs, layout, s), "dd_sap")

    def force(self, prec, phi, psi, nrhs, with_clover, G=None, F=None, stream=None):
        check(_lib.dd_force(self.h, prec, _ptr(phi), _ptr(psi), nrhs, int(with_clover),
                            _ptr(G) if G is not None else None, _ptr(F) if F is not None else None,
                            _stream(stream)), "dd_force")

    def clover_dense(self):
        import numpy as np
        A = np.empty((self.lattice.V, 12, 12), dtype=np.complex128)
        check(_lib.dd_clover_download(self.h, A.ctypes.data), "dd_clover_download")
        return A


class Decomposition:
    """Virtual-rank domain decomposition of an operator's lattice (dd_decomp)."""

    def __init__(self, op, grid):
        lib = load()
        self.op = op
        self.grid = tuple(int(g) for g in grid)
        h = ctypes.c_void_p()
        check(lib.dd_decomp_create(op.h, (ctypes.c_int * 4)(*self.grid), ctypes.byref(h)), "dd_decomp_create")
        self.h = h
        self.nranks = self.info(0)["nranks"]

    def info(self, rank):
        c, o, n = (ctypes.c_int * 4)(), (ctypes.c_int * 4)(), (ctypes.c_int * 4)()
        nb = ctypes.c_int64()
        k = _lib.dd_decomp_info(self.h, rank, c, o, n, ctypes.byref(nb))
        if k < 0:
            check(k, "dd_decomp_info")
        return {"nranks": k, "coord": tuple(c), "offset": tuple(o), "local": tuple(n), "boundary_sites": nb.value}

    def scatter(self, prec, subset, native, nrhs, stream=None):
        check(_lib.dd_decomp_scatter(self.h, prec, subset, _ptr(native), nrhs, _stream(stream)), "dd_decomp_scatter")

    def gather(self, prec, subset, native, nrhs, stream=None):
        check(_lib.dd_decomp_gather(self.h, prec, subset, _ptr(native), nrhs, _stream(stream)), "dd_decomp_gather")

    def apply(self, which, prec, nrhs, stream=None):
        check(_lib.dd_decomp_apply(self.h, which, prec, nrhs, _stream(stream)), "dd_decomp_apply")

    def dot(self, prec, subset, nrhs, stream=None):
        import numpy as np
        out = np.empty((nrhs, 2), dtype=np.float64)
        check(_lib.dd_decomp_dot(self.h, prec, subset, nrhs, out.ctypes.data, _stream(stream)), "dd_decomp_dot")
        return out[:, 0] + 1j * out[:, 1]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dd_decomp_destroy(self.h)
            self.h = None


class Amg:
    """Two-level AMG preconditioner (dd_amg_create); w0: canonical device
    test vectors [n_tv, V, 12] complex128 (a torch tensor)."""

    def __init__(self, op, prec, w0, **kw):
        p = AmgParams()
        _lib.dd_amg_params_default(ctypes.byref(p))
        for k, v in kw.items():
            if k in ("aggregate", "sap_block"):
                v = (ctypes.c_int * 4)(*v)
            setattr(p, k, v)
        self.params = p
        self.op = op  # keeps the operator alive
        h = ctypes.c_void_p()
        check(_lib.dd_amg_create(op.h, prec, ctypes.byref(p), _ptr(w0), ctypes.byref(h)), "dd_amg_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dd_amg_destroy(self.h)
            self.h = None

    def info(self):
        cd = (ctypes.c_int * 4)()
        dof, steps = ctypes.c_int(), ctypes.c_int()
        sec = ctypes.c_double()
        check(_lib.dd_amg_info(self.h, cd, ctypes.byref(dof), ctypes.byref(sec), ctypes.byref(steps)), "dd_amg_info")
        return {"coarse_dims": tuple(cd), "dof_per_aggregate": dof.value, "setup_seconds": sec.value,
                "last_coarse_steps": steps.value}

    def coarse_operator(self):
        import numpy as np
        i = self.info()
        nagg = int(np.prod(i["coarse_dims"]))
        K = i["dof_per_aggregate"]
        out = np.empty((nagg, 9, K, K), dtype=np.complex128)
        check(_lib.dd_amg_coarse_download(self.h, out.ctypes.data), "dd_amg_coarse_download")
        return out  # [agg][block][col][row]

    def apply(self, v, z, nrhs, layout=DD_LAYOUT_CANONICAL, stream=None):
        check(_lib.dd_amg_apply(self.h, _ptr(v), _ptr(z), nrhs, layout, _stream(stream)), "dd_amg_apply")
