"""Thin Python binding of libstag (include/stag.h) over ctypes.

Argument marshalling only: every step of the Dslash and the solvers runs in
the CUDA library.  If ``libstag.so`` has not been built the first call raises
``LibraryNotBuilt``; there is no fallback.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA), complex128
in the canonical layouts of ``include/stag.h``:

* gauge field ``[4][V][3][3]``
* one-parity colour field ``[Vh][3]`` in checkerboard order
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libstag.so")

OK = 0
ERR_ARG = -1
ERR_STATE = -2
ERR_CUDA = -3
ERR_NOT_CONVERGED = -4
ERR_BREAKDOWN = -5
ERR_TIMEOUT = -6
ERR_NOMEM = -7

F64, F32, F16, DF64 = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "f16": F16, "df64": DF64}
COMPRESS12 = 1 << 16
COMPRESS12_LONG = 1 << 17
EVEN, ODD = 0, 1
NET_FP16_WEIGHTS, NET_LINKS16, NET_HERMITIAN = 1, 2, 4
CG_LAUNCH_GRAPH, CG_LAUNCH_HOST = 0, 1
PTR_HOST, PTR_DEVICE = 0, 1

C1_NAIK = 9.0 / 8.0
C3_NAIK = -1.0 / 24.0
BC_DEFAULT = (1.0, 1.0, 1.0, -1.0)

# every symbol include/stag.h declares (checked by the CPU tests)
EXPORTED = [
    "stag_lattice_create", "stag_lattice_destroy", "stag_lattice_volume",
    "stag_lattice_set_cg_launch",
    "stag_gauge_upload", "stag_long_links_build",
    "stag_field_create", "stag_field_destroy", "stag_field_import", "stag_field_export",
    "stag_field_zero", "stag_field_storage",
    "stag_dslash_eo", "stag_dslash_oe", "stag_apply_M",
    "stag_cg_solve", "stag_cg_solve_mixed", "stag_cg_multishift", "stag_cg_multishift_mixed",
    "stag_cg_solve_batched", "stag_cg_solve_batched_mixed", "stag_lattice_autotune",
    "stag_lattice_autotune_all", "stag_lattice_set_tuning",
    "stag_net_create", "stag_net_destroy", "stag_net_num_weights", "stag_net_set_weights",
    "stag_net_get_weights", "stag_net_apply", "stag_net_collect_pairs", "stag_net_num_pairs",
    "stag_net_get_pair", "stag_net_loss_grad", "stag_net_train", "stag_cg_solve_learned",
    "stag_net_set_loss", "stag_cg_solve_learned_mixed",
    "stag_apply_M_noalloc",
    "stag_dd_dslash", "stag_dd_cg_solve", "stag_cg_solve_traced", "stag_cb_neighbor",
    "stag_field_bytes", "stag_field_wrap",
    "stag_ddr_layout", "stag_ddr_exchange_host", "stag_ddr_create", "stag_ddr_destroy", "stag_ddr_dslash",
    "stag_ddr_cg_solve", "stag_comm_nccl_id", "stag_comm_nccl_create", "stag_comm_nccl_destroy",
    "stag_strerror", "stag_last_error_message", "stag_version",
]


class LibraryNotBuilt(RuntimeError):
    pass


class StagError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


# communicator callbacks of the rank decomposition (stag_comm in stag.h)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)
ALLREDUCE_DEV_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p)


class CommStruct(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("rank", ctypes.c_int), ("size", ctypes.c_int),
                ("device_buffers", ctypes.c_int), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN),
                ("allreduce_dev", ALLREDUCE_DEV_FN)]


class TuneResult(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("block", ctypes.c_int), ("regs", ctypes.c_int),
                ("group", ctypes.c_int), ("us", ctypes.c_double), ("chosen", ctypes.c_int)]


TUNE_KINDS = {0: "dslash", 1: "M", 2: "batch"}


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double), ("iter_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("gflops", ctypes.c_double),
                ("gbs", ctypes.c_double), ("restarts", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None
_lock = threading.Lock()


def lib():
    """Load libstag.so (built by ``paper_1411_2087_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise LibraryNotBuilt(
                f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "stag_lattice_create": ([PP, P, P, I, P], I),
            "stag_lattice_destroy": ([P], I),
            "stag_lattice_volume": ([P, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_longlong)], I),
            "stag_lattice_set_cg_launch": ([P, I, I], I),
            "stag_gauge_upload": ([P, P, P, D, D, I, ctypes.c_uint], I),
            "stag_long_links_build": ([P, P, P, I], I),
            "stag_field_create": ([P, I, I, PP], I),
            "stag_field_destroy": ([P], I),
            "stag_field_import": ([P, P, I], I),
            "stag_field_export": ([P, P, I], I),
            "stag_field_zero": ([P], I),
            "stag_field_storage": ([P, PP, ctypes.POINTER(ctypes.c_ulonglong)], I),
            "stag_dslash_eo": ([P, P, P], I),
            "stag_dslash_oe": ([P, P, P], I),
            "stag_apply_M": ([P, P, P, D], I),
            "stag_cg_solve": ([P, P, P, D, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_apply_M_noalloc": ([P, P, D, D, P, P, D, P, P, P], I),
            "stag_cg_solve_batched": ([I, P, P, P, P, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_solve_batched_mixed": ([I, P, P, P, P, D, I, I, D, ctypes.POINTER(SolveInfo)], I),
            "stag_lattice_autotune": ([P, I, P, P], I),
            "stag_lattice_autotune_all": ([P, I, ctypes.c_uint, ctypes.POINTER(TuneResult), I,
                                           ctypes.POINTER(I), ctypes.POINTER(I)], I),
            "stag_lattice_set_tuning": ([P, I, I, I, I, I], I),
            "stag_net_create": ([P, P, I, I, ctypes.c_uint, PP], I),
            "stag_net_destroy": ([P], I),
            "stag_net_num_weights": ([P, ctypes.POINTER(I)], I),
            "stag_net_set_weights": ([P, P], I),
            "stag_net_get_weights": ([P, P], I),
            "stag_net_apply": ([P, P, P, I], I),
            "stag_net_collect_pairs": ([P, P, D, D, I, I, ctypes.POINTER(I)], I),
            "stag_net_num_pairs": ([P, ctypes.POINTER(I)], I),
            "stag_net_get_pair": ([P, I, P, P], I),
            "stag_net_loss_grad": ([P, I, I, ctypes.POINTER(D), P], I),
            "stag_net_train": ([P, I, I, D, ctypes.c_uint, P], I),
            "stag_net_set_loss": ([P, I], I),
            "stag_cg_solve_learned": ([P, P, P, D, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_solve_learned_mixed": ([P, P, P, D, D, I, I, D, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_solve_mixed": ([P, P, P, D, D, I, I, D, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_multishift": ([P, P, P, I, P, D, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_multishift_mixed": ([P, P, P, I, P, D, D, I, I, D, ctypes.POINTER(SolveInfo)], I),
            "stag_cg_solve_traced": ([P, P, P, D, D, I, P, I, ctypes.POINTER(SolveInfo)], I),
            "stag_dd_dslash": ([P, I, P, P], I),
            "stag_field_bytes": ([P, I, ctypes.POINTER(ctypes.c_ulonglong)], I),
            "stag_field_wrap": ([P, I, I, P, ctypes.c_ulonglong, PP], I),
            "stag_cb_neighbor": ([P, I, ctypes.c_longlong, I, I, ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(I)], I),
            "stag_dd_cg_solve": ([P, I, P, P, D, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_ddr_layout": ([P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
            "stag_ddr_exchange_host": ([P, I, ctypes.POINTER(CommStruct), P], I),
            "stag_ddr_create": ([P, ctypes.POINTER(CommStruct), PP], I),
            "stag_ddr_destroy": ([P], I),
            "stag_ddr_dslash": ([P, P, P], I),
            "stag_ddr_cg_solve": ([P, P, P, D, D, I, ctypes.POINTER(SolveInfo)], I),
            "stag_comm_nccl_id": ([P], I),
            "stag_comm_nccl_create": ([I, I, P, I, ctypes.POINTER(CommStruct)], I),
            "stag_comm_nccl_destroy": ([ctypes.POINTER(CommStruct)], I),
            "stag_strerror": ([I], ctypes.c_char_p),
            "stag_last_error_message": ([], ctypes.c_char_p),
            "stag_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(status: int, allow=()) -> int:
    if status != OK and status not in allow:
        msg = lib().stag_last_error_message().decode(errors="replace")
        raise StagError(status, msg or lib().stag_strerror(status).decode())
    return status


# --------------------------------------------------------------------------
# buffer marshalling
# --------------------------------------------------------------------------

def _is_torch(a) -> bool:
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _as_buffer(a, shape, writable=False):
    """(pointer, ptr_kind, keepalive) for a complex128 array of `shape`."""
    if _is_torch(a):
        import torch
        if a.dtype != torch.complex128 or tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected complex128 tensor of shape {tuple(shape)}, "
                             f"got {a.dtype} {tuple(a.shape)}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        kind = PTR_DEVICE if a.is_cuda else PTR_HOST
        return ctypes.c_void_p(a.data_ptr()), kind, a
    arr = np.asarray(a)
    if arr.dtype != np.complex128 or arr.shape != tuple(shape):
        raise ValueError(f"expected complex128 array of shape {tuple(shape)}, "
                         f"got {arr.dtype} {arr.shape}")
    if not arr.flags.c_contiguous or (writable and not arr.flags.writeable):
        raise ValueError("array must be C-contiguous" + (" and writable" if writable else ""))
    return arr.ctypes.data_as(ctypes.c_void_p), PTR_HOST, arr


# --------------------------------------------------------------------------
# objects
# --------------------------------------------------------------------------

class Field:
    """One-parity colour field in the library's internal layout."""

    def __init__(self, lattice: "Lattice", parity: int, prec="df64", wrap=None):
        """wrap: a contiguous CUDA tensor to view (stag_field_wrap) instead
        of library-owned storage; the tensor must outlive the field."""
        self.lattice = lattice
        self.parity = int(parity)
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        h = ctypes.c_void_p()
        if wrap is None:
            _check(lib().stag_field_create(lattice.handle, self.parity, self.prec, ctypes.byref(h)))
        else:
            if not getattr(wrap, "is_cuda", False) or not wrap.is_contiguous():
                raise ValueError("wrap needs a contiguous CUDA tensor")
            nbytes = wrap.numel() * wrap.element_size()
            _check(lib().stag_field_wrap(lattice.handle, self.parity, self.prec, ctypes.c_void_p(wrap.data_ptr()),
                                         nbytes, ctypes.byref(h)))
        self._wrapped = wrap
        self.handle = h
        lattice._fields.add(self)

    @property
    def shape(self):
        return (self.lattice.Vh, 3)

    def import_(self, src) -> "Field":
        p, kind, keep = _as_buffer(src, self.shape)
        _check(lib().stag_field_import(self.handle, p, kind))
        return self

    def export(self, out=None):
        """Canonical complex128 [Vh][3]; a new numpy array unless `out` is given."""
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        p, kind, keep = _as_buffer(out, self.shape, writable=True)
        _check(lib().stag_field_export(self.handle, p, kind))
        return out

    def zero(self):
        _check(lib().stag_field_zero(self.handle))

    def storage(self):
        ptr = ctypes.c_void_p()
        n = ctypes.c_ulonglong()
        _check(lib().stag_field_storage(self.handle, ctypes.byref(ptr), ctypes.byref(n)))
        return ptr.value, n.value

    def destroy(self):
        if self.handle:
            _check(lib().stag_field_destroy(self.handle))
            self.handle = None
            self.lattice._fields.discard(self)


class Lattice:
    """A lattice on one CUDA device (see stag_lattice_create)."""

    def __init__(self, dims, bc=BC_DEFAULT, device: int = 0, stream: Optional[int] = None):
        self.dims = tuple(int(d) for d in dims)
        d = (ctypes.c_int * 4)(*self.dims)
        b = (ctypes.c_double * 4)(*[float(v) for v in bc]) if bc is not None else None
        h = ctypes.c_void_p()
        _check(lib().stag_lattice_create(ctypes.byref(h), d, b, int(device),
                                         ctypes.c_void_p(stream) if stream else None))
        self.handle = h
        self._fields = set()
        V = ctypes.c_longlong()
        Vh = ctypes.c_longlong()
        _check(lib().stag_lattice_volume(h, ctypes.byref(V), ctypes.byref(Vh)))
        self.V, self.Vh = V.value, Vh.value

    def set_cg_launch(self, mode: str = "graph", chunk: int = 32):
        """'graph' (device-side loop, default) or 'host' (individual launches)."""
        m = {"graph": CG_LAUNCH_GRAPH, "host": CG_LAUNCH_HOST}[mode]
        _check(lib().stag_lattice_set_cg_launch(self.handle, m, int(chunk)))

    # gauge -----------------------------------------------------------------
    def upload_gauge(self, fat, lng=None, c1=C1_NAIK, c3=C3_NAIK, precisions=("f64", "df64"),
                     compress12=False):
        """compress12: False, True (12-real one-link and three-link links in
        the FP32 and 16-bit copies) or "long" (the three-link links only)."""
        shape = (4, self.V, 3, 3)
        pf, kind, keep_f = _as_buffer(fat, shape)
        if lng is not None:
            pl, kind_l, keep_l = _as_buffer(lng, shape)
            if kind_l != kind:
                raise ValueError("fat and long links must both be on the host or both on the device")
        else:
            pl = None
        if compress12 == "long":
            mask = COMPRESS12_LONG
        elif compress12 in (True, False):
            mask = COMPRESS12 if compress12 else 0
        else:
            raise ValueError("compress12 must be False, True or 'long'")
        for p in precisions:
            mask |= 1 << (PREC[p] if isinstance(p, str) else int(p))
        _check(lib().stag_gauge_upload(self.handle, pf, pl, float(c1), float(c3), kind, mask))

    def long_links(self, fat, out=None):
        """Three-link products of `fat` computed on the GPU (canonical layout)."""
        shape = (4, self.V, 3, 3)
        pf, kind, keep_f = _as_buffer(fat, shape)
        if out is None:
            if kind == PTR_DEVICE:
                import torch
                out = torch.empty(shape, dtype=torch.complex128, device=fat.device)
            else:
                out = np.empty(shape, dtype=np.complex128)
        po, kind_o, keep_o = _as_buffer(out, shape, writable=True)
        if kind_o != kind:
            raise ValueError("fat and output must both be on the host or both on the device")
        _check(lib().stag_long_links_build(self.handle, pf, po, kind))
        return out

    # fields ----------------------------------------------------------------
    def field(self, parity: int, prec="df64", data=None) -> Field:
        f = Field(self, parity, prec)
        if data is not None:
            f.import_(data)
        return f

    def field_bytes(self, prec="df64") -> int:
        n = ctypes.c_ulonglong()
        _check(lib().stag_field_bytes(self.handle, PREC[prec] if isinstance(prec, str) else int(prec),
                                      ctypes.byref(n)))
        return n.value

    def wrap_field(self, tensor, parity: int, prec="df64") -> Field:
        """A field viewing `tensor` (CUDA, contiguous, >= field_bytes(prec)
        bytes, internal layout): zero-copy with torch."""
        return Field(self, parity, prec, wrap=tensor)

    # operators -------------------------------------------------------------
    def dslash(self, out: Field, inp: Field):
        if out.parity == EVEN:
            _check(lib().stag_dslash_eo(self.handle, out.handle, inp.handle))
        else:
            _check(lib().stag_dslash_oe(self.handle, out.handle, inp.handle))

    def apply_M(self, out: Field, inp: Field, mass: float):
        _check(lib().stag_apply_M(self.handle, out.handle, inp.handle, float(mass)))

    def cg(self, x: Field, b: Field, mass: float, tol: float = 1e-10, max_iter: int = 20000,
           raise_on_failure: bool = False) -> dict:
        info = SolveInfo()
        st = lib().stag_cg_solve(self.handle, x.handle, b.handle, float(mass), float(tol),
                                 int(max_iter), ctypes.byref(info))
        if raise_on_failure or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def cg_traced(self, x: Field, b: Field, mass: float, n_trace: int, tol: float = 1e-10,
                  max_iter: int = 20000):
        """CG recording (alpha_k, beta_k, |r_{k+1}|^2) of the first n_trace
        iterations; returns (info, trace[min(iters, n_trace)][3])."""
        trace = np.zeros((max(int(n_trace), 1), 3))
        info = SolveInfo()
        st = lib().stag_cg_solve_traced(self.handle, x.handle, b.handle, float(mass), float(tol),
                                        int(max_iter), trace.ctypes.data_as(ctypes.c_void_p),
                                        int(n_trace), ctypes.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d, trace[: min(d["iters"], int(n_trace))].copy()

    def dd_dslash(self, out: Field, inp: Field, ndomains: int):
        """Dslash computed on `ndomains` t-slabs with depth-3 halo copies."""
        _check(lib().stag_dd_dslash(self.handle, int(ndomains), out.handle, inp.handle))

    def dd_cg(self, x: Field, b: Field, mass: float, ndomains: int, tol: float = 1e-10,
              max_iter: int = 20000, raise_on_failure: bool = False) -> dict:
        """CG on `ndomains` t-slabs with host-reduced inner products."""
        info = SolveInfo()
        st = lib().stag_dd_cg_solve(self.handle, int(ndomains), x.handle, b.handle, float(mass),
                                    float(tol), int(max_iter), ctypes.byref(info))
        if raise_on_failure or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def cg_mixed(self, x: Field, b: Field, mass: float, tol: float = 1e-10, max_iter: int = 20000,
                 inner="f32", delta: float = 0.1, raise_on_failure: bool = False) -> dict:
        info = SolveInfo()
        ip = PREC[inner] if isinstance(inner, str) else int(inner)
        st = lib().stag_cg_solve_mixed(self.handle, x.handle, b.handle, float(mass), float(tol),
                                       int(max_iter), ip, float(delta), ctypes.byref(info))
        if raise_on_failure or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def cg_multishift(self, xs, b: Field, shifts, mass: float, tol: float = 1e-10,
                      max_iter: int = 20000, mixed: Optional[str] = None, delta: float = 0.1):
        """Multi-shift CG; `mixed` = 'f32' or 'f16' refines FP32 multi-shift
        solutions with reliable-update CG.  Returns (status, [info per shift])."""
        n = len(shifts)
        if len(xs) != n:
            raise ValueError("one solution field per shift")
        hx = (ctypes.c_void_p * n)(*[x.handle.value for x in xs])
        sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
        infos = (SolveInfo * n)()
        if mixed is None:
            st = lib().stag_cg_multishift(self.handle, hx, sh, n, b.handle, float(mass), float(tol),
                                          int(max_iter), infos)
        else:
            st = lib().stag_cg_multishift_mixed(self.handle, hx, sh, n, b.handle, float(mass),
                                                float(tol), int(max_iter), PREC[mixed], float(delta),
                                                infos)
        if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        return st, [i.as_dict() for i in infos]

    def autotune(self, prec="df64"):
        """Pick the fastest block sizes for `prec`; returns the timings (us)."""
        d = (ctypes.c_double * 2)()
        b = (ctypes.c_double * 2)()
        _check(lib().stag_lattice_autotune(self.handle, PREC[prec], d, b))
        return {"dslash_us": {128: d[0], 256: d[1]}, "batch_us": {128: b[0], 256: b[1]}}

    def autotune_all(self, prec="df64", force: bool = False):
        """(results, cached): every candidate timed (or the cached choice);
        results are dicts with kernel, block, regs, group, us, chosen."""
        buf = (TuneResult * 64)()
        n, cached = ctypes.c_int(), ctypes.c_int()
        _check(lib().stag_lattice_autotune_all(self.handle, PREC[prec], 1 if force else 0, buf, 64,
                                               ctypes.byref(n), ctypes.byref(cached)))
        res = [{"kernel": TUNE_KINDS[r.kernel], "block": r.block, "regs": r.regs, "group": r.group,
                "us": r.us, "chosen": bool(r.chosen)} for r in buf[:n.value]]
        return res, bool(cached.value)

    def set_tuning(self, prec, kernel: str, block: int, regs: int = 0, group: int = 0):
        k = {v: key for key, v in TUNE_KINDS.items()}[kernel]
        _check(lib().stag_lattice_set_tuning(self.handle, PREC[prec], k, int(block), int(regs), int(group)))

    def close(self):
        for n in list(getattr(self, "_nets", [])):
            n.close()
        for f in list(self._fields):
            f.destroy()
        if self.handle:
            _check(lib().stag_lattice_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover - best effort
        try:
            if getattr(self, "handle", None) and _lib is not None:
                self.close()
        except Exception:
            pass


def cb_neighbor(dims, parity: int, cb: int, mu: int, steps: int):
    """(neighbour cb index, wraps) as the Dslash kernels compute them (host)."""
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    j = ctypes.c_longlong()
    w = ctypes.c_int()
    _check(lib().stag_cb_neighbor(d, int(parity), int(cb), int(mu), int(steps), ctypes.byref(j),
                                  ctypes.byref(w)))
    return j.value, w.value


def apply_M_noalloc(dims, fat, lng, mass, in_even, out_even, bc=BC_DEFAULT, c1=C1_NAIK,
                    c3=C3_NAIK, stream=None):
    """stag_apply_M_noalloc on CUDA tensors the caller owns (see stag.h)."""
    import torch
    V = int(np.prod(dims))
    for t, shape in ((fat, (4, V, 3, 3)), (lng, (4, V, 3, 3)), (in_even, (V // 2, 3)),
                     (out_even, (V // 2, 3))):
        p, kind, keep = _as_buffer(t, shape)
        if kind != PTR_DEVICE:
            raise ValueError("stag_apply_M_noalloc needs device tensors")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("stag_apply_M_noalloc needs tensors on the current CUDA device "
                             f"(cuda:{torch.cuda.current_device()}), got {t.device}")
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    b = (ctypes.c_double * 4)(*[float(v) for v in bc]) if bc is not None else None
    _check(lib().stag_apply_M_noalloc(d, b, float(c1), float(c3), ctypes.c_void_p(fat.data_ptr()),
                                      ctypes.c_void_p(lng.data_ptr()), float(mass),
                                      ctypes.c_void_p(in_even.data_ptr()),
                                      ctypes.c_void_p(out_even.data_ptr()),
                                      ctypes.c_void_p(stream) if stream else None))


# --------------------------------------------------------------------------
# domain decomposition over ranks
# --------------------------------------------------------------------------

def ddr_layout(dims, size: int, rank: int):
    """(t0, nt): the slab of `rank` of `size` (stag_ddr_layout)."""
    t0, nt = ctypes.c_int(), ctypes.c_int()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(lib().stag_ddr_layout(d, int(size), int(rank), ctypes.byref(t0), ctypes.byref(nt)))
    return t0.value, nt.value


class HostComm:
    """A communicator over host memory from two Python callables:
    exchange(to_prev: bytes, to_next: bytes) -> (from_prev, from_next) and
    allreduce(values: list[float]) -> list[float] (sums over the ranks).
    Exceptions in the callables become a failed call (status 1)."""

    def __init__(self, rank: int, size: int, exchange, allreduce):
        self.rank, self.size = int(rank), int(size)
        self._exchange, self._allreduce = exchange, allreduce
        self.error = None

        def ex(ctx, to_prev, to_next, from_prev, from_next, nbytes, stream):
            try:
                fp, fn = self._exchange(ctypes.string_at(to_prev, nbytes), ctypes.string_at(to_next, nbytes))
                if len(fp) != nbytes or len(fn) != nbytes:
                    raise ValueError("exchange returned messages of the wrong size")
                ctypes.memmove(from_prev, fp, nbytes)
                ctypes.memmove(from_next, fn, nbytes)
                return 0
            except BaseException as e:  # noqa: BLE001 - reported through the status
                self.error = e
                return 1

        def ar(ctx, vals, n):
            try:
                out = self._allreduce([vals[k] for k in range(n)])
                for k in range(n):
                    vals[k] = float(out[k])
                return 0
            except BaseException as e:  # noqa: BLE001
                self.error = e
                return 1

        self._cb = (EXCHANGE_FN(ex), ALLREDUCE_FN(ar))
        self.struct = CommStruct(None, self.rank, self.size, 0, self._cb[0], self._cb[1])


class NcclComm:
    """NCCL as the communicator (stag_comm_nccl_create); `uid` is the
    128-byte id from nccl_unique_id() on one rank, shared by the caller."""

    def __init__(self, rank: int, size: int, uid: bytes, device: int):
        if len(uid) != 128:
            raise ValueError("an NCCL unique id has 128 bytes")
        self.struct = CommStruct()
        buf = (ctypes.c_ubyte * 128).from_buffer_copy(uid)
        _check(lib().stag_comm_nccl_create(int(rank), int(size), buf, int(device), ctypes.byref(self.struct)))
        self.rank, self.size = int(rank), int(size)

    def close(self):
        if self.struct.ctx:
            _check(lib().stag_comm_nccl_destroy(ctypes.byref(self.struct)))


def nccl_unique_id() -> bytes:
    buf = (ctypes.c_ubyte * 128)()
    _check(lib().stag_comm_nccl_id(buf))
    return bytes(buf)


def ddr_exchange_host(dims, parity: int, comm, field):
    """stag_ddr_exchange_host on a canonical complex128 [Vh][3] numpy array
    (modified in place: its halo slices)."""
    Vh = int(np.prod(dims)) // 2
    p, kind, keep = _as_buffer(field, (Vh, 3), writable=True)
    if kind != PTR_HOST:
        raise ValueError("stag_ddr_exchange_host works on host memory")
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(lib().stag_ddr_exchange_host(d, int(parity), ctypes.byref(comm.struct), p))


class DDRank:
    """One rank's view of a lattice split in t over the ranks of `comm`
    (stag_ddr_*): `lattice` is this rank's full-size lattice."""

    def __init__(self, lattice: "Lattice", comm):
        self.lattice, self.comm = lattice, comm
        h = ctypes.c_void_p()
        _check(lib().stag_ddr_create(lattice.handle, ctypes.byref(comm.struct), ctypes.byref(h)))
        self.handle = h
        self.t0, self.nt = ddr_layout(lattice.dims, comm.size, comm.rank)
        if not hasattr(lattice, "_nets"):
            lattice._nets = set()
        lattice._nets.add(self)

    def dslash(self, out: Field, inp: Field):
        _check(lib().stag_ddr_dslash(self.handle, out.handle, inp.handle))

    def cg(self, x: Field, b: Field, mass: float, tol: float = 1e-10, max_iter: int = 20000) -> dict:
        info = SolveInfo()
        st = lib().stag_ddr_cg_solve(self.handle, x.handle, b.handle, float(mass), float(tol), int(max_iter),
                                     ctypes.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def close(self):
        if self.handle:
            _check(lib().stag_ddr_destroy(self.handle))
            self.handle = None
            getattr(self.lattice, "_nets", set()).discard(self)


def cg_batched(systems, tol: float = 1e-10, max_iter: int = 20000, mixed: Optional[str] = None,
               delta: float = 0.1):
    """Batched CG over [(lattice, x, b, mass), ...] (systems of one lattice
    consecutive).  `mixed` = 'f32' or 'f16' runs the FP32 batch and refines.
    Returns (status, [info per system])."""
    n = len(systems)
    lats = (ctypes.c_void_p * n)(*[s[0].handle.value for s in systems])
    xs = (ctypes.c_void_p * n)(*[s[1].handle.value for s in systems])
    bs = (ctypes.c_void_p * n)(*[s[2].handle.value for s in systems])
    ms = (ctypes.c_double * n)(*[float(s[3]) for s in systems])
    infos = (SolveInfo * n)()
    if mixed is None:
        st = lib().stag_cg_solve_batched(n, lats, xs, bs, ms, float(tol), int(max_iter), infos)
    else:
        st = lib().stag_cg_solve_batched_mixed(n, lats, xs, bs, ms, float(tol), int(max_iter),
                                               PREC[mixed], float(delta), infos)
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        _check(st)
    return st, [i.as_dict() for i in infos]


class Net:
    """The learned gauge-covariant preconditioner (see stag_net_* in stag.h).

    Weights are exchanged as complex128 arrays: a list of three arrays of
    shapes [9][C][1], [9][C][C], [9][1][C]."""

    def __init__(self, lattice: "Lattice", fat, channels: int = 8, seed: int = 0):
        self.lattice = lattice
        self.C = int(channels)
        p, kind, keep = _as_buffer(fat, (4, lattice.V, 3, 3))
        h = ctypes.c_void_p()
        _check(lib().stag_net_create(lattice.handle, p, kind, self.C, int(seed) & 0xffffffff,
                                     ctypes.byref(h)))
        self.handle = h
        n = ctypes.c_int()
        _check(lib().stag_net_num_weights(h, ctypes.byref(n)))
        self.nw = n.value
        if not hasattr(lattice, "_nets"):
            lattice._nets = set()
        lattice._nets.add(self)

    def _shapes(self):
        C = self.C
        return [(9, C, 1), (9, C, C), (9, 1, C)]

    def get_weights(self):
        buf = np.empty(2 * self.nw, dtype=np.float64)
        _check(lib().stag_net_get_weights(self.handle, buf.ctypes.data_as(ctypes.c_void_p)))
        z = buf[0::2] + 1j * buf[1::2]
        out, off = [], 0
        for sh in self._shapes():
            n = int(np.prod(sh))
            out.append(z[off:off + n].reshape(sh).copy())
            off += n
        return out

    def set_weights(self, ws):
        flat = np.concatenate([np.asarray(w, dtype=np.complex128).reshape(-1) for w in ws])
        if flat.size != self.nw:
            raise ValueError(f"expected {self.nw} complex weights, got {flat.size}")
        buf = np.empty(2 * self.nw, dtype=np.float64)
        buf[0::2] = flat.real
        buf[1::2] = flat.imag
        _check(lib().stag_net_set_weights(self.handle, buf.ctypes.data_as(ctypes.c_void_p)))

    def set_loss(self, kind: str = "error"):
        """'error' (|N r - e|^2/|e|^2) or 'residual' (|M N r - r|^2/|r|^2)."""
        _check(lib().stag_net_set_loss(self.handle, {"error": 0, "residual": 1}[kind]))

    def apply(self, out: Field, inp: Field, fp16_weights: bool = False, links16: bool = False,
              hermitian: bool = False):
        """out = N(inp), or its Hermitian part (N + N^+)/2; all three flags
        together are the solvers' form."""
        flags = ((NET_FP16_WEIGHTS if fp16_weights else 0) | (NET_LINKS16 if links16 else 0)
                 | (NET_HERMITIAN if hermitian else 0))
        _check(lib().stag_net_apply(self.handle, out.handle, inp.handle, flags))

    def collect_pairs(self, b: Field, mass: float, tol: float = 1e-10, stride: int = 10,
                      max_pairs: int = 64) -> int:
        n = ctypes.c_int()
        _check(lib().stag_net_collect_pairs(self.handle, b.handle, float(mass), float(tol), int(stride),
                                            int(max_pairs), ctypes.byref(n)))
        return n.value

    def num_pairs(self) -> int:
        n = ctypes.c_int()
        _check(lib().stag_net_num_pairs(self.handle, ctypes.byref(n)))
        return n.value

    def get_pair(self, k: int):
        Vh = self.lattice.Vh
        r = np.empty((Vh, 3), dtype=np.complex128)
        e = np.empty((Vh, 3), dtype=np.complex128)
        _check(lib().stag_net_get_pair(self.handle, int(k), r.ctypes.data_as(ctypes.c_void_p),
                                       e.ctypes.data_as(ctypes.c_void_p)))
        return r, e

    def loss_grad(self, first: int, count: int):
        """(loss, [dL/dW* per layer]) over pairs [first, first+count)."""
        loss = ctypes.c_double()
        buf = np.empty(2 * self.nw, dtype=np.float64)
        _check(lib().stag_net_loss_grad(self.handle, int(first), int(count), ctypes.byref(loss),
                                        buf.ctypes.data_as(ctypes.c_void_p)))
        z = buf[0::2] + 1j * buf[1::2]
        out, off = [], 0
        for sh in self._shapes():
            n = int(np.prod(sh))
            out.append(z[off:off + n].reshape(sh).copy())
            off += n
        return loss.value, out

    def train(self, epochs: int = 10, batch: int = 8, lr: float = 1e-2, seed: int = 0):
        hist = np.zeros(int(epochs))
        _check(lib().stag_net_train(self.handle, int(epochs), int(batch), float(lr), int(seed) & 0xffffffff,
                                    hist.ctypes.data_as(ctypes.c_void_p)))
        return hist

    def cg(self, x: Field, b: Field, mass: float, tol: float = 1e-10, max_iter: int = 20000,
           raise_on_failure: bool = False) -> dict:
        info = SolveInfo()
        st = lib().stag_cg_solve_learned(self.handle, x.handle, b.handle, float(mass), float(tol),
                                         int(max_iter), ctypes.byref(info))
        if raise_on_failure or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def cg_mixed(self, x: Field, b: Field, mass: float, tol: float = 1e-10, max_iter: int = 20000,
                 inner="f16", delta: float = 0.1, raise_on_failure: bool = False) -> dict:
        """Mixed-precision flexible CG with the net (stag_cg_solve_learned_mixed)."""
        info = SolveInfo()
        ip = PREC[inner] if isinstance(inner, str) else int(inner)
        st = lib().stag_cg_solve_learned_mixed(self.handle, x.handle, b.handle, float(mass), float(tol),
                                               int(max_iter), ip, float(delta), ctypes.byref(info))
        if raise_on_failure or st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(st)
        d = info.as_dict()
        d["return"] = st
        return d

    def close(self):
        if self.handle:
            _check(lib().stag_net_destroy(self.handle))
            self.handle = None
            getattr(self.lattice, "_nets", set()).discard(self)


def version() -> str:
    return lib().stag_version().decode()
