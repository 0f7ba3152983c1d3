"""The C-ABI library loads, exports every symbol include/stag.h declares, and
rejects bad arguments before touching a GPU.  No compute calls: these run on
a machine without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1411_2087_gb300 import build as stag_build
from paper_1411_2087_gb300 import stag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stag.h")


@pytest.fixture(scope="module")
def L():
    stag_build.build()
    return stag.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stag_\w+)\s*\(", text)) - {"STAG_PREC_BIT"})


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"{n} declared in stag.h but not exported"
    assert sorted(stag.EXPORTED) == names


def test_strerror_and_version(L):
    assert stag.version().count(".") == 2
    assert L.stag_strerror(stag.ERR_ARG) == b"invalid argument"
    assert L.stag_strerror(stag.ERR_NOT_CONVERGED) == b"not converged"
    assert L.stag_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("dims", [(4, 4, 4, 3), (0, 4, 4, 4), (4, 4, -2, 4), (1, 2, 2, 2)])
def test_lattice_create_rejects_bad_dims(L, dims):
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*dims)
    st = L.stag_lattice_create(ctypes.byref(h), d, None, 0, None)
    assert st == stag.ERR_ARG
    assert h.value is None
    assert b"dims" in L.stag_last_error_message()


def test_lattice_size_limit_of_32bit_link_offsets(L):
    """The kernels address the 72 link planes of one parity with 32-bit
    offsets: 64^3 x 226 (72 x 29,622,272 planes < 2^31) passes the argument
    checks (and stops at the missing device here), 64^3 x 228 is refused
    before any CUDA call."""
    h = ctypes.c_void_p()
    ok = (ctypes.c_int * 4)(64, 64, 64, 226)
    assert L.stag_lattice_create(ctypes.byref(h), ok, None, 0, None) == stag.ERR_CUDA
    big = (ctypes.c_int * 4)(64, 64, 64, 228)
    assert L.stag_lattice_create(ctypes.byref(h), big, None, 0, None) == stag.ERR_ARG
    assert b"32-bit link offsets" in L.stag_last_error_message()
    assert h.value is None


def test_lattice_create_rejects_bad_bc_and_null(L):
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    bc = (ctypes.c_double * 4)(1, 1, 0.5, -1)
    assert L.stag_lattice_create(ctypes.byref(h), d, bc, 0, None) == stag.ERR_ARG
    assert b"bc" in L.stag_last_error_message()
    assert L.stag_lattice_create(None, d, None, 0, None) == stag.ERR_ARG
    assert L.stag_lattice_create(ctypes.byref(h), None, None, 0, None) == stag.ERR_ARG
    assert L.stag_lattice_create(ctypes.byref(h), d, None, -1, None) == stag.ERR_ARG
    big = (ctypes.c_int * 4)(2048, 2048, 2048, 2048)
    assert L.stag_lattice_create(ctypes.byref(h), big, None, 0, None) == stag.ERR_ARG


def test_null_handles_rejected(L):
    assert L.stag_lattice_destroy(None) == stag.OK
    assert L.stag_field_destroy(None) == stag.OK
    assert L.stag_gauge_upload(None, None, None, 1.0, 1.0, 0, 0) == stag.ERR_ARG
    assert L.stag_dslash_eo(None, None, None) == stag.ERR_ARG
    assert L.stag_dslash_oe(None, None, None) == stag.ERR_ARG
    assert L.stag_apply_M(None, None, None, 0.1) == stag.ERR_ARG
    assert L.stag_cg_solve(None, None, None, 0.1, 1e-10, 10, None) == stag.ERR_ARG
    assert L.stag_cg_solve_traced(None, None, None, 0.1, 1e-10, 10, None, 5, None) == stag.ERR_ARG
    assert L.stag_dd_dslash(None, 2, None, None) == stag.ERR_ARG
    n = ctypes.c_ulonglong()
    assert L.stag_field_bytes(None, 0, ctypes.byref(n)) == stag.ERR_ARG
    hw = ctypes.c_void_p()
    assert L.stag_field_wrap(None, 0, 0, None, 0, ctypes.byref(hw)) == stag.ERR_ARG
    assert L.stag_field_wrap(None, 0, 0, None, 0, None) == stag.ERR_ARG
    assert L.stag_dd_cg_solve(None, 2, None, None, 0.1, 1e-10, 10, None) == stag.ERR_ARG
    assert L.stag_field_import(None, None, 0) == stag.ERR_ARG
    assert L.stag_field_export(None, None, 0) == stag.ERR_ARG
    assert L.stag_field_zero(None) == stag.ERR_ARG
    h = ctypes.c_void_p()
    assert L.stag_field_create(None, 0, 0, ctypes.byref(h)) == stag.ERR_ARG
    assert L.stag_long_links_build(None, None, None, 0) == stag.ERR_ARG


def test_no_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert L.stag_lattice_create(ctypes.byref(h), d, None, 0, None) == stag.ERR_CUDA
    assert h.value is None


def test_binding_checks_shapes():
    import numpy as np
    with pytest.raises(ValueError):
        stag._as_buffer(np.zeros((3, 3)), (4, 3))
    with pytest.raises(ValueError):
        stag._as_buffer(np.zeros((4, 3), dtype=np.float64), (4, 3))
    p, kind, keep = stag._as_buffer(np.zeros((4, 3), dtype=np.complex128), (4, 3))
    assert kind == stag.PTR_HOST


def test_noalloc_argument_checks_before_cuda(L):
    """stag_apply_M_noalloc rejects bad arguments before any CUDA call (dummy
    non-NULL pointers: none is dereferenced before the checks fail)."""
    dummy = ctypes.c_void_p(0x1000)
    other = ctypes.c_void_p(0x2000)
    d = (ctypes.c_int * 4)(4, 4, 4, 4)

    def call(dims=d, bc=None, c1=1.125, c3=-1 / 24, fat=dummy, lng=dummy, mass=0.1, i=dummy, o=other):
        st = L.stag_apply_M_noalloc(dims, bc, c1, c3, fat, lng, mass, i, o, None)
        return st, L.stag_last_error_message()

    for args in ({"dims": None}, {"fat": None}, {"lng": None}, {"i": None}, {"o": None}):
        st, msg = call(**args)
        assert st == stag.ERR_ARG and b"NULL" in msg, args
    for dims in ((4, 4, 4, 3), (4, 0, 4, 4), (1, 4, 4, 4), (4, 4, -2, 4)):
        st, msg = call(dims=(ctypes.c_int * 4)(*dims))
        assert st == stag.ERR_ARG and b"even" in msg, dims
    st, msg = call(dims=(ctypes.c_int * 4)(16, 16, 16, 64))
    assert st == stag.ERR_ARG and b"65536" in msg
    st, msg = call(bc=(ctypes.c_double * 4)(1, 1, 0.5, -1))
    assert st == stag.ERR_ARG and b"bc" in msg
    for kw in ({"c1": float("nan")}, {"c3": float("inf")}, {"mass": float("nan")}):
        st, msg = call(**kw)
        assert st == stag.ERR_ARG and b"finite" in msg, kw
    st, msg = call(o=dummy)
    assert st == stag.ERR_ARG and b"differ" in msg


def test_noalloc_binding_refuses_host_tensors():
    import torch
    dims = (4, 4, 4, 4)
    V = 256
    fat = torch.zeros((4, V, 3, 3), dtype=torch.complex128)
    vec = torch.zeros((V // 2, 3), dtype=torch.complex128)
    with pytest.raises(ValueError, match="device tensors"):
        stag.apply_M_noalloc(dims, fat, fat, 0.1, vec, vec.clone())
