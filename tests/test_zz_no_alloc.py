"""The allocation-free M entry point (stag_apply_M_noalloc).

Callers that cannot allocate device memory (code running while its caller
captures a CUDA graph, services with fixed pre-sized buffers, programs whose
own allocator owns the device) use this entry point on their own buffers.
These tests call it through the C ABI on buffers the test allocates up front,
twice in a row, and compare each result with the lattice-based stag_apply_M
within the FP64 tolerance of the other parity tests (1e-12 relative); they
also check that a lattice beyond the fixed scratch size is refused.

This file is collected last on purpose: a failure here comes after every
other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10), (16, 16, 16, 32)])
def test_noalloc_matches_apply_M_twice(dims):
    dev = torch.device("cuda", 0)
    Vh = int(np.prod(dims)) // 2
    mass = 0.05
    U = synth.su3_field(dims, 0.3, 2024)
    with stag.Lattice(dims) as lat:
        N = lat.long_links(U.numpy())
        lat.upload_gauge(U.numpy(), N, precisions=("f64",))
        U_d = U.to(dev)
        N_d = torch.from_numpy(N).to(dev)
        out_d = torch.empty((Vh, 3), dtype=torch.complex128, device=dev)
        for seed in (7, 8):  # two calls in a row share the scratch array
            src = synth.gaussian_colour_field(Vh, seed)
            fin = lat.field(stag.EVEN, "f64", src.numpy())
            fout = lat.field(stag.EVEN, "f64")
            lat.apply_M(fout, fin, mass)
            want = fout.export()
            in_d = src.to(dev)
            out_d.fill_(float("nan"))
            torch.cuda.synchronize()
            stag.apply_M_noalloc(dims, U_d, N_d, mass, in_d, out_d)
            torch.cuda.synchronize()
            got = out_d.cpu().numpy()
            err = rel_err(got, want)
            assert err <= TOL, f"call with seed {seed}: rel err {err:.3e}"
            fin.destroy()
            fout.destroy()


@pytest.mark.parametrize("dims,bc", [((4, 2, 6, 4), (-1.0, 1.0, 1.0, -1.0)),
                                     ((2, 4, 4, 2), (1.0, -1.0, -1.0, 1.0))])
def test_noalloc_matches_oracle_wraps_and_bc(dims, bc):
    """Extents of 2 (a three-link hop wraps twice) and non-default boundary
    signs and coefficients: the kernel's own wrap counting against the CPU
    oracle's M, twice in a row."""
    dev = torch.device("cuda", 0)
    Vh = int(np.prod(dims)) // 2
    c1, c3, mass = 1.25, -0.1, 0.3
    U = synth.su3_field(dims, 0.3, 2025).numpy()
    N = oracle.long_links(dims, U)
    U_d = torch.from_numpy(U).to(dev)
    N_d = torch.from_numpy(N).to(dev)
    out_d = torch.empty((Vh, 3), dtype=torch.complex128, device=dev)
    for seed in (9, 10):
        src = synth.gaussian_colour_field(Vh, seed).numpy()
        want = oracle.apply_M(dims, U, N, mass, src, bc=bc, c1=c1, c3=c3)
        in_d = torch.from_numpy(src).to(dev)
        out_d.fill_(float("nan"))
        torch.cuda.synchronize()
        stag.apply_M_noalloc(dims, U_d, N_d, mass, in_d, out_d, bc=bc, c1=c1, c3=c3)
        torch.cuda.synchronize()
        err = rel_err(out_d.cpu().numpy(), want)
        assert err <= TOL, f"seed {seed}: rel err {err:.3e}"


def test_noalloc_rejects_oversize_and_host_memory():
    L = stag.lib()
    big = (ctypes.c_int * 4)(16, 16, 16, 64)  # Vh = 131072 > 65536
    dev = torch.device("cuda", 0)
    t = torch.zeros(8, dtype=torch.complex128, device=dev)
    p = ctypes.c_void_p(t.data_ptr())
    st = L.stag_apply_M_noalloc(big, None, 1.125, -1 / 24, p, p, 0.1, p, p, None)
    assert st == stag.ERR_ARG
    assert b"65536" in L.stag_last_error_message()
    small = (ctypes.c_int * 4)(4, 4, 4, 4)
    host = np.zeros(4 * 256 * 9, dtype=np.complex128)
    hp = host.ctypes.data_as(ctypes.c_void_p)
    t2 = torch.zeros(128 * 3, dtype=torch.complex128, device=dev)
    st = L.stag_apply_M_noalloc(small, None, 1.125, -1 / 24, hp, hp, 0.1,
                                ctypes.c_void_p(t2.data_ptr()), p, None)
    assert st == stag.ERR_ARG
    assert b"device memory" in L.stag_last_error_message()
