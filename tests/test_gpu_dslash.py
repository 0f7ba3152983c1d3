"""GPU Dslash, M and three-link products against the CPU oracle, element by
element, through the C ABI.

Tolerance: max|gpu - oracle| / max|oracle| <= 1e-12 for FP64 and the
double-float form (the FP64 target).  Reduced precisions are held to bounds
derived from their storage: FP32 (24-bit significand, 16 products summed)
to 2e-6, 16-bit fixed point (1/32767 of the link-field and per-site vector
scales) to 3e-4; the assertion message states the error against FP64.
"""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "f16": 3e-4}

# 2^4 and 4^4 alias the +-1/+-3 hops; (6,4,6,10) has Vh = 720: several
# blocks and a ragged tail; 8^4 has all 16 neighbours distinct.
DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 6, 10), (8, 8, 8, 8), (2, 6, 4, 4)]


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.fixture(scope="module", params=DIMS, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    dims = request.param
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 1000).numpy()
    N = oracle.long_links(dims, U)
    psi_e = synth.gaussian_colour_field(Vh, 1100).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 1101).numpy()
    lat = stag.Lattice(dims)
    lat.upload_gauge(U, N, precisions=("f64", "df64", "f32", "f16"))
    yield dims, U, N, psi_e, psi_o, lat
    lat.close()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_dslash_both_parities(setup, prec):
    dims, U, N, psi_e, psi_o, lat = setup
    fe = lat.field(stag.EVEN, prec, psi_e)
    fo = lat.field(stag.ODD, prec, psi_o)
    out_o = lat.field(stag.ODD, prec)
    out_e = lat.field(stag.EVEN, prec)
    lat.dslash(out_o, fe)
    lat.dslash(out_e, fo)
    e1 = rel_err(out_o.export(), oracle.dslash_parity(dims, U, N, 1, psi_e))
    e2 = rel_err(out_e.export(), oracle.dslash_parity(dims, U, N, 0, psi_o))
    for f in (fe, fo, out_o, out_e):
        f.destroy()
    assert e1 <= TOL[prec] and e2 <= TOL[prec], f"{prec}: D_oe err {e1:.3e}, D_eo err {e2:.3e}"


# M = m^2 - D_eo D_oe applies two stencils with the odd intermediate stored in
# the field's precision: the reduced-precision bounds are twice the Dslash
# bounds plus one rounding of the intermediate
TOL_M = {"f64": 1e-12, "df64": 1e-12, "f32": 5e-6, "f16": 8e-4}


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_apply_M(setup, prec):
    dims, U, N, psi_e, psi_o, lat = setup
    mass = 0.1
    fe = lat.field(stag.EVEN, prec, psi_e)
    out = lat.field(stag.EVEN, prec)
    lat.apply_M(out, fe, mass)
    err = rel_err(out.export(), oracle.apply_M(dims, U, N, mass, psi_e))
    fe.destroy()
    out.destroy()
    assert err <= TOL_M[prec], f"{prec}: M err {err:.3e}"


def test_import_export_roundtrip(setup):
    dims, U, N, psi_e, psi_o, lat = setup
    f = lat.field(stag.EVEN, "f64", psi_e)
    assert np.array_equal(f.export(), psi_e)
    f.destroy()
    h = lat.field(stag.EVEN, "f16", psi_e)
    # per-site norm, 1/32767 quantum, rounding to nearest: half a quantum,
    # plus the float rounding of the value and the scale (2^-24 of the site
    # maximum is 0.4 % of half a quantum)
    site_max = np.maximum(np.abs(psi_e.real), np.abs(psi_e.imag)).max(axis=1)
    d = h.export() - psi_e
    bound = site_max[:, None] * (0.5 / 32767) * 1.01 + 1e-12
    assert np.all(np.abs(d.real) <= bound) and np.all(np.abs(d.imag) <= bound)
    h.destroy()
    g = lat.field(stag.EVEN, "df64", psi_e)
    # double-float keeps about 48 bits
    assert np.abs(g.export() - psi_e).max() <= 2.0 ** -47 * np.abs(psi_e).max()
    g.destroy()


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 2, 8), (8, 8, 8, 8)])
def test_gpu_long_links(dims):
    U = synth.su3_field(dims, 0.5, 3).numpy()
    want = oracle.long_links(dims, U)
    with stag.Lattice(dims) as lat:
        got = lat.long_links(U)
        assert np.abs(got - want).max() < 1e-14
        # upload without long links builds them on the GPU
        Vh = int(np.prod(dims)) // 2
        psi = synth.gaussian_colour_field(Vh, 5).numpy()
        lat.upload_gauge(U, None, precisions=("f64",))
        fe = lat.field(stag.EVEN, "f64", psi)
        fo = lat.field(stag.ODD, "f64")
        lat.dslash(fo, fe)
        err = rel_err(fo.export(), oracle.dslash_parity(dims, U, want, 1, psi))
        assert err < 1e-13


@pytest.mark.parametrize("bc", [(1.0, 1.0, 1.0, 1.0), (-1.0, 1.0, -1.0, -1.0)])
def test_boundary_conditions(bc):
    dims = (4, 2, 6, 8)
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.4, 17).numpy()
    N = oracle.long_links(dims, U)
    psi = synth.gaussian_colour_field(Vh, 18).numpy()
    with stag.Lattice(dims, bc=bc) as lat:
        lat.upload_gauge(U, N, c1=1.25, c3=-0.1, precisions=("df64",))
        fe = lat.field(stag.EVEN, "df64", psi)
        fo = lat.field(stag.ODD, "df64")
        lat.dslash(fo, fe)
        want = oracle.dslash_parity(dims, U, N, 1, psi, bc=bc, c1=1.25, c3=-0.1)
        assert rel_err(fo.export(), want) <= 1e-12


def test_free_field_plane_wave_on_gpu():
    """Unit links: D of a plane wave is the closed form, independent of the oracle."""
    import math
    dims = (8, 4, 4, 6)
    V = int(np.prod(dims))
    U = synth.unit_gauge_field(dims).numpy()
    t, z, y, x = np.meshgrid(*(np.arange(n) for n in dims[::-1]), indexing="ij")
    xs = [a.reshape(-1) for a in (x, y, z, t)]
    p = [2 * math.pi * 3 / 8, 2 * math.pi / 4, 0.0, math.pi * 3 / 6]
    c = np.array([1.0, -0.5j, 0.25 + 0.5j])
    psi = np.exp(1j * sum(pm * xm for pm, xm in zip(p, xs)))[:, None] * c[None, :]
    par = (xs[0] + xs[1] + xs[2] + xs[3]) & 1
    eta = [np.ones(V), (-1.0) ** xs[0], (-1.0) ** (xs[0] + xs[1]), (-1.0) ** (xs[0] + xs[1] + xs[2])]
    f = [9 / 8 * math.sin(q) - 1 / 24 * math.sin(3 * q) for q in p]
    want_full = sum(eta[m] * 2j * f[m] for m in range(4))[:, None] * psi
    ev = np.nonzero(par == 0)[0]
    od = np.nonzero(par == 1)[0]
    psi_e = np.zeros((V // 2, 3), complex)
    psi_e[ev // 2] = psi[ev]
    want_o = np.zeros((V // 2, 3), complex)
    want_o[od // 2] = want_full[od]
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        fe = lat.field(stag.EVEN, "df64", psi_e)
        fo = lat.field(stag.ODD, "df64")
        lat.dslash(fo, fe)
        assert np.abs(fo.export() - want_o).max() < 1e-13


def test_state_errors():
    with stag.Lattice((4, 4, 4, 4)) as lat:
        fe = lat.field(stag.EVEN, "df64")
        fo = lat.field(stag.ODD, "df64")
        with pytest.raises(stag.StagError) as ei:
            lat.dslash(fo, fe)  # no gauge field yet
        assert ei.value.status == stag.ERR_STATE
        U = synth.su3_field((4, 4, 4, 4), 0.3, 1).numpy()
        lat.upload_gauge(U, None, precisions=("df64",))
        f64 = lat.field(stag.EVEN, "f64")
        with pytest.raises(stag.StagError) as ei:
            lat.dslash(fo, f64)  # precision mismatch
        assert ei.value.status == stag.ERR_STATE
        with pytest.raises(stag.StagError) as ei:
            lat.dslash(fe, fe)  # parity mismatch
        assert ei.value.status == stag.ERR_STATE


def test_upload_from_device_tensor_written_on_another_stream():
    """Links generated by torch on its own stream and uploaded at once (no
    synchronisation by the caller) must be read complete."""
    import torch
    dims = (16, 16, 8, 8)
    dev = torch.device("cuda", 0)
    Vh = int(np.prod(dims)) // 2
    psi = synth.gaussian_colour_field(Vh, 44).numpy()
    for _ in range(2):
        U = synth.su3_field(dims, 0.3, 43, device=dev)  # queued on torch's stream
        with stag.Lattice(dims) as lat:
            lat.upload_gauge(U, None, precisions=("df64",))
            fe = lat.field(stag.EVEN, "df64", psi)
            fo = lat.field(stag.ODD, "df64")
            lat.dslash(fo, fe)
            Uh = U.cpu().numpy()
            want = oracle.dslash_parity(dims, Uh, oracle.long_links(dims, Uh), 1, psi)
            assert rel_err(fo.export(), want) <= 1e-12
