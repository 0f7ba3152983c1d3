"""12-real ("two-row") link compression of the FP32 and 16-bit copies: the
Dslash with the third row rebuilt from conj(row1 x row2) / (c eta b) against
the oracle, for boundary conditions and lattice sizes that exercise every
sign of the rebuild (including hops that wrap twice on L = 2), the SU(3)
check at upload, and a mixed-precision solve on compressed 16-bit links."""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-6, "f16": 3e-4}
TOL_M = {"f32": 5e-6, "f16": 8e-4}  # two stencils and one stored intermediate


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 8), (8, 8, 8, 8), (6, 4, 6, 10)])
@pytest.mark.parametrize("bc", [(1.0, 1.0, 1.0, -1.0), (-1.0, 1.0, -1.0, -1.0), (1.0, 1.0, 1.0, 1.0)])
def test_compressed_dslash(dims, bc):
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.5, 31).numpy()
    N = oracle.long_links(dims, U)
    psi_e = synth.gaussian_colour_field(Vh, 32).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 33).numpy()
    want_o = oracle.dslash_parity(dims, U, N, 1, psi_e, bc=bc, c1=1.2, c3=-0.07)
    want_e = oracle.dslash_parity(dims, U, N, 0, psi_o, bc=bc, c1=1.2, c3=-0.07)
    with stag.Lattice(dims, bc=bc) as lat:
        lat.upload_gauge(U, N, c1=1.2, c3=-0.07, precisions=("f32", "f16"), compress12=True)
        for prec in ("f32", "f16"):
            fe = lat.field(stag.EVEN, prec, psi_e)
            fo = lat.field(stag.ODD, prec, psi_o)
            oo = lat.field(stag.ODD, prec)
            oe = lat.field(stag.EVEN, prec)
            lat.dslash(oo, fe)
            lat.dslash(oe, fo)
            e1 = rel_err(oo.export(), want_o)
            e2 = rel_err(oe.export(), want_e)
            assert e1 <= TOL[prec] and e2 <= TOL[prec], (prec, e1, e2)
            # M = m^2 - D_eo D_oe on the same links (the fused m^2 p - D t epilogue)
            om = lat.field(stag.EVEN, prec)
            lat.apply_M(om, fe, 0.3)
            em = rel_err(om.export(), oracle.apply_M(dims, U, N, 0.3, psi_e, bc=bc, c1=1.2, c3=-0.07))
            assert em <= TOL_M[prec], (prec, "M", em)


def test_compression_rejects_non_su3_links():
    dims = (4, 4, 4, 4)
    U = synth.su3_field(dims, 0.3, 34).numpy()
    with stag.Lattice(dims) as lat:
        with pytest.raises(stag.StagError) as ei:
            lat.upload_gauge(1.01 * U, None, precisions=("f32",), compress12=True)
        assert ei.value.status == stag.ERR_ARG
        with pytest.raises(stag.StagError):  # DF64 copies are never compressed
            lat.upload_gauge(U, None, precisions=("df64",), compress12=True)
        # without compression the same links are accepted
        lat.upload_gauge(1.01 * U, None, precisions=("f32",))
        # the two compression flags exclude each other
        buf = np.ascontiguousarray(U)
        st = stag.lib().stag_gauge_upload(lat.handle, buf.ctypes.data, None, stag.C1_NAIK, stag.C3_NAIK,
                                          stag.PTR_HOST,
                                          stag.COMPRESS12 | stag.COMPRESS12_LONG | (1 << stag.F32))
        assert st == stag.ERR_ARG


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 8), (6, 4, 6, 10)])
@pytest.mark.parametrize("bc", [(1.0, 1.0, 1.0, -1.0), (-1.0, 1.0, -1.0, -1.0)])
def test_long_only_compression_with_smeared_fat_links(dims, bc):
    """STAG_COMPRESS12_LONG (the paper's Sec. 4 suggestion for smeared links):
    fat links off SU(3), as smeared links are, and three-link links in
    SU(3).  Compressing both is refused; compressing the three-link field
    only reproduces the oracle's Dslash (both parities) and M in FP32 and
    16-bit storage."""
    Vh = int(np.prod(dims)) // 2
    V1 = synth.su3_field(dims, 0.5, 31).numpy()
    V2 = synth.su3_field(dims, 0.4, 37).numpy()
    fat = 0.8 * V1 + 0.2 * V2
    N = oracle.long_links(dims, V1)
    psi_e = synth.gaussian_colour_field(Vh, 32).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 33).numpy()
    kw = dict(bc=bc, c1=1.2, c3=-0.07)
    want_o = oracle.dslash_parity(dims, fat, N, 1, psi_e, **kw)
    want_e = oracle.dslash_parity(dims, fat, N, 0, psi_o, **kw)
    want_m = oracle.apply_M(dims, fat, N, 0.3, psi_e, **kw)
    with stag.Lattice(dims, bc=bc) as lat:
        with pytest.raises(stag.StagError) as ei:
            lat.upload_gauge(fat, N, c1=1.2, c3=-0.07, precisions=("f32",), compress12=True)
        assert ei.value.status == stag.ERR_ARG
        lat.upload_gauge(fat, N, c1=1.2, c3=-0.07, precisions=("f32", "f16"), compress12="long")
        for prec in ("f32", "f16"):
            fe = lat.field(stag.EVEN, prec, psi_e)
            fo = lat.field(stag.ODD, prec, psi_o)
            oo, oe, om = lat.field(stag.ODD, prec), lat.field(stag.EVEN, prec), lat.field(stag.EVEN, prec)
            lat.dslash(oo, fe)
            lat.dslash(oe, fo)
            lat.apply_M(om, fe, 0.3)
            e1, e2 = rel_err(oo.export(), want_o), rel_err(oe.export(), want_e)
            em = rel_err(om.export(), want_m)
            assert e1 <= TOL[prec] and e2 <= TOL[prec] and em <= TOL_M[prec], (prec, e1, e2, em)


@pytest.mark.parametrize("compress", [True, "long"])
def test_mixed_cg_on_compressed_links(compress):
    dims, mass = (8, 8, 8, 8), 0.02
    U = synth.su3_field(dims, 0.35, 35).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 36).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32", "f16"), compress12=compress)
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        for inner in ("f32", "f16"):
            info = lat.cg_mixed(fx, fb, mass, 1e-10, 20000, inner=inner)
            assert info["return"] == stag.OK, info
            r = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, fx.export())) / np.linalg.norm(b)
            assert r <= 1.05e-10, (inner, r)
