"""Sources far from unit scale.

Double-float and FP32 keep the float exponent range: a source of magnitude
1e-25 squares to 1e-50 and one of 1e+25 to 1e+50, both outside it.  The
solvers run on b 2^-k (k the exponent of b's largest entry) and scale the
solution back by 2^k, exactly.  These tests solve with sources scaled by
1e-25 and 1e+25 and check each solution against the FP64 oracle (its M is
linear, so the scaled problem is the same problem); imports whose finite
entries lie beyond the FP32 range are refused.
"""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

DIMS, MASS = (8, 8, 8, 8), 0.1


@pytest.fixture(scope="module")
def problem():
    U = synth.su3_field(DIMS, 0.3, 1000).numpy()
    N = oracle.long_links(DIMS, U)
    Vh = int(np.prod(DIMS)) // 2
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    return U, N, b


def rel_resid(U, N, b, x, mass=MASS, shift=0.0):
    r = b - oracle.apply_M(DIMS, U, N, mass, x) - shift * x
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("scale", [1e-25, 1e25])
def test_cg_and_traced_cg_scaled_sources(problem, scale):
    U, N, b = problem
    bs = b * scale
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        fb1 = lat.field(stag.EVEN, "df64", b)
        fx1 = lat.field(stag.EVEN, "df64")
        ref = lat.cg(fx1, fb1, MASS, 1e-10, 5000)
        info1, tr1 = lat.cg_traced(fx1, fb1, MASS, 20, 1e-10, 5000)
        fb = lat.field(stag.EVEN, "df64", bs)
        fx = lat.field(stag.EVEN, "df64")
        info = lat.cg(fx, fb, MASS, 1e-10, 5000)
        x = fx.export()
        info_t, tr = lat.cg_traced(fx, fb, MASS, 20, 1e-10, 5000)
    assert info["return"] == stag.OK, info
    res = rel_resid(U, N, bs, x)
    assert res <= 1.05e-10, res
    assert abs(info["iters"] - ref["iters"]) <= 3, (info, ref)
    # alpha, beta unchanged by the scale; |r|^2 reported in the units of b
    assert np.allclose(tr[:, :2], tr1[:, :2], rtol=1e-9, atol=0)
    assert np.allclose(tr[:, 2], tr1[:, 2] * scale**2, rtol=1e-9, atol=0)


@pytest.mark.parametrize("scale", [1e-25, 1e25])
def test_mixed_multishift_batched_scaled_sources(problem, scale):
    U, N, b = problem
    bs = b * scale
    shifts = [0.0, 0.05, 0.4]
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32", "f16"))
        fb = lat.field(stag.EVEN, "df64", bs)
        fx = lat.field(stag.EVEN, "df64")
        for inner in ("f32", "f16"):
            info = lat.cg_mixed(fx, fb, MASS, 1e-10, 5000, inner)
            assert info["return"] == stag.OK, (inner, info)
            assert rel_resid(U, N, bs, fx.export()) <= 1.05e-10, inner
        xs = [lat.field(stag.EVEN, "df64") for _ in shifts]
        for mixed in (None, "f16"):
            st, infos = lat.cg_multishift(xs, fb, shifts, MASS, 1e-10, 5000, mixed=mixed)
            assert st == stag.OK, (mixed, infos)
            for sh, x in zip(shifts, xs):
                assert rel_resid(U, N, bs, x.export(), shift=sh) <= 1.05e-10, (mixed, sh)
        b2 = synth.gaussian_colour_field(len(b), 1101).numpy() * scale
        systems = [(lat, lat.field(stag.EVEN, "df64"), fb, MASS),
                   (lat, lat.field(stag.EVEN, "df64"), lat.field(stag.EVEN, "df64", b2), 0.2)]
        for mixed in (None, "f16"):
            st, infos = stag.cg_batched(systems, 1e-10, 5000, mixed=mixed)
            assert st == stag.OK, (mixed, infos)
            assert rel_resid(U, N, bs, systems[0][1].export()) <= 1.05e-10, mixed
            assert rel_resid(U, N, b2, systems[1][1].export(), mass=0.2) <= 1.05e-10, mixed
        info = lat.dd_cg(fx, fb, MASS, 2, 1e-10, 5000)
        assert info["return"] == stag.OK, info
        assert rel_resid(U, N, bs, fx.export()) <= 1.05e-10


@pytest.mark.parametrize("scale", [1e-25, 1e25])
def test_learned_solvers_scaled_sources(problem, scale):
    U, N, b = problem
    bs = b * scale
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32", "f16"))
        net = stag.Net(lat, U, channels=4, seed=1)
        fb = lat.field(stag.EVEN, "df64", bs)
        fx = lat.field(stag.EVEN, "df64")
        info = net.cg(fx, fb, MASS, 1e-10, 5000)
        assert info["return"] == stag.OK, info
        assert rel_resid(U, N, bs, fx.export()) <= 1.05e-10
        info = net.cg_mixed(fx, fb, MASS, 1e-10, 5000, "f16")
        assert info["return"] == stag.OK, info
        assert rel_resid(U, N, bs, fx.export()) <= 1.05e-10
        net.close()


def test_import_beyond_fp32_range_refused(problem):
    U, N, b = problem
    bad = b.copy()
    bad[7, 1] = 1e39 + 2e39j
    with stag.Lattice(DIMS) as lat:
        for prec in ("df64", "f32", "f16"):
            f = lat.field(stag.EVEN, prec, b)
            before = f.export()
            with pytest.raises(stag.StagError) as ei:
                f.import_(bad)
            assert ei.value.status == stag.ERR_ARG and "FP32 range" in str(ei.value)
            assert np.array_equal(f.export(), before), prec  # unchanged
        # FP64 holds it; NaN passes the import (the solvers report it)
        f = lat.field(stag.EVEN, "f64", bad)
        assert f.export()[7, 1] == bad[7, 1]
        nan = b.copy()
        nan[0, 0] = np.nan
        lat.field(stag.EVEN, "df64", nan)


def test_reduced_precision_solve_refused_before_scaling(problem):
    """CG needs F64 or DF64 fields: an FP32 or 16-bit solve is refused with
    STAG_ERR_STATE (the source normalisation does not run first)."""
    U, N, b = problem
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("f32", "f16"))
        for prec in ("f32", "f16"):
            fb = lat.field(stag.EVEN, prec, b * 1e-25)
            fx = lat.field(stag.EVEN, prec)
            with pytest.raises(stag.StagError) as ei:
                lat.cg(fx, fb, MASS, 1e-6, 100)
            assert ei.value.status == stag.ERR_STATE, (prec, ei.value)
