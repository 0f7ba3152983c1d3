"""GPU even-odd CG against the CPU oracle through the C ABI.

Criteria (CG iterates cannot agree bit for bit when reductions sum in a
different order): the GPU solution's true residual, recomputed by the oracle,
meets the tolerance; the iteration counts agree within max(3, 1%); solving
both sides to 1e-13 gives solutions that agree to 1e-12 times the condition
number estimate; edge cases return the documented status.
"""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu


def fields(dims, eps, seed):
    U = synth.su3_field(dims, eps, seed).numpy()
    return U, oracle.long_links(dims, U)


@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 8), 0.1), ((6, 4, 6, 10), 0.05),
                                       ((4, 4, 4, 4), 0.2)])
def test_cg_matches_oracle(dims, mass, prec):
    U, N = fields(dims, 0.3, 1000)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    x_o, info_o = oracle.cg(dims, U, N, mass, b, tol=1e-10)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info = lat.cg(fx, fb, mass, 1e-10, 5000)
        x = fx.export()
    assert info["return"] == stag.OK, info
    res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)
    assert res <= 1e-10 * 1.05, res
    assert abs(info["true_rel_resid"] - res) <= 1e-3 * res + 1e-15
    assert abs(info["iters"] - info_o["iters"]) <= max(3, 0.01 * info_o["iters"]), (info, info_o)


@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 8), 0.1), ((6, 4, 6, 10), 0.05)])
def test_cg_first_iterations_match_oracle(prec, dims, mass):
    """The scalar recurrence itself: alpha_k, beta_k and |r_{k+1}|^2 of the
    first 20 iterations agree with the oracle's to 1e-12 relative."""
    U, N = fields(dims, 0.3, 1000)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    _, info_o = oracle.cg(dims, U, N, mass, b, tol=1e-10, history=True)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info, trace = lat.cg_traced(fx, fb, mass, 20, 1e-10, 5000)
        fy = lat.field(stag.EVEN, prec)
        info_g = lat.cg(fy, fb, mass, 1e-10, 5000)
        same = np.array_equal(fx.export(), fy.export())
    assert info["return"] == stag.OK and trace.shape == (20, 3)
    want = info_o["history"][:20]
    rel = np.abs(trace - want) / np.abs(want)
    assert rel.max() <= 1e-12, rel.max(axis=0)
    # tracing changes how the iterations are launched, not their arithmetic
    assert info["iters"] == info_g["iters"] and same


def test_cg_trace_shorter_than_solve_and_arguments():
    dims, mass = (4, 4, 4, 4), 0.5
    U, N = fields(dims, 0.3, 9)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 10).numpy()
    _, info_o = oracle.cg(dims, U, N, mass, b, tol=1e-10, history=True)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("f64",))
        fb = lat.field(stag.EVEN, "f64", b)
        fx = lat.field(stag.EVEN, "f64")
        # a trace longer than the solve holds every iteration
        info, trace = lat.cg_traced(fx, fb, mass, 1000, 1e-10, 5000)
        assert info["return"] == stag.OK and len(trace) == info["iters"]
        assert np.abs(trace - info_o["history"]).max() <= 1e-12 * np.abs(info_o["history"]).max()
        # trace_len 0: a plain host-driven solve
        info0, trace0 = lat.cg_traced(fx, fb, mass, 0, 1e-10, 5000)
        assert info0["iters"] == info["iters"] and len(trace0) == 0
        with pytest.raises(stag.StagError):
            lat.cg_traced(fx, fb, mass, -1)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_cg_tight_solution_agrees(prec):
    dims, mass = (4, 4, 4, 8), 0.1
    U, N = fields(dims, 0.3, 77)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 78).numpy()
    x_o, info_o = oracle.cg(dims, U, N, mass, b, tol=1e-13)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info = lat.cg(fx, fb, mass, 1e-13, 5000)
        x = fx.export()
    assert info["return"] == stag.OK, info
    # kappa <= (m^2 + 16 (7/6)^2 * max|U|-ish) / m^2; free-field bound is 2180 at m = 0.1
    kappa = (mass ** 2 + 4 * 4 * (7 / 6) ** 2) / mass ** 2
    assert np.abs(x - x_o).max() / np.abs(x_o).max() <= 1e-12 * kappa


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_cg_edge_cases(prec):
    dims = (4, 4, 4, 4)
    U, N = fields(dims, 0.3, 5)
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fx = lat.field(stag.EVEN, prec)
        # zero source: x = 0, no iterations
        fz = lat.field(stag.EVEN, prec, np.zeros((Vh, 3), complex))
        info = lat.cg(fx, fz, 0.1, 1e-10, 100)
        assert info["return"] == stag.OK and info["iters"] == 0
        assert not np.any(fx.export())
        # max_iter reached
        b = synth.gaussian_colour_field(Vh, 6).numpy()
        fb = lat.field(stag.EVEN, prec, b)
        info = lat.cg(fx, fb, 0.01, 1e-14, 3)
        assert info["return"] == stag.ERR_NOT_CONVERGED and info["iters"] == 3
        # the returned x is the 3rd iterate: compare with the oracle's
        x_o, info_o = oracle.cg(dims, U, N, 0.01, b, tol=1e-14, max_iter=3)
        assert np.abs(fx.export() - x_o).max() <= 1e-12 * np.abs(x_o).max()
        # max_iter = 0
        info = lat.cg(fx, fb, 0.01, 1e-10, 0)
        assert info["return"] == stag.ERR_NOT_CONVERGED and info["iters"] == 0
        # bad mass
        with pytest.raises(stag.StagError):
            lat.cg(fx, fb, -1.0, 1e-10, 10, raise_on_failure=True)
        # a NaN in the source is reported as a breakdown, not a hang
        bn = b.copy()
        bn[3, 1] = np.nan
        fn = lat.field(stag.EVEN, prec, bn)
        info = lat.cg(fx, fn, 0.1, 1e-10, 100)
        assert info["return"] == stag.ERR_BREAKDOWN
        # a later good solve on the same lattice still works
        info = lat.cg(fx, fb, 0.1, 1e-10, 1000)
        assert info["return"] == stag.OK


def test_cg_repeated_solves_reuse_graph():
    dims = (8, 8, 8, 8)
    U, N = fields(dims, 0.3, 1000)
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        fx = lat.field(stag.EVEN, "df64")
        iters = []
        for seed, mass in ((1, 0.1), (2, 0.2), (1, 0.1)):
            b = synth.gaussian_colour_field(Vh, seed).numpy()
            fb = lat.field(stag.EVEN, "df64", b)
            info = lat.cg(fx, fb, mass, 1e-10, 5000)
            assert info["return"] == stag.OK
            res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, fx.export())) / np.linalg.norm(b)
            assert res <= 1.05e-10
            iters.append(info["iters"])
        assert iters[0] == iters[2]  # deterministic reductions


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
@pytest.mark.parametrize("bad", [np.nan, np.inf, 1e39])
def test_corrupted_gauge_field_is_rejected(prec, bad):
    """A NaN, an infinity or an FP32-overflowing entry in either link field is
    an argument error at upload (not a silent 16-bit clamp, not a trap), and
    the lattice keeps no gauge field."""
    dims = (4, 4, 4, 4)
    U, N = fields(dims, 0.3, 5)
    for which in ("fat", "long"):
        Ub, Nb = U.copy(), N.copy()
        (Ub if which == "fat" else Nb)[2, 17, 1, 2] = complex(bad, 0.0)
        with stag.Lattice(dims) as lat:
            with pytest.raises(stag.StagError) as e:
                lat.upload_gauge(Ub, Nb, precisions=(prec,))
            assert e.value.status == stag.ERR_ARG and which in str(e.value)
            fe = lat.field(stag.EVEN, prec)
            fo = lat.field(stag.ODD, prec)
            with pytest.raises(stag.StagError) as e2:
                lat.dslash(fo, fe)
            assert e2.value.status == stag.ERR_STATE
            # a clean upload afterwards works
            lat.upload_gauge(U, N, precisions=(prec,))
            lat.dslash(fo, fe)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_host_launch_mode_is_identical(prec):
    """The host-driven launch mode runs the same kernels in the same order:
    bit-identical solution and iteration count."""
    dims = (6, 4, 6, 10)
    U, N = fields(dims, 0.3, 1000)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 31).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info_g = lat.cg(fx, fb, 0.05, 1e-10, 5000)
        xg = fx.export()
        for chunk in (1, 7, 64):
            lat.set_cg_launch("host", chunk)
            info_h = lat.cg(fx, fb, 0.05, 1e-10, 5000)
            assert info_h["return"] == stag.OK
            assert info_h["iters"] == info_g["iters"]
            assert np.array_equal(fx.export(), xg)
        info_h = lat.cg(fx, fb, 0.01, 1e-14, 5)
        assert info_h["return"] == stag.ERR_NOT_CONVERGED and info_h["iters"] == 5
        with pytest.raises(stag.StagError):
            lat.set_cg_launch("host", 0)


# ---------------------------------------------------------------------------
# mixed precision with reliable updates
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("outer,inner", [("df64", "f32"), ("df64", "f16"), ("f64", "f32"),
                                         ("f64", "f16")])
@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 8), 0.1), ((6, 4, 6, 10), 0.02)])
def test_mixed_cg_reaches_true_residual(dims, mass, outer, inner):
    U, N = fields(dims, 0.35, 1002)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1102).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(outer, inner))
        fb = lat.field(stag.EVEN, outer, b)
        fx = lat.field(stag.EVEN, outer)
        info = lat.cg_mixed(fx, fb, mass, 1e-10, 20000, inner=inner, delta=0.1)
        x = fx.export()
    assert info["return"] == stag.OK, info
    res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)
    assert res <= 1e-10 * 1.05, (res, info)
    # the reported residual is the recomputed one of the returned x
    assert abs(info["true_rel_resid"] - res) <= 1e-2 * res
    assert info["restarts"] >= 1


def test_mixed_host_mode_identical_and_edges():
    dims = (6, 4, 6, 10)
    U, N = fields(dims, 0.35, 7)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 8).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f16"))
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        ig = lat.cg_mixed(fx, fb, 0.05, 1e-10, 5000, inner="f16")
        xg = fx.export()
        lat.set_cg_launch("host", 5)
        ih = lat.cg_mixed(fx, fb, 0.05, 1e-10, 5000, inner="f16")
        assert ih["iters"] == ig["iters"] and ih["restarts"] == ig["restarts"]
        assert np.array_equal(fx.export(), xg)
        lat.set_cg_launch("graph")
        # zero source
        fz = lat.field(stag.EVEN, "df64", np.zeros((Vh, 3), complex))
        iz = lat.cg_mixed(fx, fz, 0.05, 1e-10, 100, inner="f16")
        assert iz["return"] == stag.OK and iz["iters"] == 0 and not np.any(fx.export())
        # iteration limit: x is the last reliably updated iterate, its true
        # residual is the reported one
        il = lat.cg_mixed(fx, fb, 0.01, 1e-14, 7, inner="f16")
        assert il["return"] == stag.ERR_NOT_CONVERGED and il["iters"] == 7
        r = np.linalg.norm(b - oracle.apply_M(dims, U, N, 0.01, fx.export())) / np.linalg.norm(b)
        assert abs(r - il["true_rel_resid"]) <= 1e-6 * r
        # argument errors
        with pytest.raises(stag.StagError):
            lat.cg_mixed(fx, fb, 0.05, 1e-10, 100, inner="f16", delta=1.5, raise_on_failure=True)
        with pytest.raises(stag.StagError):
            lat.cg_mixed(fx, fb, 0.05, 1e-10, 100, inner="df64", raise_on_failure=True)
        f32x = lat.field(stag.EVEN, "f32")
        with pytest.raises(stag.StagError):  # no F32 gauge copy uploaded
            lat.cg_mixed(fx, fb, 0.05, 1e-10, 100, inner="f32", raise_on_failure=True)
