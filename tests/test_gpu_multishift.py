"""Multi-shift CG on the GPU against the definition: every shifted system
(M + sigma) x = b is M with mass sqrt(m^2 + sigma), so the oracle's M (FP64)
recomputes each shift's true residual; a single shift must reproduce the
plain CG."""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

SHIFTS12 = list(np.geomspace(1e-4, 0.5, 12))


def fields(dims, eps, seed):
    U = synth.su3_field(dims, eps, seed).numpy()
    return U, oracle.long_links(dims, U)


def true_res(dims, U, N, mass, shift, x, b):
    ms = np.sqrt(mass ** 2 + shift)
    return np.linalg.norm(b - oracle.apply_M(dims, U, N, ms, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("df64", 1e-10), ("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10)])
def test_multishift_all_shifts(dims, prec, tol):
    mass = 0.02
    U, N = fields(dims, 0.3, 1003)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1103).numpy()
    shifts = SHIFTS12[::-1]  # any order: the smallest is found internally
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        xs = [lat.field(stag.EVEN, prec) for _ in shifts]
        st, infos = lat.cg_multishift(xs, fb, shifts, mass, tol, 20000)
        assert st == stag.OK, infos
        sols = [x.export() for x in xs]
    iters = []
    for sigma, x, info in zip(shifts, sols, infos):
        r = true_res(dims, U, N, mass, sigma, x, b)
        # the iterated shifted residual zeta|r| drifts from the true one by the
        # working precision times the condition number
        assert r <= tol * (1.05 if prec != "f32" else 3.0), (sigma, r, info)
        assert abs(info["true_rel_resid"] - r) <= 1e-3 * r + (1e-7 if prec == "f32" else 1e-15)
        iters.append(info["iters"])
    # larger shifts are better conditioned: they stop no later
    order = np.argsort(shifts)
    it_sorted = np.array(iters)[order]
    assert np.all(np.diff(it_sorted) <= 0), it_sorted


def test_single_shift_is_plain_cg():
    dims, mass = (6, 4, 6, 10), 0.05
    U, N = fields(dims, 0.3, 5)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 6).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        info = lat.cg(fx, fb, mass, 1e-10, 5000)
        x_cg = fx.export()
        xs = [lat.field(stag.EVEN, "df64")]
        st, infos = lat.cg_multishift(xs, fb, [0.0], mass, 1e-10, 5000)
        assert st == stag.OK
        assert infos[0]["iters"] == info["iters"]
        assert np.abs(xs[0].export() - x_cg).max() <= 1e-13 * np.abs(x_cg).max()


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_multishift_mixed_refined(inner):
    dims, mass = (8, 8, 8, 8), 0.02
    U, N = fields(dims, 0.3, 1003)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1104).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32", inner))
        fb = lat.field(stag.EVEN, "df64", b)
        xs = [lat.field(stag.EVEN, "df64") for _ in SHIFTS12]
        st, infos = lat.cg_multishift(xs, fb, SHIFTS12, mass, 1e-10, 20000, mixed=inner)
        assert st == stag.OK, infos
        sols = [x.export() for x in xs]
    for sigma, x, info in zip(SHIFTS12, sols, infos):
        r = true_res(dims, U, N, mass, sigma, x, b)
        assert r <= 1.05e-10, (sigma, r, info)
        assert info["iter_rel_resid"] <= 2e-5  # after the FP32 multi-shift phase


def test_multishift_argument_errors():
    dims = (4, 4, 4, 4)
    U, N = fields(dims, 0.3, 9)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(128, 1).numpy())
        x1 = lat.field(stag.EVEN, "df64")
        x2 = lat.field(stag.EVEN, "df64")
        for xs, shifts in (([x1], [-0.1]), ([x1, x1], [0.0, 0.1]), ([fb], [0.0]),
                           ([x1, x2], [0.0, float("nan")])):
            with pytest.raises(stag.StagError) as ei:
                lat.cg_multishift(xs, fb, shifts, 0.1, 1e-10, 100)
            assert ei.value.status == stag.ERR_ARG
        many = [lat.field(stag.EVEN, "df64") for _ in range(33)]
        with pytest.raises(stag.StagError):
            lat.cg_multishift(many, fb, [0.01] * 33, 0.1, 1e-10, 100)
        # zero source: every x is zero after no iterations
        fz = lat.field(stag.EVEN, "df64", np.zeros((128, 3), complex))
        st, infos = lat.cg_multishift([x1, x2], fz, [0.0, 0.3], 0.1, 1e-10, 100)
        assert st == stag.OK and not np.any(x1.export()) and not np.any(x2.export())
