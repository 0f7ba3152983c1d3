"""Batched CG (several right-hand sides on lattices of different sizes in one
graph launch) and the autotuner, against the oracle's recomputed residuals."""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

LATS = [((4, 4, 4, 8), 2, 0.1), ((6, 4, 6, 10), 3, 0.05), ((8, 8, 8, 8), 5, 0.02)]


def build(prec_list, precs_gauge):
    out = []
    for li, (dims, nrhs, mass) in enumerate(LATS):
        U = synth.su3_field(dims, 0.3, 1003 + li).numpy()
        N = oracle.long_links(dims, U)
        lat = stag.Lattice(dims)
        lat.upload_gauge(U, N, precisions=precs_gauge)
        Vh = int(np.prod(dims)) // 2
        for k in range(nrhs):
            b = synth.gaussian_colour_field(Vh, 2000 + 10 * li + k).numpy()
            out.append((lat, dims, U, N, b, mass * (1 + 0.1 * k)))
    return out


def res(dims, U, N, mass, x, b):
    return np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("df64", 1e-10), ("f64", 1e-10), ("f32", 1e-5)])
def test_batched_matches_individual(prec, tol):
    sys = build([prec], (prec,))
    fields = []
    for lat, dims, U, N, b, m in sys:
        fields.append((lat, lat.field(stag.EVEN, prec), lat.field(stag.EVEN, prec, b), m))
    st, infos = stag.cg_batched(fields, tol, 20000)
    assert st == stag.OK, infos
    for (lat, dims, U, N, b, m), (l2, fx, fb, _), info in zip(sys, fields, infos):
        x = fx.export()
        r = res(dims, U, N, m, x, b)
        assert r <= tol * (1.05 if prec != "f32" else 3.0), (dims, m, r, info)
        assert abs(info["true_rel_resid"] - r) <= 1e-3 * r + (1e-7 if prec == "f32" else 1e-15)
        if prec != "f32":
            # the same system solved alone takes the same number of iterations (+-2:
            # partial sums are grouped differently)
            fy = lat.field(stag.EVEN, prec)
            solo = lat.cg(fy, fb, m, tol, 20000)
            assert abs(solo["iters"] - info["iters"]) <= 2
    for lat in {s[0] for s in sys}:
        lat.close()


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_batched_mixed_refined(inner):
    sys = build(["df64"], ("df64", "f32", inner))
    fields = []
    for lat, dims, U, N, b, m in sys:
        fields.append((lat, lat.field(stag.EVEN, "df64"), lat.field(stag.EVEN, "df64", b), m))
    st, infos = stag.cg_batched(fields, 1e-10, 20000, mixed=inner)
    assert st == stag.OK, infos
    for (lat, dims, U, N, b, m), (l2, fx, fb, _), info in zip(sys, fields, infos):
        r = res(dims, U, N, m, fx.export(), b)
        assert r <= 1.05e-10, (dims, m, r, info)
        assert info["iter_rel_resid"] <= 2e-5
    for lat in {s[0] for s in sys}:
        lat.close()


def test_batched_argument_errors():
    dims = (4, 4, 4, 4)
    U = synth.su3_field(dims, 0.3, 1).numpy()
    with stag.Lattice(dims) as la, stag.Lattice(dims) as lb:
        for lat in (la, lb):
            lat.upload_gauge(U, None, precisions=("df64", "f32"))
        b = synth.gaussian_colour_field(128, 2).numpy()
        sa = [(la, la.field(stag.EVEN, "df64"), la.field(stag.EVEN, "df64", b), 0.1) for _ in range(2)]
        sb = [(lb, lb.field(stag.EVEN, "df64"), lb.field(stag.EVEN, "df64", b), 0.1)]
        with pytest.raises(stag.StagError):  # systems of la not consecutive
            stag.cg_batched([sa[0], sb[0], sa[1]])
        f32 = lb.field(stag.EVEN, "f32")
        with pytest.raises(stag.StagError):  # mixed precisions
            stag.cg_batched([sa[0], (lb, f32, sb[0][2], 0.1)])
        with pytest.raises(stag.StagError):  # shared solution field
            stag.cg_batched([sa[0], (la, sa[0][1], sa[1][2], 0.1)])
        with pytest.raises(stag.StagError):  # bad mass
            stag.cg_batched([(la, sa[0][1], sa[0][2], -1.0)])
        st, infos = stag.cg_batched(sa + sb)
        assert st == stag.OK


def test_autotune_keeps_results_correct():
    dims = (8, 8, 8, 8)
    U = synth.su3_field(dims, 0.3, 3).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 4).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32"))
        for prec in ("df64", "f32"):
            t = lat.autotune(prec)
            assert all(v > 0 for v in t["dslash_us"].values())
            assert all(v > 0 for v in t["batch_us"].values())
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        info = lat.cg(fx, fb, 0.05, 1e-10, 5000)
        assert info["return"] == stag.OK
        assert res(dims, U, N, 0.05, fx.export(), b) <= 1.05e-10
