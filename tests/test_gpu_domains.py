"""Domain decomposition in t emulated on one GPU (the data movement of the
paper's multi-node runs): slab-by-slab Dslash from depth-3 halo copies and
CG with host-reduced inner products, through the C ABI.

Criteria: the slab-wise Dslash runs the same per-site arithmetic on the same
input values as the single-domain Dslash, so the two agree bit for bit, and
both match the oracle to the per-precision tolerance; any halo shallower
than the three-link reach would leave zeros in the assembled input and
change the result.  The slab-wise CG sums its inner products in another
order than the single-domain graph, so it is held to the solve criteria:
true residual within the tolerance (recomputed by the oracle), iteration
count within max(3, 1%) of the oracle's, and the solution within 1e-12
(times a condition-number estimate) of the oracle's when both solve to
1e-13.
"""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "f16": 3e-4}


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


# (6,4,6,10): Lt = 10 cut into 3 gives slabs 4,3,3 (ragged); k = Lt gives
# one slice per slab (halos of three slices on each side, wrapping at t = 0);
# Lt = 16 with k = 2 has halos that do not cover the lattice.
CASES = [((6, 4, 6, 10), 1), ((6, 4, 6, 10), 3), ((6, 4, 6, 10), 10), ((4, 4, 4, 16), 2),
         ((4, 4, 4, 16), 4), ((4, 4, 4, 16), 16), ((4, 2, 2, 8), 8)]


@pytest.mark.parametrize("dims,k", CASES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_dd_dslash_matches_single_domain_and_oracle(dims, k, prec):
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 41).numpy()
    N = oracle.long_links(dims, U)
    psi_e = synth.gaussian_colour_field(Vh, 42).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 43).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fe = lat.field(stag.EVEN, prec, psi_e)
        fo = lat.field(stag.ODD, prec, psi_o)
        ref_o, ref_e = lat.field(stag.ODD, prec), lat.field(stag.EVEN, prec)
        dd_o, dd_e = lat.field(stag.ODD, prec), lat.field(stag.EVEN, prec)
        lat.dslash(ref_o, fe)
        lat.dslash(ref_e, fo)
        lat.dd_dslash(dd_o, fe, k)
        lat.dd_dslash(dd_e, fo, k)
        got_o, got_e = dd_o.export(), dd_e.export()
        assert np.array_equal(got_o, ref_o.export()) and np.array_equal(got_e, ref_e.export())
    e1 = rel_err(got_o, oracle.dslash_parity(dims, U, N, 1, psi_e))
    e2 = rel_err(got_e, oracle.dslash_parity(dims, U, N, 0, psi_o))
    assert e1 <= TOL[prec] and e2 <= TOL[prec], (e1, e2)


@pytest.mark.parametrize("compress", [True, "long"])
def test_dd_dslash_compressed_links(compress):
    dims, k = (4, 4, 6, 12), 3
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.4, 51).numpy()
    N = oracle.long_links(dims, U)
    psi_e = synth.gaussian_colour_field(Vh, 52).numpy()
    want = oracle.dslash_parity(dims, U, N, 1, psi_e)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("f32", "f16"), compress12=compress)
        for prec in ("f32", "f16"):
            fe = lat.field(stag.EVEN, prec, psi_e)
            ref, dd = lat.field(stag.ODD, prec), lat.field(stag.ODD, prec)
            lat.dslash(ref, fe)
            lat.dd_dslash(dd, fe, k)
            got = dd.export()
            assert np.array_equal(got, ref.export())
            assert rel_err(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("dims,k,mass", [((6, 4, 6, 10), 3, 0.05), ((8, 8, 8, 8), 4, 0.1),
                                         ((4, 4, 4, 8), 8, 0.2)])
def test_dd_cg_matches_oracle(prec, dims, k, mass):
    U = synth.su3_field(dims, 0.3, 61).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 62).numpy()
    _, info_o = oracle.cg(dims, U, N, mass, b, tol=1e-10)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info = lat.dd_cg(fx, fb, mass, k, 1e-10, 5000)
        x = fx.export()
        fy = lat.field(stag.EVEN, prec)
        info1 = lat.cg(fy, fb, mass, 1e-10, 5000)
    assert info["return"] == stag.OK, info
    res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)
    assert res <= 1e-10 * 1.05, res
    assert abs(info["true_rel_resid"] - res) <= 1e-3 * res + 1e-15
    tol_it = max(3, 0.01 * info_o["iters"])
    assert abs(info["iters"] - info_o["iters"]) <= tol_it, (info, info_o)
    assert abs(info["iters"] - info1["iters"]) <= tol_it, (info, info1)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_dd_cg_tight_solution_agrees(prec):
    dims, mass, k = (4, 4, 4, 12), 0.1, 3
    U = synth.su3_field(dims, 0.3, 71).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 72).numpy()
    x_o, _ = oracle.cg(dims, U, N, mass, b, tol=1e-13)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fb = lat.field(stag.EVEN, prec, b)
        fx = lat.field(stag.EVEN, prec)
        info = lat.dd_cg(fx, fb, mass, k, 1e-13, 5000)
        x = fx.export()
    assert info["return"] == stag.OK, info
    kappa = (mass ** 2 + 4 * 4 * (7 / 6) ** 2) / mass ** 2
    assert np.abs(x - x_o).max() / np.abs(x_o).max() <= 1e-12 * kappa


def test_dd_edge_cases():
    dims = (4, 4, 4, 8)
    U = synth.su3_field(dims, 0.3, 81).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("f64",))
        fe = lat.field(stag.EVEN, "f64", synth.gaussian_colour_field(Vh, 82).numpy())
        fo = lat.field(stag.ODD, "f64")
        for bad in (0, -1, 9):
            with pytest.raises(stag.StagError) as e:
                lat.dd_dslash(fo, fe, bad)
            assert e.value.status == stag.ERR_ARG
        # same parity
        fe2 = lat.field(stag.EVEN, "f64")
        with pytest.raises(stag.StagError):
            lat.dd_dslash(fe2, fe, 2)
        # zero source: no iterations, x = 0
        fz = lat.field(stag.EVEN, "f64", np.zeros((Vh, 3), complex))
        info = lat.dd_cg(fe2, fz, 0.1, 2, 1e-10, 100)
        assert info["return"] == stag.OK and info["iters"] == 0
        assert not np.any(fe2.export())
        # iteration limit
        info = lat.dd_cg(fe2, fe, 0.01, 2, 1e-14, 3)
        assert info["return"] == stag.ERR_NOT_CONVERGED and info["iters"] == 3
