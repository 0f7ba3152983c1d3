"""The pair form of the 16-bit stencil (regs 3): two output sites
(x, y, z, t) and (x, y, z, t + Lt/2) per thread in packed FP32x2 arithmetic,
their loads through a shared-memory ring of cp.async copies, on full links,
12-real links and 12-real three-link links with full one-link links.

* D and M equal the one-site forms bit for bit, for every block size, on
  lattices whose Lt is a multiple of 4 (8, 12, 16), with every boundary sign
  (the t hops wrap on one site of the pair only), and against the oracle to
  the 16-bit tolerance;
* where Lt is not a multiple of 4 (or is 4) the setting falls back to the
  default form, again with the same bits;
* the solvers' M with <p, Mp> block partials (the pair kernel writes one
  partial per block of site pairs) gives a mixed CG with 16-bit inner
  iterations that meets 1e-10 against the oracle in the one-site form's
  iteration count (within max(3, 1 %)).
"""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

BLOCKS = (64, 128, 256, 512)
C1, C3 = 1.2, -0.07


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("compress", [True, False, "long"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 12), (4, 6, 4, 16), (6, 4, 6, 10), (4, 4, 4, 4)])
@pytest.mark.parametrize("bc", [(1.0, 1.0, 1.0, -1.0), (-1.0, 1.0, -1.0, -1.0), (1.0, -1.0, 1.0, 1.0)])
def test_pair_matches_one_site_and_oracle(dims, bc, compress):
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.5, 41).numpy()
    N = oracle.long_links(dims, U)
    psi_e = synth.gaussian_colour_field(Vh, 42).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 43).numpy()
    want_o = oracle.dslash_parity(dims, U, N, 1, psi_e, bc=bc, c1=C1, c3=C3)
    want_e = oracle.dslash_parity(dims, U, N, 0, psi_o, bc=bc, c1=C1, c3=C3)
    want_m = oracle.apply_M(dims, U, N, 0.3, psi_e, bc=bc, c1=C1, c3=C3)
    with stag.Lattice(dims, bc=bc) as lat:
        lat.upload_gauge(U, N, c1=C1, c3=C3, precisions=("f16",), compress12=compress)
        fe = lat.field(stag.EVEN, "f16", psi_e)
        fo = lat.field(stag.ODD, "f16", psi_o)
        oo, oe, om = lat.field(stag.ODD, "f16"), lat.field(stag.EVEN, "f16"), lat.field(stag.EVEN, "f16")

        def run():
            lat.dslash(oo, fe)
            lat.dslash(oe, fo)
            lat.apply_M(om, fe, 0.3)
            return oo.export(), oe.export(), om.export()

        lat.set_tuning("f16", "dslash", 128, 1)
        ref = run()
        assert rel_err(ref[0], want_o) <= 3e-4 and rel_err(ref[1], want_e) <= 3e-4
        assert rel_err(ref[2], want_m) <= 8e-4
        for block in BLOCKS:
            for regs in (2, 3):
                lat.set_tuning("f16", "dslash", block, regs)
                got = run()
                for g, w in zip(got, ref):
                    assert np.array_equal(g, w), (block, regs, dims, bc, compress)


@pytest.mark.parametrize("compress", [True, False, "long"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 6, 4, 12)])
def test_solvers_with_the_pair_form(dims, compress):
    mass = 0.1
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 44).numpy()
    N = oracle.long_links(dims, U)
    b = synth.gaussian_colour_field(Vh, 45).numpy()

    def res(x):
        return np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)

    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f16"), compress12=compress)
        fb = lat.field(stag.EVEN, "df64", b)
        iters = {}
        for block in (64, 256):
            for regs in (1, 3):
                lat.set_tuning("f16", "dslash", block, regs)
                lat.set_tuning("f16", "M", block, regs)
                # mixed CG: the 16-bit iteration's alpha comes from the M
                # kernel's block partials of <p, Mp>; double-float reliable updates
                fx = lat.field(stag.EVEN, "df64")
                info = lat.cg_mixed(fx, fb, mass, 1e-10, 20000, inner="f16")
                assert info["return"] == stag.OK, info
                assert res(fx.export()) <= 1.05e-10, (block, regs, res(fx.export()))
                iters[(block, regs)] = info["iters"]
        # the partial sums differ only in their order
        assert max(iters.values()) - min(iters.values()) <= max(3, 0.01 * min(iters.values())), iters
