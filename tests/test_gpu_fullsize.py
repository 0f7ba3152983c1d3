"""Parity at the bench's sizes and launch configuration: the whole 32^3x64
Dslash against the oracle in both parities and precisions, the CG solve there
checked by the oracle's residual, and 4096 sampled sites of the 48^3x96
Dslash."""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu


def gen(dims, eps, seed):
    dev = torch.device("cuda", 0)
    U = synth.su3_field(dims, eps, seed, device=dev)
    torch.cuda.synchronize()
    return U


def test_dslash_32x32x32x64_full():
    dims = (32, 32, 32, 64)
    Vh = int(np.prod(dims)) // 2
    U = gen(dims, 0.3, 1001)
    Uh = U.cpu().numpy()
    N = oracle.long_links(dims, Uh)
    psi_e = synth.gaussian_colour_field(Vh, 1101).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 1102).numpy()
    want_o = oracle.dslash_parity(dims, Uh, N, 1, psi_e)
    want_e = oracle.dslash_parity(dims, Uh, N, 0, psi_o)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64", "f64"))
        for prec in ("df64", "f64"):
            fe = lat.field(stag.EVEN, prec, psi_e)
            fo = lat.field(stag.ODD, prec, psi_o)
            oo = lat.field(stag.ODD, prec)
            oe = lat.field(stag.EVEN, prec)
            lat.dslash(oo, fe)
            lat.dslash(oe, fo)
            for got, want in ((oo.export(), want_o), (oe.export(), want_e)):
                err = np.abs(got - want).max() / np.abs(want).max()
                assert err <= 1e-12, (prec, err)
            for f in (fe, fo, oo, oe):
                f.destroy()
        # the bench step: CG at m = 0.02 to 1e-10, residual by the oracle
        b = synth.gaussian_colour_field(Vh, 1101).numpy()
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        info = lat.cg(fx, fb, 0.02, 1e-10, 20000)
        assert info["return"] == stag.OK
        x = fx.export()
    r = np.linalg.norm(b - oracle.apply_M(dims, Uh, N, 0.02, x)) / np.linalg.norm(b)
    assert r <= 1.05e-10, r


def test_dslash_48x48x48x96_sampled():
    dims = (48, 48, 48, 96)
    V = int(np.prod(dims))
    Vh = V // 2
    U = gen(dims, 0.35, 1002)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        N_dev = lat.long_links(U)
        Uh = U.cpu().numpy()
        Nh = N_dev.cpu().numpy()
        del N_dev
        psi = synth.gaussian_colour_field(Vh, 1103).numpy()
        fe = lat.field(stag.EVEN, "df64", psi)
        fo = lat.field(stag.ODD, "df64")
        lat.dslash(fo, fe)
        got = fo.export()
    # the long links the GPU built are checked on sampled sites too
    rng = np.random.default_rng(7)
    par = None
    sites = rng.choice(V, 20000, replace=False)
    x = sites % 48
    y = (sites // 48) % 48
    z = (sites // (48 * 48)) % 48
    t = sites // (48 * 48 * 48)
    odd = sites[((x + y + z + t) & 1) == 1][:4096]
    Noracle = oracle.long_links(dims, Uh)
    for mu in range(4):
        assert np.abs(Noracle[mu][odd] - Nh[mu][odd]).max() < 1e-13
    want = oracle.dslash_sites(dims, Uh, Noracle, odd, psi)
    err = np.abs(got[odd // 2] - want).max() / np.abs(want).max()
    assert err <= 1e-12, err


def test_mixed_f16_c12_48x48x48x96_oracle_residual():
    """The mixed-precision bench configuration (16-bit inner iterations on
    12-real links, double-float reliable updates, 48^3x96, m = 0.01), with
    the 16-bit kernels in the two-site form the bench's autotuner picks: the
    16-bit Dslash on 4096 sampled sites against the oracle, and the returned
    solution's true residual recomputed by the oracle."""
    dims, mass = (48, 48, 48, 96), 0.01
    V = int(np.prod(dims))
    Vh = V // 2
    U = gen(dims, 0.35, 1002)
    b = synth.gaussian_colour_field(Vh, 1102).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"), compress12=True)
        Uh = U.cpu().numpy()
        del U
        for kind in ("dslash", "M"):
            lat.set_tuning("f16", kind, 256, 3)
        fe16 = lat.field(stag.EVEN, "f16", b)
        fo16 = lat.field(stag.ODD, "f16")
        lat.dslash(fo16, fe16)
        d16 = fo16.export()
        fe16.destroy()
        fo16.destroy()
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        info = lat.cg_mixed(fx, fb, mass, 1e-10, 20000, inner="f16")
        x = fx.export()
    assert info["return"] == stag.OK, info
    N = oracle.long_links(dims, Uh)
    rng = np.random.default_rng(8)
    sites = rng.choice(V, 20000, replace=False)
    xs, ys, zs, ts = sites % 48, (sites // 48) % 48, (sites // 2304) % 48, sites // 110592
    odd = sites[((xs + ys + zs + ts) & 1) == 1][:4096]
    want = oracle.dslash_sites(dims, Uh, N, odd, b)
    err = np.abs(d16[odd // 2] - want).max() / np.abs(want).max()
    assert err <= 3e-4, err
    r = np.linalg.norm(b - oracle.apply_M(dims, Uh, N, mass, x)) / np.linalg.norm(b)
    assert r <= 1.05e-10, r
    assert abs(info["true_rel_resid"] - r) <= 1e-2 * r


def test_multishift_24x24x24x48_oracle_residuals():
    """The multishift bench configuration (12 shifts geomspace(1e-4, 0.5) on
    24^3x48, m = 0.02): every shifted solution's true residual recomputed by
    the oracle."""
    dims, mass = (24, 24, 24, 48), 0.02
    Vh = int(np.prod(dims)) // 2
    shifts = list(np.geomspace(1e-4, 0.5, 12))
    U = gen(dims, 0.3, 1004)
    b = synth.gaussian_colour_field(Vh, 3000).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        Uh = U.cpu().numpy()
        fb = lat.field(stag.EVEN, "df64", b)
        xs = [lat.field(stag.EVEN, "df64") for _ in shifts]
        st, infos = lat.cg_multishift(xs, fb, shifts, mass, 1e-10, 20000)
        sols = [x.export() for x in xs]
    assert st == stag.OK, infos
    N = oracle.long_links(dims, Uh)
    nb = np.linalg.norm(b)
    for sh, x in zip(shifts, sols):
        r = np.linalg.norm(b - oracle.apply_M(dims, Uh, N, mass, x) - sh * x) / nb
        assert r <= 1.05e-10, (sh, r)


def test_batched_bench_configuration_oracle_residuals():
    """The batched bench configuration (16 right-hand sides: 6 on 16^4, 5 on
    24^3x48, 5 on 32^3x64, m = 0.02, double-float, one graph launch): every
    solution's true residual recomputed by the oracle."""
    specs = [((16, 16, 16, 16), 6, 1003), ((24, 24, 24, 48), 5, 1004), ((32, 32, 32, 64), 5, 1005)]
    mass = 0.02
    lats, systems, host = [], [], []
    try:
        for dims, nrhs, seed in specs:
            U = gen(dims, 0.3, seed)
            lat = stag.Lattice(dims)
            lat.upload_gauge(U, None, precisions=("df64",))
            lats.append(lat)
            Uh = U.cpu().numpy()
            del U
            Vh = int(np.prod(dims)) // 2
            for k in range(nrhs):
                b = synth.gaussian_colour_field(Vh, 3000 + 17 * seed + k).numpy()
                systems.append((lat, lat.field(stag.EVEN, "df64"), lat.field(stag.EVEN, "df64", b), mass))
                host.append((dims, Uh, b))
        st, infos = stag.cg_batched(systems, 1e-10, 20000)
        assert st == stag.OK, infos
        sols = [s[1].export() for s in systems]
    finally:
        for lat in lats:
            lat.close()
    longs = {}
    for (dims, Uh, b), x in zip(host, sols):
        if dims not in longs:
            longs[dims] = oracle.long_links(dims, Uh)
        r = np.linalg.norm(b - oracle.apply_M(dims, Uh, longs[dims], mass, x)) / np.linalg.norm(b)
        assert r <= 1.05e-10, (dims, r)
