"""The Dslash kernels' neighbour arithmetic (checkerboard decode, hop, wrap
count), run on the host through stag_cb_neighbor, against a brute-force
table built from the site-order definition: full index
i = x + Lx (y + Ly (z + Lz t)), cb = i // 2, parity = (x + y + z + t) % 2,
periodic hops, wraps = number of times a hop crosses the boundary.  Every
site, parity, direction and hop length of lattices whose small extents make
hops alias and wrap twice.  No GPU needed: this stands in for a sanitizer
on the index maths."""
import itertools

import numpy as np
import pytest

from paper_1411_2087_gb300 import stag


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1411_2087_gb300 import build
    build.build()


def brute_force(dims):
    """{(parity, cb): coords} and coords -> (parity, cb)."""
    Lx, Ly, Lz, Lt = dims
    to_cb, from_cb = {}, {}
    for t, z, y, x in itertools.product(range(Lt), range(Lz), range(Ly), range(Lx)):
        i = x + Lx * (y + Ly * (z + Lz * t))
        par = (x + y + z + t) % 2
        to_cb[(x, y, z, t)] = (par, i // 2)
        from_cb[(par, i // 2)] = (x, y, z, t)
    return to_cb, from_cb


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 8), (6, 4, 2, 10), (2, 6, 4, 4), (8, 8, 2, 2)])
def test_every_hop_matches_brute_force(dims):
    to_cb, from_cb = brute_force(dims)
    Vh = int(np.prod(dims)) // 2
    assert len(from_cb) == 2 * Vh  # the decode is a bijection per parity
    for (par, cb), xs in from_cb.items():
        for mu in range(4):
            for s in (1, -1, 3, -3):
                y = list(xs)
                raw = xs[mu] + s
                y[mu] = raw % dims[mu]
                wraps = abs(raw // dims[mu]) if raw < 0 else raw // dims[mu]
                want_par, want_cb = to_cb[tuple(y)]
                got_cb, got_w = stag.cb_neighbor(dims, par, cb, mu, s)
                assert want_par == (par + (s % 2)) % 2
                assert (got_cb, got_w) == (want_cb, wraps), (dims, par, cb, xs, mu, s)


def test_arguments_are_checked():
    for bad in [((3, 2, 2, 2), 0, 0, 0, 1), ((2, 2, 2, 2), 2, 0, 0, 1), ((2, 2, 2, 2), 0, 8, 0, 1),
                ((2, 2, 2, 2), 0, -1, 0, 1), ((2, 2, 2, 2), 0, 0, 4, 1), ((2, 2, 2, 2), 0, 0, 0, 2)]:
        with pytest.raises(stag.StagError) as e:
            stag.cb_neighbor(*bad)
        assert e.value.status == stag.ERR_ARG


def decode(dims, par, cb):
    """Coordinates of checkerboard site cb of parity par, by integer division."""
    Lx, Ly, Lz, Lt = dims
    xh, r = cb % (Lx // 2), cb // (Lx // 2)
    y, r = r % Ly, r // Ly
    z, t = r % Lz, r // Lz
    x = 2 * xh + ((par + y + z + t) & 1)
    return [x, y, z, t]


@pytest.mark.parametrize("dims", [(64, 64, 64, 226), (94, 62, 58, 122), (2, 2, 2, 4096), (4096, 2, 2, 2)])
def test_large_lattices_sampled(dims):
    """The decode divides by multiply and shift; at the largest lattice a
    lattice object accepts (64^3 x 226) and at extents that are not powers
    of two, sampled sites (and the last ones of each parity) hop where the
    integer definition says."""
    Vh = int(np.prod(dims)) // 2
    rng = np.random.default_rng(11)
    cbs = list(rng.integers(0, Vh, 400)) + [0, 1, Vh - 2, Vh - 1]
    for cb in cbs:
        cb = int(cb)
        for par in (0, 1):
            xs = decode(dims, par, cb)
            for mu in range(4):
                for s in (1, -1, 3, -3):
                    y = list(xs)
                    raw = xs[mu] + s
                    y[mu] = raw % dims[mu]
                    wraps = abs(raw // dims[mu]) if raw < 0 else raw // dims[mu]
                    i = y[0] + dims[0] * (y[1] + dims[1] * (y[2] + dims[2] * y[3]))
                    got_cb, got_w = stag.cb_neighbor(dims, par, cb, mu, s)
                    assert (got_cb, got_w) == (i // 2, wraps), (dims, par, cb, xs, mu, s)
