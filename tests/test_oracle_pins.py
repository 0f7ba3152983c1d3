"""Pins of the CPU oracle against facts fixed by the mathematics and the paper.

None of these re-types the oracle's formula: each checks a property that a
plausible mistake (dropped term, wrong sign, wrong hop index, transposed or
un-conjugated link, wrong phase convention, wrong CG update) would break:

* free field (unit links): plane waves are eigenvectors with the closed-form
  eigenvalue, pointwise for D and for M = m^2 - D_eo D_oe; the whole dense
  spectrum of M equals the closed-form set;
* anti-Hermiticity of D (D_eo^+ = -D_oe) and Hermiticity/positivity of M;
* gauge covariance under a random SU(3) transform, for D, for the
  three-link products and for the CG solution;
* brute force on 2^4 and 4^4: the dense D assembled from boundary-folded links
  (a different construction of the same operator) equals the oracle, and
  numpy's dense solve equals the oracle CG;
* CG facts: one iteration for an eigenvector source, at most (number of
  distinct eigenvalues) iterations in the free field;
* the c3 = 0 special case is the textbook one-link staggered operator.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import synth

C1, C3 = 9.0 / 8.0, -1.0 / 24.0
BC = (1.0, 1.0, 1.0, -1.0)


def coords(dims):
    """x, y, z, t coordinate arrays in site order."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return [a.reshape(-1) for a in (x, y, z, t)]


def momenta(dims, bc):
    """All lattice momenta allowed by the boundary conditions, per direction."""
    out = []
    for L, b in zip(dims, bc):
        if b > 0:
            out.append([2 * math.pi * n / L for n in range(L)])
        else:
            out.append([math.pi * (2 * n + 1) / L for n in range(L)])
    return out


def plane_wave(dims, p, colour):
    xs = coords(dims)
    phase = np.exp(1j * sum(pm * xm for pm, xm in zip(p, xs)))
    return phase[:, None] * np.asarray(colour)[None, :]


def f_naik(p, c1=C1, c3=C3):
    return c1 * math.sin(p) + c3 * math.sin(3 * p)


def eta(dims):
    x, y, z, t = coords(dims)
    return [np.ones_like(x), (-1.0) ** x, (-1.0) ** (x + y), (-1.0) ** (x + y + z)]


def rand_colour(n, seed):
    return synth.gaussian_colour_field(n, seed).numpy()


def fields(dims, eps, seed):
    U = synth.su3_field(dims, eps, seed).numpy()
    N = oracle.long_links(dims, U)
    return U, N


def inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


# --------------------------------------------------------------------------
# generator
# --------------------------------------------------------------------------

@pytest.mark.parametrize("eps", [0.0, 0.3, 1.0])
def test_generator_special_unitary(eps):
    U = synth.su3_field((4, 4, 2, 2), eps, 7).numpy()
    eye = np.eye(3)
    err_u = np.abs(np.einsum("...ji,...jk->...ik", U.conj(), U) - eye).max()
    err_d = np.abs(np.linalg.det(U) - 1).max()
    assert err_u < 1e-14 and err_d < 1e-14
    if eps == 0.0:
        assert np.abs(U - eye).max() == 0


def test_generator_seeded_and_chunk_independent():
    a = synth.su3_field((4, 2, 2, 2), 0.3, 11).numpy()
    b = synth.su3_field((4, 2, 2, 2), 0.3, 11, chunk=5).numpy()
    # same draws; the matrix exponential may round differently per chunk
    assert np.abs(a - b).max() < 1e-14
    assert np.array_equal(a, synth.su3_field((4, 2, 2, 2), 0.3, 11).numpy())
    c = synth.su3_field((4, 2, 2, 2), 0.3, 12).numpy()
    assert not np.allclose(a, c)


# --------------------------------------------------------------------------
# three-link products
# --------------------------------------------------------------------------

def shift(field, dims, mu, s):
    """field at x + s*mu (periodic), for field shaped [V, ...]."""
    Lx, Ly, Lz, Lt = dims
    f = field.reshape((Lt, Lz, Ly, Lx) + field.shape[1:])
    axis = 3 - mu
    return np.roll(f, -s, axis=axis).reshape(field.shape)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 4), (8, 4, 4, 2)])
def test_long_links_are_three_link_products(dims):
    U = synth.su3_field(dims, 0.5, 3).numpy()
    N = oracle.long_links(dims, U)
    for mu in range(4):
        want = U[mu] @ shift(U[mu], dims, mu, 1) @ shift(U[mu], dims, mu, 2)
        assert np.abs(N[mu] - want).max() < 1e-14
    # SU(3) closure
    assert np.abs(np.linalg.det(N) - 1).max() < 1e-13


# --------------------------------------------------------------------------
# (a) free field closed form
# --------------------------------------------------------------------------

FREE_DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (8, 2, 4, 6)]


@pytest.mark.parametrize("dims", FREE_DIMS)
@pytest.mark.parametrize("bc", [BC, (1.0, 1.0, 1.0, 1.0), (-1.0, 1.0, -1.0, -1.0)])
def test_free_field_plane_wave_pointwise(dims, bc):
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    assert np.abs(N - U).max() == 0
    rng = np.random.default_rng(5)
    ps = momenta(dims, bc)
    etas = eta(dims)
    for trial in range(4):
        p = [rng.choice(pl) for pl in ps]
        c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        psi = plane_wave(dims, p, c)
        got = oracle.dslash_full(dims, U, N, psi, bc=bc)
        factor = sum(etas[mu] * 2j * f_naik(p[mu]) for mu in range(4))
        want = factor[:, None] * psi
        assert np.abs(got - want).max() < 1e-13 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("dims", FREE_DIMS)
def test_free_field_M_eigenvalue(dims):
    mass = 0.1
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    ps = momenta(dims, BC)
    rng = np.random.default_rng(6)
    for trial in range(4):
        p = [rng.choice(pl) for pl in ps]
        c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        psi_e = oracle.full_to_cb(dims, plane_wave(dims, p, c), 0)
        lam = mass ** 2 + 4 * sum(f_naik(pm) ** 2 for pm in p)
        got = oracle.apply_M(dims, U, N, mass, psi_e)
        assert np.abs(got - lam * psi_e).max() < 1e-13 * lam


def dense_M(dims, U, N, mass, bc=BC, c1=C1, c3=C3):
    n = 3 * (np.prod(dims) // 2)
    M = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        M[:, k] = oracle.apply_M(dims, U, N, mass, e.reshape(-1, 3), bc=bc, c1=c1, c3=c3).reshape(-1)
    return M


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 2, 2), (4, 4, 4, 4)])
def test_free_field_dense_spectrum(dims):
    mass = 0.2
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    M = dense_M(dims, U, N, mass)
    ev = np.linalg.eigvalsh(M)
    lams = [mass ** 2 + 4 * sum(f_naik(pm) ** 2 for pm in p)
            for p in itertools.product(*momenta(dims, BC))]
    want = np.sort(np.repeat(lams, 3))
    got = np.sort(np.repeat(ev, 2))
    assert np.abs(got - want).max() < 1e-12


def test_free_field_naik_improvement():
    """f(p) = p - (3/40) p^5 + O(p^7): with c1 = 9/8, c3 = -1/24 the Naik term
    cancels the O(p^3) error of sin p, and f(pi/2) = c1 - c3 = 7/6."""
    for p in [1e-1, 5e-2, 2e-2]:
        assert abs((f_naik(p) - p) / p ** 5 + 0.075) < 0.05
        assert abs(math.sin(p) - p) > 0.1 * p ** 3
    assert abs(f_naik(math.pi / 2) - 7 / 6) < 1e-15


# --------------------------------------------------------------------------
# (g) c3 = 0: the textbook one-link staggered operator
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_one_link_special_case(dims):
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    ps = momenta(dims, BC)
    rng = np.random.default_rng(8)
    etas = eta(dims)
    for trial in range(3):
        p = [rng.choice(pl) for pl in ps]
        c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        psi = plane_wave(dims, p, c)
        got = oracle.dslash_full(dims, U, N, psi, c1=1.0, c3=0.0)
        factor = sum(etas[mu] * 2j * math.sin(p[mu]) for mu in range(4))
        assert np.abs(got - factor[:, None] * psi).max() < 1e-13
    # with random links the long links must drop out completely
    U2, N2 = fields(dims, 0.4, 9)
    psi = rand_colour(np.prod(dims), 10)
    a = oracle.dslash_full(dims, U2, N2, psi, c1=1.0, c3=0.0)
    b = oracle.dslash_full(dims, U2, np.zeros_like(N2), psi, c1=1.0, c3=0.0)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# (b) anti-Hermiticity
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (8, 8, 8, 8)])
@pytest.mark.parametrize("eps", [0.3, 1.0])
def test_anti_hermitian(dims, eps):
    U, N = fields(dims, eps, 21)
    Vh = np.prod(dims) // 2
    xe = rand_colour(Vh, 22)
    yo = rand_colour(Vh, 23)
    lhs = inner(xe, oracle.dslash_parity(dims, U, N, 0, yo))
    rhs = -inner(oracle.dslash_parity(dims, U, N, 1, xe), yo)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # full lattice: <a, D b> = -<D a, b>
    a = rand_colour(2 * Vh, 24)
    b = rand_colour(2 * Vh, 25)
    l2 = inner(a, oracle.dslash_full(dims, U, N, b))
    r2 = -inner(oracle.dslash_full(dims, U, N, a), b)
    assert abs(l2 - r2) < 1e-13 * abs(l2)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 8)])
def test_M_hermitian_positive(dims):
    mass = 0.05
    U, N = fields(dims, 0.3, 31)
    Vh = np.prod(dims) // 2
    x = rand_colour(Vh, 32)
    y = rand_colour(Vh, 33)
    a = inner(x, oracle.apply_M(dims, U, N, mass, y))
    b = inner(oracle.apply_M(dims, U, N, mass, x), y)
    assert abs(a - b) < 1e-13 * abs(a)
    xMx = inner(x, oracle.apply_M(dims, U, N, mass, x))
    assert abs(xMx.imag) < 1e-13 * abs(xMx)
    assert xMx.real >= mass ** 2 * inner(x, x).real


# --------------------------------------------------------------------------
# (c) gauge covariance
# --------------------------------------------------------------------------

def gauge_rotate(dims, U, g):
    Up = np.empty_like(U)
    for mu in range(4):
        Up[mu] = g @ U[mu] @ shift(g, dims, mu, 1).conj().transpose(0, 2, 1)
    return Up


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (8, 8, 8, 8)])
def test_gauge_covariance_dslash(dims):
    U, N = fields(dims, 0.3, 41)
    g = synth.gauge_transform(dims, 42).numpy()
    Up = gauge_rotate(dims, U, g)
    Np = oracle.long_links(dims, Up)
    # the three-link product of rotated links is the rotated three-link product
    for mu in range(4):
        Nrot = g @ N[mu] @ shift(g, dims, mu, 3).conj().transpose(0, 2, 1)
        assert np.abs(Np[mu] - Nrot).max() < 1e-13
    psi = rand_colour(np.prod(dims), 43)
    gpsi = np.einsum("vab,vb->va", g, psi)
    lhs = oracle.dslash_full(dims, Up, Np, gpsi)
    rhs = np.einsum("vab,vb->va", g, oracle.dslash_full(dims, U, N, psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_gauge_covariance_cg():
    dims = (4, 4, 4, 4)
    mass = 0.1
    U, N = fields(dims, 0.3, 51)
    g = synth.gauge_transform(dims, 52).numpy()
    Up = gauge_rotate(dims, U, g)
    Np = oracle.long_links(dims, Up)
    Vh = np.prod(dims) // 2
    b = rand_colour(Vh, 53)
    # g restricted to even sites in checkerboard order
    par = oracle.parity_mask(dims)
    idx = np.nonzero(par == 0)[0]
    g_even = np.empty((Vh, 3, 3), dtype=np.complex128)
    g_even[idx // 2] = g[idx]
    x, info = oracle.cg(dims, U, N, mass, b, tol=1e-13)
    xp, infop = oracle.cg(dims, Up, Np, mass, np.einsum("vab,vb->va", g_even, b), tol=1e-13)
    assert info["status"] == 0 and infop["status"] == 0
    gx = np.einsum("vab,vb->va", g_even, x)
    assert np.abs(xp - gx).max() < 1e-11 * np.abs(gx).max()


# --------------------------------------------------------------------------
# (d) brute force on tiny lattices
# --------------------------------------------------------------------------

def dense_D_folded(dims, U, bc=BC, c1=C1, c3=C3):
    """Dense D assembled a second way: the boundary signs are folded into the
    links on the last slice and the three-link term uses the product of those
    folded links, with purely periodic neighbour indexing."""
    V = int(np.prod(dims))
    xs = coords(dims)
    etas = eta(dims)
    Uf = U.copy()
    for mu in range(4):
        last = xs[mu] == dims[mu] - 1
        Uf[mu][last] *= bc[mu]
    Nf = np.empty_like(Uf)
    for mu in range(4):
        Nf[mu] = Uf[mu] @ shift(Uf[mu], dims, mu, 1) @ shift(Uf[mu], dims, mu, 2)
    idx = np.arange(V)
    D = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    for mu in range(4):
        fwd1 = shift(idx, dims, mu, 1)
        bwd1 = shift(idx, dims, mu, -1)
        fwd3 = shift(idx, dims, mu, 3)
        bwd3 = shift(idx, dims, mu, -3)
        for i in range(V):
            e = etas[mu][i]
            for (j, A, c) in ((fwd1[i], Uf[mu][i], c1), (fwd3[i], Nf[mu][i], c3)):
                D[3 * i:3 * i + 3, 3 * j:3 * j + 3] += e * c * A
            for (j, A, c) in ((bwd1[i], Uf[mu][bwd1[i]], c1), (bwd3[i], Nf[mu][bwd3[i]], c3)):
                D[3 * i:3 * i + 3, 3 * j:3 * j + 3] -= e * c * A.conj().T
    return D


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2), (4, 4, 4, 4)])
@pytest.mark.parametrize("c3", [C3, 0.0])
def test_dense_D_matches_folded_construction(dims, c3):
    U, N = fields(dims, 0.6, 61)
    D = dense_D_folded(dims, U, c3=c3)
    V = int(np.prod(dims))
    psi = rand_colour(V, 62)
    got = oracle.dslash_full(dims, U, N, psi, c3=c3)
    want = (D @ psi.reshape(-1)).reshape(V, 3)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()
    assert np.abs(D + D.conj().T).max() < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_dense_solve_matches_cg(dims):
    mass = 0.1
    U, N = fields(dims, 0.3, 71)
    M = dense_M(dims, U, N, mass)
    assert np.abs(M - M.conj().T).max() < 1e-13
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= mass ** 2 * (1 - 1e-12)
    Vh = np.prod(dims) // 2
    b = rand_colour(Vh, 72)
    want = np.linalg.solve(M, b.reshape(-1)).reshape(Vh, 3)
    x, info = oracle.cg(dims, U, N, mass, b, tol=1e-13)
    assert info["status"] == 0
    assert info["true_rel_resid"] < 1e-12
    kappa = ev.max() / ev.min()
    assert np.abs(x - want).max() / np.abs(want).max() < 1e-12 * max(1.0, kappa) + 1e-12


# --------------------------------------------------------------------------
# CG facts
# --------------------------------------------------------------------------

def test_cg_eigenvector_one_iteration():
    dims = (4, 4, 4, 8)
    mass = 0.3
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    p = [math.pi / 2, 2 * math.pi / 4, 0.0, 3 * math.pi / 8]
    b = oracle.full_to_cb(dims, plane_wave(dims, p, [1.0, 0.5j, -0.25]), 0)
    lam = mass ** 2 + 4 * sum(f_naik(pm) ** 2 for pm in p)
    x, info = oracle.cg(dims, U, N, mass, b, tol=1e-12, history=True)
    assert info["iters"] == 1
    assert abs(info["history"][0][0] - 1 / lam) < 1e-14 / lam
    assert np.abs(x - b / lam).max() < 1e-13


def test_cg_free_field_distinct_eigenvalue_bound():
    dims = (4, 4, 4, 4)
    mass = 0.2
    U = synth.unit_gauge_field(dims).numpy()
    N = oracle.long_links(dims, U)
    lams = {round(mass ** 2 + 4 * sum(f_naik(pm) ** 2 for pm in p), 10)
            for p in itertools.product(*momenta(dims, BC))}
    b = rand_colour(np.prod(dims) // 2, 81)
    x, info = oracle.cg(dims, U, N, mass, b, tol=1e-12)
    assert info["status"] == 0
    assert info["iters"] <= len(lams) + 1


def test_cg_zero_source_and_maxiter():
    dims = (4, 4, 4, 4)
    U, N = fields(dims, 0.3, 91)
    Vh = np.prod(dims) // 2
    x, info = oracle.cg(dims, U, N, 0.1, np.zeros((Vh, 3)), tol=1e-10)
    assert info["iters"] == 0 and info["status"] == 0 and not np.any(x)
    b = rand_colour(Vh, 92)
    x, info = oracle.cg(dims, U, N, 0.01, b, tol=1e-14, max_iter=3)
    assert info["status"] == oracle.CG_NOT_CONVERGED and info["iters"] == 3


def test_cg_history_consistent():
    """alpha_k = |r_k|^2 / <p_k, M p_k> and beta_k = |r_{k+1}|^2/|r_k|^2; the
    recorded residual norms must agree with the residual recomputed from x
    after the last iteration."""
    dims = (4, 4, 4, 4)
    mass = 0.1
    U, N = fields(dims, 0.3, 93)
    b = rand_colour(np.prod(dims) // 2, 94)
    x, info = oracle.cg(dims, U, N, mass, b, tol=1e-10, history=True)
    h = info["history"]
    rr = np.concatenate([[np.vdot(b, b).real], h[:, 2]])
    assert np.allclose(h[:, 1], rr[1:] / rr[:-1], rtol=1e-14)
    true_r = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)
    assert abs(true_r - info["true_rel_resid"]) < 1e-14
    assert info["true_rel_resid"] < 1e-10 * 1.5


def test_dslash_sites_equals_full_parity():
    dims = (4, 6, 2, 8)
    U, N = fields(dims, 0.3, 95)
    Vh = np.prod(dims) // 2
    psi = rand_colour(Vh, 96)
    full = oracle.dslash_parity(dims, U, N, 1, psi)
    par = oracle.parity_mask(dims)
    odd = np.nonzero(par == 1)[0]
    pick = odd[::7]
    got = oracle.dslash_sites(dims, U, N, pick, psi)
    assert np.array_equal(got, full[pick // 2])
