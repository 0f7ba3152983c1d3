"""Pins of the oracle's gauge-covariant convolution (the learned
preconditioner's layer): identity weights, the free-field closed form of a
plane wave, gauge covariance, the adjoint relation that defines the backward
pass, and finite differences of the training loss against the gradient the
adjoint relation gives."""
import math

import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import synth

BC = (1.0, 1.0, 1.0, -1.0)


def rand_w(cout, cin, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal((9, cout, cin)) + 1j * rng.standard_normal((9, cout, cin)))


def adjoint_w(W):
    """W^+[dbar][i][o] = conj(W[d][o][i]) with dbar the reversed hop."""
    A = np.conj(np.transpose(W, (0, 2, 1))).copy()
    out = A.copy()
    for mu in range(4):
        out[1 + 2 * mu] = A[2 + 2 * mu]
        out[2 + 2 * mu] = A[1 + 2 * mu]
    return out


def colour(n, c, seed):
    return np.stack([synth.gaussian_colour_field(n, seed + k).numpy() for k in range(c)])


def coords(dims):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return [a.reshape(-1) for a in (x, y, z, t)]


def shift(field, dims, mu, s):
    Lx, Ly, Lz, Lt = dims
    f = field.reshape((Lt, Lz, Ly, Lx) + field.shape[1:])
    return np.roll(f, -s, axis=3 - mu).reshape(field.shape)


def test_identity_weights():
    dims = (4, 2, 4, 2)
    U = synth.su3_field(dims, 0.5, 1).numpy()
    V = int(np.prod(dims))
    psi = colour(V, 3, 10)
    W = np.zeros((9, 3, 3), complex)
    W[0] = np.eye(3)
    assert np.array_equal(oracle.covconv(dims, U, W, psi), psi)


@pytest.mark.parametrize("bc", [BC, (1.0, -1.0, 1.0, 1.0)])
def test_free_field_plane_wave(bc):
    dims = (4, 6, 2, 8)
    V = int(np.prod(dims))
    U = synth.unit_gauge_field(dims).numpy()
    xs = coords(dims)
    rng = np.random.default_rng(3)
    p = [(2 * math.pi * rng.integers(L) + (math.pi if b < 0 else 0)) / L for L, b in zip(dims, bc)]
    c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    wave = np.exp(1j * sum(pm * xm for pm, xm in zip(p, xs)))[:, None] * c
    W = rand_w(2, 1, 4)
    y = oracle.covconv(dims, U, W, wave[None], bc)
    for o in range(2):
        factor = W[0, o, 0] + sum(W[1 + 2 * m, o, 0] * np.exp(1j * p[m]) +
                                  W[2 + 2 * m, o, 0] * np.exp(-1j * p[m]) for m in range(4))
        assert np.abs(y[o] - factor * wave).max() < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 2, 6)
    V = int(np.prod(dims))
    U = synth.su3_field(dims, 0.6, 5).numpy()
    g = synth.gauge_transform(dims, 6).numpy()
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ shift(g, dims, mu, 1).conj().transpose(0, 2, 1)
    psi = colour(V, 2, 20)
    W = rand_w(3, 2, 7)
    gpsi = np.einsum("vab,cvb->cva", g, psi)
    lhs = oracle.covconv(dims, Ug, W, gpsi)
    rhs = np.einsum("vab,cvb->cva", g, oracle.covconv(dims, U, W, psi))
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 4)])
def test_adjoint_relation(dims):
    V = int(np.prod(dims))
    U = synth.su3_field(dims, 0.7, 8).numpy()
    W = rand_w(3, 2, 9)
    a = colour(V, 3, 30)
    b = colour(V, 2, 40)
    lhs = np.vdot(a.reshape(-1), oracle.covconv(dims, U, W, b).reshape(-1))
    rhs = np.vdot(oracle.covconv(dims, U, adjoint_w(W), a).reshape(-1), b.reshape(-1))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def analytic_grad(dims, U, Ws, rs, es):
    """dL/dW* from the adjoint relation: backward pass of the linear net."""
    grads = [np.zeros_like(W) for W in Ws]
    V = int(np.prod(dims))
    for r, e in zip(rs, es):
        acts = [oracle.cb_to_full(dims, r, 0)[None]]
        for W in Ws:
            acts.append(oracle.covconv(dims, U, W, acts[-1]))
        z = oracle.full_to_cb(dims, acts[-1][0], 0)
        g = oracle.cb_to_full(dims, (z - e) / np.vdot(e, e).real, 0)[None]
        for li in range(len(Ws) - 1, -1, -1):
            W = Ws[li]
            a = acts[li]
            cout, cin = W.shape[1], W.shape[2]
            for d in range(9):
                sel = np.zeros((9, 1, 1), complex)
                sel[d] = 1
                for i in range(cin):
                    h = oracle.covconv(dims, U, sel, a[i:i + 1])[0]
                    for o in range(cout):
                        grads[li][d, o, i] += np.vdot(h.reshape(-1), g[o].reshape(-1))
            g = oracle.covconv(dims, U, adjoint_w(W), g)
    return grads


def test_loss_gradient_finite_differences():
    dims = (2, 2, 2, 4)
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.5, 11).numpy()
    Ws = [rand_w(2, 1, 12), rand_w(2, 2, 13), rand_w(1, 2, 14)]
    rs = [synth.gaussian_colour_field(Vh, 50 + k).numpy() for k in range(2)]
    es = [synth.gaussian_colour_field(Vh, 60 + k).numpy() for k in range(2)]
    grads = analytic_grad(dims, U, Ws, rs, es)
    h = 1e-6
    for li, W in enumerate(Ws):
        for idx in np.ndindex(W.shape):
            for unit in (1.0, 1j):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[li][idx] += unit * h
                Wm[li][idx] -= unit * h
                fd = (oracle.net_loss(dims, U, Wp, rs, es) - oracle.net_loss(dims, U, Wm, rs, es)) / (2 * h)
                an = 2 * (grads[li][idx].real if unit == 1.0 else grads[li][idx].imag)
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, idx, unit, fd, an)


def test_net_ignores_odd_input_and_is_linear():
    dims = (4, 4, 2, 2)
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.4, 15).numpy()
    Ws = [rand_w(4, 1, 16), rand_w(4, 4, 17), rand_w(1, 4, 18)]
    r1 = synth.gaussian_colour_field(Vh, 70).numpy()
    r2 = synth.gaussian_colour_field(Vh, 71).numpy()
    z = oracle.net_apply(dims, U, Ws, 2.0 * r1 - 0.5j * r2)
    z1 = oracle.net_apply(dims, U, Ws, r1)
    z2 = oracle.net_apply(dims, U, Ws, r2)
    assert np.abs(z - (2.0 * z1 - 0.5j * z2)).max() < 1e-12 * np.abs(z).max()


@pytest.mark.parametrize("dims,bc", [((4, 4, 2, 6), BC), ((2, 4, 4, 4), (-1.0, 1.0, -1.0, 1.0))])
def test_phased_links_give_the_one_link_dslash(dims, bc):
    """One layer on the phased links with weight +1 on every forward hop and
    -1 on every backward hop is the one-link staggered operator: the oracle's
    Dslash with c1 = 1 and c3 = 0 (pinned itself by the free-field closed
    form).  A wrong phase convention, a phase on the wrong site or a missing
    phase in one direction breaks the equality."""
    V = int(np.prod(dims))
    U = synth.su3_field(dims, 0.4, 31).numpy()
    N = oracle.long_links(dims, U)
    psi = synth.gaussian_colour_field(V, 32).numpy()
    W = np.zeros((9, 1, 1), complex)
    for mu in range(4):
        W[1 + 2 * mu] = 1.0
        W[2 + 2 * mu] = -1.0
    got = oracle.covconv(dims, oracle.phased_links(dims, U), W, psi[None], bc)[0]
    want = oracle.dslash_full(dims, U, N, psi, bc, c1=1.0, c3=0.0)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # the raw links do not give it
    raw = oracle.covconv(dims, U, W, psi[None], bc)[0]
    assert np.abs(raw - want).max() > 0.1 * np.abs(want).max()


def _path_weights(c0, C):
    """Layer weights (1 -> 8 -> 8 -> 1) whose even-to-even action is
    c0 r + sum_{a,b} C[a][b] T_a T_b r (hop index 2 mu: +mu, 2 mu + 1: -mu):
    hop b into channel b, the identity in between, hop a out of channel b
    with weight C[a][b]; paths of odd length land on odd sites."""
    W1 = np.zeros((9, 8, 1), complex)
    W2 = np.zeros((9, 8, 8), complex)
    W3 = np.zeros((9, 1, 8), complex)
    for d in range(1, 9):
        W1[d, d - 1, 0] = 1.0
    W1[0, 0, 0] = 1.0
    W2[0] = np.eye(8)
    for a in range(1, 9):
        W3[a, 0, :] = C[a - 1, :]
    W3[0, 0, 0] = c0
    return [W1, W2, W3]


def test_phased_links_let_the_net_precondition_further():
    """The least-squares optimum of the residual loss over the net's 65 path
    coefficients, on CG residuals of the oracle's M (4^4, m = 0.05): with
    phased links flexible CG needs clearly fewer iterations than with raw
    links, whose translation-invariant weights cannot form the operator's
    turning two-hop paths."""
    dims, mass = (4, 4, 4, 4), 0.05
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 41).numpy()
    N = oracle.long_links(dims, U)

    def M(x):
        return oracle.apply_M(dims, U, N, mass, x)

    def cg(b, prec):
        x = np.zeros_like(b)
        r = b.copy()
        z = prec(r)
        p = z.copy()
        rz = np.vdot(r, z).real
        res = []
        for k in range(1, 2000):
            Ap = M(p)
            al = rz / np.vdot(p, Ap).real
            x += al * p
            r -= al * Ap
            res.append(r.copy())
            if np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b):
                return k, res
            z = prec(r)
            rz2 = np.vdot(r, z).real
            p = z + (rz2 / rz) * p
            rz = rz2
        return -1, res

    b0 = synth.gaussian_colour_field(Vh, 42).numpy()
    plain, res = cg(b0, lambda r: r)
    pairs = res[:: max(1, len(res) // 8)][:8]
    b = synth.gaussian_colour_field(Vh, 43).numpy()
    iters = {}
    for name, L in (("raw", U), ("phased", oracle.phased_links(dims, U))):
        A, y = [], []
        for r in pairs:
            w = 1.0 / np.linalg.norm(r)
            cols = [M(r)]
            for a in range(8):
                for bb in range(8):
                    C = np.zeros((8, 8), complex)
                    C[a, bb] = 1.0
                    cols.append(M(oracle.net_apply(dims, L, _path_weights(0.0, C), r)))
            A.append(np.stack([c.reshape(-1) for c in cols], 1) * w)
            y.append(r.reshape(-1) * w)
        th = np.linalg.lstsq(np.concatenate(A), np.concatenate(y), rcond=None)[0]
        W = _path_weights(th[0], th[1:].reshape(8, 8))
        iters[name] = cg(b, lambda r: oracle.net_apply(dims, L, W, r))[0]
    assert 0 < iters["phased"] < iters["raw"] < plain
    assert plain / iters["phased"] >= 1.15 * plain / iters["raw"], (plain, iters)


@pytest.mark.parametrize("mistake", ["own_coordinate", "later_coordinates", "t_only", "y_coordinate_missing"])
def test_phased_link_pin_catches_plausible_mistakes(mistake):
    """Phase conventions a reader could plausibly write instead: each, used
    in place of oracle.phased_links, breaks the one-link Dslash equality
    that pins the helper."""
    dims, bc = (4, 4, 2, 6), BC
    V = int(np.prod(dims))
    U = synth.su3_field(dims, 0.4, 31).numpy()
    N = oracle.long_links(dims, U)
    psi = synth.gaussian_colour_field(V, 32).numpy()
    x = coords(dims)
    out = U.copy()
    zero = np.zeros(V, dtype=np.int64)
    for mu in range(4):
        if mistake == "own_coordinate":
            e = sum((x[nu] for nu in range(mu + 1)), zero)
        elif mistake == "later_coordinates":
            e = sum((x[nu] for nu in range(mu + 1, 4)), zero)
        elif mistake == "t_only":
            e = sum((x[nu] for nu in range(mu)), zero) if mu == 3 else zero
        else:
            e = sum((x[nu] for nu in range(mu) if nu != 1), zero)
        out[mu] = U[mu] * np.where(e % 2 == 1, -1.0, 1.0)[:, None, None]
    W = np.zeros((9, 1, 1), complex)
    for mu in range(4):
        W[1 + 2 * mu] = 1.0
        W[2 + 2 * mu] = -1.0
    got = oracle.covconv(dims, out, W, psi[None], bc)[0]
    want = oracle.dslash_full(dims, U, N, psi, bc, c1=1.0, c3=0.0)
    assert np.abs(got - want).max() > 1e-3 * np.abs(want).max()
