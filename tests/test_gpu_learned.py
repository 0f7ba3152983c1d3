"""The learned gauge-covariant preconditioner on the GPU: the forward pass
against the oracle's FP64 net, gauge covariance, the training gradient
against the oracle's finite differences (central, h = 1e-6, FP64), training
lowering the loss, and flexible CG with the trained net reaching the true
residual in fewer iterations than without it."""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu


def rand_weights(C, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    shapes = [(9, C, 1), (9, C, C), (9, 1, C)]
    return [scale * (rng.standard_normal(s) + 1j * rng.standard_normal(s)) for s in shapes]


def shift(field, dims, mu, s):
    Lx, Ly, Lz, Lt = dims
    f = field.reshape((Lt, Lz, Ly, Lx) + field.shape[1:])
    return np.roll(f, -s, axis=3 - mu).reshape(field.shape)


@pytest.mark.parametrize("dims,C", [((4, 4, 4, 4), 4), ((6, 4, 6, 10), 8), ((2, 2, 2, 2), 2)])
def test_forward_matches_oracle(dims, C):
    U = synth.su3_field(dims, 0.4, 5).numpy()
    Vh = int(np.prod(dims)) // 2
    r = synth.gaussian_colour_field(Vh, 6).numpy()
    Ws = rand_weights(C, 7)
    # the net transports with the staggered-phased links
    want = oracle.net_apply(dims, oracle.phased_links(dims, U), Ws, r)
    with stag.Lattice(dims) as lat:
        net = stag.Net(lat, U, channels=C)
        net.set_weights(Ws)
        got_w = net.get_weights()
        assert all(np.array_equal(a, b) for a, b in zip(got_w, Ws))
        for prec in ("f32", "df64"):
            fin = lat.field(stag.EVEN, prec, r)
            fout = lat.field(stag.EVEN, prec)
            net.apply(fout, fin)
            err = np.abs(fout.export() - want).max() / np.abs(want).max()
            assert err < 1e-5, (prec, err)
        # binary16 weights: error of the rounding only; with the 16-bit
        # links as well (the solver's form), 1/32767 of the largest entry more
        fin = lat.field(stag.EVEN, "f32", r)
        fout = lat.field(stag.EVEN, "f32")
        net.apply(fout, fin, fp16_weights=True)
        err = np.abs(fout.export() - want).max() / np.abs(want).max()
        assert err < 5e-3
        for prec in ("f32", "df64"):
            fin = lat.field(stag.EVEN, prec, r)
            fout = lat.field(stag.EVEN, prec)
            net.apply(fout, fin, fp16_weights=True, links16=True)
            err = np.abs(fout.export() - want).max() / np.abs(want).max()
            assert err < 5e-3, (prec, err)
        fin = lat.field(stag.EVEN, "f32", r)
        fout = lat.field(stag.EVEN, "f32")
        net.apply(fout, fin, links16=True)
        err = np.abs(fout.export() - want).max() / np.abs(want).max()
        assert err < 5e-4, err
        net.close()


@pytest.mark.parametrize("dims,bc,unitary", [((4, 4, 4, 8), (1.0, 1.0, 1.0, -1.0), True),
                                             ((6, 4, 2, 4), (-1.0, 1.0, -1.0, -1.0), True),
                                             ((4, 4, 4, 8), (1.0, 1.0, 1.0, -1.0), False)])
def test_solver_form_links(dims, bc, unitary):
    """The solver's 16-bit net links: with special unitary fat links the
    kernels read rows 0 and 1 and rebuild row 2 with the link's phase and
    boundary sign (every boundary-sign pattern of direction and wrap); with
    other links they read all nine entries.  Both against the oracle's FP64
    net on the phased links."""
    U = synth.su3_field(dims, 0.4, 15).numpy()
    if not unitary:
        U = 0.97 * U
    Vh = int(np.prod(dims)) // 2
    r = synth.gaussian_colour_field(Vh, 16).numpy()
    Ws = rand_weights(8, 17)
    want = oracle.net_apply(dims, oracle.phased_links(dims, U), Ws, r, bc)
    with stag.Lattice(dims, bc=bc) as lat:
        net = stag.Net(lat, U, channels=8)
        net.set_weights(Ws)
        for prec in ("f32", "df64"):
            fin = lat.field(stag.EVEN, prec, r)
            fout = lat.field(stag.EVEN, prec)
            net.apply(fout, fin, fp16_weights=True, links16=True)
            err = np.abs(fout.export() - want).max() / np.abs(want).max()
            assert err < 5e-3, (prec, err)
        net.close()


def adjoint_net(Ws):
    """Layers of N^+: reversed order, each W^+[dbar][i][o] = conj(W[d][o][i])
    with dbar the reversed hop (d = 1 + 2 mu <-> 2 + 2 mu)."""
    out = []
    for W in reversed(Ws):
        A = np.conj(np.transpose(W, (0, 2, 1))).copy()
        B = A.copy()
        for mu in range(4):
            B[1 + 2 * mu] = A[2 + 2 * mu]
            B[2 + 2 * mu] = A[1 + 2 * mu]
        out.append(B)
    return out


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 4)])
def test_hermitian_part_matches_oracle(dims):
    """The solvers' preconditioner (N + N^+)/2, formed on the GPU from the
    path coefficients, against the oracle's net and its adjoint net (layers
    reversed and adjointed) on the phased links."""
    U = synth.su3_field(dims, 0.4, 18).numpy()
    Vh = int(np.prod(dims)) // 2
    r = synth.gaussian_colour_field(Vh, 19).numpy()
    Ws = rand_weights(8, 20)
    Up = oracle.phased_links(dims, U)
    want = 0.5 * (oracle.net_apply(dims, Up, Ws, r) + oracle.net_apply(dims, Up, adjoint_net(Ws), r))
    # the adjoint net really is the adjoint: <s, N r> = <N^+ s, r>
    sv = synth.gaussian_colour_field(Vh, 21).numpy()
    lhs = np.vdot(sv, oracle.net_apply(dims, Up, Ws, r))
    rhs = np.vdot(oracle.net_apply(dims, Up, adjoint_net(Ws), sv), r)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    with stag.Lattice(dims) as lat:
        net = stag.Net(lat, U, channels=8)
        net.set_weights(Ws)
        for prec in ("f32", "df64"):
            fin = lat.field(stag.EVEN, prec, r)
            fout = lat.field(stag.EVEN, prec)
            net.apply(fout, fin, hermitian=True)
            err = np.abs(fout.export() - want).max() / np.abs(want).max()
            assert err < 1e-5, (prec, err)
        fin = lat.field(stag.EVEN, "f32", r)
        fout = lat.field(stag.EVEN, "f32")
        net.apply(fout, fin, fp16_weights=True, links16=True, hermitian=True)
        err = np.abs(fout.export() - want).max() / np.abs(want).max()
        assert err < 5e-3, err
        net.close()


def test_gpu_net_is_gauge_covariant():
    dims = (4, 4, 4, 6)
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.5, 8).numpy()
    g = synth.gauge_transform(dims, 9).numpy()
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ shift(g, dims, mu, 1).conj().transpose(0, 2, 1)
    par = oracle.parity_mask(dims)
    idx = np.nonzero(par == 0)[0]
    g_even = np.empty((Vh, 3, 3), complex)
    g_even[idx // 2] = g[idx]
    r = synth.gaussian_colour_field(Vh, 10).numpy()
    Ws = rand_weights(4, 11)
    outs = []
    for links, src in ((U, r), (Ug, np.einsum("vab,vb->va", g_even, r))):
        with stag.Lattice(dims) as lat:
            net = stag.Net(lat, links, channels=4)
            net.set_weights(Ws)
            fin = lat.field(stag.EVEN, "df64", src)
            fout = lat.field(stag.EVEN, "df64")
            net.apply(fout, fin)
            outs.append(fout.export())
            net.close()
    want = np.einsum("vab,vb->va", g_even, outs[0])
    assert np.abs(outs[1] - want).max() < 1e-5 * np.abs(want).max()


def resid_loss_oracle(dims, U, N, mass, Ws, rs):
    tot = 0.0
    Up = oracle.phased_links(dims, U)
    for r in rs:
        z = oracle.net_apply(dims, Up, Ws, r)
        q = oracle.apply_M(dims, U, N, mass, z) - r
        tot += float(np.vdot(q, q).real / np.vdot(r, r).real)
    return tot


@pytest.mark.parametrize("kind", ["error", "residual"])
def test_gradient_against_oracle_finite_differences(kind):
    dims = (4, 4, 2, 4)
    mass = 0.1
    U = synth.su3_field(dims, 0.3, 12).numpy()
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 13).numpy()
    C = 2
    Ws = rand_weights(C, 14, scale=0.4)
    N = oracle.long_links(dims, U)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32"))
        net = stag.Net(lat, U, channels=C)
        fb = lat.field(stag.EVEN, "df64", b)
        assert net.collect_pairs(fb, mass, 1e-10, stride=3, max_pairs=3) == 3
        net.set_loss(kind)
        net.set_weights(Ws)
        loss, grads = net.loss_grad(0, 3)
        pairs = [net.get_pair(k) for k in range(3)]
        net.close()
    rs = [p[0] for p in pairs]
    es = [p[1] for p in pairs]
    if kind == "error":
        Up = oracle.phased_links(dims, U)

        def L(ws):
            return oracle.net_loss(dims, Up, ws, rs, es)
    else:
        def L(ws):
            return resid_loss_oracle(dims, U, N, mass, ws, rs)
    assert abs(loss - L(Ws)) <= 1e-5 * loss
    h = 1e-6
    fd_all, an_all = [], []
    for li, W in enumerate(Ws):
        for idx in np.ndindex(W.shape):
            for unit in (1.0, 1j):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[li][idx] += unit * h
                Wm[li][idx] -= unit * h
                fd = (L(Wp) - L(Wm)) / (2 * h)
                an = 2 * (grads[li][idx].real if unit == 1.0 else grads[li][idx].imag)
                fd_all.append(fd)
                an_all.append(an)
    fd_all = np.array(fd_all)
    an_all = np.array(an_all)
    # FP32 forward/backward against FP64 finite differences
    assert np.linalg.norm(fd_all - an_all) <= 2e-4 * np.linalg.norm(fd_all), \
        np.abs(fd_all - an_all).max()


def test_training_lowers_loss_and_net_cuts_iterations():
    """What the trained net gains: flexible CG with it against the same
    solve without it (plain CG), on a source it was not trained on."""
    dims = (8, 8, 8, 8)
    mass = 0.05
    U = synth.su3_field(dims, 0.3, 1010).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64", "f32", "f16"))
        net = stag.Net(lat, U, channels=8, seed=1)
        for s in range(4):
            fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1200 + s).numpy())
            net.collect_pairs(fb, mass, 1e-10, stride=8, max_pairs=16)
        assert net.num_pairs() >= 32
        net.set_loss("residual")
        hist = net.train(epochs=100, batch=8, lr=1e-2, seed=3)
        assert hist[-1] < 0.9 * hist[0], hist
        b = synth.gaussian_colour_field(Vh, 1300).numpy()
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        plain = lat.cg(fx, fb, mass, 1e-10, 20000)
        learned = net.cg(fx, fb, mass, 1e-10, 20000)
        x = fx.export()
        # the same net inside the mixed-precision flexible CG (FP32 and 16-bit
        # iteration, double-float reliable updates) against the mixed CG
        mixed = {}
        for inner in ("f32", "f16"):
            plain_m = lat.cg_mixed(fx, fb, mass, 1e-10, 20000, inner)
            learned_m = net.cg_mixed(fx, fb, mass, 1e-10, 20000, inner)
            mixed[inner] = (plain_m, learned_m, fx.export())
        net.close()
    res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)
    assert learned["return"] == stag.OK, learned
    assert res <= 1.05e-10, res
    # a degree-one polynomial in M can at best quarter the condition number
    # (up to 2x fewer iterations); on the phased links the trained net gets
    # about 1.8x here, beyond the 1.42x of the same net on raw links
    assert learned["iters"] <= 0.7 * plain["iters"], (learned, plain)
    assert learned["restarts"] == 0
    for inner, (plain_m, learned_m, xm) in mixed.items():
        res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, xm)) / np.linalg.norm(b)
        assert learned_m["return"] == stag.OK, (inner, learned_m)
        assert res <= 1.05e-10, (inner, res)
        # no fallback (a fallback adds a whole plain solve to the count)
        assert learned_m["iters"] <= 0.8 * plain_m["iters"], (inner, learned_m, plain_m)


def test_briefly_trained_net_does_no_harm():
    """A net trained for a few steps is far from Hermitian; the solver
    applies its Hermitian part, with which flexible CG needs no more
    iterations than plain CG (the net itself had made CG slower)."""
    dims = (8, 8, 8, 8)
    mass = 0.05
    U = synth.su3_field(dims, 0.3, 1011).numpy()
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"))
        net = stag.Net(lat, U, channels=8, seed=2)
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1210).numpy())
        assert net.collect_pairs(fb, mass, 1e-10, stride=6, max_pairs=16) == 16
        net.set_loss("residual")
        net.train(epochs=1, batch=8, lr=1e-2, seed=3)
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1310).numpy())
        fx = lat.field(stag.EVEN, "df64")
        plain = lat.cg(fx, fb, mass, 1e-10, 20000)
        learned = net.cg(fx, fb, mass, 1e-10, 20000)
        net.close()
    assert learned["return"] == stag.OK, learned
    assert learned["iters"] <= plain["iters"], (learned, plain)


def test_error_loss_training_runs():
    dims = (4, 4, 4, 8)
    U = synth.su3_field(dims, 0.3, 21).numpy()
    Vh = int(np.prod(dims)) // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        net = stag.Net(lat, U, channels=4, seed=2)
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 22).numpy())
        net.collect_pairs(fb, 0.1, 1e-10, stride=4, max_pairs=8)
        hist = net.train(epochs=20, batch=4, lr=1e-2, seed=1)
        assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
        with pytest.raises(stag.StagError):  # the residual loss needs an F32 gauge copy
            net.set_loss("residual")
        net.close()


def test_learned_solver_edges():
    dims = (4, 4, 4, 4)
    U = synth.su3_field(dims, 0.3, 20).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        net = stag.Net(lat, U, channels=4)
        fz = lat.field(stag.EVEN, "df64", np.zeros((128, 3), complex))
        fx = lat.field(stag.EVEN, "df64")
        info = net.cg(fx, fz, 0.1, 1e-10, 100)
        assert info["return"] == stag.OK and not np.any(fx.export())
        with pytest.raises(stag.StagError):
            net.train(epochs=1)  # no pairs yet
        with pytest.raises(stag.StagError):
            stag.Net(lat, U, channels=3)
        net.close()
