"""Fields that view caller-owned device memory (stag_field_wrap): zero-copy
with torch, bit-identical results to library-owned fields, the caller keeps
ownership, and bad buffers are argument errors."""
import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_wrapped_field_matches_owned(prec):
    dims, mass = (6, 4, 6, 10), 0.1
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 91).numpy()
    N = oracle.long_links(dims, U)
    psi = synth.gaussian_colour_field(Vh, 92).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        nb = lat.field_bytes(prec)
        tin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        tout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        win = lat.wrap_field(tin, stag.EVEN, prec)
        wout = lat.wrap_field(tout, stag.ODD, prec)
        win.import_(psi)                          # writes into the tensor
        torch.cuda.synchronize()
        assert int(tin.count_nonzero()) > 0
        fin = lat.field(stag.EVEN, prec, psi)
        fout = lat.field(stag.ODD, prec)
        lat.dslash(wout, win)
        lat.dslash(fout, fin)
        assert np.array_equal(wout.export(), fout.export())
        # same size as the owned field's storage
        ptr, n = fout.storage()
        assert n == nb
        # destroying the view leaves the tensor usable
        wout.destroy()
        win.destroy()
        assert int(tout.count_nonzero()) > 0


def test_wrapped_fields_in_cg():
    dims, mass = (8, 8, 8, 8), 0.1
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 93).numpy()
    N = oracle.long_links(dims, U)
    b = synth.gaussian_colour_field(Vh, 94).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        nb = lat.field_bytes("df64")
        tb = torch.empty(nb, dtype=torch.uint8, device="cuda")
        tx = torch.empty(nb, dtype=torch.uint8, device="cuda")
        wb = lat.wrap_field(tb, stag.EVEN, "df64").import_(b)
        wx = lat.wrap_field(tx, stag.EVEN, "df64")
        info = lat.cg(wx, wb, mass, 1e-10, 5000)
        fx = lat.field(stag.EVEN, "df64")
        info2 = lat.cg(fx, lat.field(stag.EVEN, "df64", b), mass, 1e-10, 5000)
        assert info["return"] == stag.OK and info["iters"] == info2["iters"]
        assert np.array_equal(wx.export(), fx.export())


def test_wrap_rejects_bad_buffers():
    dims = (4, 4, 4, 4)
    with stag.Lattice(dims) as lat:
        nb = lat.field_bytes("df64")
        small = torch.zeros(nb - 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(stag.StagError) as e:
            lat.wrap_field(small, stag.EVEN, "df64")
        assert e.value.status == stag.ERR_ARG
        big = torch.zeros(nb + 64, dtype=torch.uint8, device="cuda")
        with pytest.raises(stag.StagError) as e:
            lat.wrap_field(big[8:], stag.EVEN, "df64")   # 8-byte offset: misaligned
        assert e.value.status == stag.ERR_ARG
        with pytest.raises(ValueError):
            lat.wrap_field(torch.zeros(nb, dtype=torch.uint8), stag.EVEN, "df64")  # host tensor
        host = np.zeros(nb, dtype=np.uint8)
        h = stag.ctypes.c_void_p()
        st = stag.lib().stag_field_wrap(lat.handle, 0, stag.PREC["df64"],
                                        host.ctypes.data_as(stag.ctypes.c_void_p), nb, stag.ctypes.byref(h))
        assert st == stag.ERR_ARG


def test_lattice_on_caller_stream_is_identical():
    """A lattice bound to the caller's CUDA stream (a torch stream) runs the
    same kernels, graphs included, as one on the library's own stream."""
    dims, mass = (6, 4, 6, 10), 0.05
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 95).numpy()
    N = oracle.long_links(dims, U)
    b = synth.gaussian_colour_field(Vh, 96).numpy()
    user = torch.cuda.Stream()
    results = []
    for stream in (None, user.cuda_stream):
        with stag.Lattice(dims, stream=stream) as lat:
            lat.upload_gauge(U, N, precisions=("df64", "f16"))
            fb = lat.field(stag.EVEN, "df64", b)
            fo = lat.field(stag.ODD, "df64")
            lat.dslash(fo, fb)
            fx = lat.field(stag.EVEN, "df64")
            i1 = lat.cg(fx, fb, mass, 1e-10, 5000)
            fy = lat.field(stag.EVEN, "df64")
            i2 = lat.cg_mixed(fy, fb, mass, 1e-10, 5000, inner="f16")
            results.append((fo.export(), fx.export(), fy.export(), i1["iters"], i2["iters"]))
    a, c = results
    assert all(np.array_equal(u, v) for u, v in zip(a[:3], c[:3])) and a[3:] == c[3:]
    res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, c[1])) / np.linalg.norm(b)
    assert res <= 1.05e-10


def test_two_lattices_interleaved():
    """Two lattices of different sizes, used alternately, keep separate
    graphs, scalars and workspaces."""
    specs = [((4, 4, 4, 8), 0.1, 97), ((6, 4, 6, 10), 0.05, 98)]
    lats, data = [], []
    for dims, mass, seed in specs:
        Vh = int(np.prod(dims)) // 2
        U = synth.su3_field(dims, 0.3, seed).numpy()
        N = oracle.long_links(dims, U)
        b = synth.gaussian_colour_field(Vh, seed + 1).numpy()
        lat = stag.Lattice(dims)
        lat.upload_gauge(U, N, precisions=("df64",))
        lats.append(lat)
        data.append((dims, mass, U, N, b, lat.field(stag.EVEN, "df64", b), lat.field(stag.EVEN, "df64")))
    try:
        for _ in range(2):
            for lat, (dims, mass, U, N, b, fb, fx) in zip(lats, data):
                info = lat.cg(fx, fb, mass, 1e-10, 5000)
                assert info["return"] == stag.OK
                res = np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, fx.export())) / np.linalg.norm(b)
                assert res <= 1.05e-10
    finally:
        for lat in lats:
            lat.close()
