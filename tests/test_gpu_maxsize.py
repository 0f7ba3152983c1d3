"""The Dslash and M at (nearly) the largest lattice a lattice object accepts.

The kernels address one parity's 72 link planes with 32-bit offsets, and a
lattice is refused once 72 x stride reaches 2^31; 64^3 x 224 (Vh =
29,360,128, 98.6 % of that limit, Lt a multiple of 4 so that the two-site
16-bit form applies) puts every offset near the top of that range.  The
oracle would need the whole 68 GB of canonical links on the host there, so
the check is a property that holds at any size, gauge covariance: with
U'_mu(x) = g(x) U_mu(x) g(x+mu)^+ and the three-link products rebuilt from
U', D'(g psi) = g (D psi) and M'(g psi) = g (M psi) on every site.  A wrong
index anywhere in the stencil breaks it by O(1)."""
import numpy as np
import pytest
import torch

from paper_1411_2087_gb300 import stag

pytestmark = pytest.mark.gpu

DIMS = (64, 64, 64, 224)
MASS = 0.02


def su3_on_device(n, gen, chunk=1 << 23):
    """n random SU(3) matrices from a seeded CUDA generator: rows u, v by
    Gram-Schmidt from Gaussian complex vectors, row 3 = conj(u x v) (so det
    = 1).  Built with elementwise ops on the device: batched 3 x 3 matrix
    functions of 240 M matrices take minutes, and covariance holds for any
    SU(3) links (no oracle reads these fields)."""
    dev = gen.device
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=dev)

    def cvec(m):
        re = torch.randn((m, 3), dtype=torch.float64, device=dev, generator=gen)
        im = torch.randn((m, 3), dtype=torch.float64, device=dev, generator=gen)
        return torch.complex(re, im)

    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        u = cvec(m)
        u = u / torch.linalg.vector_norm(u, dim=1, keepdim=True)
        v = cvec(m)
        v = v - (u.conj() * v).sum(1, keepdim=True) * u
        v = v / torch.linalg.vector_norm(v, dim=1, keepdim=True)
        w = torch.stack([u[:, 1] * v[:, 2] - u[:, 2] * v[:, 1],
                         u[:, 2] * v[:, 0] - u[:, 0] * v[:, 2],
                         u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]], dim=1).conj()
        out[s:s + m, 0] = u
        out[s:s + m, 1] = v
        out[s:s + m, 2] = w
    return out


def mul33(A, B):
    """Batched 3 x 3 products as three broadcast multiply-adds (the batched
    library product of tiny matrices is far slower at this count)."""
    C = A[..., :, 0:1] * B[..., 0:1, :]
    for k in (1, 2):
        C += A[..., :, k:k + 1] * B[..., k:k + 1, :]
    return C


def matvec(A, x):
    return (A * x.unsqueeze(-2)).sum(-1)


def full_index(dims, parity, dev):
    """Full site index i = x + Lx (y + Ly (z + Lz t)) of every checkerboard
    site c of one parity, in cb order (i = 2c + the parity bit of its row)."""
    Lx, Ly, Lz, Lt = dims
    Vh = Lx * Ly * Lz * Lt // 2
    c = torch.arange(Vh, device=dev, dtype=torch.int64)
    r = c // (Lx // 2)
    y = r % Ly
    r = r // Ly
    z = r % Lz
    t = r // Lz
    return 2 * c + ((parity + y + z + t) & 1)


def transform_links(U, g, dims):
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^+ in place (periodic in index space)."""
    Lx, Ly, Lz, Lt = dims
    g5 = g.view(Lt, Lz, Ly, Lx, 3, 3)
    for mu, axis in enumerate((3, 2, 1, 0)):
        gs = torch.roll(g5, shifts=-1, dims=axis).reshape(-1, 3, 3)
        for a in range(0, g.shape[0], 1 << 23):
            b = a + (1 << 23)
            U[mu, a:b] = mul33(mul33(g[a:b], U[mu, a:b]), gs[a:b].conj().transpose(-1, -2))
        del gs


def apply_ops(U, psi_e, precs):
    """{prec: (D_oe psi, M psi)} as device tensors; f16 on 12-real links in
    the two-site form."""
    out = {}
    Vh = psi_e.shape[0]
    dev = psi_e.device
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, None, precisions=precs, compress12=("f16" in precs))
        torch.cuda.empty_cache()
        for prec in precs:
            if prec == "f16":
                lat.set_tuning("f16", "dslash", 256, 3)
                lat.set_tuning("f16", "M", 256, 3)
            fe = lat.field(stag.EVEN, prec, psi_e)
            fo = lat.field(stag.ODD, prec)
            fm = lat.field(stag.EVEN, prec)
            lat.dslash(fo, fe)
            lat.apply_M(fm, fe, MASS)
            d = torch.empty((Vh, 3), dtype=torch.complex128, device=dev)
            m = torch.empty((Vh, 3), dtype=torch.complex128, device=dev)
            fo.export(d)
            fm.export(m)
            torch.cuda.synchronize()
            out[prec] = (d, m)
            for f in (fe, fo, fm):
                f.destroy()
    torch.cuda.empty_cache()
    return out


def test_gauge_covariance_near_the_size_limit():
    dev = torch.device("cuda", 0)
    Vh = int(np.prod(DIMS)) // 2
    torch.cuda.empty_cache()
    gen = torch.Generator(device=dev)
    gen.manual_seed(1301)
    V = 2 * Vh
    U = su3_on_device(4 * V, gen).view(4, V, 3, 3)
    psi = torch.complex(torch.randn((Vh, 3), dtype=torch.float64, device=dev, generator=gen),
                        torch.randn((Vh, 3), dtype=torch.float64, device=dev, generator=gen))
    precs = ("df64", "f16")
    before = apply_ops(U, psi, precs)

    g = su3_on_device(V, gen)
    transform_links(U, g, DIMS)
    ie, io = full_index(DIMS, 0, dev), full_index(DIMS, 1, dev)
    g_e, g_o = g[ie], g[io]
    del g, ie, io
    psi_t = matvec(g_e, psi)
    torch.cuda.empty_cache()
    after = apply_ops(U, psi_t, precs)
    del U

    tol = {"df64": 1e-12, "f16": 2e-3}
    for prec in precs:
        d0, m0 = before[prec]
        d1, m1 = after[prec]
        for got, ref, gx in ((d1, d0, g_o), (m1, m0, g_e)):
            want = matvec(gx, ref)
            err = ((got - want).abs().max() / want.abs().max()).item()
            assert err <= tol[prec], (prec, err)
