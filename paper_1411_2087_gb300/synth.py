"""Seeded synthetic inputs: SU(3) gauge fields, random gauge transforms and
Gaussian colour-vector sources.

This module is shared by the CUDA path's callers and by the tests that feed
the CPU oracle.  It holds none of the Dslash/CG arithmetic: it only draws
random numbers and turns them into group elements and sources.

Recipe (the paper runs on real MILC configurations that are not available;
these synthetic fields stand in for them):

* fat link  U_mu(x) = exp(i * eps * H_mu(x)),  H = sum_a omega_a * lambda_a / 2
  with the eight Gell-Mann matrices lambda_a and omega_a ~ N(0, 1) drawn from
  numpy's PCG64(seed) in the order (mu, site, a).  U is special unitary.
* source    re, im i.i.d. N(0, 1), drawn from PCG64(seed) in (site, colour,
  re/im) order.
* a random gauge transform is one SU(3) matrix per site with eps = 1.

Canonical layouts (all complex128, C order):

* gauge field ``[4][V][3][3]``: direction mu (0..3 = x, y, z, t), site
  ``i = x + Lx*(y + Ly*(z + Lz*t))``, row, column.
* colour field on one parity ``[Vh][3]`` in checkerboard order: site i of
  parity (x+y+z+t)&1 sits at position ``i >> 1``.
* colour field on the full lattice ``[V][3]`` in site order.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = [
    "volume",
    "gell_mann",
    "su3_field",
    "gauge_transform",
    "gaussian_colour_field",
    "unit_gauge_field",
]


def volume(dims) -> int:
    """Number of lattice sites V = Lx*Ly*Lz*Lt."""
    v = 1
    for d in dims:
        v *= int(d)
    return v


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape [8][3][3] complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _exp_i_eps_h(omega: np.ndarray, eps: float, device) -> torch.Tensor:
    """exp(i*eps*H) for H = sum_a omega_a lambda_a / 2; omega has shape [..., 8]."""
    lam = torch.from_numpy(gell_mann() / 2).to(device)
    om = torch.from_numpy(np.ascontiguousarray(omega)).to(device=device, dtype=torch.complex128)
    h = torch.einsum("...a,aij->...ij", om, lam)
    return torch.linalg.matrix_exp((1j * eps) * h)


def su3_field(dims, eps: float, seed: int, n_dir: int = 4, device="cpu",
              chunk: int = 1 << 22) -> torch.Tensor:
    """Seeded SU(3) link field, shape [n_dir][V][3][3] complex128 on ``device``.

    eps = 0 gives unit links (the free field).  Draws are made in chunks of
    ``chunk`` matrices so that large lattices do not need all omegas at once;
    the draw order (mu, site, a) does not depend on the chunk size.
    """
    v = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = torch.empty((n_dir, v, 3, 3), dtype=torch.complex128, device=device)
    flat = out.view(n_dir * v, 3, 3)
    total = n_dir * v
    start = 0
    while start < total:
        n = min(chunk, total - start)
        omega = rng.standard_normal((n, 8))
        flat[start:start + n] = _exp_i_eps_h(omega, eps, device)
        start += n
    return out


def unit_gauge_field(dims, n_dir: int = 4, device="cpu") -> torch.Tensor:
    """Unit links, shape [n_dir][V][3][3] complex128."""
    v = volume(dims)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    return eye.expand(n_dir, v, 3, 3).contiguous()


def gauge_transform(dims, seed: int, device="cpu") -> torch.Tensor:
    """Random SU(3) matrix per site (eps = 1), shape [V][3][3] complex128."""
    return su3_field(dims, 1.0, seed, n_dir=1, device=device)[0]


def gaussian_colour_field(n_sites: int, seed: int, device="cpu") -> torch.Tensor:
    """Gaussian colour field, shape [n_sites][3] complex128, re/im ~ N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ri = rng.standard_normal((n_sites, 3, 2))
    z = ri[..., 0] + 1j * ri[..., 1]
    return torch.from_numpy(z).to(device)
