"""CPU oracle for the improved-staggered Dslash and even-odd CG (FP64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the library's product path.
It shares no code with the CUDA path.

The arithmetic lives in ``stag_oracle.c`` (plain C99 complex, OpenMP over
output sites); this module compiles it with gcc on first use and wraps it
with ctypes on numpy complex128 arrays in the canonical layouts:

* gauge field ``[4][V][3][3]``, site ``i = x + Lx*(y + Ly*(z + Lz*t))``
* full-lattice colour field ``[V][3]``
* one-parity colour field ``[Vh][3]``, site i of that parity at position i//2

Every function follows the operator definition stated in the header of
``stag_oracle.c`` (the paper's Sec. 3 operation description, with the
readings listed there).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stag_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

C1_NAIK = 9.0 / 8.0
C3_NAIK = -1.0 / 24.0
BC_DEFAULT = (1.0, 1.0, 1.0, -1.0)

CG_CONVERGED = 0
CG_NOT_CONVERGED = 1
CG_BREAKDOWN = 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # STAG_ORACLE_SO lets the mutation tests load a deliberately broken
        # copy of the oracle in a child process.
        so = os.environ.get("STAG_ORACLE_SO")
        if not so:
            build()
            so = _SO
        lib = ctypes.CDLL(so)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_long_links.argtypes = [P, P, P]
        lib.orc_long_links.restype = None
        lib.orc_dslash_full.argtypes = [P, P, D, D, P, P, P, P]
        lib.orc_dslash_full.restype = None
        lib.orc_dslash_parity.argtypes = [P, P, D, D, P, P, I, P, P]
        lib.orc_dslash_parity.restype = None
        lib.orc_apply_M.argtypes = [P, P, D, D, P, P, D, P, P]
        lib.orc_apply_M.restype = None
        lib.orc_cg.argtypes = [P, P, D, D, P, P, D, P, P, D, I,
                               ctypes.POINTER(I), ctypes.POINTER(D), P]
        lib.orc_cg.restype = I
        lib.orc_dslash_sites.argtypes = [P, P, D, D, P, P, P, P, ctypes.c_long, P]
        lib.orc_dslash_sites.restype = None
        lib.orc_covconv.argtypes = [P, P, P, I, I, P, P, P]
        lib.orc_covconv.restype = None
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = I
        lib.orc_set_num_threads.argtypes = [I]
        lib.orc_set_num_threads.restype = None
        _lib = lib
        return lib


def _dims(dims) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    if d.shape != (4,) or np.any(d < 2) or np.any(d % 2):
        raise ValueError(f"lattice dims must be four even numbers >= 2, got {dims}")
    return d


def _bc(bc) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(bc, dtype=np.float64).reshape(4))


def _c(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def long_links(dims, U) -> np.ndarray:
    """Three-link products N_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu) (Sec. 4)."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = np.empty_like(U)
    _load().orc_long_links(_ptr(d), _ptr(U), _ptr(N))
    return N


def dslash_full(dims, U, N, psi, bc=BC_DEFAULT, c1=C1_NAIK, c3=C3_NAIK) -> np.ndarray:
    """(D psi)(x) on every site; psi and the result are full-lattice [V][3]."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = _c(N, (4, V, 3, 3))
    psi = _c(psi, (V, 3))
    out = np.empty_like(psi)
    _load().orc_dslash_full(_ptr(d), _ptr(_bc(bc)), c1, c3, _ptr(U), _ptr(N), _ptr(psi), _ptr(out))
    return out


def dslash_parity(dims, U, N, out_parity: int, psi_cb, bc=BC_DEFAULT,
                  c1=C1_NAIK, c3=C3_NAIK) -> np.ndarray:
    """D_eo (out_parity 0) or D_oe (out_parity 1) in checkerboard order."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = _c(N, (4, V, 3, 3))
    psi = _c(psi_cb, (V // 2, 3))
    out = np.empty_like(psi)
    _load().orc_dslash_parity(_ptr(d), _ptr(_bc(bc)), c1, c3, _ptr(U), _ptr(N),
                              int(out_parity), _ptr(psi), _ptr(out))
    return out


def dslash_sites(dims, U, N, sites, psi_cb, bc=BC_DEFAULT, c1=C1_NAIK, c3=C3_NAIK) -> np.ndarray:
    """(D psi)(x) at the full-lattice sites `sites` (all of one parity);
    psi_cb is the other parity in checkerboard order.  Returns [n][3]."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = _c(N, (4, V, 3, 3))
    psi = _c(psi_cb, (V // 2, 3))
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((idx.size, 3), dtype=np.complex128)
    _load().orc_dslash_sites(_ptr(d), _ptr(_bc(bc)), c1, c3, _ptr(U), _ptr(N), _ptr(psi), _ptr(idx),
                             idx.size, _ptr(out))
    return out


def apply_M(dims, U, N, mass: float, x_even, bc=BC_DEFAULT, c1=C1_NAIK,
            c3=C3_NAIK) -> np.ndarray:
    """M x = m^2 x - D_eo D_oe x on the even checkerboard."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = _c(N, (4, V, 3, 3))
    x = _c(x_even, (V // 2, 3))
    out = np.empty_like(x)
    _load().orc_apply_M(_ptr(d), _ptr(_bc(bc)), c1, c3, _ptr(U), _ptr(N), float(mass),
                        _ptr(x), _ptr(out))
    return out


def cg(dims, U, N, mass: float, b_even, tol: float = 1e-10, max_iter: int = 20000,
       bc=BC_DEFAULT, c1=C1_NAIK, c3=C3_NAIK, history: bool = False):
    """Solve M x = b (x0 = 0) by CG; returns (x, info).

    info: ``status`` (0 converged, 1 not converged, 2 breakdown), ``iters``,
    ``true_rel_resid`` = |b - M x| / |b| recomputed at exit, and with
    ``history`` an array [iters][3] of (alpha_k, beta_k, |r_{k+1}|^2).
    """
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    N = _c(N, (4, V, 3, 3))
    b = _c(b_even, (V // 2, 3))
    x = np.empty_like(b)
    iters = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    hist = np.zeros((max(max_iter, 1), 3)) if history else None
    status = _load().orc_cg(_ptr(d), _ptr(_bc(bc)), c1, c3, _ptr(U), _ptr(N), float(mass),
                            _ptr(b), _ptr(x), float(tol), int(max_iter),
                            ctypes.byref(iters), ctypes.byref(res),
                            _ptr(hist) if hist is not None else None)
    info = {"status": int(status), "iters": int(iters.value),
            "true_rel_resid": float(res.value)}
    if hist is not None:
        info["history"] = hist[: iters.value].copy()
    return x, info


def parity_mask(dims) -> np.ndarray:
    """parity (x+y+z+t) & 1 of every site, in site order."""
    d = np.asarray(dims)
    t, z, y, x = np.meshgrid(*(np.arange(n) for n in d[::-1]), indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1)


def full_to_cb(dims, psi_full, parity: int) -> np.ndarray:
    """Sites of one parity of a full-lattice field, in checkerboard order."""
    par = parity_mask(dims)
    idx = np.nonzero(par == parity)[0]
    out = np.zeros((volume(dims) // 2, 3), dtype=np.complex128)
    out[idx // 2] = np.asarray(psi_full)[idx]
    return out


def cb_to_full(dims, psi_cb, parity: int) -> np.ndarray:
    """Full-lattice field that is psi_cb on one parity and zero on the other."""
    par = parity_mask(dims)
    idx = np.nonzero(par == parity)[0]
    out = np.zeros((volume(dims), 3), dtype=np.complex128)
    out[idx] = np.asarray(psi_cb)[idx // 2]
    return out


# --------------------------------------------------------------------------
# learned preconditioner: gauge-covariant convolution net (oracle side)
# --------------------------------------------------------------------------

def covconv(dims, U, W, psi, bc=BC_DEFAULT) -> np.ndarray:
    """One covariant convolution layer (see orc_covconv in stag_oracle.c).

    W: complex [9][cout][cin]; psi: complex [cin][V][3] -> [cout][V][3]."""
    d = _dims(dims)
    V = volume(d)
    U = _c(U, (4, V, 3, 3))
    W = _c(W)
    if W.ndim != 3 or W.shape[0] != 9:
        raise ValueError("W must have shape [9][cout][cin]")
    cout, cin = W.shape[1], W.shape[2]
    psi = _c(psi, (cin, V, 3))
    y = np.empty((cout, V, 3), dtype=np.complex128)
    _load().orc_covconv(_ptr(d), _ptr(_bc(bc)), _ptr(U), cin, cout, _ptr(W), _ptr(psi), _ptr(y))
    return y


def phased_links(dims, U) -> np.ndarray:
    """eta_mu(x) U_mu(x) with the Kogut-Susskind phases
    eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) (x fastest): the links the
    library's net transports with (the boundary sign is applied by covconv)."""
    d = [int(n) for n in dims]
    V = volume(d)
    t, z, y, x = np.meshgrid(*(np.arange(n) for n in d[::-1]), indexing="ij")
    coords = [c.reshape(-1) for c in (x, y, z, t)]
    out = np.array(_c(U, (4, V, 3, 3)), copy=True)
    for mu in range(4):
        esum = sum(coords[:mu], np.zeros(V, dtype=np.int64))
        out[mu] *= np.where(esum % 2 == 1, -1.0, 1.0)[:, None, None]
    return out


def net_apply(dims, U, weights, r_even, bc=BC_DEFAULT) -> np.ndarray:
    """The preconditioner: r (even sites) zero-extended to the full lattice,
    the layers applied in order (no nonlinearity), the result restricted to
    the even sites.  weights: list of complex [9][cout][cin]."""
    psi = cb_to_full(dims, r_even, 0)[None]
    for W in weights:
        psi = covconv(dims, U, W, psi, bc)
    return full_to_cb(dims, psi[0], 0)


def net_loss(dims, U, weights, rs, es, bc=BC_DEFAULT) -> float:
    """sum over pairs of |N(r) - e|^2 / |e|^2."""
    tot = 0.0
    for r, e in zip(rs, es):
        z = net_apply(dims, U, weights, r, bc)
        tot += float(np.vdot(z - e, z - e).real / np.vdot(e, e).real)
    return tot
