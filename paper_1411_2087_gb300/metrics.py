"""Operation and byte accounting used for every reported rate.

The counts follow the paper's Sec. 3: per site the improved staggered Dslash
does 16 SU(3) matrix-vector products (36 real multiplies + 30 real adds each)
and 15 colour-vector additions (6 real adds each), 1146 flops in all, on 16
link matrices and 16 neighbour colour vectors.

The byte model is the one behind the paper's GB/s columns (Tables 1 and 2):
every link matrix and the output vector move once, the input vector moves
once per site (perfect neighbour reuse in cache), and without streaming
stores the output is read before it is written:

    bytes/site = w * (n_links * reals_per_link + 6 + 6 + 6 * [no streaming store])

with w the bytes per real.  The GPU rates in this project use the streaming
form (no read-for-ownership), which is also the minimum traffic a Dslash
launch has to move: 2400 B/site in FP64.
"""
from __future__ import annotations

REALS_PER_LINK = 18          # 3x3 complex
REALS_PER_LINK_COMPRESSED = 12  # two rows, third reconstructed (Sec. 4)
REALS_PER_VECTOR = 6         # 3 complex colour components
N_LINKS_NAIK = 16            # 8 one-link + 8 three-link matrices per site
N_LINKS_NAIVE = 8            # one-link term only


def matvec_flops() -> int:
    """36 real multiplies + 30 real adds for one SU(3) matrix times vector."""
    return 36 + 30


def dslash_flops_per_site(n_links: int = N_LINKS_NAIK) -> int:
    """n_links mat-vec products plus (n_links - 1) colour-vector adds."""
    return n_links * matvec_flops() + (n_links - 1) * REALS_PER_VECTOR


def dslash_bytes_per_site(real_bytes: int = 8, n_links: int = N_LINKS_NAIK,
                          reals_per_link: int = REALS_PER_LINK,
                          streaming_store: bool = True) -> int:
    """Algorithmic bytes per output site of one Dslash launch."""
    reals = n_links * reals_per_link + REALS_PER_VECTOR + REALS_PER_VECTOR
    if not streaming_store:
        reals += REALS_PER_VECTOR
    return real_bytes * reals


def dslash_half_bytes_per_site(n_links: int = N_LINKS_NAIK) -> int:
    """FP16 storage: 2-byte links and vectors plus one 4-byte norm per vector."""
    return 2 * n_links * REALS_PER_LINK + 2 * (2 * REALS_PER_VECTOR + 4)


def cg_vector_bytes_per_site(real_bytes: int = 8) -> int:
    """Vector traffic of one CG iteration per even site outside the stencils.

    M p = m^2 p - D_eo t reads p once more (48 B in FP64); the fused update
    reads x, p, r, Mp and writes x, r; the direction update reads r, p and
    writes p.
    """
    v = REALS_PER_VECTOR * real_bytes
    return v + 6 * v + 3 * v


def cg_bytes_per_iteration_per_site(real_bytes: int = 8) -> int:
    """Two Dslash launches (D_oe then D_eo) plus the vector passes, per even site."""
    return 2 * dslash_bytes_per_site(real_bytes) + cg_vector_bytes_per_site(real_bytes)


def cg_flops_per_iteration_per_site() -> int:
    """Two Dslash + m^2 p - (D t) (12) + dot <p,Mp> (12) + x,r updates (24)
    + |r|^2 (12) + p = r + beta p (12), per even site."""
    return 2 * dslash_flops_per_site() + 12 + 12 + 24 + 12 + 12


def multishift_cg_flops_per_iteration(volume: int, n_masses: int) -> int:
    """The paper's count for one multishift CG iteration: (1205 + 15 N_m) V (Sec. 3)."""
    return (1205 + 15 * n_masses) * volume


def multishift_memory_bytes_per_site(n_masses: int) -> int:
    """The paper's memory model for the multishift solver: (36 + 2 N_m) * 48 B (Sec. 3)."""
    return (36 + 2 * n_masses) * 48
