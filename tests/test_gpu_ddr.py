"""The rank decomposition on the GPU.

Every run here has one GPU, so the ranks are host threads of one process,
each with its own lattice and stream on that GPU, talking through an
in-process mailbox (a communicator in host memory).  No kernel waits for
another: the ranks meet only on the host, in the mailbox's exchange and
allreduce.  Checks:

* each rank's slab of stag_ddr_dslash equals the single-domain Dslash
  bit for bit (same kernel, same links, the received halo), also where the
  slab's interior is computed while the halo is exchanged;
* the CG over 1, 2 and 3 ranks (F64 and double float) gives a solution whose
  true residual, recomputed by the FP64 oracle on the ranks' slabs put
  together, meets 1e-10, in the oracle's iteration count (within max(3, 1%));
* NCCL as the communicator, with one rank, gives the same Dslash and solution
  as the mailbox: its device allreduce drives the CG with one host wait per
  eight iterations, the mailbox's host allreduce with one per sum, and the
  device-side scalar recurrence is the same; its exchange (a rank sending to
  itself) and allreduces are checked on device buffers directly.
"""
import ctypes
import threading

import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

DIMS, MASS = (6, 4, 4, 12), 0.1
DIMS16 = (4, 4, 6, 16)  # slabs of 8 and 16 slices: the interior stencil overlaps the exchange


class Mailbox:
    """Exchange and allreduce between threads; sums in rank order, so every
    rank gets the same result."""

    def __init__(self, size):
        self.size = size
        self.barrier = threading.Barrier(size, timeout=120)
        self.slots = {}

    def comm(self, rank):
        def exchange(to_prev, to_next):
            self.slots[(rank, "prev")] = to_prev
            self.slots[(rank, "next")] = to_next
            self.barrier.wait()
            fp = self.slots[((rank - 1) % self.size, "next")]
            fn = self.slots[((rank + 1) % self.size, "prev")]
            self.barrier.wait()
            return fp, fn

        def allreduce(vals):
            self.slots[(rank, "sum")] = list(vals)
            self.barrier.wait()
            out = [sum(self.slots[(r, "sum")][k] for r in range(self.size)) for k in range(len(vals))]
            self.barrier.wait()
            return out

        return stag.HostComm(rank, self.size, exchange, allreduce)


def make_problem(dims):
    U = synth.su3_field(dims, 0.3, 1000).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    psi_o = synth.gaussian_colour_field(Vh, 1101).numpy()
    return U, N, b, psi_o


@pytest.fixture(scope="module")
def problem():
    return make_problem(DIMS)


def run_ranks(size, fn):
    """fn(rank, comm) in one thread per rank; the results by rank."""
    mb = Mailbox(size)
    out, errs = [None] * size, []

    def body(r):
        try:
            out[r] = fn(r, mb.comm(r))
        except BaseException as e:  # noqa: BLE001
            errs.append(e)
            mb.barrier.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(size)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out


def rank_job(U, N, b, psi_o, prec, dims=DIMS):
    def job(rank, comm):
        with stag.Lattice(dims) as lat:
            lat.upload_gauge(U, N, precisions=(prec,))
            d = stag.DDRank(lat, comm)
            fo = lat.field(stag.ODD, prec, psi_o)
            fe = lat.field(stag.EVEN, prec)
            d.dslash(fe, fo)
            de = fe.export()
            fb = lat.field(stag.EVEN, prec, b)
            fx = lat.field(stag.EVEN, prec)
            info = d.cg(fx, fb, MASS, 1e-10, 5000)
            x = fx.export()
            t0, nt = d.t0, d.nt
            d.close()
        return t0, nt, de, x, info
    return job


@pytest.mark.parametrize("prec", ["f64", "df64"])
@pytest.mark.parametrize("dims,size", [(DIMS, 1), (DIMS, 2), (DIMS, 3), (DIMS16, 2)])
def test_ranks_dslash_and_cg(dims, size, prec):
    U, N, b, psi_o = make_problem(dims)
    Vh = len(b)
    per = dims[0] * dims[1] * dims[2] // 2
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,))
        fo = lat.field(stag.ODD, prec, psi_o)
        fe = lat.field(stag.EVEN, prec)
        lat.dslash(fe, fo)
        want_d = fe.export()
    res = run_ranks(size, rank_job(U, N, b, psi_o, prec, dims))
    x = np.zeros_like(b)
    covered = np.zeros(Vh, bool)
    for t0, nt, de, xr, info in res:
        sl = slice(t0 * per, (t0 + nt) * per)
        assert np.array_equal(de[sl], want_d[sl]), (t0, nt)
        x[sl] = xr[sl]
        covered[sl] = True
        assert info["return"] == stag.OK, info
    assert covered.all()
    # every rank took the same decisions
    assert len({r[4]["iters"] for r in res}) == 1
    assert len({r[4]["true_rel_resid"] for r in res}) == 1
    rel = np.linalg.norm(b - oracle.apply_M(dims, U, N, MASS, x)) / np.linalg.norm(b)
    assert rel <= 1.05e-10, rel
    assert abs(rel - res[0][4]["true_rel_resid"]) <= 1e-3 * rel
    _, info_o = oracle.cg(dims, U, N, MASS, b, tol=1e-10)
    it = res[0][4]["iters"]
    assert abs(it - info_o["iters"]) <= max(3, 0.01 * info_o["iters"]), (it, info_o["iters"])


def test_nccl_single_rank_matches_mailbox(problem):
    U, N, b, psi_o = problem
    try:
        uid = stag.nccl_unique_id()
    except stag.StagError as e:
        pytest.skip(f"libstag built without NCCL: {e}")
    comm = stag.NcclComm(0, 1, uid, 0)
    try:
        t0, nt, de, x, info = rank_job(U, N, b, psi_o, "df64")(0, comm)
    finally:
        comm.close()
    t0m, ntm, dem, xm, infom = run_ranks(1, rank_job(U, N, b, psi_o, "df64"))[0]
    assert (t0, nt) == (t0m, ntm) == (0, DIMS[3])
    assert np.array_equal(de, dem)
    assert info["return"] == stag.OK and info["iters"] == infom["iters"]
    assert np.array_equal(x, xm)


def test_nccl_callbacks_single_rank():
    """The NCCL communicator's callbacks on device buffers, one rank (a rank
    that owns the whole lattice exchanges nothing, so the solver tests do not
    reach them): the exchange delivers what the rank sent to its next
    neighbour into from_prev and what it sent to its previous one into
    from_next; both allreduces return the values unchanged."""
    import torch
    try:
        uid = stag.nccl_unique_id()
    except stag.StagError as e:
        pytest.skip(f"libstag built without NCCL: {e}")
    comm = stag.NcclComm(0, 1, uid, 0)
    try:
        c = comm.struct
        n = 3 * 4096
        to_prev = torch.arange(n, dtype=torch.uint8, device="cuda")
        to_next = torch.flip(to_prev, [0]).contiguous()
        from_prev = torch.zeros(n, dtype=torch.uint8, device="cuda")
        from_next = torch.zeros(n, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = c.exchange(c.ctx, to_prev.data_ptr(), to_next.data_ptr(), from_prev.data_ptr(), from_next.data_ptr(),
                        n, stream)
        torch.cuda.synchronize()
        assert rc == 0
        assert torch.equal(from_prev, to_next) and torch.equal(from_next, to_prev)
        vals = torch.tensor([1.5, -2.25, 3e-300], dtype=torch.float64, device="cuda")
        want = vals.clone()
        assert c.allreduce_dev(c.ctx, vals.data_ptr(), 3, stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(vals, want)
        host = (ctypes.c_double * 2)(0.5, 7.0)
        assert c.allreduce(c.ctx, host, 2) == 0 and list(host) == [0.5, 7.0]
    finally:
        comm.close()


@pytest.mark.parametrize("max_iter", [0, 5, 13])
def test_nccl_max_iter_stops_exactly(problem, max_iter):
    """The device-driven CG enqueues chunks of eight iterations; max_iter cuts
    it off at the same iteration count as the host-driven path."""
    U, N, b, psi_o = problem
    try:
        uid = stag.nccl_unique_id()
    except stag.StagError as e:
        pytest.skip(f"libstag built without NCCL: {e}")
    comm = stag.NcclComm(0, 1, uid, 0)
    try:
        with stag.Lattice(DIMS) as lat:
            lat.upload_gauge(U, N, precisions=("df64",))
            d = stag.DDRank(lat, comm)
            fb = lat.field(stag.EVEN, "df64", b)
            fx = lat.field(stag.EVEN, "df64")
            info = d.cg(fx, fb, MASS, 1e-10, max_iter)
            x = fx.export()
            d.close()
    finally:
        comm.close()
    assert info["return"] == stag.ERR_NOT_CONVERGED and info["iters"] == max_iter, info
    hm = run_ranks(1, lambda rank, c: _short_cg(U, N, b, max_iter, c))[0]
    assert hm[1]["iters"] == max_iter and np.array_equal(x, hm[0])


def _short_cg(U, N, b, max_iter, comm):
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        d = stag.DDRank(lat, comm)
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        info = d.cg(fx, fb, MASS, 1e-10, max_iter)
        x = fx.export()
        d.close()
    return x, info


def test_ranks_refuse_bad_layouts(problem):
    U, N, b, psi_o = problem
    with stag.Lattice(DIMS) as lat:
        lat.upload_gauge(U, N, precisions=("f64",))
        mb = Mailbox(5)  # 12 slices over 5 ranks: slabs of 2 or 3
        with pytest.raises(stag.StagError):
            stag.DDRank(lat, mb.comm(0))
