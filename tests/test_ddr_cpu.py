"""The rank decomposition's host protocol with real gloo ranks on the CPU.

Each rank (a process, world size 2 or 3) owns a t-slab of the lattice.  With
the library's own exchange (stag_ddr_exchange_host: which slices go to which
neighbour, in which order, and where the received ones land) and gloo as the
communicator, the test checks that

* the halo a rank receives equals the single-domain field on those slices,
  and nothing outside slab and halo is written;
* a CG over the ranks, each applying the oracle's Dslash to its slab plus
  halo and summing its inner products with an allreduce, reproduces the
  one-process oracle CG's scalar history (alpha_k, beta_k, |r_{k+1}|^2) to
  1e-12 relative for the first 20 iterations.

The GPU path runs the same exchange (tests/test_gpu_ddr.py)."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CHILD = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, os.environ["ROOT"])
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1411_2087_gb300 import stag, synth

    rank, size = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=size)
    dims = tuple(json.loads(os.environ["DIMS"]))
    mass = 0.1
    Vh = int(np.prod(dims)) // 2
    per = dims[0] * dims[1] * dims[2] // 2
    Lt = dims[3]
    prev, nxt = (rank - 1) % size, (rank + 1) % size

    def exchange(to_prev, to_next):
        # one message each way to each neighbour; tags tell the two apart
        # when both neighbours are the same rank
        bufs = [torch.frombuffer(bytearray(to_next), dtype=torch.uint8),
                torch.frombuffer(bytearray(to_prev), dtype=torch.uint8)]
        fp = torch.empty(len(to_prev), dtype=torch.uint8)
        fn = torch.empty(len(to_next), dtype=torch.uint8)
        reqs = [dist.isend(bufs[0], nxt, tag=0), dist.isend(bufs[1], prev, tag=1),
                dist.irecv(fp, prev, tag=0), dist.irecv(fn, nxt, tag=1)]
        for r in reqs:
            r.wait()
        return fp.numpy().tobytes(), fn.numpy().tobytes()

    def allreduce(vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t)
        return t.tolist()

    comm = stag.HostComm(rank, size, exchange, allreduce)
    t0, nt = stag.ddr_layout(dims, size, rank)
    slab = np.zeros(Vh, bool)
    slab[t0 * per:(t0 + nt) * per] = True
    halo = np.zeros(Vh, bool)
    for t in list(range(t0 - 3, t0)) + list(range(t0 + nt, t0 + nt + 3)):
        tt = t % Lt
        halo[tt * per:(tt + 1) * per] = True
    out = {"t0": t0, "nt": nt}

    # 1. the halo of both parities
    ok = True
    for parity in (0, 1):
        g = synth.gaussian_colour_field(Vh, 50 + parity).numpy()
        loc = np.where(slab[:, None], g, 0)
        stag.ddr_exchange_host(dims, parity, comm, loc)
        ok &= np.array_equal(loc[halo], g[halo]) and np.array_equal(loc[slab], g[slab])
        ok &= not np.any(loc[~(slab | halo)])
    out["halo_ok"] = bool(ok)

    # 2. CG over the ranks: oracle Dslash on slab + halo, sums by allreduce
    U = synth.su3_field(dims, 0.3, 1000).numpy()
    N = oracle.long_links(dims, U)
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    s = slab[:, None]

    def with_halo(v, parity):
        w = np.where(s, v, 0)
        stag.ddr_exchange_host(dims, parity, comm, w)
        return w

    def gsum(v):
        return allreduce([float(v)])[0]

    x = np.zeros_like(b)
    r = np.where(s, b, 0)
    p = r.copy()
    rr = gsum(np.vdot(r, r).real)
    hist = []
    for k in range(20):
        t = oracle.dslash_parity(dims, U, N, 1, with_halo(p, 0))
        Ap = mass * mass * p - oracle.dslash_parity(dims, U, N, 0, with_halo(t, 1))
        Ap = np.where(s, Ap, 0)
        alpha = rr / gsum(np.vdot(p, Ap).real)
        x += alpha * p
        r -= alpha * Ap
        rr_new = gsum(np.vdot(r, r).real)
        beta = rr_new / rr
        hist.append([alpha, beta, rr_new])
        rr = rr_new
        p = r + beta * p
    out["hist"] = hist
    dist.barrier()
    print(json.dumps(out))
    dist.destroy_process_group()
""")


@pytest.mark.parametrize("size,dims", [(2, (4, 4, 2, 12)), (3, (4, 2, 4, 12))])
def test_gloo_ranks_exchange_and_cg_history(size, dims):
    import numpy as np

    import oracle
    from paper_1411_2087_gb300 import build as stag_build
    from paper_1411_2087_gb300 import synth

    stag_build.build()
    port = free_port()
    procs = []
    for rank in range(size):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(size), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), ROOT=ROOT, CUDA_VISIBLE_DEVICES="", DIMS=json.dumps(dims))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    # the slabs tile the lattice
    assert sorted((o["t0"], o["nt"]) for o in outs)[0][0] == 0
    assert sum(o["nt"] for o in outs) == dims[3]
    assert all(o["halo_ok"] for o in outs)
    # the one-process oracle CG
    U = synth.su3_field(dims, 0.3, 1000).numpy()
    N = oracle.long_links(dims, U)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, 1100).numpy()
    _, info = oracle.cg(dims, U, N, 0.1, b, tol=1e-10, history=True)
    want = np.array(info["history"][:20])
    for o in outs:
        got = np.array(o["hist"])
        rel = np.abs(got - want) / np.abs(want)
        assert rel.max() <= 1e-12, rel.max(axis=0)


def test_layout_rules():
    from paper_1411_2087_gb300 import stag
    assert stag.ddr_layout((4, 4, 4, 8), 1, 0) == (0, 8)
    assert stag.ddr_layout((4, 4, 4, 8), 2, 1) == (4, 4)
    # uneven: the first Lt % size ranks take one slice more
    assert [stag.ddr_layout((4, 4, 4, 10), 3, r) for r in range(3)] == [(0, 4), (4, 3), (7, 3)]
    with pytest.raises(stag.StagError):
        stag.ddr_layout((4, 4, 4, 8), 3, 0)  # slabs of 2 slices: thinner than the reach
    with pytest.raises(stag.StagError):
        stag.ddr_layout((4, 4, 4, 8), 2, 2)
