"""The bench's multi-rank path on the CPU: two gloo ranks aggregate their
timings (largest over ranks) and their work (sum) the way bench.py reports
the whole-job rate under torchrun."""
import json
import os
import socket
import subprocess
import sys
import textwrap

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
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=2)
    r = dist.get_rank()
    out = bench.aggregate_ranks(dist, [10.0 + r, 5.0 - r, 1.0 + 2 * r], [100.0 * (r + 1), 7.0])
    dist.barrier()
    print(json.dumps(out))
    dist.destroy_process_group()
""")


def test_two_gloo_ranks_aggregate():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        # times: max over ranks; work: sum
        assert o == [11.0, 5.0, 3.0, 300.0, 14.0]


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(None, [1, 2], [3]) == [1.0, 2.0, 3.0]
