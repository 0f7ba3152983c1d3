"""Benchmark: even-odd CG solve to a 1e-10 true residual on a 32^3x64 lattice.

One step is one full solve of M x = b, M = m^2 - D_eo D_oe, m = 0.02, on
synthetic eps = 0.3 SU(3) fat links with their three-link products (every
row of the hot path: two Dslash per iteration, the fused M epilogue and dot
products, the fused vector updates, the device-side stopping test and the
final true residual).  Inputs are resident in HBM when the timed region
starts; they are larger than L2 (the links alone are 2.4 GB), so no flush is
needed between steps.

value  = algorithmic GB/s sustained over the solve
         (iterations * bytes per iteration / solve time),
plus the Dslash kernel's own GB/s (algorithmic bytes per launch / launch time
from CUDA events on the lattice stream) in "roofline", the solve time in
"cg", the end-to-end rate through the C ABI with host buffers in "e2e", and
the CPU oracle on a bounded sample in "cpu_baseline".

--impl reference runs the CPU oracle (the reference arm of this project) on
the host cores instead.  N > 1 (torchrun) runs one independent solve per rank
per step (different sources; no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

DIMS = (32, 32, 32, 64)
MASS = 0.02
TOL = 1e-10
EPS = 0.3
SEED_LINKS = 1001
SEED_SOURCE = 1101
METRIC = "Dslash GB/s (% HBM peak) & CG time-to-1e-10 residual, mixed/learned vs FP64"
DSLASH_SOURCES = ["common.cuh", "fields.cuh", "dslash.cuh", "dslash_launch.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="df64", choices=["df64", "f64"])
    ap.add_argument("--dims", default=None, help="override lattice, e.g. 16,16,16,32")
    ap.add_argument("--dslash-launches", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision comparison on the 48^3x96 workload")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-preconditioner comparison on the 32^3x64, m=0.005 workload")
    ap.add_argument("--no-dd", action="store_true",
                    help="skip the one-lattice-over-the-ranks (domain decomposition) section")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the IEEE FP64 and reduced-precision-error sections")
    ap.add_argument("--learned-pairs", type=int, default=4096)
    ap.add_argument("--learned-epochs", type=int, default=2)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched / multi-shift comparison (16 RHS on three lattices, 12 shifts)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time the Dslash kernels of every precision on --dims (autotuner launches) and exit")
    ap.add_argument("--compress12", action="store_true",
                    help="with --kernels-only: 12-real links for the FP32 and 16-bit copies")
    ap.add_argument("--kernels-prec", default="f64,df64,f32,f16",
                    help="with --kernels-only: the precisions to time (comma-separated)")
    ap.add_argument("--net-only", action="store_true",
                    help="time one application of the learned preconditioner (solver form) and exit")
    ap.add_argument("--cg-launch", default="graph", choices=["graph", "host"],
                    help="host: the same CG kernels launched one by one (per-kernel profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dslash_source_hash() -> str:
    h = hashlib.sha256()
    for n in DSLASH_SOURCES:
        with open(os.path.join(ROOT, "paper_1411_2087_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(prec: str, dims):
    """DRAM bytes per Dslash launch from the committed ncu summary, if it was
    taken on the current kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", "dslash_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    key = f"bytes_per_site_{prec}"
    if rec.get("source_hash") != dslash_source_hash() or key not in rec:
        return None
    return float(rec[key]) * (int(np.prod(dims)) // 2)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region
    (read through a pipe by a background thread)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = self.smi_id(device_index)
        self.proc = None
        self.reader = None
        self.lines = []
        self.first = threading.Event()

    @staticmethod
    def smi_id(device_index: int) -> str:
        """The GPU's UUID for nvidia-smi (the CUDA index differs from
        nvidia-smi's when CUDA_VISIBLE_DEVICES remaps devices)."""
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device_index).uuid)
            if u:
                return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        return str(device_index)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)
            self.first.set()
        self.first.set()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        if self.proc is not None:
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            # nvidia-smi's start-up (process, NVML) must not overlap the timed
            # region: wait for its first sample (at most 3 s)
            self.first.wait(timeout=3.0)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.reader is not None:
                self.reader.join(timeout=5)

    def summary(self):
        rows = []
        for line in list(self.lines):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def make_inputs(dims, device, rank):
    import torch
    from paper_1411_2087_gb300 import synth
    U = synth.su3_field(dims, EPS, SEED_LINKS, device=device)
    Vh = int(np.prod(dims)) // 2
    b = synth.gaussian_colour_field(Vh, SEED_SOURCE + rank)
    return U, b


def aggregate_ranks(pg, times, work):
    """Whole-job figures: the largest time of each kind over the ranks and
    the sum of the work, through torch.distributed `pg` (None: one rank).
    Returns times followed by work, as floats."""
    import torch
    if pg is None:
        return [float(t) for t in times] + [float(w) for w in work]
    t = torch.tensor([float(v) for v in times], dtype=torch.float64)
    w = torch.tensor([float(v) for v in work], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(w, op=pg.ReduceOp.SUM)
    return [float(v) for v in t] + [float(v) for v in w]


def cg_bytes_per_iter_site(prec):
    from paper_1411_2087_gb300 import metrics
    return metrics.cg_bytes_per_iteration_per_site(8)


def run_native(args):
    import torch
    from paper_1411_2087_gb300 import metrics, stag

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else DIMS
    Vh = int(np.prod(dims)) // 2
    prec = args.prec

    U, b_host = make_inputs(dims, dev, rank)
    torch.cuda.synchronize()
    # all library work goes to this stream; CUDA events are recorded on it
    stream = torch.cuda.Stream(dev)
    lat = stag.Lattice(dims, device=local, stream=stream.cuda_stream)
    lat.upload_gauge(U, None, precisions=(prec,))
    lat.set_cg_launch(args.cg_launch)
    tuned = lat.autotune(prec)
    block = min(tuned["dslash_us"], key=tuned["dslash_us"].get)
    del U
    torch.cuda.empty_cache()
    b_pinned = b_host.pin_memory()
    x_pinned = torch.empty_like(b_pinned).pin_memory()
    fb = lat.field(stag.EVEN, prec, b_pinned)
    fx = lat.field(stag.EVEN, prec)

    def barrier():
        if pg is not None:
            pg.barrier()

    # warm-up (also builds the solve graph)
    for _ in range(args.warmup):
        info = lat.cg(fx, fb, MASS, TOL, 20000)
    assert info["return"] == stag.OK, info

    # ---- timed: device-resident solves
    iters = []
    solve_ms = []
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            info = lat.cg(fx, fb, MASS, TOL, 20000)
            iters.append(info["iters"])
            solve_ms.append(info["seconds"] * 1e3)
            assert info["return"] == stag.OK, info
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        # ---- Dslash launches alone, CUDA events on the lattice stream
        fo = lat.field(stag.ODD, prec)
        fo2 = lat.field(stag.EVEN, prec)
        for _ in range(10):
            lat.dslash(fo, fb)
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for k in range(args.dslash_launches):
            if k % 2 == 0:
                lat.dslash(fo, fb)
            else:
                lat.dslash(fo2, fo)
        d1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    clocks = clk.summary()
    total_ms = e0.elapsed_time(e1)
    dslash_ms = d0.elapsed_time(d1) / args.dslash_launches

    # ---- end to end through the C ABI with host buffers
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.steps):
        fb.import_(b_pinned)              # host -> device
        info = lat.cg(fx, fb, MASS, TOL, 20000)
        fx.export(x_pinned)               # device -> host
        e2e_iters += info["iters"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # ---- aggregate over ranks (max time, sum of work)
    bpi = cg_bytes_per_iter_site(prec) * Vh
    total_ms, e2e_s, dslash_ms, work_bytes, e2e_bytes = aggregate_ranks(
        pg, [total_ms, e2e_s, dslash_ms], [sum(iters) * bpi, e2e_iters * bpi])
    value = work_bytes / (total_ms * 1e-3) / 1e9
    e2e_value = e2e_bytes / e2e_s / 1e9

    peak, peak_kind = measured_peak()
    alg_dslash = metrics.dslash_bytes_per_site(8) * Vh
    achieved = alg_dslash / (dslash_ms * 1e-3) / 1e9
    # per iteration: D_oe, M with <p, Mp> partials, their sum, update, p update;
    # per solve: init and the two kernels of the true residual
    launches_per_solve = [5 * k + 3 for k in iters]
    gpu_launches = sum(launches_per_solve) + args.dslash_launches

    lat.close()
    torch.cuda.empty_cache()

    # the comparison sections are single-GPU measurements: reported on the
    # one-GPU line, skipped when several ranks run (the scaling runs)
    small = small_config(local) if world == 1 else None
    mixed = None
    if not args.no_mixed and world == 1:
        mixed = mixed_comparison(local, rank, args.cg_launch)
    batched = None
    if not args.no_batched and world == 1:
        batched = batched_comparison(local, rank)
    # one lattice split over the ranks (strong scaling), on every N
    ddr = None if args.no_dd else dd_section(local, rank, world, pg, args.steps)
    fp64 = None
    precision = None
    if not args.no_precision and world == 1:
        fp64 = fp64_ieee_section(local, rank)
        precision = precision_error_section(local, rank)
    learned = None
    if not args.no_learned and world == 1:
        learned = learned_comparison(local, rank, args.learned_pairs, args.learned_epochs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(dims, rank)

    if rank != 0:
        return None
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "df64" if prec == "df64" else "f64",
        "data": "synthetic (seeded SU(3) links eps=0.3, three-link products, Gaussian source)",
        "config": {
            "workload": f"even-odd CG to 1e-10 true residual, {'x'.join(map(str, dims))} lattice, m={MASS}",
            "lattice": list(dims), "mass": MASS, "tol": TOL, "eps": EPS,
            "prec": prec, "global_batch": world, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (links 2.4 GB), no flush",
            "step": "one CG solve (init, iterations, true residual)",
            "cg_launch": args.cg_launch,
        },
        "cg": {"iters": iters[0], "seconds_per_solve": round(statistics.median(solve_ms) * 1e-3, 4),
               "true_rel_resid": info["true_rel_resid"], "gflops": round(info["gflops"], 1)},
        "dslash": {"gbs": round(achieved, 1), "pct_hbm": round(100 * achieved / peak, 1),
                   "gflops": round(1146 * Vh / (dslash_ms * 1e-3) / 1e9, 1),
                   "us_per_launch": round(dslash_ms * 1e3, 2)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic(prec, dims),
                     "kernel": f"dslash_kernel<{prec}, EPI_NONE, {block}>",
                     "peak_source": peak_kind},
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s",
                "h2d_bytes_per_step": Vh * 48, "d2h_bytes_per_step": Vh * 48},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "small_8x8x8x8": small,
        "mixed_vs_fp64": mixed,
        "batched_multishift": batched,
        "learned_vs_fp64": learned,
        "fp64_ieee": fp64,
        "precision_error": precision,
        "domain_decomposition": ddr,
    }
    return line


def dd_section(local, rank, world, pg, steps):
    """The main workload (32^3x64, m = 0.02, to 1e-10, double float) as one
    lattice cut in t over the N ranks (stag_ddr_*), NCCL as the communicator:
    strong scaling.  Seconds per solve are the largest over the ranks; GB/s
    counts the whole lattice's CG bytes (iterations x 5280 B x Vh)."""
    import torch
    from paper_1411_2087_gb300 import stag
    if DIMS[3] // world < 3:
        return {"skipped": f"{world} ranks leave slabs thinner than 3 of {DIMS[3]} slices"}
    dev = torch.device("cuda", local)
    # rank 0 makes the NCCL id; every rank learns the id or why there is
    # none, so that no rank waits in the broadcast for one that gave up
    uid, err = None, None
    if rank == 0:
        try:
            uid = stag.nccl_unique_id()
        except stag.StagError as e:
            err = str(e)
    if pg is not None:
        box = [(uid, err)]
        pg.broadcast_object_list(box, src=0)
        uid, err = box[0]
    if err is not None:
        return {"skipped": err}
    U, b_host = make_inputs(DIMS, dev, 0)
    torch.cuda.synchronize()
    Vh = int(np.prod(DIMS)) // 2
    stream = torch.cuda.Stream(dev)
    comm = stag.NcclComm(rank, world, uid, local)
    # NCCL may print a banner through C stdio: out before the JSON line
    ctypes.CDLL(None).fflush(None)
    try:
        with stag.Lattice(DIMS, device=local, stream=stream.cuda_stream) as lat:
            lat.upload_gauge(U, None, precisions=("df64",))
            del U
            torch.cuda.empty_cache()
            lat.autotune("df64")
            d = stag.DDRank(lat, comm)
            fb = lat.field(stag.EVEN, "df64", b_host)
            fx = lat.field(stag.EVEN, "df64")
            info = d.cg(fx, fb, MASS, TOL, 20000)
            n = max(1, min(int(steps), 5))
            if pg is not None:
                pg.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n):
                info = d.cg(fx, fb, MASS, TOL, 20000)
            torch.cuda.synchronize()
            secs = (time.perf_counter() - t0) / n
            d.close()
    finally:
        comm.close()
    secs, _ = aggregate_ranks(pg, [secs], [0.0])
    return {"workload": f"{'x'.join(map(str, DIMS))}, m={MASS}, tol={TOL}, double float, one lattice over "
                        f"{world} rank(s) split in t",
            "ranks": world, "scaling": "strong", "comm": "nccl",
            "seconds_per_solve": round(secs, 4), "iters": info["iters"],
            "gbs": round(info["iters"] * cg_bytes_per_iter_site("df64") * Vh / secs / 1e9, 1),
            "true_rel_resid": info["true_rel_resid"], "ok": info["return"] == stag.OK,
            "slab": stag.ddr_layout(DIMS, world, rank)}


# nominal GB300 FP64 rate (FLOP/s); the stencil needs 576 FP64 multiply-adds
# (1146 flops with the sums) per site
FP64_NOMINAL_FLOPS = 1.25e12


def fp64_ieee_section(local, rank):
    """The main workload (32^3x64, m = 0.02, to 1e-10) in IEEE FP64 storage
    and arithmetic: CG seconds and iterations, and the Dslash rate against
    both the HBM roof and the FP64-pipe bound (1146 flops per site at the
    nominal 1.25 TFLOP/s)."""
    import torch
    from paper_1411_2087_gb300 import metrics, stag
    dev = torch.device("cuda", local)
    U, b_host = make_inputs(DIMS, dev, rank)
    torch.cuda.synchronize()
    Vh = int(np.prod(DIMS)) // 2
    stream = torch.cuda.Stream(dev)
    out = {"workload": f"{'x'.join(map(str, DIMS))}, m={MASS}, tol={TOL}, IEEE FP64"}
    with stag.Lattice(DIMS, device=local, stream=stream.cuda_stream) as lat:
        lat.upload_gauge(U, None, precisions=("f64",))
        del U
        torch.cuda.empty_cache()
        tuned = lat.autotune("f64")
        fb = lat.field(stag.EVEN, "f64", b_host)
        fx = lat.field(stag.EVEN, "f64")
        fo = lat.field(stag.ODD, "f64")
        lat.cg(fx, fb, MASS, TOL, 20000)
        info = lat.cg(fx, fb, MASS, TOL, 20000)
        for _ in range(5):
            lat.dslash(fo, fb)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(50):
            lat.dslash(fo, fb)
        ev1.record(stream)
        torch.cuda.synchronize()
        us = ev0.elapsed_time(ev1) / 50 * 1e3
    peak, peak_kind = measured_peak()
    gbs = metrics.dslash_bytes_per_site(8) * Vh / (us * 1e-6) / 1e9
    flops = 1146 * Vh / (us * 1e-6)
    out["cg"] = {"seconds": round(info["seconds"], 4), "iters": info["iters"],
                 "true_rel_resid": info["true_rel_resid"], "ok": info["return"] == stag.OK}
    out["dslash"] = {"us_per_launch": round(us, 2), "gbs": round(gbs, 1),
                     "frac_hbm": round(gbs / peak, 4), "hbm_peak_source": peak_kind,
                     "tflops": round(flops / 1e12, 3),
                     "frac_fp64_pipe": round(flops / FP64_NOMINAL_FLOPS, 4),
                     "fp64_pipe_peak_tflops": FP64_NOMINAL_FLOPS / 1e12,
                     "fp64_pipe_peak_source": "nominal",
                     "block": min(tuned["dslash_us"], key=tuned["dslash_us"].get)}
    return out


def precision_error_section(local, rank):
    """Error of every reduced-precision operator against the double-float
    one on the main workload's lattice and source (32^3x64): max-norm
    relative error of D_oe b and of M b = m^2 b - D_eo D_oe b, for FP32 and
    16-bit storage with full and 12-real (two-row) links, against double
    float (itself within 1e-12 of the FP64 oracle in the GPU tests)."""
    import torch
    from paper_1411_2087_gb300 import stag
    dev = torch.device("cuda", local)
    U, b_host = make_inputs(DIMS, dev, rank)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)
    out = {"workload": f"{'x'.join(map(str, DIMS))}, eps={EPS}, Gaussian source; reference: double-float",
           "norm": "max |got - ref| / max |ref|"}
    with stag.Lattice(DIMS, device=local, stream=stream.cuda_stream) as lat:
        ref = {}
        for compress in (False, True):
            lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"), compress12=compress)
            for prec in (("df64", "f32", "f16") if not compress else ("f32", "f16")):
                fb = lat.field(stag.EVEN, prec, b_host)
                fo = lat.field(stag.ODD, prec)
                fm = lat.field(stag.EVEN, prec)
                lat.dslash(fo, fb)
                lat.apply_M(fm, fb, MASS)
                d, m = fo.export(), fm.export()
                for f in (fb, fo, fm):
                    f.destroy()
                if prec == "df64":
                    ref = {"dslash": d, "M": m}
                    continue
                key = prec + ("_c12" if compress else "")
                out[key] = {op: float(np.abs(v - ref[op]).max() / np.abs(ref[op]).max())
                            for op, v in (("dslash", d), ("M", m))}
    del U
    torch.cuda.empty_cache()
    return out


LEARNED_DIMS = (32, 32, 32, 64)
LEARNED_MASS = 0.005


def learned_comparison(local, rank, n_pairs, epochs):
    """32^3x64, eps = 0.3, m = 0.005 to a 1e-10 true residual: double-float
    CG against flexible CG with the trained gauge-covariant net (3 layers,
    8 channels, residual loss; in the solve binary16 weights, 16-bit links,
    FP32 arithmetic), and mixed 16-bit CG against the same mixed iteration
    with the net (flexible, double-float reliable updates).  Training pairs
    (r_k, x* - x_k) come from plain CG on as many sources of the same gauge
    field as the pair count needs; the timed solves use another source.
    Collection and training times are reported separately, and the net's
    application time (CUDA events, solver form) beside them."""
    import torch
    from paper_1411_2087_gb300 import stag, synth
    dev = torch.device("cuda", local)
    U = synth.su3_field(LEARNED_DIMS, 0.3, 1010, device=dev)
    torch.cuda.synchronize()
    Vh = int(np.prod(LEARNED_DIMS)) // 2
    out = {"workload": f"{'x'.join(map(str, LEARNED_DIMS))}, m={LEARNED_MASS}, eps=0.3, tol=1e-10"}
    stream = torch.cuda.Stream(dev)
    with stag.Lattice(LEARNED_DIMS, device=local, stream=stream.cuda_stream) as lat:
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"))
        for p in ("df64", "f16"):
            lat.autotune(p)
        net = stag.Net(lat, U, channels=8, seed=1)
        del U
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("learned_collect")
        # half the pairs from each of two sources, spread over the solve; a
        # request beyond what two solves hold (one pair per iteration) draws
        # further sources
        per_src = max(1, (n_pairs + 1) // 2)
        fx = lat.field(stag.EVEN, "df64")
        left, src = n_pairs, 0
        while left > 0 and src < 64:
            fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1400 + src))
            iters = lat.cg(fx, fb, LEARNED_MASS, 1e-10, 20000)["iters"]
            want = min(left, per_src)
            left -= net.collect_pairs(fb, LEARNED_MASS, 1e-10, stride=max(1, iters // (want + 1)),
                                      max_pairs=want)
            fb.destroy()
            src += 1
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        t1 = time.perf_counter()
        net.set_loss("residual")
        torch.cuda.nvtx.range_push("learned_train")
        hist = net.train(epochs=epochs, batch=8, lr=1e-2, seed=3)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        t2 = time.perf_counter()
        b = synth.gaussian_colour_field(Vh, 1500 + rank)
        fb = lat.field(stag.EVEN, "df64", b)
        fr = lat.field(stag.EVEN, "df64")

        def resid():
            lat.apply_M(fr, fx, LEARNED_MASS)
            r = fr.export() - b.numpy()
            return float(np.linalg.norm(r) / np.linalg.norm(b.numpy()))

        # one application of the net in the solver's form (DF64 in and out)
        fz = lat.field(stag.EVEN, "df64")
        for _ in range(3):
            net.apply(fz, fb, fp16_weights=True, links16=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(20):
            net.apply(fz, fb, fp16_weights=True, links16=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        out["net_apply_ms"] = round(ev0.elapsed_time(ev1) / 20, 4)
        fz.destroy()
        runs = {}
        for name, fn in (("fp64_df64_cg", lambda: lat.cg(fx, fb, LEARNED_MASS, 1e-10, 20000)),
                         ("mixed_f16_cg", lambda: lat.cg_mixed(fx, fb, LEARNED_MASS, 1e-10, 20000, "f16")),
                         ("learned_fcg_df64", lambda: net.cg(fx, fb, LEARNED_MASS, 1e-10, 20000)),
                         ("learned_mixed_f16",
                          lambda: net.cg_mixed(fx, fb, LEARNED_MASS, 1e-10, 20000, "f16"))):
            fn()
            torch.cuda.synchronize()
            ta = time.perf_counter()
            info = fn()
            torch.cuda.synchronize()
            tb = time.perf_counter()
            res = resid()
            runs[name] = {"seconds": round(tb - ta, 4), "iters": info["iters"], "true_rel_resid": res,
                          "ok": info["return"] == stag.OK and res <= 1.05e-10}
        base = runs["fp64_df64_cg"]
        for name in ("mixed_f16_cg", "learned_fcg_df64", "learned_mixed_f16"):
            runs[name]["speedup_vs_fp64"] = round(base["seconds"] / runs[name]["seconds"], 3)
            runs[name]["iteration_ratio_vs_fp64"] = round(base["iters"] / max(1, runs[name]["iters"]), 3)
        # what the net adds to the mixed iteration by itself
        runs["learned_mixed_f16"]["speedup_vs_mixed_f16"] = round(
            runs["mixed_f16_cg"]["seconds"] / runs["learned_mixed_f16"]["seconds"], 3)
        out.update(runs)
        out["training"] = {"pairs": net.num_pairs(), "epochs": epochs, "collect_seconds": round(t1 - t0, 2),
                           "train_seconds": round(t2 - t1, 2), "loss_first": float(hist[0]),
                           "loss_last": float(hist[-1]), "loss": "residual |M N r - r|^2/|r|^2"}
        net.close()
    return out


BATCH_LATTICES = (((16, 16, 16, 16), 6, 1003), ((24, 24, 24, 48), 5, 1004), ((32, 32, 32, 64), 5, 1005))
BATCH_MASS = 0.02
MS_DIMS = (24, 24, 24, 48)
MS_SHIFTS = list(np.geomspace(1e-4, 0.5, 12))


def batched_comparison(local, rank):
    """16 Gaussian right-hand sides on 16^4, 24^3x48 and 32^3x64 (6 + 5 + 5,
    m = 0.02, eps = 0.3) to a 1e-10 true residual: one after another with
    double-float CG, in one batched double-float graph, and as one batched
    FP32 graph refined per system with FP32- or 16-bit-inner reliable
    updates.  Then 12 shifts 1e-4..0.5 (log-spaced) on 24^3x48: 12 separate
    double-float solves against one double-float multi-shift solve and against
    the mixed multi-shift solve (double-float vectors, the Dslash pair in FP32
    on 12-real links once |r| < 1e-4 |b|, reliable updates; shifts refined
    only if they miss the tolerance).  One warm-up each; wall time of the
    timed call."""
    import torch
    from paper_1411_2087_gb300 import stag, synth
    dev = torch.device("cuda", local)
    out = {"batched_workload": "16 RHS: 6 on 16^4, 5 on 24^3x48, 5 on 32^3x64; m=0.02, eps=0.3, tol=1e-10",
           "multishift_workload": "12 shifts geomspace(1e-4, 0.5) on 24^3x48, m=0.02, eps=0.3, tol=1e-10"}
    lats, systems = [], []
    for dims, nrhs, seed in BATCH_LATTICES:
        U = synth.su3_field(dims, 0.3, seed, device=dev)
        torch.cuda.synchronize()
        lat = stag.Lattice(dims, device=local)
        # 12-real FP32 / 16-bit copies for the stencils of the mixed solvers
        # (the batched FP32 kernels keep the full copies)
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"), compress12=True)
        del U
        for p in ("df64", "f32", "f16"):
            lat.autotune(p)
        lats.append(lat)
        Vh = int(np.prod(dims)) // 2
        for k in range(nrhs):
            b = synth.gaussian_colour_field(Vh, 3000 + 17 * seed + k + 100 * rank)
            systems.append((lat, lat.field(stag.EVEN, "df64"), lat.field(stag.EVEN, "df64", b), BATCH_MASS))
    torch.cuda.empty_cache()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    maxit = 5000  # bounds the section's run time should a solve misbehave

    def one_by_one():
        return [lat.cg(x, b, m, 1e-10, maxit) for lat, x, b, m in systems]

    t_seq, infos = timed(one_by_one)
    ok_seq = all(i["return"] == stag.OK for i in infos)
    t_b, (st_b, infos_b) = timed(lambda: stag.cg_batched(systems, 1e-10, maxit))
    t_m32, (st_m32, infos_m32) = timed(lambda: stag.cg_batched(systems, 1e-10, maxit, mixed="f32"))
    t_m16, (st_m16, infos_m16) = timed(lambda: stag.cg_batched(systems, 1e-10, maxit, mixed="f16"))

    def worst(infs):
        return max(i["true_rel_resid"] for i in infs)

    out["sequential_df64_cg"] = {"seconds": round(t_seq, 4), "ok": ok_seq,
                                 "iters": [i["iters"] for i in infos]}
    out["batched_df64"] = {"seconds": round(t_b, 4), "ok": st_b == stag.OK,
                           "max_true_rel_resid": worst(infos_b),
                           "speedup_vs_sequential": round(t_seq / t_b, 3)}
    out["batched_f32_refined_f32"] = {"seconds": round(t_m32, 4), "ok": st_m32 == stag.OK,
                                      "max_true_rel_resid": worst(infos_m32),
                                      "speedup_vs_sequential": round(t_seq / t_m32, 3)}
    out["batched_f32_refined_f16"] = {"seconds": round(t_m16, 4), "ok": st_m16 == stag.OK,
                                      "max_true_rel_resid": worst(infos_m16),
                                      "speedup_vs_sequential": round(t_seq / t_m16, 3)}
    # multi-shift on the 24^3x48 lattice of the batch
    lat = lats[1]
    b = systems[6][2]
    xs = [lat.field(stag.EVEN, "df64") for _ in MS_SHIFTS]

    def separate():
        return [lat.cg(x, b, float(np.sqrt(BATCH_MASS ** 2 + s)), 1e-10, maxit)
                for x, s in zip(xs, MS_SHIFTS)]

    t_sep, inf_sep = timed(separate)
    t_ms, (st_ms, inf_ms) = timed(lambda: lat.cg_multishift(xs, b, MS_SHIFTS, BATCH_MASS, 1e-10, maxit))
    t_msm, (st_msm, inf_msm) = timed(lambda: lat.cg_multishift(xs, b, MS_SHIFTS, BATCH_MASS, 1e-10, maxit,
                                                               mixed="f16"))
    out["separate_df64_cg_12_shifts"] = {"seconds": round(t_sep, 4),
                                         "ok": all(i["return"] == stag.OK for i in inf_sep),
                                         "iters": [i["iters"] for i in inf_sep]}
    out["multishift_df64"] = {"seconds": round(t_ms, 4), "ok": st_ms == stag.OK,
                              "iters": max(i["iters"] for i in inf_ms),
                              "max_true_rel_resid": worst(inf_ms),
                              "speedup_vs_separate": round(t_sep / t_ms, 3)}
    out["multishift_mixed"] = {"seconds": round(t_msm, 4), "ok": st_msm == stag.OK,
                               "iters": max(i["iters"] for i in inf_msm),
                               "refinement_iters": sum(i["restarts"] for i in inf_msm),
                               "max_true_rel_resid": worst(inf_msm),
                               "speedup_vs_separate": round(t_sep / t_msm, 3),
                               "speedup_vs_multishift_df64": round(t_ms / t_msm, 3)}
    for lat in lats:
        lat.close()
    return out


def small_config(local):
    """The 8^4 parity configuration (eps = 0.3, seed 1000, m = 0.1, tol
    1e-10): too small to fill the GPU (2048 sites per parity), reported for
    completeness.  Median of 5 double-float CG solves after 2 warm-ups."""
    import torch
    from paper_1411_2087_gb300 import stag, synth
    dims, mass = (8, 8, 8, 8), 0.1
    Vh = int(np.prod(dims)) // 2
    U = synth.su3_field(dims, 0.3, 1000, device=torch.device("cuda", local))
    torch.cuda.synchronize()
    with stag.Lattice(dims, device=local) as lat:
        lat.upload_gauge(U, None, precisions=("df64",))
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1100))
        fx = lat.field(stag.EVEN, "df64")
        for _ in range(2):
            lat.cg(fx, fb, mass, 1e-10, 5000)
        runs = [lat.cg(fx, fb, mass, 1e-10, 5000) for _ in range(5)]
    sec = statistics.median(r["seconds"] for r in runs)
    return {"workload": "even-odd CG to 1e-10, 8x8x8x8, m=0.1, eps=0.3 (launch-bound)",
            "iters": runs[0]["iters"], "seconds_per_solve": round(sec, 6),
            "us_per_iteration": round(1e6 * sec / max(1, runs[0]["iters"]), 2),
            "true_rel_resid": runs[0]["true_rel_resid"],
            "ok": all(r["return"] == stag.OK for r in runs)}


MIXED_DIMS = (48, 48, 48, 96)
MIXED_MASS = 0.01
MIXED_EPS = 0.35
MIXED_DELTA = 0.1


def mixed_comparison(local, rank, cg_launch):
    """Time to a 1e-10 true residual on the 48^3x96, m = 0.01, eps = 0.35
    workload: double-float CG against mixed precision (FP32 and 16-bit inner
    iterations with double-float reliable updates, delta = 0.1) on full
    links, on 12-real links and (16-bit) on 12-real three-link links only.
    One warm-up and one timed solve each; the true residual of every
    returned x is recomputed in double-float."""
    import torch
    from paper_1411_2087_gb300 import stag, synth
    dev = torch.device("cuda", local)
    U = synth.su3_field(MIXED_DIMS, MIXED_EPS, 1002, device=dev)
    Vh = int(np.prod(MIXED_DIMS)) // 2
    b = synth.gaussian_colour_field(Vh, 1102 + rank)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)
    out = {"workload": f"{'x'.join(map(str, MIXED_DIMS))}, m={MIXED_MASS}, eps={MIXED_EPS}, tol=1e-10"}
    with stag.Lattice(MIXED_DIMS, device=local, stream=stream.cuda_stream) as lat:
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"))
        lat.set_cg_launch(cg_launch)
        del U
        torch.cuda.empty_cache()
        fb = lat.field(stag.EVEN, "df64", b)
        fx = lat.field(stag.EVEN, "df64")
        fr = lat.field(stag.EVEN, "df64")
        runs = (("fp64_df64", lambda: lat.cg(fx, fb, MIXED_MASS, 1e-10, 20000)),
                ("mixed_f32", lambda: lat.cg_mixed(fx, fb, MIXED_MASS, 1e-10, 20000, "f32", MIXED_DELTA)),
                ("mixed_f16", lambda: lat.cg_mixed(fx, fb, MIXED_MASS, 1e-10, 20000, "f16", MIXED_DELTA)))

        def run_all(tag, which):
            for name, fn in which:
                fn()
                # an NVTX range per timed solve, e.g. "mixed_f16_c12", so that a
                # profiler can select one solve's kernels
                torch.cuda.nvtx.range_push(name + tag)
                info = fn()
                torch.cuda.nvtx.range_pop()
                lat.apply_M(fr, fx, MIXED_MASS)
                r = fr.export() - b.numpy()
                res = float(np.linalg.norm(r) / np.linalg.norm(b.numpy()))
                out[name + tag] = {"seconds": round(info["seconds"], 4), "iters": info["iters"],
                                   "reliable_updates": info["restarts"], "true_rel_resid": res,
                                   "ok": info["return"] == stag.OK and res <= 1.05e-10}

        for p in ("df64", "f32", "f16"):
            lat.autotune(p)
        run_all("", runs)
        # the same inner solves on 12-real (two-row) links, the paper's compression
        U = synth.su3_field(MIXED_DIMS, MIXED_EPS, 1002, device=dev)
        lat.upload_gauge(U, None, precisions=("df64", "f32", "f16"), compress12=True)
        del U
        torch.cuda.empty_cache()
        for p in ("f32", "f16"):
            lat.autotune(p)
        run_all("_c12", runs[1:])
        # 12-real three-link links only, full one-link links (the form for
        # smeared fat links, which are not in SU(3))
        U = synth.su3_field(MIXED_DIMS, MIXED_EPS, 1002, device=dev)
        lat.upload_gauge(U, None, precisions=("df64", "f16"), compress12="long")
        del U
        torch.cuda.empty_cache()
        lat.autotune("f16")
        run_all("_c12long", runs[2:])
        base = out["fp64_df64"]["seconds"]
        for name in ("mixed_f32", "mixed_f16", "mixed_f32_c12", "mixed_f16_c12", "mixed_f16_c12long"):
            out[name]["speedup_vs_fp64"] = round(base / out[name]["seconds"], 3)
    return out


class OracleWorkload:
    """The bench workload on the host, for the CPU oracle."""

    def __init__(self, dims, rank):
        import oracle
        from paper_1411_2087_gb300 import synth
        self.oracle = oracle
        self.dims = dims
        self.U = synth.su3_field(dims, EPS, SEED_LINKS).numpy()
        self.N = oracle.long_links(dims, self.U)
        Vh = int(np.prod(dims)) // 2
        self.b = synth.gaussian_colour_field(Vh, SEED_SOURCE + rank).numpy()

    def run(self, n_iter):
        """Time `n_iter` CG iterations (plus the final true-residual check)."""
        t0 = time.perf_counter()
        x, info = self.oracle.cg(self.dims, self.U, self.N, MASS, self.b, tol=TOL, max_iter=n_iter)
        return info["iters"], time.perf_counter() - t0, self.oracle.num_threads()

    def dslash_ms(self, reps=3):
        """Median time of one oracle D_oe on the source."""
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            self.oracle.dslash_parity(self.dims, self.U, self.N, 1, self.b)
            ts.append(time.perf_counter() - t0)
        return 1e3 * float(np.median(ts))


def cpu_baseline(dims, rank, n_iter=150, n_iter_1=5):
    """The oracle on the host cores: n_iter CG iterations with every core,
    n_iter_1 with one thread, and the median of three Dslash applications."""
    Vh = int(np.prod(dims)) // 2
    wl = OracleWorkload(dims, rank)
    it, dt, cores = wl.run(n_iter)
    gbs = it * cg_bytes_per_iter_site("f64") * Vh / dt / 1e9
    dslash_ms = wl.dslash_ms()
    wl.oracle.set_num_threads(1)
    try:
        it1, dt1, _ = wl.run(n_iter_1)
    finally:
        wl.oracle.set_num_threads(cores)
    gbs1 = it1 * cg_bytes_per_iter_site("f64") * Vh / dt1 / 1e9
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{it} CG iterations of the FP64 oracle on the same {'x'.join(map(str, dims))} "
                      f"workload ({dt:.1f} s incl. the final true-residual check), "
                      f"rate = iterations * bytes/iteration / time",
            "single_thread": {"value": round(gbs1, 3), "unit": "GB/s", "cores": 1,
                              "sample": f"{it1} CG iterations ({dt1:.1f} s incl. the true-residual check)"},
            "dslash_ms": {"value": round(dslash_ms, 1), "cores": cores,
                          "sample": "median of 3 oracle D_oe applications on the workload's source"}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else DIMS
    Vh = int(np.prod(dims)) // 2
    wl = OracleWorkload(dims, 0)
    for _ in range(args.warmup):
        wl.run(1)
    times, its = [], []
    cores = 1
    for _ in range(args.steps):
        it, dt, cores = wl.run(3)
        times.append(dt)
        its.append(it)
    bpi = cg_bytes_per_iter_site("f64") * Vh
    value = sum(its) * bpi / sum(times) / 1e9
    return {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(times) / len(times), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SU(3) links eps=0.3, three-link products, Gaussian source)",
        "config": {"workload": f"even-odd CG to 1e-10 true residual, {'x'.join(map(str, dims))} "
                               f"lattice, m={MASS}", "lattice": list(dims), "mass": MASS,
                   "tol": TOL, "eps": EPS, "prec": "f64"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: 3 CG iterations of the FP64 CPU oracle on the "
                                   "same workload (plus its final true-residual check)"},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_kernels_only(args):
    """Dslash kernel timings per precision (and of the batched multi-RHS
    kernel) on one lattice: the autotuner's CUDA-event timings of both block
    sizes, with GB/s from the algorithmic bytes per site."""
    import torch
    from paper_1411_2087_gb300 import metrics, stag, synth
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else DIMS
    Vh = int(np.prod(dims)) // 2
    dev = torch.device("cuda", 0)
    U = synth.su3_field(dims, EPS, SEED_LINKS, device=dev)
    torch.cuda.synchronize()
    out = {"kernels_only": True, "lattice": list(dims), "compress12": bool(args.compress12)}
    link_reals = 12 if args.compress12 else 18
    want = [p for p in args.kernels_prec.split(",") if p]
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=tuple(want), compress12=args.compress12)
        for prec, rb in (("f64", 8), ("df64", 8), ("f32", 4), ("f16", 2)):
            if prec not in want:
                continue
            t = lat.autotune(prec)
            best = min(t["dslash_us"].values())
            if prec == "f16":
                byts = metrics.dslash_half_bytes_per_site() if not args.compress12 else 16 * 24 + 32
            elif prec in ("f32",):
                byts = metrics.dslash_bytes_per_site(rb, reals_per_link=link_reals)
            else:
                byts = metrics.dslash_bytes_per_site(rb)
            out[prec] = {"us": {str(k): round(v, 2) for k, v in t["dslash_us"].items()},
                         "gbs": round(byts * Vh / (best * 1e-6) / 1e9, 1),
                         "batched_us": {str(k): round(v, 2) for k, v in t["batch_us"].items()}}
    return out


def run_net_only(args):
    """The learned preconditioner's application in the solver's form
    (binary16 weights, 16-bit links, DF64 in and out) on 32^3x64, CUDA
    events over 20 applications after 3 warm-ups; the net's weights do not
    change its cost, so it is not trained here."""
    import torch
    from paper_1411_2087_gb300 import stag, synth
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else LEARNED_DIMS
    dev = torch.device("cuda", 0)
    U = synth.su3_field(dims, 0.3, 1010, device=dev)
    torch.cuda.synchronize()
    Vh = int(np.prod(dims)) // 2
    stream = torch.cuda.Stream(dev)
    with stag.Lattice(dims, stream=stream.cuda_stream) as lat:
        net = stag.Net(lat, U, channels=8, seed=1)
        del U
        fb = lat.field(stag.EVEN, "df64", synth.gaussian_colour_field(Vh, 1400))
        fz = lat.field(stag.EVEN, "df64")
        for _ in range(3):
            net.apply(fz, fb, fp16_weights=True, links16=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(20):
            net.apply(fz, fb, fp16_weights=True, links16=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / 20
        net.close()
    return {"net_only": True, "lattice": list(dims), "apply_ms": round(ms, 4),
            "form": "binary16 weights, 16-bit links, DF64 fields"}


def main():
    args = parse()
    world = dist_env()[1]
    if args.gpus != world:
        sys.exit(f"bench.py: --gpus {args.gpus} needs that many ranks (torch.distributed.run "
                 f"--nproc-per-node {args.gpus}); this launch has WORLD_SIZE={world}")
    if args.kernels_only:
        print(json.dumps(run_kernels_only(args)), flush=True)
        return
    if args.net_only:
        print(json.dumps(run_net_only(args)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_native(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
