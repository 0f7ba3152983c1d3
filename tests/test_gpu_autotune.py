"""The autotuner (stag_lattice_autotune_all, stag_lattice_set_tuning).

* Every Dslash candidate (block 64..512, both register variants) gives the
  same output bit for bit, in every precision and link layout; so does M
  (the two-site 16-bit form, a third candidate where it applies, is checked
  bit for bit in tests/test_gpu_pair16.py).
* The solvers meet the r11 criteria with every M-Dslash and batched
  candidate (block sizes reorder the partial sums, so not bit for bit).
* The first call times every candidate and keeps one per kind; later calls
  for the same (dims, precision, layout, device) take the cached choice
  without timing, also on a new lattice, and STAG_TUNE_FORCE times again;
  with STAG_TUNE_CACHE a second process reads the choice from the file.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from paper_1411_2087_gb300 import stag, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BLOCKS = (64, 128, 256, 512)


def fields(dims, seed=1000):
    U = synth.su3_field(dims, 0.3, seed).numpy()
    return U, oracle.long_links(dims, U)


@pytest.mark.parametrize("prec,compress", [("f64", False), ("df64", False), ("f32", False), ("f32", True),
                                           ("f16", False), ("f16", True)])
def test_every_dslash_candidate_bit_identical(prec, compress):
    dims = (6, 4, 6, 10)
    U, N = fields(dims)
    Vh = int(np.prod(dims)) // 2
    psi = synth.gaussian_colour_field(Vh, 3).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec,), compress12=compress)
        fe = lat.field(stag.EVEN, prec, psi)
        fo = lat.field(stag.ODD, prec)
        fm = lat.field(stag.EVEN, prec)
        lat.dslash(fo, fe)
        lat.apply_M(fm, fe, 0.1)
        want_d, want_m = fo.export(), fm.export()
        for block in BLOCKS:
            for regs in (1, 2):
                lat.set_tuning(prec, "dslash", block, regs)
                lat.dslash(fo, fe)
                lat.apply_M(fm, fe, 0.1)
                assert np.array_equal(fo.export(), want_d), (block, regs)
                assert np.array_equal(fm.export(), want_m), (block, regs)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_solvers_with_every_m_and_batched_candidate(prec):
    dims, mass = (4, 4, 4, 6), 0.1
    U, N = fields(dims)
    Vh = int(np.prod(dims)) // 2
    bs = [synth.gaussian_colour_field(Vh, 10 + k).numpy() for k in range(8)]

    def res(b, x):
        return np.linalg.norm(b - oracle.apply_M(dims, U, N, mass, x)) / np.linalg.norm(b)

    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=(prec, "f32"))
        fb = lat.field(stag.EVEN, prec, bs[0])
        fx = lat.field(stag.EVEN, prec)
        for block in BLOCKS:
            for regs in (1, 2):
                lat.set_tuning(prec, "M", block, regs)
                info = lat.cg(fx, fb, mass, 1e-10, 2000)
                assert info["return"] == stag.OK and res(bs[0], fx.export()) <= 1.05e-10, (block, regs)
        kmin = 2
        for p in (prec, "f32"):
            for block in (128, 256):
                for group in ((kmin, 4) if p != "f32" else (4, 8)):
                    lat.set_tuning(p, "batch", block, 0, group)
                    fbs = [lat.field(stag.EVEN, p, b) for b in bs]
                    fxs = [lat.field(stag.EVEN, p) for _ in bs]
                    st, infos = stag.cg_batched([(lat, x, b, mass) for x, b in zip(fxs, fbs)], 1e-10 if p == prec
                                                else 1e-5, 2000)
                    assert st == stag.OK, (p, block, group, infos)
                    for x, b in zip(fxs, bs):
                        assert res(b, x.export()) <= (1.05e-10 if p == prec else 2e-5), (p, block, group)
        with pytest.raises(stag.StagError):
            lat.set_tuning(prec, "dslash", 96, 1)
        with pytest.raises(stag.StagError):
            lat.set_tuning("f32", "batch", 128, 0, 3)


def test_cache_in_process_and_force():
    dims = (4, 6, 4, 10)  # a shape no other test tunes
    U, N = fields(dims)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("df64",))
        res, cached = lat.autotune_all("df64")
        assert not cached
        kinds = [r["kernel"] for r in res]
        assert kinds.count("dslash") == 8 and kinds.count("M") == 8 and kinds.count("batch") == 4
        for k in ("dslash", "M", "batch"):
            chosen = [r for r in res if r["kernel"] == k and r["chosen"]]
            assert len(chosen) == 1 and all(r["us"] > 0 for r in res if r["kernel"] == k)
        best = {r["kernel"]: r for r in res if r["chosen"]}
        res2, cached2 = lat.autotune_all("df64")
        assert cached2 and all(r["us"] == 0 for r in res2)
        assert {r["kernel"]: (r["block"], r["regs"], r["group"]) for r in res2} == \
            {k: (r["block"], r["regs"], r["group"]) for k, r in best.items()}
    with stag.Lattice(dims) as lat2:
        lat2.upload_gauge(U, N, precisions=("df64",))
        _, cached3 = lat2.autotune_all("df64")
        assert cached3
        res4, cached4 = lat2.autotune_all("df64", force=True)
        assert not cached4 and len(res4) == 20


CHILD = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, os.environ["ROOT"])
    from paper_1411_2087_gb300 import stag, synth
    dims = (6, 6, 4, 8)
    U = synth.su3_field(dims, 0.3, 7).numpy()
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, None, precisions=("f32",))
        res, cached = lat.autotune_all("f32")
    print(json.dumps({"cached": cached, "chosen": [r for r in res if r["chosen"]]}))
""")


def test_cache_file_across_processes(tmp_path):
    path = tmp_path / "tune.txt"
    env = dict(os.environ, ROOT=ROOT, STAG_TUNE_CACHE=str(path))
    outs = []
    for _ in range(2):
        p = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=300)
        assert p.returncode == 0, p.stderr
        outs.append(json.loads(p.stdout.strip().splitlines()[-1]))
    assert not outs[0]["cached"] and outs[1]["cached"]
    strip = [[(r["kernel"], r["block"], r["regs"], r["group"]) for r in o["chosen"]] for o in outs]
    assert strip[0] == strip[1]
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("stag-tune2 6 6 4 8 1 0 ")


@pytest.mark.parametrize("dims,pairs", [((4, 4, 4, 8), True), ((6, 4, 6, 10), False)])
def test_pair_candidate_only_where_it_applies(dims, pairs):
    """The two-site 16-bit form (regs 3) is a candidate on 12-real links with
    Lt a multiple of 4 (and at least 8) only."""
    U, N = fields(dims)
    with stag.Lattice(dims) as lat:
        lat.upload_gauge(U, N, precisions=("f16",), compress12=True)
        res, _ = lat.autotune_all("f16", force=True)
        for kind in ("dslash", "M"):
            regs = [r["regs"] for r in res if r["kernel"] == kind]
            assert len(regs) == (12 if pairs else 8)
            assert (3 in regs) == pairs
        assert not any(r["kernel"] == "batch" for r in res)


def test_cache_file_lines_out_of_range_are_ignored(tmp_path):
    """A cache line whose choices stag_lattice_set_tuning would refuse (a
    block size or batched group the kernels do not have) is not applied: the
    next process times the candidates again."""
    path = tmp_path / "tune.txt"
    env = dict(os.environ, ROOT=ROOT, STAG_TUNE_CACHE=str(path))
    p = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    first = json.loads(p.stdout.strip().splitlines()[-1])
    key = " ".join(path.read_text().split()[1:8])
    bad = [f"stag-tune2 {key} 1000 0 128 0 128 8",   # no 1000-thread Dslash
           f"stag-tune2 {key} 128 0 128 7 128 8",    # no register variant 7
           f"stag-tune2 {key} 128 0 128 0 128 64"]   # a group beyond the kernels' arrays
    path.write_text("\n".join(bad) + "\n")
    p = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    out = json.loads(p.stdout.strip().splitlines()[-1])
    assert not out["cached"]
    for r in out["chosen"]:
        assert r["block"] in (64, 128, 256, 512) and 0 <= r["regs"] <= 3
        if r["kernel"] == "batch":
            assert r["group"] in (4, 8)
    assert len(first["chosen"]) == len(out["chosen"])
    lines = path.read_text().splitlines()
    assert len(lines) == 4 and lines[3].startswith("stag-tune2 6 6 4 8 1 0 ")
