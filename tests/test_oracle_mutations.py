"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source, compiles it
on the CPU, and runs the pin suite against it in a child process; the suite
must fail.  The unmodified source must pass.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stag_oracle.c")

MUTATIONS = {
    "drop_backward_naik": ("-eta * c3 * b", "0.0 * c3 * b"),
    "sign_backward_one_link": ("-eta * c1 * b", "eta * c1 * b"),
    "adjoint_without_conj": ("conj(A[b * 3 + a]) * v[b]", "A[b * 3 + a] * v[b]"),
    "transposed_forward_link": ("t += A[a * 3 + b] * v[b];", "t += A[b * 3 + a] * v[b];"),
    "naik_hop_distance": ("j = hop(L, bc, x, mu, +3, &b);", "j = hop(L, bc, x, mu, +1, &b);"),
    "eta_convention": ("for (int nu = 0; nu < mu; nu++)", "for (int nu = 0; nu <= mu; nu++)"),
    "wrap_sign_once": ("*sign = pow(bc[mu], (double)w);", "*sign = (w != 0) ? bc[mu] : 1.0;"),
    "long_link_order": ("mat_mul(T, link_at(U, V, mu, i), link_at(U, V, mu, j1));",
                        "mat_mul(T, link_at(U, V, mu, j1), link_at(U, V, mu, i));"),
    "backward_link_site": ("add_adj_mat_vec(out, -eta * c1 * b, link_at(U, V, mu, j)",
                           "add_adj_mat_vec(out, -eta * c1 * b, link_at(U, V, mu, i)"),
    "cg_beta_inverted": ("const double beta = rr_new / rr;", "const double beta = rr / rr_new;"),
    "cg_x_update": ("x[q] += alpha * p[q];", "x[q] += alpha * r[q];"),
    "mass_not_squared": ("out_even[k] = mass * mass * in_even[k]", "out_even[k] = mass * in_even[k]"),
    "covconv_backward_link_site": (
        "add_adj_mat_vec(t, b, link_at(U, V, mu, j), psi + ((long)c * V + j) * 3);",
        "add_adj_mat_vec(t, b, link_at(U, V, mu, i), psi + ((long)c * V + j) * 3);"),
    "covconv_backward_weight": ("const cplx wb = W[((2 + 2 * mu) * cout + o) * cin + c];",
                                "const cplx wb = W[((1 + 2 * mu) * cout + o) * cin + c];"),
    "covconv_forward_no_transport": (
        "add_mat_vec(t, b, link_at(U, V, mu, i), psi + ((long)c * V + j) * 3);",
        "add_adj_mat_vec(t, b, link_at(U, V, mu, i), psi + ((long)c * V + j) * 3);"),
}


def _compile(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", so, c, "-lm"],
                   check=True)
    return so


def _run_pins(so):
    env = dict(os.environ, STAG_ORACLE_SO=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_net_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_passes(source, tmp_path):
    assert _run_pins(_compile(source, str(tmp_path), "clean")) == 0


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(source, tmp_path, name):
    old, new = MUTATIONS[name]
    assert source.count(old) >= 1, f"mutation anchor not found: {old}"
    mutated = source.replace(old, new, 1)
    assert _run_pins(_compile(mutated, str(tmp_path), name)) != 0, f"pins missed: {name}"
