"""include/stag.h is a plain C header: a C99 program compiles against it with
warnings as errors, links against libstag.so and reaches the library's
argument checks.  Only calls that return before any CUDA work are made, so
this runs on a machine without a GPU (and gives the same answers on one)."""
import os
import shutil
import subprocess

import pytest

from paper_1411_2087_gb300 import build as stag_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "stag.h"

static int expect(int got, int want, const char *what) {
    if (got != want) {
        fprintf(stderr, "%s: got %d, want %d (%s)\n", what, got, want, stag_last_error_message());
        return 1;
    }
    return 0;
}

int main(void) {
    int bad = 0;
    stag_lattice lat = NULL;
    stag_field f = NULL;
    stag_solve_info info;
    int odd_dims[4] = {4, 4, 5, 4};
    int zero_dims[4] = {4, 0, 4, 4};
    double bad_bc[4] = {1.0, 1.0, 0.5, -1.0};
    int dims[4] = {4, 4, 4, 4};
    memset(&info, 0, sizeof info);

    if (strchr(stag_version(), '.') == NULL) bad |= 1;
    if (strcmp(stag_strerror(STAG_ERR_ARG), "invalid argument") != 0) bad |= 1;
    bad |= expect(stag_lattice_create(&lat, odd_dims, NULL, 0, NULL), STAG_ERR_ARG, "odd extent");
    bad |= expect(stag_lattice_create(&lat, zero_dims, NULL, 0, NULL), STAG_ERR_ARG, "zero extent");
    bad |= expect(stag_lattice_create(&lat, dims, bad_bc, 0, NULL), STAG_ERR_ARG, "boundary phase");
    bad |= expect(stag_lattice_create(NULL, dims, NULL, 0, NULL), STAG_ERR_ARG, "null out");
    bad |= expect(lat == NULL, 1, "no handle on failure");
    bad |= expect(stag_field_create(NULL, STAG_EVEN, STAG_DF64, &f), STAG_ERR_ARG, "null lattice");
    bad |= expect(stag_cg_solve(NULL, NULL, NULL, 0.1, 1e-10, 100, &info), STAG_ERR_ARG, "null solve");
    bad |= expect(stag_dslash_oe(NULL, NULL, NULL), STAG_ERR_ARG, "null dslash");
    printf("%s\n", bad ? "FAIL" : "ok");
    return bad;
}
"""


@pytest.fixture(scope="module")
def lib_dir():
    return os.path.dirname(stag_build.build())


@pytest.mark.parametrize("std", ["c99", "c11"])
def test_header_compiles_as_c_and_links(lib_dir, tmp_path, std):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_stag.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_stag"
    cmd = [cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", lib_dir, "-lstag", f"-Wl,-rpath,{lib_dir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
