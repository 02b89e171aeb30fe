"""The boundary as a C program sees it: include/pmrf.h compiles as plain C11
with every warning an error, a C program links against the library and calls
the entry points that need no GPU, and the Python binding's ctypes structures
have the size and field offsets that C gives the header's structures (a
mismatch there would pass garbage through every call that takes them)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1809_05018_b300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

STRUCTS = {
    "pmrf_config": (_native.Config, ["n_labels", "max_iters", "conv_window", "init_from_labels", "potts_scope",
                                     "replica_rule", "beta", "conv_tol", "sigma_min", "init_lo", "init_hi"]),
    "pmrf_build_options": (_native.BuildOptions, ["hood_depth", "volume_depth"]),
    "pmrf_tuning": (_native.Tuning, ["hood_tile", "hood_lanes", "use_cuda_graph", "profile"]),
}

PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "pmrf.h"

#define LAYOUT(T, f) printf(#T " " #f " %zu %zu\n", offsetof(T, f), sizeof(((T*)0)->f))

int main(void) {
    pmrf_config c;
    pmrf_build_options o;
    memset(&c, 0xff, sizeof c);
    memset(&o, 0xff, sizeof o);
    if (pmrf_config_default(&c) != PMRF_OK) return 2;
    if (pmrf_build_options_default(&o) != PMRF_OK) return 3;
    if (pmrf_config_default(NULL) != PMRF_ERR_ARG) return 4;
    printf("defaults %d %d %d %g %g %g %d %d\n", c.n_labels, c.max_iters, c.conv_window, c.beta, c.conv_tol,
           c.sigma_min, o.hood_depth, o.volume_depth);
    printf("error %s\n", pmrf_last_error()[0] ? "set" : "empty");
    printf("version %s\n", pmrf_version());
    printf("size pmrf_config %zu\nsize pmrf_build_options %zu\nsize pmrf_tuning %zu\n", sizeof(pmrf_config),
           sizeof(pmrf_build_options), sizeof(pmrf_tuning));
    %LAYOUT%
    %CONSTS%
    printf("count PMRF_ARR_COUNT %d\n", (int)PMRF_ARR_COUNT);
    return 0;
}
"""


def _constants():
    """The header's named constants against the binding's copies of them."""
    c = {f"PMRF_ARR_{k}": v for k, v in _native.ARR.items()}
    c.update({name: code for code, name in _native.STATUS_NAMES.items()})
    c.update(PMRF_MAX_LABELS=_native.MAX_LABELS, PMRF_MAX_DEGREE=_native.MAX_DEGREE)
    return c


def _program():
    lines = []
    for name, (_, fields) in STRUCTS.items():
        lines += [f"LAYOUT({name}, {f});" for f in fields]
    consts = [f'printf("const {k} %lld\\n", (long long)({k}));' for k in _constants()]
    return PROGRAM.replace("%LAYOUT%", "\n    ".join(lines)).replace("%CONSTS%", "\n    ".join(consts))


@pytest.fixture(scope="module")
def c_output(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    _native.load()  # the library is built
    d = tmp_path_factory.mktemp("cabi")
    src = d / "abi.c"
    src.write_text(_program())
    exe = d / "abi"
    libdir = os.path.dirname(_native.LIB_PATH)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INCLUDE, str(src),
                    "-L", libdir, "-Wl,-rpath," + libdir, "-lpmrf", "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    return r.stdout.splitlines()


def test_c_program_calls_the_library(c_output):
    out = {ln.split(" ", 1)[0]: ln.split(" ", 1)[1] for ln in c_output if ln.split(" ", 1)[0] in
           ("defaults", "error", "version")}
    n, it, w, beta, tol, smin, depth, vdepth = out["defaults"].split()
    assert (int(n), int(it), int(w), float(beta), float(tol), float(smin)) == (2, 20, 3, 1.0, 1e-4, 1e-6)
    assert (int(depth), int(vdepth)) == (1, 1)
    assert out["error"] == "set"  # the NULL call left its message
    assert "sm_103a" in out["version"]


def test_ctypes_structures_match_the_c_layout(c_output):
    sizes = {ln.split()[1]: int(ln.split()[2]) for ln in c_output if ln.startswith("size ")}
    layout = {(ln.split()[0], ln.split()[1]): (int(ln.split()[2]), int(ln.split()[3])) for ln in c_output
              if ln.split()[0] in STRUCTS}
    for name, (cls, fields) in STRUCTS.items():
        assert ctypes.sizeof(cls) == sizes[name], name
        assert [f for f, _ in cls._fields_] == fields, name
        for f, _ in cls._fields_:
            desc = getattr(cls, f)
            assert (desc.offset, desc.size) == layout[(name, f)], (name, f)


def test_binding_constants_match_the_header(c_output):
    got = {ln.split()[1]: int(ln.split()[2]) for ln in c_output if ln.startswith("const ")}
    want = _constants()
    assert got == want
    count = [int(ln.split()[2]) for ln in c_output if ln.startswith("count PMRF_ARR_COUNT")]
    assert count == [len(_native.ARR)]  # the binding names every array the header lists
