"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/pmrf.h declares; the binding declares the same set."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1809_05018_b300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pmrf.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"PMRF_API\s+[\w\s\*]+?\b(pmrf_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pmrf_build_graph", "pmrf_em", "pmrf_map_sweep", "pmrf_params", "pmrf_pll", "pmrf_pll_grad",
              "pmrf_label_image", "pmrf_graph_destroy", "pmrf_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(pmrf_\w+)", out))
    declared = set(_declared())
    assert declared <= exported, declared - exported
    for n in declared:
        assert getattr(lib, n) is not None
    # nothing exported that the header does not declare
    assert exported <= declared, exported - declared
    # the binding declares exactly the header's entry points
    assert set(_native.exported_symbols()) == declared


def test_calls_that_need_no_gpu():
    lib = _native.load()
    c = _native.Config()
    assert lib.pmrf_config_default(ctypes.byref(c)) == 0
    assert (c.n_labels, c.max_iters, c.conv_window) == (2, 20, 3)
    assert c.conv_tol == 1e-4 and c.beta == 1.0
    assert b"sm_103a" in lib.pmrf_version()
    # argument checks fail before touching the device
    assert lib.pmrf_config_default(None) == 1
    assert b"NULL" in lib.pmrf_last_error()
    g = ctypes.c_void_p()
    H = (ctypes.c_int64 * 1)(4)
    W = (ctypes.c_int64 * 1)(4)
    assert lib.pmrf_build_graph(None, None, 0, H, W, None, ctypes.byref(g)) == 1
    assert lib.pmrf_build_graph(None, None, 1, None, W, None, ctypes.byref(g)) == 1
    assert lib.pmrf_graph_stats(None, None, None, None, None, None) == 1
    assert lib.pmrf_em(None, None, None, None, None, None, None, None) == 1
    assert lib.pmrf_graph_destroy(None) == 0


def test_library_is_built_for_sm_103a():
    # the fatbinary carries sm_103a code: cuobjdump-free check through the
    # ELF note nvcc writes (the arch list string) is not portable, so check
    # the build flags the package uses instead
    from paper_1809_05018_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
