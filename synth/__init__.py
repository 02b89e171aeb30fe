"""Seeded synthetic inputs: noisy disk phantoms and jittered-grid Voronoi
oversegmentations (the input of the paper's Algorithm 2: an image, an
oversegmentation and a number of labels).

This module produces inputs only and holds none of the segmentation method.
The named workloads below describe the five synthetic workloads the tests and
the benchmark use; they stand in for the paper's porous-media and beamline
stacks (Section 4.1.1), which are not available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, replace  # noqa: F401  (replace is re-exported)

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libpmrf_synth.so")


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (plain gcc, -O2)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int64), ("width", ctypes.c_int64),
        ("n_phases", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("phase_mu", ctypes.c_double * 3), ("noise_sigma", ctypes.c_double),
        ("r_min", ctypes.c_double), ("r_max", ctypes.c_double),
        ("area_frac", ctypes.c_double),
        ("pitch_min", ctypes.c_double), ("pitch_max", ctypes.c_double),
        ("jitter", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


_lib = None


def _get():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_slice.restype = ctypes.c_double
        _lib.synth_slice.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return _lib


@dataclass(frozen=True)
class SliceSpec:
    """Generator parameters of one slice."""
    height: int
    width: int
    n_phases: int = 2
    phase_mu: tuple = (0.3, 0.7, 0.0)
    noise_sigma: float = 0.08
    r_min: float = 6.0
    r_max: float = 20.0
    area_frac: float = 0.4
    pitch_min: float = 8.0
    pitch_max: float = 8.0
    jitter: float = 3.0
    seed: int = 0


@dataclass
class Slice:
    image: np.ndarray       # f64 [H, W]
    region_ids: np.ndarray  # i32 [H, W], raw Voronoi cell ids (may have gaps)
    truth: np.ndarray       # u8 [H, W], phase map
    pitch: float


def make_slice(spec: SliceSpec) -> Slice:
    lib = _get()
    H, W = int(spec.height), int(spec.width)
    img = np.empty((H, W), dtype=np.float64)
    ids = np.empty((H, W), dtype=np.int32)
    tru = np.empty((H, W), dtype=np.uint8)
    mu = (list(spec.phase_mu) + [0.0, 0.0, 0.0])[:3]
    cfg = _Cfg(H, W, spec.n_phases, 0, (ctypes.c_double * 3)(*mu), spec.noise_sigma,
               spec.r_min, spec.r_max, spec.area_frac, spec.pitch_min, spec.pitch_max,
               spec.jitter, spec.seed & 0xFFFFFFFFFFFFFFFF)
    p = lib.synth_slice(ctypes.byref(cfg), img.ctypes.data, ids.ctypes.data, tru.ctypes.data)
    if p <= 0:
        raise ValueError(f"synth_slice failed ({p}) for {spec}")
    return Slice(img, ids, tru, p)


@dataclass
class Workload:
    """A named synthetic workload: a list of slice specs plus the EM settings
    it is run with."""
    name: str
    slices: list
    n_labels: int
    beta: float
    max_iters: int


def _spec(H, W, **kw):
    return SliceSpec(height=H, width=W, **kw)


def workload(name: str, n_slices: int | None = None, first_slice: int = 0) -> Workload:
    """The five synthetic workloads.

    slice256   : one 256x256 two-phase slice, pitch 8, sigma 0.08, r in [6,20],
                 2 labels, beta 1.0, <= 20 iterations.
    slice2048  : one 2048x2048 slice, pitch 6, sigma 0.12, r in [10,60], 2 labels,
                 beta 1.0, <= 50 iterations.
    stack512   : 512 slices of 1024x1024 (slice256's generator), per-slice seed
                 s and pitch U[4,10]; 2 labels, beta 1.0, <= 50 iterations.
    grad64     : 64 slices of 2048x2048 (slice2048's generator), per-slice seed.
    large8192  : one 8192x8192 three-phase slice (0.2/0.5/0.8, two disk families
                 each newly covering 20% of the area), r in [8,40], sigma 0.1,
                 pitch 5, 3 labels, beta 1.5, <= 100 iterations.

    `n_slices`/`first_slice` select a sub-range of a stack (for sampled runs).
    """
    if name == "slice256":
        s = [_spec(256, 256, seed=0)]
        wl = Workload(name, s, 2, 1.0, 20)
    elif name == "slice2048":
        s = [_spec(2048, 2048, noise_sigma=0.12, r_min=10.0, r_max=60.0, pitch_min=6.0, pitch_max=6.0, seed=0)]
        wl = Workload(name, s, 2, 1.0, 50)
    elif name == "stack512":
        n = 512 if n_slices is None else n_slices
        s = [_spec(1024, 1024, pitch_min=4.0, pitch_max=10.0, seed=1000 + k)
             for k in range(first_slice, first_slice + n)]
        wl = Workload(name, s, 2, 1.0, 50)
    elif name == "grad64":
        n = 64 if n_slices is None else n_slices
        s = [_spec(2048, 2048, noise_sigma=0.12, r_min=10.0, r_max=60.0, pitch_min=6.0, pitch_max=6.0,
                   seed=5000 + k) for k in range(first_slice, first_slice + n)]
        wl = Workload(name, s, 2, 1.0, 50)
    elif name == "large8192":
        s = [_spec(8192, 8192, n_phases=3, phase_mu=(0.2, 0.5, 0.8), noise_sigma=0.1, r_min=8.0, r_max=40.0,
                   area_frac=0.2, pitch_min=5.0, pitch_max=5.0, seed=7)]
        wl = Workload(name, s, 3, 1.5, 100)
    else:
        raise KeyError(name)
    return wl


def scaled(spec: SliceSpec, height: int, width: int, seed: int | None = None) -> SliceSpec:
    """Same generator at another size (and optionally another seed)."""
    return replace(spec, height=height, width=width, seed=spec.seed if seed is None else seed)


def make_stack(specs, threads: int | None = None):
    """Generate several slices in parallel (the C generator releases the GIL).
    Returns (images, region_ids, truths) as lists of 2-D arrays."""
    _get()
    threads = threads or min(len(specs), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        out = list(ex.map(make_slice, specs))
    return out
