"""B300 (sm_103a) engine for DPP-PMRF's MRF region-labelling EM path.

Thin Python binding of the C ABI in include/pmrf.h.  Every step of the path
runs in the CUDA library (lib/libpmrf.so); this module only marshals torch
tensors (device memory) and the current CUDA stream into the C calls.  The
names follow the C entry points: build_graph, em, map_sweep, params,
init_labels, label_image, pll, pll_grad, autotune.

    import paper_1809_05018_b300 as pmrf
    g = pmrf.build_graph(images, region_ids)        # CUDA f64 / i32 tensors
    out = g.em(pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=50))
    seg = g.label_image(region_ids, out["labels"])
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N
from ._native import PmrfError

__all__ = ["EMConfig", "Graph", "build_graph", "PmrfError", "lib_path", "PLL", "memory_usage", "trim_memory"]


def lib_path() -> str:
    return N.LIB_PATH


def _lib():
    return N.load()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib().pmrf_launch_count())


def memory_usage() -> tuple[int, int]:
    """(reserved, used) bytes of the library's device memory pool on the
    current device."""
    r, u = N._I64(0), N._I64(0)
    N.check(_lib().pmrf_memory_usage(ctypes.byref(r), ctypes.byref(u)), "pmrf_memory_usage")
    return int(r.value), int(u.value)


def trim_memory(keep_bytes: int = 0) -> None:
    """Return the pool's unused device memory to the driver, keeping at least
    keep_bytes reserved."""
    N.check(_lib().pmrf_trim_memory(int(keep_bytes)), "pmrf_trim_memory")


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, name, numel=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


@dataclass
class EMConfig:
    """EM settings; see pmrf_config in include/pmrf.h."""
    n_labels: int = 2
    beta: float = 1.0
    max_iters: int = 20
    conv_window: int = 3
    conv_tol: float = 1e-4
    sigma_min: float = 1e-6
    init_lo: float = 0.0
    init_hi: float = 1.0
    init_from_labels: int = 0
    potts_scope: int = 0   # 0 hood, 1 full neighbourhood
    replica_rule: int = 0  # 0 min, 1 mean energy, 2 vote

    def c(self) -> N.Config:
        return N.Config(self.n_labels, self.max_iters, self.conv_window, self.init_from_labels, self.potts_scope,
                        self.replica_rule, self.beta, self.conv_tol, self.sigma_min, self.init_lo, self.init_hi)


class Graph:
    """Device-resident region graph of a batch of slices (pmrf_graph)."""

    def __init__(self, handle, heights, widths, device):
        self._h = handle
        self.heights = list(heights)
        self.widths = list(widths)
        self.device = device
        S, V, E, C, Nel = (ctypes.c_int64() for _ in range(5))
        N.check(_lib().pmrf_graph_stats(self._h, ctypes.byref(S), ctypes.byref(V), ctypes.byref(E),
                                        ctypes.byref(C), ctypes.byref(Nel)), "pmrf_graph_stats")
        self.S, self.V, self.E, self.C, self.N_el = S.value, V.value, E.value, C.value, Nel.value
        self.n_pix = sum(h * w for h, w in zip(self.heights, self.widths))

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if self._h is not None:
            _lib().pmrf_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _handle(self):
        if self._h is None:
            raise RuntimeError("graph has been closed")
        return self._h

    # -- inspection -----------------------------------------------------------
    _DT = dict(VERT_OFF=torch.int64, HOOD_SLICE_OFF=torch.int64, Y=torch.float64, NPIX=torch.int32,
               ADJ_OFF=torch.int64, ADJ=torch.int32, CLQ_OFF=torch.int64, CLQ=torch.int32, HOOD_OFF=torch.int64,
               HOOD=torch.int32, REP_OFF=torch.int64, REP_HOOD=torch.int32, RANK_OFF=torch.int64, RANK=torch.int32)

    def array(self, name: str, device: str = "cpu") -> torch.Tensor:
        """Copy one of the graph's arrays (see pmrf_array) into a new tensor."""
        which = N.ARR[name]
        n = ctypes.c_int64()
        N.check(_lib().pmrf_graph_len(self._handle(), which, ctypes.byref(n)), "pmrf_graph_len")
        out = torch.empty(n.value, dtype=self._DT[name], device=device)
        to_host = 1 if out.device.type == "cpu" else 0
        N.check(_lib().pmrf_graph_get(self._handle(), which, _ptr(out) if n.value else None,
                                      out.numel() * out.element_size(), to_host, _stream_ptr()), "pmrf_graph_get")
        return out

    def sync_status(self):
        d = ctypes.c_int64()
        N.check(_lib().pmrf_sync_status(self._handle(), _stream_ptr(), ctypes.byref(d)), "device status")

    def tuning(self):
        t = N.Tuning()
        N.check(_lib().pmrf_get_tuning(self._handle(), ctypes.byref(t)), "pmrf_get_tuning")
        return dict(hood_tile=t.hood_tile, hood_lanes=t.hood_lanes, use_cuda_graph=t.use_cuda_graph,
                    profile=t.profile)

    def set_tuning(self, hood_tile=0, hood_lanes=0, use_cuda_graph=1, profile=0):
        t = N.Tuning(hood_tile, hood_lanes, use_cuda_graph, profile)
        N.check(_lib().pmrf_set_tuning(self._handle(), ctypes.byref(t)), "pmrf_set_tuning")

    def em_kernel_times(self, max_n=1000):
        """Per-iteration (vertex pass ms, hood pass ms) of the last profiled em()."""
        a = (ctypes.c_float * max_n)()
        b = (ctypes.c_float * max_n)()
        n = ctypes.c_int32()
        N.check(_lib().pmrf_em_kernel_times(self._handle(), max_n, a, b, ctypes.byref(n), _stream_ptr()),
                "pmrf_em_kernel_times")
        return list(a[:n.value]), list(b[:n.value])

    def autotune(self, cfg: EMConfig):
        t = N.Tuning()
        c = cfg.c()
        N.check(_lib().pmrf_autotune(self._handle(), ctypes.byref(c), _stream_ptr(), ctypes.byref(t)),
                "pmrf_autotune")
        return dict(hood_tile=t.hood_tile, hood_lanes=t.hood_lanes, use_cuda_graph=t.use_cuda_graph,
                    profile=t.profile)

    # -- the method -----------------------------------------------------------
    def init_labels(self, cfg: EMConfig) -> torch.Tensor:
        x = torch.empty(self.V, dtype=torch.uint8, device=self.device)
        c = cfg.c()
        N.check(_lib().pmrf_init_labels(self._handle(), ctypes.byref(c), _ptr(x), _stream_ptr()), "pmrf_init_labels")
        return x

    def params(self, cfg: EMConfig, labels, vertex_energy, params_prev, out=None) -> torch.Tensor:
        L = cfg.n_labels
        _need(labels, torch.uint8, "labels", self.V)
        if vertex_energy is not None:
            _need(vertex_energy, torch.float64, "vertex_energy", self.V)
        _need(params_prev, torch.float64, "params_prev", self.S * L * 4)
        out = torch.empty((self.S, L, 4), dtype=torch.float64, device=self.device) if out is None else out
        c = cfg.c()
        N.check(_lib().pmrf_params(self._handle(), ctypes.byref(c), _ptr(labels), _ptr(vertex_energy),
                                   _ptr(params_prev), _ptr(out), _stream_ptr()), "pmrf_params")
        return out

    def map_sweep(self, cfg: EMConfig, labels, params):
        L = cfg.n_labels
        _need(labels, torch.uint8, "labels", self.V)
        _need(params, torch.float64, "params", self.S * L * 4)
        x_out = torch.empty(self.V, dtype=torch.uint8, device=self.device)
        e_v = torch.empty(self.V, dtype=torch.float64, device=self.device)
        e_h = torch.empty(self.C, dtype=torch.float64, device=self.device)
        c = cfg.c()
        N.check(_lib().pmrf_map_sweep(self._handle(), ctypes.byref(c), _ptr(labels), _ptr(params), _ptr(x_out),
                                      _ptr(e_v), _ptr(e_h), _stream_ptr()), "pmrf_map_sweep")
        return x_out, e_v, e_h

    def em(self, cfg: EMConfig, labels=None, want_T=False, out=None, params=None):
        """Run the EM loop on every slice.  Returns a dict of CUDA tensors:
        labels u8 [V], params f64 [S, L, 4] (n, mu, sigma, U), iters i32 [S],
        converged i32 [S] and, with want_T, T_hist f64 [S, max_iters].
        labels: start from these labels (their moments as parameters);
        labels and params [S, L, 4]: start from both (e.g. random_init)."""
        L = cfg.n_labels
        dev = self.device
        if out is None:
            out = dict(labels=torch.empty(self.V, dtype=torch.uint8, device=dev),
                       params=torch.empty((self.S, L, 4), dtype=torch.float64, device=dev),
                       iters=torch.empty(self.S, dtype=torch.int32, device=dev),
                       converged=torch.empty(self.S, dtype=torch.int32, device=dev))
            if want_T:
                out["T_hist"] = torch.empty((self.S, cfg.max_iters), dtype=torch.float64, device=dev)
        if params is not None and labels is None:
            raise ValueError("a parameter start needs starting labels too")
        if labels is not None:
            _need(labels, torch.uint8, "labels", self.V)
            out["labels"].copy_(labels)
            cfg = EMConfig(**{**cfg.__dict__, "init_from_labels": 1})
        if params is not None:
            _need(params, torch.float64, "params", self.S * L * 4)
            out["params"].copy_(params.reshape(self.S, L, 4))
            cfg = EMConfig(**{**cfg.__dict__, "init_from_labels": 2})
        c = cfg.c()
        N.check(_lib().pmrf_em(self._handle(), ctypes.byref(c), _ptr(out["labels"]), _ptr(out["params"]),
                               _ptr(out["iters"]), _ptr(out["converged"]), _ptr(out.get("T_hist")), _stream_ptr()),
                "pmrf_em")
        return out

    def label_image(self, region_ids, labels, out=None) -> torch.Tensor:
        _need(labels, torch.uint8, "labels", self.V)
        ids = _flat_ids(region_ids)
        out = torch.empty(ids.numel(), dtype=torch.uint8, device=self.device) if out is None else out
        N.check(_lib().pmrf_label_image(self._handle(), _ptr(ids), _ptr(labels), _ptr(out), _stream_ptr()),
                "pmrf_label_image")
        return out

    def random_init(self, n_labels, seed, lo=0.0, hi=255.0):
        """The paper's random start (Algorithm 2 step 3): (labels u8 [V],
        params f64 [S, L, 4] = (0, mu, sigma, 0)) for em(init_from_labels=2)."""
        x = torch.empty(self.V, dtype=torch.uint8, device=self.device)
        th = torch.empty((self.S, n_labels, 4), dtype=torch.float64, device=self.device)
        N.check(_lib().pmrf_random_init(self._handle(), n_labels, seed, lo, hi, _ptr(x), _ptr(th), _stream_ptr()),
                "pmrf_random_init")
        return x, th

    def quality(self, n_labels, pred, truth):
        """Segmentation quality of a pixel label image against a ground truth
        (Section 4.2.1): (confusion i64 [S, L, L] truth-major, metrics f64
        [S, L, 5] = precision, recall, accuracy, predicted and true fraction)."""
        pred = pred.reshape(-1)
        truth = truth.reshape(-1)
        for t, name in ((pred, "pred"), (truth, "truth")):
            if t.dtype != torch.uint8 or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n_pix:
                raise ValueError(f"{name} must be a contiguous CUDA uint8 tensor of {self.n_pix} pixels")
        conf = torch.empty((self.S, n_labels, n_labels), dtype=torch.int64, device=self.device)
        met = torch.empty((self.S, n_labels, 5), dtype=torch.float64, device=self.device)
        N.check(_lib().pmrf_quality(self._handle(), n_labels, _ptr(pred), _ptr(truth), _ptr(conf), _ptr(met),
                                    _stream_ptr()), "pmrf_quality")
        return conf, met

    def pll(self, n_labels, labels, mu, sigma, beta) -> torch.Tensor:
        _need(labels, torch.uint8, "labels", self.V)
        _need(mu, torch.float64, "mu", self.S * n_labels)
        _need(sigma, torch.float64, "sigma", self.S * n_labels)
        out = torch.empty(self.S, dtype=torch.float64, device=self.device)
        N.check(_lib().pmrf_pll(self._handle(), n_labels, _ptr(labels), _ptr(mu), _ptr(sigma), float(beta),
                                _ptr(out), _stream_ptr()), "pmrf_pll")
        return out

    def pll_grad(self, n_labels, labels, mu, sigma, beta, gout):
        _need(labels, torch.uint8, "labels", self.V)
        _need(mu, torch.float64, "mu", self.S * n_labels)
        _need(sigma, torch.float64, "sigma", self.S * n_labels)
        _need(gout, torch.float64, "gout", self.S)
        gmu = torch.empty((self.S, n_labels), dtype=torch.float64, device=self.device)
        gsg = torch.empty((self.S, n_labels), dtype=torch.float64, device=self.device)
        gb = torch.empty(1, dtype=torch.float64, device=self.device)
        N.check(_lib().pmrf_pll_grad(self._handle(), n_labels, _ptr(labels), _ptr(mu), _ptr(sigma), float(beta),
                                     _ptr(gout), _ptr(gmu), _ptr(gsg), _ptr(gb), _stream_ptr()), "pmrf_pll_grad")
        return gmu, gsg, gb


    def pll_value_and_grad(self, n_labels, labels, mu, sigma, beta, gout):
        """pll() and pll_grad() in one pass: (pll [S], gmu, gsigma, gbeta)."""
        _need(labels, torch.uint8, "labels", self.V)
        _need(mu, torch.float64, "mu", self.S * n_labels)
        _need(sigma, torch.float64, "sigma", self.S * n_labels)
        _need(gout, torch.float64, "gout", self.S)
        pll = torch.empty(self.S, dtype=torch.float64, device=self.device)
        gmu = torch.empty((self.S, n_labels), dtype=torch.float64, device=self.device)
        gsg = torch.empty((self.S, n_labels), dtype=torch.float64, device=self.device)
        gb = torch.empty(1, dtype=torch.float64, device=self.device)
        N.check(_lib().pmrf_pll_value_and_grad(self._handle(), n_labels, _ptr(labels), _ptr(mu), _ptr(sigma),
                                               float(beta), _ptr(gout), _ptr(pll), _ptr(gmu), _ptr(gsg), _ptr(gb),
                                               _stream_ptr()), "pmrf_pll_value_and_grad")
        return pll, gmu, gsg, gb


def _flat_ids(region_ids):
    if isinstance(region_ids, (list, tuple)):
        return torch.cat([_need(r, torch.int32, "region_ids").reshape(-1) for r in region_ids])
    return _need(region_ids, torch.int32, "region_ids").reshape(-1)


def build_graph(images, region_ids, stream=None, hood_depth=1, volume_depth=1) -> Graph:
    """Build the graph of one slice (2-D tensors), a stack (3-D tensors) or a
    list of slices of different sizes (lists of 2-D tensors).  images: CUDA
    float64, region_ids: CUDA int32 of the same shapes; hood_depth: k of the
    k-neighbourhoods (Section 3.1; 1 in the paper's study); volume_depth D > 1:
    every D consecutive slices are the layers of one 3-D volume (6-connected
    voxels, region ids per volume), and the graph's slices are the volumes."""
    lib = _lib()
    if isinstance(images, (list, tuple)):
        shapes = [tuple(t.shape) for t in images]
        if [tuple(r.shape) for r in region_ids] != shapes or any(len(s) != 2 for s in shapes):
            raise ValueError("images and region_ids must be lists of matching 2-D tensors")
        img = torch.cat([_need(t, torch.float64, "image").reshape(-1) for t in images])
        ids = torch.cat([_need(t, torch.int32, "region_ids").reshape(-1) for t in region_ids])
        hs = [s[0] for s in shapes]
        ws = [s[1] for s in shapes]
    else:
        _need(images, torch.float64, "images")
        _need(region_ids, torch.int32, "region_ids")
        if images.shape != region_ids.shape or images.dim() not in (2, 3):
            raise ValueError("images and region_ids must be 2-D or 3-D tensors of the same shape")
        img, ids = images, region_ids
        if images.dim() == 2:
            hs, ws = [images.shape[0]], [images.shape[1]]
        else:
            hs, ws = [images.shape[1]] * images.shape[0], [images.shape[2]] * images.shape[0]
    S = len(hs)
    H = (ctypes.c_int64 * S)(*hs)
    W = (ctypes.c_int64 * S)(*ws)
    h = ctypes.c_void_p()
    opt = N.BuildOptions(hood_depth, volume_depth)
    N.check(lib.pmrf_build_graph_ex(_ptr(img), _ptr(ids), S, H, W, ctypes.byref(opt), _stream_ptr(stream),
                                    ctypes.byref(h)), "pmrf_build_graph_ex")
    return Graph(h, hs, ws, img.device)


from .autograd import PLL  # noqa: E402
