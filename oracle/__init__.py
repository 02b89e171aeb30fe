"""CPU oracle for the MRF region-labelling EM path -- TEST INFRASTRUCTURE.

A plain serial C implementation (``pmrf_oracle.c``) of what DPP-PMRF's
optimisation phase computes (Lessley et al., LDAV 2018: Sections 2.1, 3.1,
3.2, Algorithms 1-2), wrapped with ctypes and numpy.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package; the CUDA library never calls it and shares no code with it.

Batches are handled here by looping over slices: every oracle routine works on
one slice (one graph), which is how the paper itself processes a stack
(Section 4.3.1: slice by slice).

Parity pins for every function live in ``tests/test_oracle_*.py``.  The
per-slice functions and the readings they encode:

* regions / edges / cliques / hoods  -- Section 2.1, 3.1, 3.2.1, 3.2.2
  (Construction of Neighborhoods); readings G1, G2.
* replicate                          -- Section 3.2.2 EM step 1 (worked arrays).
* map_sweep                          -- Section 3.2.2 EM step 2-3; G4-G7.
* params / init                      -- Section 3.2.2 EM step 4, Algorithm 2
  step 3; G3, G8.
* em, stop_rule                     -- Algorithm 2 steps 6-11, EM step 5; G9.
* pll, fit_beta                      -- the differentiable form (G10, G11).
* quality                            -- Section 4.2.1 evaluation metrics; G12.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libpmrf_oracle.so")

ORC_OK, ORC_ERR_ARG, ORC_ERR_OOM = 0, 1, 3
SCOPE_HOOD, SCOPE_FULL = 0, 1
RULE_MIN, RULE_SUM, RULE_VOTE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc -O2 (no fast-math: the C source fixes
    the order of every floating-point operation; OpenMP for the optional
    multi-core sweep only)."""
    src = os.path.join(_HERE, "pmrf_oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(ctypes.Structure):
    _fields_ = [
        ("max_id", ctypes.c_int32), ("V", ctypes.c_int32), ("n_adj", ctypes.c_int64),
        ("C", ctypes.c_int64), ("n_clq", ctypes.c_int64), ("N_el", ctypes.c_int64),
        ("rank", ctypes.POINTER(ctypes.c_int32)), ("npix", ctypes.POINTER(ctypes.c_int64)),
        ("y", ctypes.POINTER(ctypes.c_double)), ("adj_off", ctypes.POINTER(ctypes.c_int64)),
        ("adj", ctypes.POINTER(ctypes.c_int32)), ("clq_off", ctypes.POINTER(ctypes.c_int64)),
        ("clq", ctypes.POINTER(ctypes.c_int32)), ("hood_off", ctypes.POINTER(ctypes.c_int64)),
        ("hood", ctypes.POINTER(ctypes.c_int32)),
    ]


class _Config(ctypes.Structure):
    _fields_ = [("n_labels", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("conv_window", ctypes.c_int32),
                ("potts_scope", ctypes.c_int32), ("replica_rule", ctypes.c_int32), ("init_mode", ctypes.c_int32),
                ("beta", ctypes.c_double), ("conv_tol", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("init_lo", ctypes.c_double), ("init_hi", ctypes.c_double),
                ("n_threads", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        GP = ctypes.POINTER(_Graph)
        lib.orc_build_graph.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(GP)]
        lib.orc_graph_from_adjacency.argtypes = [ctypes.c_int32, _P, _P, _P, ctypes.POINTER(GP)]
        lib.orc_graph_free.argtypes = [GP]
        lib.orc_graph_free.restype = None
        lib.orc_replicate.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P]
        lib.orc_map_sweep.argtypes = [GP, ctypes.c_int32, ctypes.c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
        lib.orc_params.argtypes = [GP, ctypes.c_int32, _P, _P, _P, ctypes.c_double, _P]
        lib.orc_init_labels.argtypes = [GP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P]
        lib.orc_init_params.argtypes = [GP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P]
        lib.orc_em.argtypes = [GP, ctypes.POINTER(_Config), _P, _P, _P, _P, _P]
        lib.orc_em_ex.argtypes = [GP, ctypes.POINTER(_Config), _P, _P, _P, _P, _P, _P]
        lib.orc_stop_rule.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int64, _P, _P, _P,
                                      _P]
        lib.orc_replica_lists.argtypes = [GP, ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                          ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))]
        lib.orc_map_sweep_par.argtypes = [GP, ctypes.c_int32, ctypes.c_double, _P, _P, _P, _P, _P, ctypes.c_int32,
                                          _P, _P, _P]
        libc = ctypes.CDLL(None)
        libc.free.argtypes = [ctypes.c_void_p]
        lib._free = libc.free
        lib.orc_fit_beta.argtypes = [ctypes.POINTER(GP), ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_void_p), _P, _P, ctypes.c_double, ctypes.c_int32,
                                     ctypes.c_double, _P]
        lib.orc_pll.argtypes = [GP, ctypes.c_int32, _P, _P, _P, ctypes.c_double, _P, _P, _P, _P]
        lib.orc_label_image.argtypes = [GP, _P, ctypes.c_int64, _P, _P]
        lib.orc_quality.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P]
        lib.orc_graph_set_hood_depth.argtypes = [GP, ctypes.c_int32]
        lib.orc_build_volume.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(GP)]
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_random_init.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_double, _P, _P]
        lib.orc_map_sweep_v.argtypes = [GP, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                        _P, _P, _P, _P, _P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != ORC_OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _arr(p, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(p, shape=(n,)).astype(dtype, copy=True)


@dataclass
class EMConfig:
    """EM settings (defaults: window W = 3 and tolerance 1e-4 of Section 3.2.2;
    the iteration cap is per workload; sigma floor and threshold-init range are
    readings G8 and G3)."""
    n_labels: int = 2
    beta: float = 1.0
    max_iters: int = 20
    conv_window: int = 3
    conv_tol: float = 1e-4
    sigma_min: float = 1e-6
    init_lo: float = 0.0
    init_hi: float = 1.0
    potts_scope: int = 0   # SCOPE_HOOD (G4) or SCOPE_FULL (G13)
    replica_rule: int = 0  # RULE_MIN (G6), RULE_SUM or RULE_VOTE (G14)
    init_mode: int = 0     # 0 threshold (G3), 1 given labels, 2 given labels and parameters
    n_threads: int = 1     # > 1: the default sweep on that many threads (identical results)

    def _c(self):
        return _Config(self.n_labels, self.max_iters, self.conv_window, self.potts_scope, self.replica_rule,
                       self.init_mode, self.beta, self.conv_tol, self.sigma_min, self.init_lo, self.init_hi,
                       self.n_threads)


class Graph:
    """One slice's region graph with its cliques and hoods (oracle side)."""

    def __init__(self, handle):
        self._h = handle
        g = handle.contents
        self.V = int(g.V)
        self.max_id = int(g.max_id)
        self.C = int(g.C)
        self.N_el = int(g.N_el)
        self.rank = _arr(g.rank, self.max_id + 1, np.int32)
        self.npix = _arr(g.npix, self.V, np.int64)
        self.y = _arr(g.y, self.V, np.float64)
        self.adj_off = _arr(g.adj_off, self.V + 1, np.int64)
        self.adj = _arr(g.adj, int(g.n_adj), np.int32)
        self.clq_off = _arr(g.clq_off, self.C + 1, np.int64)
        self.clq = _arr(g.clq, int(g.n_clq), np.int32)
        self.hood_off = _arr(g.hood_off, self.C + 1, np.int64)
        self.hood = _arr(g.hood, self.N_el, np.int32)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_graph_free(h)
            self._h = None

    @property
    def E(self):
        return len(self.adj) // 2

    # -- constructors --------------------------------------------------------
    @classmethod
    def from_image(cls, image: np.ndarray, region_ids: np.ndarray, hood_depth: int = 1) -> "Graph":
        lib = _get()
        img = np.ascontiguousarray(image, dtype=np.float64)
        ids = np.ascontiguousarray(region_ids, dtype=np.int32)
        if img.shape != ids.shape or img.ndim != 2:
            raise ValueError("image and region_ids must be 2-D of the same shape")
        h = ctypes.POINTER(_Graph)()
        _check(lib.orc_build_graph(_ptr(img), _ptr(ids), img.shape[0], img.shape[1], ctypes.byref(h)), "build_graph")
        if hood_depth != 1:
            _check(lib.orc_graph_set_hood_depth(h, hood_depth), "set_hood_depth")
        return cls(h)

    @classmethod
    def from_volume(cls, volume: np.ndarray, region_ids: np.ndarray, hood_depth: int = 1) -> "Graph":
        """3-D region graph of one volume [D, H, W] (reading G16: 6-connected
        voxels, means in storage order)."""
        lib = _get()
        img = np.ascontiguousarray(volume, dtype=np.float64)
        ids = np.ascontiguousarray(region_ids, dtype=np.int32)
        if img.shape != ids.shape or img.ndim != 3:
            raise ValueError("volume and region_ids must be 3-D of the same shape")
        h = ctypes.POINTER(_Graph)()
        _check(lib.orc_build_volume(_ptr(img), _ptr(ids), *img.shape, ctypes.byref(h)), "build_volume")
        if hood_depth != 1:
            _check(lib.orc_graph_set_hood_depth(h, hood_depth), "set_hood_depth")
        return cls(h)

    @classmethod
    def from_adjacency(cls, y, neighbours, hood_depth: int = 1) -> "Graph":
        """neighbours: list of iterables (symmetric, no self loops)."""
        lib = _get()
        V = len(neighbours)
        lists = [sorted(set(int(u) for u in nb)) for nb in neighbours]
        off = np.zeros(V + 1, dtype=np.int64)
        for v, nb in enumerate(lists):
            off[v + 1] = off[v] + len(nb)
        adj = np.array([u for nb in lists for u in nb], dtype=np.int32)
        if adj.size == 0:
            adj = np.zeros(1, dtype=np.int32)
        yy = np.ascontiguousarray(y, dtype=np.float64)
        h = ctypes.POINTER(_Graph)()
        _check(lib.orc_graph_from_adjacency(V, _ptr(yy), _ptr(off), _ptr(adj), ctypes.byref(h)), "from_adjacency")
        if hood_depth != 1:
            _check(lib.orc_graph_set_hood_depth(h, hood_depth), "set_hood_depth")
        return cls(h)

    # -- method steps --------------------------------------------------------
    def neighbours(self, v):
        return self.adj[self.adj_off[v]:self.adj_off[v + 1]]

    def cliques(self):
        return [tuple(self.clq[self.clq_off[c]:self.clq_off[c + 1]]) for c in range(self.C)]

    def hoods(self):
        return [tuple(self.hood[self.hood_off[c]:self.hood_off[c + 1]]) for c in range(self.C)]

    def map_sweep(self, L, beta, x, mu, sigma, want_elements=False, want_second=False):
        """One MAP sweep; returns dict with x_new, E_star, S (per hood) and
        optionally E_el [N_el, L], Emin_el, lab_el, E_second."""
        lib = _get()
        x = np.ascontiguousarray(x, dtype=np.uint8)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        out = dict(x_new=np.zeros(self.V, np.uint8), E_star=np.zeros(self.V), S=np.zeros(self.C))
        E_el = np.zeros((self.N_el, L)) if want_elements else None
        Emin_el = np.zeros(self.N_el) if want_elements else None
        lab_el = np.zeros(self.N_el, np.uint8) if want_elements else None
        E2 = np.zeros(self.V) if want_second else None
        _check(lib.orc_map_sweep(self._h, L, beta, _ptr(x), _ptr(mu), _ptr(sigma), _ptr(out["x_new"]),
                                 _ptr(out["E_star"]), _ptr(out["S"]), _ptr(E_el), _ptr(Emin_el), _ptr(lab_el),
                                 _ptr(E2)), "map_sweep")
        if want_elements:
            out.update(E_el=E_el, Emin_el=Emin_el, lab_el=lab_el)
        if want_second:
            out["E_second"] = E2
        return out

    def map_sweep_par(self, L, beta, x, mu, sigma, n_threads):
        """The default sweep on n_threads threads (orc_map_sweep_par): x_new,
        E_star, S -- identical to map_sweep's."""
        lib = _get()
        x = np.ascontiguousarray(x, dtype=np.uint8)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        ro = ctypes.POINTER(ctypes.c_int64)()
        re = ctypes.POINTER(ctypes.c_int64)()
        _check(lib.orc_replica_lists(self._h, ctypes.byref(ro), ctypes.byref(re)), "replica_lists")
        out = dict(x_new=np.zeros(self.V, np.uint8), E_star=np.zeros(self.V), S=np.zeros(self.C))
        try:
            _check(lib.orc_map_sweep_par(self._h, L, beta, _ptr(x), _ptr(mu), _ptr(sigma),
                                         ctypes.cast(ro, ctypes.c_void_p), ctypes.cast(re, ctypes.c_void_p),
                                         n_threads, _ptr(out["x_new"]), _ptr(out["E_star"]), _ptr(out["S"])),
                   "map_sweep_par")
        finally:
            lib._free(ctypes.cast(ro, ctypes.c_void_p))
            lib._free(ctypes.cast(re, ctypes.c_void_p))
        return out

    def map_sweep_variant(self, L, beta, x, mu, sigma, scope=SCOPE_HOOD, rule=RULE_MIN):
        """One MAP sweep with a Potts scope and a replica rule (G13, G14);
        returns dict with x_new, E_star, S (per hood) and gap (per vertex:
        the relative distance of its decision from a floating-point tie)."""
        lib = _get()
        x = np.ascontiguousarray(x, dtype=np.uint8)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        out = dict(x_new=np.zeros(self.V, np.uint8), E_star=np.zeros(self.V), S=np.zeros(self.C),
                   gap=np.zeros(self.V))
        _check(lib.orc_map_sweep_v(self._h, L, beta, scope, rule, _ptr(x), _ptr(mu), _ptr(sigma), _ptr(out["x_new"]),
                                   _ptr(out["E_star"]), _ptr(out["S"]), _ptr(out["gap"])), "map_sweep_v")
        return out

    def params(self, L, x, E_star, theta_prev, sigma_min=1e-6):
        lib = _get()
        th = np.zeros((L, 4))
        x = np.ascontiguousarray(x, dtype=np.uint8)
        es = None if E_star is None else np.ascontiguousarray(E_star, dtype=np.float64)
        prev = np.ascontiguousarray(theta_prev, dtype=np.float64).reshape(L, 4)
        _check(lib.orc_params(self._h, L, _ptr(x), _ptr(es), _ptr(prev), sigma_min, _ptr(th)), "params")
        return th

    def init_labels(self, L, lo=0.0, hi=1.0):
        x = np.zeros(self.V, np.uint8)
        _check(_get().orc_init_labels(self._h, L, lo, hi, _ptr(x)), "init_labels")
        return x

    def init_params(self, L, x, lo=0.0, hi=1.0, sigma_min=1e-6):
        th = np.zeros((L, 4))
        x = np.ascontiguousarray(x, dtype=np.uint8)
        _check(_get().orc_init_params(self._h, L, lo, hi, sigma_min, _ptr(x), _ptr(th)), "init_params")
        return th

    def em(self, cfg: EMConfig, x0=None, theta0=None):
        """Full EM loop from the start cfg.init_mode selects (threshold; the
        labels x0; the labels x0 and parameters theta0 [L,4]).  Returns dict
        with labels, theta [L,4] (n, mu, sigma, U), iters, converged, T_hist
        and stop (which convergence tests held at the last iteration: bit 0 the
        MAP check over every hood, bit 1 the EM check on the total; 0 when the
        iteration cap ended the loop)."""
        lib = _get()
        x = np.zeros(self.V, np.uint8) if x0 is None else np.array(x0, dtype=np.uint8)
        th = np.zeros((cfg.n_labels, 4)) if theta0 is None else np.array(theta0, dtype=np.float64).reshape(-1, 4)
        it = ctypes.c_int32(0)
        cv = ctypes.c_int32(0)
        why = ctypes.c_int32(0)
        Th = np.zeros(cfg.max_iters)
        c = cfg._c()
        _check(lib.orc_em_ex(self._h, ctypes.byref(c), _ptr(x), _ptr(th), ctypes.byref(it), ctypes.byref(cv),
                             _ptr(Th), ctypes.byref(why)), "em")
        return dict(labels=x, theta=th, iters=int(it.value), converged=int(cv.value), T_hist=Th[:it.value].copy(),
                    stop=int(why.value))

    def pll(self, L, x, mu, sigma, beta):
        """Pseudo-log-likelihood and its gradient: (pll, g_mu[L], g_sigma[L], g_beta)."""
        lib = _get()
        x = np.ascontiguousarray(x, dtype=np.uint8)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        p = ctypes.c_double(0)
        gb = ctypes.c_double(0)
        gm = np.zeros(L)
        gs = np.zeros(L)
        _check(lib.orc_pll(self._h, L, _ptr(x), _ptr(mu), _ptr(sigma), beta, ctypes.byref(p), _ptr(gm), _ptr(gs),
                           ctypes.byref(gb)), "pll")
        return float(p.value), gm, gs, float(gb.value)

    def label_image(self, region_ids, x):
        ids = np.ascontiguousarray(region_ids, dtype=np.int32)
        out = np.zeros(ids.shape, np.uint8)
        x = np.ascontiguousarray(x, dtype=np.uint8)
        _check(_get().orc_label_image(self._h, _ptr(ids), ids.size, _ptr(x), _ptr(out)), "label_image")
        return out


def stop_rule(S_seq, T_seq, W=3, tol=1e-4):
    """The two convergence tests (Section 3.2.2; reading G9) after the last
    iteration of the given histories, as the EM loop applies them:
    S_seq [t, C] the hood sums of iterations 1..t, T_seq [t] the totals.
    Returns (hood_ok, total_ok)."""
    S = np.ascontiguousarray(S_seq, dtype=np.float64)
    T = np.ascontiguousarray(T_seq, dtype=np.float64)
    if S.ndim != 2 or T.shape != (S.shape[0],):
        raise ValueError("S_seq must be [t, C] and T_seq [t]")
    h = ctypes.c_int32(0)
    k = ctypes.c_int32(0)
    _check(_get().orc_stop_rule(S.shape[0], W, tol, S.shape[1], _ptr(S), _ptr(T), ctypes.byref(h),
                                ctypes.byref(k)), "stop_rule")
    return bool(h.value), bool(k.value)


def fit_beta(graphs, labels, mu, sigma, beta0=0.2, steps=30, lr=1.0):
    """Fit of beta by gradient ascent on the summed pseudo-log-likelihood of a
    batch (reading G11): beta <- max(0, beta + lr * sum_s dPLL_s/dbeta / sum_s
    V_s), labels and per-slice (mu, sigma) [S, L] fixed.  Returns the
    trajectory beta_0 .. beta_steps."""
    lib = _get()
    n = len(graphs)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    L = mu.shape[1]
    GP = ctypes.POINTER(_Graph)
    gs = (GP * n)(*[g._h for g in graphs])
    xs_np = [np.ascontiguousarray(x, dtype=np.uint8) for x in labels]
    xs = (ctypes.c_void_p * n)(*[x.ctypes.data for x in xs_np])
    traj = np.zeros(steps + 1)
    _check(lib.orc_fit_beta(gs, n, L, xs, _ptr(mu), _ptr(sigma), beta0, steps, lr, _ptr(traj)), "fit_beta")
    return traj


def replicate(hood_off, hood, L):
    """Literal replication of the hoods by label: (testLabel, oldIndex, hoodId,
    repHoods), each of length L * N_el."""
    lib = _get()
    hood_off = np.ascontiguousarray(hood_off, dtype=np.int64)
    hood = np.ascontiguousarray(hood, dtype=np.int32)
    C = len(hood_off) - 1
    n = L * len(hood)
    outs = [np.zeros(max(n, 1), np.int32) for _ in range(4)]
    _check(lib.orc_replicate(_ptr(hood_off), _ptr(hood), C, L, *[_ptr(o) for o in outs]), "replicate")
    return tuple(o[:n] for o in outs)


def quality(pred, truth, L):
    """Segmentation quality of one slice against its ground truth (Section
    4.2.1; reading G12): the L x L confusion counts (truth-major) and, per
    label, [precision, recall, accuracy, predicted fraction, true fraction]."""
    pred = np.ascontiguousarray(pred, dtype=np.uint8).ravel()
    truth = np.ascontiguousarray(truth, dtype=np.uint8).ravel()
    if pred.size != truth.size:
        raise ValueError("pred and truth differ in size")
    conf = np.zeros((L, L), np.int64)
    met = np.zeros((L, 5), np.float64)
    _check(_get().orc_quality(_ptr(pred), _ptr(truth), pred.size, L, _ptr(conf), _ptr(met)), "quality")
    return conf, met


def splitmix64(key, i):
    """Output of the (i+1)-th SplitMix64 step from state key."""
    return int(_get().orc_splitmix64(key, i))


def random_init(V, L, seed, slice_index, lo=0.0, hi=255.0):
    """Random start of one slice (Algorithm 2 step 3; reading G15): labels
    [V] and theta [L,4] = (0, mu, sigma, 0)."""
    x = np.zeros(max(V, 1), np.uint8)
    th = np.zeros((L, 4))
    _check(_get().orc_random_init(V, L, seed, slice_index, lo, hi, _ptr(x), _ptr(th)), "random_init")
    return x[:V], th


def segment_slices(images, region_ids, cfg: EMConfig):
    """Run the whole per-slice pipeline (graph, EM, label image) on a list of
    slices; returns a list of (graph, em_result, label_image)."""
    res = []
    for img, ids in zip(images, region_ids):
        g = Graph.from_image(img, ids)
        r = g.em(cfg)
        res.append((g, r, g.label_image(ids, r["labels"])))
    return res
