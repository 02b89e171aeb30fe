#!/usr/bin/env python
"""Throughput of the B300 MRF region-labelling engine (DPP-PMRF's EM path).

One step = the whole path on one batch of synthetic slices: region graph +
maximal cliques + hoods + replica structures (pmrf_build_graph), the EM loop
(pmrf_em: MAP sweeps, replica reduction, parameter update, convergence tests),
the label image (pmrf_label_image) and one pseudo-log-likelihood value plus its
adjoint at the final labels (pmrf_pll_value_and_grad: both in one pass).

Default workload: stack512 -- 512 slices of 1024x1024, per-slice seed and
Voronoi pitch U[4,10] (10k-65k regions each), 2 labels, beta 1, <= 50 EM
iterations; the inputs (6.4 GB) are larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank processes its own
batch (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0

# DRAM traffic of the dominant kernel, from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum on a launch with every slice
# active, taken on the first 64 slices of stack512 (a capture of the full
# batch would hold far more device memory than a counter capture should),
# stored as bytes per algorithmic byte of the same launch, with the SHA-1 of
# the sources it was taken on: the opening section of em.cu (constants and
# shared structures), its hood-pass section (from the "// hood pass" header to
# the next section) and the headers em.cu includes.  bench.py reports it,
# scaled to its own average launch by the algorithmic bytes, only while those
# sources are unchanged; otherwise the field is null.
TRAFFIC_CAPTURE = {"kernel": "k_hood", "workload": "stack512", "per_alg_byte": 0.8874,
                   "sources_sha1": "294ba24c69b4e6bb35c6081cd0c602f42bbfc3e2"}
TRAFFIC_SECTION = ("paper_1809_05018_b300/csrc/em.cu", "// hood pass\n")
TRAFFIC_SOURCES = ("paper_1809_05018_b300/csrc/graph.cuh", "paper_1809_05018_b300/csrc/common.cuh")


def sources_sha1() -> str:
    h = hashlib.sha1()
    rel, header = TRAFFIC_SECTION
    with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
        text = f.read()
    first = text.find("\n// ----")
    h.update(text[:first if first >= 0 else len(text)].encode())
    a = text.index(header)
    b = text.find("\n// ----", a)
    h.update(text[a:b if b >= 0 else len(text)].encode())
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(kernel: str, workload: str, per_launch: float):
    c = TRAFFIC_CAPTURE
    if (c["per_alg_byte"] is None or kernel != c["kernel"] or workload != c["workload"]
            or c["sources_sha1"] != sources_sha1()):
        return None
    return round(c["per_alg_byte"] * per_launch, 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="stack512")
    ap.add_argument("--slices", type=int, default=None, help="slices per rank (default: the workload's)")
    ap.add_argument("--plain-sample", type=int, default=16, help="slices timed one call per slice")
    ap.add_argument("--cpu-slices", type=int, default=2, help="slices the oracle baseline runs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="run with the default hood-pass launch shape")
    ap.add_argument("--e2e-chunks", type=int, default=4, help="chunks per step in the end-to-end leg")
    # variants of the method beside the paper's form, measured on the same workload
    ap.add_argument("--hood-depth", type=int, default=1, help="k of the k-neighbourhoods")
    ap.add_argument("--potts-scope", type=int, default=0, choices=[0, 1], help="0 hood, 1 full neighbourhood")
    ap.add_argument("--replica-rule", type=int, default=0, choices=[0, 1, 2], help="0 min, 1 mean energy, 2 vote")
    ap.add_argument("--volume-depth", type=int, default=1, help="layers per 3-D volume (1: 2-D slices)")
    ap.add_argument("--slab", type=int, default=4, help="layers of a volume sharing one slice's partition")
    return ap.parse_args()


def variant(a):
    """The non-default build and sweep choices of this run (empty: the paper's form)."""
    v = {}
    if a.hood_depth != 1:
        v["hood_depth"] = a.hood_depth
    if a.potts_scope:
        v["potts_scope"] = a.potts_scope
    if a.replica_rule:
        v["replica_rule"] = a.replica_rule
    if a.volume_depth > 1:
        v.update(volume_depth=a.volume_depth, slab=a.slab)
    return v


def volumize(img, ids, D, t):
    """Stack the slices into volumes of D layers: layers of a slab of t share
    the partition and intensities of the slab's first slice, ids offset per
    slab (regions are prisms t layers tall; neighbouring slabs' partitions
    differ, so regions touch several others across the slab boundary)."""
    S = img.shape[0]
    if S % D:
        raise SystemExit(f"--volume-depth {D} must divide the {S} slices")
    off = int(ids.max()) + 1
    img2, ids2 = np.empty_like(img), np.empty_like(ids)
    for v in range(S // D):
        for z in range(D):
            src = v * D + (z // t) * t
            img2[v * D + z] = img[src]
            ids2[v * D + z] = ids[src] + (z // t) * off
    return img2, ids2


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
# clocks during the timed region

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = list(csv.reader(io.StringIO(self.out)))
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, n in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------

def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


STACKS = ("stack512", "grad64")


def shard_workload(name: str, n: int | None, rank: int):
    """Rank `rank`'s batch.  Stacks are split into consecutive runs of n slices,
    one run per rank (disjoint: every rank adds n new slices -- weak scaling);
    single-slice workloads are replicated on every rank."""
    base = synth.workload(name)
    if name not in STACKS:
        return base
    n = n or len(base.slices)
    return synth.workload(name, n_slices=n, first_slice=rank * n)


def max_over_ranks(x: float, world: int, device):
    """The largest value over all ranks (the step time of the slowest rank)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def host_inputs(wl, threads=None):
    sl = synth.make_stack(wl.slices, threads=threads or os.cpu_count())
    img = np.stack([s.image for s in sl])
    ids = np.stack([s.region_ids for s in sl])
    return sl, img, ids


def sweep_bytes(g, L, W):
    """Algorithmic bytes of one MAP sweep of every slice, split by kernel, plus
    the per-slice vectors needed to weight iterations by the slices still
    active.  A vertex record carries D_min (8 B) and, per other label, its
    excess (8 B) and a label mask (4 B): 8 + 12 (L - 1) bytes."""
    vo = g.array("VERT_OFF").numpy()
    hso = g.array("HOOD_SLICE_OFF").numpy()
    ho = g.array("HOOD_OFF").numpy()
    ao = g.array("ADJ_OFF").numpy()
    ro = g.array("REP_OFF").numpy()
    Vs = np.diff(vo)
    Cs = np.diff(hso)
    Es = ho[hso[1:]] - ho[hso[:-1]]
    Adj = ao[vo[1:]] - ao[vo[:-1]]
    Rep = ro[vo[1:]] - ro[vo[:-1]]  # replica words (== replicas when every degree <= 32)
    rec = 8 + 12 * (L - 1)
    # vertex pass: per vertex adj_off, rep_woff, y (8 each), label in + out (2), its record written;
    # per adjacency entry 4 B (neighbour id; its label byte comes with it), per replica mask word 4 B
    vb = Vs * (24 + 2 + rec) + 4 * Adj + 4 * Rep
    # hood pass: per hood its element offset (8) and the W-deep history ring (8W read + 8 write);
    # per element member id + slot mask (8); per vertex its record, read once
    hb = Cs * (8 + 8 * W + 8) + 8 * Es + Vs * rec
    return vb.astype(np.float64), hb.astype(np.float64), dict(V=int(Vs.sum()), C=int(Cs.sum()), N_el=int(Es.sum()),
                                                               E=int(Adj.sum() // 2), Es=Es)


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_1809_05018_b300 as pmrf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = shard_workload(a.workload, a.slices, rank)
    t0 = time.time()
    sl, img_np, ids_np = host_inputs(wl)
    D = a.volume_depth
    if D > 1:
        img_np, ids_np = volumize(img_np, ids_np, D, a.slab)
    gen_s = time.time() - t0
    S = img_np.shape[0]
    L, beta = wl.n_labels, wl.beta
    cfg = pmrf.EMConfig(n_labels=L, beta=beta, max_iters=wl.max_iters, potts_scope=a.potts_scope,
                        replica_rule=a.replica_rule)
    bopt = dict(hood_depth=a.hood_depth, volume_depth=D)
    img_h = torch.from_numpy(img_np).pin_memory()
    ids_h = torch.from_numpy(ids_np).pin_memory()
    img_d = img_h.cuda()
    ids_d = ids_h.cuda()
    ones = torch.ones(S, dtype=torch.float64, device="cuda")

    def step(img, ids):
        g = pmrf.build_graph(img, ids, **bopt)
        out = g.em(cfg)
        seg = g.label_image(ids, out["labels"])
        mu = out["params"][:, :, 1].contiguous()
        sg = out["params"][:, :, 2].contiguous()
        # the pseudo-log-likelihood and its adjoint in one pass
        pll, gm, gs, gb = g.pll_value_and_grad(L, out["labels"], mu, sg, beta, ones[:g.S])
        return g, out, seg, pll

    # A batch's graph is released before the next batch is built (the release
    # runs inside the step): the next build then reuses the memory, at the
    # same addresses, that the previous step just worked on; built while the
    # previous graph is still alive it took about 3.7 ms longer on stack512
    tuned = None
    gw = None
    for k in range(a.warmup):
        gw = None
        gw, _, _, _ = step(img_d, ids_d)
        if k == 0 and not a.no_autotune:
            # the hood pass's launch shape for this batch's shape, kept by the
            # library for the graphs the timed steps build
            tuned = gw.autotune(cfg)
    gw = None
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = pmrf.launch_count()
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record()
        g = None
        for _ in range(a.steps):
            g = out = seg = pll = None
            g, out, seg, pll = step(img_d, ids_d)
        e1.record()
        torch.cuda.synchronize()
    barrier()
    launches = pmrf.launch_count() - n0
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, world, "cuda")
    value = S * world / (ms / 1e3)

    # ---- the EM loop alone (the step's graph, same inputs), then once more with
    # events around every vertex and hood pass (an unrolled graph) for per-kernel times
    iters = out["iters"].cpu().numpy()
    g.em(cfg)
    torch.cuda.synchronize()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, a.steps)
    ee0.record()
    for _ in range(reps):
        o2 = g.em(cfg)
    ee1.record()
    torch.cuda.synchronize()
    em_ms = ee0.elapsed_time(ee1) / reps
    # the same loop launched kernel by kernel (no CUDA graph replay)
    g.set_tuning(use_cuda_graph=0)
    g.em(cfg)
    torch.cuda.synchronize()
    ee0.record()
    for _ in range(reps):
        g.em(cfg)
    ee1.record()
    torch.cuda.synchronize()
    em_ms_direct = ee0.elapsed_time(ee1) / reps
    g.set_tuning(profile=1)
    g.em(cfg)  # capture
    g.em(cfg)
    torch.cuda.synchronize()
    msv, msh = g.em_kernel_times()
    g.set_tuning()
    # the graph build alone (same inputs; each graph released before the next)
    ee0.record()
    for _ in range(reps):
        gb_ = pmrf.build_graph(img_d, ids_d, **bopt)
        del gb_
    ee1.record()
    torch.cuda.synchronize()
    build_ms = ee0.elapsed_time(ee1) / reps
    extra = {}
    if wl.name == "grad64":
        # the adjoint of the summed pseudo-log-likelihood (value and gradient in
        # one pass) and the 30-step beta fit through torch.autograd, at the
        # final labels
        from paper_1809_05018_b300.autograd import fit_beta
        mu = o2["params"][:, :, 1].contiguous()
        sg = o2["params"][:, :, 2].contiguous()
        g.pll_value_and_grad(L, o2["labels"], mu, sg, 0.2, ones)
        torch.cuda.synchronize()
        ee0.record()
        for _ in range(reps):
            g.pll_value_and_grad(L, o2["labels"], mu, sg, 0.2, ones)
        ee1.record()
        torch.cuda.synchronize()
        adj_ms = ee0.elapsed_time(ee1) / reps
        # one step first: torch's autograd engine starts its device threads on
        # the first backward pass (seconds), which is not part of the fit
        fit_beta(g, o2["labels"], mu, sg, beta0=0.2, steps=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        traj = fit_beta(g, o2["labels"], mu, sg, beta0=0.2, steps=30)
        torch.cuda.synchronize()
        extra.update(adjoint_ms=round(adj_ms, 3), beta_fit_ms=round((time.perf_counter() - t0) * 1e3, 3),
                     beta_fit_final=traj[-1])
    vb, hb, st = sweep_bytes(g, L, cfg.conv_window)
    # bytes per iteration t: slices still iterating at t
    tb_v, tb_h = [], []
    for t in range(1, len(msv) + 1):
        act = iters >= t
        tb_v.append(float(vb[act].sum()))
        tb_h.append(float(hb[act].sum()))
    evals = float((iters.astype(np.float64) * st["Es"]).sum() * L)
    hbm, peak_kind = load_peaks()
    bw_v = sum(tb_v) / (sum(msv) / 1e3) / 1e9 if msv else 0.0
    bw_h = sum(tb_h) / (sum(msh) / 1e3) / 1e9 if msh else 0.0
    dom = "k_hood" if sum(msh) >= sum(msv) else "k_vertex"
    ach = bw_h if dom == "k_hood" else bw_v
    per_launch = (sum(tb_h) / len(tb_h)) if dom == "k_hood" else (sum(tb_v) / len(tb_v))
    all_active = float(hb.sum()) if dom == "k_hood" else float(vb.sum())
    traffic = captured_traffic(dom, wl.name, per_launch)
    n_sw = len(msv)  # iterations of the longest slice (the loop's sweeps)

    # ---- plain: one call per slice on a sample of slices
    ps = min(a.plain_sample, S)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ones1 = ones[:1]

    def step1(k):
        if D > 1:  # one volume per call
            g1 = pmrf.build_graph(img_d[k * D:(k + 1) * D], ids_d[k * D:(k + 1) * D], **bopt)
            o1 = g1.em(cfg)
            g1.label_image(ids_d[k * D:(k + 1) * D], o1["labels"])
            mu1 = o1["params"][:, :, 1].contiguous()
            sg1 = o1["params"][:, :, 2].contiguous()
            g1.pll_value_and_grad(L, o1["labels"], mu1, sg1, beta, ones1)
            return
        g1 = pmrf.build_graph(img_d[k], ids_d[k], **bopt)
        o1 = g1.em(cfg)
        g1.label_image(ids_d[k], o1["labels"])
        mu1 = o1["params"][:, :, 1].contiguous()
        sg1 = o1["params"][:, :, 2].contiguous()
        g1.pll_value_and_grad(L, o1["labels"], mu1, sg1, beta, ones1)

    units = ps if D == 1 else max(1, ps // D)  # slices, or volumes of D slices
    for k in range(min(2, units)):  # warm the per-slice path
        step1(k)
    torch.cuda.synchronize()
    p0.record()
    for k in range(units):
        step1(k)
    p1.record()
    torch.cuda.synchronize()
    plain = units * D / (p0.elapsed_time(p1) / 1e3)

    # ---- end to end: host buffers in, label image out, copies inside the timed region.
    # Every step copies its inputs from pinned host memory and reads its label
    # image back.  A step's slices go through the public API in a few chunks, so
    # that the copy of the next chunk (own stream, second device buffer) runs
    # while this chunk computes and each read-back runs beside the next chunk:
    # the host-to-device link, the bound here, stays busy from the first copy on.
    e2e = None
    if not a.no_e2e:
        nc = max(1, a.e2e_chunks)
        if S % (nc * D):
            nc = 1
        Sc = S // nc  # input slices per chunk (whole volumes)
        npx = int(img_np[0].size)
        seg_h = torch.empty(int(img_np.size), dtype=torch.uint8).pin_memory()
        bufs = [(img_d[:Sc], ids_d[:Sc]), (torch.empty_like(img_d[:Sc]), torch.empty_like(ids_d[:Sc]))]
        cs, xs, ds = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_steps(n):
            units = [j for _ in range(n) for j in range(nc)]  # chunk index of each unit, step after step
            ready = [torch.cuda.Event(), torch.cuda.Event()]
            free = [torch.cuda.Event(), torch.cuda.Event()]

            def fetch(u):
                j, b = units[u], u % 2
                with torch.cuda.stream(xs):
                    if u >= 2:
                        xs.wait_event(free[b])  # unit u-2 has finished with that buffer
                    bufs[b][0].copy_(img_h[j * Sc:(j + 1) * Sc], non_blocking=True)
                    bufs[b][1].copy_(ids_h[j * Sc:(j + 1) * Sc], non_blocking=True)
                    ready[b].record(xs)

            fetch(0)
            for u in range(len(units)):
                j, b = units[u], u % 2
                if u + 1 < len(units):
                    fetch(u + 1)
                with torch.cuda.stream(cs):
                    cs.wait_event(ready[b])
                    _, _, sg_, _ = step(*bufs[b])
                    free[b].record(cs)
                with torch.cuda.stream(ds):
                    ds.wait_event(free[b])
                    sg_.record_stream(ds)
                    seg_h[j * Sc * npx:(j + 1) * Sc * npx].copy_(sg_, non_blocking=True)

        e2e_steps(2)
        torch.cuda.synchronize()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        x0.record(xs)
        e2e_steps(a.steps)
        for st_ in (cs, ds):
            torch.cuda.current_stream().wait_stream(st_)
        x1.record()
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(x0.elapsed_time(x1) / a.steps, world, "cuda")
        e2e = {"value": S * world / (ems / 1e3), "unit": "slices/s",
               "h2d_bytes_per_step": int(img_np.nbytes + ids_np.nbytes), "d2h_bytes_per_step": int(img_np.size),
               "pipelined": f"each step in {nc} chunks of {Sc} slices: a chunk's input copies run while the "
                            f"previous chunk computes, its label image is read back beside the next"}

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = cpu_omp = None
    if rank == 0 and world == 1 and not a.no_cpu:
        if D > 1:
            cpu = cpu_baseline_volume(img_np[:D], ids_np[:D], wl, a)
        else:
            cpu = cpu_baseline(sl[:a.cpu_slices], wl, a)
            cpu_omp = cpu_baseline(sl[:a.cpu_slices], wl, a, threads=os.cpu_count() or 1)

    if rank == 0:
        line = {
            "metric": "EM slices/s (graph build + EM loop + label image + PLL adjoint per step), batched",
            "value": round(value, 3), "unit": "slices/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "slices_per_gpu": S, "height": int(img_np.shape[1]),
                       "width": int(img_np.shape[2]), "n_labels": L, "beta": beta, "max_iters": wl.max_iters,
                       "V": st["V"], "E": st["E"], "C": st["C"], "N_el": st["N_el"],
                       "l2_policy": "inputs larger than L2 (6.4 GB per step)", "parallelism": f"replicas{world}",
                       **({"variant": variant(a)} if variant(a) else {})},
            "energy_evals_per_s": round(evals / (em_ms / 1e3), 1),
            "em_ms": round(em_ms, 3), "em_slices_per_s": round(S / (em_ms / 1e3), 3),
            "em_ms_direct_launches": round(em_ms_direct, 3), "build_ms": round(build_ms, 3),
            "us_per_iteration": round(em_ms / max(1, int(iters.max())) * 1e3, 2),
            "us_per_sweep": round((sum(msv) + sum(msh)) / max(1, n_sw) * 1e3, 2), **extra,
            "plain_slices_per_s": round(plain, 3), "plain_sample": ps,
            "iters_mean": float(iters.mean()), "iters_max": int(iters.max()),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": traffic,
                         "peak_source": peak_kind, "bytes_per_launch": per_launch,
                         "bytes_per_launch_all_active": all_active, "sources_sha1": sources_sha1(),
                         "k_vertex_GBs": round(bw_v, 1), "k_hood_GBs": round(bw_h, 1),
                         "k_vertex_ms": round(sum(msv), 3), "k_hood_ms": round(sum(msh), 3)},
            "hood_pass_tuning": None if tuned is None else {k: tuned[k] for k in ("hood_tile", "hood_lanes")},
            "cpu_baseline": cpu, "cpu_baseline_multicore": cpu_omp, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(), "gen_s": round(gen_s, 1),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(slices, wl, a=None, threads=1):
    """The oracle as it stands (serial C), full per-slice pipeline; with
    threads > 1 its MAP sweep runs on that many threads (the oracle's
    multi-core form, identical results; the rest stays serial)."""
    import oracle
    k = a.hood_depth if a else 1
    cfg = oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters,
                          potts_scope=a.potts_scope if a else 0, replica_rule=a.replica_rule if a else 0,
                          n_threads=threads)
    t0 = time.perf_counter()
    for s in slices:
        g = oracle.Graph.from_image(s.image, s.region_ids, hood_depth=k)
        r = g.em(cfg)
        g.label_image(s.region_ids, r["labels"])
        g.pll(wl.n_labels, r["labels"], r["theta"][:, 1], r["theta"][:, 2], wl.beta)
    dt = time.perf_counter() - t0
    form = "serial C oracle" if threads == 1 else f"C oracle, MAP sweep on {threads} threads (OpenMP over hoods)"
    return {"value": round(len(slices) / dt, 4), "unit": "slices/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(slices)} slices of {wl.name} ({slices[0].image.shape[0]}x{slices[0].image.shape[1]}), "
                      f"{form}: graph, cliques, hoods, EM, label image, PLL"}


def cpu_baseline_volume(img, ids, wl, a):
    """The oracle on one volume of the run (serial C, full pipeline)."""
    import oracle
    cfg = oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters, potts_scope=a.potts_scope,
                          replica_rule=a.replica_rule)
    t0 = time.perf_counter()
    g = oracle.Graph.from_volume(img, ids, hood_depth=a.hood_depth)
    r = g.em(cfg)
    g.label_image(ids.reshape(-1, ids.shape[-1]), r["labels"])
    g.pll(wl.n_labels, r["labels"], r["theta"][:, 1], r["theta"][:, 2], wl.beta)
    dt = time.perf_counter() - t0
    D = img.shape[0]
    return {"value": round(D / dt, 4), "unit": "slices/s", "cores": 1, "kind": "oracle",
            "sample": f"one volume of {D} layers of {img.shape[1]}x{img.shape[2]}, serial C oracle: graph, "
                      f"cliques, hoods, EM, label image, PLL"}


def run_reference(a):
    """The oracle, timed on the host cores on this arm's workload; each step is
    one slice of the batch (a bounded sample)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    base = synth.workload(a.workload)
    n = max(1, min(a.steps + a.warmup, len(base.slices)))
    wl = shard_workload(a.workload, n, 0)
    sl = synth.make_stack(wl.slices)
    cfg = oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)

    def one(s):
        g = oracle.Graph.from_image(s.image, s.region_ids)
        r = g.em(cfg)
        g.label_image(s.region_ids, r["labels"])
        g.pll(wl.n_labels, r["labels"], r["theta"][:, 1], r["theta"][:, 2], wl.beta)

    for k in range(a.warmup):
        one(sl[k % len(sl)])
    t0 = time.perf_counter()
    for k in range(a.steps):
        one(sl[(a.warmup + k) % len(sl)])
    dt = (time.perf_counter() - t0) / a.steps
    v = 1.0 / dt
    print(json.dumps({
        "impl": "reference", "metric": "EM slices/s (graph build + EM loop + label image + PLL adjoint per step), "
                                       "batched", "value": round(v, 4), "unit": "slices/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "slices_per_step": 1, "n_labels": wl.n_labels, "beta": wl.beta,
                   "max_iters": wl.max_iters},
        "cpu_baseline": {"value": round(v, 4), "unit": "slices/s", "cores": 1, "kind": "oracle",
                         "sample": f"one {wl.slices[0].height}x{wl.slices[0].width} slice per step"},
        "e2e": {"value": round(v, 4), "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
