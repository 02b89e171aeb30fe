"""Helpers shared by the GPU parity tests: run the oracle slice by slice and
the CUDA path on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle
import synth

# tolerances (labels equal wherever the oracle's label-energy gap
# exceeds 1e-9 relative; parameters within 1e-10 relative; hood and total
# energies within 1e-12 relative, i.e. summation order only)
GAP_TOL = 1e-9
PARAM_RTOL = 1e-10
ENERGY_RTOL = 1e-12


def dev_tensors(slices):
    import torch
    imgs = [torch.from_numpy(s.image).cuda() for s in slices]
    ids = [torch.from_numpy(s.region_ids).cuda() for s in slices]
    return imgs, ids


def gpu_arrays(g):
    names = ["VERT_OFF", "HOOD_SLICE_OFF", "Y", "NPIX", "ADJ_OFF", "ADJ", "CLQ_OFF", "CLQ", "HOOD_OFF", "HOOD",
             "REP_OFF", "REP_HOOD", "RANK_OFF", "RANK"]
    return {n: g.array(n).numpy() for n in names}


def slice_view(arrs, s):
    """The per-slice graph of slice s in the oracle's local numbering."""
    v0, v1 = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
    c0, c1 = arrs["HOOD_SLICE_OFF"][s], arrs["HOOD_SLICE_OFF"][s + 1]
    ao = arrs["ADJ_OFF"][v0:v1 + 1]
    adj = arrs["ADJ"][ao[0]:ao[-1]] - v0
    co = arrs["CLQ_OFF"][c0:c1 + 1]
    clq = arrs["CLQ"][co[0]:co[-1]] - v0
    ho = arrs["HOOD_OFF"][c0:c1 + 1]
    hood = arrs["HOOD"][ho[0]:ho[-1]] - v0
    return dict(V=v1 - v0, y=arrs["Y"][v0:v1], npix=arrs["NPIX"][v0:v1], adj_off=ao - ao[0], adj=adj,
                clq_off=co - co[0], clq=clq, hood_off=ho - ho[0], hood=hood, v0=v0, c0=c0)


def assert_graph_equal(og: "oracle.Graph", gv):
    assert og.V == gv["V"]
    assert np.array_equal(og.y, gv["y"]), "region means differ (both sum in row-major order)"
    assert np.array_equal(og.npix, gv["npix"])
    assert np.array_equal(og.adj_off, gv["adj_off"]) and np.array_equal(og.adj, gv["adj"])
    assert np.array_equal(og.clq_off, gv["clq_off"]) and np.array_equal(og.clq, gv["clq"])
    assert np.array_equal(og.hood_off, gv["hood_off"]) and np.array_equal(og.hood, gv["hood"])


def rep_lists_from_oracle(og):
    """hoods containing each vertex, ascending (from the oracle's hoods)."""
    lists = [[] for _ in range(og.V)]
    for c in range(og.C):
        for v in og.hood[og.hood_off[c]:og.hood_off[c + 1]]:
            lists[v].append(c)
    return lists


def label_gap(E_star, E_second):
    den = np.maximum(np.maximum(np.abs(E_star), np.abs(E_second)), 1e-300)
    return (E_second - E_star) / den


def assert_labels_match(x_gpu, x_orc, gap, what=""):
    bad = np.nonzero(x_gpu != x_orc)[0]
    if len(bad):
        g = gap[bad]
        assert (g <= GAP_TOL).all(), (f"{what}: {len(bad)} label mismatches, {int((g > GAP_TOL).sum())} above the "
                                      f"gap tolerance (first: v={bad[0]}, gap={g[0]:.3e})")


def rel_close(a, b, rtol, atol=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(a), np.abs(b)) + atol)


def small_specs(n=4, seed0=0, sizes=((64, 80), (96, 64), (40, 128), (72, 72), (33, 47), (128, 96))):
    base = synth.workload("slice256").slices[0]
    return [synth.scaled(base, sizes[k % len(sizes)][0], sizes[k % len(sizes)][1], seed=seed0 + k) for k in range(n)]
