"""bench.py's algorithmic-byte model of one MAP sweep (the numerator of the
roofline fraction), checked on CPU against counts taken independently from the
oracle's graphs of a two-slice batch, for two and three labels.

Per vertex the vertex pass reads adj_off, rep_woff and y (8 B each), reads and
writes a label byte, writes the hood-pass record, and reads 4 B per adjacency
entry and per replica mask word; the hood pass reads per hood its element
offset and the W-deep sum history and writes one sum (8 + 8 W + 8 B), per
element its member id and slot mask (8 B), and each vertex record once.  The
record holds D_min (8 B) and, for every label but the least, an excess (8 B)
and a 4-byte label mask: 20 B for two labels, 32 B for three."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402
from pmrf_testutil import small_specs  # noqa: E402


class _BatchArrays:
    """The batched graph's arrays that the byte model reads, assembled from the
    oracle's per-slice graphs (slices back to back, vertex ids global)."""

    def __init__(self, graphs):
        vo, hso, ho, ao, ro = [0], [0], [0], [0], [0]
        for og in graphs:
            base_v, base_e, base_a = vo[-1], ho[-1], ao[-1]
            # replicas of each vertex: the hoods that contain it (one mask word
            # each while its degree is at most 32)
            reps = np.bincount(og.hood, minlength=og.V)
            deg = np.diff(og.adj_off)
            assert deg.max() <= 32
            vo.append(base_v + og.V)
            hso.append(hso[-1] + og.C)
            ho.extend(base_e + og.hood_off[1:])
            ao.extend(base_a + og.adj_off[1:])
            ro.extend(ro[-1] + np.cumsum(reps))
        self._a = {k: np.asarray(v, dtype=np.int64) for k, v in
                   dict(VERT_OFF=vo, HOOD_SLICE_OFF=hso, HOOD_OFF=ho, ADJ_OFF=ao, REP_OFF=ro).items()}

    def array(self, name):
        import torch
        return torch.from_numpy(self._a[name])


@pytest.mark.parametrize("L,rec", [(2, 20), (3, 32)])
def test_sweep_bytes_counts_each_slice(L, rec):
    sl = synth.make_stack(small_specs(2, seed0=3100))
    ogs = [oracle.Graph.from_image(s.image, s.region_ids) for s in sl]
    W = 3
    vb, hb, st = bench.sweep_bytes(_BatchArrays(ogs), L, W)
    assert vb.shape == (2,) and hb.shape == (2,)
    for s, og in enumerate(ogs):
        n_adj = int(og.adj_off[-1])  # 2 E
        n_rep = sum(og.hood_off[c + 1] - og.hood_off[c] for c in range(og.C))  # one word per element
        assert vb[s] == og.V * (8 + 8 + 8 + 2 + rec) + 4 * n_adj + 4 * n_rep
        assert hb[s] == og.C * (8 + 8 * W + 8) + 8 * og.N_el + og.V * rec
    assert st["V"] == sum(og.V for og in ogs)
    assert st["C"] == sum(og.C for og in ogs)
    assert st["N_el"] == sum(og.N_el for og in ogs)
    assert st["E"] == sum(og.E for og in ogs)
    assert list(st["Es"]) == [og.N_el for og in ogs]
