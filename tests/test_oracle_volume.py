"""Pins of the oracle's 3-D region graphs (reading G16: 6-connected voxels,
means in storage order): a hand-worked volume, the 3-D grid graph, D = 1
against the 2-D build, stacked identical layers, and pair enumeration by
array shifts on random volumes."""
import networkx as nx
import numpy as np
import pytest

import oracle
import synth


def _edges(g):
    return {(v, int(u)) for v in range(g.V) for u in g.neighbours(v) if v < u}


def test_hand_worked_two_layers():
    """Layers [a; b] over [c; d] (one column): a-b and c-d in-layer, a-c and
    b-d across layers, and no b-c (adjacent only in the flattened rows)."""
    ids = np.array([[[10], [11]], [[12], [13]]], np.int32)
    img = np.array([[[1.0], [2.0]], [[3.0], [4.0]]])
    g = oracle.Graph.from_volume(img, ids)
    assert _edges(g) == {(0, 1), (2, 3), (0, 2), (1, 3)}
    assert [tuple(int(v) for v in K) for K in g.cliques()] == [(0, 1), (0, 2), (1, 3), (2, 3)]
    assert g.y.tolist() == [1.0, 2.0, 3.0, 4.0]


@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 1, 5), (4, 4, 2)])
def test_unique_ids_give_the_grid_graph(shape):
    D, H, W = shape
    ids = np.arange(D * H * W, dtype=np.int32).reshape(shape)
    g = oracle.Graph.from_volume(np.zeros(shape), ids)
    G = nx.grid_graph(dim=[W, H, D])  # nodes (z, r, c)
    want = {tuple(sorted((z0 * H * W + r0 * W + c0, z1 * H * W + r1 * W + c1)))
            for (z0, r0, c0), (z1, r1, c1) in G.edges()}
    assert _edges(g) == want


def test_one_layer_is_the_slice_graph():
    sp = synth.scaled(synth.workload("slice256").slices[0], 40, 52, seed=8)
    s = synth.make_slice(sp)
    a = oracle.Graph.from_image(s.image, s.region_ids)
    b = oracle.Graph.from_volume(s.image[None], s.region_ids[None])
    for k in ("y", "npix", "adj_off", "adj", "clq_off", "clq", "hood_off", "hood"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def test_stacked_identical_layers():
    """The same ids in every layer: no new edge (z-neighbours share an id),
    and each region's mean is over all of its voxels."""
    sp = synth.scaled(synth.workload("slice256").slices[0], 32, 36, seed=9)
    s = synth.make_slice(sp)
    D = 3
    rng = np.random.default_rng(4)
    vol = rng.random((D,) + s.image.shape)
    ids = np.repeat(s.region_ids[None], D, axis=0)
    g2 = oracle.Graph.from_image(s.image, s.region_ids)
    g3 = oracle.Graph.from_volume(vol, ids)
    assert np.array_equal(g2.adj_off, g3.adj_off) and np.array_equal(g2.adj, g3.adj)
    assert np.array_equal(g3.npix, D * g2.npix)
    raw = np.unique(s.region_ids)
    for v, rid in enumerate(raw):
        vals = vol[ids == rid]  # storage order
        acc = 0.0
        for x in vals:
            acc += x
        assert g3.y[v] == acc / vals.size


@pytest.mark.parametrize("seed", range(4))
def test_random_volumes_by_array_shifts(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(n) for n in rng.integers(2, 7, 3))
    ids = rng.integers(0, 12, shape).astype(np.int32) * 3
    g = oracle.Graph.from_volume(rng.random(shape), ids)
    rank = {int(r): k for k, r in enumerate(np.unique(ids))}
    want = set()
    for ax in range(3):
        a = np.moveaxis(ids, ax, 0)
        for x, y in zip(a[:-1].ravel(), a[1:].ravel()):
            if x != y:
                u, v = rank[int(x)], rank[int(y)]
                want.add((min(u, v), max(u, v)))
    assert _edges(g) == want
