"""Pins of the oracle's graph construction (regions, edges, maximal cliques,
1-neighbourhoods, replication by label) against things other than itself:
the paper's worked arrays, a hand-derived example, brute force on tiny inputs
and networkx's clique enumerator."""
import itertools
import json
import os

import networkx as nx
import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# hand-derived strip example

def test_strip_regions_edges_cliques_hoods():
    fx = _load("strip_overseg.json")
    g = oracle.Graph.from_image(np.array(fx["image"]), np.array(fx["ids"], dtype=np.int32))
    assert g.V == fx["V"]
    # dyadic pixel values: the means are exact
    assert g.y.tolist() == fx["y"]
    assert g.npix.tolist() == fx["npix"]
    edges = sorted((int(v), int(u)) for v in range(g.V) for u in g.neighbours(v) if v < u)
    assert edges == [tuple(e) for e in fx["edges"]]
    assert [list(c) for c in g.cliques()] == fx["cliques"]
    assert [list(h) for h in g.hoods()] == fx["hoods"]


def test_raw_ids_compact_in_ascending_order():
    fx = _load("strip_overseg.json")
    ids = np.array(fx["ids"], dtype=np.int32)
    g = oracle.Graph.from_image(np.array(fx["image"]), ids)
    assert g.max_id == 61
    present = np.unique(ids)
    assert (g.rank[present] == np.arange(len(present))).all()
    absent = np.setdiff1d(np.arange(62), present)
    assert (g.rank[absent] == -1).all()


# --------------------------------------------------------------------------
# brute force on tiny random id maps

def _brute_edges(ids):
    H, W = ids.shape
    pairs = set()
    for r1, c1, r2, c2 in itertools.product(range(H), range(W), range(H), range(W)):
        if abs(r1 - r2) + abs(c1 - c2) == 1 and ids[r1, c1] != ids[r2, c2]:
            a, b = ids[r1, c1], ids[r2, c2]
            pairs.add((min(a, b), max(a, b)))
    return pairs


@pytest.mark.parametrize("seed", range(6))
def test_edges_and_means_vs_brute_force(seed):
    rng = np.random.default_rng(seed)
    H, W = rng.integers(3, 9), rng.integers(3, 9)
    raw = rng.choice(np.arange(0, 40, 3), size=(H, W)).astype(np.int32)
    img = rng.random((H, W))
    g = oracle.Graph.from_image(img, raw)
    present = np.unique(raw)
    assert g.V == len(present)
    # edges by brute force over all pixel pairs at Manhattan distance 1
    want = _brute_edges(raw)
    got = set()
    for v in range(g.V):
        nb = g.neighbours(v)
        assert (np.diff(nb) > 0).all()
        for u in nb:
            got.add((int(present[min(v, u)]), int(present[max(v, u)])))
    assert got == {(int(a), int(b)) for a, b in want}
    # means: row-major sequential sums, compared with an independent sum
    for k, rid in enumerate(present):
        vals = img[raw == rid]
        assert g.npix[k] == len(vals)
        assert abs(g.y[k] - vals.mean()) <= 4e-16 * max(1.0, abs(vals.mean()))


# --------------------------------------------------------------------------
# maximal cliques

def _brute_maximal_cliques(n, E):
    adj = [[False] * n for _ in range(n)]
    for a, b in E:
        adj[a][b] = adj[b][a] = True
    cl = []
    for mask in range(1, 1 << n):
        S = [i for i in range(n) if mask >> i & 1]
        if all(adj[a][b] for a, b in itertools.combinations(S, 2)):
            cl.append(S)
    sets = [frozenset(s) for s in cl]
    maximal = [s for s in sets if not any(s < t for t in sets)]
    return sorted(sorted(s) for s in maximal)


def _graph_from_edges(n, E, y=None):
    nb = [[] for _ in range(n)]
    for a, b in E:
        nb[a].append(b)
        nb[b].append(a)
    return oracle.Graph.from_adjacency(np.zeros(n) if y is None else y, nb)


@pytest.mark.parametrize("seed", range(12))
def test_cliques_vs_subset_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 13))
    p = rng.uniform(0.1, 0.8)
    E = [(a, b) for a, b in itertools.combinations(range(n), 2) if rng.random() < p]
    g = _graph_from_edges(n, E)
    assert [list(c) for c in g.cliques()] == _brute_maximal_cliques(n, E)


@pytest.mark.parametrize("seed", range(5))
def test_cliques_vs_networkx(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(20, 120))
    G = nx.gnp_random_graph(n, rng.uniform(0.03, 0.25), seed=int(seed))
    g = _graph_from_edges(n, list(G.edges()))
    want = sorted(sorted(c) for c in nx.find_cliques(G))
    assert [list(c) for c in g.cliques()] == want


def test_cliques_of_a_generated_slice_vs_networkx():
    sp = synth.scaled(synth.workload("slice256").slices[0], 96, 80, seed=3)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    G = nx.Graph()
    G.add_nodes_from(range(g.V))
    G.add_edges_from((v, int(u)) for v in range(g.V) for u in g.neighbours(v))
    assert [list(c) for c in g.cliques()] == sorted(sorted(c) for c in nx.find_cliques(G))


def test_special_graphs():
    # complete graph: one clique, one hood holding every vertex
    n = 6
    g = _graph_from_edges(n, list(itertools.combinations(range(n), 2)))
    assert g.cliques() == [tuple(range(n))]
    assert g.hoods() == [tuple(range(n))]
    # path 0-1-2-3: cliques are its edges; hood of {1,2} is everything
    g = _graph_from_edges(4, [(0, 1), (1, 2), (2, 3)])
    assert g.cliques() == [(0, 1), (1, 2), (2, 3)]
    assert g.hoods() == [(0, 1, 2), (0, 1, 2, 3), (1, 2, 3)]
    # star: centre 0 with 4 leaves: four edge cliques, each hood is the star
    g = _graph_from_edges(5, [(0, k) for k in range(1, 5)])
    assert g.cliques() == [(0, k) for k in range(1, 5)]
    assert all(h == (0, 1, 2, 3, 4) for h in g.hoods())
    # isolated vertices are cliques of size one; their hood is themselves
    g = _graph_from_edges(3, [])
    assert g.cliques() == [(0,), (1,), (2,)]
    assert g.hoods() == [(0,), (1,), (2,)]


# --------------------------------------------------------------------------
# 1-neighbourhoods via an adjacency-matrix computation

@pytest.mark.parametrize("seed", range(6))
def test_hoods_vs_adjacency_matrix(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 40))
    G = nx.gnp_random_graph(n, rng.uniform(0.05, 0.3), seed=int(seed) + 7)
    g = _graph_from_edges(n, list(G.edges()))
    A = nx.to_numpy_array(G, nodelist=range(n)) + np.eye(n)
    for K, H in zip(g.cliques(), g.hoods()):
        want = np.nonzero(A[list(K)].any(axis=0))[0].tolist()
        assert list(H) == want


# --------------------------------------------------------------------------
# replication by label: the paper's worked arrays

def test_replication_reproduces_the_paper_arrays():
    fx = _load("paper_replication.json")
    tl, oi, hid, rep = oracle.replicate(fx["hood_off"], fx["hoods"], fx["L"])
    assert tl.tolist() == fx["testLabel"]
    assert oi.tolist() == fx["oldIndex"]
    assert hid.tolist() == fx["hoodId"]
    assert rep.tolist() == fx["repHoods"]
    # gathers of the worked example: vertex label and intensity per element
    lab = {int(k): v for k, v in fx["vertex_label"].items()}
    inten = {int(k): v for k, v in fx["vertex_intensity"].items()}
    assert [lab[v] for v in rep] == fx["vertLabel"]
    assert [inten[v] for v in rep] == fx["vertMu"]
    # the printed labelMu is the mean of the element's current label (G7)
    mu = {int(k): v for k, v in fx["label_mu"].items()}
    assert [mu[lab[v]] for v in rep] == fx["labelMu"]
    assert [mu[t] for t in tl] != fx["labelMu"]


def test_label_image_maps_regions_back_to_pixels():
    fx = _load("strip_overseg.json")
    ids = np.array(fx["ids"], dtype=np.int32)
    g = oracle.Graph.from_image(np.array(fx["image"]), ids)
    x = np.array([1, 0, 1, 0, 1, 1, 0], np.uint8)
    img = g.label_image(ids, x)
    present = np.unique(ids)
    for k, rid in enumerate(present):
        assert (img[ids == rid] == x[k]).all()


def test_empty_image():
    g = oracle.Graph.from_image(np.zeros((0, 5)), np.zeros((0, 5), np.int32))
    assert g.V == 0 and g.C == 0 and g.N_el == 0
    r = g.em(oracle.EMConfig())
    assert r["iters"] == 0 and r["converged"] == 1


def test_single_region():
    g = oracle.Graph.from_image(np.full((4, 4), 0.3), np.full((4, 4), 9, np.int32))
    assert g.V == 1 and g.E == 0
    assert g.cliques() == [(0,)] and g.hoods() == [(0,)]
