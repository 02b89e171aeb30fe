"""Pins of the oracle's k-neighbourhoods (Section 3.1: the clique's vertices
and every vertex within k edges of one of them): networkx shortest-path balls,
k = 1 against the pinned 1-hoods, nesting in k, and whole components."""
import networkx as nx
import numpy as np
import pytest

import oracle
import synth


def _random_graph(seed, n=None, p=None):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 30)) if n is None else n
    p = rng.uniform(0.05, 0.3) if p is None else p
    G = nx.gnp_random_graph(n, p, seed=seed)
    return G, rng.random(n)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("seed", range(6))
def test_k_hoods_are_shortest_path_balls(seed, k):
    G, y = _random_graph(seed)
    nb = [list(G.neighbors(v)) for v in range(G.number_of_nodes())]
    g1 = oracle.Graph.from_adjacency(y, nb)
    gk = oracle.Graph.from_adjacency(y, nb, hood_depth=k)
    assert np.array_equal(gk.clq, g1.clq) and np.array_equal(gk.clq_off, g1.clq_off)
    for c, K in enumerate(g1.cliques()):
        ball = set()
        for u in K:
            ball |= set(nx.single_source_shortest_path_length(G, int(u), cutoff=k))
        assert list(gk.hoods()[c]) == sorted(ball), (c, K)


def test_depth_one_is_the_one_hood_and_depths_nest():
    sp = synth.scaled(synth.workload("slice256").slices[0], 40, 56, seed=5)
    s = synth.make_slice(sp)
    g1 = oracle.Graph.from_image(s.image, s.region_ids)
    gd = oracle.Graph.from_image(s.image, s.region_ids, hood_depth=1)
    assert np.array_equal(g1.hood_off, gd.hood_off) and np.array_equal(g1.hood, gd.hood)
    prev = g1
    for k in (2, 3, 4):
        gk = oracle.Graph.from_image(s.image, s.region_ids, hood_depth=k)
        assert gk.N_el > prev.N_el
        for a, b in zip(prev.hoods(), gk.hoods()):
            assert set(a) <= set(b)
        prev = gk


def test_deep_hoods_are_components():
    """k at least the diameter: every hood is its clique's connected component."""
    G = nx.disjoint_union(nx.path_graph(5), nx.cycle_graph(4))
    nb = [list(G.neighbors(v)) for v in range(G.number_of_nodes())]
    g = oracle.Graph.from_adjacency(np.zeros(9), nb, hood_depth=8)
    for K, H in zip(g.cliques(), g.hoods()):
        comp = nx.node_connected_component(G, int(K[0]))
        assert list(H) == sorted(comp)


def test_em_runs_on_two_hoods():
    sp = synth.scaled(synth.workload("slice256").slices[0], 40, 56, seed=6)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids, hood_depth=2)
    r = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20))
    assert 1 <= r["iters"] <= 20
    for l in range(2):
        sel = r["labels"] == l
        assert r["theta"][l, 0] == sel.sum()
