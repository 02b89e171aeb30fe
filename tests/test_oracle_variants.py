"""Pins of the oracle's sweep variants (Potts scope G13, replica rule G14):
a worked example, brute force over networkx subgraphs on small random graphs,
special cases with closed forms, and order relations between the rules."""
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "replica_rules_path4.json")
RULES = (oracle.RULE_MIN, oracle.RULE_SUM, oracle.RULE_VOTE)


def test_worked_path_example():
    f = json.load(open(GOLDEN))
    g = oracle.Graph.from_adjacency(np.array(f["y"]), f["neighbours"])
    assert [tuple(int(v) for v in h) for h in g.hoods()] == [(0, 1, 2), (0, 1, 2, 3), (1, 2, 3)]
    for c in f["cases"]:
        r = g.map_sweep_variant(f["L"], f["beta"], np.array(f["x"]), np.array(f["mu"]), np.array(f["sigma"]),
                                c["scope"], c["rule"])
        assert r["x_new"].tolist() == c["x_new"], c
        assert r["E_star"].tolist() == c["E_star"], c
        assert r["S"].tolist() == c["S"], c


def _random_graph(seed, n=None, p=None):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 16)) if n is None else n
    p = rng.uniform(0.15, 0.6) if p is None else p
    G = nx.gnp_random_graph(n, p, seed=seed)
    y = rng.random(n)
    return G, oracle.Graph.from_adjacency(y, [list(G.neighbors(v)) for v in range(n)]), y, rng


@pytest.mark.parametrize("scope", [0, 1])
@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("seed", range(5))
def test_rules_vs_brute_force(seed, L, scope):
    """Every replica's energies from networkx neighbourhoods (the hood's
    induced subgraph, or the whole graph), then each rule applied per vertex."""
    G, g, y, rng = _random_graph(100 + seed)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    mu = np.sort(rng.random(L))
    sigma = rng.uniform(0.05, 0.5, L)
    beta = float(rng.uniform(0.1, 2.0))
    reps = {v: [] for v in range(g.V)}
    S = []
    for H in g.hoods():
        sub = G if scope == 1 else G.subgraph(H)
        s = 0.0
        for v in H:
            E = [(y[v] - mu[l]) ** 2 / (2 * sigma[l] ** 2) + math.log(sigma[l])
                 + beta * sum(1 for u in sub.neighbors(v) if x[u] != l) for l in range(L)]
            lab = min(range(L), key=lambda l: (E[l], l))
            reps[v].append((E, lab))
            s += E[lab]
        S.append(s)
    for rule in RULES:
        r = g.map_sweep_variant(L, beta, x, mu, sigma, scope, rule)
        assert np.allclose(r["S"], S, rtol=1e-12, atol=0)
        for v in range(g.V):
            if r["gap"][v] < 1e-9:
                continue
            if rule == oracle.RULE_MIN:
                e, lab = min((E[lab], lab) for E, lab in reps[v])
            elif rule == oracle.RULE_SUM:
                mean = [sum(E[l] for E, _ in reps[v]) / len(reps[v]) for l in range(L)]
                lab = min(range(L), key=lambda l: (mean[l], l))
                e = mean[lab]
            else:
                votes = [sum(1 for _, b in reps[v] if b == l) for l in range(L)]
                lab = min(range(L), key=lambda l: (-votes[l], l))
                e = min(E[b] for E, b in reps[v] if b == lab)
            assert r["x_new"][v] == lab, (rule, v)
            assert abs(r["E_star"][v] - e) <= 1e-12 * max(1.0, abs(e)), (rule, v)


@pytest.mark.parametrize("seed", range(4))
def test_full_scope_rules_agree_and_dominate(seed):
    """With the full neighbourhood every replica of v carries the same
    energies: the three rules give the same labels and energies; and no hood
    sum can drop when more neighbours are counted."""
    G, g, y, rng = _random_graph(200 + seed, n=24, p=0.25)
    L = 2
    x = rng.integers(0, L, g.V).astype(np.uint8)
    mu, sg = np.array([0.3, 0.7]), np.array([0.15, 0.2])
    full = [g.map_sweep_variant(L, 0.8, x, mu, sg, oracle.SCOPE_FULL, r) for r in RULES]
    # (the mean of R equal values can round differently from the value)
    for r in full[1:]:
        assert np.array_equal(r["x_new"], full[0]["x_new"])
        assert np.allclose(r["E_star"], full[0]["E_star"], rtol=1e-14, atol=1e-15)
    assert np.array_equal(full[2]["E_star"], full[0]["E_star"])
    hood = g.map_sweep_variant(L, 0.8, x, mu, sg, oracle.SCOPE_HOOD, oracle.RULE_MIN)
    assert (full[0]["S"] >= hood["S"] - 1e-12).all()


def test_complete_graph_scopes_coincide():
    """K_n: one clique whose hood holds every neighbourhood, so both scopes give
    the same sweep under every rule."""
    n = 6
    rng = np.random.default_rng(3)
    y = rng.random(n)
    g = oracle.Graph.from_adjacency(y, [[u for u in range(n) if u != v] for v in range(n)])
    x = rng.integers(0, 2, n).astype(np.uint8)
    for rule in RULES:
        a = g.map_sweep_variant(2, 1.3, x, np.array([0.2, 0.8]), np.array([0.3, 0.3]), 0, rule)
        b = g.map_sweep_variant(2, 1.3, x, np.array([0.2, 0.8]), np.array([0.3, 0.3]), 1, rule)
        for k in ("x_new", "E_star", "S"):
            assert np.array_equal(a[k], b[k])


def test_beta_zero_every_variant_is_the_gaussian_classifier():
    G, g, y, rng = _random_graph(7, n=40, p=0.15)
    x = rng.integers(0, 2, g.V).astype(np.uint8)
    from scipy.stats import norm
    mu, sg = np.array([0.3, 0.6]), np.array([0.05, 0.3])
    want = (norm.logpdf(y, mu[1], sg[1]) > norm.logpdf(y, mu[0], sg[0])).astype(np.uint8)
    for scope in (0, 1):
        for rule in RULES:
            r = g.map_sweep_variant(2, 0.0, x, mu, sg, scope, rule)
            assert (r["x_new"] == want).all(), (scope, rule)


@pytest.mark.parametrize("seed", range(3))
def test_min_rule_energy_is_the_lowest(seed):
    """E* under MIN is the smallest replica energy: the mean (SUM) and the
    voting replicas' minimum (VOTE) cannot be below it."""
    G, g, y, rng = _random_graph(300 + seed, n=30, p=0.2)
    x = rng.integers(0, 2, g.V).astype(np.uint8)
    mu, sg = np.array([0.35, 0.65]), np.array([0.2, 0.2])
    rmin = g.map_sweep_variant(2, 1.0, x, mu, sg, 0, oracle.RULE_MIN)
    for rule in (oracle.RULE_SUM, oracle.RULE_VOTE):
        r = g.map_sweep_variant(2, 1.0, x, mu, sg, 0, rule)
        assert (r["E_star"] >= rmin["E_star"] - 1e-12).all()


@pytest.mark.parametrize("scope,rule", [(0, 1), (0, 2), (1, 0)])
def test_em_variants_keep_the_moment_invariant(scope, rule):
    """Any variant's EM result: the parameters are the label-conditional
    moments of the returned labels, and the default variant is unchanged."""
    sp = synth.scaled(synth.workload("slice256").slices[0], 48, 64, seed=21)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    cfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=25, potts_scope=scope, replica_rule=rule)
    r = g.em(cfg)
    assert 1 <= r["iters"] <= 25
    for l in range(2):
        sel = r["labels"] == l
        assert r["theta"][l, 0] == sel.sum()
        if sel.any():
            assert abs(r["theta"][l, 1] - g.y[sel].mean()) <= 1e-12
