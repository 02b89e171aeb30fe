"""Pins of the oracle's MAP sweep, parameter update, EM loop and
pseudo-log-likelihood: hand-derived energies, brute-force Potts counts computed
with networkx, invariants, closed-form special cases and finite differences."""
import itertools
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _strip():
    with open(os.path.join(GOLD, "strip_overseg.json")) as f:
        fx = json.load(f)
    g = oracle.Graph.from_image(np.array(fx["image"]), np.array(fx["ids"], dtype=np.int32))
    return fx, g


def _D_closed(y, l):
    # closed forms of the fixture (mu = (0.25, 0.75), sigma = (0.25, 0.5))
    return 8.0 * (y - 0.25) ** 2 + math.log(0.25) if l == 0 else 2.0 * (y - 0.75) ** 2 + math.log(0.5)


def test_strip_sweep_matches_hand_derivation():
    fx, g = _strip()
    r = g.map_sweep(2, fx["beta"], fx["x"], fx["mu"], fx["sigma"], want_elements=True, want_second=True)
    k = 0
    want_S = []
    for c, h in enumerate(fx["hoods"]):
        S = 0.0
        for v in h:
            m0, m1 = fx["m"][str(c)][str(v)]
            e = [_D_closed(fx["y"][v], 0) + fx["beta"] * m0, _D_closed(fx["y"][v], 1) + fx["beta"] * m1]
            assert np.allclose(r["E_el"][k], e, rtol=0, atol=1e-14), (c, v)
            assert r["lab_el"][k] == int(np.argmin(e))
            S += min(e)
            k += 1
        want_S.append(S)
    assert np.allclose(r["S"], want_S, rtol=0, atol=1e-13)
    assert r["x_new"].tolist() == fx["x_new"]


def test_strip_init_moments_exact():
    fx, g = _strip()
    x = g.init_labels(2)
    assert x.tolist() == fx["init_labels"]
    th = g.init_params(2, x)
    assert th[:, 0].tolist() == [3.0, 4.0]
    assert abs(th[0, 1] - 5 / 24) < 1e-16 and th[1, 1] == 25 / 32
    assert abs(th[0, 2] - math.sqrt(1 / 288)) < 1e-16 and abs(th[1, 2] - math.sqrt(3 / 1024)) < 1e-16


def _random_graph(seed, n=None, p=None):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 16)) if n is None else n
    p = rng.uniform(0.15, 0.6) if p is None else p
    G = nx.gnp_random_graph(n, p, seed=seed)
    y = rng.random(n)
    nb = [list(G.neighbors(v)) for v in range(n)]
    return G, oracle.Graph.from_adjacency(y, nb), y, rng


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("seed", range(6))
def test_sweep_vs_networkx_brute_force(seed, L):
    G, g, y, rng = _random_graph(seed)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    mu = np.sort(rng.random(L))
    sigma = rng.uniform(0.05, 0.5, L)
    beta = float(rng.uniform(0.1, 2.0))
    r = g.map_sweep(L, beta, x, mu, sigma, want_elements=True, want_second=True)
    k = 0
    best = {}
    for c, H in enumerate(g.hoods()):
        sub = G.subgraph(H)
        S = 0.0
        for v in H:
            # disagreement counts over in-hood neighbours, via networkx
            m = [sum(1 for u in sub.neighbors(v) if x[u] != l) for l in range(L)]
            E = r["E_el"][k]
            # the Potts part is beta * m: differences between labels are exact multiples
            for l in range(L):
                d = (y[v] - mu[l]) ** 2 / (2 * sigma[l] ** 2) + math.log(sigma[l])
                assert abs(E[l] - (d + beta * m[l])) < 1e-12
            lab = min(range(L), key=lambda l: (E[l], l))
            assert r["lab_el"][k] == lab and r["Emin_el"][k] == E[lab]
            S += E[lab]
            cand = (E[lab], lab)
            best[v] = min(best.get(v, cand), cand)
            k += 1
        assert abs(r["S"][c] - S) <= 1e-12 * max(1, abs(S))
    for v in range(g.V):
        assert r["x_new"][v] == best[v][1] and r["E_star"][v] == best[v][0]
    # second-best distinct-label energy
    for v in range(g.V):
        others = [r["E_el"][i][l] for i in range(g.N_el) if g.hood[i] == v for l in range(L) if l != r["x_new"][v]]
        assert r["E_second"][v] == min(others)


@pytest.mark.parametrize("seed", range(4))
def test_sweep_never_raises_an_element_energy(seed):
    """Within one sweep the chosen label's energy is never above the energy of
    the element's current label (the argmin includes it)."""
    G, g, y, rng = _random_graph(40 + seed, n=30, p=0.2)
    L = 2
    x = rng.integers(0, L, g.V).astype(np.uint8)
    r = g.map_sweep(L, 0.7, x, np.array([0.3, 0.7]), np.array([0.1, 0.2]), want_elements=True)
    cur = r["E_el"][np.arange(g.N_el), x[g.hood]]
    assert (r["Emin_el"] <= cur).all()


def test_beta_zero_is_the_gaussian_classifier():
    """beta = 0: every replica sees the same energies, so the label is the
    per-vertex Gaussian maximum-likelihood class; with equal sigma it is the
    threshold at the midpoint of the two means."""
    G, g, y, rng = _random_graph(7, n=40, p=0.15)
    x = rng.integers(0, 2, g.V).astype(np.uint8)
    mu = np.array([0.3, 0.6])
    r = g.map_sweep(2, 0.0, x, mu, np.array([0.2, 0.2]))
    assert (r["x_new"] == (y >= 0.45).astype(np.uint8)).all()
    # unequal sigma: compare the two Gaussian log-densities (scipy)
    from scipy.stats import norm
    sg = np.array([0.05, 0.3])
    r = g.map_sweep(2, 0.0, x, mu, sg)
    want = (norm.logpdf(y, mu[1], sg[1]) > norm.logpdf(y, mu[0], sg[0])).astype(np.uint8)
    assert (r["x_new"] == want).all()
    # and E* is minus the log-density up to the constant 0.5 ln(2 pi)
    lp = np.maximum(norm.logpdf(y, mu[0], sg[0]), norm.logpdf(y, mu[1], sg[1]))
    assert np.allclose(r["E_star"], -lp - 0.5 * math.log(2 * math.pi), rtol=0, atol=1e-12)


def test_params_are_label_conditional_moments():
    sp = synth.scaled(synth.workload("slice256").slices[0], 64, 64, seed=11)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    L = 3
    rng = np.random.default_rng(1)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    x[x == 2] = 1  # label 2 left empty: keeps its previous mu and sigma
    Es = rng.normal(size=g.V)
    prev = np.array([[0, 0.1, 0.2, 0], [0, 0.5, 0.6, 0], [0, 0.9, 0.7, 0.0]])
    th = g.params(L, x, Es, prev, sigma_min=1e-6)
    for l in range(2):
        sel = x == l
        assert th[l, 0] == sel.sum()
        assert abs(th[l, 1] - g.y[sel].mean()) < 1e-15
        assert abs(th[l, 2] - g.y[sel].std(ddof=0)) < 1e-14
        assert abs(th[l, 3] - Es[sel].sum()) < 1e-12
    assert th[2].tolist() == [0.0, 0.9, 0.7, 0.0]
    # sigma floor on a single-member label
    x2 = np.zeros(g.V, np.uint8)
    x2[5] = 1
    th = g.params(2, x2, None, prev[:2], sigma_min=1e-6)
    assert th[1, 2] == 1e-6 and th[1, 1] == g.y[5]


# --------------------------------------------------------------------------
# EM loop: convergence rule

def _two_cluster_graph():
    # tightly clustered intensities: threshold labels are already optimal, so
    # every sweep repeats the same state
    y = np.array([0.10, 0.12, 0.11, 0.90, 0.88, 0.91, 0.13, 0.89])
    E = [(0, 1), (1, 2), (2, 6), (0, 2), (3, 4), (4, 5), (5, 7), (3, 5), (2, 3)]
    nb = [[] for _ in y]
    for a, b in E:
        nb[a].append(b)
        nb[b].append(a)
    return oracle.Graph.from_adjacency(y, nb)


def test_em_stops_after_window_when_state_repeats():
    g = _two_cluster_graph()
    r = g.em(oracle.EMConfig(n_labels=2, beta=0.5, max_iters=20))
    # S^1 = S^2 = S^3 = S^4 exactly, so the MAP test first holds at t = W + 1
    assert r["iters"] == 4 and r["converged"] == 1
    assert r["labels"].tolist() == (g.y >= 0.5).astype(int).tolist()
    assert len(set(r["T_hist"].tolist())) == 1


def test_em_cap_and_window_parameters():
    g = _two_cluster_graph()
    r = g.em(oracle.EMConfig(n_labels=2, beta=0.5, max_iters=3))
    assert r["iters"] == 3 and r["converged"] == 0
    r = g.em(oracle.EMConfig(n_labels=2, beta=0.5, max_iters=20, conv_window=5))
    assert r["iters"] == 6 and r["converged"] == 1
    # tolerance 0 can never be met: runs to the cap
    r = g.em(oracle.EMConfig(n_labels=2, beta=0.5, max_iters=9, conv_tol=0.0))
    assert r["iters"] == 9 and r["converged"] == 0


def test_em_output_is_consistent_with_its_last_sweep():
    sp = synth.scaled(synth.workload("slice256").slices[0], 96, 96, seed=5)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    cfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20)
    r = g.em(cfg)
    assert 1 <= r["iters"] <= 20
    # replay the loop step by step with the public sweep/params
    x = g.init_labels(2)
    th = g.init_params(2, x)
    T = []
    for t in range(r["iters"]):
        sw = g.map_sweep(2, cfg.beta, x, th[:, 1], th[:, 2])
        x = sw["x_new"]
        th = g.params(2, x, sw["E_star"], th)
        T.append(sw["S"].sum())
    assert (x == r["labels"]).all()
    assert np.array_equal(th, r["theta"])
    assert np.allclose(T, r["T_hist"], rtol=1e-13, atol=0)
    # theta equals the label-conditional moments of the returned labels
    for l in range(2):
        sel = r["labels"] == l
        if sel.any():
            assert abs(r["theta"][l, 1] - g.y[sel].mean()) < 1e-14


# --------------------------------------------------------------------------
# brute force over labelings of a tiny graph (quality reference, plus the
# single-site optimality the sweep guarantees)

def test_each_replica_label_is_the_exact_conditional_minimiser():
    G, g, y, rng = _random_graph(21, n=9, p=0.4)
    L, beta = 2, 0.8
    mu, sg = np.array([0.3, 0.7]), np.array([0.15, 0.15])
    for x in itertools.islice(itertools.product(range(L), repeat=g.V), 0, 512, 7):
        x = np.array(x, np.uint8)
        r = g.map_sweep(L, beta, x, mu, sg, want_elements=True)
        # the local energy of the hood with v's label changed alone is minimal at lab
        k = 0
        for c, H in enumerate(g.hoods()):
            for v in H:
                def local(l):
                    xx = x.copy()
                    xx[v] = l
                    d = (y[v] - mu[l]) ** 2 / (2 * sg[l] ** 2) + math.log(sg[l])
                    return d + beta * sum(1 for u in G.neighbors(v) if u in H and xx[u] != l)
                vals = [local(l) for l in range(L)]
                assert r["lab_el"][k] == int(np.argmin(vals))
                k += 1


# --------------------------------------------------------------------------
# pseudo-log-likelihood

def _pll_setup(seed=3, L=2):
    sp = synth.scaled(synth.workload("slice256").slices[0], 48, 48, seed=seed)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    r = g.em(oracle.EMConfig(n_labels=L, beta=1.0, max_iters=20))
    return g, r["labels"], r["theta"]


def test_pll_gradient_vs_central_differences():
    g, x, th = _pll_setup()
    mu, sg, beta = th[:, 1].copy(), th[:, 2].copy(), 0.7
    f0, gm, gs, gb = g.pll(2, x, mu, sg, beta)
    h = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (g.pll(2, x, mu + e, sg, beta)[0] - g.pll(2, x, mu - e, sg, beta)[0]) / (2 * h)
        assert abs(fd - gm[k]) <= 1e-5 * max(1, abs(gm[k]))
        fd = (g.pll(2, x, mu, sg + e, beta)[0] - g.pll(2, x, mu, sg - e, beta)[0]) / (2 * h)
        assert abs(fd - gs[k]) <= 1e-5 * max(1, abs(gs[k]))
    fd = (g.pll(2, x, mu, sg, beta + h)[0] - g.pll(2, x, mu, sg, beta - h)[0]) / (2 * h)
    assert abs(fd - gb) <= 1e-5 * max(1, abs(gb))


def test_pll_two_vertex_closed_form():
    # path 0-1, labels (0, 1), mu = (0, 1), sigma = (1, 1) (so ln sigma = 0), beta = b.
    # vertex 0 (y=0, neighbour has label 1): E(0) = 0 + b, E(1) = 0.5 + 0
    # vertex 1 (y=1, neighbour has label 0): E(0) = 0.5 + 0, E(1) = 0 + b
    b = 0.3
    g = oracle.Graph.from_adjacency(np.array([0.0, 1.0]), [[1], [0]])
    x = np.array([0, 1], np.uint8)
    f, gm, gs, gbeta = g.pll(2, x, np.array([0.0, 1.0]), np.array([1.0, 1.0]), b)
    # each vertex: -E(own) - log(exp(-b) + exp(-0.5)) with E(own) = b
    want = 2 * (-b - math.log(math.exp(-b) + math.exp(-0.5)))
    assert abs(f - want) < 1e-15
    # dPLL/dbeta = sum_v sum_l p_v(l) m_v(l) - m_v(x_v) = 2 * (p_own * 1 - 1)
    p_own = math.exp(-b) / (math.exp(-b) + math.exp(-0.5))
    assert abs(gbeta - 2 * (p_own - 1)) < 1e-15


def test_pll_is_concave_in_beta():
    g, x, th = _pll_setup(seed=4)
    bs = np.linspace(0.0, 3.0, 13)
    f = np.array([g.pll(2, x, th[:, 1], th[:, 2], b)[0] for b in bs])
    assert (np.diff(f, 2) <= 1e-9).all()
