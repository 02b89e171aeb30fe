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


# --------------------------------------------------------------------------
# the two convergence tests of Section 3.2.2 (reading G9), on hand-written
# histories and on two hand-derived EM runs

TAU = 1e-4


def test_stop_rule_total_test_alone():
    # two hoods move by +-1 every iteration in opposite directions; the total
    # does not move: only the EM (total) check holds
    S = [[0.0, 0.0], [1.0, -1.0], [0.0, 0.0], [1.0, -1.0]]
    T = [0.0, 0.0, 0.0, 0.0]
    assert oracle.stop_rule(S, T) == (False, True)


def test_stop_rule_hood_test_alone():
    # three hoods each move by 0.6 tau (below tau) at the last iteration: their
    # total moves by 1.8 tau: only the MAP (hood) check holds
    d = 0.6 * TAU
    S = [[0.0] * 3, [0.0] * 3, [0.0] * 3, [d] * 3]
    T = [0.0, 0.0, 0.0, 3 * d]
    assert oracle.stop_rule(S, T) == (True, False)


def test_stop_rule_compares_every_iteration_of_the_window():
    # constant for the last two iterations only: k = 1 and 2 agree, k = 3
    # does not, so neither check holds at t = 4; one iteration later both do
    assert oracle.stop_rule([[5.0], [7.0], [7.0], [7.0]], [10.0, 20.0, 20.0, 20.0]) == (False, False)
    assert oracle.stop_rule([[5.0], [7.0], [7.0], [7.0], [7.0]], [10.0, 20.0, 20.0, 20.0, 20.0]) == (True, True)
    # a change at k = 2 only
    assert oracle.stop_rule([[7.0], [7.0], [5.0], [7.0]], [7.0, 7.0, 5.0, 7.0]) == (False, False)
    # the window W sets how far back: with W = 1 only the last change counts
    assert oracle.stop_rule([[5.0], [7.0], [7.0]], [5.0, 7.0, 7.0], W=1) == (True, True)
    assert oracle.stop_rule([[5.0], [7.0], [7.0]], [5.0, 7.0, 7.0], W=2) == (False, False)


def test_stop_rule_needs_more_than_window_iterations():
    S = [[1.0, 2.0]] * 3
    T = [3.0] * 3
    assert oracle.stop_rule(S, T) == (False, False)  # t = W
    assert oracle.stop_rule(S + [[1.0, 2.0]], T + [3.0]) == (True, True)  # t = W + 1


def test_stop_rule_is_strict_and_absolute():
    # a change of exactly tol is not below it
    assert oracle.stop_rule([[0.0], [0.0], [0.0], [0.5]], [0.0, 0.0, 0.0, 0.5], tol=0.5) == (False, False)
    assert oracle.stop_rule([[0.0], [0.0], [0.0], [0.25]], [0.0, 0.0, 0.0, 0.25], tol=0.5) == (True, True)
    # absolute, not relative: a change of 1 on a value of 1e6 fails tau = 1e-4
    big = 1e6
    assert oracle.stop_rule([[big]] * 3 + [[big + 1.0]], [big] * 3 + [big + 1.0]) == (False, False)


def _anchored_pairs(two_components):
    """Hand-derived EM runs (adjacency given directly).  Vertices: f0 (y 0.00,
    isolated), a1 (0.55) - a2 (0.45) an edge, [b1 (0.55) - b2 (0.45) an edge],
    f1 (1.00, isolated).  Hoods: {f0}, {a1, a2}, [{b1, b2}], {f1}."""
    if two_components:
        y = [0.0, 0.55, 0.45, 0.55, 0.45, 1.0]
        nb = [[], [2], [1], [4], [3], []]
    else:
        y = [0.0, 0.55, 0.45, 1.0]
        nb = [[], [2], [1], []]
    return oracle.Graph.from_adjacency(np.array(y), nb)


def test_em_total_test_alone_ends_a_symmetric_two_cycle():
    # Start x = (f0, a1, a2, b1, b2, f1) = (0, 0, 1, 1, 0, 1): label 0 holds
    # {0, 0.55, 0.45} and label 1 {0.45, 0.55, 1}, so mu = (1/3, 2/3) and the
    # two sigmas are equal (mirror sets).  At y = 0.55 the data terms differ by
    # D_0 - D_1 = ((0.55 - 1/3)^2 - (0.55 - 2/3)^2) / (2 sigma^2) = 0.291 (and the
    # opposite at 0.45), less than beta = 1: each pair member takes the label
    # its partner holds, so both pairs swap every iteration, and the swapped
    # state has the same label sets, so theta never changes.  Hood {a1, a2}
    # alternates between D_1(0.55) + D_0(0.45) and D_0(0.55) + D_1(0.45) (apart
    # by 0.58 > tau), hood {b1, b2} does the opposite, the total is constant:
    # only the EM check can stop the loop, first at t = W + 1 = 4.
    g = _anchored_pairs(True)
    x0 = np.array([0, 0, 1, 1, 0, 1], np.uint8)
    cfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20, init_mode=1)
    r = g.em(cfg, x0=x0)
    assert r["iters"] == 4 and r["converged"] == 1 and r["stop"] == 2
    assert r["labels"].tolist() == x0.tolist()  # four swaps
    var = (1 / 9 + (0.55 - 1 / 3) ** 2 + (0.45 - 1 / 3) ** 2) / 3
    assert np.allclose(r["theta"][:, 1], [1 / 3, 2 / 3], rtol=0, atol=1e-15)
    assert np.allclose(r["theta"][:, 2], [math.sqrt(var)] * 2, rtol=1e-14, atol=0)
    assert np.ptp(r["T_hist"]) < 1e-12
    # without the total test the hoods never settle: the run ends at the cap
    no_total = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20, init_mode=1, conv_tol=0.0), x0=x0)
    assert no_total["iters"] == 20 and no_total["converged"] == 0
    # the hood sums really alternate by more than tau
    s1 = g.map_sweep(2, 1.0, x0, r["theta"][:, 1], r["theta"][:, 2])["S"]
    x1 = np.array([0, 1, 0, 0, 1, 1], np.uint8)
    s2 = g.map_sweep(2, 1.0, x1, r["theta"][:, 1], r["theta"][:, 2])["S"]
    assert abs(s1[1] - s2[1]) > 0.5 and abs(s1[2] - s2[2]) > 0.5 and abs(s1[1] - s2[2]) < 1e-12


def test_em_window_reaches_back_w_iterations():
    # One pair only: x0 = (f0, a1, a2, f1) = (0, 0, 1, 1): mu = (0.275, 0.725),
    # sigma = (0.275, 0.275).  Sweep 1: a1 (0.55) -> 1 and a2 (0.45) -> 0 on the
    # data term alone.  Then mu = (0.225, 0.775), sigma = 0.225, and at y =
    # 0.55 the data terms differ by D_0 - D_1 = (0.325^2 - 0.225^2) / (2 0.225^2)
    # = 0.543 > beta = 0.2, so the labels (0, 1, 0, 1) never change again: the
    # sums of iterations 2, 3, ... are equal and those of iteration 1 differ.
    # Both checks compare against W = 3 earlier iterations, so they first hold
    # at t = 5 (at t = 4 the window still reaches iteration 1).
    g = _anchored_pairs(False)
    x0 = np.array([0, 0, 1, 1], np.uint8)
    r = g.em(oracle.EMConfig(n_labels=2, beta=0.2, max_iters=20, init_mode=1), x0=x0)
    assert r["labels"].tolist() == [0, 1, 0, 1]
    assert r["iters"] == 5 and r["converged"] == 1 and r["stop"] == 3
    assert np.allclose(r["theta"][:, 1], [0.225, 0.775], rtol=0, atol=1e-15)
    assert np.allclose(r["theta"][:, 2], [0.225, 0.225], rtol=1e-14, atol=0)
    T = r["T_hist"]
    assert abs(T[0] - T[1]) > 0.1 and T[1] == T[2] == T[3] == T[4]
    # with a window of 1 the same run stops at t = 3 (first t > W with an
    # unchanged predecessor)
    r1 = g.em(oracle.EMConfig(n_labels=2, beta=0.2, max_iters=20, init_mode=1, conv_window=1), x0=x0)
    assert r1["iters"] == 3 and r1["stop"] == 3


# --------------------------------------------------------------------------
# beta fit (reading G11): gradient ascent on the summed pseudo-log-likelihood

def _fit_batch(seeds=(31, 32), L=2):
    gs, xs, mus, sgs = [], [], [], []
    for sd in seeds:
        g, x, th = _pll_setup(seed=sd, L=L)
        gs.append(g)
        xs.append(x)
        mus.append(th[:, 1])
        sgs.append(th[:, 2])
    return gs, xs, np.array(mus), np.array(sgs)


def _pll_total(gs, xs, mu, sg, b):
    return sum(g.pll(mu.shape[1], x, m, s, b)[0] for g, x, m, s in zip(gs, xs, mu, sg))


def test_fit_beta_first_step_is_the_scaled_derivative():
    gs, xs, mu, sg = _fit_batch()
    V = sum(g.V for g in gs)
    traj = oracle.fit_beta(gs, xs, mu, sg, beta0=0.2, steps=1, lr=1.0)
    h = 1e-6
    fd = (_pll_total(gs, xs, mu, sg, 0.2 + h) - _pll_total(gs, xs, mu, sg, 0.2 - h)) / (2 * h)
    assert traj[0] == 0.2
    assert abs(traj[1] - (0.2 + fd / V)) <= 1e-7
    traj2 = oracle.fit_beta(gs, xs, mu, sg, beta0=0.2, steps=1, lr=0.5)
    assert abs((traj2[1] - 0.2) - 0.5 * (traj[1] - 0.2)) <= 1e-15


def test_fit_beta_climbs_to_the_maximiser():
    from scipy.optimize import minimize_scalar
    gs, xs, mu, sg = _fit_batch()
    # a larger step than the default so that 300 steps reach the maximiser
    traj = oracle.fit_beta(gs, xs, mu, sg, beta0=0.2, steps=300, lr=20.0)
    f = [_pll_total(gs, xs, mu, sg, b) for b in traj[:31]]
    assert all(b2 >= b1 - 1e-9 for b1, b2 in zip(f, f[1:]))  # ascent
    best = minimize_scalar(lambda b: -_pll_total(gs, xs, mu, sg, b), bounds=(0.0, 20.0), method="bounded",
                           options=dict(xatol=1e-10))
    assert abs(traj[-1] - best.x) <= 1e-6


def test_fit_beta_normalises_by_the_batch_size():
    # a batch of two copies of one slice has twice the derivative and twice
    # the vertices: the same trajectory as the slice alone
    gs, xs, mu, sg = _fit_batch(seeds=(31,))
    one = oracle.fit_beta(gs, xs, mu, sg, steps=10)
    two = oracle.fit_beta(gs * 2, xs * 2, np.vstack([mu, mu]), np.vstack([sg, sg]), steps=10)
    assert np.allclose(one, two, rtol=1e-13, atol=0)


def test_fit_beta_stops_at_zero():
    # labels that disagree with every neighbour: the likelihood grows as beta
    # falls, so the ascent reaches the bound beta = 0 and stays there
    g = oracle.Graph.from_adjacency(np.array([0.4, 0.6, 0.4, 0.6]), [[1], [0, 2], [1, 3], [2]])
    x = np.array([0, 1, 0, 1], np.uint8)
    mu, sg = np.array([[0.45, 0.55]]), np.array([[0.2, 0.2]])
    assert g.pll(2, x, mu[0], sg[0], 0.2)[3] < 0
    traj = oracle.fit_beta([g], [x], mu, sg, beta0=0.2, steps=50, lr=1.0)
    assert traj[-1] == 0.0 and (np.diff(traj) <= 0).all()


# --------------------------------------------------------------------------
# the multi-core sweep gives the serial sweep's results exactly

@pytest.mark.parametrize("L", [2, 3])
def test_parallel_sweep_equals_serial(L):
    sp = synth.scaled(synth.workload("slice256").slices[0], 120, 100, seed=77)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    rng = np.random.default_rng(L)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    mu, sg = np.sort(rng.random(L)), rng.uniform(0.05, 0.3, L)
    a = g.map_sweep(L, 0.9, x, mu, sg)
    b = g.map_sweep_par(L, 0.9, x, mu, sg, n_threads=4)
    assert np.array_equal(a["x_new"], b["x_new"])
    assert np.array_equal(a["E_star"], b["E_star"]) and np.array_equal(a["S"], b["S"])


def test_parallel_em_equals_serial():
    sp = synth.scaled(synth.workload("slice256").slices[0], 96, 112, seed=78)
    s = synth.make_slice(sp)
    g = oracle.Graph.from_image(s.image, s.region_ids)
    a = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20))
    b = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20, n_threads=4))
    assert a["iters"] == b["iters"] and a["stop"] == b["stop"]
    assert np.array_equal(a["labels"], b["labels"]) and np.array_equal(a["theta"], b["theta"])
    assert np.array_equal(a["T_hist"], b["T_hist"])
