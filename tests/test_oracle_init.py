"""Pins of the oracle's starts (Algorithm 2 step 3): the SplitMix64 draws
against the generator's published outputs, the random start's ranges and
frequencies, and the EM start modes against one another."""
import numpy as np
import pytest

import oracle
import synth


def test_splitmix64_published_outputs():
    """First outputs of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014; the
    reference splitmix64.c) from states 0 and 1234567."""
    assert [oracle.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                           0x06C45D188009454F]
    assert [oracle.splitmix64(1234567, i) for i in range(3)] == [0x599ED017FB08FC85, 0x2C73F08458540FA5,
                                                                 0x883EBCE5A3F27C77]


@pytest.mark.parametrize("L", [2, 3, 5])
def test_random_labels_are_uniform(L):
    V = 60000
    x, th = oracle.random_init(V, L, seed=2018, slice_index=7)
    assert x.max() < L
    n = np.bincount(x, minlength=L)
    p = 1.0 / L
    assert np.all(np.abs(n - V * p) < 5 * np.sqrt(V * p * (1 - p)))
    # consecutive labels are not correlated
    same = (x[1:] == x[:-1]).mean()
    assert abs(same - p) < 5 * np.sqrt(p * (1 - p) / (V - 1))


def test_random_parameters_in_range_and_uniform():
    L = 4
    mus, sgs = [], []
    for s in range(500):
        _, th = oracle.random_init(3, L, seed=11, slice_index=s, lo=0.0, hi=255.0)
        assert (th[:, 0] == 0).all() and (th[:, 3] == 0).all()
        mus.append(th[:, 1])
        sgs.append(th[:, 2])
    mus, sgs = np.concatenate(mus), np.concatenate(sgs)
    for a in (mus, sgs):
        assert a.min() >= 0.0 and a.max() < 255.0
        assert abs(a.mean() - 127.5) < 5 * 255 / np.sqrt(12 * a.size)
    # slices and seeds give different draws; equal arguments equal draws
    a = oracle.random_init(50, 2, 5, 0)
    b = oracle.random_init(50, 2, 5, 1)
    c = oracle.random_init(50, 2, 6, 0)
    d = oracle.random_init(50, 2, 5, 0)
    assert not np.array_equal(a[0], b[0]) and not np.array_equal(a[0], c[0])
    assert np.array_equal(a[0], d[0]) and np.array_equal(a[1], d[1])


def _slice_graph():
    sp = synth.scaled(synth.workload("slice256").slices[0], 48, 64, seed=31)
    s = synth.make_slice(sp)
    return oracle.Graph.from_image(s.image, s.region_ids)


def test_em_start_modes_agree():
    """Given labels equal to the threshold start reproduce the threshold run;
    given parameters equal to those labels' moments reproduce it too."""
    g = _slice_graph()
    base = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=25)
    r0 = g.em(base)
    x0 = g.init_labels(2)
    th0 = g.init_params(2, x0)
    r1 = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=25, init_mode=1), x0=x0)
    r2 = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=25, init_mode=2), x0=x0, theta0=th0)
    for r in (r1, r2):
        assert r["iters"] == r0["iters"] and np.array_equal(r["labels"], r0["labels"])
        assert np.array_equal(r["theta"], r0["theta"]) and np.array_equal(r["T_hist"], r0["T_hist"])


def test_em_from_random_start():
    """The paper's random start: the run ends, its parameters are the moments
    of its labels, and a sigma drawn below the floor is raised to it."""
    g = _slice_graph()
    x0, th0 = oracle.random_init(g.V, 2, seed=99, slice_index=0, lo=0.0, hi=1.0)
    th0[1, 2] = 1e-9
    cfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=40, init_mode=2)
    r = g.em(cfg, x0=x0, theta0=th0)
    assert 1 <= r["iters"] <= 40
    for l in range(2):
        sel = r["labels"] == l
        assert r["theta"][l, 0] == sel.sum()
        if sel.any():
            assert abs(r["theta"][l, 1] - g.y[sel].mean()) <= 1e-12
    # one iteration from the floored start equals a sweep at sigma_min
    r1 = g.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=1, init_mode=2), x0=x0, theta0=th0)
    sw = g.map_sweep(2, 1.0, x0, th0[:, 1], np.maximum(th0[:, 2], 1e-6))
    assert np.array_equal(r1["labels"], sw["x_new"])


def test_bad_start_labels_rejected():
    g = _slice_graph()
    x0 = np.full(g.V, 2, np.uint8)
    with pytest.raises(RuntimeError):
        g.em(oracle.EMConfig(n_labels=2, init_mode=1), x0=x0)
