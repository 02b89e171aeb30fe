"""k-neighbourhoods (Section 3.1) on the GPU against the oracle: the hoods,
replica lists and the EM path built on them."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import (ENERGY_RTOL, PARAM_RTOL, assert_graph_equal, assert_labels_match, gpu_arrays, label_gap,
                           rel_close, rep_lists_from_oracle, slice_view, small_specs)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def _pairs(seed0):
    sl = synth.make_stack(small_specs(4, seed0=seed0))
    pairs = [(s.image, s.region_ids) for s in sl]
    H, W = 24, 140  # a region touching 70 cells: degree > 32, wide hoods
    ids = np.zeros((H, W), np.int32)
    ids[1:, :] = 1000
    for k in range(70):
        ids[0, 2 * k:2 * k + 2] = 7 + 3 * k
    pairs.append((np.random.default_rng(0).random((H, W)), ids))
    return pairs


def _build(pairs, k):
    return _pmrf().build_graph([torch.from_numpy(a).cuda() for a, _ in pairs],
                               [torch.from_numpy(b).cuda() for _, b in pairs], hood_depth=k)


@pytest.mark.parametrize("k", [2, 3])
def test_k_hoods_match_oracle(k):
    pairs = _pairs(950 + k)
    g = _build(pairs, k)
    arrs = gpu_arrays(g)
    for s, (a, b) in enumerate(pairs):
        og = oracle.Graph.from_image(a, b, hood_depth=k)
        gv = slice_view(arrs, s)
        assert_graph_equal(og, gv)
        ro = arrs["REP_OFF"]
        want = rep_lists_from_oracle(og)
        for v in range(og.V):
            got = (arrs["REP_HOOD"][ro[gv["v0"] + v]:ro[gv["v0"] + v + 1]] - gv["c0"]).tolist()
            assert got == want[v], (s, v)


def test_em_on_two_hoods_matches_oracle():
    pmrf = _pmrf()
    pairs = _pairs(960)
    g = _build(pairs, 2)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=30)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    T = out["T_hist"].cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    for s, (a, b) in enumerate(pairs):
        og = oracle.Graph.from_image(a, b, hood_depth=2)
        r = og.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=30))
        assert it[s] == r["iters"], (s, it[s], r["iters"])
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert rel_close(T[s, :r["iters"]], r["T_hist"], ENERGY_RTOL)


def test_em_sparse_loop_on_two_hoods():
    """The sparse EM loop with two lanes per hood (64-hood tiles, the launch
    shape of 2-neighbourhoods, whose hoods hold 23 members on average here): 24
    small slices whose oracle runs keep several slices iterating in the sparse
    loop.  Every slice matches the oracle's run; the whole output equals the
    kernel-by-kernel loop's."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(24, seed0=700))
    pairs = [(s.image, s.region_ids) for s in sl]
    ocfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    ogs = [oracle.Graph.from_image(a, b, hood_depth=2) for a, b in pairs]
    runs = [og.em(ocfg) for og in ogs]
    its = np.array([r["iters"] for r in runs])
    assert sum(og.N_el for og in ogs) >= 16 * sum(og.C for og in ogs)  # two lanes per hood
    tiles = np.array([-(-og.V // 128) + -(-og.C // 64) for og in ogs])
    sparse = [t for t in range(1, its.max() + 1) if 4 * tiles[its >= t].sum() < tiles.sum()]
    assert sum((its >= t).sum() >= 2 for t in sparse) >= 2
    g = _build(pairs, 2)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    T = out["T_hist"].cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    assert list(out["iters"].cpu().numpy()) == list(its)
    for s, r in enumerate(runs):
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert rel_close(T[s, :r["iters"]], r["T_hist"], ENERGY_RTOL)
    g.set_tuning(use_cuda_graph=0)
    od = g.em(cfg, want_T=True)
    g.sync_status()
    for k in ("labels", "params", "iters", "converged", "T_hist"):
        assert torch.equal(out[k], od[k]), k


def test_sweep_on_three_hoods_three_labels():
    pmrf = _pmrf()
    pairs = _pairs(970)
    g = _build(pairs, 3)
    L = 3
    rng = np.random.default_rng(9)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    theta = np.zeros((g.S, L, 4))
    theta[:, :, 1] = np.sort(rng.uniform(0.2, 0.8, (g.S, L)), axis=1)
    theta[:, :, 2] = rng.uniform(0.05, 0.3, (g.S, L))
    cfg = pmrf.EMConfig(n_labels=L, beta=0.7)
    xo, ev, eh = g.map_sweep(cfg, torch.from_numpy(x).cuda(), torch.from_numpy(theta).cuda())
    xo, ev, eh = xo.cpu().numpy(), ev.cpu().numpy(), eh.cpu().numpy()
    arrs = gpu_arrays(g)
    for s, (a, b) in enumerate(pairs):
        og = oracle.Graph.from_image(a, b, hood_depth=3)
        v0, v1 = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        c0, c1 = arrs["HOOD_SLICE_OFF"][s], arrs["HOOD_SLICE_OFF"][s + 1]
        r = og.map_sweep(L, cfg.beta, x[v0:v1], theta[s, :, 1], theta[s, :, 2], want_second=True)
        assert_labels_match(xo[v0:v1], r["x_new"], label_gap(r["E_star"], r["E_second"]), f"slice {s}")
        assert rel_close(ev[v0:v1], r["E_star"], 1e-12, 1e-13)
        assert rel_close(eh[c0:c1], r["S"], ENERGY_RTOL, 1e-12)


def test_hood_depth_out_of_range():
    pmrf = _pmrf()
    pairs = _pairs(980)[:1]
    for k in (0, 9):
        with pytest.raises(pmrf.PmrfError):
            _build(pairs, k)
