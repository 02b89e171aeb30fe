"""Limits and degenerate cases: the largest label count and the largest
degree the library accepts (against the oracle), one label, inputs beyond the
documented limits, and configurations out of range."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import PARAM_RTOL, assert_graph_equal, dev_tensors, gpu_arrays, rel_close, slice_view, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def _em_vs_oracle(pairs, L, beta=1.0, max_iters=20):
    pmrf = _pmrf()
    g = pmrf.build_graph([torch.from_numpy(a).cuda() for a, _ in pairs],
                         [torch.from_numpy(b).cuda() for _, b in pairs])
    out = g.em(pmrf.EMConfig(n_labels=L, beta=beta, max_iters=max_iters))
    g.sync_status()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    for s, (a, b) in enumerate(pairs):
        og = oracle.Graph.from_image(a, b)
        r = og.em(oracle.EMConfig(n_labels=L, beta=beta, max_iters=max_iters))
        assert it[s] == r["iters"], (s, it[s], r["iters"])
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert np.array_equal(th[s, :, 0], r["theta"][:, 0])
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
    return g


def test_largest_label_count():
    """L = 8 (PMRF_MAX_LABELS): intensities spread over [0, 1] so that every
    threshold bin starts non-empty."""
    sl = synth.make_stack(small_specs(3, seed0=1200))
    pairs = [(s.image, s.region_ids) for s in sl]
    _em_vs_oracle(pairs, 8, beta=0.5)


def test_one_label():
    sl = synth.make_stack(small_specs(2, seed0=1210))
    g = _em_vs_oracle([(s.image, s.region_ids) for s in sl], 1)
    assert int(g.em(_pmrf().EMConfig(n_labels=1))["labels"].max()) == 0


def _star(n_cells):
    """A background region touched by n_cells small cells along its top row."""
    W = 2 * n_cells
    ids = np.zeros((3, W), np.int32)
    ids[1:, :] = 1
    ids[0, :] = 2 + np.arange(W) // 2
    img = np.random.default_rng(n_cells).random((3, W))
    return img, ids


def test_largest_degree_accepted_and_beyond_rejected():
    pmrf = _pmrf()
    img, ids = _star(4096)  # the background has PMRF_MAX_DEGREE neighbours
    g = pmrf.build_graph(torch.from_numpy(img).cuda(), torch.from_numpy(ids).cuda())
    og = oracle.Graph.from_image(img, ids)
    assert int(np.diff(og.adj_off).max()) == 4096
    assert_graph_equal(og, slice_view(gpu_arrays(g), 0))
    _em_vs_oracle([(img, ids)], 2, max_iters=10)
    img, ids = _star(4097)
    with pytest.raises(pmrf.PmrfError) as e:
        pmrf.build_graph(torch.from_numpy(img).cuda(), torch.from_numpy(ids).cuda())
    assert e.value.code == 6  # PMRF_ERR_UNSUPPORTED


@pytest.mark.parametrize("bad", [dict(n_labels=0), dict(n_labels=9), dict(beta=-0.5), dict(beta=2.0 ** 32),
                                 dict(max_iters=0), dict(conv_window=0), dict(sigma_min=0.0),
                                 dict(init_lo=1.0, init_hi=0.5), dict(potts_scope=2), dict(replica_rule=3)])
def test_configurations_out_of_range(bad):
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(1, seed0=1220))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    with pytest.raises(pmrf.PmrfError) as e:
        g.em(pmrf.EMConfig(**bad))
    assert e.value.code == 1  # PMRF_ERR_ARG
    g.em(pmrf.EMConfig(n_labels=2))  # the graph stays usable
