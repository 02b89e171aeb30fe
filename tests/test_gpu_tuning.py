"""Tuning and profiling hooks: results do not depend on the tile sizes or on
the graph replay, the autotuner returns a valid tuning, and the profiled run
reports one time per iteration."""
import numpy as np
import pytest

import synth
from pmrf_testutil import dev_tensors, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def test_results_independent_of_tiles_and_replay():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(6, seed0=1100))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=30)
    ref = g.em(cfg, want_T=True)
    ref = {k: v.clone() for k, v in ref.items()}
    for tuning in (dict(hood_tile=32), dict(hood_tile=256), dict(hood_tile=1024), dict(hood_lanes=1),
                   dict(hood_lanes=2), dict(hood_lanes=8), dict(hood_tile=32, hood_lanes=8),
                   dict(use_cuda_graph=0), dict(profile=1)):
        g.set_tuning(**tuning)
        out = g.em(cfg, want_T=True)
        for k in ("labels", "params", "iters", "converged", "T_hist"):
            assert torch.equal(out[k], ref[k]), (tuning, k)
    g.sync_status()


def test_autotune_and_kernel_times():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(4, seed0=1110))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=25)
    ref = g.em(cfg)
    ref = {k: v.clone() for k, v in ref.items()}
    best = g.autotune(cfg)
    assert 32 <= best["hood_tile"] <= 1024 and best["hood_tile"] % 32 == 0
    assert best["hood_lanes"] in (1, 2, 4, 8)
    assert g.tuning()["hood_tile"] == best["hood_tile"] and g.tuning()["hood_lanes"] == best["hood_lanes"]
    # a second graph of the same shape left at the defaults runs with the kept result
    g2 = pmrf.build_graph(imgs, ids)
    assert g2.tuning()["hood_tile"] == 0 and g2.tuning()["hood_lanes"] == 0
    out2 = g2.em(cfg)
    for k in ("labels", "params", "iters"):
        assert torch.equal(out2[k], ref[k]), k
    out = g.em(cfg)
    for k in ("labels", "params", "iters"):
        assert torch.equal(out[k], ref[k]), k
    g.set_tuning(hood_tile=best["hood_tile"], hood_lanes=best["hood_lanes"], profile=1)
    out = g.em(cfg)
    tv, th = g.em_kernel_times()
    n_run = int(out["iters"].max())
    assert len(tv) == len(th) == n_run
    assert all(t > 0 for t in tv) and all(t > 0 for t in th)
