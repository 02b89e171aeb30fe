"""The two convergence tests of Section 3.2.2 on the GPU (reading G9): a run
that the EM (total) check alone ends, and runs whose window must reach back W
iterations, compared with the oracle's runs (iteration counts, stop flags,
labels, parameters)."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import PARAM_RTOL, rel_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_both(s, L, beta, tol, W=3, max_iters=40):
    import paper_1809_05018_b300 as pmrf
    g = pmrf.build_graph(torch.from_numpy(s.image).cuda(), torch.from_numpy(s.region_ids).cuda())
    out = g.em(pmrf.EMConfig(n_labels=L, beta=beta, max_iters=max_iters, conv_tol=tol, conv_window=W), want_T=True)
    g.sync_status()
    og = oracle.Graph.from_image(s.image, s.region_ids)
    r = og.em(oracle.EMConfig(n_labels=L, beta=beta, max_iters=max_iters, conv_tol=tol, conv_window=W))
    return out, r


def test_em_total_check_alone_ends_the_run():
    # a 64x64 slice on which, with tolerance 1, the labels settle after the
    # second iteration and the hoods' sums of iterations 1 and 4 still differ by
    # up to 2.1 (25 hoods at or above the tolerance, the nearest 0.016 from it)
    # while the totals of iterations 1..4 differ by at most 0.557: the EM check
    # ends the run at t = 4, one iteration before the MAP check would
    s = synth.make_slice(synth.scaled(synth.workload("slice256").slices[0], 64, 64, seed=3056))
    out, r = _run_both(s, 2, 1.0, 1.0)
    assert r["stop"] == 2 and r["iters"] == 4 and r["converged"] == 1  # the EM check only
    assert int(out["iters"][0]) == 4 and int(out["converged"][0]) == 1
    assert np.array_equal(out["labels"].cpu().numpy(), r["labels"])
    assert rel_close(out["params"][0].cpu().numpy()[:, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
    assert rel_close(out["T_hist"][0].cpu().numpy()[:4], r["T_hist"], 1e-12, 1e-12)


@pytest.mark.parametrize("W,tol", [(1, 1e-4), (2, 1e-4), (5, 1e-4), (3, 0.5)])
def test_em_window_and_tolerance_match_the_oracle(W, tol):
    sl = synth.make_stack([synth.scaled(synth.workload("slice256").slices[0], 96, 80, seed=3100 + k)
                           for k in range(3)])
    for s in sl:
        out, r = _run_both(s, 2, 1.0, tol, W=W)
        assert int(out["iters"][0]) == r["iters"] and int(out["converged"][0]) == r["converged"]
        assert np.array_equal(out["labels"].cpu().numpy(), r["labels"])
        assert rel_close(out["params"][0].cpu().numpy()[:, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
