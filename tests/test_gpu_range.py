"""Energies far from the unit range: 8-bit-scaled intensities (the paper's
data are 8-bit grayscale), a label whose deviation collapses to sigma_min, and
the paper's random start drawn over [0, 255].  The device keeps every energy
sum in a per-slice fixed point whose unit follows the size of that slice's
energies, so these runs must equal the oracle's (iteration counts, labels,
parameters, totals) rather than lose range."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import ENERGY_RTOL, PARAM_RTOL, rel_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _slice(seed, scale, noise=None, H=96, W=112):
    sp = synth.scaled(synth.workload("slice256").slices[0], H, W, seed=seed)
    if noise is not None:
        sp = synth.replace(sp, noise_sigma=noise)
    s = synth.make_slice(sp)
    return s.image * scale, s.region_ids


def _compare(out, r, what):
    assert int(out["iters"][0]) == r["iters"], what
    assert int(out["converged"][0]) == r["converged"], what
    assert np.array_equal(out["labels"].cpu().numpy(), r["labels"]), what
    th = out["params"][0].cpu().numpy()
    assert np.array_equal(th[:, 0], r["theta"][:, 0]), what
    assert rel_close(th[:, 1:3], r["theta"][:, 1:3], PARAM_RTOL), what
    assert rel_close(out["T_hist"][0].cpu().numpy()[:r["iters"]], r["T_hist"], ENERGY_RTOL, 1e-12), what


def _graph(img, ids):
    import paper_1809_05018_b300 as pmrf
    return pmrf.build_graph(torch.from_numpy(np.ascontiguousarray(img)).cuda(),
                            torch.from_numpy(np.ascontiguousarray(ids)).cuda())


@pytest.mark.parametrize("L,beta", [(2, 1.0), (3, 25.0)])
def test_eight_bit_intensities_match_the_oracle(L, beta):
    import paper_1809_05018_b300 as pmrf
    img, ids = _slice(4100 + L, 255.0)
    g = _graph(img, ids)
    out = g.em(pmrf.EMConfig(n_labels=L, beta=beta, max_iters=40, init_lo=0.0, init_hi=255.0), want_T=True)
    g.sync_status()
    og = oracle.Graph.from_image(img, ids)
    r = og.em(oracle.EMConfig(n_labels=L, beta=beta, max_iters=40, init_lo=0.0, init_hi=255.0))
    _compare(out, r, "8-bit")
    assert np.abs(r["T_hist"]).max() > 1e3  # the totals are far beyond the unit range


def test_collapsed_deviation_matches_the_oracle():
    # every region constant; the regions of label 0 all exactly 50: that
    # label's deviation is 0, floored to sigma_min = 1e-6, so the other
    # label's vertices see a label-0 data term near 100^2 / 2e-12 = 5e15 (an
    # excess the device saturates) beside their own of a few units
    import paper_1809_05018_b300 as pmrf
    _, ids = _slice(4200, 255.0)
    r_id = ids.astype(np.int64)
    img = np.where(r_id % 3 == 0, 50.0, 150.0 + (r_id % 7)).astype(np.float64)
    og = oracle.Graph.from_image(img, ids)
    cfg = dict(n_labels=2, beta=1.0, max_iters=30, init_lo=0.0, init_hi=255.0)
    r = og.em(oracle.EMConfig(**cfg))
    assert r["theta"][0, 2] == 1e-6  # the collapse happened
    g = _graph(img, ids)
    out = g.em(pmrf.EMConfig(**cfg), want_T=True)
    g.sync_status()
    _compare(out, r, "collapsed sigma")
    # the hood sums of the last sweep, against the oracle's, at the large range
    xo, ev, eh = g.map_sweep(pmrf.EMConfig(**cfg), out["labels"], out["params"].contiguous())
    th = r["theta"]
    rs = og.map_sweep(2, 1.0, r["labels"], th[:, 1], th[:, 2], want_elements=True)
    assert rs["E_el"].max() > 1e15
    assert rel_close(eh.cpu().numpy(), rs["S"], ENERGY_RTOL, 1e-12)
    assert np.array_equal(xo.cpu().numpy(), rs["x_new"])


@pytest.mark.parametrize("lo,hi", [(0.0, 255.0), (0.0, 1e-5)])
def test_random_start_over_eight_bit_range_matches_the_oracle(lo, hi):
    # the paper's random start (labels, means and deviations drawn between lo
    # and hi); with hi = 1e-5 every drawn deviation is at or near sigma_min
    import paper_1809_05018_b300 as pmrf
    img, ids = _slice(4300, 255.0)
    g = _graph(img, ids)
    x0, th0 = g.random_init(2, seed=99, lo=lo, hi=hi)
    out = g.em(pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=30), labels=x0, params=th0, want_T=True)
    g.sync_status()
    og = oracle.Graph.from_image(img, ids)
    xo, tho = oracle.random_init(og.V, 2, 99, 0, lo, hi)
    assert np.array_equal(x0.cpu().numpy(), xo)
    r = og.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=30, init_mode=2), x0=xo, theta0=tho)
    _compare(out, r, f"random start [{lo}, {hi}]")
    if hi < 1.0:
        assert np.abs(r["T_hist"]).max() > 1e15  # every least data term is huge
