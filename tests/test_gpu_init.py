"""EM starts on the GPU against the oracle: the paper's random start
(SplitMix64 draws, bit-exact), and EM runs from given labels and from given
labels and parameters."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import ENERGY_RTOL, PARAM_RTOL, dev_tensors, rel_close, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def _graph(seed0, n=5):
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(n, seed0=seed0))
    imgs, ids = dev_tensors(sl)
    return sl, pmrf.build_graph(imgs, ids)


@pytest.mark.parametrize("L", [1, 2, 3, 8])
def test_random_start_bit_exact(L):
    sl, g = _graph(900)
    x, th = g.random_init(L, seed=0xC0FFEE + L, lo=0.0, hi=255.0)
    x, th = x.cpu().numpy(), th.cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    for s in range(g.S):
        ox, oth = oracle.random_init(int(vo[s + 1] - vo[s]), L, 0xC0FFEE + L, s, 0.0, 255.0)
        assert np.array_equal(x[vo[s]:vo[s + 1]], ox), s
        assert np.array_equal(th[s], oth), s


@pytest.mark.parametrize("mode", [1, 2])
def test_em_from_given_start_matches_oracle(mode):
    pmrf = _pmrf()
    sl, g = _graph(910)
    x0, th0 = g.random_init(2, seed=77, lo=0.0, hi=1.0)
    th0[1, 0, 2] = 1e-9  # below sigma_min: floored at the start
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=40)
    out = g.em(cfg, labels=x0, params=th0 if mode == 2 else None, want_T=True)
    g.sync_status()
    xs, ths = x0.cpu().numpy(), th0.cpu().numpy()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    T = out["T_hist"].cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    ocfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=40, init_mode=mode)
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        r = og.em(ocfg, x0=xs[vo[s]:vo[s + 1]], theta0=ths[s] if mode == 2 else None)
        assert it[s] == r["iters"], (s, it[s], r["iters"])
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert np.array_equal(th[s, :, 0], r["theta"][:, 0])
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert rel_close(T[s, :r["iters"]], r["T_hist"], ENERGY_RTOL)


def test_bad_start_mode_rejected():
    pmrf = _pmrf()
    sl, g = _graph(920, n=2)
    with pytest.raises(pmrf.PmrfError):
        g.em(pmrf.EMConfig(n_labels=2, init_from_labels=3))
