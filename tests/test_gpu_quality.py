"""Segmentation quality (Section 4.2.1) on the GPU against the oracle: the
confusion counts must be identical and the ratios bit-equal (the same IEEE
divisions of the same integers), NaN where the oracle has NaN."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import dev_tensors, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def _same(a, b):
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


def _check(g, L, pred, truth, sizes):
    conf, met = g.quality(L, pred, truth)
    conf, met = conf.cpu().numpy(), met.cpu().numpy()
    p = pred.reshape(-1).cpu().numpy()
    t = truth.reshape(-1).cpu().numpy()
    o = 0
    for s, n in enumerate(sizes):
        oc, om = oracle.quality(p[o:o + n], t[o:o + n], L)
        assert np.array_equal(conf[s], oc), s
        assert _same(met[s], om), s
        o += n


def test_quality_of_em_segmentation_matches_oracle():
    """Slices of mixed sizes (odd pixel counts put later slices off 4-byte
    alignment): EM labels -> label image -> quality against the phase maps."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(6, seed0=700))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=30))
    pred = g.label_image(ids, out["labels"])
    truth = torch.from_numpy(np.concatenate([s.truth.ravel() for s in sl])).cuda()
    _check(g, 2, pred, truth, [s.truth.size for s in sl])
    g.sync_status()


@pytest.mark.parametrize("L", [1, 3, 8])
def test_quality_random_labels_and_misaligned_buffers(L):
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(5, seed0=710))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    n = g.n_pix
    rng = np.random.default_rng(L)
    # label L-1 absent from the truth when L > 1: its precision stays defined,
    # its recall is NaN
    tr = rng.integers(0, max(1, L - 1), size=n).astype(np.uint8)
    pr = rng.integers(0, L, size=n).astype(np.uint8)
    buf_p = torch.zeros(n + 1, dtype=torch.uint8, device="cuda")
    buf_t = torch.zeros(n + 3, dtype=torch.uint8, device="cuda")
    buf_p[1:] = torch.from_numpy(pr).cuda()
    buf_t[3:] = torch.from_numpy(tr).cuda()
    _check(g, L, buf_p[1:], buf_t[3:], [s.truth.size for s in sl])
    g.sync_status()


def test_quality_label_out_of_range_is_reported():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(2, seed0=720))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    pred = torch.zeros(g.n_pix, dtype=torch.uint8, device="cuda")
    truth = torch.zeros(g.n_pix, dtype=torch.uint8, device="cuda")
    pred[1234] = 2
    conf, _ = g.quality(2, pred, truth)
    with pytest.raises(pmrf.PmrfError) as e:
        g.sync_status()
    assert e.value.code == 1  # PMRF_ERR_ARG
    assert int(conf.sum()) == g.n_pix - 1
