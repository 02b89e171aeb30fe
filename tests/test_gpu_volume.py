"""3-D region graphs of volumes on the GPU (6-connected voxels, reading G16)
against the oracle: the graph, hoods and the EM path built on it."""
import numpy as np
import pytest

import oracle
from pmrf_testutil import ENERGY_RTOL, PARAM_RTOL, assert_graph_equal, gpu_arrays, rel_close, slice_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def voronoi_volume(D, H, W, pitch, seed):
    """A seeded synthetic volume: nearest-seed regions on a jittered 3-D grid
    (raw ids = seed index, some cells empty), two phases (spheres) with
    Gaussian noise."""
    rng = np.random.default_rng(seed)
    g = [np.arange(p / 2, n, p) for n, p in zip((D, H, W), (max(1.0, pitch / 2), pitch, pitch))]
    cz, cy, cx = np.meshgrid(*g, indexing="ij")
    seeds = np.stack([cz.ravel(), cy.ravel(), cx.ravel()], 1) + rng.uniform(-1, 1, (cz.size, 3))
    z, y, x = np.meshgrid(np.arange(D) + 0.5, np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    pts = np.stack([z.ravel(), y.ravel(), x.ravel()], 1)
    d2 = ((pts[:, None, :] - seeds[None, :, :]) ** 2).sum(-1)
    ids = np.argmin(d2, 1).astype(np.int32).reshape(D, H, W) * 2 + 1
    phase = np.zeros((D, H, W))
    for _ in range(4):
        c = rng.uniform(0, 1, 3) * np.array([D, H, W])
        r = rng.uniform(3, 8)
        phase[((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) < r * r] = 1.0
    img = 0.3 + 0.4 * phase + rng.normal(0, 0.1, (D, H, W))
    return img, ids


def _build(vols, **kw):
    img = torch.from_numpy(np.concatenate([v[0] for v in vols])).cuda()
    ids = torch.from_numpy(np.concatenate([v[1] for v in vols])).cuda()
    return _pmrf().build_graph(img, ids, volume_depth=vols[0][0].shape[0], **kw)


def test_volume_graphs_match_oracle():
    vols = [voronoi_volume(5, 24, 28, 4.0, seed) for seed in (1, 2, 3)]
    g = _build(vols)
    assert g.S == 3
    arrs = gpu_arrays(g)
    for s, (a, b) in enumerate(vols):
        og = oracle.Graph.from_volume(a, b)
        assert_graph_equal(og, slice_view(arrs, s))


def test_em_on_volumes_matches_oracle():
    pmrf = _pmrf()
    vols = [voronoi_volume(6, 20, 20, 4.0, seed) for seed in (11, 12)]
    g = _build(vols)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=30)
    out = g.em(cfg, want_T=True)
    seg = g.label_image(torch.from_numpy(np.concatenate([v[1] for v in vols])).cuda(), out["labels"])
    g.sync_status()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    T = out["T_hist"].cpu().numpy()
    seg = seg.cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    p0 = 0
    for s, (a, b) in enumerate(vols):
        og = oracle.Graph.from_volume(a, b)
        r = og.em(oracle.EMConfig(n_labels=2, beta=1.0, max_iters=30))
        assert it[s] == r["iters"], (s, it[s], r["iters"])
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert rel_close(T[s, :r["iters"]], r["T_hist"], ENERGY_RTOL)
        assert np.array_equal(seg[p0:p0 + b.size], og.label_image(b.reshape(-1, b.shape[-1]), r["labels"]).ravel())
        p0 += b.size


def test_volume_with_two_hoods():
    vols = [voronoi_volume(4, 16, 18, 4.0, 21)]
    g = _build(vols, hood_depth=2)
    og = oracle.Graph.from_volume(*vols[0], hood_depth=2)
    assert_graph_equal(og, slice_view(gpu_arrays(g), 0))


def test_volume_arguments_rejected():
    pmrf = _pmrf()
    a, b = voronoi_volume(3, 8, 8, 4.0, 31)
    img = torch.from_numpy(a).cuda()
    ids = torch.from_numpy(b).cuda()
    with pytest.raises(pmrf.PmrfError):  # 3 slices, volumes of 2
        pmrf.build_graph(img, ids, volume_depth=2)
    with pytest.raises(pmrf.PmrfError):  # layers of unequal size
        pmrf.build_graph([img[0], img[1][:7]], [ids[0], ids[1][:7]], volume_depth=2)
