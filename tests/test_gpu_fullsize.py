"""Parity at the full workload sizes, in the launch configuration bench.py
times (one build over the whole batch, the EM loop replayed from its CUDA
graph), on outputs the oracle can compute one slice at a time."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import PARAM_RTOL, ENERGY_RTOL, assert_graph_equal, assert_labels_match, gpu_arrays, label_gap, \
    rel_close, slice_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


def _stack_tensors(sl):
    img = torch.from_numpy(np.stack([s.image for s in sl])).cuda()
    ids = torch.from_numpy(np.stack([s.region_ids for s in sl])).cuda()
    return img, ids


def test_stack512_sampled_slices_match_oracle():
    """512 slices of 1024x1024 in one batch (the bench workload); three
    sampled slices checked end to end against the oracle, segmentation quality
    against the phase maps included."""
    pmrf = _pmrf()
    wl = synth.workload("stack512")
    sl = synth.make_stack(wl.slices)
    img, ids = _stack_tensors(sl)
    g = pmrf.build_graph(img, ids)
    cfg = pmrf.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    out = g.em(cfg)
    segd = g.label_image(ids, out["labels"])
    conf, met = g.quality(wl.n_labels, segd, torch.from_numpy(np.stack([s.truth for s in sl])).cuda())
    seg = segd.cpu().numpy().reshape(len(sl), -1)
    conf, met = conf.cpu().numpy(), met.cpu().numpy()
    g.sync_status()
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    assert g.S == 512 and (it >= 1).all() and (it <= wl.max_iters).all()
    ocfg = oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    for s in (0, 257, 511):
        og = oracle.Graph.from_image(sl[s].image, sl[s].region_ids)
        assert og.V == vo[s + 1] - vo[s]
        r = og.em(ocfg)
        assert it[s] == r["iters"]
        assert np.array_equal(x[vo[s]:vo[s + 1]], r["labels"]), s
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert np.array_equal(seg[s], og.label_image(sl[s].region_ids, r["labels"]).ravel())
        oc, om = oracle.quality(seg[s], sl[s].truth, wl.n_labels)
        assert np.array_equal(conf[s], oc) and np.array_equal(met[s], om)


def test_slice2048_matches_oracle():
    """The 2048x2048 single-slice workload, end to end."""
    pmrf = _pmrf()
    wl = synth.workload("slice2048")
    s = synth.make_slice(wl.slices[0])
    g = pmrf.build_graph(torch.from_numpy(s.image).cuda(), torch.from_numpy(s.region_ids).cuda())
    cfg = pmrf.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    out = g.em(cfg, want_T=True)
    og = oracle.Graph.from_image(s.image, s.region_ids)
    assert_graph_equal(og, slice_view(gpu_arrays(g), 0))
    r = og.em(oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters))
    assert int(out["iters"][0]) == r["iters"] and int(out["converged"][0]) == r["converged"]
    assert np.array_equal(out["labels"].cpu().numpy(), r["labels"])
    assert rel_close(out["params"][0].cpu().numpy()[:, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
    assert rel_close(out["T_hist"][0].cpu().numpy()[:r["iters"]], r["T_hist"], ENERGY_RTOL)


def test_large8192_three_phase():
    """8192x8192, three labels, beta 1.5: the full graph equals the oracle's;
    one sweep from the GPU's final state agrees with the oracle's sweep (labels
    at the gap rule, vertex and hood energies); the parameters are the
    label-conditional moments of the returned labels."""
    pmrf = _pmrf()
    wl = synth.workload("large8192")
    s = synth.make_slice(wl.slices[0])
    g = pmrf.build_graph(torch.from_numpy(s.image).cuda(), torch.from_numpy(s.region_ids).cuda())
    cfg = pmrf.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    out = g.em(cfg)
    g.sync_status()
    og = oracle.Graph.from_image(s.image, s.region_ids)
    arrs = gpu_arrays(g)
    assert_graph_equal(og, slice_view(arrs, 0))
    x = out["labels"]
    th = out["params"]
    xo, ev, eh = g.map_sweep(cfg, x, th.contiguous())
    xn = x.cpu().numpy()
    thn = th[0].cpu().numpy()
    r = og.map_sweep(wl.n_labels, wl.beta, xn, thn[:, 1], thn[:, 2], want_second=True)
    assert_labels_match(xo.cpu().numpy(), r["x_new"], label_gap(r["E_star"], r["E_second"]), "large8192")
    assert rel_close(ev.cpu().numpy(), r["E_star"], 1e-12, 1e-13)
    assert rel_close(eh.cpu().numpy(), r["S"], ENERGY_RTOL, 1e-12)
    for l in range(wl.n_labels):
        sel = xn == l
        assert thn[l, 0] == sel.sum()
        if sel.any():
            assert abs(thn[l, 1] - og.y[sel].mean()) <= 1e-12 * max(1.0, abs(thn[l, 1]))
            assert abs(thn[l, 2] - max(og.y[sel].std(ddof=0), 1e-6)) <= 1e-9 * thn[l, 2]


def test_grad64_adjoint_and_beta_fit():
    """64 slices of 2048x2048: the adjoint of the summed pseudo-log-likelihood
    on one sampled slice equals the oracle's gradient; the beta fit runs 30
    steps."""
    pmrf = _pmrf()
    from paper_1809_05018_b300.autograd import fit_beta
    wl = synth.workload("grad64")
    sl = synth.make_stack(wl.slices)
    img, ids = _stack_tensors(sl)
    g = pmrf.build_graph(img, ids)
    out = g.em(pmrf.EMConfig(n_labels=2, beta=wl.beta, max_iters=wl.max_iters))
    lab = out["labels"]
    mu = out["params"][:, :, 1].contiguous()
    sg = out["params"][:, :, 2].contiguous()
    gout = torch.ones(g.S, dtype=torch.float64, device="cuda")
    beta = 0.2
    gmu, gsg, gb = g.pll_grad(2, lab, mu, sg, beta, gout)
    pll = g.pll(2, lab, mu, sg, beta).cpu().numpy()
    vo = g.array("VERT_OFF").numpy()
    xs = lab.cpu().numpy()
    s = 33
    og = oracle.Graph.from_image(sl[s].image, sl[s].region_ids)
    f, om, osg, ob = og.pll(2, xs[vo[s]:vo[s + 1]], mu[s].cpu().numpy(), sg[s].cpu().numpy(), beta)
    assert rel_close(pll[s], f, 1e-12, 1e-9)
    assert rel_close(gmu[s].cpu().numpy(), om, 1e-10, 1e-8)
    assert rel_close(gsg[s].cpu().numpy(), osg, 1e-10, 1e-8)
    traj = fit_beta(g, lab, mu, sg, beta0=0.2, steps=30)
    assert len(traj) == 31 and all(np.isfinite(traj)) and min(traj) >= 0.0
