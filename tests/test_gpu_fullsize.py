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


def _oracle_graphs(sl):
    """Oracle graphs of the slices, built on all host cores (the C oracle
    releases the GIL)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda one: oracle.Graph.from_image(one.image, one.region_ids), sl))


def test_large8192_three_phase():
    """8192x8192, three labels, beta 1.5, <= 100 iterations, one slice of about
    2.7 M regions: the full graph equals the oracle's, and the whole EM run
    equals the oracle's (iteration count, stop, labels, parameters, the total
    of every iteration).  The oracle's sweep runs on all host cores here
    (its multi-core form gives the serial sweep's results exactly)."""
    import os
    pmrf = _pmrf()
    wl = synth.workload("large8192")
    s = synth.make_slice(wl.slices[0])
    g = pmrf.build_graph(torch.from_numpy(s.image).cuda(), torch.from_numpy(s.region_ids).cuda())
    cfg = pmrf.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    og = oracle.Graph.from_image(s.image, s.region_ids)
    assert_graph_equal(og, slice_view(gpu_arrays(g), 0))
    r = og.em(oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters,
                              n_threads=os.cpu_count() or 1))
    it = int(out["iters"][0])
    assert it == r["iters"] and int(out["converged"][0]) == r["converged"]
    xg = out["labels"].cpu().numpy()
    assert np.array_equal(xg, r["labels"]), f"{int((xg != r['labels']).sum())} labels differ"
    th = out["params"][0].cpu().numpy()
    assert rel_close(th[:, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
    assert np.array_equal(th[:, 0], r["theta"][:, 0])
    assert rel_close(out["T_hist"][0].cpu().numpy()[:it], r["T_hist"], ENERGY_RTOL, 1e-12)
    # one more sweep from the final state: labels at the gap rule, vertex and
    # hood energies
    xo, ev, eh = g.map_sweep(cfg, out["labels"], out["params"].contiguous())
    rs = og.map_sweep(wl.n_labels, wl.beta, xg, th[:, 1], th[:, 2], want_second=True)
    assert_labels_match(xo.cpu().numpy(), rs["x_new"], label_gap(rs["E_star"], rs["E_second"]), "large8192")
    assert rel_close(ev.cpu().numpy(), rs["E_star"], 1e-12, 1e-13)
    assert rel_close(eh.cpu().numpy(), rs["S"], ENERGY_RTOL, 1e-12)


def test_grad64_adjoint_and_beta_fit():
    """64 slices of 2048x2048 with their converged labels: the adjoint of the
    summed pseudo-log-likelihood equals the oracle's gradient on every slice;
    the summed dPLL/dbeta equals the oracle's and central differences of the
    GPU's summed PLL (h = 1e-6); the 30-step beta fit from 0.2 follows the
    oracle's fit."""
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
    ogs = _oracle_graphs(sl)
    mu_h, sg_h = mu.cpu().numpy(), sg.cpu().numpy()
    gmu_h, gsg_h = gmu.cpu().numpy(), gsg.cpu().numpy()
    xsl = [xs[vo[s]:vo[s + 1]] for s in range(g.S)]
    ob = []
    for s, og in enumerate(ogs):
        f, om, osg, b = og.pll(2, xsl[s], mu_h[s], sg_h[s], beta)
        assert rel_close(pll[s], f, 1e-12, 1e-9), s
        assert rel_close(gmu_h[s], om, 1e-10, 1e-8), s
        assert rel_close(gsg_h[s], osg, 1e-10, 1e-8), s
        ob.append(b)
    gbeta = float(gb.reshape(-1)[0])
    assert rel_close(gbeta, float(np.sum(ob)), 1e-10, 1e-8)
    h = 1e-6
    fd = (g.pll(2, lab, mu, sg, beta + h).sum().item() - g.pll(2, lab, mu, sg, beta - h).sum().item()) / (2 * h)
    assert abs(fd - gbeta) <= 1e-6 * max(1.0, abs(gbeta))
    traj = fit_beta(g, lab, mu, sg, beta0=0.2, steps=30)
    want = oracle.fit_beta(ogs, xsl, mu_h, sg_h, beta0=0.2, steps=30, lr=1.0)
    assert len(traj) == 31
    assert rel_close(traj, want, 1e-10, 1e-12)
