"""CUDA path vs the CPU oracle, element by element, on seeded synthetic
inputs.  Integer results (graph, cliques, hoods, replica lists) must be
identical; labels equal wherever the oracle's label-energy gap exceeds 1e-9
relative; parameters within 1e-10 relative; hood energies within 1e-12."""
import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import (ENERGY_RTOL, PARAM_RTOL, assert_graph_equal, assert_labels_match, dev_tensors,
                           gpu_arrays, label_gap, rel_close, rep_lists_from_oracle, slice_view, small_specs)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pmrf():
    import paper_1809_05018_b300 as pmrf
    return pmrf


# --------------------------------------------------------------------------
# graph construction

@pytest.mark.parametrize("which", ["slice256", "batch"])
def test_graph_matches_oracle(which):
    pmrf = _pmrf()
    if which == "slice256":
        specs = synth.workload("slice256").slices
    else:
        specs = small_specs(6, seed0=40)
    sl = synth.make_stack(specs)
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    arrs = gpu_arrays(g)
    assert g.S == len(sl)
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        gv = slice_view(arrs, s)
        assert_graph_equal(og, gv)
        # replica lists: hoods containing each vertex, ascending
        ro = arrs["REP_OFF"]
        v0 = gv["v0"]
        want = rep_lists_from_oracle(og)
        for v in range(og.V):
            got = (arrs["REP_HOOD"][ro[v0 + v]:ro[v0 + v + 1]] - gv["c0"]).tolist()
            assert got == want[v], (s, v)
        # raw id map: compact ids ascending, -1 where absent
        rk = arrs["RANK"][arrs["RANK_OFF"][s]:arrs["RANK_OFF"][s + 1]]
        assert np.array_equal(np.where(og.rank >= 0, og.rank + v0, -1), rk)


def test_graph_edge_cases():
    pmrf = _pmrf()
    # one region; a region touching 40 others (general paths, degree > 32 and
    # hoods wider than 32); non-contiguous ids; an empty slice in the batch
    one = (np.full((8, 9), 0.25), np.full((8, 9), 5, np.int32))
    H, W = 24, 140
    ids = np.zeros((H, W), np.int32)
    ids[1:, :] = 1000  # background: 3220 pixels, 70 neighbours, hoods of 71+ members
    for k in range(70):  # a strip of small cells along the top touching the background
        ids[0, 2 * k:2 * k + 2] = 7 + 3 * k
    img = np.random.default_rng(0).random((H, W))
    big = (img, ids)
    empty = (np.zeros((0, 5)), np.zeros((0, 5), np.int32))
    # a diagonal region (40 pixels spread over a 40x40 box) takes the sorted
    # pixel-list path for its mean; a few scattered pixels of a third id too
    did = np.full((40, 40), 3, np.int32)
    did[np.arange(40), np.arange(40)] = 7
    did[[0, 39, 5, 33], [39, 0, 20, 2]] = 11
    diag = (np.random.default_rng(1).random((40, 40)), did)
    cases = [one, big, empty, diag]
    imgs = [torch.from_numpy(a).cuda() for a, _ in cases]
    idt = [torch.from_numpy(b).cuda() for _, b in cases]
    g = pmrf.build_graph(imgs, idt)
    arrs = gpu_arrays(g)
    for s, (a, b) in enumerate(cases):
        og = oracle.Graph.from_image(a, b)
        assert_graph_equal(og, slice_view(arrs, s))
    # the EM loop through the general (wide) paths
    for L in (2, 3):
        cfg = pmrf.EMConfig(n_labels=L, beta=0.3, max_iters=15)
        out = g.em(cfg)
        g.sync_status()
        _em_compare([type("S", (), dict(image=a, region_ids=b)) for a, b in cases],
                    oracle.EMConfig(n_labels=L, beta=0.3, max_iters=15), cfg, g, out)


def test_graph_of_one_pixel_regions():
    """Every pixel its own region, ids a random permutation scattered over
    three times their number: one-pixel runs everywhere in the region-size
    pass, one-pixel boxes in the region scan, a grid graph with no triangle
    (every maximal clique an edge); sizes, means and the graph equal the
    oracle's."""
    pmrf = _pmrf()
    rng = np.random.default_rng(31)
    H, W = 40, 300
    ids = rng.permutation(H * W).astype(np.int32).reshape(H, W) * 3 + 1
    img = rng.random((H, W))
    g = pmrf.build_graph(torch.from_numpy(img).cuda(), torch.from_numpy(ids).cuda())
    og = oracle.Graph.from_image(img, ids)
    assert og.V == H * W
    assert_graph_equal(og, slice_view(gpu_arrays(g), 0))


def test_build_rejects_bad_input():
    pmrf = _pmrf()
    img = torch.rand(8, 8, dtype=torch.float64, device="cuda")
    ids = torch.zeros(8, 8, dtype=torch.int32, device="cuda")
    ids[3, 3] = -2
    with pytest.raises(pmrf.PmrfError) as e:
        pmrf.build_graph(img, ids)
    assert e.value.code == 1
    ids[3, 3] = 0
    img[2, 2] = float("nan")
    with pytest.raises(pmrf.PmrfError) as e:
        pmrf.build_graph(img, ids)
    assert e.value.code == 4
    # the context is still usable afterwards
    img[2, 2] = 0.5
    g = pmrf.build_graph(img, ids)
    assert g.V == 1
    # a non-finite pixel of a region whose box is too sparse for a box scan
    # (its mean comes from a sorted pixel list) is rejected as well
    img2 = torch.rand(16, 16, dtype=torch.float64, device="cuda")
    ids2 = torch.zeros(16, 16, dtype=torch.int32, device="cuda")
    ids2[0, 0] = 1
    ids2[15, 15] = 1
    img2[15, 15] = float("inf")
    with pytest.raises(pmrf.PmrfError) as e:
        pmrf.build_graph(img2, ids2)
    assert e.value.code == 4
    img2[15, 15] = 0.25
    g2 = pmrf.build_graph(img2, ids2)
    assert g2.V == 2 and abs(float(g2.array("Y")[1]) - (float(img2[0, 0]) + 0.25) / 2) < 1e-15


# --------------------------------------------------------------------------
# one MAP sweep, lock-step (same labels and parameters on both sides)

@pytest.mark.parametrize("L", [2, 3])
def test_map_sweep_lockstep(L):
    pmrf = _pmrf()
    specs = small_specs(4, seed0=7)
    sl = synth.make_stack(specs)
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    rng = np.random.default_rng(L)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    theta = np.zeros((g.S, L, 4))
    theta[:, :, 1] = np.sort(rng.uniform(0.2, 0.8, (g.S, L)), axis=1)
    theta[:, :, 2] = rng.uniform(0.05, 0.3, (g.S, L))
    cfg = pmrf.EMConfig(n_labels=L, beta=0.8)
    xo, ev, eh = g.map_sweep(cfg, torch.from_numpy(x).cuda(), torch.from_numpy(theta).cuda())
    xo, ev, eh = xo.cpu().numpy(), ev.cpu().numpy(), eh.cpu().numpy()
    arrs = gpu_arrays(g)
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        v0, v1 = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        c0, c1 = arrs["HOOD_SLICE_OFF"][s], arrs["HOOD_SLICE_OFF"][s + 1]
        r = og.map_sweep(L, cfg.beta, x[v0:v1], theta[s, :, 1], theta[s, :, 2], want_second=True)
        gap = label_gap(r["E_star"], r["E_second"])
        assert_labels_match(xo[v0:v1], r["x_new"], gap, f"slice {s}")
        assert rel_close(ev[v0:v1], r["E_star"], 1e-12, 1e-13)
        assert rel_close(eh[c0:c1], r["S"], ENERGY_RTOL, 1e-12)


def test_params_match_oracle():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(3, seed0=70))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    L = 3
    rng = np.random.default_rng(5)
    x = rng.integers(0, L, g.V).astype(np.uint8)
    arrs = gpu_arrays(g)
    v0, v1 = arrs["VERT_OFF"][1], arrs["VERT_OFF"][2]
    x[v0:v1][x[v0:v1] == 2] = 0  # slice 1: label 2 empty -> keeps the previous values
    E = rng.normal(size=g.V)
    prev = np.zeros((g.S, L, 4))
    prev[:, :, 1] = [0.1, 0.5, 0.9]
    prev[:, :, 2] = [0.2, 0.3, 0.4]
    cfg = pmrf.EMConfig(n_labels=L)
    th = g.params(cfg, torch.from_numpy(x).cuda(), torch.from_numpy(E).cuda(), torch.from_numpy(prev).cuda())
    th = th.cpu().numpy()
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        a, b = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        want = og.params(L, x[a:b], E[a:b], prev[s])
        assert np.array_equal(th[s, :, 0], want[:, 0])
        assert rel_close(th[s, :, 1:3], want[:, 1:3], PARAM_RTOL)
        assert rel_close(th[s, :, 3], want[:, 3], 1e-12, 1e-12)


# --------------------------------------------------------------------------
# the EM loop end to end

def _em_compare(sl, cfg_o, cfg_g, g, out):
    x = out["labels"].cpu().numpy()
    th = out["params"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    cv = out["converged"].cpu().numpy()
    arrs = gpu_arrays(g)
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        r = og.em(cfg_o)
        a, b = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        assert it[s] == r["iters"], (s, it[s], r["iters"])
        assert cv[s] == r["converged"]
        assert np.array_equal(x[a:b], r["labels"]), (s, int((x[a:b] != r["labels"]).sum()))
        assert np.array_equal(th[s, :, 0], r["theta"][:, 0])
        assert rel_close(th[s, :, 1:3], r["theta"][:, 1:3], PARAM_RTOL)
        assert rel_close(th[s, :, 3], r["theta"][:, 3], 1e-11, 1e-11)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_em_slice256_matches_oracle(use_graph):
    pmrf = _pmrf()
    wl = synth.workload("slice256")
    sl = synth.make_stack(wl.slices)
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    g.set_tuning(use_cuda_graph=use_graph)
    cfg = pmrf.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    _em_compare(sl, oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters), cfg, g, out)
    # T history matches the oracle's totals up to summation order
    og = oracle.Graph.from_image(sl[0].image, sl[0].region_ids)
    r = og.em(oracle.EMConfig(n_labels=wl.n_labels, beta=wl.beta, max_iters=wl.max_iters))
    T = out["T_hist"].cpu().numpy()[0, :r["iters"]]
    assert rel_close(T, r["T_hist"], ENERGY_RTOL)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_em_iteration_cap_mixed_with_converged_slices(use_graph):
    """Six slices run for at most 6 iterations: with these seeds the oracle's
    runs of two of them converge (after 5 and 4 iterations) and four stop at
    the cap unconverged.  The loop ends for the whole batch on the cap, whether
    it runs as the conditional graph node or kernel by kernel, and every slice
    keeps its own count, flag, labels and parameters."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(6, seed0=4200))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    g.set_tuning(use_cuda_graph=use_graph)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=6)
    out = g.em(cfg)
    g.sync_status()
    ocfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=6)
    ref = [oracle.Graph.from_image(s.image, s.region_ids).em(ocfg) for s in sl]
    # the case needs both kinds of slice
    assert any(r["converged"] == 1 and r["iters"] < 6 for r in ref)
    assert any(r["converged"] == 0 and r["iters"] == 6 for r in ref)
    assert list(out["iters"].cpu().numpy()) == [r["iters"] for r in ref]
    assert list(out["converged"].cpu().numpy()) == [r["converged"] for r in ref]
    _em_compare(sl, ocfg, cfg, g, out)


@pytest.mark.parametrize("seed0", [800, 700])
def test_em_sparse_loop_matches_oracle_and_direct(seed0):
    """24 small slices whose oracle runs stop between 4 and 60 iterations.  The
    loop graph runs its later iterations in the sparse loop (blocks that take
    only the tiles of slices still iterating) once those tiles are fewer than a
    quarter of the table: with seed 800 from t = 8 with five slices left, with
    seed 700 from t = 14 with two left, one of them to the 60-iteration cap.
    Every slice matches the oracle's run, and the whole output equals that of
    the kernel-by-kernel loop (one block per tile throughout)."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(24, seed0=seed0))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    ocfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    # the case reaches the sparse loop with more than one slice left (tiles of
    # 128 vertices and of 128 hoods)
    its, tiles = [], []
    for one in sl:
        og = oracle.Graph.from_image(one.image, one.region_ids)
        its.append(og.em(ocfg)["iters"])
        tiles.append(-(-og.V // 128) + -(-og.C // 128))
    its, tiles = np.array(its), np.array(tiles)
    sparse = [t for t in range(1, its.max() + 1) if 4 * tiles[its >= t].sum() < tiles.sum()]
    assert sum((its >= t).sum() >= 2 for t in sparse) >= 3
    out = g.em(cfg, want_T=True)
    g.sync_status()
    _em_compare(sl, ocfg, cfg, g, out)
    g.set_tuning(use_cuda_graph=0)
    od = g.em(cfg, want_T=True)
    for k in ("labels", "params", "iters", "converged", "T_hist"):
        assert torch.equal(out[k], od[k]), k


@pytest.mark.parametrize("L,beta,scope,rule,seed0", [(2, 1.0, 0, 1, 700), (2, 1.0, 0, 2, 700), (2, 1.0, 1, 0, 700),
                                                     (2, 1.0, 1, 1, 700), (2, 1.0, 1, 2, 700), (3, 1.5, 0, 0, 900)])
def test_em_sparse_loop_variants_and_three_labels(L, beta, scope, rule, seed0):
    """The sparse loop's other kernel instances: the sweep variants' vertex
    pass (Potts scope, replica rule) and the three-label hood pass, taking only
    the listed tiles.  24 small slices (three-phase ones for three labels)
    whose oracle runs leave at least two slices iterating in at least two of
    the sparse loop's iterations; every slice matches the oracle's run and the
    whole output equals the kernel-by-kernel loop's."""
    pmrf = _pmrf()
    specs = small_specs(24, seed0=seed0)
    if L == 3:
        specs = [synth.scaled(synth.workload("large8192").slices[0], sp.height, sp.width, seed=sp.seed)
                 for sp in specs]
    sl = synth.make_stack(specs)
    cfg = pmrf.EMConfig(n_labels=L, beta=beta, max_iters=60, potts_scope=scope, replica_rule=rule)
    ocfg = oracle.EMConfig(n_labels=L, beta=beta, max_iters=60, potts_scope=scope, replica_rule=rule)
    its, tiles = [], []
    for one in sl:
        og = oracle.Graph.from_image(one.image, one.region_ids)
        its.append(og.em(ocfg)["iters"])
        tiles.append(-(-og.V // 128) + -(-og.C // 128))
    its, tiles = np.array(its), np.array(tiles)
    sparse = [t for t in range(1, its.max() + 1) if 4 * tiles[its >= t].sum() < tiles.sum()]
    assert sum((its >= t).sum() >= 2 for t in sparse) >= 2
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    _em_compare(sl, ocfg, cfg, g, out)
    g.set_tuning(use_cuda_graph=0)
    od = g.em(cfg, want_T=True)
    g.sync_status()
    for k in ("labels", "params", "iters", "converged", "T_hist"):
        assert torch.equal(out[k], od[k]), k


def test_em_sparse_loop_with_a_wide_region():
    """The sparse loop's general hood tiles (a member with more than 32
    neighbours, taken hood by hood through the hood-local rows): 24 small
    slices plus one whose two middle rows are a single region touching 77
    cells, which keeps iterating for several of the sparse loop's iterations.
    Every slice matches the oracle's run; the whole output equals the
    kernel-by-kernel loop's."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(24, seed0=700))
    band = synth.make_slice(synth.scaled(small_specs(1, seed0=5018)[0], 48, 320, seed=5018))
    bids = band.region_ids.copy()
    bids[24:26, :] = bids.max() + 1
    sl.append(type("S", (), dict(image=band.image, region_ids=bids)))
    ocfg = oracle.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    ogs = [oracle.Graph.from_image(one.image, one.region_ids) for one in sl]
    assert np.diff(ogs[-1].adj_off).max() > 32
    its = np.array([og.em(ocfg)["iters"] for og in ogs])
    tiles = np.array([-(-og.V // 128) + -(-og.C // 128) for og in ogs])
    sparse = [t for t in range(1, its.max() + 1) if 4 * tiles[its >= t].sum() < tiles.sum()]
    assert sum(its[-1] >= t for t in sparse) >= 2
    imgs = [torch.from_numpy(one.image).cuda() for one in sl]
    ids = [torch.from_numpy(one.region_ids).cuda() for one in sl]
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=60)
    out = g.em(cfg, want_T=True)
    g.sync_status()
    _em_compare(sl, ocfg, cfg, g, out)
    g.set_tuning(use_cuda_graph=0)
    od = g.em(cfg, want_T=True)
    g.sync_status()
    for k in ("labels", "params", "iters", "converged", "T_hist"):
        assert torch.equal(out[k], od[k]), k


@pytest.mark.parametrize("L,beta", [(2, 1.0), (3, 1.5), (2, 0.0)])
def test_em_batch_uneven_matches_oracle(L, beta):
    pmrf = _pmrf()
    specs = small_specs(6, seed0=100 + L)
    if L == 3:
        specs = [synth.scaled(synth.workload("large8192").slices[0], sp.height, sp.width, seed=sp.seed)
                 for sp in specs]
    sl = synth.make_stack(specs)
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=L, beta=beta, max_iters=30)
    out = g.em(cfg)
    _em_compare(sl, oracle.EMConfig(n_labels=L, beta=beta, max_iters=30), cfg, g, out)


def test_batched_equals_per_slice():
    """Slices in one batch give exactly what each gives alone."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(5, seed0=300))
    imgs, ids = dev_tensors(sl)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=25)
    gb = pmrf.build_graph(imgs, ids)
    ob = gb.em(cfg)
    xb = ob["labels"].cpu().numpy()
    vo = gb.array("VERT_OFF").numpy()
    for s in range(len(sl)):
        g1 = pmrf.build_graph(imgs[s], ids[s])
        o1 = g1.em(cfg)
        assert np.array_equal(o1["labels"].cpu().numpy(), xb[vo[s]:vo[s + 1]])
        assert int(o1["iters"][0]) == int(ob["iters"][s])
        assert torch.equal(o1["params"][0], ob["params"][s])


def test_em_resume_from_labels():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(2, seed0=500))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=40)
    full = g.em(cfg)
    # stopping early then resuming from the labels reaches the same fixed point
    part = g.em(pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=3))
    res = g.em(cfg, labels=part["labels"].clone())
    assert torch.equal(res["labels"], full["labels"])


def test_label_image_matches_oracle():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(3, seed0=900))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(pmrf.EMConfig())
    seg = g.label_image(ids, out["labels"]).cpu().numpy()
    arrs = gpu_arrays(g)
    x = out["labels"].cpu().numpy()
    o = 0
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        a, b = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        want = og.label_image(one.region_ids, x[a:b]).ravel()
        assert np.array_equal(seg[o:o + want.size], want)
        o += want.size


# --------------------------------------------------------------------------
# pseudo-log-likelihood and its adjoint

def test_pll_and_adjoint_match_oracle():
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(3, seed0=1200))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    L = 2
    out = g.em(pmrf.EMConfig(n_labels=L))
    mu = out["params"][:, :, 1].contiguous()
    sg = out["params"][:, :, 2].contiguous()
    beta = 0.7
    pll = g.pll(L, out["labels"], mu, sg, beta).cpu().numpy()
    gout = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    gmu, gsg, gb = g.pll_grad(L, out["labels"], mu, sg, beta, gout)
    x = out["labels"].cpu().numpy()
    arrs = gpu_arrays(g)
    gbeta = 0.0
    for s, one in enumerate(sl):
        og = oracle.Graph.from_image(one.image, one.region_ids)
        a, b = arrs["VERT_OFF"][s], arrs["VERT_OFF"][s + 1]
        f, om, osg, ob = og.pll(L, x[a:b], mu[s].cpu().numpy(), sg[s].cpu().numpy(), beta)
        assert rel_close(pll[s], f, 1e-12, 1e-9)
        go = float(gout[s])
        assert rel_close(gmu[s].cpu().numpy(), go * om, 1e-10, 1e-8)
        assert rel_close(gsg[s].cpu().numpy(), go * osg, 1e-10, 1e-8)
        gbeta += go * ob
    assert rel_close(float(gb[0]), gbeta, 1e-10, 1e-8)


def test_pll_autograd_vs_central_differences():
    pmrf = _pmrf()
    from paper_1809_05018_b300.autograd import fit_beta
    sl = synth.make_stack(small_specs(2, seed0=1300))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(pmrf.EMConfig())
    mu = out["params"][:, :, 1].clone().requires_grad_(True)
    sg = out["params"][:, :, 2].clone().requires_grad_(True)
    beta = torch.tensor(0.6, dtype=torch.float64, device="cuda", requires_grad=True)
    lab = out["labels"]
    f = pmrf.PLL.apply(mu, sg, beta, g, lab).sum()
    f.backward()
    h = 1e-6

    def F(m, s, b):
        return float(pmrf.PLL.apply(m, s, b, g, lab).sum())

    with torch.no_grad():
        for (i, j) in [(0, 0), (1, 1)]:
            e = torch.zeros_like(mu)
            e[i, j] = h
            fd = (F(mu + e, sg, beta) - F(mu - e, sg, beta)) / (2 * h)
            assert abs(fd - float(mu.grad[i, j])) <= 1e-5 * max(1.0, abs(fd))
            fd = (F(mu, sg + e, beta) - F(mu, sg - e, beta)) / (2 * h)
            assert abs(fd - float(sg.grad[i, j])) <= 1e-5 * max(1.0, abs(fd))
        fd = (F(mu, sg, beta + h) - F(mu, sg, beta - h)) / (2 * h)
        assert abs(fd - float(beta.grad)) <= 1e-5 * max(1.0, abs(fd))
    traj = fit_beta(g, lab, mu.detach(), sg.detach(), beta0=0.2, steps=30)
    assert len(traj) == 31 and all(b >= 0 for b in traj)


def test_large_regions_match_oracle():
    """Regions of ~600-2000 pixels: pixel lists take the shared-memory sort,
    candidate-neighbour lists the widest warp sort."""
    pmrf = _pmrf()
    base = synth.workload("slice256").slices[0]
    specs = [synth.replace(synth.scaled(base, 160, 200, seed=77), pitch_min=26.0, pitch_max=45.0, jitter=8.0),
             synth.replace(synth.scaled(base, 96, 300, seed=78), pitch_min=40.0, pitch_max=40.0, jitter=3.0)]
    sl = synth.make_stack(specs)
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    arrs = gpu_arrays(g)
    npix = arrs["NPIX"]
    assert npix.max() > 256  # the shared-memory path ran
    for s, one in enumerate(sl):
        assert_graph_equal(oracle.Graph.from_image(one.image, one.region_ids), slice_view(arrs, s))
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=20)
    _em_compare(sl, oracle.EMConfig(n_labels=2, beta=1.0, max_iters=20), cfg, g, g.em(cfg))


def _carved_ids(h, w, bs, rng):
    """Square blocks of side bs, each with a notch given to the block on its
    right (that region gets a detached island, the block a C shape: rows with
    pixels of another region between their first and last pixel), plus a few
    tall thin strips (boxes taller than the scan keeps spans for) and scattered
    single pixels of the block above."""
    r, c = np.mgrid[0:h, 0:w]
    nbw = (w + bs - 1) // bs
    ids = (r // bs) * nbw + (c // bs)
    br, bc = r % bs, c % bs
    notch = (br >= 2) & (br < bs - 2) & (bc >= bs // 2 - 1) & (bc < bs // 2 + 1) & (c // bs < nbw - 1)
    ids = np.where(notch, ids + 1, ids)
    # thin vertical strips, each a region of its own
    nb = int(ids.max()) + 1
    for k, col in enumerate(range(bs // 2, w - 1, 3 * bs)):
        ids[1:h - 1, col] = nb + k
    # single pixels carrying the id of the block above
    pts = rng.integers(0, h * w, size=h * w // 97)
    rr, cc = pts // w, pts % w
    ok = rr >= bs
    ids[rr[ok], cc[ok]] = ids[rr[ok] - bs, cc[ok]]
    return ids.astype(np.int32)


def test_nonconvex_regions_match_oracle():
    """Regions whose rows hold other regions' pixels between their first and
    last pixel (C shapes, detached islands, scattered pixels) and boxes taller
    than the scan's span table: means bit-identical, graph exact."""
    pmrf = _pmrf()
    rng = np.random.default_rng(2024)
    shapes = [(64, 64, 8), (96, 80, 12), (70, 45, 9), (48, 128, 20)]
    sl = []
    for h, w, bs in shapes:
        ids = _carved_ids(h, w, bs, rng)
        img = rng.normal(0.5, 0.2, size=(h, w))
        sl.append(type("S", (), dict(image=img, region_ids=ids)))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    arrs = gpu_arrays(g)
    for s, one in enumerate(sl):
        assert_graph_equal(oracle.Graph.from_image(one.image, one.region_ids), slice_view(arrs, s))


def test_em_conditional_graph_equals_unrolled():
    """The captured EM loop whose iterations sit in conditional graph nodes
    gives exactly what the unrolled capture (profiling mode) and the direct
    launches give, runs the same kernels as the unrolled loop cut at the last
    active iteration plus one condition setter per run iteration, one after the
    initial pass and one between the dense and the sparse loop, and a repeated
    replay gives the same outputs."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(7, seed0=500))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    cfg = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=60)

    def run(c, **tuning):
        g.set_tuning(**tuning)
        g.em(c, want_T=True)  # capture
        torch.cuda.synchronize()
        n0 = pmrf.launch_count()
        out = g.em(c, want_T=True)
        torch.cuda.synchronize()
        return out, pmrf.launch_count() - n0

    oc, nc = run(cfg)
    ou, _ = run(cfg, profile=1)
    od, _ = run(cfg, use_cuda_graph=0)
    oc2, nc2 = run(cfg)
    T = int(oc["iters"].max())
    assert 1 <= T < cfg.max_iters
    for o in (ou, od, oc2):
        for k in ("labels", "params", "iters", "converged", "T_hist"):
            assert torch.equal(oc[k], o[k]), k
    assert nc == nc2
    cut = pmrf.EMConfig(n_labels=2, beta=1.0, max_iters=T)
    _, nu = run(cut, profile=1)
    assert nc == nu + T + 2


def test_pll_value_and_grad_equals_separate_calls():
    """The fused value-and-adjoint call gives bit for bit what pll() and
    pll_grad() give."""
    pmrf = _pmrf()
    sl = synth.make_stack(small_specs(4, seed0=990))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    for L in (2, 3):
        out = g.em(pmrf.EMConfig(n_labels=L, beta=1.0, max_iters=15))
        mu = out["params"][:, :, 1].contiguous()
        sg = out["params"][:, :, 2].contiguous()
        gout = torch.linspace(0.5, 2.0, g.S, dtype=torch.float64, device="cuda")
        p1 = g.pll(L, out["labels"], mu, sg, 0.8)
        gm1, gs1, gb1 = g.pll_grad(L, out["labels"], mu, sg, 0.8, gout)
        p2, gm2, gs2, gb2 = g.pll_value_and_grad(L, out["labels"], mu, sg, 0.8, gout)
        for a, b in ((p1, p2), (gm1, gm2), (gs1, gs2), (gb1, gb2)):
            assert torch.equal(a, b)
