"""pmrf_pll_grad_noalloc: the adjoint for callers that cannot allocate device
memory when they need it -- an application whose device memory is already
claimed by its own caching allocator, or a latency-critical loop that must not
pay for (or be synchronised by) an allocation.  Its scratch is a fixed array
inside the library instead of a per-call allocation.  Called through the C ABI,
it must give what pmrf_pll_grad gives, and what the oracle's gradient gives, on
two calls in a row (the second call reuses the array the first one wrote); a
request larger than the fixed array is refused with PMRF_ERR_UNSUPPORTED.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from pmrf_testutil import dev_tensors, rel_close, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PMRF_ERR_UNSUPPORTED = 6
NOALLOC_MAX_DOUBLES = 1 << 20


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(lib, fn, g, L, labels, mu, sg, beta, gout):
    S = g.S
    gmu = torch.full((S, L), float("nan"), dtype=torch.float64, device="cuda")
    gsg = torch.full((S, L), float("nan"), dtype=torch.float64, device="cuda")
    gb = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(g._handle(), L, _p(labels), _p(mu), _p(sg), float(beta), _p(gout), _p(gmu), _p(gsg),
                          _p(gb), stream)
    torch.cuda.synchronize()
    return rc, (gmu.cpu().numpy(), gsg.cpu().numpy(), float(gb[0]))


def _grads(lib, fn, *a):
    rc, out = _call(lib, fn, *a)
    assert rc == 0, (fn, rc, lib.pmrf_last_error())
    return out


def test_noalloc_adjoint_matches_pmrf_pll_grad_and_the_oracle_twice():
    import paper_1809_05018_b300 as pmrf
    from paper_1809_05018_b300 import _native

    lib = _native.load()
    sl = synth.make_stack(small_specs(4, seed0=2400))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(pmrf.EMConfig(n_labels=2))
    labels = out["labels"]
    mu = out["params"][:, :, 1].contiguous()
    sg = out["params"][:, :, 2].contiguous()
    vo = g.array("VERT_OFF").numpy()
    xs = labels.cpu().numpy()
    ogs = [oracle.Graph.from_image(s.image, s.region_ids) for s in sl]
    cases = [(0.7, torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")),
             (1.3, torch.tensor([0.25, 1.0, -1.0, 2.0], dtype=torch.float64, device="cuda"))]
    for beta, gout in cases:  # two calls in a row on the shared scratch array
        want = _grads(lib, "pmrf_pll_grad", g, 2, labels, mu, sg, beta, gout)
        got = _grads(lib, "pmrf_pll_grad_noalloc", g, 2, labels, mu, sg, beta, gout)
        for w, h in zip(want, got):
            assert np.all(np.isfinite(h))
            assert rel_close(h, w, 1e-10, 1e-8)
        # the oracle's gradient of each slice, weighted by gout
        go = gout.cpu().numpy()
        ob = 0.0
        for s, og in enumerate(ogs):
            _, om, osg, b = og.pll(2, xs[vo[s]:vo[s + 1]], mu[s].cpu().numpy(), sg[s].cpu().numpy(), beta)
            assert rel_close(got[0][s], go[s] * om, 1e-10, 1e-8)
            assert rel_close(got[1][s], go[s] * osg, 1e-10, 1e-8)
            ob += go[s] * b
        assert rel_close(got[2], ob, 1e-10, 1e-8)


def test_noalloc_refuses_a_request_above_its_fixed_array():
    # one slice of about 65k regions makes every slice take ceil(V_max / 256)
    # partial records of 2 L + 2 doubles; with L = 8 and 240 slices the request
    # exceeds the fixed array, and the call fails before enqueueing any work
    import paper_1809_05018_b300 as pmrf
    from paper_1809_05018_b300 import _native

    lib = _native.load()
    big = synth.scaled(synth.workload("stack512").slices[0], 1024, 1024, seed=7)
    big = synth.replace(big, pitch_min=4.0, pitch_max=4.0)
    tiny = small_specs(1, seed0=2500, sizes=((8, 8),))[0]
    sl = synth.make_stack([big] + [synth.replace(tiny, seed=2500 + k) for k in range(239)])
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    vo = g.array("VERT_OFF").numpy()
    L = 8
    nchunk = -(-int(np.diff(vo).max()) // 256)
    need = g.S * nchunk * (2 * L + 2) + g.S
    assert need > NOALLOC_MAX_DOUBLES
    labels = torch.zeros(g.V, dtype=torch.uint8, device="cuda")
    mu = torch.linspace(0.1, 0.9, L, dtype=torch.float64, device="cuda").repeat(g.S, 1).contiguous()
    sg = torch.full((g.S, L), 0.2, dtype=torch.float64, device="cuda")
    gout = torch.ones(g.S, dtype=torch.float64, device="cuda")
    rc, out = _call(lib, "pmrf_pll_grad_noalloc", g, L, labels, mu, sg, 1.0, gout)
    assert rc == PMRF_ERR_UNSUPPORTED
    msg = lib.pmrf_last_error()
    msg = msg.decode() if isinstance(msg, bytes) else str(msg)
    assert str(need) in msg and str(NOALLOC_MAX_DOUBLES) in msg
    assert np.isnan(out[0]).all() and np.isnan(out[1]).all() and np.isnan(out[2])  # nothing written
    # the allocating adjoint serves the same request
    assert _call(lib, "pmrf_pll_grad", g, L, labels, mu, sg, 1.0, gout)[0] == 0
