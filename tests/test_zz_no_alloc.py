"""pmrf_pll_grad_noalloc: the adjoint for callers that cannot allocate device
memory when they need it (for instance while a stream is being captured into a
CUDA graph, or when an application's own allocator holds the device memory).
Its scratch is a fixed array inside the library instead of a per-call
allocation.  Called through the C ABI, it must give what pmrf_pll_grad gives,
on two calls in a row (the second call reuses the array the first one wrote).

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from pmrf_testutil import dev_tensors, rel_close, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _grads(lib, fn, g, L, labels, mu, sg, beta, gout):
    S = g.S
    gmu = torch.full((S, L), float("nan"), dtype=torch.float64, device="cuda")
    gsg = torch.full((S, L), float("nan"), dtype=torch.float64, device="cuda")
    gb = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(g._handle(), L, _p(labels), _p(mu), _p(sg), float(beta), _p(gout), _p(gmu), _p(gsg),
                          _p(gb), stream)
    assert rc == 0, (fn, rc, lib.pmrf_last_error())
    torch.cuda.synchronize()
    return gmu.cpu().numpy(), gsg.cpu().numpy(), float(gb[0])


def test_noalloc_adjoint_matches_pmrf_pll_grad_twice():
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
    cases = [(0.7, torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")),
             (1.3, torch.tensor([0.25, 1.0, -1.0, 2.0], dtype=torch.float64, device="cuda"))]
    for beta, gout in cases:  # two calls in a row on the shared scratch array
        want = _grads(lib, "pmrf_pll_grad", g, 2, labels, mu, sg, beta, gout)
        got = _grads(lib, "pmrf_pll_grad_noalloc", g, 2, labels, mu, sg, beta, gout)
        for w, h in zip(want, got):
            assert np.all(np.isfinite(h))
            assert rel_close(h, w, 1e-10, 1e-8)
