"""The library's device memory pool: a destroyed graph's arrays go back to the
pool (used bytes fall, reserved bytes stay), a rebuild of the same batch reuses
them (reserving little or nothing more), and trimming returns the unused
memory."""
import gc

import pytest

import synth
from pmrf_testutil import dev_tensors, small_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_pool_keeps_and_trims_memory():
    import paper_1809_05018_b300 as pmrf
    gc.collect()  # graphs that earlier tests left in reference cycles go back to the pool first
    sl = synth.make_stack(small_specs(3, seed0=2600))
    imgs, ids = dev_tensors(sl)
    g = pmrf.build_graph(imgs, ids)
    g.em(pmrf.EMConfig(n_labels=2))
    torch.cuda.synchronize()
    r1, u1 = pmrf.memory_usage()
    assert u1 > 0 and r1 >= u1
    del g
    gc.collect()
    r2, u2 = pmrf.memory_usage()
    assert u2 < u1 and r2 >= r1 - (1 << 20)
    g = pmrf.build_graph(imgs, ids)
    out = g.em(pmrf.EMConfig(n_labels=2))
    torch.cuda.synchronize()
    r3, u3 = pmrf.memory_usage()
    assert u3 == u1 and r3 <= r2 + r2 // 4  # same sizes, served mostly from the kept memory
    assert int(out["iters"].min()) >= 1
    del g, out
    gc.collect()
    pmrf.trim_memory(0)
    r4, u4 = pmrf.memory_usage()
    assert u4 == u2 and u4 <= r4 < r3


def test_destroy_orders_release_after_pending_work():
    """pmrf_graph_destroy does not wait on the host: the arrays of a graph
    whose EM run may still be executing on one stream go back to the pool
    after that run, so a graph built at once on another stream (possibly on
    the same memory) cannot disturb it.  Both runs must equal a reference run
    made with nothing else in flight."""
    import paper_1809_05018_b300 as pmrf
    sl = synth.make_stack(small_specs(4, seed0=2700))
    imgs, ids = dev_tensors(sl)
    cfg = pmrf.EMConfig(n_labels=2, max_iters=30)
    g = pmrf.build_graph(imgs, ids)
    ref = g.em(cfg)
    torch.cuda.synchronize()
    ref_lab, ref_par = ref["labels"].cpu(), ref["params"].cpu()
    del g
    gc.collect()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(sa):
            ga = pmrf.build_graph(imgs, ids)
            out_a = ga.em(cfg)
        del ga  # released without a host wait; sa's EM run may still be executing
        gc.collect()
        with torch.cuda.stream(sb):
            gb = pmrf.build_graph(imgs, ids)
            out_b = gb.em(cfg)
        torch.cuda.synchronize()
        for out in (out_a, out_b):
            assert torch.equal(out["labels"].cpu(), ref_lab)
            assert torch.equal(out["params"].cpu(), ref_par)
        del gb
        gc.collect()
    r, u = pmrf.memory_usage()
    assert 0 <= u <= r
