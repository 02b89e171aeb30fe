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
