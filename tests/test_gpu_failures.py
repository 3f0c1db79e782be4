"""Failure handling without faulting the GPU: every failure is made on the
host (an allocator that refuses a block or returns a misaligned one) and
must come back as an error code with everything released."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

CFG = workloads.custom(grid_x=2, grid_y=2, fanout=60, pct_ring=(40, 30, 20, 10), seed=71)


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


class Counting:
    """Wraps torch's caching allocator; fails the fail_at-th request (1-based)."""

    def __init__(self, fail_at=0, offset=0):
        from paper_1310_8478_gb300 import snn
        self.alloc0, self.free0 = snn.torch_allocator()
        self.fail_at, self.offset = fail_at, offset
        self.calls, self.live = 0, {}

    def alloc(self, n, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            return 0
        p = self.alloc0(n + self.offset, stream)
        self.live[p + self.offset] = p
        return p + self.offset

    def free(self, ptr):
        self.free0(self.live.pop(ptr))


def _run(eng, steps=300):
    with eng.Network(CFG, raster_capacity=1 << 20) as n:
        n.run(steps)
        t, g = n.raster()
        w, sd = n.weights()
    return t, g, w, sd


def test_torch_allocator_gives_the_same_run_and_returns_its_memory(eng):
    import torch
    from paper_1310_8478_gb300 import snn
    ref = _run(eng)
    a = Counting()
    base = torch.cuda.memory_allocated()
    snn.set_allocator(a.alloc, a.free)
    try:
        got = _run(eng)
    finally:
        snn.set_allocator(None)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    assert a.calls > 5 and not a.live
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("fail_at", [1, 3, 7, 12])
def test_a_refused_allocation_fails_the_build_and_releases_everything(eng, fail_at):
    from paper_1310_8478_gb300 import snn
    a = Counting(fail_at=fail_at)
    snn.set_allocator(a.alloc, a.free)
    try:
        with pytest.raises(snn.SnnError) as e:
            eng.Network(CFG, raster_capacity=1 << 20)
        assert e.value.code == snn.ENOMEM
    finally:
        snn.set_allocator(None)
    assert a.calls >= fail_at and not a.live
    _run(eng, 50)                         # the library stays usable


def test_a_misaligned_block_is_refused(eng):
    from paper_1310_8478_gb300 import snn
    a = Counting(offset=16)
    snn.set_allocator(a.alloc, a.free)
    try:
        with pytest.raises(snn.SnnError) as e:
            eng.Network(CFG, raster_capacity=1 << 20)
        assert e.value.code == snn.ENOMEM and "aligned" in str(e.value)
    finally:
        snn.set_allocator(None)
    assert not a.live
