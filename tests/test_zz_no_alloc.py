"""The no-allocation read-back entry point, for callers that cannot allocate
device memory while networks run (a serving loop whose HBM budget is fully
committed, code that must not synchronize the device through cudaMalloc /
cudaFree while other streams step other networks).

It must return exactly what the allocating snn_read_synapses returns, call
after call (the staging array is shared and keeps the previous call's
contents), and refuse ranges larger than its fixed staging array.  This file
is collected last so that a stop at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _read(lib, fn, h, first, count):
    n = ctypes.c_size_t(0)
    rc = fn(h, first, count, None, None, None, None, 0, ctypes.byref(n))
    assert rc in (0, -6)
    m = n.value
    tgt = np.empty(max(m, 1), np.int32)
    dl = np.empty(max(m, 1), np.uint8)
    w = np.empty(max(m, 1), np.int32)
    sd = np.empty(max(m, 1), np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = fn(h, first, count, p(tgt), p(dl), p(w), p(sd), m, ctypes.byref(n))
    assert rc == 0, lib.snn_last_error()
    return tgt[:m], dl[:m], w[:m], sd[:m]


def test_noalloc_read_matches_allocating_read_on_consecutive_calls():
    import paper_1310_8478_gb300 as eng
    from paper_1310_8478_gb300 import snn
    eng.build_engine()
    lib = snn.load()
    cfg = workloads.custom(grid_x=3, grid_y=2, fanout=300, pct_ring=(40, 30, 20, 10), seed=71)
    with eng.Network(cfg, raster_capacity=1 << 20) as net:
        net.run(1050)                       # crosses a long-term update; LTP owed at the end
        # two calls in a row on different ranges, then the first range again
        for first, count in [(0, 1250), (2000, 1700), (0, 1250)]:
            ref = _read(lib, lib.snn_read_synapses, net.h, first, count)
            got = _read(lib, lib.snn_read_synapses_noalloc, net.h, first, count)
            assert len(got[0]) == count * 300
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
        assert np.any(ref[3] != 0)          # the derivatives moved: a real comparison
        # a range above the staging size is refused, nothing is written
        big = snn.SNN_NOALLOC_MAX_SYNAPSES // 300 + 1
        n = ctypes.c_size_t(0)
        out = np.zeros(big * 300, np.int32)
        rc = lib.snn_read_synapses_noalloc(net.h, 0, big, None, None, out.ctypes.data_as(ctypes.c_void_p), None,
                                           out.size, ctypes.byref(n))
        assert rc == -1 and b"split" in lib.snn_last_error()
        assert n.value == big * 300 and not out.any()


def test_noalloc_read_of_an_explicit_net_and_a_range_at_the_limit():
    import paper_1310_8478_gb300 as eng
    from paper_1310_8478_gb300 import snn
    eng.build_engine()
    lib = snn.load()
    # explicit synapse lists with uneven rows (the row offsets are looked up
    # on the device and every synapse keeps its own delay)
    rng = np.random.default_rng(5)
    cfg = workloads.custom(grid_x=2, grid_y=1, fanout=1, seed=73)
    N = 2 * 1250
    lens = rng.integers(0, 40, N)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    S = int(row_off[-1])
    tgt = rng.integers(0, N, S).astype(np.int32)
    src = np.repeat(np.arange(N), lens)
    tgt[tgt == src] = (tgt[tgt == src] + 1) % N
    dly = np.where((src % 1250) < 1000, rng.integers(1, 21, S), 1).astype(np.uint8)
    w = np.where((src % 1250) < 1000, 6 * 65536, -5 * 65536).astype(np.int32)
    with eng.Network(cfg, explicit=dict(row_off=row_off, tgt=tgt, delay=dly, w=w), raster_capacity=1 << 20) as net:
        net.run(1020)
        for first, count in [(3, 700), (1200, 1300), (3, 700)]:
            ref = _read(lib, lib.snn_read_synapses, net.h, first, count)
            got = _read(lib, lib.snn_read_synapses_noalloc, net.h, first, count)
            assert len(got[0]) == row_off[first + count] - row_off[first]
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
    # a range of exactly SNN_NOALLOC_MAX_SYNAPSES synapses is accepted
    M = 1024
    cfg = workloads.custom(grid_x=1, grid_y=1, fanout=M, seed=74)
    rows = snn.SNN_NOALLOC_MAX_SYNAPSES // M
    with eng.Network(cfg, raster_capacity=1 << 20) as net:
        net.run(30)
        ref = _read(lib, lib.snn_read_synapses, net.h, 0, rows)
        got = _read(lib, lib.snn_read_synapses_noalloc, net.h, 0, rows)
        assert len(got[0]) == snn.SNN_NOALLOC_MAX_SYNAPSES
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
