"""Host logic of the serving loop (admission under the device budget, FIFO
order, chunked advance, batch re-formation, release on completion), driven
by a fake engine on the CPU: no GPU, no device memory.  The GPU test
test_gpu_serve.py checks the same loop on the real engine."""
import types

import numpy as np
import pytest

import workloads
from paper_1310_8478_gb300 import serve

ENOMEM = -2


class FakeError(Exception):
    def __init__(self, code):
        super().__init__(code)
        self.code = code


class FakeNet:
    """A net whose device size is its neuron count times a fixed factor."""
    live = []

    def __init__(self, cfg, stream=None, hbm_budget_bytes=0, raster_capacity=0):
        n = cfg["grid_x"] * cfg["grid_y"] * cfg["neurons_per_col"]
        self.device_bytes = n * 1000
        if self.device_bytes > hbm_budget_bytes:
            raise FakeError(ENOMEM)
        self.t = 0
        self.n = n
        self.closed = False
        FakeNet.live.append(self)

    def counters(self):
        return {"t": self.t, "spikes": self.t * 2, "e_all": self.t * self.n}

    def run(self, n_ms):
        self.t += n_ms

    def raster(self):
        return np.arange(self.t), np.zeros(self.t)

    def weights(self):
        return np.zeros(1), np.zeros(1)

    def close(self):
        assert not self.closed
        self.closed = True
        FakeNet.live.remove(self)


class FakeBatch:
    formed = []

    def __init__(self, nets, graph_steps=10):
        self.nets = list(nets)
        self.closed = False
        FakeBatch.formed.append(len(self.nets))

    def run(self, steps):
        assert not self.closed and steps > 0
        for n in self.nets:
            assert not n.closed
            n.t += steps

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    eng = types.SimpleNamespace(Network=FakeNet, Batch=FakeBatch, SnnError=FakeError, ENOMEM=ENOMEM)
    monkeypatch.setattr(serve, "snn", eng)
    FakeNet.live.clear()
    FakeBatch.formed.clear()
    return eng


class Clock:
    """Simulated time: each call advances it by a fixed tick."""

    def __init__(self, tick=0.001):
        self.now, self.tick = 0.0, tick

    def __call__(self):
        self.now += self.tick
        return self.now

    def sleep(self, dt):
        self.now += dt


def _req(i, side, ms, arrival):
    cfg = workloads.custom(grid_x=side, grid_y=side, neurons_per_col=10, exc_per_col=8, fanout=5, seed=i)
    return serve.Request(i, cfg, ms, arrival)


def test_every_request_completes_with_its_own_duration(fake):
    reqs = [_req(i, 1 + i % 3, 30 + 7 * i, 0.01 * i) for i in range(12)]
    clock = Clock()
    res = serve.Server(budget_bytes=10**9, chunk_ms=10).serve(reqs, clock=clock, sleep=clock.sleep)
    assert sorted(r.rid for r in res) == list(range(12))
    for r in res:
        req = reqs[r.rid]
        assert r.steps == req.duration_ms                 # no step more or less than asked
        assert r.events == req.duration_ms * req.cfg["grid_x"] ** 2 * 10
        assert r.admitted_s >= req.arrival_s and r.done_s >= r.admitted_s
    assert not FakeNet.live                                # every net released


def test_admission_respects_the_budget_and_fifo_order(fake):
    # each net holds 90 kB (3x3 columns of 10 neurons); the budget fits two
    reqs = [_req(i, 3, 50, 0.0) for i in range(5)]
    clock = Clock()
    srv = serve.Server(budget_bytes=200_000, chunk_ms=10)
    peak = []
    orig_run = FakeBatch.run

    def run(self, steps):
        peak.append(sum(n.device_bytes for n in FakeNet.live))
        orig_run(self, steps)
    FakeBatch.run = run
    try:
        res = srv.serve(reqs, clock=clock, sleep=clock.sleep)
    finally:
        FakeBatch.run = orig_run
    assert max(peak) <= 200_000 and max(FakeBatch.formed) == 2
    order = [r.rid for r in sorted(res, key=lambda r: (r.admitted_s, r.rid))]
    assert order == sorted(order)                          # admitted in arrival order
    assert srv.used == 0 and not FakeNet.live


def test_a_request_larger_than_the_budget_is_reported(fake):
    clock = Clock()
    with pytest.raises(RuntimeError):
        serve.Server(budget_bytes=1000, chunk_ms=10).serve([_req(0, 4, 20, 0.0)], clock=clock, sleep=clock.sleep)


def test_late_arrivals_join_at_chunk_boundaries(fake):
    # a long request and a short one arriving later: the batch is re-formed
    # when the short one joins and when it leaves
    reqs = [_req(0, 2, 200, 0.0), _req(1, 1, 20, 0.05)]
    clock = Clock(tick=0.01)
    srv = serve.Server(budget_bytes=10**9, chunk_ms=10)
    res = {r.rid: r for r in srv.serve(reqs, clock=clock, sleep=clock.sleep)}
    assert res[0].steps == 200 and res[1].steps == 20
    assert res[1].admitted_s >= 0.05 and res[1].done_s < res[0].done_s
    assert FakeBatch.formed[:3] == [1, 2, 1] and srv.rebatches >= 3


def test_poisson_requests_are_reproducible():
    a = serve.poisson_requests(20, 200.0, lambda i, rng: {"i": i}, lambda i, rng: 100 + i, seed=3)
    b = serve.poisson_requests(20, 200.0, lambda i, rng: {"i": i}, lambda i, rng: 100 + i, seed=3)
    assert [r.arrival_s for r in a] == [r.arrival_s for r in b]
    assert all(x.arrival_s < y.arrival_s for x, y in zip(a, a[1:]))
    st = serve.latency_stats([serve.Result(i, 0.0, 0.0, float(i), 1, 0, 0) for i in range(1, 101)])
    assert st["p50_s"] == pytest.approx(50.5) and st["max_s"] == 100.0
