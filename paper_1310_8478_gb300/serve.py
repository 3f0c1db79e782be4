"""Continuous batching of simulation requests on one GPU.

A request is one network (a parameter dictionary, its seed included) and a
duration in simulated milliseconds.  Requests enter a FIFO queue at their
arrival time; the server admits the head of the queue as soon as the network
fits the device budget (the engine checks the footprint before allocating),
keeps every admitted network resident, and advances all of them together in
chunks of `chunk_ms` steps through one batch (one CUDA graph per chunk, each
network a parallel branch).  The batch is re-formed whenever a request joins
or finishes, so requests that arrive while others run start at the next chunk
boundary and their work overlaps on the device.  A finished request releases
its memory at once.  Networks keep their own clocks: a request's results are
identical whether it runs alone or in a mix.

Everything on the device is the engine's (include/snn.h); this module only
orders the calls.
"""
from __future__ import annotations

import collections
import dataclasses
import hashlib
import time

import numpy as np

from . import snn


@dataclasses.dataclass
class Request:
    rid: int
    cfg: dict
    duration_ms: int
    arrival_s: float = 0.0
    keep_raster: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    done_s: float
    steps: int
    spikes: int
    events: int
    raster_digest: str | None = None
    weights_digest: str | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


class Server:
    def __init__(self, budget_bytes: int, chunk_ms: int = 10, stream=None, digests: bool = False):
        self.budget = int(budget_bytes)
        self.chunk = max(1, int(chunk_ms))
        self.stream = stream
        self.digests = digests
        self.used = 0
        self.active = collections.OrderedDict()     # rid -> [net, request, remaining, admitted_s]
        self.batch = None
        self.results: list[Result] = []
        self.chunks = 0
        self.rebatches = 0

    # -- admission -------------------------------------------------------
    def _try_admit(self, req: Request, now: float) -> bool:
        left = self.budget - self.used
        if left <= 0:
            return False
        n_neurons = req.cfg["grid_x"] * req.cfg["grid_y"] * req.cfg["neurons_per_col"]
        cap = n_neurons * (req.duration_ms + 2) if req.keep_raster else 0
        try:
            net = snn.Network(req.cfg, stream=self.stream, hbm_budget_bytes=left, raster_capacity=cap)
        except snn.SnnError as e:
            if e.code == snn.ENOMEM:
                return False
            raise
        self.used += net.device_bytes
        self.active[req.rid] = [net, req, req.duration_ms, now]
        self._drop_batch()
        return True

    def _drop_batch(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None

    def _finish(self, rid: int, now: float):
        net, req, _, admitted = self.active.pop(rid)
        c = net.counters()
        rd = wd = None
        if self.digests:
            if req.keep_raster:
                rd = digest(*net.raster())
            wd = digest(*net.weights())
        self.results.append(Result(rid, req.arrival_s, admitted, now, c["t"], c["spikes"], c["e_all"], rd, wd))
        self._drop_batch()                  # the batch goes before the nets it holds
        self.used -= net.device_bytes
        net.close()

    # -- the loop ----------------------------------------------------------
    def serve(self, requests, clock=time.perf_counter, sleep=time.sleep) -> list[Result]:
        """Run `requests` (arrival_s relative to the start) to completion."""
        queue = collections.deque(sorted(requests, key=lambda r: (r.arrival_s, r.rid)))
        t0 = clock()
        while queue or self.active:
            now = clock() - t0
            while queue and queue[0].arrival_s <= now:
                if not self._try_admit(queue[0], now):
                    break
                queue.popleft()
            if not self.active:
                if queue and queue[0].arrival_s > now:
                    sleep(min(0.05, queue[0].arrival_s - now))
                    continue
                if queue:      # the head does not fit even on an empty device
                    raise RuntimeError("request %d does not fit the budget" % queue[0].rid)
                break
            step = min(self.chunk, min(a[2] for a in self.active.values()))
            if self.batch is None:
                self.batch = snn.Batch([a[0] for a in self.active.values()],
                                       graph_steps=self.chunk if self.chunk % 2 == 0 else 10)
                self.rebatches += 1
            self.batch.run(step)
            self.chunks += 1
            now = clock() - t0
            for rid in [rid for rid, a in self.active.items() if a[2] - step <= 0]:
                self.active[rid][2] = 0
                self._finish(rid, now)
            for a in self.active.values():
                a[2] -= step
        self._drop_batch()
        return self.results


def poisson_requests(n: int, rate_per_s: float, cfg_of, duration_of, seed: int = 5) -> list[Request]:
    """n requests with exponential inter-arrival times of mean 1 / rate; the
    i-th request's parameters come from cfg_of(i, rng) and duration_of(i, rng)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        out.append(Request(i, cfg_of(i, rng), int(duration_of(i, rng)), t))
    return out


def latency_stats(results) -> dict:
    lat = np.array([r.latency_s for r in results]) if results else np.zeros(1)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
