#!/usr/bin/env python
"""Benchmark of the DPSNN-STDP per-millisecond step on GB300.

A bench step is one 1 ms step of the whole hot path (delivery + LTD, thalamic
drive + neuron update, spike compaction + raster, LTP, and the long-term
plasticity update whenever the step closes a 1000 ms period) on the 64x64
torus workload (5.12 M neurons, 1125 synapses per neuron, 5.76 G synapses).
Warm-up steps run first, untimed; then exactly --steps steps are timed with
CUDA events on the stream the kernels run on.  The value is synaptic events
per second (one event = one spike reaching one synapse).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
instead, on a bounded sample of the same column model.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

DEFAULT_WORKLOAD = "grid64_m1125"
# the oracle's bounded sample: the same column model, fan-out and projection
# mix on the 16x16 torus (the 64x64 net does not fit a bounded CPU sample),
# over the same simulated steps as the GPU's timed region, single core
CPU_SAMPLE_WORKLOAD = "grid16_m1125"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=None, help="steps of the end-to-end leg (default: --steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the oracle sample")
    ap.add_argument("--ref-budget-s", type=float, default=150.0, help="wall bound of the reference arm")
    ap.add_argument("--no-small", action="store_true", help="skip the 1-column latency line")
    ap.add_argument("--batch-bench", type=int, default=0, metavar="NETS",
                    help="instead: the uneven batched workload (first NETS of 256 nets), batched vs one at a time")
    ap.add_argument("--batch-budget-gb", type=float, default=150.0, help="device budget of one wave of nets")
    ap.add_argument("--batch-steps", type=int, default=100, help="steps of each net in the batch leg")
    ap.add_argument("--batch-nets", type=int, default=256, help="nets of the batch leg of the default line (0: none)")
    ap.add_argument("--batch-autotune-ms", type=int, default=0,
                    help="probe steps of the batch autotuner before the timed batch (0: default shape)")
    ap.add_argument("--serve-bench", type=int, default=0, metavar="REQUESTS",
                    help="instead: the serving workload (Poisson arrivals) with this many requests")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--no-atomics", dest="atomics", action="store_false",
                    help="skip the L2-reduction / gather / shared-atomic microbenchmark")
    ap.add_argument("--no-steady", dest="steady", action="store_false",
                    help="skip the dense-regime and period-end legs after the timed region")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the serving leg of the default line (0: no serving leg)")
    return ap.parse_args()


def combine_ranks(ms: float, events: float, dist=None, device="cpu"):
    """Whole-job figures of a replicas run: the slowest rank's time and the
    sum of every rank's synaptic events."""
    if dist is None:
        return ms, events
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(events)], dtype=torch.float64, device=device)
    dist.all_reduce(e)
    return float(t.item()), float(e.item())


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ---------------------------------------------------------------------------
# the oracle's bounded sample (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(seconds: float, t0: int, t1: int):
    """The oracle on the CPU sample workload, timed over steps [t0, t1) (the
    GPU leg's window) or until `seconds` have passed, whichever comes first;
    construction and the steps before t0 are not timed."""
    import oracle
    cfg = workloads.workload(CPU_SAMPLE_WORKLOAD)
    sim = oracle.Oracle(cfg)
    sim.run(t0)
    c0 = sim.counters()
    t_start = time.perf_counter()
    steps = 0
    while t0 + steps < t1:
        sim.run(1)
        steps += 1
        if time.perf_counter() - t_start >= seconds:
            break
    el = time.perf_counter() - t_start
    c1 = sim.counters()
    ev = c1["e_all"] - c0["e_all"]
    sample = ("oracle on the %dx%d torus (%s: same column model, fan-out and mix), steps %d..%d of its run "
              "(the GPU leg's timed steps), 1 thread" % (
                  cfg["grid_x"], cfg["grid_y"], CPU_SAMPLE_WORKLOAD, t0, t0 + steps - 1))
    return dict(value=ev / el, unit="events/s", cores=1, kind="oracle", sample=sample,
                steps=steps, seconds=el, events=ev)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    r = oracle_sample(args.ref_budget_s, args.warmup, args.warmup + args.steps)
    cfg = workloads.workload(args.workload)
    line = {
        "impl": "reference", "metric": "synaptic events/s", "value": r["value"], "unit": "events/s",
        "n_gpus": args.gpus, "steps": r["steps"], "warmup": args.warmup,
        "ms_per_step": 1000.0 * r["seconds"] / max(1, r["steps"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32", "data": "synthetic",
        "config": {"workload": args.workload,
                   "stands_in": "%s torus of the same column model, same steps (CPU bound)" % CPU_SAMPLE_WORKLOAD,
                   "grid": [cfg["grid_x"], cfg["grid_y"]], "fanout": cfg["fanout"]},
        "cpu_baseline": {"value": r["value"], "unit": "events/s", "cores": 1, "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": r["value"], "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(period_ms)], stdout=self.f, stderr=subprocess.DEVNULL)
            # the first sample is taken before the timed region starts
            self._wait_lines(1, 5.0)
        except Exception:
            self.proc = None

    def _lines(self) -> int:
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def _wait_lines(self, n: int, timeout_s: float):
        t0 = time.perf_counter()
        while self._lines() < n and time.perf_counter() - t0 < timeout_s and self.proc.poll() is None:
            time.sleep(0.005)

    def stop(self):
        if self.proc is None:
            return None
        # a sample after the timed region too, so that a short region is
        # bracketed by samples on both sides
        self._wait_lines(self._lines() + 1, 2.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_digest(kernel: str = "dense"):
    """sha256 of the sources a step kernel is compiled from (the dense pass
    has its own file; the other step kernels share snn_step.cu)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("snn_dense.cu" if kernel == "dense" else "snn_step.cu", "snn_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1310_8478_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of
    this workload, or None when there is none or the kernel changed since."""
    p = os.path.join(ROOT, "profiles", "k_%s_%s_dram.json" % (kernel, workload))
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != kernel_source_digest(kernel):
        return None
    return d.get("dram_bytes_per_launch")


def deriv_updates(t0: int, t1: int, period: int) -> int:
    """Long-term updates carried out by the launches of steps t0 .. t1 - 1: the
    update that closes step m runs with the launch of step m + 1, so these are
    the multiples of the period in [max(t0, 1), t1)."""
    if period <= 0 or t1 <= t0:
        return 0
    below = (t0 - 1) // period if t0 >= 1 else 0
    return (t1 - 1) // period - below


def algorithmic_bytes(d_events, d_exc, d_ltp, n_neurons, neuron_launches, n_exc_syn, updates, dd):
    """Algorithmic bytes moved by each kernel over the timed region, from the
    per-unit figures: 8 B per delivered event (target + weight), 8 B per event
    on a plastic synapse (sd read + write), 12 B per potentiation visit, 16 B
    per plastic synapse per long-term update, 32 B per neuron per step.  The
    work the dense pass did (dd: its own counts) is charged to it and taken
    out of the event-driven kernels' share."""
    return {
        "deliver": 8.0 * (d_events - dd["dense_events"]) + 8.0 * (d_exc - dd["dense_exc_events"]),
        "ltp": 12.0 * max(0, d_ltp - dd["dense_ltp_visits"]),
        "neuron": 32.0 * n_neurons * neuron_launches,
        "deriv": 16.0 * n_exc_syn * max(0, updates - dd["dense_deriv_steps"]),
        "dense": (8.0 * dd["dense_events"] + 8.0 * dd["dense_exc_events"] + 12.0 * dd["dense_ltp_visits"]
                  + 16.0 * n_exc_syn * dd["dense_deriv_steps"]),
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def batch_leg(n_nets: int, steps: int, budget_gb: float, stream, autotune_ms: int = 0, warm: int = 10):
    """Independent uneven networks (grid side 1..16, M in {100, 400, 1125},
    seeds 1000..): every wave of nets that fits the budget runs twice from
    the initial state, once one net after another (each with its own CUDA
    graphs) and once as one batch (one graph per chunk, one launch per kind
    of kernel per step for all nets): `warm` untimed steps (graph capture),
    then `steps` timed steps; throughput = synaptic events of the timed steps
    / their time (CUDA events around the whole wave, host launch overhead
    included).  Each net's raster digest must be the same both ways."""
    import torch
    import paper_1310_8478_gb300 as eng
    cfgs = workloads.batch_workloads()[:n_nets]
    budget = int(budget_gb * 1e9)
    T = warm + steps
    seq_ms = bat_ms = 0.0
    seq_ev = bat_ev = 0
    waves = 0
    same = True
    shape = None
    ev_a = torch.cuda.Event(enable_timing=True)
    ev_b = torch.cuda.Event(enable_timing=True)
    by_kind = {}

    def kind_of(c):
        side = "side 1-4" if c["grid_x"] <= 4 else ("side 5-10" if c["grid_x"] <= 10 else "side 11-16")
        return "M=%d, %s" % (c["fanout"], side)

    def timed(fn):
        torch.cuda.synchronize()
        ev_a.record(stream)
        fn()
        ev_b.record(stream)
        torch.cuda.synchronize()
        return ev_a.elapsed_time(ev_b)

    i = 0
    while i < len(cfgs):
        wave, used = [], 0
        while i < len(cfgs):
            n = eng.Network(cfgs[i], stream=stream, raster_capacity=workloads.n_neurons(cfgs[i]) * T + 1024)
            if wave and used + n.device_bytes > budget:
                n.close()
                break
            wave.append(n)
            used += n.device_bytes
            i += 1
        waves += 1
        # one at a time
        for n in wave:
            n.run(warm)
        e0 = sum(n.counters()["e_all"] for n in wave)

        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in wave]
        c_before = [n.counters()["e_all"] for n in wave]

        def alone():
            for n, (a, b) in zip(wave, evs):
                a.record(stream)
                n.run(steps)
                b.record(stream)
        seq_ms += timed(alone)
        seq_ev += sum(n.counters()["e_all"] for n in wave) - e0
        for n, (a, b), c0 in zip(wave, evs, c_before):
            kind = kind_of(n.cfg)
            k = by_kind.setdefault(kind, {"nets": 0, "one_at_a_time_ms": 0.0, "events": 0})
            k["nets"] += 1
            k["one_at_a_time_ms"] += a.elapsed_time(b)
            k["events"] += n.counters()["e_all"] - c0
        ref = [raster_digest(n, 0, T) for n in wave]
        for n in wave:
            n.reset()
        # batched
        with eng.Batch(wave, graph_steps=10) as b:
            if autotune_ms and shape is None:
                shape = b.autotune(autotune_ms)
            elif shape is not None:
                b.set_launch(**{k: shape[k] for k in ("deliver_block", "deliver_blocks_per_sm",
                                                      "ltp_blocks_per_sm", "graph_steps")})
            b.run(warm)
            e0 = sum(n.counters()["e_all"] for n in wave)
            bat_ms += timed(lambda: b.run(steps))
        bat_ev += sum(n.counters()["e_all"] for n in wave) - e0
        same = same and all(raster_digest(n, 0, T) == d for n, d in zip(wave, ref))
        for n in wave:
            n.close()
    out = {"workload": "%d independent nets, grid side uniform 1..16, M in {100, 400, 1125}, seeds 1000..%d, "
                       "steps %d..%d of each (after %d untimed), waves under %.0f GB" % (
                           len(cfgs), 999 + len(cfgs), warm, T - 1, warm, budget_gb),
           "nets": len(cfgs), "waves": waves, "steps": steps, "unit": "events/s",
           "value": bat_ev / (bat_ms / 1e3), "batched_ms": round(bat_ms, 3),
           "one_at_a_time": seq_ev / (seq_ms / 1e3), "one_at_a_time_ms": round(seq_ms, 3),
           "speedup": (bat_ev / bat_ms) / (seq_ev / seq_ms), "same_events": seq_ev == bat_ev,
           "raster_digests_equal": same, "events": bat_ev,
           # where the one-at-a-time time goes: batching can only take away
           # the launch-bound share of the small nets
           "one_at_a_time_by_kind": {k: {"nets": v["nets"], "ms": round(v["one_at_a_time_ms"], 3),
                                         "share": round(v["one_at_a_time_ms"] / max(seq_ms, 1e-9), 4),
                                         "events_per_s": v["events"] / max(v["one_at_a_time_ms"] / 1e3, 1e-12)}
                                     for k, v in sorted(by_kind.items())}}
    if shape is not None:
        out["autotuned"] = {k: shape[k] for k in ("deliver_block", "deliver_blocks_per_sm", "graph_steps")}
    return out


def run_batch_bench(args):
    """The batched workload alone (see batch_leg), --batch-bench nets."""
    import torch
    import paper_1310_8478_gb300 as eng
    torch.cuda.set_device(0)
    eng.build_engine()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        leg = batch_leg(args.batch_bench, args.batch_steps, args.batch_budget_gb, stream, args.batch_autotune_ms)
    line = {"metric": "synaptic events/s", "mode": "batch", "n_gpus": 1, "config": {"workload": leg["workload"]}}
    line.update(leg)
    print(json.dumps(line), flush=True)
    return 0


SERVE_WORKLOAD = ("Poisson requests, grid side log-uniform 1..32, M in {100, 400, 1125}, "
                  "duration uniform 100..5000 ms, seeds 5000..")


def serve_leg(n_requests: int, rate: float, budget_gb: float, stream, one_at_a_time: bool = True):
    """Simulation requests arriving as a Poisson stream (mean `rate` per
    second; grid side log-uniform 1..32, M in {100, 400, 1125}, duration
    uniform 100..5000 ms, seeds 5000..) served with continuous batching under
    a device budget of `budget_gb`; latency = completion - arrival."""
    from paper_1310_8478_gb300 import serve
    params = {}

    def cfg_of(i, rng):
        c, d = workloads.serve_request_params(i, rng)
        params[i] = d
        return c

    reqs = serve.poisson_requests(n_requests, rate, cfg_of, lambda i, rng: params[i])
    srv = serve.Server(int(budget_gb * 1e9), chunk_ms=10, stream=stream)
    t0 = time.perf_counter()
    res = srv.serve(reqs)
    wall = time.perf_counter() - t0
    ev = sum(r.events for r in res)
    out = {"requests": len(res), "rate_per_s": rate, "budget_gb": budget_gb,
           "value": ev / wall, "unit": "events/s", "wall_s": wall, "events": ev,
           "latency": serve.latency_stats(res), "chunks": srv.chunks, "rebatches": srv.rebatches,
           "sim_ms_total": int(sum(r.steps for r in res))}
    if one_at_a_time:
        # the same requests, each run alone to completion one after another
        # (no waiting for arrivals), wall time around the whole sequence
        ev1 = 0
        by_kind = {}
        t0 = time.perf_counter()
        for r in reqs:
            tr = time.perf_counter()
            n = serve.snn.Network(r.cfg, stream=stream, hbm_budget_bytes=int(budget_gb * 1e9), raster_capacity=0)
            try:
                n.run(r.duration_ms)
                e = n.counters()["e_all"]
                ev1 += e
            finally:
                n.close()
            side = r.cfg["grid_x"]
            kind = "M=%d, side %s" % (r.cfg["fanout"], "1-8" if side <= 8 else ("9-16" if side <= 16 else "17-32"))
            k = by_kind.setdefault(kind, {"requests": 0, "s": 0.0, "events": 0})
            k["requests"] += 1
            k["s"] += time.perf_counter() - tr
            k["events"] += e
        wall1 = time.perf_counter() - t0
        for k in by_kind.values():
            k["share"] = round(k["s"] / wall1, 4)
            k["events_per_s"] = k["events"] / max(k["s"], 1e-9)
            k["s"] = round(k["s"], 3)
        out["one_at_a_time"] = {"value": ev1 / wall1, "wall_s": wall1, "same_events": ev1 == ev}
        out["one_at_a_time_by_kind"] = dict(sorted(by_kind.items()))
        out["speedup"] = (ev / wall) / (ev1 / wall1)
    return out


def run_serve_bench(args):
    """The serving workload alone (see serve_leg), --serve-bench requests."""
    import torch
    import paper_1310_8478_gb300 as eng
    torch.cuda.set_device(0)
    eng.build_engine()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        leg = serve_leg(args.serve_bench, args.serve_rate, args.batch_budget_gb, stream)
    line = {"metric": "synaptic events/s", "mode": "serve", "n_gpus": 1, "config": {"workload": SERVE_WORKLOAD}}
    line.update(leg)
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_bench:
        return run_batch_bench(args)
    if args.serve_bench:
        return run_serve_bench(args)
    rank, local_rank, world = dist_env()
    import torch
    import paper_1310_8478_gb300 as eng
    from paper_1310_8478_gb300 import snn

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # before any GPU work; same process, no fork
        cpu = oracle_sample(args.cpu_seconds, args.warmup, args.warmup + args.steps)

    # rank 0 compiles whatever is stale; the other ranks then find it built
    if rank == 0:
        eng.build_engine()
    barrier()
    eng.build_engine()
    cfg = workloads.workload(args.workload)
    K, W = args.steps, args.warmup
    n_neurons = workloads.n_neurons(cfg)
    raster_cap = int(n_neurons * (K + W + 2) * 0.8) + (1 << 20)
    # the raster takes what the net leaves of the device (net: 10 B per
    # synapse slot, 12 B per reverse entry, ~200 B per neuron), so that a
    # large net over many steps still builds; a full raster counts its drops
    n_rin = cfg["grid_x"] * cfg["grid_y"] * cfg["exc_per_col"] * cfg["fanout"]
    net_est = workloads.n_synapses(cfg) * 10 + n_rin * 12 + n_neurons * 200
    free = torch.cuda.mem_get_info()[0]
    raster_cap = max(1 << 20, min(raster_cap, (free - net_est - (8 << 30)) // 4))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t_build = time.perf_counter()
        net = eng.Network(cfg, stream=stream, raster_capacity=raster_cap)
        t_build = time.perf_counter() - t_build
        device_bytes = net.device_bytes
        net.run(W)
        c0 = net.counters()
        clocks = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.run(K)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        c1 = net.counters()
        # the raster digest reads the window's spikes to the host: skipped
        # for windows of more than RASTER_DIGEST_MAX_SPIKES spikes (the full
        # 2000-step run holds ~1e10), where the counters are compared alone
        device_digest = (raster_digest(net, W, W + K)
                         if c1["raster_dropped"] == 0 and c1["spikes"] - c0["spikes"] <= RASTER_DIGEST_MAX_SPIKES
                         else None)

        # the kernels of the same steps, timed one by one: the net restarted
        # and the same steps run again with profiling on, in which the library
        # launches the step's kernels one after another, each between CUDA
        # events on its own stream (in the timed run above the potentiation
        # overlaps the delivery on a side stream, so their own durations
        # would count each other's time)
        # The launches of steps t0 .. t1 - 1 potentiate the spikers of steps
        # t0 - 1 .. t1 - 2 (step t takes the potentiation owed by t - 1), so
        # their potentiation visits are l_exc(t1 - 1) - l_exc(t0 - 1): the
        # counters are read one step before each end of the region.
        net.reset()
        net.run(max(0, W - 1))
        ca = net.counters()
        net.run(W - max(0, W - 1))
        net.set_profile(True)
        prof0 = net.profile()
        cp0 = net.counters()
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        net.run(K - 1)
        cb = net.counters()
        net.run(1)
        p1.record(stream)
        torch.cuda.synchronize()
        ms_profiled = p0.elapsed_time(p1)
        cp1 = net.counters()
        ltp_visits = cb["l_exc"] - ca["l_exc"]
        prof = net.profile()
        prof1 = prof
        net.set_profile(False)
        profiled_same_events = (cp1["e_all"] - cp0["e_all"]) == (c1["e_all"] - c0["e_all"])

        # end-to-end leg: the same workload restarted, driven from host memory
        # (the thalamic events of every step are copied in from pinned host
        # memory, the step's counters are read back)
        e2e = None
        if not args.no_e2e:
            KE = args.e2e_steps if args.e2e_steps is not None else K
            net.reset()
            net.set_thalamic(False)
            stim = snn.snn_thalamic_events(cfg, 0, W + KE)
            pinned = torch.empty(stim.nbytes, dtype=torch.uint8, pin_memory=True)
            stim_host = pinned.numpy().view(snn.STIM_DTYPE)
            stim_host[:] = stim
            per_step = cfg["grid_x"] * cfg["grid_y"] * cfg["thal_per_col_per_ms"]
            for s in range(W):
                net.run_host_counts(1, stim_host[s * per_step:(s + 1) * per_step])
            net.raster_reset()
            ce0 = net.counters()
            barrier()
            t0 = time.perf_counter()
            for s in range(W, W + KE):
                net.run_host_counts(1, stim_host[s * per_step:(s + 1) * per_step])
            el = time.perf_counter() - t0
            barrier()
            ce1 = net.counters()
            e2e = {"value": (ce1["e_all"] - ce0["e_all"]) / el, "unit": "events/s",
                   "h2d_bytes_per_step": per_step * snn.STIM_DTYPE.itemsize,
                   "d2h_bytes_per_step": 2 * DEVICE_COUNTERS_BYTES, "steps": KE,
                   "same_events_as_device_run": bool(ce1["e_all"] - ce0["e_all"] == c1["e_all"] - c0["e_all"]
                                                     and KE == K)}
            if KE == K and device_digest is not None and ce1["raster_dropped"] == 0:  # digest taken above
                e2e["raster_sha256_equals_device_run"] = raster_digest(net, W, W + K) == device_digest
            net.set_thalamic(True)

        # the regime that dominates the workload's first simulated second (the
        # net runs away to nearly every neuron firing every step, so the dense
        # pass takes the steps) and a step that closes a plasticity period
        steady = None
        if args.steady and rank == 0:
            steady = steady_leg(net, cfg, stream, n_neurons, args)
        net.close()

        # the rates of scattered L2 reductions, gathers and shared atomics on
        # an array the size of the net's input array: the roof of the
        # event-driven delivery, which is bound by them rather than by HBM
        atomics = None
        if rank == 0 and args.atomics:
            clk_a = ClockSampler(local_rank)
            atomics = snn.snn_microbench_atomics(n_neurons * 4, 4096, stream)
            atomics["clocks"] = clk_a.stop()

        # the 1-column, M = 100 workload is launch/latency bound: its figure is
        # microseconds per step with CUDA-graph replays (50 steps per graph)
        small = None
        if not args.no_small and rank == 0:
            scfg = workloads.workload("col1_m100")
            with eng.Network(scfg, stream=stream, raster_capacity=1 << 22) as sn:
                sn.run(100)
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                sn.run(1000)
                a1.record(stream)
                torch.cuda.synchronize()
                small = {"workload": "col1_m100 (1 column, 1250 neurons, M=100)", "steps": 1000,
                         "us_per_step": round(1000.0 * a0.elapsed_time(a1) / 1000.0, 2),
                         "graph_steps": sn.get_launch()["graph_steps"]}

        # batching: the 256 uneven nets, batched against one at a time
        batched = None
        if args.batch_nets > 0 and rank == 0:
            try:
                batched = batch_leg(args.batch_nets, args.batch_steps, args.batch_budget_gb, stream,
                                    args.batch_autotune_ms)
            except Exception as e:  # noqa: BLE001
                batched = {"error": "%s: %s" % (type(e).__name__, e)}

        # serving: p50 / p99 latency and throughput of a Poisson request
        # stream under continuous batching, after the main net is released;
        # a failure here is reported in the line instead of losing it
        served = None
        if args.serve_requests > 0 and rank == 0:
            try:
                served = {"workload": SERVE_WORKLOAD}
                served.update(serve_leg(args.serve_requests, args.serve_rate, args.batch_budget_gb, stream))
            except Exception as e:  # noqa: BLE001
                served = {"error": "%s: %s" % (type(e).__name__, e)}

    d_events = c1["e_all"] - c0["e_all"]
    d_exc = c1["e_exc"] - c0["e_exc"]
    d_ltp = ltp_visits
    d_spikes = c1["spikes"] - c0["spikes"]
    ms, total_events = combine_ranks(ms, d_events, dist, "cuda")
    if rank != 0:
        return 0

    secs = ms / 1000.0
    value = total_events / secs
    rate_hz = d_spikes / n_neurons / (K / 1000.0)
    n_exc_syn = cfg["grid_x"] * cfg["grid_y"] * cfg["exc_per_col"] * cfg["fanout"]
    dd = {k: prof1[k] - prof0[k] for k in ("dense_steps", "dense_deriv_steps", "dense_events",
                                             "dense_exc_events", "dense_ltp_visits")}
    updates = deriv_updates(c0["t"], c1["t"], cfg["deriv_period_ms"])
    alg = algorithmic_bytes(d_events, d_exc, d_ltp, n_neurons, prof["neuron"][0], n_exc_syn, updates, dd)
    peak, peak_kind = measured_peaks()
    names = ("deliver", "neuron", "ltp", "deriv", "dense")
    kernel_ms = {k: prof[k][1] for k in names}
    dom = max(kernel_ms, key=kernel_ms.get)
    achieved = alg[dom] / (kernel_ms[dom] / 1000.0) / 1e9
    per_kernel = {k: {"launches": prof[k][0], "ms": round(prof[k][1], 3),
                      "share": round(prof[k][1] / max(1e-9, sum(kernel_ms.values())), 4),
                      "alg_gbs": round(alg[k] / (prof[k][1] / 1000.0) / 1e9, 1) if prof[k][1] > 0 else None}
                  for k in names}
    per_kernel["dense"]["steps_taken"] = dd["dense_steps"]
    traffic = committed_traffic(dom, args.workload)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic}
    if traffic is not None and dom == "dense" and dd["dense_steps"] > 0:
        # measured DRAM bytes of a dense launch (committed ncu capture) over
        # this run's dense time: what the fused pass really moves
        dram = traffic * dd["dense_steps"] / (kernel_ms[dom] / 1000.0) / 1e9
        roofline["dram_achieved"] = round(dram, 1)
        roofline["dram_frac"] = round(dram / peak, 4)
    elif traffic is not None and prof[dom][0] > 0:
        # the committed capture's DRAM bytes per launch (the same timed steps
        # of the same workload) over this run's time of the kernel: what it
        # really moves, next to its algorithmic bytes
        dram = traffic * prof[dom][0] / (kernel_ms[dom] / 1000.0) / 1e9
        roofline["dram_achieved"] = round(dram, 1)
        roofline["dram_frac"] = round(dram / peak, 4)
        roofline["traffic_vs_algorithmic"] = round(traffic * prof[dom][0] / max(alg[dom], 1.0), 4)
    if atomics is not None and prof["deliver"][1] > 0:
        # events delivered by the event-driven kernels per second of their
        # time, split by where they land: an event on another column is one
        # scattered L2 reduction (the excitatory synapses outside the source
        # column: 1 - pct_ring[0] of them, exact on tori of side >= 5), an
        # event on the source column (every inhibitory one, the local share of
        # the excitatory ones) a shared-memory atomic; each against its
        # measured rate
        ev_sparse = d_events - dd["dense_events"]
        exc_sparse = d_exc - dd["dense_exc_events"]
        secs_d = prof["deliver"][1] / 1e3
        l2_red = exc_sparse * (1.0 - cfg["pct_ring"][0] / 100.0)
        smem = ev_sparse - l2_red
        red_rate = atomics["red_global_window_gops"] * 1e9
        smem_rate = atomics["atom_shared_window_gops"] * 1e9
        roofline["atomic"] = {"kernel": "deliver", "events_per_s": round(ev_sparse / secs_d),
                              "red_global_window_per_s": round(red_rate),
                              "atom_shared_window_per_s": round(smem_rate),
                              "l2_reductions_per_s": round(l2_red / secs_d),
                              "frac_of_l2_reduction_rate": round(l2_red / secs_d / red_rate, 4),
                              "shared_atomics_per_s": round(smem / secs_d),
                              "frac_of_shared_atomic_rate": round(smem / secs_d / smem_rate, 4)}
    line = {
        "metric": "synaptic events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32", "data": "synthetic",
        "config": {"workload": "%s: %dx%d torus, %d neurons, M=%d, %d synapses, mix %s" % (
            args.workload, cfg["grid_x"], cfg["grid_y"], n_neurons, cfg["fanout"], workloads.n_synapses(cfg),
            "/".join(str(p) for p in cfg["pct_ring"])),
            "step": "1 ms of simulated time", "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (%.1f GB resident on the device)" % (device_bytes / 1e9),
            "sim_ms_timed": [W, W + K]},
        "wall_s_per_sim_s_per_hz": (secs / (K / 1000.0)) / rate_hz if rate_hz > 0 else None,
        "wall_s_per_sim_s": secs / (K / 1000.0),
        "rate_hz": rate_hz,
        "events": d_events, "spikes": d_spikes,
        "raster": {"capacity": raster_cap, "dropped": c1["raster_dropped"]},
        "roofline": roofline,
        "kernels": per_kernel,
        "kernels_timed_in": {"what": "the same steps again from a reset, profiled: kernels one after another",
                             "ms_per_step": round(ms_profiled / K, 5), "same_events": bool(profiled_same_events)},
        "gpu_launches": int(prof1["kernels"] - prof0["kernels"]),
        "build_s": round(t_build, 2),
        "e2e": e2e,
        "steady": steady,
        "atomics": atomics,
        "small_net": small,
        "batch": batched,
        "serve": served,
        "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def raster_digest(net, t0: int, t1: int) -> str:
    """sha256 of the raster of steps [t0, t1) as little-endian int32 (t, gid)
    pairs sorted by (t, gid)."""
    import hashlib
    import numpy as np
    t, g = net.raster(t0, t1)
    return hashlib.sha256(np.stack([t, g], axis=1).astype("<i4").tobytes()).hexdigest()


def fused_dense_bytes(cfg) -> float:
    """Bytes one dense step must move by the fused pass's own count: every
    synapse's 2-byte target, and on excitatory rows the weight (4 B) and the
    derivative's read and write (8 B)."""
    s_all = workloads.n_synapses(cfg)
    s_exc = cfg["grid_x"] * cfg["grid_y"] * cfg["exc_per_col"] * cfg["fanout"]
    return 2.0 * s_all + 12.0 * s_exc


def timed_window(net, stream, n_steps: int, device: int = 0):
    """n_steps steps with per-kernel profiling, CUDA events and sampled clocks."""
    import torch
    net.set_profile(True)
    p0, c0 = net.profile(), net.counters()
    clocks = ClockSampler(device)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    net.run(n_steps)
    a1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    p1, c1 = net.profile(), net.counters()
    net.set_profile(False)
    return a0.elapsed_time(a1), p0, p1, c0, c1, clk


def steady_leg(net, cfg, stream, n_neurons, args, dense_at: int = 60, n_dense: int = 10, period_from: int = 995,
               n_period: int = 10):
    """After the timed region: n_dense steps from step dense_at (the run-away
    regime, dense pass), and n_period steps from period_from (they cross the
    long-term update that closes step period - 1)."""
    peak, peak_kind = measured_peaks()
    out = {}
    for name, start, steps in (("dense_regime", dense_at, n_dense), ("period_end", period_from, n_period)):
        t = net.t
        if t > start:
            continue
        if start > t:
            net.run(start - t)
        ms, p0, p1, c0, c1, clk = timed_window(net, stream, steps)
        ev = c1["e_all"] - c0["e_all"]
        spikes = c1["spikes"] - c0["spikes"]
        rate = spikes / n_neurons / (steps / 1000.0)
        dense_steps = p1["dense_steps"] - p0["dense_steps"]
        dense_ms = p1["dense"][1] - p0["dense"][1]
        leg = {"steps": [start, start + steps], "ms_per_step": ms / steps, "value": ev / (ms / 1000.0),
               "unit": "events/s", "rate_hz": rate,
               "wall_s_per_sim_s_per_hz": (ms / 1000.0 / (steps / 1000.0)) / rate if rate > 0 else None,
               "dense_steps": dense_steps, "clocks": clk,
               "kernel_ms": {k: round(p1[k][1] - p0[k][1], 3) for k in ("deliver", "neuron", "ltp", "deriv", "dense")}}
        if dense_steps > 0 and dense_ms > 0:
            fused = fused_dense_bytes(cfg) * dense_steps
            ach = fused / (dense_ms / 1000.0) / 1e9
            leg["dense_fused"] = {"bytes_per_step": fused_dense_bytes(cfg), "achieved": round(ach, 1), "peak": peak,
                                  "peak_kind": peak_kind, "unit": "GB/s", "frac": round(ach / peak, 4)}
        out[name] = leg
    return out


# largest window whose raster bench.py reads back for a digest (4 GB of host memory)
RASTER_DIGEST_MAX_SPIKES = 500_000_000

# bytes of the device counter block that snn_run_host copies to the host
# before and after the steps it runs (its result: the spikes of the window)
DEVICE_COUNTERS_BYTES = 184


if __name__ == "__main__":
    sys.exit(main())
