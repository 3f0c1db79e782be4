"""Host-side pieces of bench.py that need no GPU: the committed DRAM traffic
follows the kernel's source digest, the clock samples are summarised as the
JSON line reports them, the reference arm prints its line (rank 0 only)
with the keys the line must carry, and the per-kernel algorithmic bytes
charge each kernel the work it did (long-term updates counted per period
closed inside the timed launches, not per launch).  bench.main runs end to
end against a fake engine and fake CUDA calls, and its line carries every key
of the contract."""
import io
import json
import os
import sys
import types
from contextlib import redirect_stdout

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_committed_traffic_follows_the_source_digest(monkeypatch):
    p = os.path.join(ROOT, "profiles", "k_dense_grid64_m1125_dram.json")
    rec = json.load(open(p))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda kernel="dense": rec["source_sha256"])
    got = bench.committed_traffic("dense", "grid64_m1125")
    assert got == rec["dram_bytes_per_launch"]
    # the bytes per launch are the mean of the recorded launches
    per = [x["dram_read"] + x["dram_write"] for x in rec["launches"]]
    assert got == pytest.approx(sum(per) / len(per), rel=1e-9)
    monkeypatch.setattr(bench, "kernel_source_digest", lambda kernel="dense": "0" * 64)
    assert bench.committed_traffic("dense", "grid64_m1125") is None
    assert bench.committed_traffic("dense", "no_such_workload") is None


def test_kernel_source_digest_tracks_the_right_files():
    d_dense, d_step = bench.kernel_source_digest("dense"), bench.kernel_source_digest("ltp")
    assert len(d_dense) == 64 and len(d_step) == 64 and d_dense != d_step
    assert bench.kernel_source_digest("deliver_ordered") == d_step


def test_end_to_end_read_back_bytes_are_the_counter_block(tmp_path):
    """The end-to-end leg states its device-to-host bytes per step as two
    copies of the device counter block (before and after the step, inside
    snn_run_host): the constant must be that block's size as compiled."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "sz.cu"
    src.write_text('#include "snn_internal.cuh"\n#include <cstdio>\n'
                   'int main() { std::printf("%zu\\n", sizeof(snn::DevCounters)); return 0; }\n')
    exe = tmp_path / "sz"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1310_8478_gb300", "csrc"), "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert int(out) == bench.DEVICE_COUNTERS_BYTES


def test_clock_samples_are_summarised(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("1965, 2070, 900.1, Not Active, Not Active, Not Active, Active\n"
                    "1980, 2070, 910.0, Not Active, Not Active, Not Active, Not Active\n"
                    "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active\n"
                    "2010, 2070, 905.5, Not Active, Not Active, Not Active, Not Active\n"
                    "truncated line\n")
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.path = str(path)
    s.f = open(os.devnull, "w")
    s.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None,
                                   poll=lambda: 0)
    out = s.stop()
    assert out == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()


def test_clock_sampler_without_nvidia_smi_reports_nothing():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    assert s.stop() is None


def _args(**kw):
    a = dict(gpus=1, steps=5, warmup=3, impl="reference", workload=bench.DEFAULT_WORKLOAD, ref_budget_s=1.0)
    a.update(kw)
    return types.SimpleNamespace(**a)


def _fake_sample(seconds, t0, t1):
    # the oracle is timed over the GPU leg's window of steps
    return dict(value=1.5e7, unit="events/s", cores=1, kind="oracle", sample="fake sample",
                steps=t1 - t0, seconds=0.5, events=7.5e6)


def test_reference_arm_prints_one_complete_line(monkeypatch):
    monkeypatch.setattr(bench, "oracle_sample", _fake_sample)
    monkeypatch.setattr(bench, "dist_env", lambda: (0, 0, 1))
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args()) == 0
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] == 1.5e7 and line["steps"] == 5
    assert line["ms_per_step"] == pytest.approx(100.0)
    assert line["config"]["workload"] == bench.DEFAULT_WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": 1.5e7, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_off_rank_0(monkeypatch):
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: pytest.fail("rank 1 must not run the oracle"))
    monkeypatch.setattr(bench, "dist_env", lambda: (1, 1, 2))
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_args(gpus=2)) == 0
    assert buf.getvalue() == ""


@pytest.mark.parametrize("t0,t1,period,n", [
    (3, 2003, 1000, 2),      # the bench's default: updates closing steps 999 and 1999
    (0, 1000, 1000, 0),      # the update closing step 999 runs with step 1000's launch
    (0, 1001, 1000, 1),
    (1000, 1001, 1000, 1),
    (1001, 2000, 1000, 0),
    (5, 5, 1000, 0),
    (0, 5000, 0, 0),         # no long-term plasticity
    (0, 21, 7, 2),
])
def test_deriv_updates_counts_the_periods_closed_in_the_timed_launches(t0, t1, period, n):
    assert bench.deriv_updates(t0, t1, period) == n


def test_algorithmic_bytes_charge_each_kernel_its_own_work():
    dd = dict(dense_steps=1, dense_deriv_steps=1, dense_events=100, dense_exc_events=60, dense_ltp_visits=50)
    alg = bench.algorithmic_bytes(d_events=1000, d_exc=700, d_ltp=400, n_neurons=10, neuron_launches=4,
                                  n_exc_syn=30, updates=2, dd=dd)
    assert alg == {"deliver": 8.0 * 900 + 8.0 * 640, "ltp": 12.0 * 350, "neuron": 32.0 * 40,
                   "deriv": 16.0 * 30 * 1, "dense": 8.0 * 100 + 8.0 * 60 + 12.0 * 50 + 16.0 * 30}
    # a long-term update done by the dense pass is not charged to k_deriv
    alg = bench.algorithmic_bytes(1000, 700, 400, 10, 4, 30, updates=1, dd=dd)
    assert alg["deriv"] == 0.0


def test_serving_leg_reports_latency_and_throughput(monkeypatch):
    # the serving leg of the default line, driven by the fake engine of
    # test_serve_host.py (host logic only; the GPU run is the bench's own)
    import test_serve_host as ts
    from paper_1310_8478_gb300 import serve
    monkeypatch.setattr(serve, "snn", types.SimpleNamespace(Network=ts.FakeNet, Batch=ts.FakeBatch,
                                                            SnnError=ts.FakeError, ENOMEM=ts.ENOMEM))
    ts.FakeNet.live.clear()
    leg = bench.serve_leg(6, 200.0, 150.0, None)
    assert leg["requests"] == 6 and leg["unit"] == "events/s" and leg["value"] > 0
    assert set(leg["latency"]) == {"p50_s", "p99_s", "mean_s", "max_s"}
    assert leg["latency"]["p50_s"] <= leg["latency"]["p99_s"] <= leg["latency"]["max_s"]
    assert leg["sim_ms_total"] >= 6 * 100 and not ts.FakeNet.live
    # the same requests one at a time: same events, and the ratio reported
    assert leg["one_at_a_time"]["same_events"] and leg["speedup"] > 0


class _FakeBenchNet:
    """Stands in for snn.Network in bench.main: fixed work per step, no device."""

    def __init__(self, cfg, stream=None, raster_capacity=0, **kw):
        self.n = cfg["grid_x"] * cfg["grid_y"] * cfg["neurons_per_col"]
        self.device_bytes = self.n * 100
        self.t = 0
        self.prof_on = False
        self.prof_steps = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, n):
        self.t += n
        if self.prof_on:
            self.prof_steps += n

    def run_host_counts(self, n, events):
        assert len(events) > 0
        self.run(n)

    def set_profile(self, on):
        self.prof_on = bool(on)
        self.prof_steps = 0

    def profile(self):
        k = self.prof_steps
        out = {"deliver": (k, 0.1 * k), "neuron": (k, 0.05 * k), "ltp": (k, 0.02 * k),
               "deriv": (k, 0.01 * k), "dense": (k, 1.0 * k)}
        out.update(dense_steps=k // 2, dense_deriv_steps=0, dense_events=1000 * k, dense_exc_events=800 * k,
                   dense_ltp_visits=500 * k, kernels=7 * k)
        return out

    def counters(self):
        # potentiation visits grow with the step (as over an onset): the
        # visits of step s's spikers are 900 * (2 s + 1)
        return {"t": self.t, "spikes": 10 * self.t, "e_all": 2000 * self.t, "e_exc": 1500 * self.t,
                "l_exc": 900 * self.t * self.t, "raster_dropped": 0}

    def reset(self):
        self.t = 0

    def set_thalamic(self, on):
        pass

    def raster_reset(self):
        pass

    def raster(self, t0=0, t1=None):
        import numpy as np
        t = np.arange(t0, t1, dtype=np.int32)
        return t, (t * 7) % self.n

    def get_launch(self):
        return {"graph_steps": 50}

    def close(self):
        pass


def test_main_line_carries_every_key_with_a_fake_engine(monkeypatch, capsys):
    # bench.main end to end on the CPU: a fake engine and fake CUDA calls
    # stand in for the device; the line must parse and carry every key of
    # the contract, with the arithmetic of its derived figures
    import contextlib

    import torch

    import paper_1310_8478_gb300 as pkg
    import test_serve_host as ts
    from paper_1310_8478_gb300 import serve

    class Ev:
        def __init__(self, **kw):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 5.0 * 4.0                       # 4 ms per step over the 5 timed steps

    cuda = types.SimpleNamespace(is_available=lambda: True, set_device=lambda i: None,
                                 mem_get_info=lambda: (280e9, 285e9),
                                 Stream=lambda: types.SimpleNamespace(cuda_stream=0),
                                 stream=lambda s: contextlib.nullcontext(), synchronize=lambda: None, Event=Ev)
    monkeypatch.setattr(torch, "cuda", cuda)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, pin_memory=False, **k: real_empty(*a, **k))
    monkeypatch.setattr(pkg, "Network", _FakeBenchNet)
    monkeypatch.setattr(pkg, "build_engine", lambda *a, **k: None)
    monkeypatch.setattr(serve, "snn", types.SimpleNamespace(Network=ts.FakeNet, Batch=ts.FakeBatch,
                                                            SnnError=ts.FakeError, ENOMEM=ts.ENOMEM))
    ts.FakeNet.live.clear()
    monkeypatch.setattr(bench, "oracle_sample", lambda seconds, t0, t1: _fake_sample(seconds, t0, t1))
    monkeypatch.setattr(pkg.snn, "snn_microbench_atomics",
                        lambda nbytes, ops, stream=None: {"red_global_window_gops": 200.0,
                                                          "atom_shared_window_gops": 2000.0})
    monkeypatch.setattr(bench, "dist_env", lambda: (0, 0, 1))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "5", "--warmup", "3", "--serve-requests", "4",
                                      "--batch-nets", "0"])
    assert bench.main() == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks", "serve"):
        assert key in line, key
    assert line["steps"] == 5 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["ms_per_step"] == pytest.approx(4.0)
    assert line["value"] == pytest.approx(2000 * 5 / 0.020)
    assert line["gpu_launches"] == 35
    assert line["config"]["workload"].startswith(bench.DEFAULT_WORKLOAD)
    r = line["roofline"]
    assert r["kernel"] == "dense" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert line["e2e"]["h2d_bytes_per_step"] == 64 * 64 * 12      # one 12-byte event per column and step
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["serve"]["requests"] == 4 and "p99_s" in line["serve"]["latency"]
    assert line["kernels"]["deriv"]["alg_gbs"] == 0.0                # no period closes in steps 3..7
    # the launches of steps 3..7 potentiate the spikers of steps 2..6:
    # 900 * (7^2 - 2^2) visits, less the 500 per step the dense pass took,
    # 12 B each, over the fake's 0.02 ms per launch
    assert line["kernels"]["ltp"]["alg_gbs"] == pytest.approx(
        12.0 * (900 * (7 ** 2 - 2 ** 2) - 500 * 5) / (0.02 * 5 / 1000.0) / 1e9, abs=0.051)   # rounded to 0.1
    # the oracle is timed over the GPU leg's steps; the end-to-end leg
    # compares its raster with the device run's
    assert line["e2e"]["raster_sha256_equals_device_run"] is True
    assert line["roofline"]["atomic"]["red_global_window_per_s"] == 200e9
    st = line["steady"]
    assert st["dense_regime"]["steps"] == [60, 70] and st["period_end"]["steps"] == [995, 1005]
    assert st["dense_regime"]["dense_fused"]["bytes_per_step"] == pytest.approx(
        2.0 * 64 * 64 * 1250 * 1125 + 12.0 * 64 * 64 * 1000 * 1125)
