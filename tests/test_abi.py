"""The C-ABI library builds, loads and exports every symbol include/snn.h
declares; the ctypes mirrors of its structs (and of the oracle's) match the
compiled headers field by field; host-side argument checks answer without a
GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads
from conftest import ROOT, build_readme_c_example

import paper_1310_8478_gb300 as eng
from paper_1310_8478_gb300 import snn


def declared_functions():
    src = open(os.path.join(ROOT, "include", "snn.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    names = re.findall(r"\b(snn_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = eng.build_engine()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(snn._SIGS)


def test_config_struct_layout_matches_header():
    # offsets the header fixes (all fields naturally aligned)
    c = snn.SnnConfig
    assert c.pct_ring.offset == 20 and c.max_delay_ms.offset == 36
    assert c.a_plus_mv.offset == 56 and c.seed.offset == 112 and c.raster_capacity.offset == 128
    assert ctypes.sizeof(c) == 136
    assert ctypes.sizeof(snn.SnnCounters) == 64
    assert ctypes.sizeof(snn.SnnLaunch) == 48
    assert ctypes.sizeof(snn.SnnProfile) == 128


def _compiled_layout(tmp_path, include_dir, header, structs):
    """sizeof and offsetof of every field of the ctypes mirrors in `structs`
    ({C type name: ctypes class}), printed by a C program built against the
    header itself."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "%s"' % header, 'int main(void) {']
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", include_dir, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return dict(line.split() for line in out.splitlines())


def _assert_layout(got, structs):
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert int(got["%s.%s" % (cname, field)]) == getattr(py, field).offset, (cname, field)


def test_every_struct_field_matches_the_compiled_header(tmp_path):
    structs = {"snn_config": snn.SnnConfig, "snn_spike": snn.SnnSpike, "snn_stimulus": snn.SnnStimulus,
               "snn_counters": snn.SnnCounters, "snn_launch": snn.SnnLaunch, "snn_profile": snn.SnnProfile}
    _assert_layout(_compiled_layout(tmp_path, os.path.join(ROOT, "include"), "snn.h", structs), structs)


def test_oracle_binding_matches_its_header(tmp_path):
    import oracle
    structs = {"orc_config": oracle.OrcConfig, "orc_stim": oracle.OrcStim}
    _assert_layout(_compiled_layout(tmp_path, os.path.join(ROOT, "oracle"), "oracle.h", structs), structs)


def _rc_build(cfg, budget=0):
    lib = snn.load()
    h = ctypes.c_void_p()
    c = snn.make_config(cfg)
    return lib.snn_build_network(ctypes.byref(c), None, budget, ctypes.byref(h)), h


@pytest.mark.parametrize("bad", [
    dict(grid_x=0), dict(neurons_per_col=1), dict(exc_per_col=0), dict(fanout=0), dict(fanout=70000),
    dict(pct_ring=(40, 30, 20, 11)), dict(max_delay_ms=0), dict(max_delay_ms=32), dict(wmax_q16=-1),
    dict(tau_plus_ms=0.0), dict(a_minus_mv=-0.1), dict(flags=8),
    dict(grid_x=2, thal_per_col_per_ms=1 << 30),
])
def test_bad_config_is_rejected_before_any_device_work(bad):
    rc, h = _rc_build(workloads.custom(**bad))
    assert rc == snn.EINVAL and not h.value
    assert snn.load().snn_last_error()


def test_budget_is_checked_before_any_device_work():
    rc, h = _rc_build(workloads.workload("grid64_m1125"), budget=1 << 30)
    assert rc == snn.ENOMEM and not h.value
    assert b"budget" in snn.load().snn_last_error()


def test_strerror_covers_every_code():
    lib = snn.load()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.snn_strerror(code) and lib.snn_strerror(code) != b"unknown error"
    assert lib.snn_strerror(-99) == b"unknown error"


def test_free_null_is_harmless():
    snn.load().snn_free(None)


def test_compact_target_slot_decode_is_exact():
    """Compact targets store slot * npc + local in 16 bits; the device recovers
    the slot as the high word of v * ceil(2^32 / npc).  The rounding error of
    the reciprocal times v < 2^16 stays below 2^-16 < 1 / npc, so the quotient
    is exact for every column size the compact format admits (2 <= npc <= 4096)."""
    for npc in range(2, 4097):
        r = np.uint64(((1 << 32) + npc - 1) // npc)
        assert r < 2 ** 32
        v = np.arange(13 * npc, dtype=np.uint64)
        assert np.array_equal((v * r) >> np.uint64(32), v // np.uint64(npc)), npc


def test_readme_c_example_builds_and_fails_loudly_without_a_gpu(tmp_path):
    # the example C program compiles warning-free against the header
    # and links against the library; on a machine without a GPU the first
    # call reports a CUDA error and the program exits 1 (there is no CPU path)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: tests/test_zz_readme_example.py runs the program")
    exe = build_readme_c_example(tmp_path, eng.build_engine())
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 1
    assert "CUDA" in r.stderr and r.stdout == ""


def test_readme_c_example_configures_the_one_column_workload():
    # every "c.field = value;" of the example program, evaluated, equals the
    # col1_m100 workload (the GPU test compares the program's output with the
    # oracle on that workload)
    code = open(os.path.join(ROOT, "examples", "readme_example.c")).read()
    got = {}
    for field, idx, expr in re.findall(r"\bc\.(\w+)(?:\[(\d)\])?\s*=\s*([^;]+);", code):
        value = eval(expr, {})
        if idx:
            got.setdefault(field, [0, 0, 0, 0])[int(idx)] = value
        else:
            got[field] = value
    cfg = workloads.workload("col1_m100")
    want = snn.make_config(cfg)
    for field, _ in snn.SnnConfig._fields_:
        if field in ("reserved", "flags"):
            continue
        if field == "pct_ring":
            assert got["pct_ring"] == list(cfg["pct_ring"])
        elif field == "raster_capacity":
            assert got[field] > 0
        else:
            assert got[field] == getattr(want, field), field


@pytest.mark.parametrize("cfg", [
    workloads.custom(grid_x=3, grid_y=2, seed=77),
    workloads.custom(grid_x=2, grid_y=2, neurons_per_col=997, exc_per_col=800, thal_per_col_per_ms=3,
                     thal_amp_q16=7 * 65536, seed=(1 << 40) + 12345),
])
def test_host_thalamic_events_equal_the_oracle(orc, cfg):
    # snn_thalamic_events is host code of the library (no GPU): every event it
    # lists -- step, target and amount -- equals the oracle's draw for that
    # (step, column, k), in step order, at the start and far into a run
    C = cfg["grid_x"] * cfg["grid_y"]
    K = cfg["thal_per_col_per_ms"]
    for t0, n_ms in ((0, 5), (123456, 3)):
        ev = snn.snn_thalamic_events(cfg, t0, n_ms)
        assert len(ev) == n_ms * C * K
        assert np.all(np.diff(ev["t"]) >= 0) and ev["t"][0] == t0 and ev["t"][-1] == t0 + n_ms - 1
        assert np.all(ev["q16"] == cfg["thal_amp_q16"])
        want = sorted((t, orc.thalamic_target(cfg, t, col, k))
                      for t in range(t0, t0 + n_ms) for col in range(C) for k in range(K))
        assert sorted(zip(ev["t"].tolist(), ev["gid"].tolist())) == want
