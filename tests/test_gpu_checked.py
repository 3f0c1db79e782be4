"""The checked build (-DSNN_CHECKED: every step kernel verifies its computed
indices, records a bad one in the device error word and skips the access)
runs every pass bit-exact against the oracle with the error word clear.  It
runs in a child process, since a process loads one build of the library."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MODES = {"auto": {}, "sparse": dict(dense_permille=1001, staged_permille=0xffffffff),
         "staged": dict(dense_permille=1001, staged_permille=1), "dense": dict(dense_permille=1)}


def _main():
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    import paper_1310_8478_gb300 as eng
    from paper_1310_8478_gb300 import snn
    assert snn.checked() and snn.library_path().endswith("libsnn_checked.so")
    cases = [(workloads.workload("col1_m100"), 600),
             (workloads.custom(grid_x=3, grid_y=3, fanout=100, pct_ring=(40, 30, 20, 10), seed=32), 1050),
             (workloads.custom(grid_x=2, grid_y=1, neurons_per_col=4200, exc_per_col=3360, fanout=24,
                               pct_ring=(40, 30, 20, 10), seed=35, w_exc0_q16=12 * 65536), 200),
             (workloads.workload("grid8_m1125"), 24)]
    for cfg, T in cases:
        o = oracle.Oracle(cfg)
        o.run(T)
        ot, og = o.raster()
        s = o.synapses()
        for mode, shape in MODES.items():
            with eng.Network(cfg, raster_capacity=1 << 23) as n:
                if shape:
                    n.set_launch(**shape)
                n.run(T)
                t, g = n.raster()
                w, sd = n.weights()
                c = n.counters()
                assert c["error"] == 0, (cfg["name"], mode, c["error"])
                assert np.array_equal(t, ot) and np.array_equal(g, og), (cfg["name"], mode)
                assert np.array_equal(w, s["w"]) and np.array_equal(sd, s["sd"]), (cfg["name"], mode)
                assert c["e_all"] == o.counters()["e_all"], (cfg["name"], mode)
    print("checked build: all paths bit-exact, error word clear")


def test_checked_build_runs_every_pass_bitexact():
    env = dict(os.environ, SNN_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "import test_gpu_checked as t; t._main()"], cwd=HERE, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all paths bit-exact" in r.stdout
