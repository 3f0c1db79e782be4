"""The plain-C example program (examples/readme_example.c), run on the GPU: what it prints (spike and
event counts of one simulated second, first spike of the raster) equals the
oracle's figures for the same one-column workload.  Collected after the other
GPU tests, so that a stop at the first failure has run everything else."""
import subprocess

import pytest

import workloads
from conftest import build_readme_c_example

pytestmark = pytest.mark.gpu


def test_readme_c_example_matches_the_oracle(tmp_path, orc):
    import paper_1310_8478_gb300 as e
    exe = build_readme_c_example(tmp_path, e.build_engine())
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    # the example's configuration is the one-column benchmark workload
    o = orc.Oracle(workloads.workload("col1_m100"))
    o.run(1000)
    c = o.counters()
    rt, rg = o.raster()
    expect = "%d spikes, %d synaptic events, first spike: neuron %d at %d ms" % (
        c["spikes"], c["e_all"], int(rg[0]), int(rt[0]))
    assert r.stdout.strip() == expect
