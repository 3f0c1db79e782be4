"""Per-kernel timing (snn_set_profile / snn_read_profile): a profiled run
launches every step eagerly with a CUDA-event pair around each kind of
kernel, counts every kernel it launches, and gives the same results as the
graph-replayed run the oracle is compared with.  The kernel count is what
bench.py reports as its launches.  This file is collected after the other
GPU tests, so that a stop at the first failure has run everything else."""
import pytest

import workloads
from test_gpu_parity import assert_same_run, gpu_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


def test_profile_counts_every_kernel_and_keeps_results(eng, orc):
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=44)
    T, T0 = 1100, 100
    o = orc.Oracle(cfg)
    o.run(T)
    with gpu_net(eng, cfg) as n:
        # make the column-staged delivery eligible, so that a step launches
        # the five step kernels k_ltp, k_deliver_ordered, k_deliver_cols,
        # k_dense, k_neuron_f32, and the step closing a period also k_fold
        # and k_deriv (the ring-list delivery of compact nets is off by
        # default and not launched)
        n.set_launch(staged_permille=1)
        n.run(T0)
        n.set_profile(True)
        n.run(T - T0)
        p = n.profile()
        n.set_profile(False)
        assert_same_run(o, n)
    # eager steps launch the long-term update's kernels (k_fold, k_deriv)
    # only in the step that closes a period (t = 1000 here)
    steps = T - T0
    for kind in eng.snn.KERNELS:
        launches, ms = p[kind]
        assert launches == (1 if kind == "deriv" else steps), (kind, launches)
        assert ms > 0, kind
    assert p["kernels"] == 5 * steps + 2
