"""Parity with the oracle when the two sides of the STDP pair rule (Sec. 2,
"Synaptic update") take different amplitudes and time constants, and when a
depression amount no longer fits the 15 bits in which the dense pass and the
column-staged delivery stage it (the engine then keeps to the event-driven,
column-ordered delivery).  Bar: bit-exact, as in test_gpu_parity.py."""
import pytest

import workloads
from test_gpu_parity import assert_same_run, gpu_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


def _cfg(seed, **stdp):
    return workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=seed, **stdp)


@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense"])
def test_distinct_branch_constants_bitexact(eng, orc, mode):
    # every amount of both tables rounds to 0 before lag 255 (A+ e^{-25.5},
    # A- e^{-10.2}, both below half a Q16 unit)
    cfg = _cfg(41, a_plus_mv=0.2, tau_plus_ms=10.0, a_minus_mv=0.05, tau_minus_ms=25.0)
    o = orc.Oracle(cfg)
    o.run(1100)
    with gpu_net(eng, cfg, mode) as n:
        n.run(1100)
        assert_same_run(o, n)
        assert n.counters()["e_exc"] > 0


@pytest.mark.parametrize("mode", ["auto", "dense", "staged"])
def test_wide_depression_amounts_keep_to_the_ordered_delivery(eng, orc, mode):
    # A- = 1 mV puts 65536 in the first depression entry, above 0x7fff: the
    # dense pass and the staged delivery must stay off whatever the launch asks
    cfg = _cfg(42, a_minus_mv=1.0)
    o = orc.Oracle(cfg)
    o.run(1100)
    with gpu_net(eng, cfg, mode) as n:
        n.run(1100)
        assert_same_run(o, n)
        assert n.profile()["dense_steps"] == 0
