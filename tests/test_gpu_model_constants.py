"""Parity with the oracle away from the benchmark's model constants: the two
sides of the STDP pair rule (Sec. 2, "Synaptic update") with different
amplitudes and time constants; a depression amount too wide for the 15 bits in
which the dense pass and the column-staged delivery stage it (the engine then
keeps to the event-driven, column-ordered delivery); several thalamic events
per column per ms with another amplitude (Sec. 2, thalamic stimulus) and a
long-term update (Table 2) with another period, bias, decay and weight bound.
Bar: bit-exact, as in test_gpu_parity.py."""
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


@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense"])
def test_drive_and_long_term_constants_bitexact(eng, orc, mode):
    # 3 thalamic events of 20 mV per column per ms (Philox counters
    # (t, col, 1, k), k = 0..2); long-term update every 250 ms with bias 1000,
    # decay 50000/65536 and wmax 6.5 mV, which about a tenth of the
    # excitatory weights reach by 1.1 s
    cfg = _cfg(43, thal_per_col_per_ms=3, thal_amp_q16=20 * 65536, deriv_period_ms=250,
               deriv_bias_q16=1000, deriv_decay_q16=50000, wmax_q16=425984)
    o = orc.Oracle(cfg)
    o.run(1100)
    with gpu_net(eng, cfg, mode) as n:
        n.run(1100)
        assert_same_run(o, n)
        w, _ = n.weights()
        assert (w == 425984).sum() > 1000
