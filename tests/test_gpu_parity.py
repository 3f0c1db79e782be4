"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Bar: rasters, weights, derivatives, counters and the fp32 neuron state are
bit-exact (integer Q16 synaptic arithmetic; fp32 neuron update with the same
operation order and no contraction on either side).
"""
import numpy as np
import pytest

import workloads
from conftest import stdp_tables

pytestmark = pytest.mark.gpu

FORCE_Q16 = 300 * 65536


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


MODES = {"auto": None,
         "sparse": dict(dense_permille=1001, staged_permille=0xffffffff),
         "staged": dict(dense_permille=1001, staged_permille=1),
         "dense": dict(dense_permille=1),
         # the column walk in every event-driven step, and the ring-list
         # delivery in every one
         "ordered": dict(dense_permille=1001, staged_permille=0xffffffff, ring_permille=1),
         "ring": dict(dense_permille=1001, staged_permille=0xffffffff, ring_permille=0xffffffff)}


def gpu_net(eng, cfg, mode="auto", **kw):
    """mode: 'auto' (device picks per step), 'sparse' (event-driven kernels
    with global reductions only), 'staged' (event-driven delivery column by
    column through shared memory whenever anything is due) or 'dense' (the
    dense synapse pass whenever any neuron fired)."""
    kw.setdefault("raster_capacity", 1 << 22)
    n = eng.Network(cfg, **kw)
    if MODES[mode] is not None:
        n.set_launch(**MODES[mode])
    return n


def assert_same_run(orc_sim, net, check_state=True):
    ot, og = orc_sim.raster()
    gt, gg = net.raster()
    assert len(gt) == len(ot), (len(gt), len(ot))
    assert np.array_equal(gt, ot) and np.array_equal(gg, og)
    s = orc_sim.synapses()
    w, sd = net.weights()
    assert np.array_equal(w, s["w"])
    assert np.array_equal(sd, s["sd"])
    oc, gc = orc_sim.counters(), net.counters()
    for k in ("spikes", "e_all", "e_exc", "l_exc"):
        assert gc[k] == oc[k], (k, gc[k], oc[k])
    assert gc["error"] == 0
    if check_state:
        on = orc_sim.neurons()
        gn = net.neurons()
        assert np.array_equal(gn["v"].view(np.int32), on["v"].view(np.int32))
        assert np.array_equal(gn["u"].view(np.int32), on["u"].view(np.int32))


# ---------------------------------------------------------------------------
# construction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", [
    workloads.workload("col1_m100"),
    workloads.custom(grid_x=3, grid_y=2, fanout=300, pct_ring=(40, 30, 20, 10), seed=12),
    workloads.custom(grid_x=2, grid_y=2, fanout=1125, pct_ring=(40, 30, 20, 10), seed=4),
    workloads.custom(grid_x=7, grid_y=6, neurons_per_col=50, exc_per_col=40, fanout=200,
                     pct_ring=(76, 12, 8, 4), seed=11),
], ids=["col1", "3x2", "2x2_m1125", "paper_mix"])
def test_generated_network_equals_oracle(eng, orc, cfg):
    o = orc.Oracle(cfg)
    s = o.synapses()
    with gpu_net(eng, cfg) as n:
        g = n.synapses()
        assert np.array_equal(g["tgt"], s["tgt"])
        assert np.array_equal(g["delay"], s["delay"])
        assert np.array_equal(g["w"], s["w"])
        assert np.all(g["sd"] == 0)


# ---------------------------------------------------------------------------
# whole runs, bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense", "ordered", "ring"])
def test_col1_m100_full_second_bitexact(eng, orc, mode):
    cfg = workloads.workload("col1_m100")
    o = orc.Oracle(cfg)
    o.run(1000)
    with gpu_net(eng, cfg, mode) as n:
        n.run(1000)
        assert_same_run(o, n)
        assert n.counters()["spikes"] > 1000
        if mode == "dense":
            assert n.profile()["dense_steps"] > 300


@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense", "ordered", "ring"])
@pytest.mark.parametrize("gx,gy,m,T,seed", [
    (2, 2, 60, 1100, 31),        # ring members coincide on a 2x2 torus; crosses a derivative update
    (3, 3, 100, 1050, 32),
    (1, 1, 100, 2100, 33),       # two derivative updates
    (5, 3, 40, 1030, 34),        # ragged grid
])
def test_small_grids_bitexact_across_derivative_updates(eng, orc, gx, gy, m, T, seed, mode):
    cfg = workloads.custom(grid_x=gx, grid_y=gy, fanout=m,
                           pct_ring=(40, 30, 20, 10) if gx * gy > 1 else (100, 0, 0, 0), seed=seed)
    o = orc.Oracle(cfg)
    o.run(T)
    with gpu_net(eng, cfg, mode) as n:
        n.run(T)
        assert_same_run(o, n)


DEGENERATE = {
    # no thalamic drive and no stimulus: nothing ever fires, neurons settle
    "quiet": dict(grid_x=2, grid_y=2, neurons_per_col=100, exc_per_col=80, fanout=60,
                  pct_ring=(40, 30, 20, 10), seed=36, thal_per_col_per_ms=0),
    # one synapse per neuron, one delay
    "m1_d1": dict(grid_x=3, grid_y=3, neurons_per_col=100, exc_per_col=80, fanout=1,
                  pct_ring=(100, 0, 0, 0), seed=37, max_delay_ms=1, w_exc0_q16=9 * 65536),
    # the longest delay the layout allows, fan-out not a multiple of 8
    "d31": dict(grid_x=2, grid_y=2, neurons_per_col=100, exc_per_col=80, fanout=33,
                pct_ring=(40, 30, 20, 10), seed=38, max_delay_ms=31),
    # excitatory columns only / a single excitatory neuron per column
    "all_exc": dict(grid_x=2, grid_y=1, neurons_per_col=50, exc_per_col=50, fanout=40,
                    pct_ring=(40, 30, 20, 10), seed=39),
    "one_exc": dict(grid_x=2, grid_y=2, neurons_per_col=20, exc_per_col=1, fanout=15,
                    pct_ring=(40, 30, 20, 10), seed=40),
}


@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense", "ordered", "ring"])
@pytest.mark.parametrize("name", sorted(DEGENERATE))
def test_degenerate_networks_bitexact(eng, orc, name, mode):
    cfg = workloads.custom(**DEGENERATE[name])
    o = orc.Oracle(cfg)
    o.run(1100)                                   # crosses one long-term update
    with gpu_net(eng, cfg, mode) as n:
        n.run(1100)
        assert_same_run(o, n)
        c = n.counters()
        if name == "quiet":
            assert c["spikes"] == 0 and c["e_all"] == 0
        else:
            assert c["spikes"] > 0


def test_big_columns_with_32_bit_targets_bitexact(eng, orc):
    # columns above 4096 neurons keep 32-bit target ids: the ring-order
    # event-driven delivery (no column passes) against the oracle
    cfg = workloads.custom(grid_x=2, grid_y=1, neurons_per_col=4200, exc_per_col=3360, fanout=24,
                           pct_ring=(40, 30, 20, 10), seed=35, w_exc0_q16=12 * 65536)
    o = orc.Oracle(cfg)
    o.run(300)
    with gpu_net(eng, cfg) as n:
        n.run(300)
        assert_same_run(o, n)
        assert n.counters()["spikes"] > 100


@pytest.fixture(scope="module")
def grid8_onset(orc):
    # the 8x8, M = 1125 workload over its first 32 ms: activity grows from the
    # thalamic drive to ~70 % of the neurons firing every step
    o = orc.Oracle(workloads.workload("grid8_m1125"))
    o.run(32)
    return o


@pytest.mark.parametrize("mode", ["auto", "sparse", "staged", "dense", "ordered", "ring"])
def test_grid8_m1125_onset_bitexact(eng, grid8_onset, mode):
    with gpu_net(eng, workloads.workload("grid8_m1125"), mode) as n:
        n.run(32)
        assert_same_run(grid8_onset, n)
        assert n.counters()["spikes"] > 100000


@pytest.mark.parametrize("mode", ["sparse", "staged", "dense", "ordered", "ring"])
@pytest.mark.parametrize("flag_pair", [("STDP_OFF", 1, 1), ("DELIVERY_OFF", 2, 2)])
def test_debug_flags_bitexact(eng, orc, flag_pair, mode):
    _, of, gf = flag_pair
    cfg = workloads.custom(grid_x=2, grid_y=1, fanout=100, pct_ring=(40, 30, 20, 10), seed=41, flags=gf)
    o = orc.Oracle(cfg, flags=of)
    o.run(1200)
    with gpu_net(eng, cfg, mode) as n:
        n.run(1200)
        assert_same_run(o, n)


# ---------------------------------------------------------------------------
# STDP through the device path (explicit networks + forced spikes)
# ---------------------------------------------------------------------------
def _pair_cfg():
    return workloads.custom(grid_x=1, grid_y=1, neurons_per_col=2, exc_per_col=2, fanout=1,
                            pct_ring=(100, 0, 0, 0), thal_per_col_per_ms=0, deriv_period_ms=0)


@pytest.mark.parametrize("d", [1, 7, 20])
def test_stdp_pair_closed_form_on_gpu(eng, d):
    ltp, ltd = stdp_tables()
    net = dict(row_off=[0, 1, 1], tgt=[1], delay=[d], w=[0])
    t_pre = 60
    for lag in range(-40, 41):
        t_post = t_pre + d + lag
        with gpu_net(eng, _pair_cfg(), explicit=net) as n:
            n.set_stimulus([t_pre, t_post], [0, 1], [FORCE_Q16] * 2)
            n.run(max(t_pre + d, t_post) + 3)
            t, g = n.raster()
            assert sorted(zip(t.tolist(), g.tolist())) == sorted([(t_pre, 0), (t_post, 1)])
            sd = int(n.weights()[1][0])
            assert sd == (ltp[lag] if lag >= 0 else -ltd[-lag]), (d, lag)


def test_explicit_trains_equal_oracle(eng, orc):
    # random small explicit networks with forced spike trains and random rows
    rng = np.random.default_rng(7)
    for trial in range(6):
        n_neu, ne = 12, 9
        rows = [int(rng.integers(0, 6)) for _ in range(n_neu)]
        row_off = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
        S = int(row_off[-1])
        tgt = rng.integers(0, n_neu, S).astype(np.int32)
        dl = rng.integers(1, 21, S).astype(np.uint8)
        w = rng.integers(-3 * 65536, 3 * 65536, S).astype(np.int32)
        cfg = workloads.custom(grid_x=1, grid_y=1, neurons_per_col=n_neu, exc_per_col=ne, fanout=1,
                               pct_ring=(100, 0, 0, 0), thal_per_col_per_ms=0, deriv_period_ms=150,
                               seed=100 + trial)
        ex = dict(row_off=row_off, tgt=tgt, delay=dl, w=w)
        st_t = rng.integers(0, 400, 60)
        st_g = rng.integers(0, n_neu, 60)
        st_q = rng.integers(0, 40 * 65536, 60)
        o = orc.Oracle(cfg, explicit=ex)
        o.set_stimulus(st_t, st_g, st_q)
        o.run(420)
        with gpu_net(eng, cfg, explicit=ex) as n:
            n.set_stimulus(st_t, st_g, st_q)
            n.run(420)
            assert_same_run(o, n)


# ---------------------------------------------------------------------------
# layout invariance (Sec. 3: identical spikes for any distribution of the
# network): any launch shape, with or without graphs, gives identical results
# ---------------------------------------------------------------------------
SHAPES = [
    dict(deliver_block=256, deliver_blocks_per_sm=8, neuron_block=256, ltp_block=256, ltp_blocks_per_sm=8,
         graph_steps=50),
    dict(deliver_block=64, deliver_blocks_per_sm=1, neuron_block=32, ltp_block=32, ltp_blocks_per_sm=1,
         graph_steps=1, dense_permille=1001),
    dict(deliver_block=1024, deliver_blocks_per_sm=3, neuron_block=1024, ltp_block=512, ltp_blocks_per_sm=5,
         graph_steps=20, deriv_block=64, dense_permille=1, dense_block=128, dense_rows=37),
    dict(graph_steps=10, dense_permille=1, dense_block=512, dense_rows=1250),
    dict(graph_steps=2, dense_permille=20, dense_block=32, dense_rows=1),
    dict(graph_steps=4, dense_permille=1001, staged_permille=1),
    dict(graph_steps=1, dense_permille=200, staged_permille=300, deliver_block=128),
]


def test_layout_invariance_under_launch_shapes(eng):
    cfg = workloads.custom(grid_x=3, grid_y=2, fanout=200, pct_ring=(40, 30, 20, 10), seed=51)
    ref = None
    for shape in SHAPES:
        with gpu_net(eng, cfg) as n:
            n.set_launch(**shape)
            n.run(1010)
            r = (n.raster(), n.weights(), n.counters()["e_all"])
        if ref is None:
            ref = r
        else:
            assert np.array_equal(r[0][0], ref[0][0]) and np.array_equal(r[0][1], ref[0][1])
            assert np.array_equal(r[1][0], ref[1][0]) and np.array_equal(r[1][1], ref[1][1])
            assert r[2] == ref[2]


def test_step_by_step_equals_run(eng):
    cfg = workloads.workload("col1_m100")
    with gpu_net(eng, cfg) as a, gpu_net(eng, cfg) as b:
        a.run(230)
        for _ in range(230):
            b.step()
        assert np.array_equal(a.raster()[1], b.raster()[1])
        assert np.array_equal(a.weights()[1], b.weights()[1])


# ---------------------------------------------------------------------------
# checkpoint / resume, host end-to-end call
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["auto", "staged", "dense"])
def test_checkpoint_resume_is_bitexact(eng, mode):
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=61)
    with gpu_net(eng, cfg, mode) as a:
        a.run(1200)
        ref_r = a.raster(600, 1200)
        ref_w = a.weights()
    with gpu_net(eng, cfg, mode) as b:
        b.run(600)
        blob = b.save_state()
    with gpu_net(eng, cfg, mode) as c:
        c.load_state(blob)
        assert c.counters()["t"] == 600
        c.run(600)
        r = c.raster(600, 1200)
        assert np.array_equal(r[0], ref_r[0]) and np.array_equal(r[1], ref_r[1])
        w = c.weights()
        assert np.array_equal(w[0], ref_w[0]) and np.array_equal(w[1], ref_w[1])


def test_checkpoint_changing_an_inhibitory_weight_is_rejected(eng):
    """Inhibitory synapses are not plastic (Sec. 2 "Synaptic update": STDP acts
    on excitatory synapses); a checkpoint that changes one is refused."""
    from paper_1310_8478_gb300 import snn
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=63)
    with gpu_net(eng, cfg) as a:
        a.run(50)
        blob = bytearray(a.save_state())
    # the first inhibitory row's weights: the first run of 100 equal values
    # w_inh0 in the buffer (excitatory rows, currents and state hold none)
    w_inh = np.int32(cfg["w_inh0_q16"])
    hit = None
    for shift in range(4):
        v = np.frombuffer(bytes(blob[shift:len(blob) - (len(blob) - shift) % 4]), dtype=np.int32)
        eq = np.concatenate([[0], (v == w_inh).astype(np.int8), [0]])
        d = np.diff(eq)
        starts, ends = np.flatnonzero(d == 1), np.flatnonzero(d == -1)
        runs = [(s0, e0) for s0, e0 in zip(starts, ends) if e0 - s0 >= 100]
        if runs:
            off = shift + 4 * int(runs[0][0])
            hit = off if hit is None else min(hit, off)
    assert hit is not None
    with gpu_net(eng, cfg) as b:
        b.load_state(bytes(blob))                      # unchanged: accepted
        blob[hit:hit + 4] = np.int32(w_inh + 1).tobytes()
        with pytest.raises(snn.SnnError) as e:
            b.load_state(bytes(blob))
        assert e.value.code == snn.EINVAL


def test_run_host_equals_run_and_raster(eng):
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=62)
    with gpu_net(eng, cfg) as a, gpu_net(eng, cfg, "dense") as b:
        a.run(300)
        ref = a.raster(0, 300)
        t1, g1 = b.run_host(150)
        t2, g2 = b.run_host(150)
        assert np.array_equal(np.concatenate([t1, t2]), ref[0])
        assert np.array_equal(np.concatenate([g1, g2]), ref[1])


def test_overflow_bound_is_enforced(eng):
    cfg = workloads.custom(grid_x=1, grid_y=1, fanout=2000, wmax_q16=2 ** 30)
    with pytest.raises(eng.SnnError) as e:
        eng.Network(cfg)
    assert e.value.code == -4


def test_raster_capacity_overflow_is_reported(eng):
    cfg = workloads.workload("col1_m100")
    with gpu_net(eng, cfg, raster_capacity=100) as n:
        n.run(400)
        c = n.counters()
        assert c["raster_kept"] == 100 and c["raster_dropped"] == c["spikes"] - 100
        with pytest.raises(eng.SnnError) as e:
            n.raster(0, 400)
        assert e.value.code == -6


def test_host_thalamic_events_reproduce_the_internal_drive(eng):
    # the drive drawn on the host and fed as external stimulus, with the
    # net's own draws switched off, gives the same run
    cfg = workloads.custom(grid_x=3, grid_y=2, fanout=150, pct_ring=(40, 30, 20, 10), seed=63)
    from paper_1310_8478_gb300 import snn
    with gpu_net(eng, cfg) as a, gpu_net(eng, cfg) as b:
        a.run(400)
        b.set_thalamic(False)
        ev = snn.snn_thalamic_events(cfg, 0, 400)
        for k in range(4):
            b.run_host_counts(100, ev[k * 600:(k + 1) * 600])
        ra, rb = a.raster(), b.raster()
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        wa, wb = a.weights(), b.weights()
        assert np.array_equal(wa[0], wb[0]) and np.array_equal(wa[1], wb[1])


def test_run_host_counts_one_step_at_a_time(eng):
    # the end-to-end pattern of one call per step: each call's stimulus is
    # that step's drive (given in reverse order, so the library sorts it)
    # and each call returns that step's spike count; the run equals the
    # net's own drive, and a stimulus set on its own then run equals it too
    cfg = workloads.custom(grid_x=3, grid_y=2, fanout=150, pct_ring=(40, 30, 20, 10), seed=65)
    from paper_1310_8478_gb300 import snn
    T = 60
    with gpu_net(eng, cfg) as a, gpu_net(eng, cfg) as b, gpu_net(eng, cfg) as c:
        a.run(T)
        ta, ga = a.raster()
        b.set_thalamic(False)
        c.set_thalamic(False)
        ev = snn.snn_thalamic_events(cfg, 0, T)
        per = len(ev) // T
        for t in range(T):
            got = b.run_host_counts(1, ev[t * per:(t + 1) * per][::-1])
            assert got == int(np.count_nonzero(ta == t)), t
        c.set_stimulus(ev["t"], ev["gid"], ev["q16"])
        c.run(T)
        for n in (b, c):
            tb, gb = n.raster()
            assert np.array_equal(ta, tb) and np.array_equal(ga, gb)
            assert n.counters()["e_all"] == a.counters()["e_all"]


def test_reset_restarts_the_same_run(eng):
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=100, pct_ring=(40, 30, 20, 10), seed=64)
    with gpu_net(eng, cfg) as n:
        n.run(1100)
        r1, w1 = n.raster(), n.weights()
        n.reset()
        n.run(1100)
        r2, w2 = n.raster(), n.weights()
        assert np.array_equal(r1[1], r2[1]) and np.array_equal(w1[1], w2[1])


def test_repeated_runs_are_identical(eng):
    # the same net run three times (CUDA graphs, then eager steps) gives the
    # same raster, weights and derivatives: no result may depend on the
    # order in which threads or blocks happen to run (a 19x19 torus of the
    # serving mix, across a long-term update)
    cfg = workloads.custom(grid_x=19, grid_y=19, fanout=100, pct_ring=(40, 30, 20, 10), seed=5004)
    runs = []
    for shape in (None, None, dict(graph_steps=1)):
        with gpu_net(eng, cfg, raster_capacity=19 * 19 * 1250 * 1400) as n:
            if shape:
                n.set_launch(**shape)
            n.run(1400)
            t, g = n.raster()
            w, sd = n.weights()
            runs.append((t, g, w, sd, n.counters()["e_all"]))
    for r in runs[1:]:
        for a, b in zip(r[:4], runs[0][:4]):
            assert np.array_equal(a, b)
        assert r[4] == runs[0][4]
