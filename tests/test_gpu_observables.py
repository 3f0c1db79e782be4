"""Observables: the FP64 physics mode and membrane-trace probes (paper Sec. 2,
"Production of observables"), against the oracle."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


@pytest.mark.parametrize("gx,m,T", [(1, 100, 1100), (2, 60, 1050)])
def test_fp64_mode_equals_oracle_fp64(eng, orc, gx, m, T):
    cfg = workloads.custom(grid_x=gx, grid_y=gx, fanout=m, pct_ring=(40, 30, 20, 10) if gx > 1 else (100, 0, 0, 0),
                           seed=120 + gx, flags=eng.snn.FP64)
    o = orc.Oracle(cfg, flags=orc.FP64)
    o.run(T)
    with eng.Network(cfg, raster_capacity=1 << 22) as n:
        n.run(T)
        ot, og = o.raster()
        gt, gg = n.raster()
        assert np.array_equal(ot, gt) and np.array_equal(og, gg)
        s = o.synapses()
        w, sd = n.weights()
        assert np.array_equal(s["w"], w) and np.array_equal(s["sd"], sd)
        on, gn = o.neurons(), n.neurons_f64()
        assert np.array_equal(on["vd"].view(np.int64), gn["v"].view(np.int64))
        assert np.array_equal(on["ud"].view(np.int64), gn["u"].view(np.int64))


def _isi_histogram(t, g, n_neurons, bins):
    """Normalised histogram of the inter-spike intervals of every neuron."""
    order = np.lexsort((t, g))
    ts, gs = t[order].astype(np.int64), g[order]
    same = gs[1:] == gs[:-1]
    isi = (ts[1:] - ts[:-1])[same]
    h, _ = np.histogram(isi, bins=bins)
    return h / max(1, h.sum())


def test_fp64_rate_within_2_percent_of_fp32(eng):
    # stated physics check: the chaotic network's rasters diverge, its mean
    # rate may not move by more than 2 %; the distance between the two
    # inter-spike-interval histograms (total variation, 10 ms bins up to
    # 500 ms: ~15 k intervals, so sampling noise stays near 0.03) is reported
    # and bounded
    base = workloads.workload("col1_m100")
    rates, hists = [], []
    bins = np.arange(0, 501, 10)
    for flags in (0, eng.snn.FP64):
        with eng.Network(dict(base, flags=flags), raster_capacity=1 << 22) as n:
            n.run(2000)
            rates.append(n.counters()["spikes"] / 1250 / 2.0)
            t, g = n.raster()
            hists.append(_isi_histogram(t, g, 1250, bins))
    tv = 0.5 * float(np.abs(hists[0] - hists[1]).sum())
    print("fp32 rate %.3f Hz, fp64 rate %.3f Hz, ISI histogram total variation %.4f" % (rates[0], rates[1], tv))
    assert abs(rates[0] - rates[1]) <= 0.02 * rates[0], rates
    assert tv <= 0.1, tv


@pytest.mark.parametrize("fp64", [False, True])
def test_probe_traces_equal_oracle_step_by_step(eng, orc, fp64):
    cfg = workloads.custom(grid_x=2, grid_y=1, fanout=100, pct_ring=(40, 30, 20, 10), seed=130,
                           flags=eng.snn.FP64 if fp64 else 0)
    gids = [0, 17, 999, 1000, 1249, 2400]
    T0, T = 40, 120
    o = orc.Oracle(cfg, flags=orc.FP64 if fp64 else 0)
    o.run(T0)
    want_v, want_u = [], []
    for _ in range(T):
        o.run(1)
        nv = o.neurons()
        want_v.append((nv["vd"] if fp64 else nv["v"])[gids].astype(np.float32))
        want_u.append((nv["ud"] if fp64 else nv["u"])[gids].astype(np.float32))
    with eng.Network(cfg, raster_capacity=1 << 20) as n:
        n.run(T0)
        n.set_probe(gids, max_steps=T + 10)
        n.run(T)
        pv, pu = n.probe()
        assert pv.shape == (T, len(gids))
        assert np.array_equal(pv.view(np.int32), np.array(want_v).view(np.int32))
        assert np.array_equal(pu.view(np.int32), np.array(want_u).view(np.int32))
        n.set_probe([], 0)
        n.run(5)


def test_fp64_checkpoint_resume(eng):
    cfg = workloads.custom(grid_x=2, grid_y=1, fanout=100, pct_ring=(40, 30, 20, 10), seed=131,
                           flags=eng.snn.FP64)
    with eng.Network(cfg, raster_capacity=1 << 22) as a:
        a.run(700)
        ref = a.neurons_f64(), a.weights()
    with eng.Network(cfg, raster_capacity=1 << 22) as b:
        b.run(300)
        blob = b.save_state()
    with eng.Network(cfg, raster_capacity=1 << 22) as c:
        c.load_state(blob)
        c.run(400)
        got = c.neurons_f64(), c.weights()
    assert np.array_equal(ref[0]["v"], got[0]["v"]) and np.array_equal(ref[1][1], got[1][1])
