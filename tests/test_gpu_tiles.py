"""The torus partitioned into column tiles (paper Sec. 2 "Delivery of
spiking messages"), run as several handles on the one GPU that exchange
their spikes through host buffers after every step (counts, then payload):
the tiles together must reproduce the oracle's run of the whole torus bit for
bit -- the union of their rasters, the event counters summed over tiles, and
every synapse's weight and derivative as kept by the tile that owns its
target."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


@pytest.mark.parametrize("gx,gy,n_tiles,fanout,T", [(4, 2, 2, 100, 1050), (4, 2, 3, 60, 1020),
                                                     (5, 3, 4, 100, 300)])
def test_tiles_reproduce_the_whole_torus(eng, orc, gx, gy, n_tiles, fanout, T):
    from paper_1310_8478_gb300 import tiles
    cfg = workloads.custom(grid_x=gx, grid_y=gy, fanout=fanout, pct_ring=(40, 30, 20, 10), seed=300 + n_tiles)
    npc = cfg["neurons_per_col"]
    o = orc.Oracle(cfg)
    o.run(T)
    ranges = tiles.column_ranges(gx * gy, n_tiles)
    dest = tiles.destinations(cfg, ranges)
    nets = [eng.Network(cfg, raster_capacity=workloads.n_neurons(cfg) * (T + 2)) for _ in ranges]
    try:
        for n, (first, count) in zip(nets, ranges):
            n.set_tile(first, count)
        tiles.step_local(nets, cfg, ranges, dest, n_ms=T)
        # rasters: every tile holds its own neurons' spikes
        ts, gs = zip(*[n.raster() for n in nets])
        t = np.concatenate(ts)
        g = np.concatenate(gs)
        order = np.lexsort((g, t))
        ot, og = o.raster()
        assert np.array_equal(t[order], ot) and np.array_equal(g[order], og)
        for n, (first, count) in zip(nets, ranges):
            assert np.all((g_ := n.raster()[1]) // npc >= first) and np.all(g_ // npc < first + count)
        # counters: each event, spike and potentiation visit is counted by one tile
        oc = o.counters()
        for k in ("spikes", "e_all", "e_exc", "l_exc"):
            assert sum(n.counters()[k] for n in nets) == oc[k], k
        assert all(n.counters()["error"] == 0 for n in nets)
        # synapses: the tile owning the target keeps the synapse
        s = o.synapses()
        owner = tiles.tile_of_column(ranges)[s["tgt"] // npc]
        w = np.empty_like(s["w"])
        sd = np.empty_like(s["sd"])
        for k, n in enumerate(nets):
            wk, sdk = n.weights()
            w[owner == k] = wk[owner == k]
            sd[owner == k] = sdk[owner == k]
        assert np.array_equal(w, s["w"]) and np.array_equal(sd, s["sd"])
        # the neuron state of every tile's own neurons
        on = o.neurons()
        for n, (first, count) in zip(nets, ranges):
            a, b = first * npc, (first + count) * npc
            nn = n.neurons(a, b - a)
            assert np.array_equal(nn["v"].view(np.int32), on["v"][a:b].view(np.int32))
            assert np.array_equal(nn["u"].view(np.int32), on["u"][a:b].view(np.int32))
    finally:
        for n in nets:
            n.close()


def test_tile_calls_refuse_what_does_not_fit(eng):
    cfg = workloads.custom(grid_x=2, grid_y=2, fanout=50, pct_ring=(40, 30, 20, 10), seed=5)
    with eng.Network(cfg, raster_capacity=1 << 16) as n:
        with pytest.raises(eng.SnnError):
            n.set_tile(3, 2)                       # beyond the torus
        with pytest.raises(eng.SnnError):
            n.inject_spikes([1])                   # not a tile
        n.set_tile(0, 2)
        with pytest.raises(eng.SnnError):
            n.inject_spikes([1])                   # no step run yet
        n.run(1)
        with pytest.raises(eng.SnnError):
            n.inject_spikes([5])                   # owned by the tile itself
        with pytest.raises(eng.SnnError):
            n.inject_spikes([2600, 2600])          # repeated
        n.inject_spikes([2600, 4999])
        with pytest.raises(eng.SnnError):
            n.set_tile(0, 4)                       # the net has stepped
