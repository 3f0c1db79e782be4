"""The workload definitions: the paper's geometry against its Table 1, and
the reproducibility and ranges of the batch and serving mixes."""
import os

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _table1():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_table1_sizes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                gx, gy, neu, syn = line.split()
                rows.append((int(gx), int(gy), float(neu), float(syn)))
    return rows


def test_paper_geometry_matches_table_1():
    rows = _table1()
    assert len(rows) == len(workloads.PAPER_GRIDS)
    for gx, gy, neu, syn in rows:
        cfg = workloads.workload("paper_%dx%d" % (gx, gy))
        assert (cfg["grid_x"], cfg["grid_y"]) == (gx, gy)
        assert cfg["neurons_per_col"] == 1000 and cfg["fanout"] == 200
        assert cfg["exc_per_col"] == 800                        # 80 % excitatory (Sec. 3)
        assert tuple(cfg["pct_ring"]) == (76, 12, 8, 4)          # Sec. 2, grid of columns
        # Table 1 rounds its totals to two or three digits
        assert workloads.n_neurons(cfg) == pytest.approx(neu, rel=0.03)
        assert workloads.n_synapses(cfg) == pytest.approx(syn, rel=0.03)


def test_batch_mix_is_reproducible_and_in_range():
    a = workloads.batch_workloads()
    b = workloads.batch_workloads()
    assert len(a) == 256 and a == b
    sides = np.array([c["grid_x"] for c in a])
    assert sides.min() >= 1 and sides.max() <= 16 and len(set(sides)) > 10
    assert all(c["grid_x"] == c["grid_y"] for c in a)
    assert {c["fanout"] for c in a} == {100, 400, 1125}
    assert [c["seed"] for c in a] == list(range(1000, 1256))


def test_serving_requests_are_in_range():
    rng = np.random.default_rng(5)
    sides, durs = [], []
    for i in range(500):
        cfg, dur = workloads.serve_request_params(i, rng)
        sides.append(cfg["grid_x"])
        durs.append(dur)
        assert cfg["fanout"] in (100, 400, 1125) and cfg["seed"] == 5000 + i
    assert min(sides) >= 1 and max(sides) <= 32 and 100 <= min(durs) and max(durs) <= 5000
    # log-uniform sides: about as many requests below side 6 as above
    assert 0.35 < np.mean(np.array(sides) <= 5) < 0.65
