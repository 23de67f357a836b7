"""The seeded input generators follow the recipe they state: the SplitMix64
finaliser against its published outputs, counter-addressed streams, the two
pin-count laws (their point masses and means), distinct cells within a net,
fixed cells on the die perimeter, signals over the die with fixed rows at
their positions, the named workloads' sizes, and the batch and arrival
recipes."""
import math

import numpy as np
import pytest

from paper_2502_17632_gb300 import synth


def test_splitmix64_reference_outputs():
    """SplitMix64 seeded with 0 (the state advances by the golden gamma before
    each output): its first three outputs as published with the generator."""
    g = int(synth.GAMMA)
    z = np.array([(k * g) % 2 ** 64 for k in (1, 2, 3)], dtype=np.uint64)
    assert [int(v) for v in synth._mix64(z)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_counter_addressed():
    a = synth.u64(5, 3, np.arange(100, dtype=np.uint64))
    b = synth.u64(5, 3, np.array([42, 7], dtype=np.uint64))
    assert b[0] == a[42] and b[1] == a[7]
    assert not np.array_equal(synth.u64(5, 4, np.arange(100, dtype=np.uint64)), a)
    assert not np.array_equal(synth.u64(6, 3, np.arange(100, dtype=np.uint64)), a)
    u = synth.uniform(1, 1, np.arange(200_000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)


def test_geometric_pin_count_law():
    """2 pins with probability 0.6, else min(2 + G, 50), G ~ Geometric(0.35)
    on {1, 2, ...}: P(M = 3 | M > 2) = 0.35, mean 1.2 + 0.4 (2 + 1/0.35)."""
    n = 400_000
    m = synth.pin_counts("geom", n, 11, 50)
    assert m.min() == 2 and m.max() <= 50
    assert abs((m == 2).mean() - 0.6) < 4 * math.sqrt(0.24 / n)
    tail = m[m > 2]
    assert abs((tail == 3).mean() - 0.35) < 4 * math.sqrt(0.35 * 0.65 / tail.size)
    mean = 0.6 * 2 + 0.4 * (2 + 1 / 0.35)
    assert abs(m.mean() - mean) < 4 * m.std() / math.sqrt(n)
    assert mean == pytest.approx(3.142857, abs=1e-6)


def test_zipf_pin_count_law():
    """min(1 + Z, cap), Z ~ Zipf(2.2) on {1, 2, ...}: P(M = 2) = 1/zeta(2.2),
    P(M = 3) = 2^-2.2 / zeta(2.2), every count in [2, cap]."""
    special = pytest.importorskip("scipy.special")
    n = 400_000
    m = synth.pin_counts("zipf", n, 13, 2000)
    z = float(special.zeta(2.2, 1))
    assert m.min() == 2 and m.max() <= 2000
    for k, p in ((2, 1 / z), (3, 2 ** -2.2 / z), (4, 3 ** -2.2 / z)):
        assert abs((m == k).mean() - p) < 4 * math.sqrt(p * (1 - p) / n)
    assert (m == 2000).any()  # the cap is reached at this size


def test_netlist_cells_fixed_and_signals():
    nl = synth.make_netlist(5_000, 120, 6_000, 21)
    assert nl.num_cells == 5_120 and nl.num_nets == 6_000
    for e in range(nl.num_nets):
        cells = nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]
        assert len(set(cells.tolist())) == len(cells)  # distinct cells within a net
    assert nl.pin_cell.min() >= 0 and nl.pin_cell.max() < nl.num_cells
    fx = nl.is_fixed.astype(bool)
    assert fx.sum() == 120 and fx[-120:].all()  # the last cells are the fixed ones
    xy = nl.fixed_xy[fx].astype(np.float64)
    on_edge = np.isclose(xy, 0.0, atol=1e-3) | np.isclose(xy, 1000.0, atol=1e-3)
    assert on_edge.any(axis=1).all() and (xy >= 0).all() and (xy <= 1000.0).all()
    g = synth.make_signals(nl, 3, 21)
    assert g.shape == (5_120, 3, 2) and g.dtype == np.float32
    assert (g[~fx] >= 0).all() and (g[~fx] < 1000.0).all()
    np.testing.assert_array_equal(g[fx], np.repeat(nl.fixed_xy[fx][:, None, :], 3, axis=1))


def test_perimeter_positions_cover_the_four_sides():
    xy = synth.perimeter_xy(40_000, 1000.0, 3)
    side = np.select([xy[:, 1] == 0.0, xy[:, 0] == 1000.0, xy[:, 1] == 1000.0], [0, 1, 2], 3)
    counts = np.bincount(side, minlength=4) / len(xy)
    assert np.all(np.abs(counts - 0.25) < 0.01)


def test_named_workload_sizes():
    nl, g = synth.workload("plain-10k")
    assert (nl.num_cells, nl.num_nets, int(nl.is_fixed.sum()), g.shape) == (10_200, 12_000, 200, (10_200, 1, 2))
    nl, g = synth.workload("large-2.2m")
    assert (nl.num_cells, nl.num_nets, int(nl.is_fixed.sum())) == (2_202_000, 2_300_000, 2_000)
    assert nl.num_pins == 7_222_533 and g.shape == (2_202_000, 8, 2)


def test_batch_and_arrival_recipes():
    batch = synth.batch_workload(num_graphs=8)
    for nl, g in batch:
        n = nl.num_cells
        assert 5_000 - 1 <= n <= 300_000 + 1
        assert 1.0 * n - 1 <= nl.num_nets <= 1.2 * n + 1
        assert int(nl.is_fixed.sum()) == int(round(n * 0.01))
        assert g.shape == (n, 4, 2)
    t = synth.arrival_times(20_000, 40.0, 5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all() and abs(gaps.mean() - 1 / 40.0) < 4 * (1 / 40.0) / math.sqrt(len(gaps))
