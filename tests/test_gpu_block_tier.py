"""The block tier of the graph build (rows of more than 512 raw entries) on
netlists shaped to reach each of its cases, bit-exact against the FP64
oracle: structure, stored weights and degrees.

A row's slots are its raw entries plus its incidences (every pin of every
net of the row, its own included).  The cases: a row of exactly 1,024 slots
(the smallest class, full); a row of exactly 15,360 slots (the largest
shared-memory class on this device, full) with 256 incidences (the most
that one-byte incidence indices allow); a row of 300 incidences in a
shared-memory class (two-byte indices); more than 32 incidences (the
incidences sorted block-wide rather than in one warp) with more than 2^16
cells and nets (three radix passes on each, the result on the other side of
the buffers); cells repeated inside long nets, the long row's cell twice in
one net, and two nets with the same pins (runs of several entries per column,
some with the same net twice); and a row beyond the shared-memory classes
(global scratch) among more than 2^16 cells.
"""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def from_nets(num_cells, nets):
    net_ptr = np.concatenate([[0], np.cumsum([len(n) for n in nets])]).astype(np.int64)
    pin_cell = np.array([c for n in nets for c in n], dtype=np.int32)
    fx = np.zeros(num_cells, np.uint8)
    fx[-2:] = 1
    return synth.Netlist(num_cells, len(nets), net_ptr, pin_cell, fx, np.zeros((num_cells, 2), np.float32))


def distinct_cells(seed, stream, count, num_cells, avoid):
    """count distinct cells of [0, num_cells) other than those in avoid, drawn by the counter generator."""
    u = synth.u64(seed, stream, np.arange(8 * count + 64, dtype=np.uint64)) % np.uint64(num_cells)
    out, seen = [], set(avoid)
    for v in u.astype(np.int64):
        if int(v) not in seen:
            seen.add(int(v))
            out.append(int(v))
            if len(out) == count:
                return out
    raise AssertionError("not enough draws")


def hub_nets(seed, num_cells, hub, count, pins):
    return [[hub] + distinct_cells(seed, 100 + e, pins - 1, num_cells, [hub]) for e in range(count)]


def small_nets(seed, num_cells, count, max_pins=6):
    s = synth.random_small(seed, num_cells, count, max_pins, min_pins=2)
    return [[int(c) for c in s.pin_cell[s.net_ptr[e]:s.net_ptr[e + 1]]] for e in range(s.num_nets)]


def slots(nl, cell):
    """Raw entries + incidences of a cell's row (the block tier's slot count)."""
    m = np.diff(nl.net_ptr)
    total = 0
    for e in range(nl.num_nets):
        if m[e] < 2:
            continue
        k = int((nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]] == cell).sum())
        total += k * int(m[e])
    return total


def case_need_1024():
    nets = hub_nets(31, 5000, 7, 16, 64) + [n for n in small_nets(32, 5000, 3000) if 7 not in n]
    return from_nets(5000, nets), 7, 1024


def case_top_class():
    nets = hub_nets(33, 20000, 11, 256, 60) + [n for n in small_nets(34, 20000, 6000) if 11 not in n]
    return from_nets(20000, nets), 11, 15360


def case_wide_ids():
    N = 70000
    nets = hub_nets(35, N, 3, 40, 50) + [n for n in small_nets(36, N, 70000) if 3 not in n]
    return from_nets(N, nets), 3, None


def case_repeats():
    N = 3000
    hub = 5
    nets = []
    for e in range(50):
        cells = [hub] + distinct_cells(37, 200 + e, 39, N, [hub])
        if e % 3 == 0:
            cells.append(cells[1 + e % 10])   # a neighbour twice in the net
        if e % 7 == 0:
            cells.append(hub)                 # the long row's own cell twice
        nets.append(cells)
    nets.append(list(nets[4]))                # two nets with the same pins
    nets.append(list(reversed(nets[9])))
    nets += [n for n in small_nets(38, N, 2000) if hub not in n]
    return from_nets(N, nets), hub, None


def case_many_incidences():
    nets = hub_nets(41, 5000, 9, 300, 3) + [n for n in small_nets(42, 5000, 3000) if 9 not in n]
    return from_nets(5000, nets), 9, 900


def case_global_wide_ids():
    N = 70000
    nets = hub_nets(39, N, 2, 400, 45) + [n for n in small_nets(40, N, 3000) if 2 not in n]
    return from_nets(N, nets), 2, None


CASES = {"need-1024": case_need_1024, "top-class": case_top_class, "wide-ids": case_wide_ids,
         "repeats": case_repeats, "many-incidences": case_many_incidences,
         "global-wide-ids": case_global_wide_ids}
_BUILT = {}


def get_case(name):
    if name not in _BUILT:
        nl, hub, want = CASES[name]()
        _BUILT[name] = (nl, hub, want, oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell))
    return _BUILT[name]


@pytest.mark.parametrize("wd", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_block_tier_bit_exact(ctx, name, wd):
    nl, hub, want, og64 = get_case(name)
    need = slots(nl, hub)
    if want is not None:
        assert need == want
    assert need > 512 + 1
    if name.startswith("global"):
        assert need > 15360
    if name in ("wide-ids", "global-wide-ids"):
        assert nl.num_cells > 1 << 16 and (name == "global-wide-ids" or nl.num_nets > 1 << 16)
    if name in ("wide-ids", "repeats", "many-incidences", "global-wide-ids"):
        assert int((nl.pin_cell == hub).sum()) > 32
    if name == "top-class":  # the most incidences a row may have for one-byte indices
        assert int((nl.pin_cell == hub).sum()) == 256
    if name == "many-incidences":  # more: two-byte indices, in a shared-memory class
        assert int((nl.pin_cell == hub).sum()) == 300
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                              gift.WEIGHT[wd])
    try:
        rp, col, val, deg = gift.gift_graph_export(h)
    finally:
        gift.gift_graph_free(h)
    og = oracle.stored(og64, wd)
    np.testing.assert_array_equal(rp, og.row_ptr)
    np.testing.assert_array_equal(col, og.col)
    np.testing.assert_array_equal(val, og.val)
    np.testing.assert_array_equal(deg, oracle.degrees(og))
