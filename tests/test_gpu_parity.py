"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars: graph structure (row_ptr, col) bit-exact; stored weights and FP64
degrees bit-exact (same FP64 summation order, same round-to-nearest-even);
filter output within 1e-5 relative per coordinate in FP32 arithmetic; fixed
rows bit-exact; HPWL within 1e-12 relative (FP64 sums in another order).
"""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5  # FP32 filter vs FP64 oracle, per coordinate


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def build(ctx, nl, wd="f32", device=True):
    if device:
        return gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                                     gift.WEIGHT[wd])
    return gift.gift_build_graph(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, gift.WEIGHT[wd])


def rel_err(got, ref, g):
    floor = 1e-3 * max(float(np.abs(g).max()), 1e-30)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)


def star_netlist(num_cells, hub_nets, pins_per_net, seed, extra_nets=0):
    """Cell 0 sits in `hub_nets` nets of `pins_per_net` pins (a long row) plus random small nets."""
    nets = []
    for e in range(hub_nets):
        u = synth.u64(seed, 77, np.arange(e * 1000, e * 1000 + 4 * pins_per_net, dtype=np.uint64))
        cells = [0]
        for v in (u % np.uint64(num_cells - 1) + np.uint64(1)).astype(np.int64):
            if v not in cells:
                cells.append(int(v))
            if len(cells) == pins_per_net:
                break
        nets.append(cells)
    small = synth.random_small(seed, num_cells, extra_nets, 6, min_pins=2) if extra_nets else None
    if small is not None:
        for e in range(small.num_nets):
            nets.append(list(small.pin_cell[small.net_ptr[e]:small.net_ptr[e + 1]]))
    net_ptr = np.concatenate([[0], np.cumsum([len(n) for n in nets])]).astype(np.int64)
    pin_cell = np.array([c for n in nets for c in n], dtype=np.int32)
    fx = np.zeros(num_cells, dtype=np.uint8)
    fx[-3:] = 1
    return synth.Netlist(num_cells, len(nets), net_ptr, pin_cell, fx, np.zeros((num_cells, 2), np.float32))


def netlists():
    out = {
        "plain-10k": synth.workload("plain-10k")[0],
        "repeat-cells": synth.random_small(3, 300, 420, 9, num_fixed=10, allow_repeat=True),
        "tiny": synth.random_small(4, 7, 5, 4, num_fixed=1),
        "no-nets": synth.random_small(5, 9, 0, 3),
        "single-pin-nets": synth.random_small(6, 20, 30, 1),
        "one-cell": synth.Netlist(1, 2, np.array([0, 1, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                                  np.zeros(1, np.uint8), np.zeros((1, 2), np.float32)),
        "block-tier-row": star_netlist(1000, 20, 40, 8, extra_nets=300),
        "global-tier-row": star_netlist(3000, 400, 45, 9, extra_nets=500),
    }
    return out


NETLISTS = netlists()


@pytest.mark.parametrize("wd", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", sorted(NETLISTS))
def test_graph_bit_exact(ctx, name, wd):
    nl = NETLISTS[name]
    h = build(ctx, nl, wd)
    try:
        rp, col, val, deg = gift.gift_graph_export(h)
        info = gift.gift_graph_info(h)
    finally:
        gift.gift_graph_free(h)
    og = oracle.stored(oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell), wd)
    np.testing.assert_array_equal(rp, og.row_ptr)
    np.testing.assert_array_equal(col, og.col)
    np.testing.assert_array_equal(val, og.val)
    np.testing.assert_array_equal(deg, oracle.degrees(og))
    assert info.nnz == og.nnz
    m = nl.net_ptr[1:] - nl.net_ptr[:-1]
    assert info.raw_pairs == int((m * (m - 1))[m >= 2].sum())
    # rows keep their raw positions (zero-weight padding) when at most 1/1024 of them collapse
    padded = info.raw_pairs - og.nnz <= info.raw_pairs // 1024
    assert info.stored == (info.raw_pairs if padded else og.nnz)
    if og.nnz:
        assert info.max_row_nnz == int((og.row_ptr[1:] - og.row_ptr[:-1]).max())


_WIDE = {}


def wide_net_case():
    """One net of 4,200 pins over cells 0..4199 of 4,400 plus 600 small nets:
    the wide net's weight 2/4200 lies below 2^-11, so the degrees of its rows
    (block tier, 4,199 or more raw entries) take the one-thread FP64 sum, not
    the integer count; the other rows mix both."""
    if not _WIDE:
        M, N = 4200, 4400
        nets = [list(range(M))]
        small = synth.random_small(12, N, 600, 6, min_pins=2)
        for e in range(small.num_nets):
            nets.append([int(c) for c in small.pin_cell[small.net_ptr[e]:small.net_ptr[e + 1]]])
        net_ptr = np.concatenate([[0], np.cumsum([len(n) for n in nets])]).astype(np.int64)
        pin_cell = np.array([c for n in nets for c in n], dtype=np.int32)
        nl = synth.Netlist(N, len(nets), net_ptr, pin_cell, np.zeros(N, np.uint8), np.zeros((N, 2), np.float32))
        _WIDE["nl"] = nl
        _WIDE["og"] = oracle.build_graph(N, net_ptr, pin_cell)
    return _WIDE["nl"], _WIDE["og"]


@pytest.mark.parametrize("wd", ["f32", "bf16", "f16"])
def test_block_tier_fp64_degrees(ctx, wd):
    nl, og64 = wide_net_case()
    assert 2.0 / 4200 < 2.0 ** -11
    h = build(ctx, nl, wd)
    try:
        rp, col, val, deg = gift.gift_graph_export(h)
    finally:
        gift.gift_graph_free(h)
    og = oracle.stored(og64, wd)
    np.testing.assert_array_equal(rp, og.row_ptr)
    np.testing.assert_array_equal(col, og.col)
    np.testing.assert_array_equal(val, og.val)
    np.testing.assert_array_equal(deg, oracle.degrees(og))


def test_host_and_device_inputs_agree(ctx):
    nl = NETLISTS["repeat-cells"]
    a, b = build(ctx, nl, device=True), build(ctx, nl, device=False)
    try:
        for x, y in zip(gift.gift_graph_export(a), gift.gift_graph_export(b)):
            np.testing.assert_array_equal(x, y)
    finally:
        gift.gift_graph_free(a)
        gift.gift_graph_free(b)


def run_filter(ctx, nl, g, wd="f32", spec=None, device=True):
    h = build(ctx, nl, wd)
    try:
        if device:
            gi = dev(g)
            go = torch.empty_like(gi)
            gift.gift_filter(ctx, h, gi, go, spec)
            torch.cuda.synchronize()
            return go.cpu().numpy()
        out = np.empty_like(g)
        gift.gift_filter(ctx, h, g, out, spec)
        return out
    finally:
        gift.gift_graph_free(h)


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("S", [1, 2, 3, 8])
@pytest.mark.parametrize("schedule", [0, 416, 1016, 1004, 3002, 4042, 14044, 4148, 4244, 4644, 4724,
                                      4844, 5044, 5244, 5844, 6444, 14844, 16444])
def test_filter_parity(ctx, name, S, schedule):
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 1234 + S)
    got = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=schedule))
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    ref = ref.reshape(g.shape)
    assert rel_err(got, ref, g).max() <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])


@pytest.mark.parametrize("S", [1, 2, 4, 5, 8, 9, 16])
@pytest.mark.parametrize("schedule", [0, 4, 8, 16, 32, 108, 132, 204, 216, 408, 416, 432,
                                      1002, 1004, 1008, 1016, 2008, 2016, 3002, 3004, 3008, 3016,
                                      4012, 4014, 4022, 4024, 4042, 4044, 4082, 4084, 4112, 4118, 4142,
                                      4148, 4182, 4188, 4244, 4342, 4388, 4414, 4424, 4444, 4484, 4514, 4524,
                                      4644, 4744, 4784, 10408, 13008, 14042, 14148, 14244, 14644,
                                      4812, 4822, 4842, 4844, 4914, 4988, 5014, 5044, 5244, 5644, 5814, 5844,
                                      6412, 6444, 6544, 6644, 14844, 15044, 16444])
def test_filter_shapes_and_schedules(ctx, S, schedule):
    nl = NETLISTS["repeat-cells"]
    g = synth.make_signals(nl, S, 99 + S)
    spec = gift.make_spec(schedule=schedule)
    K = 2 * S
    bad_tma = 2000 <= schedule < 3000 and K % (schedule - 2000) != 0
    if bad_tma:
        with pytest.raises(gift.GiftError) as e:
            run_filter(ctx, nl, g, spec=spec)
        assert e.value.status == gift.GIFT_ERR_INVALID
        return
    got = run_filter(ctx, nl, g, spec=spec)
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    assert rel_err(got, ref.reshape(g.shape), g).max() <= RTOL


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("S,schedule", [(4, 2008), (8, 2016), (8, 2008), (16, 2016), (4, 3008), (8, 3016),
                                        (8, 3008), (16, 3016), (2, 3004)])
def test_filter_tma_and_sell(ctx, name, S, schedule):
    """The TMA gather4 pipeline and the sliced-ELL format on every netlist shape
    (empty rows, long rows, one cell)."""
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 4321 + S)
    got = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=schedule))
    gift.gift_ctx_device_status(ctx)
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    assert rel_err(got, ref.reshape(g.shape), g).max() <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])


@pytest.mark.parametrize("terms,norm,reimpose", [
    (((2.0, 2, 0.1), (4.0, 2, 0.7), (4.0, 4, 0.2)), "rw", True),
    (((2.0, 2, 0.1), (4.0, 2, 0.7), (4.0, 4, 0.2)), "sym", False),
    (((1.0, 1, 0.25), (3.0, 3, 0.5), (0.5, 2, 0.25)), "sym", True),   # three chains at once
    (((4.0, 4, 1.0),), "sym", True),
    (((2.0, 1, 0.3), (2.0, 3, 0.7)), "sym", True),
    (((1.0, 1, 0.2), (2.0, 2, 0.2), (3.0, 3, 0.2), (4.0, 4, 0.2), (5.0, 5, 0.2)), "sym", True),
    (((1.0, 1, 0.25), (2.0, 2, 0.25), (3.0, 3, 0.25), (4.0, 4, 0.25)), "sym", True),  # two chain pairs
    (((1.0, 1, 0.25), (2.0, 2, 0.25), (3.0, 3, 0.25), (4.0, 4, 0.25)), "rw", True),
])
@pytest.mark.parametrize("schedule", [0, 3008, 4042, 14042, 408, 4842, 5842, 6442, 16442])
def test_filter_general_specs(ctx, terms, norm, reimpose, schedule):
    """Chains grouped in pairs, one chain left over, both normalisations; the
    first sweep of every pair gathers g once with that pair's two scales."""
    nl = NETLISTS["plain-10k"]
    g = synth.make_signals(nl, 2, 5)
    spec = gift.make_spec(terms=terms, norm=gift.GIFT_NORM_RW if norm == "rw" else gift.GIFT_NORM_SYM,
                          reimpose=reimpose, schedule=schedule)
    got = run_filter(ctx, nl, g, spec=spec)
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1), terms=terms, norm=norm, reimpose=reimpose)
    assert rel_err(got, ref.reshape(g.shape), g).max() <= RTOL


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("S", [1, 8])
def test_row_order_does_not_change_sums(ctx, name, S):
    """Direct row groups sum every row alone in CSR order, so walking the rows
    in natural order, in the window order, in length order over the CSR or
    from the sorted copy of the CSR gives the same bits.  (Running a chain
    pair as two launches combines the terms in another order, and the
    pre-scaled first sweep rounds s_j g_j once more: each is compared with its
    own kind, and all meet the FP32 bar.)"""
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 77)
    for base_sched, same in ((4244, (4044, 4844, 5044)), (14244, (14044, 14844, 15044))):
        base = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=base_sched))
        for sched in same:
            np.testing.assert_array_equal(run_filter(ctx, nl, g, spec=gift.make_spec(schedule=sched)), base,
                                          err_msg=f"schedule {sched} vs {base_sched}")
    pre = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=6444))
    np.testing.assert_array_equal(run_filter(ctx, nl, g, spec=gift.make_spec(schedule=5844)), pre)
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    assert rel_err(pre, ref.reshape(g.shape), g).max() <= RTOL


@pytest.mark.parametrize("S", [2, 8])
@pytest.mark.parametrize("schedule", [4244, 4844, 5044, 4224, 408, 14244])
def test_long_rows_compensated_by_default(ctx, S, schedule):
    """The default spec sums the rows of at least 1024 entries (the hub row of
    17,600 here) with Neumaier compensation and every other row plainly: on
    one product, the hub row equals the all-rows compensated result and the
    other rows the plain result, bit for bit; and the default filter meets
    the FP32 bar against the oracle."""
    nl = NETLISTS["global-tier-row"]
    g = synth.make_signals(nl, S, 31)
    one = ((2.0, 1, 1.0),)
    auto = run_filter(ctx, nl, g, spec=gift.make_spec(terms=one, schedule=schedule, compensated=0))
    comp = run_filter(ctx, nl, g, spec=gift.make_spec(terms=one, schedule=schedule, compensated=1))
    plain = run_filter(ctx, nl, g, spec=gift.make_spec(terms=one, schedule=schedule, compensated=2))
    rp = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell).row_ptr
    long_rows = np.diff(rp) >= 1024
    assert long_rows.sum() == 1 and long_rows[0]
    np.testing.assert_array_equal(auto[long_rows], comp[long_rows])
    np.testing.assert_array_equal(auto[~long_rows], plain[~long_rows])
    got = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=schedule))
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    assert rel_err(got, ref.reshape(g.shape), g).max() <= RTOL


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("schedule", [0, 4644, 4424, 408])
def test_compensated_sums(ctx, name, schedule):
    """spec.compensated = 1: warp-row kernels with Neumaier sums (the schedule's
    lane count kept for direct shapes, the default warp-row shape otherwise);
    the same 1e-5 bar, including the star netlists' hub rows of 1,000 and
    17,000 nonzeros."""
    nl = NETLISTS[name]
    g = synth.make_signals(nl, 4, 2024)
    got = run_filter(ctx, nl, g, spec=gift.make_spec(schedule=schedule, compensated=True))
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    assert rel_err(got, ref.reshape(g.shape), g).max() <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])
    sched = gift.gift_ctx_last_schedule(ctx)
    assert all(c == 0 or 4400 <= c % 10000 < 4800 for c in sched)  # warp-row direct kernels


@pytest.mark.parametrize("wd", ["bf16", "f16"])
def test_reduced_precision_weights(ctx, wd):
    """Against the oracle on the same rounded weights: the FP32 bar.  Against the
    exact-weight oracle: the weight-rounding error, bounded as measured."""
    nl = NETLISTS["plain-10k"]
    g = synth.make_signals(nl, 4, 17)
    got = run_filter(ctx, nl, g, wd=wd)
    _, _, ref_q = oracle.run(nl, g.reshape(nl.num_cells, -1), fmt=wd)
    assert rel_err(got, ref_q.reshape(g.shape), g).max() <= RTOL
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    bound = {"bf16": 5e-3, "f16": 1e-3}[wd]
    assert rel_err(got, ref.reshape(g.shape), g).max() <= bound


def test_host_memory_filter_matches_device(ctx):
    nl = NETLISTS["plain-10k"]
    g = synth.make_signals(nl, 3, 3)
    np.testing.assert_array_equal(run_filter(ctx, nl, g, device=True), run_filter(ctx, nl, g, device=False))


def test_filter_is_deterministic(ctx):
    nl = NETLISTS["repeat-cells"]
    g = synth.make_signals(nl, 8, 1)
    np.testing.assert_array_equal(run_filter(ctx, nl, g), run_filter(ctx, nl, g))


@pytest.mark.parametrize("S", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("name", ["plain-10k", "repeat-cells", "global-tier-row", "single-pin-nets"])
def test_hpwl_parity(ctx, name, S):
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 8)
    h = build(ctx, nl)
    try:
        got_d = gift.gift_hpwl(ctx, h, dev(g))
        got_h = gift.gift_hpwl(ctx, h, g)
    finally:
        gift.gift_graph_free(h)
    ref = oracle.hpwl(nl.net_ptr, nl.pin_cell, g)
    np.testing.assert_allclose(got_d, ref, rtol=1e-12)
    np.testing.assert_array_equal(got_d, got_h)


# ---------------------------------------------------------------- errors
def test_invalid_netlists_rejected(ctx):
    nl = NETLISTS["tiny"]
    bad_pin = nl.pin_cell.copy()
    bad_pin[0] = nl.num_cells
    with pytest.raises(gift.GiftError) as e:
        gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(bad_pin), None)
    assert e.value.status == gift.GIFT_ERR_INVALID
    bad_pin[0] = -1
    with pytest.raises(gift.GiftError) as e:
        gift.gift_build_graph(ctx, nl.num_cells, nl.net_ptr, bad_pin, None)
    assert e.value.status == gift.GIFT_ERR_INVALID
    bad_ptr = nl.net_ptr.copy()
    bad_ptr[1] = bad_ptr[2] + 1  # net 1 ends before it starts
    with pytest.raises(gift.GiftError) as e:
        gift.gift_build_graph(ctx, nl.num_cells, dev(bad_ptr), dev(nl.pin_cell), None)
    assert e.value.status == gift.GIFT_ERR_INVALID
    with pytest.raises(gift.GiftError) as e:
        gift.gift_build_graph(ctx, 0, nl.net_ptr, nl.pin_cell, None)
    assert e.value.status == gift.GIFT_ERR_INVALID


def test_invalid_filter_args(ctx):
    nl = NETLISTS["tiny"]
    h = build(ctx, nl)
    g = dev(synth.make_signals(nl, 2, 1))
    out = torch.empty_like(g)
    try:
        for terms in [((0.0, 2, 1.0),), ((2.0, 0, 1.0),), ((2.0, 65, 1.0),), ((float("nan"), 1, 1.0),)]:
            with pytest.raises(gift.GiftError) as e:
                gift.gift_filter(ctx, h, g, out, gift.make_spec(terms=terms))
            assert e.value.status == gift.GIFT_ERR_INVALID
        for bad in (3, -1):
            spec = gift.make_spec()
            spec.compensated = bad
            with pytest.raises(gift.GiftError):
                gift.gift_filter(ctx, h, g, out, spec)
        spec = gift.make_spec()
        spec.num_terms = 9
        with pytest.raises(gift.GiftError):
            gift.gift_filter(ctx, h, g, out, spec)
        with pytest.raises(gift.GiftError):
            gift.gift_filter(ctx, h, g, g, None)  # overlap
        with pytest.raises(gift.GiftError):
            gift.gift_filter(ctx, h, g, out, None, num_signals=0)
        for bad in (1, 2, 3, 404 + 1, 800 + 16, 216 + 100, 1161, 1003, 1032, 4043, 4062, 4442, 4041,
                    4642, 5046, 5644 + 2, 7244, 9999, 10000, 10003, 19999, 20000):
            with pytest.raises(gift.GiftError) as e:
                gift.gift_filter(ctx, h, g, out, gift.make_spec(schedule=bad))
            assert e.value.status == gift.GIFT_ERR_INVALID
    finally:
        gift.gift_graph_free(h)


def test_injected_oom_leaves_library_usable(ctx):
    nl = NETLISTS["repeat-cells"]
    g = synth.make_signals(nl, 2, 4)
    for n in (1, 3, 6, 9):
        gift.gift_ctx_debug_fail_alloc(ctx, n)
        try:
            h = build(ctx, nl)
        except gift.GiftError as e:
            assert e.status == gift.GIFT_ERR_OOM
            continue
        finally:
            gift.gift_ctx_debug_fail_alloc(ctx, 0)
        gift.gift_graph_free(h)
    h = build(ctx, nl)
    try:
        gift.gift_ctx_debug_fail_alloc(ctx, 2)
        gi = dev(g)
        go = torch.empty_like(gi)
        with pytest.raises(gift.GiftError) as e:
            gift.gift_filter(ctx, h, gi, go)
        assert e.value.status == gift.GIFT_ERR_OOM
        gift.gift_ctx_debug_fail_alloc(ctx, 0)
        gift.gift_filter(ctx, h, gi, go)
        torch.cuda.synchronize()
        _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
        assert rel_err(go.cpu().numpy(), ref.reshape(g.shape), g).max() <= RTOL
    finally:
        gift.gift_graph_free(h)


def lane_tier_netlist(seed):
    """Rows that drive every width of the lane tier's sorting networks, one
    such row per warp (cells 0, 32, 64, ...), and the rows just past its
    caps: cell 0 in 32 two-pin nets and cell 32 in 20 (more than the 16
    incidences the lane tier takes: the warp tier), cell 64 in 16 (the
    incidence cap, 16 keys), cell 96 in 12; cell 128 in one net of 33 pins
    (32 keys, the raw-entry cap), cell 160 in two nets of 15 pins (28 keys),
    cell 192 in three of 9 (24), cell 224 in four of 6 (20); cells 256..258
    share a cell pair through runs of 2, 3 and 5 nets (summed in FP64 in net
    order), cell 288 holds a net twice (a repeated pin); the rest random
    small nets with repeats on cells 320..899."""
    nets = []
    for c, k in ((0, 32), (32, 20), (64, 16), (96, 12)):
        for t in range(k):
            nets.append([c, 320 + (7 * t + 13 * c) % 580])
    for c, count, pins in ((128, 1, 33), (160, 2, 15), (192, 3, 9), (224, 4, 6)):
        for t in range(count):
            nets.append([c] + [320 + (37 * t + 11 * q + c) % 580 for q in range(pins - 1)])
    for c, run in ((256, 2), (257, 3), (258, 5)):
        for r in range(run):
            nets.append([c, 330, 331 + r])  # cell pair (c, 330) in `run` nets of 3 pins
    nets.append([288, 340, 288, 341])  # cell 288 twice in one net
    small = synth.random_small(seed, 580, 900, 7, allow_repeat=True, min_pins=2)
    for e in range(small.num_nets):  # on cells 320..899, away from the rows above
        nets.append([320 + int(c) for c in small.pin_cell[small.net_ptr[e]:small.net_ptr[e + 1]]])
    order = synth.u64(seed, 91, np.arange(len(nets), dtype=np.uint64)).argsort(kind="stable")  # shuffle the net ids
    nets = [nets[i] for i in order]
    net_ptr = np.concatenate([[0], np.cumsum([len(n) for n in nets])]).astype(np.int64)
    pin_cell = np.array([c for n in nets for c in n], dtype=np.int32)
    return synth.Netlist(900, len(nets), net_ptr, pin_cell, np.zeros(900, np.uint8), np.zeros((900, 2), np.float32))


@pytest.mark.parametrize("wd", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("seed", [1, 2])
def test_lane_tier_network_widths(ctx, wd, seed):
    nl = lane_tier_netlist(seed)
    raw = np.zeros(nl.num_cells, dtype=np.int64)
    inc = np.zeros(nl.num_cells, dtype=np.int64)
    for e in range(nl.num_nets):
        cells = nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]
        for c in cells:
            raw[c] += len(cells) - 1
            inc[c] += 1
    # incidences past the lane tier's 16, at its cap, and below it
    assert (inc[0], inc[32], inc[64], inc[96]) == (32, 20, 16, 12)
    # keys: the raw-entry cap and the 28-, 24- and 20-key networks with few incidences
    assert (raw[128], raw[160], raw[192], raw[224]) == (32, 28, 24, 20)
    assert inc[128] == 1 and inc[160] == 2 and inc[192] == 3 and inc[224] == 4
    assert raw[320:].max() <= 512
    h = build(ctx, nl, wd)
    try:
        rp, col, val, deg = gift.gift_graph_export(h)
    finally:
        gift.gift_graph_free(h)
    og = oracle.stored(oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell), wd)
    np.testing.assert_array_equal(rp, og.row_ptr)
    np.testing.assert_array_equal(col, og.col)
    np.testing.assert_array_equal(val, og.val)
    np.testing.assert_array_equal(deg, oracle.degrees(og))
