"""Batches: many uneven netlists as one block-diagonal graph, filtered by the
same launches, and a filter replayed as one CUDA-graph launch.

Graph b's rows of the batch are the rows of graph b built alone (columns
offset by its first cell): structure, weights and degrees bit-identical.
With the same kernel shape the batch filter gives bit-identical per-graph
results; every graph matches the FP64 oracle within 1e-5; per-graph HPWL
matches gift_hpwl on the graph alone within 1e-12 (FP64 sums in another
order).
"""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5
SCHEDULE = 4244


def rel_err(got, ref, g):
    floor = 1e-3 * max(float(np.abs(g).max()), 1e-30)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


@pytest.fixture(scope="module")
def batch():
    """12 graphs, cells log-uniform in [500, 20000], S = 4 (the batched law, scaled down),
    plus a graph without nets and a one-cell graph."""
    out = synth.batch_workload(num_graphs=12, lo=500, hi=20_000, S=4)
    empty = synth.random_small(21, 40, 0, 3)
    out.insert(3, (empty, synth.make_signals(empty, 4, 3)))
    one = synth.Netlist(1, 1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                        np.zeros(1, np.uint8), np.zeros((1, 2), np.float32))
    out.insert(7, (one, synth.make_signals(one, 4, 4)))
    return out


def build_batch(ctx, batch, wd="f32", device=True):
    conv = dev if device else (lambda a: a)
    nets = [(nl.num_cells, conv(nl.net_ptr), conv(nl.pin_cell), conv(nl.is_fixed)) for nl, _ in batch]
    return gift.gift_build_batch(ctx, nets, gift.WEIGHT[wd])


def alone(ctx, nl, g, wd="f32"):
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed), gift.WEIGHT[wd])
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go, gift.make_spec(schedule=SCHEDULE))
        hp = gift.gift_hpwl(ctx, h, go)
        torch.cuda.synchronize()
        return h, go.cpu().numpy(), hp
    except Exception:
        gift.gift_graph_free(h)
        raise


@pytest.mark.parametrize("device", [True, False])
@pytest.mark.parametrize("wd", ["f32", "bf16"])
def test_batch_equals_graphs_alone(ctx, batch, device, wd):
    h, offs = build_batch(ctx, batch, wd, device)
    try:
        np.testing.assert_array_equal(offs, np.concatenate([[0], np.cumsum([nl.num_cells for nl, _ in batch])]))
        rp, col, val, deg = gift.gift_graph_export(h)
        sig = np.concatenate([g for _, g in batch], axis=0)
        gi = dev(sig)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go, gift.make_spec(schedule=SCHEDULE))
        hp = gift.gift_hpwl_batch(ctx, h, go, len(batch))
        torch.cuda.synchronize()
        out = go.cpu().numpy()
    finally:
        gift.gift_graph_free(h)
    for b, (nl, g) in enumerate(batch):
        c0, c1 = offs[b], offs[b + 1]
        hb, out_b, hp_b = alone(ctx, nl, g, wd)
        try:
            rpb, colb, valb, degb = gift.gift_graph_export(hb)
        finally:
            gift.gift_graph_free(hb)
        # rows of graph b: same structure (columns offset), weights and degrees
        np.testing.assert_array_equal(rp[c0:c1 + 1] - rp[c0], rpb)
        np.testing.assert_array_equal(col[rp[c0]:rp[c1]] - c0, colb)
        np.testing.assert_array_equal(val[rp[c0]:rp[c1]], valb)
        np.testing.assert_array_equal(deg[c0:c1], degb)
        # same launches for all graphs, bit-identical per graph
        np.testing.assert_array_equal(out[c0:c1], out_b)
        np.testing.assert_allclose(hp[b], hp_b, rtol=1e-12)
        if wd == "f32":
            _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
            assert rel_err(out[c0:c1], ref.reshape(g.shape), g).max() <= RTOL
            np.testing.assert_allclose(hp[b], oracle.hpwl(nl.net_ptr, nl.pin_cell, out[c0:c1]), rtol=1e-12)


def test_hpwl_batch_on_a_single_graph_equals_gift_hpwl(ctx, batch):
    nl, g = batch[0]
    h, out, hp = alone(ctx, nl, g)
    try:
        one = gift.gift_hpwl_batch(ctx, h, dev(out), 1)
    finally:
        gift.gift_graph_free(h)
    np.testing.assert_allclose(one[0], hp, rtol=1e-12)


@pytest.mark.parametrize("schedule", [0, SCHEDULE, 3008, 408])
def test_captured_filter_replays(ctx, batch, schedule):
    h, offs = build_batch(ctx, batch)
    try:
        sig = np.concatenate([g for _, g in batch], axis=0)
        gi = dev(sig)
        ref = torch.empty_like(gi)
        spec = gift.make_spec(schedule=schedule)
        gift.gift_filter(ctx, h, gi, ref, spec)
        go = torch.full_like(gi, float("nan"))
        ex = gift.gift_filter_capture(ctx, h, gi, go, spec)
        try:
            go.fill_(float("nan"))
            gift.gift_exec_launch(ex, torch.cuda.current_stream())
            torch.cuda.synchronize()
            np.testing.assert_array_equal(go.cpu().numpy(), ref.cpu().numpy())
            # new signals in the same buffer, replay again
            sig2 = sig[:, ::-1, :].copy()
            gi.copy_(torch.from_numpy(sig2))
            gift.gift_exec_launch(ex, torch.cuda.current_stream())
            ref2 = torch.empty_like(gi)
            gift.gift_filter(ctx, h, dev(sig2), ref2, spec)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(go.cpu().numpy(), ref2.cpu().numpy())
        finally:
            gift.gift_exec_free(ex)
    finally:
        gift.gift_graph_free(h)


@pytest.mark.parametrize("device", [True, False])
def test_batch_rejects_pins_outside_their_netlist(ctx, batch, device):
    nl, g = batch[1]
    bad = nl.pin_cell.copy()
    bad[-1] = nl.num_cells  # a cell of the next graph, not of this one
    conv = dev if device else (lambda a: a)
    nets = [(n.num_cells, conv(n.net_ptr), conv(n.pin_cell), conv(n.is_fixed)) for n, _ in batch]
    nets[1] = (nl.num_cells, conv(nl.net_ptr), conv(bad), conv(nl.is_fixed))
    with pytest.raises(gift.GiftError) as e:
        gift.gift_build_batch(ctx, nets)
    assert e.value.status == gift.GIFT_ERR_INVALID


def test_gift_run_equals_separate_calls(ctx, batch):
    """gift_run (host netlist and signal, upload overlapping the build) gives
    the same output and HPWL as build + filter + HPWL called one by one; an
    invalid netlist is rejected and leaves the context usable."""
    nl, g = batch[0]
    out = np.empty_like(g)
    hp = gift.gift_run(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g, out)
    h = gift.gift_build_graph(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed)
    try:
        ref = np.empty_like(g)
        gift.gift_filter(ctx, h, g, ref)
        hp_ref = gift.gift_hpwl(ctx, h, ref)
    finally:
        gift.gift_graph_free(h)
    np.testing.assert_array_equal(out, ref)
    np.testing.assert_array_equal(hp, hp_ref)
    bad = nl.pin_cell.copy()
    bad[0] = nl.num_cells + 5
    with pytest.raises(gift.GiftError) as e:
        gift.gift_run(ctx, nl.num_cells, nl.net_ptr, bad, nl.is_fixed, g, out)
    assert e.value.status == gift.GIFT_ERR_INVALID
    hp2 = gift.gift_run(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g, out,
                        implicit_min_pins=4, weight_dtype=gift.GIFT_WEIGHT_BF16)
    assert np.all(np.isfinite(hp2)) and np.all(np.isfinite(out))


def test_results_written_straight_to_pinned_host_memory(ctx, batch):
    """Page-locked output: the last sweep stores the result into it directly
    (no copy after the filter).  Same bits as pageable output, through
    gift_run and through gift_filter with host buffers, for every kernel
    family's epilogue."""
    nl, g = batch[0]
    pinned = torch.empty(g.shape, dtype=torch.float32).pin_memory()
    out_p = pinned.numpy()
    out = np.empty_like(g)
    hp_p = gift.gift_run(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g, out_p)
    hp = gift.gift_run(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g, out)
    np.testing.assert_array_equal(out_p, out)
    np.testing.assert_array_equal(hp_p, hp)
    h = gift.gift_build_graph(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed)
    try:
        for schedule in (0, 408, 1004, 3008, 4244, 4644, 4844, 6444):
            spec = gift.make_spec(schedule=schedule)
            ref = np.empty_like(g)
            gift.gift_filter(ctx, h, g, ref, spec)
            out_p[...] = np.nan
            gift.gift_filter(ctx, h, g, out_p, spec)
            np.testing.assert_array_equal(out_p, ref)
    finally:
        gift.gift_graph_free(h)


def test_nonfinite_host_signals_rejected(ctx, batch):
    """A NaN or an infinity in a host signal: GIFT_ERR_INVALID from gift_filter
    (host memory) and gift_run, the output left untouched, the context
    usable afterwards."""
    nl, g = batch[0]
    h = gift.gift_build_graph(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed)
    try:
        for val in (np.nan, np.inf, -np.inf):
            bad = g.copy()
            bad[nl.num_cells // 2, 0, 1] = val
            out = np.full_like(g, 7.0)
            with pytest.raises(gift.GiftError) as e:
                gift.gift_filter(ctx, h, bad, out)
            assert e.value.status == gift.GIFT_ERR_INVALID
            assert np.all(out == 7.0)
            with pytest.raises(gift.GiftError) as e:
                gift.gift_run(ctx, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, bad, out)
            assert e.value.status == gift.GIFT_ERR_INVALID
            assert np.all(out == 7.0)
        ref = np.empty_like(g)
        gift.gift_filter(ctx, h, g, ref)
        assert np.all(np.isfinite(ref))
    finally:
        gift.gift_graph_free(h)
