"""Implicit cliques (build option implicit_min_pins): the nets of at least T
pins stay out of the CSR and every sweep applies their cliques through net
sums -- the same operator as the full expansion.

Bars: the CSR of the smaller nets, its stored weights and the degrees (CSR
part plus the implicit cliques' part) bit-exact against the oracle's cut
expansion and implicit degrees; the filter within 1e-5 of the FP64 oracle
of the full expansion (FP32 weights), and within 8u + 2e-5 for BF16 weights
(the implicit part is not rounded to the storage type, the CSR part is).
"""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


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


def netlists():
    from tests.test_gpu_parity import star_netlist
    return {
        "plain-10k": synth.workload("plain-10k")[0],
        "repeat-cells": synth.random_small(3, 300, 420, 9, num_fixed=10, allow_repeat=True),
        "zipf-20k": synth.make_netlist(19_800, 200, 22_000, 77, law="zipf", cap=400),
        "block-tier-row": star_netlist(1000, 20, 40, 8, extra_nets=300),
        "single-pin-nets": synth.random_small(6, 20, 30, 1),
    }


NETLISTS = netlists()
REF = {}


def exact(name, g):
    """FP64 oracle of the full expansion for the netlist and signal."""
    nl = NETLISTS[name]
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    return ref.reshape(g.shape)


def build(ctx, nl, cut, wd="f32"):
    return gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                                 gift.WEIGHT[wd], implicit_min_pins=cut)


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("cut", [2, 3, 8, 40])
@pytest.mark.parametrize("wd", ["f32", "bf16"])
def test_structure_and_degrees_bit_exact(ctx, name, cut, wd):
    nl = NETLISTS[name]
    h = build(ctx, nl, cut, wd)
    try:
        rp, col, val, deg = gift.gift_graph_export(h)
        info = gift.gift_graph_info(h)
    finally:
        gift.gift_graph_free(h)
    G = oracle.stored(oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut), wd)
    np.testing.assert_array_equal(rp, G.row_ptr)
    np.testing.assert_array_equal(col, G.col)
    np.testing.assert_array_equal(val, G.val)
    d = oracle.implicit_degrees(oracle.degrees(G), nl.net_ptr, nl.pin_cell, cut)
    np.testing.assert_array_equal(deg, d)
    M = np.diff(nl.net_ptr)
    big = M >= cut
    assert info.implicit_min_pins == cut
    assert info.implicit_nets == int(big.sum()) and info.implicit_pins == int(M[big].sum())


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("cut", [3, 8, 40])
@pytest.mark.parametrize("S", [1, 4, 8])
@pytest.mark.parametrize("schedule", [0, 408, 1016, 3008, 4244, 4644, 14244, 4844, 6444, 16444])
def test_filter_matches_full_expansion(ctx, name, cut, S, schedule):
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 300 + S)
    key = (name, S)
    if key not in REF:
        REF[key] = exact(name, g)
    h = build(ctx, nl, cut)
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go, gift.make_spec(schedule=schedule))
        torch.cuda.synchronize()
        got = go.cpu().numpy()
    finally:
        gift.gift_graph_free(h)
    assert rel_err(got, REF[key], g).max() <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])


@pytest.mark.parametrize("name", ["zipf-20k", "repeat-cells"])
def test_compensated_bf16_noalloc_and_tma(ctx, name):
    nl = NETLISTS[name]
    g = synth.make_signals(nl, 8, 41)
    ref = exact(name, g)
    h = build(ctx, nl, 8)
    hb = build(ctx, nl, 8, "bf16")
    try:
        gi = dev(g)
        outs = {}
        for tag, spec, graph in [("comp", gift.make_spec(compensated=True), h), ("tma", gift.make_spec(schedule=2016), h),
                                 ("bf16", gift.make_spec(), hb), ("plain", gift.make_spec(schedule=4244), h)]:
            go = torch.empty_like(gi)
            gift.gift_filter(ctx, graph, gi, go, spec)
            outs[tag] = go
        na = torch.empty_like(gi)
        gift.gift_filter_noalloc(ctx, h, gi, na, gift.make_spec(schedule=4244))
        torch.cuda.synchronize()
        gift.gift_ctx_device_status(ctx)
    finally:
        gift.gift_graph_free(h)
        gift.gift_graph_free(hb)
    for tag in ("comp", "tma", "plain"):
        assert rel_err(outs[tag].cpu().numpy(), ref, g).max() <= RTOL, tag
    assert rel_err(outs["bf16"].cpu().numpy(), ref, g).max() <= 8 * 2.0 ** -9 + 2 * RTOL
    np.testing.assert_array_equal(na.cpu().numpy(), outs["plain"].cpu().numpy())


def test_batch_with_implicit_cliques(ctx):
    batch = [(NETLISTS[n], synth.make_signals(NETLISTS[n], 4, 9)) for n in ("zipf-20k", "repeat-cells", "plain-10k")]
    nets = [(nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed)) for nl, _ in batch]
    hb, offs = gift.gift_build_batch(ctx, nets, implicit_min_pins=8)
    try:
        sig = dev(np.concatenate([g for _, g in batch], axis=0))
        out = torch.empty_like(sig)
        gift.gift_filter(ctx, hb, sig, out, gift.make_spec(schedule=4244))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        gift.gift_graph_free(hb)
    for b, (nl, g) in enumerate(batch):
        h = build(ctx, nl, 8)
        try:
            gi = dev(g)
            go = torch.empty_like(gi)
            gift.gift_filter(ctx, h, gi, go, gift.make_spec(schedule=4244))
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got[offs[b]:offs[b + 1]], go.cpu().numpy())
        finally:
            gift.gift_graph_free(h)


def test_bad_option_rejected(ctx):
    nl = NETLISTS["plain-10k"]
    with pytest.raises(gift.GiftError) as e:
        build(ctx, nl, 1)
    assert e.value.status == gift.GIFT_ERR_INVALID
