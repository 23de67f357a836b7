"""gift_filter_noalloc: the filter for callers that cannot allocate device
memory while they filter (a budget set aside in advance, real-time loops,
hosts that own the allocator).  Its scratch is the library's fixed device
area, so its output must equal gift_filter's on the same inputs -- also on
repeated calls, which find the previous call's data in that area.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5  # the FP32 filter tolerance used by the parity tests


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, ref):
    floor = 1e-3 * max(float(np.abs(ref).max()), 1e-30)
    return float((np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)).max())


def _graph(ctx, nl):
    return gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed))


@pytest.mark.parametrize("S", [1, 8])
def test_noalloc_matches_gift_filter_twice(ctx, S):
    nl, _ = synth.workload("plain-10k")
    other = synth.random_small(7, 500, 600, 8, num_fixed=5)
    g = synth.make_signals(nl, S, 77 + S)
    go = synth.make_signals(other, S, 5)
    h, h2 = _graph(ctx, nl), _graph(ctx, other)
    try:
        gi = dev(g)
        ref = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy().astype(np.float64)
        outs = []
        for _ in range(2):  # two calls in a row on the shared scratch
            out = torch.full_like(gi, float("nan"))
            gift.gift_filter_noalloc(ctx, h, gi, out)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        # another graph in between, then the first again
        oi = dev(go)
        oo = torch.empty_like(oi)
        gift.gift_filter_noalloc(ctx, h2, oi, oo)
        out = torch.empty_like(gi)
        gift.gift_filter_noalloc(ctx, h, gi, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
        gift.gift_ctx_device_status(ctx)
    finally:
        gift.gift_graph_free(h)
        gift.gift_graph_free(h2)
    for o in outs:
        assert np.isfinite(o).all()
        assert rel_err(o, ref) <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(outs[0][fx], g[fx])


def test_noalloc_rejects_too_large(ctx):
    nl, _ = synth.workload("plain-10k")
    # N x S x 8 bytes per signal buffer; 5 buffers at S = 400 exceed the 64 MiB area
    S = 400
    g = dev(synth.make_signals(nl, S, 1))
    out = torch.empty_like(g)
    h = _graph(ctx, nl)
    try:
        with pytest.raises(gift.GiftError) as e:
            gift.gift_filter_noalloc(ctx, h, g, out)
        assert e.value.status == gift.GIFT_ERR_INVALID
        assert "scratch" in str(e.value)
    finally:
        gift.gift_graph_free(h)
