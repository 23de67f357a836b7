"""gift_filter_noalloc: the filter for callers that cannot allocate device
memory while they filter (a budget set aside in advance, real-time loops,
hosts that own the allocator).  Its scratch is the library's fixed device
area, so its output must equal gift_filter's on the same inputs -- also on
repeated calls, which find the previous call's data in that area -- and
match the FP64 oracle within the FP32 filter tolerance.

That the call allocates nothing is checked with the context's allocation
fault injection: a failure armed for the next device allocation must still
be pending after the no-alloc calls, and the next gift_filter (which does
allocate) must hit it.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
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


def _graph(ctx, nl, implicit_min_pins=0):
    return gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                                 implicit_min_pins=implicit_min_pins)


def _noalloc_armed(ctx, h, gi, out, spec=None):
    """One no-alloc call with a device-allocation failure armed: the call must
    succeed and leave the failure pending for the next allocating call."""
    gift.gift_ctx_debug_fail_alloc(ctx, 1)
    try:
        gift.gift_filter_noalloc(ctx, h, gi, out, spec)
        torch.cuda.synchronize()
        probe_in = torch.zeros_like(gi)
        probe_out = torch.empty_like(gi)
        with pytest.raises(gift.GiftError) as e:
            gift.gift_filter(ctx, h, probe_in, probe_out, spec)
        assert e.value.status == gift.GIFT_ERR_OOM and "injected" in str(e.value)
    finally:
        gift.gift_ctx_debug_fail_alloc(ctx, 0)


@pytest.mark.parametrize("S", [1, 8])
def test_noalloc_matches_gift_filter_twice(ctx, S):
    nl, _ = synth.workload("plain-10k")
    other = synth.random_small(7, 500, 600, 8, num_fixed=5)
    g = synth.make_signals(nl, S, 77 + S)
    go = synth.make_signals(other, S, 5)
    exact = oracle.run(nl, g.reshape(nl.num_cells, -1))[2].reshape(g.shape)
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
            _noalloc_armed(ctx, h, gi, out)
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
    assert rel_err(ref.astype(np.float32), exact) <= RTOL
    for o in outs:
        assert np.isfinite(o).all()
        assert rel_err(o, ref) <= RTOL
        assert rel_err(o, exact) <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(outs[0][fx], g[fx])


@pytest.mark.parametrize("case", ["implicit", "compensated", "random-walk"])
def test_noalloc_other_forms_against_oracle(ctx, case):
    """Net sums of implicit cliques, compensated warp rows and the random-walk
    normalisation all run on the fixed area too."""
    nl = synth.random_small(11, 3000, 3300, 40, num_fixed=30)
    S = 4
    g = synth.make_signals(nl, S, 123)
    norm = "rw" if case == "random-walk" else "sym"
    exact = oracle.run(nl, g.reshape(nl.num_cells, -1), norm=norm)[2].reshape(g.shape)
    spec = gift.make_spec(norm=gift.GIFT_NORM_RW if case == "random-walk" else gift.GIFT_NORM_SYM,
                          compensated=case == "compensated")
    h = _graph(ctx, nl, implicit_min_pins=6 if case == "implicit" else 0)
    try:
        if case == "implicit":
            assert gift.gift_graph_info(h).implicit_nets > 0
        gi = dev(g)
        ref = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, ref, spec)
        outs = []
        for _ in range(2):
            out = torch.full_like(gi, float("nan"))
            _noalloc_armed(ctx, h, gi, out, spec)
            outs.append(out.cpu().numpy())
        ref = ref.cpu().numpy()
    finally:
        gift.gift_graph_free(h)
    for o in outs:
        assert rel_err(o, ref.astype(np.float64)) <= RTOL
        assert rel_err(o, exact) <= RTOL


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


def test_noalloc_rejects_bad_term_count(ctx):
    """A spec whose num_terms is beyond the term array is refused before the
    terms are read."""
    nl = synth.random_small(2, 200, 240, 6)
    g = dev(synth.make_signals(nl, 1, 3))
    out = torch.empty_like(g)
    h = _graph(ctx, nl)
    try:
        for n in (0, gift.GIFT_MAX_TERMS + 1, 1 << 20):
            spec = gift.make_spec()
            spec.num_terms = n
            with pytest.raises(gift.GiftError) as e:
                gift.gift_filter_noalloc(ctx, h, g, out, spec)
            assert e.value.status == gift.GIFT_ERR_INVALID
            assert "num_terms" in str(e.value)
    finally:
        gift.gift_graph_free(h)
