"""Bounded device waits: every mbarrier wait of the TMA sweep pipeline gives up
after a limit and records GIFT_ERR_TIMEOUT in the context's device error word
instead of hanging.  The test makes the waits run out the allowed way -- a
short limit, and a producer that announces its stages without issuing their
copies, so no copy is ever in flight -- then checks that the error is
reported once, through gift_ctx_device_status and through a host-memory call,
and that the next normal call succeeds with correct results."""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5
TMA = 2016  # TMA gather4 pipeline, 16-column slab (K = 16: 8 signals)


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_debug_waits(c, 0, False)
    gift.gift_ctx_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_wait_runs_out_then_recovers(ctx):
    nl, _ = synth.workload("plain-10k")
    g = synth.make_signals(nl, 8, 17)
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed))
    spec = gift.make_spec(schedule=TMA)
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_ctx_device_status(ctx)  # clean to begin with
        gift.gift_ctx_debug_waits(ctx, 2000, True)
        try:
            gift.gift_filter(ctx, h, gi, go, spec)  # device memory: queued, returns at once
            with pytest.raises(gift.GiftError) as e:
                gift.gift_ctx_device_status(ctx)
            assert e.value.status == gift.GIFT_ERR_TIMEOUT
            gift.gift_ctx_device_status(ctx)  # reported once: the word is clear again
            out = np.empty_like(g)
            with pytest.raises(gift.GiftError) as e:  # a host-memory call checks the word itself
                gift.gift_filter(ctx, h, g, out, spec)
            assert e.value.status == gift.GIFT_ERR_TIMEOUT
        finally:
            gift.gift_ctx_debug_waits(ctx, 0, False)
        gift.gift_ctx_device_status(ctx)
        gift.gift_filter(ctx, h, gi, go, spec)
        torch.cuda.synchronize()
        gift.gift_ctx_device_status(ctx)
        got = go.cpu().numpy()
    finally:
        gift.gift_graph_free(h)
    _, _, ref = oracle.run(nl, g.reshape(nl.num_cells, -1))
    floor = 1e-3 * np.abs(g).max()
    err = np.abs(got.reshape(nl.num_cells, -1).astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)
    assert err.max() <= RTOL
