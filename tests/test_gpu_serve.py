"""The request loop (gift_serve_*): continuous batching on one GPU.

Each request's result must be the same alone and in the mix: a request run by
itself through gift_build_graph + gift_filter + gift_hpwl (same schedule, same
weight type) and the same request served while others of different sizes
and weight types overlap on the device -- their filters sharing sweep
launches -- give bit-identical outputs (every row is computed as the
request's own filter computes it), and the FP32 requests match the FP64
oracle within the 1e-5 bar.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5
SERVE_SCHEDULE = 4244  # the server's fixed shape when spec.schedule is 0


def rel_err(got, ref, g):
    floor = 1e-3 * max(float(np.abs(g).max()), 1e-30)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)


def mix(num=12, seed=11):
    """Netlists of uneven sizes (log-uniform 2k..80k cells), S in {1, 2, 4}, FP32 and BF16."""
    u = synth.uniform(seed, synth.T_MISC, np.arange(3 * num, dtype=np.uint64)).reshape(num, 3)
    out = []
    for k in range(num):
        n = int(np.exp(np.log(2000) + u[k, 0] * (np.log(80000) - np.log(2000))))
        nf = max(1, n // 100)
        nl = synth.make_netlist(n - nf, nf, int(n * (1.0 + 0.2 * u[k, 1])), seed * 100 + k)
        S = (1, 2, 4)[k % 3]
        wd = "bf16" if k % 2 else "f32"
        out.append((nl, synth.make_signals(nl, S, seed * 100 + k), wd))
    return out


def alone(ctx, nl, g, wd, cut=0):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed), gift.WEIGHT[wd],
                              implicit_min_pins=cut)
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go, gift.make_spec(schedule=SERVE_SCHEDULE))
        hp = gift.gift_hpwl(ctx, h, go)
        torch.cuda.synchronize()
        return go.cpu().numpy(), hp
    finally:
        gift.gift_graph_free(h)


@pytest.fixture(scope="module")
def requests():
    return mix()


def submit_all(srv, reqs):
    return [gift.gift_serve_submit(srv, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g, gift.WEIGHT[wd])
            for nl, g, wd in reqs]


def test_results_same_alone_and_in_mix(requests):
    ctx = gift.gift_ctx_create(0)
    try:
        ref = [alone(ctx, nl, g, wd) for nl, g, wd in requests]
    finally:
        gift.gift_ctx_destroy(ctx)
    srv = gift.gift_serve_create(max_slots=4)
    try:
        tickets = submit_all(srv, requests)
        got = [gift.gift_serve_wait(srv, t, nl.num_cells, g.shape[1]) for t, (nl, g, _) in zip(tickets, requests)]
        st = gift.gift_serve_stats_get(srv)
    finally:
        gift.gift_serve_destroy(srv)
    for (nl, g, wd), (out, hp, rs), (out_a, hp_a) in zip(requests, got, ref):
        np.testing.assert_array_equal(out, out_a)  # same alone and in the mix
        np.testing.assert_array_equal(hp, hp_a)
        assert rs.weight_dtype == gift.WEIGHT[wd] and rs.num_signals == g.shape[1]
        assert rs.latency_ms >= rs.run_ms > 0 and rs.queue_ms >= 0
    assert st.completed == len(requests) and st.failed == 0 and st.waiting == 0 and st.running == 0
    assert st.peak_running >= 2  # requests overlapped
    assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
    assert st.edge_updates_per_s > 0 and st.requests_per_s > 0
    # the FP32 requests against the FP64 oracle
    for (nl, g, wd), (out, hp, _) in zip(requests[:4], got[:4]):
        if wd != "f32":
            continue
        _, _, o = oracle.run(nl, g.reshape(nl.num_cells, -1))
        assert rel_err(out, o.reshape(g.shape), g).max() <= RTOL
        np.testing.assert_allclose(hp, oracle.hpwl(nl.net_ptr, nl.pin_cell, out), rtol=1e-12)


def test_admission_respects_the_budget(requests):
    """With a budget of 1.5x the largest request's footprint, the admitted
    requests never hold more than the budget together, and results are
    unchanged."""
    reqs = requests[:6]
    big = max(reqs, key=lambda r: r[0].num_cells)
    probe = gift.gift_serve_create(max_slots=1)
    try:
        t = submit_all(probe, [big])[0]
        fp = gift.gift_serve_wait(probe, t, big[0].num_cells, big[1].shape[1])[2].footprint_bytes
    finally:
        gift.gift_serve_destroy(probe)
    budget = int(fp * 1.5)
    srv = gift.gift_serve_create(max_slots=4, hbm_budget_bytes=budget)
    try:
        tickets = submit_all(srv, reqs)
        outs = [gift.gift_serve_wait(srv, t, nl.num_cells, g.shape[1]) for t, (nl, g, _) in zip(tickets, reqs)]
        st = gift.gift_serve_stats_get(srv)
    finally:
        gift.gift_serve_destroy(srv)
    assert st.completed == len(reqs) and st.budget_bytes == budget
    assert 0 < st.peak_footprint_bytes <= budget
    ctx = gift.gift_ctx_create(0)
    try:
        for (nl, g, wd), (out, _, _) in zip(reqs, outs):
            np.testing.assert_array_equal(out, alone(ctx, nl, g, wd)[0])
    finally:
        gift.gift_ctx_destroy(ctx)


def test_oversized_and_invalid_requests_rejected(requests):
    nl, g, _ = requests[0]
    srv = gift.gift_serve_create(max_slots=2, hbm_budget_bytes=1 << 16)
    try:
        with pytest.raises(gift.GiftError) as e:  # footprint above the budget
            gift.gift_serve_submit(srv, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g)
        assert e.value.status == gift.GIFT_ERR_INVALID
    finally:
        gift.gift_serve_destroy(srv)
    srv = gift.gift_serve_create(max_slots=2)
    try:
        bad = nl.pin_cell.copy()
        bad[0] = nl.num_cells  # pin on a cell that does not exist
        with pytest.raises(gift.GiftError) as e:
            gift.gift_serve_submit(srv, nl.num_cells, nl.net_ptr, bad, nl.is_fixed, g)
        assert e.value.status == gift.GIFT_ERR_INVALID
        gn = g.copy()
        gn[0, 0, 0] = np.nan
        with pytest.raises(gift.GiftError):
            gift.gift_serve_submit(srv, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, gn)
        with pytest.raises(gift.GiftError) as e:
            gift.gift_serve_poll(srv, 12345, nl.num_cells, g.shape[1])
        assert e.value.status == gift.GIFT_ERR_INVALID
        t = gift.gift_serve_submit(srv, nl.num_cells, nl.net_ptr, nl.pin_cell, nl.is_fixed, g)
        r = None
        t0 = time.time()
        while r is None and time.time() - t0 < 60:  # poll until done
            r = gift.gift_serve_poll(srv, t, nl.num_cells, g.shape[1])
            time.sleep(0.001)
        assert r is not None
        with pytest.raises(gift.GiftError):  # a result is taken once
            gift.gift_serve_poll(srv, t, nl.num_cells, g.shape[1])
        assert gift.gift_serve_stats_get(srv).failed == 0
    finally:
        gift.gift_serve_destroy(srv)


def test_destroy_with_requests_pending(requests):
    srv = gift.gift_serve_create(max_slots=1)
    submit_all(srv, requests)  # most are still waiting when the server stops
    gift.gift_serve_destroy(srv)  # cancels the waiting ones, lets the running one finish


def test_implicit_cliques_in_the_mix(requests):
    """Requests built with implicit cliques (nets of 6+ pins) give the same
    results as the same builds alone."""
    ctx = gift.gift_ctx_create(0)
    try:
        ref = [alone(ctx, nl, g, wd, cut=6) for nl, g, wd in requests[:6]]
    finally:
        gift.gift_ctx_destroy(ctx)
    srv = gift.gift_serve_create(max_slots=3, implicit_min_pins=6)
    try:
        tickets = submit_all(srv, requests[:6])
        got = [gift.gift_serve_wait(srv, t, nl.num_cells, g.shape[1]) for t, (nl, g, _) in zip(tickets, requests[:6])]
    finally:
        gift.gift_serve_destroy(srv)
    for (out, hp, _), (out_a, hp_a) in zip(got, ref):
        np.testing.assert_array_equal(out, out_a)
        np.testing.assert_array_equal(hp, hp_a)


@pytest.mark.parametrize("separate,window", [(0, 0), (0, 20000), (1, 0)])
def test_burst_shares_filter_launches(requests, separate, window):
    """A burst of requests: with shared filters (the default) several
    requests run per launch -- FP32 and BF16 graphs in the same launch,
    requests grouped by their number of signals -- and every result is still
    bit-identical to the request alone (a batch window of 20 ms makes the
    batches gather); with separate_filters = 1 every request runs its own
    launches."""
    reqs = requests * 3  # 36 requests, S in {1, 2, 4}, both weight types
    ctx = gift.gift_ctx_create(0)
    try:
        ref = [alone(ctx, nl, g, wd) for nl, g, wd in requests]
    finally:
        gift.gift_ctx_destroy(ctx)
    srv = gift.gift_serve_create(max_slots=16, separate_filters=separate, batch_window_us=window)
    try:
        tickets = submit_all(srv, reqs)
        got = [gift.gift_serve_wait(srv, t, nl.num_cells, g.shape[1]) for t, (nl, g, _) in zip(tickets, reqs)]
        st = gift.gift_serve_stats_get(srv)
    finally:
        gift.gift_serve_destroy(srv)
    for k, (out, hp, _) in enumerate(got):
        np.testing.assert_array_equal(out, ref[k % len(requests)][0])
        np.testing.assert_array_equal(hp, ref[k % len(requests)][1])
    assert st.completed == len(reqs) and st.failed == 0
    if separate:
        assert st.batches == 0 and st.batched_requests == 0
    else:
        assert st.batched_requests == len(reqs) and st.peak_batch <= 16
        if window:
            assert st.batches < len(reqs) and st.peak_batch >= 2  # requests shared launches


def test_compensated_spec_runs_unbatched(requests):
    """A server whose spec asks for compensated sums filters each request on
    its own (warp-row kernels); the results equal the request's own
    compensated filter."""
    reqs = requests[:4]
    spec = gift.make_spec(compensated=True)
    ctx = gift.gift_ctx_create(0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ref = []
    try:
        for nl, g, wd in reqs:
            h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                                      gift.WEIGHT[wd])
            gi = dev(g)
            go = torch.empty_like(gi)
            s2 = gift.make_spec(compensated=True, schedule=SERVE_SCHEDULE)
            gift.gift_filter(ctx, h, gi, go, s2)
            torch.cuda.synchronize()
            ref.append(go.cpu().numpy())
            gift.gift_graph_free(h)
    finally:
        gift.gift_ctx_destroy(ctx)
    srv = gift.gift_serve_create(max_slots=4, spec=spec)
    try:
        tickets = submit_all(srv, reqs)
        got = [gift.gift_serve_wait(srv, t, nl.num_cells, g.shape[1]) for t, (nl, g, _) in zip(tickets, reqs)]
        st = gift.gift_serve_stats_get(srv)
    finally:
        gift.gift_serve_destroy(srv)
    for (out, _, _), r in zip(got, ref):
        np.testing.assert_array_equal(out, r)
    assert st.batches == 0
