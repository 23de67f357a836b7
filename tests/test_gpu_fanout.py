"""The high-fanout workload at full size (1.3M cells, Zipf(2.2) pin counts
capped at 2,000: 828M expanded nonzeros, rows of up to 10,600), expanded and
with implicit cliques, against values computed from the netlist alone.

The FP64 oracle cannot expand this netlist in test time, so:
- one sweep (A~_2 x) is checked on sampled rows -- the longest rows and a
  seeded random sample -- each computed by its definition in FP64 on the
  CPU (row i sums, over its pins' nets e, (2/M_e) s_q x_q over the net's pins
  q on other cells, s = (d + sigma)^-1/2 with the exact degrees of the
  netlist);
- the filter's fixed point: A~_4^4 (d + 4)^1/2 = (d + 4)^1/2 (Theorem 1);
- the filter operator without reimposed cells is symmetric.
"""
import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def fanout():
    nl, _ = synth.workload("fanout-1.3m")
    # exact degrees of the full expansion: every net's clique, from the netlist
    d = oracle.implicit_degrees(np.zeros(nl.num_cells), nl.net_ptr, nl.pin_cell, cut=2)
    order = np.argsort(nl.pin_cell, kind="stable")
    pin_net = np.repeat(np.arange(nl.num_nets, dtype=np.int64), np.diff(nl.net_ptr))
    inc_ptr = np.concatenate([[0], np.cumsum(np.bincount(nl.pin_cell, minlength=nl.num_cells))]).astype(np.int64)
    inc_net = pin_net[order]
    u = synth.uniform(2024, synth.T_MISC, np.arange(200, dtype=np.uint64))
    rows = np.unique(np.concatenate([np.argsort(-d)[:40], (u * nl.num_cells).astype(np.int64)]))
    return nl, d, inc_ptr, inc_net, rows


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


def rows_by_definition(nl, d, inc_ptr, inc_net, sigma, x, rows):
    s = 1.0 / np.sqrt(d + sigma)
    out = np.empty((len(rows), x.shape[1]))
    for r, i in enumerate(rows):
        acc = np.zeros(x.shape[1])
        for e in inc_net[inc_ptr[i]:inc_ptr[i + 1]]:  # once per pin of cell i in net e
            pins = nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]
            q = pins[pins != i]
            acc += (2.0 / len(pins)) * (s[q, None] * x[q]).sum(axis=0)
        acc += sigma * s[i] * x[i]
        out[r] = s[i] * acc
    return out


def run(ctx, nl, cut, g, spec):
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                              implicit_min_pins=cut)
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go, spec)
        torch.cuda.synchronize()
        gift.gift_ctx_device_status(ctx)
        return go.cpu().numpy()
    finally:
        gift.gift_graph_free(h)


CASES = [(0, False), (0, True), (8, False), (64, True)]  # (implicit_min_pins, compensated)


@pytest.mark.parametrize("cut,comp", CASES)
def test_one_sweep_on_sampled_rows(ctx, fanout, cut, comp):
    nl, d, inc_ptr, inc_net, rows = fanout
    g = synth.make_signals(nl, 2, 5)
    spec = gift.make_spec(terms=((2.0, 1, 1.0),), reimpose=False, compensated=comp)
    got = run(ctx, nl, cut, g, spec).reshape(nl.num_cells, -1)
    x = g.reshape(nl.num_cells, -1).astype(np.float64)
    ref = rows_by_definition(nl, d, inc_ptr, inc_net, 2.0, x, rows)
    floor = 1e-3 * np.abs(x).max()
    err = np.abs(got[rows] - ref) / np.maximum(np.abs(ref), floor)
    assert err.max() <= RTOL


@pytest.mark.parametrize("cut,comp", CASES)
def test_theorem1_fixed_point(ctx, fanout, cut, comp):
    nl, d = fanout[0], fanout[1]
    v = np.sqrt(d + 4.0).astype(np.float32)
    g = np.stack([np.stack([v, v], axis=1), np.stack([2 * v, 3 * v], axis=1)], axis=1)  # [N][2][2]
    spec = gift.make_spec(terms=((4.0, 4, 1.0),), reimpose=False, compensated=comp)
    got = run(ctx, nl, cut, g, spec)
    assert np.abs(got.astype(np.float64) / g - 1.0).max() <= 4 * RTOL


@pytest.mark.parametrize("cut,comp", [(0, False), (8, False)])
def test_filter_is_symmetric(ctx, fanout, cut, comp):
    nl = fanout[0]
    u = synth.make_signals(nl, 2, 8)  # columns: u_x, u_y, v_x, v_y
    spec = gift.make_spec(reimpose=False, compensated=comp)
    Gu = run(ctx, nl, cut, u, spec).reshape(nl.num_cells, -1).astype(np.float64)
    x = u.reshape(nl.num_cells, -1).astype(np.float64)
    for a, b in ((0, 2), (1, 3)):
        lhs, rhs = np.dot(Gu[:, a], x[:, b]), np.dot(x[:, a], Gu[:, b])
        assert abs(lhs - rhs) <= RTOL * abs(lhs)
