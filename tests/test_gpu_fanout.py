"""The high-fanout workload at full size (1.3M cells, Zipf(2.2) pin counts
capped at 2,000: 828M expanded nonzeros, rows of up to 10,600), expanded and
with implicit cliques, against the FP64 oracle.

The oracle applies the cliques of the nets of 8 or more pins from the netlist
(oracle.run with cut = 8: the same operator as the full expansion, whose 828M
FP64 pairs it could not sort in test time) and expands the rest; it filters
signal 0 of the GPU run, every cell, and the GPU's whole filter output (all
three terms, fixed cells) is compared element by element at the FP32 bar.
Also checked: the filter's fixed point A~_4^4 (d + 4)^1/2 = (d + 4)^1/2
(Theorem 1) and the symmetry of the filter operator without reimposed cells.
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


ORACLE_CUT = 8  # nets of at least this many pins: cliques applied from the netlist by the oracle


@pytest.fixture(scope="module")
def fanout():
    nl, g = synth.workload("fanout-1.3m")
    # exact degrees of the full expansion: every net's clique, from the netlist
    d = oracle.implicit_degrees(np.zeros(nl.num_cells), nl.net_ptr, nl.pin_cell, cut=2)
    # the FP64 filter of signal 0 (x and y of every cell)
    _, _, ref = oracle.run(nl, np.ascontiguousarray(g[:, 0, :]), cut=ORACLE_CUT)
    return nl, d, g, ref


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


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


@pytest.mark.parametrize("cut,comp", CASES + [(2, False)])
def test_whole_filter_against_oracle(ctx, fanout, cut, comp):
    """The paper's filter on all 4 signals, expanded or with implicit
    cliques, plain or compensated sums: signal 0 of every cell against the
    FP64 oracle, fixed cells bit-exact."""
    nl, _, g, ref = fanout
    got = run(ctx, nl, cut, g, gift.make_spec(compensated=comp))
    x0 = g[:, 0, :].astype(np.float64)
    floor = 1e-3 * np.abs(x0).max()
    err = np.abs(got[:, 0, :].astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)
    assert err.max() <= RTOL
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])


@pytest.fixture(scope="module")
def fanout_bf16(fanout):
    """The oracle with the expanded nets' weights rounded to bfloat16 (the
    implicit cliques keep 2/M), degrees over those weights."""
    nl, _, g, _ = fanout
    return oracle.run(nl, np.ascontiguousarray(g[:, 0, :]), fmt="bf16", cut=ORACLE_CUT)[2]


@pytest.mark.parametrize("cut", [0, ORACLE_CUT])
def test_bf16_weights_against_oracle(ctx, fanout, fanout_bf16, cut):
    """BF16 weights: with the oracle's cut the GPU computes the same rounded
    operator (FP32 bar); fully expanded, every weight is rounded, and the
    result stays within the derived bound 8u + the FP32 bar of the exact
    filter (u = 2^-8)."""
    nl, _, g, ref = fanout
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                              gift.GIFT_WEIGHT_BF16, implicit_min_pins=cut)
    try:
        gi = dev(g)
        go = torch.empty_like(gi)
        gift.gift_filter(ctx, h, gi, go)
        torch.cuda.synchronize()
        got = go.cpu().numpy()[:, 0, :].astype(np.float64)
    finally:
        gift.gift_graph_free(h)
    floor = 1e-3 * np.abs(g[:, 0, :]).max()
    if cut == ORACLE_CUT:
        err = np.abs(got - fanout_bf16) / np.maximum(np.abs(fanout_bf16), floor)
        assert err.max() <= RTOL
    else:
        err = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
        assert err.max() <= 8 * 2.0 ** -8 + RTOL


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
