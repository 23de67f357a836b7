"""gift_tikhonov: the exact smoothing GiFt approximates, by conjugate
gradients on the sweep kernels, against the oracle's FP64 sparse direct
solve of the same system.

Bar: 1e-5 relative per coordinate (FP32 vectors; after 30 steps the CG
error bound 2 q^30, q = (sqrt(1 + 2 lam) - 1) / (sqrt(1 + 2 lam) + 1), is
below 1e-12 for lam <= 1, so the FP32 arithmetic decides), and with the
default step count the derived bound 5e-7 plus that bar.
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


def rel_err(got, ref, g):
    floor = 1e-3 * max(float(np.abs(g).max()), 1e-30)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), floor)


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
        "no-nets": synth.random_small(5, 9, 0, 3),
    }


NETLISTS = netlists()


def reference(nl, g, sigma, lam, reimpose=True):
    G = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell)
    d = oracle.degrees(G)
    x = g.reshape(nl.num_cells, -1)
    return oracle.tikhonov(G, d, x, sigma, lam, nl.is_fixed, reimpose).reshape(g.shape)


def run(ctx, nl, g, sigma, lam, iterations, reimpose=True, cut=0, device=True):
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed),
                              implicit_min_pins=cut)
    try:
        if device:
            gi = dev(g)
            go = torch.empty_like(gi)
            res = gift.gift_tikhonov(ctx, h, gi, go, sigma, lam, iterations, reimpose)
            torch.cuda.synchronize()
            return go.cpu().numpy(), res
        out = np.empty_like(g)
        res = gift.gift_tikhonov(ctx, h, g, out, sigma, lam, iterations, reimpose)
        return out, res
    finally:
        gift.gift_graph_free(h)


@pytest.mark.parametrize("name", sorted(NETLISTS))
@pytest.mark.parametrize("sigma,lam", [(2.0, 1.0), (4.0, 0.5), (1.0, 1.0)])
@pytest.mark.parametrize("S", [1, 4])
def test_matches_direct_solve(ctx, name, sigma, lam, S):
    nl = NETLISTS[name]
    g = synth.make_signals(nl, S, 50 + S)
    got, res = run(ctx, nl, g, sigma, lam, 30)
    ref = reference(nl, g, sigma, lam)
    assert rel_err(got, ref, g).max() <= RTOL
    assert np.all(res <= 1e-5)
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(got[fx], g[fx])


def test_default_steps_implicit_cliques_and_host_memory(ctx):
    nl = NETLISTS["zipf-20k"]
    g = synth.make_signals(nl, 4, 8)
    ref = reference(nl, g, 2.0, 1.0)
    dflt, _ = run(ctx, nl, g, 2.0, 1.0, 0)  # default step count: bound 5e-7
    assert rel_err(dflt, ref, g).max() <= RTOL
    imp, _ = run(ctx, nl, g, 2.0, 1.0, 30, cut=8)  # the same operator with implicit cliques
    assert rel_err(imp, ref, g).max() <= RTOL
    host, _ = run(ctx, nl, g, 2.0, 1.0, 30, device=False)
    dv, _ = run(ctx, nl, g, 2.0, 1.0, 30)
    np.testing.assert_array_equal(host, dv)
    raw, _ = run(ctx, nl, g, 2.0, 1.0, 30, reimpose=False)
    assert rel_err(raw, reference(nl, g, 2.0, 1.0, reimpose=False), g).max() <= RTOL


def test_invalid_arguments(ctx):
    nl = NETLISTS["plain-10k"]
    h = gift.gift_build_graph(ctx, nl.num_cells, dev(nl.net_ptr), dev(nl.pin_cell), dev(nl.is_fixed))
    try:
        for S, sigma, lam, it in [(129, 2.0, 1.0, 5), (1, 0.0, 1.0, 5), (1, 2.0, -1.0, 5), (1, 2.0, 1.0, -1),
                                  (1, float("nan"), 1.0, 5)]:
            g = dev(synth.make_signals(nl, S, 1))
            with pytest.raises(gift.GiftError) as e:
                gift.gift_tikhonov(ctx, h, g, torch.empty_like(g), sigma, lam, it)
            assert e.value.status == gift.GIFT_ERR_INVALID
    finally:
        gift.gift_graph_free(h)
