"""The OpenMP build of the oracle (the timed CPU baseline on all host cores)
gives the single-threaded build's results bit for bit: every parallel loop
writes each output element from one thread, summed in the same order.  (Both
builds pass every pin and catch every planted mistake: test_oracle_mutants.)"""
import numpy as np

import oracle
from paper_2502_17632_gb300 import synth


def _both(fn):
    out = []
    for th in (False, True):
        oracle.use_threads(th)
        try:
            out.append(fn())
        finally:
            oracle.use_threads(False)
    return out


def test_threaded_build_same_bits():
    nl = synth.random_small(5, 2000, 2400, 30, num_fixed=20, allow_repeat=True)
    g = synth.make_signals(nl, 3, 8).reshape(nl.num_cells, -1)

    def run():
        G, d, out = oracle.run(nl, g)
        _, d16, out16 = oracle.run(nl, g, fmt="f16", norm="rw", reimpose=False)
        _, dc, outc = oracle.run(nl, g, cut=7)
        y = oracle.apply_cut(oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=5), dc, 4.0, g,
                             nl.net_ptr, nl.pin_cell, 5)
        return G.row_ptr, G.col, G.val, d, out, d16, out16, dc, outc, y, oracle.threads()

    serial, threaded = _both(run)
    assert serial[-1] == 1 and threaded[-1] >= 1
    for a, b in zip(serial[:-1], threaded[:-1]):
        np.testing.assert_array_equal(a, b)
