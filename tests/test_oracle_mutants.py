"""The pins catch plausible oracle mistakes.

Each case compiles a copy of the oracle source with one planted mistake into a
temporary directory (the committed oracle is untouched) and checks that at
least one pin -- the hand-derived K_M closed form or the dense brute force --
rejects the mutant.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "gift_oracle.c")

MUTANTS = {
    # weight rule: the classic clique weight 1/(M-1) instead of 2/M
    "weight_1_over_m_minus_1": ("double w = 2.0 / (double)m;", "double w = 1.0 / (double)(m - 1);"),
    # self-loop dropped from A + sigma I
    "no_self_loop": ("acc += sigma * si * x[(int64_t)i * K + c];", "acc += 0.0;"),
    # normaliser D instead of D + sigma I
    "scale_without_sigma": ("double sj = 1.0 / sqrt(d[j] + sigma);", "double sj = 1.0 / sqrt(d[j] + 1e-300);"),
    # wrong sign of the neighbour sum
    "neighbour_sign": ("acc += val[k] * sj * x[(int64_t)j * K + c];", "acc -= val[k] * sj * x[(int64_t)j * K + c];"),
    # own row used instead of the neighbour (wrong index)
    "wrong_index": ("acc += val[k] * sj * x[(int64_t)j * K + c];", "acc += val[k] * sj * x[(int64_t)i * K + c];"),
    # one application short for every term
    "power_off_by_one": ("for (int32_t p = 0; p < power[term]; ++p)", "for (int32_t p = 1; p < power[term]; ++p)"),
    # self pairs kept
    "self_pairs_kept": ("if (i == j) continue;", "if (0) continue;"),
    # fixed rows not reimposed
    "no_reimpose": ("if (reimpose && is_fixed)", "if (0)"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    return str(so)


def _pins_pass(so_path):
    """Run two pins against the library at so_path; True if both pass."""
    saved = oracle._lib
    try:
        oracle._lib = None
        L = C.CDLL(so_path)
        orig_build = oracle.build
        oracle.build = lambda: so_path
        try:
            L2 = oracle.lib()
        finally:
            oracle.build = orig_build
        assert L2 is not None
        ok = True
        # closed form on K_3 with no fixed cells
        M = 3
        g = oracle.build_graph(M, np.array([0, M]), np.arange(M, dtype=np.int32))
        x = np.array([[1.0, 2.0], [5.0, 7.0], [9.0, 3.0]])
        y = oracle.gift(g, oracle.degrees(g), x, None)
        f = 163817 / 512000
        ok &= np.allclose(y, x.mean(0) + f * (x - x.mean(0)), rtol=1e-12)
        # dense brute force with fixed cells and a repeated cell
        from tests.test_oracle_pins import _dense_reference
        nl = synth.random_small(2, num_cells=20, num_nets=25, max_pins=6, num_fixed=3, allow_repeat=True)
        xs = synth.uniform(1, 1, np.arange(40, dtype=np.uint64)).reshape(20, 2) * 100
        try:
            _, want = _dense_reference(nl, xs)
            _, _, got = oracle.run(nl, xs)
            ok &= np.allclose(got, want, rtol=1e-10, atol=1e-8)
        except Exception:
            ok = False
        return bool(ok)
    finally:
        oracle._lib = saved


def test_unmutated_copy_passes(tmp_path):
    so = _compile(tmp_path, "identity", "#include <math.h>", "#include <math.h>")
    assert _pins_pass(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    so = _compile(tmp_path, name, old, new)
    assert not _pins_pass(so), f"planted mistake {name} passed the pins"
