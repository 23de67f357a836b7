"""The pins catch plausible oracle mistakes.

Each case plants one mistake in a copy of the oracle (the committed oracle is
untouched) and runs every pin of tests/test_oracle_pins.py and
tests/test_oracle_eigen.py, with all their parameters, against the copy: at
least one pin must fail.  C mistakes are compiled from a patched copy of
gift_oracle.c into a temporary directory and swapped in as the oracle's
library; Python mistakes are executed from a patched copy of the package
source and their functions swapped into the ``oracle`` module.  Every planted
mistake keeps its memory accesses in bounds.
"""
import ctypes as C
import itertools
import os
import subprocess
import sys
import types
import warnings

import pytest

# the OpenMP builds run the tiny pin inputs: a couple of threads each keeps
# parallel test runs from oversubscribing the host (read when the first
# OpenMP build is loaded)
os.environ.setdefault("OMP_NUM_THREADS", "2")

import oracle  # noqa: E402
from tests import test_oracle_eigen, test_oracle_pins  # noqa: E402

C_SRC = os.path.join(os.path.dirname(oracle.__file__), "gift_oracle.c")
PY_SRC = os.path.join(os.path.dirname(oracle.__file__), "__init__.py")

# name -> [(text, replacement, occurrence)] applied to gift_oracle.c
C_MUTANTS = {
    # clique expansion (Sec. 3.2.3, weight rule after Eq. 4)
    "weight_1_over_m_minus_1": [("double w = 2.0 / (double)m;", "double w = 1.0 / (double)(m - 1);", 0)],
    "self_pairs_kept": [("if (i == j) continue;", "if (0) continue;", 0)],
    "duplicates_overwritten": [("g->val[nnz - 1] += pairs[t].w;", "g->val[nnz - 1] = pairs[t].w;", 0)],
    "columns_descending": [("if (a->j != b->j) return a->j < b->j ? -1 : 1;",
                            "if (a->j != b->j) return a->j > b->j ? -1 : 1;", 0)],
    "cut_off_by_one": [("if (m >= 2 && (cut <= 0 || m < cut)) npairs", "if (m >= 2 && (cut <= 0 || m <= cut)) npairs", 0),
                       ("if (cut > 0 && m >= cut) continue;", "if (cut > 0 && m > cut) continue;", 0)],
    "accepts_decreasing_net_ptr": [("if (m < 0) return NULL;", "if (m < 0) continue;", 0)],
    # implicit clique degrees
    "implicit_weight": [("double w = 2.0 / (double)m;", "double w = 1.0 / (double)(m - 1);", 1)],
    "implicit_ignores_repeats": [("d[cells[r]] += ((double)k * w) * (double)(m - k);",
                                  "d[cells[r]] += ((double)k * w) * (double)(m - 1);", 0)],
    "implicit_cut_off_by_one": [("if (m < 2 || m < cut) continue;", "if (m < 2 || m <= cut) continue;", 0)],
    # cliques applied from the netlist (same operator as the expansion)
    "implicit_apply_weight": [("double w = 2.0 / (double)m;", "double w = 1.0 / (double)(m - 1);", 2)],
    "implicit_apply_ignores_repeats": [("(S[c] - (double)k * xh[i * K + c])", "(S[c] - xh[i * K + c])", 0)],
    "implicit_apply_once_per_cell": [("acc[i * K + c] += (double)k * w *", "acc[i * K + c] += w *", 0)],
    "implicit_apply_unscaled": [("double sj = norm == 0 ? 1.0 / sqrt(d[j] + sigma) : 1.0;", "double sj = 1.0;", 0)],
    "implicit_apply_cut_off_by_one": [("if (m < 2 || m < cut) continue;", "if (m < 2 || m <= cut) continue;", 1)],
    "implicit_apply_self_loop_dropped": [("double a = acc[(int64_t)i * K + c] + sigma * xh[(int64_t)i * K + c];",
                                         "double a = acc[(int64_t)i * K + c];", 0)],
    "implicit_apply_last_pin_dropped": [("for (int64_t p = 0; p < m; ++p) t += xh", "for (int64_t p = 0; p < m - 1; ++p) t += xh", 0)],
    # degrees (Sec. 2.1)
    "degree_drops_first_entry": [("for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += val[k];",
                                  "for (int64_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) s += val[k];", 0)],
    # storage rounding
    "round_truncates": [("return nearbyint(v / ulp) * ulp;", "return trunc(v / ulp) * ulp;", 0)],
    "round_ties_away": [("return nearbyint(v / ulp) * ulp;", "return round(v / ulp) * ulp;", 0)],
    "round_one_bit_short": [("double ulp = ldexp(1.0, lead - (prec - 1));",
                             "double ulp = ldexp(1.0, lead - (prec - 2));", 0)],
    "f16_without_subnormals": [("case 3: out[t] = round_to(in[t], 11, -14);", "case 3: out[t] = round_to(in[t], 11, -126);", 0)],
    # augmented normalised adjacency (Eq. 16)
    "no_self_loop": [("acc += sigma * si * x[(int64_t)i * K + c];", "acc += 0.0;", 0)],
    "scale_without_sigma": [("double sj = 1.0 / sqrt(d[j] + sigma);", "double sj = 1.0 / sqrt(d[j] + 1e-300);", 0)],
    "neighbour_sign": [("acc += val[k] * sj * x[(int64_t)j * K + c];", "acc -= val[k] * sj * x[(int64_t)j * K + c];", 0)],
    "wrong_index": [("acc += val[k] * sj * x[(int64_t)j * K + c];", "acc += val[k] * sj * x[(int64_t)i * K + c];", 0)],
    "missing_post_scale": [("y[(int64_t)i * K + c] = si * acc;", "y[(int64_t)i * K + c] = acc;", 0)],
    "random_walk_normaliser": [("y[(int64_t)i * K + c] = acc / (d[i] + sigma);", "y[(int64_t)i * K + c] = acc / (d[i] + 1.0);", 0)],
    # the filter (Eq. 15) and the fixed cells
    "power_off_by_one": [("for (int32_t p = 0; p < power[term]; ++p)", "for (int32_t p = 1; p < power[term]; ++p)", 0)],
    "terms_chained": [("memcpy(v, g, len * sizeof(double));", "if (term == 0) memcpy(v, g, len * sizeof(double));", 0)],
    "first_alpha_everywhere": [("out[q] += alpha[term] * v[q];", "out[q] += alpha[0] * v[q];", 0)],
    "first_sigma_everywhere": [("oracle_apply(n, K, row_ptr, col, val, d, sigma[term], norm, v, t);",
                                "oracle_apply(n, K, row_ptr, col, val, d, sigma[0], norm, v, t);", 0)],
    "no_reimpose": [("if (reimpose && is_fixed)", "if (0)", 0)],
    # HPWL
    "hpwl_x_only": [("total += (xhi - xlo) + (yhi - ylo);", "total += (xhi - xlo);", 0)],
    "hpwl_y_reads_x": [("y = xy[(c * S + s) * 2 + 1];", "y = xy[(c * S + s) * 2 + 0];", 0)],
    "hpwl_first_signal_only": [("double x = xy[(c * S + s) * 2 + 0], y = xy[(c * S + s) * 2 + 1];",
                                "double x = xy[(c * S) * 2 + 0], y = xy[(c * S) * 2 + 1];", 0)],
    "hpwl_last_pin_dropped": [("for (int64_t p = 0; p < m; ++p) {", "for (int64_t p = 0; p < m - 1; ++p) {", 0)],
}

# name -> [(text, replacement)] applied to the oracle package source
PY_MUTANTS = {
    # exact smoothing (Sec. 3.2.2, Eq. 18)
    "tikhonov_identity_unweighted": [("return (1.0 + lam) * v - lam * At_v", "return v - lam * At_v")],
    "tikhonov_self_loop_dropped": [("At_v = s[:, None] * (A @ (s[:, None] * v) + sigma * s[:, None] * v)",
                                    "At_v = s[:, None] * (A @ (s[:, None] * v))")],
    "tikhonov_loose_stop": [("<= 1e-13 * np.maximum(bn, 1e-300)", "<= 1e-3 * np.maximum(bn, 1e-300)")],
    "tikhonov_no_reimpose": [("out[fx] = np.asarray(sig, dtype=np.float64)[fx]", "out[fx] = out[fx]")],
    # bin density (Eq. 5)
    "density_full_extent": [("hw, hh = 0.5 * w.astype(np.float64), 0.5 * h.astype(np.float64)",
                             "hw, hh = w.astype(np.float64), h.astype(np.float64)")],
    "density_left_edge_unclipped": [("np.maximum(np.minimum(hi, b1) - np.maximum(lo, b0), 0.0)",
                                     "np.maximum(np.minimum(hi, b1) - lo, 0.0)")],
    "density_bin_index_rounded": [("np.clip(np.floor((lo - o) / step), 0, n - 1)", "np.clip(np.rint((lo - o) / step), 0, n - 1)")],
    "density_y_reads_x": [("x, y = xy[:, s, 0].astype(np.float64), xy[:, s, 1].astype(np.float64)",
                           "x, y = xy[:, s, 0].astype(np.float64), xy[:, s, 0].astype(np.float64)")],
    "density_overflow_whole_bin": [("acc += c - tq", "acc += c")],
    "density_overflow_unclamped": [("if c > tq:\n                acc += c - tq", "if True:\n                acc += c - tq")],
    # storage format applied after the degrees
    "degrees_before_rounding": [("    g = build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut)\n    if fmt != \"f64\":\n"
                                 "        g = stored(g, fmt)\n    d = degrees(g)",
                                 "    g = build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut)\n    d = degrees(g)\n"
                                 "    if fmt != \"f64\":\n        g = stored(g, fmt)")],
    "implicit_drops_expanded_part": [("out = np.array(d, dtype=np.float64, copy=True)",
                                      "out = np.zeros(np.shape(d), dtype=np.float64)")],
    "run_cut_degrees_of_small_nets_only": [("        d = implicit_degrees(d, nl.net_ptr, nl.pin_cell, cut)\n",
                                            "        d = d\n")],
    "run_cut_ignores_large_nets": [("implicit=(nl.net_ptr, nl.pin_cell, cut) if cut > 0 else None)", "implicit=None)")],
    # the wrappers' arguments to the C library
    "apply_norm_flag_swapped": [("float(sigma), 0 if norm == \"sym\" else 1, _p(x), _p(y))",
                                 "float(sigma), 1 if norm == \"sym\" else 0, _p(x), _p(y))")],
    "filter_norm_flag_swapped": [("0 if norm == \"sym\" else 1, 1 if reimpose else 0, _p(fx), _p(x), _p(out))",
                                  "1 if norm == \"sym\" else 0, 1 if reimpose else 0, _p(fx), _p(x), _p(out))")],
    "filter_cut_norm_flag_swapped": [("0 if norm == \"sym\" else 1, 1 if reimpose else 0, _p(fx), int(npt.size - 1),",
                                      "1 if norm == \"sym\" else 0, 1 if reimpose else 0, _p(fx), int(npt.size - 1),")],
    "apply_cut_norm_flag_swapped": [("float(sigma), 0 if norm == \"sym\" else 1, int(npt.size - 1)",
                                     "float(sigma), 1 if norm == \"sym\" else 0, int(npt.size - 1)")],
    "rounding_format_ignored": [("_p(out), FMT[fmt])", "_p(out), FMT[\"f32\"])")],
    "stored_weights_unrounded": [("return Graph(g.n, g.row_ptr, g.col, round_values(g.val, fmt))",
                                  "return Graph(g.n, g.row_ptr, g.col, np.array(g.val, copy=True))")],
    # eigenvector placement (Sec. 3.3.1, Eq. 23-24)
    "component_smallest": [("best = np.lexsort((first, -sizes))[0]", "best = np.lexsort((first, sizes))[0]")],
    "component_tie_largest_id": [("best = np.lexsort((first, -sizes))[0]", "best = np.lexsort((-first, -sizes))[0]")],
    "eigen_signless_laplacian": [("lap = (diags(np.asarray(d, dtype=np.float64)[idx]) - a).tocsc()",
                                  "lap = (diags(np.asarray(d, dtype=np.float64)[idx]) + a).tocsc()")],
    "eigen_constant_vector": [("u[idx, 0] = v[:, 1]", "u[idx, 0] = v[:, 0]")],
    "eigen_u2_twice": [("u[idx, 1] = v[:, 2]", "u[idx, 1] = v[:, 1]")],
    "eigen_lambda_shifted": [("return u, (float(w[1]), float(w[2])), mask", "return u, (float(w[0]), float(w[1])), mask")],
}

_OUTCOME = (pytest.fail.Exception, pytest.skip.Exception)


def _pin_cases():
    """(label, function, kwargs) for every pin, parameters expanded."""
    for mod in (test_oracle_pins, test_oracle_eigen):
        for name in sorted(vars(mod)):
            f = getattr(mod, name)
            if not (name.startswith("test_") and callable(f)):
                continue
            axes = []
            for m in getattr(f, "pytestmark", []):
                if m.name != "parametrize":
                    continue
                names = [a.strip() for a in m.args[0].split(",")]
                axes.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]])
            for combo in itertools.product(*axes):
                kw = {k: v for part in combo for k, v in part.items()}
                yield f"{mod.__name__.split('.')[-1]}::{name}{kw or ''}", f, kw


def _failing_pins():
    failed = []
    for label, f, kw in _pin_cases():
        try:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                f(**kw)
        except pytest.skip.Exception:
            pass
        except (Exception, pytest.fail.Exception):
            failed.append(label)
    return failed


def _patch(src, edits):
    for edit in edits:
        old, new, nth = edit if len(edit) == 3 else (*edit, 0)
        at = -1
        for _ in range(nth + 1):
            at = src.find(old, at + 1)
            assert at >= 0, old
        src = src[:at] + new + src[at + len(old):]
    return src


def _compile(tmp_path, name, src, threads=False):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           *(["-fopenmp"] if threads else []), "-o", str(so), str(c), "-lm"])
    return str(so)


def _with_c_library(so_path, run):
    """Run `run()` with the oracle bound to the library at so_path."""
    saved_lib, saved_build = oracle._lib, oracle.build
    try:
        oracle._lib = None
        oracle.build = lambda threads=False: so_path
        oracle.lib()
        return run()
    finally:
        oracle._lib, oracle.build = saved_lib, saved_build


def _with_python_source(src, run):
    """Run `run()` with the oracle's functions taken from the source src."""
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = PY_SRC
    sys.modules["oracle_mutant"] = mod  # the dataclass decorator looks its module up
    try:
        exec(compile(src, PY_SRC, "exec"), mod.__dict__)
    finally:
        del sys.modules["oracle_mutant"]
    swapped = {k: v for k, v in vars(mod).items()
               if isinstance(v, types.FunctionType) and v.__module__ == "oracle_mutant" and k not in ("build", "lib")}
    saved = {k: getattr(oracle, k) for k in swapped}
    try:
        for k, v in swapped.items():
            setattr(oracle, k, v)
        return run()
    finally:
        for k, v in saved.items():
            setattr(oracle, k, v)


@pytest.mark.parametrize("threads", [False, True])
def test_unmutated_copies_pass_every_pin(tmp_path, threads):
    so = _compile(tmp_path, "identity", open(C_SRC).read(), threads)
    assert _with_c_library(so, _failing_pins) == []
    if not threads:
        assert _with_python_source(open(PY_SRC).read(), _failing_pins) == []
    assert len(list(_pin_cases())) >= 60


@pytest.mark.parametrize("threads", [False, True])
@pytest.mark.parametrize("name", sorted(C_MUTANTS))
def test_c_mutant_is_caught(tmp_path, name, threads):
    """Every planted C mistake fails a pin, in the single-threaded and in the
    OpenMP build."""
    so = _compile(tmp_path, name, _patch(open(C_SRC).read(), C_MUTANTS[name]), threads)
    assert _with_c_library(so, _failing_pins), f"planted mistake {name} passed every pin"


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_is_caught(name):
    src = _patch(open(PY_SRC).read(), PY_MUTANTS[name])
    assert _with_python_source(src, _failing_pins), f"planted mistake {name} passed every pin"
