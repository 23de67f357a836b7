"""The C-ABI library builds, loads and exports every symbol include/gift.h
declares; the ctypes structures match the C layout.  No GPU needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2502_17632_gb300 import gift

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        txt = open(h).read()
        names += re.findall(r"GIFT_API\s+[\w\s\*]+?\b(gift_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = gift.load()
    names = declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", gift.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gift_\w+)", out))
    assert set(names) <= exported
    # nothing exported beyond the header's API
    assert exported <= set(names), exported - set(names)


def test_binding_names_match_header():
    for n in declared_functions():
        if n in ("gift_last_error",):
            continue
        assert hasattr(gift, n), f"binding lacks {n}"


LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "gift.h"
#define P(T) printf(#T " %zu\n", sizeof(T));
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  P(gift_netlist) O(gift_netlist, net_ptr) O(gift_netlist, mem)
  P(gift_build_opts)
  P(gift_term) O(gift_term, alpha)
  P(gift_filter_spec) O(gift_filter_spec, term) O(gift_filter_spec, norm) O(gift_filter_spec, schedule)
  P(gift_graph_desc) O(gift_graph_desc, nnz) O(gift_graph_desc, device_bytes) O(gift_graph_desc, degree)
  O(gift_graph_desc, stored)
  P(gift_kernel_stat) O(gift_kernel_stat, launches) O(gift_kernel_stat, kernels) O(gift_kernel_stat, alg_bytes)
  P(gift_eigen_result) O(gift_eigen_result, residual) O(gift_eigen_result, iterations) O(gift_eigen_result, converged)
  return 0;
}
"""


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    ref = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    py = {
        "gift_netlist": gift.gift_netlist, "gift_build_opts": gift.gift_build_opts, "gift_term": gift.gift_term,
        "gift_filter_spec": gift.gift_filter_spec, "gift_graph_desc": gift.gift_graph_desc,
        "gift_kernel_stat": gift.gift_kernel_stat, "gift_eigen_result": gift.gift_eigen_result,
    }
    for key, val in ref.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(py[t], f).offset == int(val), key
        else:
            assert C.sizeof(py[key]) == int(val), key


def test_default_spec_is_the_papers():
    s = gift.gift_filter_spec_default()
    terms = [(s.term[i].sigma, s.term[i].power, s.term[i].alpha) for i in range(s.num_terms)]
    assert terms == [(2.0, 2, 0.1), (4.0, 2, 0.7), (4.0, 4, 0.2)]
    assert s.norm == gift.GIFT_NORM_SYM and s.reimpose_fixed == 1


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gift.GiftError) as ei:
        gift.gift_ctx_create(0)
    assert ei.value.status in (gift.GIFT_ERR_CUDA, gift.GIFT_ERR_INVALID)


def test_no_gpu_server_fails_loudly():
    """The request loop needs a device too: creating a server without one is
    an error status, not a silent host fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gift.GiftError) as ei:
        gift.gift_serve_create()
    assert ei.value.status in (gift.GIFT_ERR_CUDA, gift.GIFT_ERR_INVALID)


def test_serve_structs_match_header():
    """ctypes layouts of the serving structs equal the C compiler's."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "gift.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gift_serve_opts), offsetof(gift_serve_opts, spec),
         offsetof(gift_serve_opts, separate_filters), offsetof(gift_serve_opts, batch_window_us),
         offsetof(gift_serve_opts, reserved), sizeof(gift_req_stats));
  printf("%zu %zu %zu %zu %zu\n", sizeof(gift_serve_stats), offsetof(gift_serve_stats, budget_bytes),
         offsetof(gift_serve_stats, peak_running), offsetof(gift_serve_stats, batched_requests),
         offsetof(gift_serve_stats, peak_batch));
  return 0;
}
"""
    import ctypes as C
    root = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as d:
        with open(f"{d}/t.c", "w") as f:
            f.write(src)
        subprocess.run([cc, "-I", f"{root}/include", f"{d}/t.c", "-o", f"{d}/t"], check=True)
        out = subprocess.run([f"{d}/t"], check=True, capture_output=True, text=True).stdout.split()
    want = [C.sizeof(gift.gift_serve_opts), gift.gift_serve_opts.spec.offset,
            gift.gift_serve_opts.separate_filters.offset, gift.gift_serve_opts.batch_window_us.offset,
            gift.gift_serve_opts.reserved.offset,
            C.sizeof(gift.gift_req_stats), C.sizeof(gift.gift_serve_stats),
            gift.gift_serve_stats.budget_bytes.offset, gift.gift_serve_stats.peak_running.offset,
            gift.gift_serve_stats.batched_requests.offset, gift.gift_serve_stats.peak_batch.offset]
    assert [int(x) for x in out] == want
