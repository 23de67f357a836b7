"""Thin ctypes binding of libgift (include/gift.h): same names, argument
marshalling only.  Every step of the GiFt path runs in the library's CUDA
kernels; nothing here computes.

Arrays may be numpy arrays (host memory, ``GIFT_MEM_HOST``) or torch CUDA
tensors (device memory, ``GIFT_MEM_DEVICE``); torch is used only for device
memory and streams.  A missing or unloadable library raises immediately --
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GIFT_OK, GIFT_ERR_INVALID, GIFT_ERR_OOM, GIFT_ERR_CUDA, GIFT_ERR_TIMEOUT, GIFT_ERR_BUSY, GIFT_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = ["GIFT_OK", "GIFT_ERR_INVALID", "GIFT_ERR_OOM", "GIFT_ERR_CUDA", "GIFT_ERR_TIMEOUT",
                "GIFT_ERR_BUSY", "GIFT_ERR_UNSUPPORTED"]
GIFT_MEM_HOST, GIFT_MEM_DEVICE = 0, 1
GIFT_WEIGHT_F32, GIFT_WEIGHT_BF16, GIFT_WEIGHT_F16 = 0, 1, 2
WEIGHT = {"f32": 0, "bf16": 1, "f16": 2}
GIFT_NORM_SYM, GIFT_NORM_RW = 0, 1
GIFT_MAX_TERMS = 8


class GiftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")


class gift_netlist(C.Structure):
    _fields_ = [("num_cells", C.c_int32), ("num_nets", C.c_int32), ("net_ptr", C.c_void_p),
                ("pin_cell", C.c_void_p), ("is_fixed", C.c_void_p), ("mem", C.c_int32)]


class gift_build_opts(C.Structure):
    _fields_ = [("weight_dtype", C.c_int32), ("reserved", C.c_int32 * 7)]


class gift_term(C.Structure):
    _fields_ = [("sigma", C.c_float), ("power", C.c_int32), ("alpha", C.c_double)]


class gift_filter_spec(C.Structure):
    _fields_ = [("num_terms", C.c_int32), ("term", gift_term * GIFT_MAX_TERMS), ("norm", C.c_int32),
                ("reimpose_fixed", C.c_int32), ("compensated", C.c_int32), ("schedule", C.c_int32)]


class gift_graph_desc(C.Structure):
    _fields_ = [("num_cells", C.c_int32), ("num_nets", C.c_int32), ("num_pins", C.c_int64), ("nnz", C.c_int64),
                ("raw_pairs", C.c_int64), ("weight_dtype", C.c_int32), ("max_row_nnz", C.c_int32),
                ("device_bytes", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("degree", C.c_void_p)]


class gift_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("kernels", C.c_int64),
                ("total_ms", C.c_double), ("alg_bytes", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgift.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libgift.so is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "gift_ctx_create": (I32, [I32, C.POINTER(P)]),
        "gift_ctx_destroy": (None, [P]),
        "gift_ctx_set_profiling": (I32, [P, I32]),
        "gift_ctx_kernel_stats": (I32, [P, P, I32]),
        "gift_ctx_reset_stats": (None, [P]),
        "gift_ctx_debug_fail_alloc": (None, [P, I32]),
        "gift_ctx_last_schedule": (I32, [P, P]),
        "gift_ctx_device_status": (I32, [P]),
        "gift_filter_spec_default": (None, [P]),
        "gift_build_opts_default": (None, [P]),
        "gift_build_graph": (I32, [P, P, P, C.POINTER(P), P]),
        "gift_graph_info": (I32, [P, P]),
        "gift_graph_export": (I32, [P, P, P, P, P]),
        "gift_graph_free": (None, [P]),
        "gift_graph_free_async": (None, [P, P]),
        "gift_filter": (I32, [P, P, P, P, I32, P, I32, P]),
        "gift_hpwl": (I32, [P, P, P, I32, P, I32, P]),
        "gift_filter_noalloc": (I32, [P, P, P, P, I32, P, P]),
        "gift_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int):
    if st != GIFT_OK:
        raise GiftError(st, load().gift_last_error().decode())


def _ptr(a):
    """(pointer, mem kind) of a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, GIFT_MEM_HOST
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr(), (GIFT_MEM_DEVICE if a.is_cuda else GIFT_MEM_HOST)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ context
def gift_ctx_create(device: int = 0):
    h = C.c_void_p()
    _check(load().gift_ctx_create(device, C.byref(h)))
    return h


def gift_ctx_destroy(ctx):
    load().gift_ctx_destroy(ctx)


def gift_ctx_set_profiling(ctx, enable: bool):
    _check(load().gift_ctx_set_profiling(ctx, 1 if enable else 0))


def gift_ctx_kernel_stats(ctx) -> dict:
    L = load()
    n = L.gift_ctx_kernel_stats(ctx, None, 0)
    arr = (gift_kernel_stat * max(n, 1))()
    n = L.gift_ctx_kernel_stats(ctx, arr, n)
    return {arr[i].name.decode(): dict(launches=arr[i].launches, kernels=arr[i].kernels, total_ms=arr[i].total_ms,
                                       alg_bytes=arr[i].alg_bytes) for i in range(n)}


def gift_ctx_reset_stats(ctx):
    load().gift_ctx_reset_stats(ctx)


def gift_ctx_last_schedule(ctx) -> list:
    """Schedule codes of the last filter call, per launch kind (two chains first
    sweep, two chains later, one chain first sweep, one chain later)."""
    out = (C.c_int32 * 4)()
    load().gift_ctx_last_schedule(ctx, out)
    return [int(v) for v in out]


def gift_ctx_device_status(ctx):
    _check(load().gift_ctx_device_status(ctx))


def gift_ctx_debug_fail_alloc(ctx, n: int):
    load().gift_ctx_debug_fail_alloc(ctx, n)


def gift_filter_spec_default() -> gift_filter_spec:
    s = gift_filter_spec()
    load().gift_filter_spec_default(C.byref(s))
    return s


def make_spec(terms=None, norm: int = GIFT_NORM_SYM, reimpose: bool = True, schedule: int = 0,
              compensated: bool = False) -> gift_filter_spec:
    s = gift_filter_spec_default()
    if terms is not None:
        s.num_terms = len(terms)
        for i, (sg, k, al) in enumerate(terms):
            s.term[i] = gift_term(sg, k, al)
    s.norm = norm
    s.reimpose_fixed = 1 if reimpose else 0
    s.schedule = schedule
    s.compensated = 1 if compensated else 0
    return s


def gift_build_opts_default() -> gift_build_opts:
    o = gift_build_opts()
    load().gift_build_opts_default(C.byref(o))
    return o


# ------------------------------------------------------------------ graph
def gift_build_graph(ctx, num_cells: int, net_ptr, pin_cell, is_fixed=None, weight_dtype: int = GIFT_WEIGHT_F32,
                     stream=None):
    """Build the clique graph; arrays are all host (numpy) or all device (torch)."""
    npp, mem = _ptr(net_ptr)
    pcp, mem2 = _ptr(pin_cell)
    fxp, mem3 = _ptr(is_fixed)
    nets = (net_ptr.shape[0] if hasattr(net_ptr, "shape") else len(net_ptr)) - 1
    nl = gift_netlist(num_cells, nets, npp, pcp, fxp, mem)
    opts = gift_build_opts_default()
    opts.weight_dtype = weight_dtype
    h = C.c_void_p()
    _check(load().gift_build_graph(ctx, C.byref(nl), C.byref(opts), C.byref(h), _stream(stream)))
    return h


def gift_graph_info(graph) -> gift_graph_desc:
    d = gift_graph_desc()
    _check(load().gift_graph_info(graph, C.byref(d)))
    return d


def gift_graph_export(graph):
    """Host copies (row_ptr int64, col int32, val float64, degree float64)."""
    d = gift_graph_info(graph)
    rp = np.zeros(d.num_cells + 1, dtype=np.int64)
    col = np.zeros(max(d.nnz, 1), dtype=np.int32)
    val = np.zeros(max(d.nnz, 1), dtype=np.float64)
    deg = np.zeros(d.num_cells, dtype=np.float64)
    _check(load().gift_graph_export(graph, rp.ctypes.data, col.ctypes.data, val.ctypes.data, deg.ctypes.data))
    return rp, col[:d.nnz], val[:d.nnz], deg


def gift_graph_free(graph):
    load().gift_graph_free(graph)


def gift_graph_free_async(graph, stream=None):
    load().gift_graph_free_async(graph, _stream(stream))


# ------------------------------------------------------------------ filter / hpwl
def gift_filter(ctx, graph, g_in, g_out, spec: gift_filter_spec | None = None, num_signals: int | None = None,
                stream=None):
    """g_out <- GiFt(g_in); g_in/g_out are [N, S, 2] float32 (both numpy or both CUDA tensors)."""
    pi, mem = _ptr(g_in)
    po, mem_o = _ptr(g_out)
    if mem != mem_o:
        raise ValueError("g_in and g_out must live in the same memory")
    S = num_signals if num_signals is not None else int(g_in.shape[1])
    _check(load().gift_filter(ctx, graph, C.byref(spec) if spec is not None else None, pi, S, po, mem,
                              _stream(stream)))
    return g_out


def gift_filter_noalloc(ctx, graph, g_in, g_out, spec: gift_filter_spec | None = None,
                        num_signals: int | None = None, stream=None):
    """gift_filter on device tensors without any device allocation: scratch comes
    from the library's fixed GIFT_NOALLOC_SCRATCH_BYTES area (for callers that
    cannot allocate while filtering).  Overlapping calls race on that area."""
    pi, mem = _ptr(g_in)
    po, mem_o = _ptr(g_out)
    if mem != GIFT_MEM_DEVICE or mem_o != GIFT_MEM_DEVICE:
        raise ValueError("gift_filter_noalloc takes device tensors")
    S = num_signals if num_signals is not None else int(g_in.shape[1])
    _check(load().gift_filter_noalloc(ctx, graph, C.byref(spec) if spec is not None else None, pi, S, po,
                                      _stream(stream)))
    return g_out


GIFT_NOALLOC_SCRATCH_BYTES = 64 << 20


def gift_hpwl(ctx, graph, xy, num_signals: int | None = None, stream=None) -> np.ndarray:
    p, mem = _ptr(xy)
    S = num_signals if num_signals is not None else int(xy.shape[1])
    out = np.zeros(S, dtype=np.float64)
    _check(load().gift_hpwl(ctx, graph, p, S, out.ctypes.data, mem, _stream(stream)))
    return out
