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
    _fields_ = [("weight_dtype", C.c_int32), ("implicit_min_pins", C.c_int32), ("reserved", C.c_int32 * 6)]


class gift_term(C.Structure):
    _fields_ = [("sigma", C.c_float), ("power", C.c_int32), ("alpha", C.c_double)]


class gift_filter_spec(C.Structure):
    _fields_ = [("num_terms", C.c_int32), ("term", gift_term * GIFT_MAX_TERMS), ("norm", C.c_int32),
                ("reimpose_fixed", C.c_int32), ("compensated", C.c_int32), ("schedule", C.c_int32)]


class gift_graph_desc(C.Structure):
    _fields_ = [("num_cells", C.c_int32), ("num_nets", C.c_int32), ("num_pins", C.c_int64), ("nnz", C.c_int64),
                ("raw_pairs", C.c_int64), ("weight_dtype", C.c_int32), ("max_row_nnz", C.c_int32),
                ("device_bytes", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("degree", C.c_void_p), ("implicit_min_pins", C.c_int32), ("reserved0", C.c_int32),
                ("implicit_nets", C.c_int64), ("implicit_pins", C.c_int64), ("stored", C.c_int64)]


class gift_eigen_result(C.Structure):
    _fields_ = [("lambda_", C.c_double * 2), ("residual", C.c_double * 2), ("iterations", C.c_int32),
                ("component_cells", C.c_int32), ("converged", C.c_int32), ("reserved", C.c_int32)]


class gift_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("kernels", C.c_int64),
                ("total_ms", C.c_double), ("alg_bytes", C.c_double)]


class gift_serve_opts(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_slots", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("weight_dtype", C.c_int32), ("compute_hpwl", C.c_int32), ("spec", gift_filter_spec),
                ("implicit_min_pins", C.c_int32), ("separate_filters", C.c_int32),
                ("batch_window_us", C.c_int32), ("reserved", C.c_int32 * 5)]


class gift_req_stats(C.Structure):
    _fields_ = [("latency_ms", C.c_double), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("nnz", C.c_int64), ("footprint_bytes", C.c_int64), ("weight_dtype", C.c_int32),
                ("num_signals", C.c_int32)]


class gift_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("waiting", C.c_int64), ("running", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mean_ms", C.c_double), ("max_ms", C.c_double), ("uptime_s", C.c_double),
                ("requests_per_s", C.c_double), ("edge_updates_per_s", C.c_double), ("budget_bytes", C.c_int64),
                ("peak_footprint_bytes", C.c_int64), ("max_slots", C.c_int32), ("peak_running", C.c_int32),
                ("batches", C.c_int64), ("batched_requests", C.c_int64), ("peak_batch", C.c_int32),
                ("reserved0", C.c_int32)]


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
        "gift_ctx_debug_waits": (None, [P, C.c_uint32, I32]),
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
        "gift_build_batch": (I32, [P, P, I32, P, C.POINTER(P), P, P]),
        "gift_hpwl_batch": (I32, [P, P, P, I32, P, I32, P]),
        "gift_filter_capture": (I32, [P, P, P, P, I32, P, C.POINTER(P)]),
        "gift_exec_launch": (I32, [P, P]),
        "gift_exec_free": (None, [P]),
        "gift_tikhonov": (I32, [P, P, C.c_float, C.c_float, I32, I32, P, I32, P, P, I32, P]),
        "gift_eigen_placement": (I32, [P, P, I32, C.c_double, C.c_uint64, P, P, I32, P]),
        "gift_run": (I32, [P, P, P, P, P, I32, P, P, P]),
        "gift_density": (I32, [P, P, I32, I32, P, P, C.c_float, C.c_float, P, I32, I32, C.c_double, P, P, I32, P]),
        "gift_serve_opts_default": (None, [P]),
        "gift_serve_create": (I32, [P, C.POINTER(P)]),
        "gift_serve_submit": (I32, [P, P, P, I32, I32, C.POINTER(C.c_uint64)]),
        "gift_serve_poll": (I32, [P, C.c_uint64, P, P, P]),
        "gift_serve_wait": (I32, [P, C.c_uint64, I32, P, P, P]),
        "gift_serve_stats_get": (I32, [P, P]),
        "gift_serve_destroy": (None, [P]),
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


# element types the C ABI reads through each kind of pointer
_KINDS = {"i64": ("int64",), "i32": ("int32",), "u8": ("uint8", "bool"), "f32": ("float32",),
          "f64": ("float64",)}


def _ptr(a, kind: str | None = None, count: int | None = None, what: str = "array"):
    """(pointer, mem kind) of a numpy array or a torch tensor.  `kind` names
    the element type the library reads through the pointer and `count` the
    elements it reads at most; an array of another type or fewer elements is
    rejected here, before the library could read past its end."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: arrays must be C-contiguous")
        dtype, n, p, mem = a.dtype.name, a.size, a.ctypes.data, GIFT_MEM_HOST
    else:  # torch tensor
        if not a.is_contiguous():
            raise ValueError(f"{what}: tensors must be contiguous")
        dtype = str(a.dtype).replace("torch.", "")
        n, p, mem = a.numel(), a.data_ptr(), (GIFT_MEM_DEVICE if a.is_cuda else GIFT_MEM_HOST)
    if kind is not None and dtype not in _KINDS[kind]:
        raise TypeError(f"{what}: element type {dtype}, the library reads {_KINDS[kind][0]}")
    if count is not None and n < count:
        raise ValueError(f"{what}: {n} elements, the library reads {count}")
    return p, mem


def _cells(graph) -> int:
    return int(gift_graph_info(graph).num_cells)


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


def gift_ctx_debug_waits(ctx, polls: int, drop_copies: bool = False):
    """Test hook: bound the TMA pipeline's waits to `polls` polls (0: default)
    and optionally drop its copies so that the waits run out."""
    load().gift_ctx_debug_waits(ctx, polls, 1 if drop_copies else 0)


def gift_filter_spec_default() -> gift_filter_spec:
    s = gift_filter_spec()
    load().gift_filter_spec_default(C.byref(s))
    return s


def make_spec(terms=None, norm: int = GIFT_NORM_SYM, reimpose: bool = True, schedule: int = 0,
              compensated: int = 0) -> gift_filter_spec:
    """compensated: 0 (or False) long rows only, 1 (or True) every row, 2 none."""
    s = gift_filter_spec_default()
    if terms is not None:
        s.num_terms = len(terms)
        for i, (sg, k, al) in enumerate(terms):
            s.term[i] = gift_term(sg, k, al)
    s.norm = norm
    s.reimpose_fixed = 1 if reimpose else 0
    s.schedule = schedule
    s.compensated = int(compensated)
    return s


def gift_build_opts_default() -> gift_build_opts:
    o = gift_build_opts()
    load().gift_build_opts_default(C.byref(o))
    return o


# ------------------------------------------------------------------ graph
def gift_build_graph(ctx, num_cells: int, net_ptr, pin_cell, is_fixed=None, weight_dtype: int = GIFT_WEIGHT_F32,
                     stream=None, implicit_min_pins: int = 0):
    """Build the clique graph; arrays are all host (numpy) or all device (torch)."""
    npp, mem = _ptr(net_ptr, "i64", 1, "net_ptr")
    pins = int(net_ptr[-1]) if isinstance(net_ptr, np.ndarray) else None  # device: the library checks
    pcp, mem2 = _ptr(pin_cell, "i32", pins, "pin_cell")
    fxp, mem3 = _ptr(is_fixed, "u8", num_cells, "is_fixed")
    nets = (net_ptr.shape[0] if hasattr(net_ptr, "shape") else len(net_ptr)) - 1
    nl = gift_netlist(num_cells, nets, npp, pcp, fxp, mem)
    opts = gift_build_opts_default()
    opts.weight_dtype = weight_dtype
    opts.implicit_min_pins = implicit_min_pins
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
    S = num_signals if num_signals is not None else int(g_in.shape[1])
    n = _cells(graph) * 2 * max(S, 0)
    pi, mem = _ptr(g_in, "f32", n, "g_in")
    po, mem_o = _ptr(g_out, "f32", n, "g_out")
    if mem != mem_o:
        raise ValueError("g_in and g_out must live in the same memory")
    _check(load().gift_filter(ctx, graph, C.byref(spec) if spec is not None else None, pi, S, po, mem,
                              _stream(stream)))
    return g_out


def gift_filter_noalloc(ctx, graph, g_in, g_out, spec: gift_filter_spec | None = None,
                        num_signals: int | None = None, stream=None):
    """gift_filter on device tensors without any device allocation: scratch comes
    from the library's fixed GIFT_NOALLOC_SCRATCH_BYTES area (for callers that
    cannot allocate while filtering).  Overlapping calls race on that area."""
    S = num_signals if num_signals is not None else int(g_in.shape[1])
    n = _cells(graph) * 2 * max(S, 0)
    pi, mem = _ptr(g_in, "f32", n, "g_in")
    po, mem_o = _ptr(g_out, "f32", n, "g_out")
    if mem != GIFT_MEM_DEVICE or mem_o != GIFT_MEM_DEVICE:
        raise ValueError("gift_filter_noalloc takes device tensors")
    _check(load().gift_filter_noalloc(ctx, graph, C.byref(spec) if spec is not None else None, pi, S, po,
                                      _stream(stream)))
    return g_out


GIFT_NOALLOC_SCRATCH_BYTES = 64 << 20


def gift_hpwl(ctx, graph, xy, num_signals: int | None = None, stream=None) -> np.ndarray:
    S = num_signals if num_signals is not None else int(xy.shape[1])
    p, mem = _ptr(xy, "f32", _cells(graph) * 2 * max(S, 0), "xy")
    out = np.zeros(S, dtype=np.float64)
    _check(load().gift_hpwl(ctx, graph, p, S, out.ctypes.data, mem, _stream(stream)))
    return out


# ------------------------------------------------------------------ serving
def gift_serve_opts_default() -> gift_serve_opts:
    o = gift_serve_opts()
    load().gift_serve_opts_default(C.byref(o))
    return o


def gift_serve_create(opts: gift_serve_opts | None = None, **fields):
    """Start a server; ``fields`` override members of the default options."""
    o = opts if opts is not None else gift_serve_opts_default()
    for k, v in fields.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(load().gift_serve_create(C.byref(o), C.byref(h)))
    return h


def gift_serve_submit(srv, num_cells: int, net_ptr, pin_cell, is_fixed, g_in, weight_dtype: int = -1) -> int:
    """Queue a request (host numpy arrays); returns its ticket."""
    g_in = np.ascontiguousarray(g_in, dtype=np.float32)
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pin_cell = np.ascontiguousarray(pin_cell, dtype=np.int32)
    fx = None if is_fixed is None else np.ascontiguousarray(is_fixed, dtype=np.uint8)
    nl = gift_netlist(num_cells, len(net_ptr) - 1, net_ptr.ctypes.data, pin_cell.ctypes.data,
                      None if fx is None else fx.ctypes.data, GIFT_MEM_HOST)
    t = C.c_uint64()
    _check(load().gift_serve_submit(srv, C.byref(nl), g_in.ctypes.data, g_in.shape[1], weight_dtype, C.byref(t)))
    return t.value


def _result(fn, srv, ticket, num_cells, num_signals, *extra):
    out = np.empty((num_cells, num_signals, 2), dtype=np.float32)
    hp = np.empty(num_signals, dtype=np.float64)
    st = gift_req_stats()
    s = fn(srv, ticket, *extra, out.ctypes.data, hp.ctypes.data, C.byref(st))
    if s == GIFT_ERR_BUSY:
        return None
    _check(s)
    return out, hp, st


def gift_serve_poll(srv, ticket: int, num_cells: int, num_signals: int):
    """(output, hpwl, stats) of a finished request, None while it waits or runs."""
    return _result(load().gift_serve_poll, srv, ticket, num_cells, num_signals)


def gift_serve_wait(srv, ticket: int, num_cells: int, num_signals: int, timeout_ms: int = -1):
    """As gift_serve_poll, waiting up to timeout_ms (-1: no limit)."""
    return _result(load().gift_serve_wait, srv, ticket, num_cells, num_signals, timeout_ms)


def gift_serve_stats_get(srv) -> gift_serve_stats:
    s = gift_serve_stats()
    _check(load().gift_serve_stats_get(srv, C.byref(s)))
    return s


def gift_serve_destroy(srv):
    load().gift_serve_destroy(srv)


# ------------------------------------------------------------------ batches
def gift_build_batch(ctx, netlists, weight_dtype: int = GIFT_WEIGHT_F32, stream=None, implicit_min_pins: int = 0):
    """netlists: sequence of (num_cells, net_ptr, pin_cell, is_fixed), all numpy
    arrays or all torch CUDA tensors.  Returns (graph, cell_offsets [B+1])."""
    B = len(netlists)
    arr = (gift_netlist * B)()
    keep = []
    for b, (n, net_ptr, pin_cell, is_fixed) in enumerate(netlists):
        p_np, mem = _ptr(net_ptr, "i64", 1, "net_ptr")
        pins = int(net_ptr[-1]) if isinstance(net_ptr, np.ndarray) else None
        p_pc, _ = _ptr(pin_cell, "i32", pins, "pin_cell")
        p_fx, _ = _ptr(is_fixed, "u8", n, "is_fixed")
        arr[b] = gift_netlist(n, (len(net_ptr) if isinstance(net_ptr, np.ndarray) else net_ptr.numel()) - 1,
                              p_np, p_pc, p_fx, mem)
        keep.append((net_ptr, pin_cell, is_fixed))
    opts = gift_build_opts()
    load().gift_build_opts_default(C.byref(opts))
    opts.weight_dtype = weight_dtype
    opts.implicit_min_pins = implicit_min_pins
    h = C.c_void_p()
    offs = np.zeros(B + 1, dtype=np.int64)
    _check(load().gift_build_batch(ctx, arr, B, C.byref(opts), C.byref(h), offs.ctypes.data, _stream(stream)))
    return h, offs


def gift_hpwl_batch(ctx, graph, xy, num_graphs: int, stream=None) -> np.ndarray:
    """HPWL per graph and signal, [num_graphs][S]."""
    S = xy.shape[1]
    p, mem = _ptr(xy, "f32", _cells(graph) * 2 * S, "xy")
    out = np.empty((num_graphs, S), dtype=np.float64)
    _check(load().gift_hpwl_batch(ctx, graph, p, S, out.ctypes.data, mem, _stream(stream)))
    return out


def gift_filter_capture(ctx, graph, g_in, g_out, spec=None):
    """Record the filter g_in -> g_out (torch CUDA tensors) as a CUDA graph."""
    n = _cells(graph) * 2 * int(g_in.shape[1])
    pi, mi = _ptr(g_in, "f32", n, "g_in")
    po, mo = _ptr(g_out, "f32", n, "g_out")
    if mi != GIFT_MEM_DEVICE or mo != GIFT_MEM_DEVICE:
        raise ValueError("gift_filter_capture takes device tensors")
    h = C.c_void_p()
    _check(load().gift_filter_capture(ctx, graph, None if spec is None else C.byref(spec), pi, g_in.shape[1], po,
                                      C.byref(h)))
    return h


def gift_exec_launch(exec_, stream=None):
    _check(load().gift_exec_launch(exec_, _stream(stream)))


def gift_exec_free(exec_):
    load().gift_exec_free(exec_)


# ------------------------------------------------------------------ Tikhonov
def gift_tikhonov(ctx, graph, g_in, g_out, sigma: float = 2.0, lam: float = 1.0, iterations: int = 0,
                  reimpose: bool = True, stream=None) -> np.ndarray:
    """g_out = (I + lam (I - A~_sigma))^-1 g_in by CG; returns ||r|| / ||g|| per column."""
    S = g_in.shape[1]
    n = _cells(graph) * 2 * S
    pi, mi = _ptr(g_in, "f32", n, "g_in")
    po, mo = _ptr(g_out, "f32", n, "g_out")
    if mi != mo:
        raise ValueError("g_in and g_out must be in the same memory")
    res = np.zeros(2 * S, dtype=np.float64)
    _check(load().gift_tikhonov(ctx, graph, sigma, lam, iterations, 1 if reimpose else 0, pi, S, po,
                                res.ctypes.data, mi, _stream(stream)))
    return res


# ------------------------------------------------------------------ eigenvector placement
def gift_eigen_placement(ctx, graph, out=None, max_iterations: int = 300, tol: float = 1e-10, seed: int = 1,
                         stream=None):
    """(u_2, u_3) of L = D - A on the largest component into out ([N][2]
    float64, numpy or CUDA tensor; a new numpy array if None); returns
    (out, gift_eigen_result)."""
    N = _cells(graph)
    if out is None:
        out = np.zeros((N, 2), dtype=np.float64)
    p, mem = _ptr(out, "f64", 2 * N, "out")
    res = gift_eigen_result()
    _check(load().gift_eigen_placement(ctx, graph, max_iterations, tol, seed, p, C.byref(res), mem,
                                       _stream(stream)))
    return out, res


# ------------------------------------------------------------------ density
def gift_density(ctx, xy, die=(0.0, 0.0, 1000.0, 1000.0), bins=(32, 32), target: float = 1.0, unit=(1.0, 1.0),
                 cell_w=None, cell_h=None, stream=None):
    """Bin density (Eq. 5) of every signal of xy [N][S][2] and its overflow:
    returns (density [S][bins_y][bins_x], overflow [S])."""
    N, S = xy.shape[0], xy.shape[1]
    p, mem = _ptr(xy, "f32", N * S * 2, "xy")
    pw, _ = _ptr(cell_w, "f32", N, "cell_w")
    ph, _ = _ptr(cell_h, "f32", N, "cell_h")
    d = np.ascontiguousarray(die, dtype=np.float64)
    out = np.empty((S, bins[1], bins[0]), dtype=np.float64)
    ov = np.empty(S, dtype=np.float64)
    _check(load().gift_density(ctx, p, N, S, pw, ph, unit[0], unit[1], d.ctypes.data, bins[0], bins[1], target,
                               out.ctypes.data, ov.ctypes.data, mem, _stream(stream)))
    return out, ov


# ------------------------------------------------------------------ whole path
def gift_run(ctx, num_cells: int, net_ptr, pin_cell, is_fixed, g_in, g_out, spec=None,
             weight_dtype: int = GIFT_WEIGHT_F32, implicit_min_pins: int = 0, stream=None) -> np.ndarray:
    """Build + filter + HPWL from host (numpy) arrays in one call; returns the HPWL per signal."""
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pin_cell = np.ascontiguousarray(pin_cell, dtype=np.int32)
    fx = None if is_fixed is None else np.ascontiguousarray(is_fixed, dtype=np.uint8)
    nl = gift_netlist(num_cells, len(net_ptr) - 1, net_ptr.ctypes.data, pin_cell.ctypes.data,
                      None if fx is None else fx.ctypes.data, GIFT_MEM_HOST)
    opts = gift_build_opts_default()
    opts.weight_dtype = weight_dtype
    opts.implicit_min_pins = implicit_min_pins
    if not (isinstance(g_in, np.ndarray) and isinstance(g_out, np.ndarray)):
        raise ValueError("gift_run takes host (numpy) signals")
    S = g_in.shape[1]
    _ptr(g_in, "f32", num_cells * 2 * S, "g_in")
    _ptr(g_out, "f32", num_cells * 2 * S, "g_out")
    if len(pin_cell) < int(net_ptr[-1]):
        raise ValueError(f"pin_cell: {len(pin_cell)} elements, the netlist has {int(net_ptr[-1])} pins")
    hp = np.empty(S, dtype=np.float64)
    _check(load().gift_run(ctx, C.byref(nl), C.byref(opts), None if spec is None else C.byref(spec),
                           g_in.ctypes.data, S, g_out.ctypes.data, hp.ctypes.data, _stream(stream)))
    return hp
