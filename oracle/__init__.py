"""FP64 CPU oracle of the GiFt filter path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check and the CPU-baseline leg of ``bench.py`` may
import this package.  The product path (the CUDA library and its binding)
never calls it.  The arithmetic lives in ``gift_oracle.c`` (plain C, FP64);
this module compiles it with gcc -- single-threaded, and with OpenMP for the
timed CPU baseline (:func:`use_threads`; the same results) -- and marshals
numpy arrays.

Every function states the paper passage it follows:

* :func:`build_graph`   -- clique net model, weight 2/M (Sec. 2.2 after Eq. 4,
  Sec. 3.2.3); duplicates summed in net order (Sec. 2.1, single w_ij).
* :func:`round_values`  -- storage rounding of the edge weights (round to
  nearest even into binary32 / bfloat16 / binary16), an implementation choice
  the paper does not make (its precision is unstated).
* :func:`degrees`       -- d_i = sum_j w_ij (Sec. 2.1).
* :func:`apply`         -- one product with A~_sigma (Eq. 16) or its random-walk form.
* :func:`gift`          -- Eq. 15 with the Sec. 4.1 coefficients; fixed cells
  reimposed (Sec. 3.2.2, Algorithm 1).
* :func:`hpwl`          -- half-perimeter wirelength (Sec. 4.1 reports it).
* :func:`largest_component`, :func:`eigen_placement` -- the eigenvector
  placer the paper analyses (Sec. 3.3.1, Eq. 23-24): eigenvectors of the
  graph Laplacian L = D - A (Sec. 2.1) for its second and third smallest
  eigenvalues, on the largest connected component.

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gift_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libgift_oracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "libgift_oracle_omp.so")

DEFAULT_TERMS = ((2.0, 2, 0.1), (4.0, 2, 0.7), (4.0, 4, 0.2))  # Eq. 15 + Sec. 4.1
FMT = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}


def build(threads: bool = False) -> str:
    """Compile the oracle library (gcc, -O2, no fast-math); threads=True: the
    OpenMP build (same results, the row loops over the host's cores)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    lib_path = _LIB_OMP if threads else _LIB
    if (not os.path.exists(lib_path)) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
        tmp = lib_path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", *(["-fopenmp"] if threads else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib_path)
    return lib_path


_lib = None
_threads = False


def use_threads(on: bool) -> None:
    """Switch between the single-threaded and the OpenMP build."""
    global _lib, _threads
    if on != _threads:
        _threads = on
        _lib = None


def threads() -> int:
    """Threads the loaded build runs its parallel loops on."""
    return int(lib().oracle_threads())


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build(_threads))
        P = C.c_void_p
        L.oracle_build.restype = P
        L.oracle_build.argtypes = [C.c_int32, C.c_int32, P, P]
        L.oracle_build_cut.restype = P
        L.oracle_build_cut.argtypes = [C.c_int32, C.c_int32, P, P, C.c_int64]
        L.oracle_implicit_degrees.restype = C.c_int
        L.oracle_implicit_degrees.argtypes = [C.c_int32, C.c_int32, P, P, C.c_int64, P]
        L.oracle_graph_nnz.restype = C.c_int64
        L.oracle_graph_nnz.argtypes = [P]
        L.oracle_graph_copy.argtypes = [P, P, P, P]
        L.oracle_graph_free.argtypes = [P]
        L.oracle_round.argtypes = [C.c_int64, P, P, C.c_int32]
        L.oracle_degrees.argtypes = [C.c_int32, P, P, P]
        L.oracle_apply.argtypes = [C.c_int32, C.c_int32, P, P, P, P, C.c_double, C.c_int32, P, P]
        L.oracle_filter.restype = C.c_int
        L.oracle_filter.argtypes = [C.c_int32, C.c_int32, P, P, P, P, C.c_int32, P, P, P,
                                    C.c_int32, C.c_int32, P, P, P]
        L.oracle_hpwl.argtypes = [C.c_int32, P, P, C.c_int32, P, P]
        L.oracle_threads.restype = C.c_int
        L.oracle_threads.argtypes = []
        L.oracle_apply_cut.restype = C.c_int
        L.oracle_apply_cut.argtypes = [C.c_int32, C.c_int32, P, P, P, P, C.c_double, C.c_int32, C.c_int32, P, P,
                                       C.c_int64, P, P]
        L.oracle_filter_cut.restype = C.c_int
        L.oracle_filter_cut.argtypes = [C.c_int32, C.c_int32, P, P, P, P, C.c_int32, P, P, P, C.c_int32, C.c_int32,
                                        P, C.c_int32, P, P, C.c_int64, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def build_graph(num_cells: int, net_ptr: np.ndarray, pin_cell: np.ndarray, cut: int = 0) -> Graph:
    """Clique expansion (weight 2/M, duplicates summed in net order) to CSR.
    cut > 0 leaves out the nets of at least `cut` pins (implicit cliques)."""
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pin_cell = np.ascontiguousarray(pin_cell, dtype=np.int32)
    if pin_cell.size == 0:
        pin_cell = np.zeros(1, dtype=np.int32)
    if cut > 0:
        h = lib().oracle_build_cut(int(num_cells), int(net_ptr.size - 1), _p(net_ptr), _p(pin_cell), int(cut))
    else:
        h = lib().oracle_build(int(num_cells), int(net_ptr.size - 1), _p(net_ptr), _p(pin_cell))
    if not h:
        raise ValueError("oracle_build rejected the netlist")
    try:
        nnz = lib().oracle_graph_nnz(h)
        rp = np.zeros(num_cells + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1), dtype=np.float64)
        lib().oracle_graph_copy(h, _p(rp), _p(col), _p(val))
    finally:
        lib().oracle_graph_free(h)
    return Graph(num_cells, rp, col[:nnz], val[:nnz])


def round_values(v: np.ndarray, fmt: str) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    if v.size:
        lib().oracle_round(v.size, _p(v), _p(out), FMT[fmt])
    return out


def stored(g: Graph, fmt: str) -> Graph:
    """The graph with its weights rounded to the storage format."""
    return Graph(g.n, g.row_ptr, g.col, round_values(g.val, fmt))


def degrees(g: Graph) -> np.ndarray:
    d = np.zeros(g.n, dtype=np.float64)
    val = g.val if g.val.size else np.zeros(1)
    lib().oracle_degrees(g.n, _p(g.row_ptr), _p(val), _p(d))
    return d


def implicit_degrees(d: np.ndarray, net_ptr: np.ndarray, pin_cell: np.ndarray, cut: int) -> np.ndarray:
    """d plus the degrees of the cliques of the nets of at least `cut` pins
    (nets in increasing order; k pins of a net of M on one cell add
    (k * 2/M) * (M - k))."""
    out = np.array(d, dtype=np.float64, copy=True)
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pin_cell = np.ascontiguousarray(pin_cell, dtype=np.int32)
    if pin_cell.size == 0:
        pin_cell = np.zeros(1, dtype=np.int32)
    if lib().oracle_implicit_degrees(out.size, int(net_ptr.size - 1), _p(net_ptr), _p(pin_cell), int(cut),
                                     _p(out)) != 0:
        raise MemoryError("oracle_implicit_degrees")
    return out


def tikhonov(g: Graph, d: np.ndarray, sig: np.ndarray, sigma: float, lam: float,
             is_fixed: np.ndarray | None = None, reimpose: bool = True) -> np.ndarray:
    """The exact smoothing GiFt approximates (Sec. 3.2.2, Eq. 18 with a weight
    lam on the smoothness term and the self-loop Laplacian I - A~_sigma):
    the solution of ((1 + lam) I - lam A~_sigma) g' = g in FP64, then the
    fixed rows put back.  The system's spectrum lies in [1, 1 + 2 lam), so
    conjugate gradients (written out below, one sparse product per step) run
    to a relative residual of 1e-13 put g' within (1 + 2 lam) 1e-13 of the
    exact solution, per column."""
    import scipy.sparse as sp
    n = g.n
    s = 1.0 / np.sqrt(d + sigma)
    A = sp.csr_matrix((g.val, g.col, g.row_ptr), shape=(n, n))

    def M(v):  # ((1 + lam) I - lam A~_sigma) v
        At_v = s[:, None] * (A @ (s[:, None] * v) + sigma * s[:, None] * v)
        return (1.0 + lam) * v - lam * At_v

    b = np.asarray(sig, dtype=np.float64).reshape(n, -1)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rs = (r * r).sum(axis=0)
    bn = np.sqrt((b * b).sum(axis=0))
    for _ in range(1000):
        if np.all(np.sqrt(rs) <= 1e-13 * np.maximum(bn, 1e-300)):
            break
        q = M(p)
        pq = (p * q).sum(axis=0)
        alpha = np.where(pq > 0, rs / np.where(pq > 0, pq, 1.0), 0.0)
        x += alpha * p
        r -= alpha * q
        rs_new = (r * r).sum(axis=0)
        beta = np.where(rs > 0, rs_new / np.where(rs > 0, rs, 1.0), 0.0)
        p = r + beta * p
        rs = rs_new
    else:
        raise RuntimeError("oracle tikhonov: no convergence")
    out = x.reshape(np.shape(sig))
    if reimpose and is_fixed is not None:
        fx = np.asarray(is_fixed).astype(bool)
        out[fx] = np.asarray(sig, dtype=np.float64)[fx]
    return out


def density(xy: np.ndarray, die, nx: int, ny: int, target: float, unit=(1.0, 1.0), cell_w=None, cell_h=None):
    """Bin density of a placement (Eq. 5): bins of the die, each cell a
    rectangle centred on its location, rho_b = area of the cells inside bin
    b.  Overlaps in FP64, quantised to (bin area) * 2^-40 (round half to
    even) and summed as integers; overflow = sum over bins (in order) of
    max(0, rho_b - target * bin area) / total cell area.
    Returns (integer bin sums [S][ny][nx], density [S][ny][nx], overflow [S])."""
    xy = np.asarray(xy, dtype=np.float32)
    N, S = xy.shape[0], xy.shape[1]
    x0, y0, x1, y1 = (float(v) for v in die)
    bw, bh = (x1 - x0) / nx, (y1 - y0) / ny
    inv_q = math.ldexp(1.0, 40) / (bw * bh)
    w = np.full(N, unit[0], np.float32) if cell_w is None else np.asarray(cell_w, np.float32)
    h = np.full(N, unit[1], np.float32) if cell_h is None else np.asarray(cell_h, np.float32)
    hw, hh = 0.5 * w.astype(np.float64), 0.5 * h.astype(np.float64)
    total = int(np.rint((2.0 * hw) * (2.0 * hh) * inv_q).astype(np.int64).sum())

    def first(lo, o, step, n):
        return np.clip(np.floor((lo - o) / step), 0, n - 1).astype(np.int64)

    def overlap(lo, hi, o, step, i):
        b0 = o + i.astype(np.float64) * step
        b1 = o + (i + 1).astype(np.float64) * step
        return np.maximum(np.minimum(hi, b1) - np.maximum(lo, b0), 0.0)

    counts = np.zeros((S, ny * nx), dtype=np.int64)
    for s in range(S):
        x, y = xy[:, s, 0].astype(np.float64), xy[:, s, 1].astype(np.float64)
        xl, xh, yl, yh = x - hw, x + hw, y - hh, y + hh
        i0, i1 = first(xl, x0, bw, nx), first(xh, x0, bw, nx)
        j0, j1 = first(yl, y0, bh, ny), first(yh, y0, bh, ny)
        for dj in range(int((j1 - j0).max()) + 1 if N else 0):
            for di in range(int((i1 - i0).max()) + 1):
                i, j = i0 + di, j0 + dj
                ok = (i <= i1) & (j <= j1)
                lx = overlap(xl, xh, x0, bw, i)
                ly = overlap(yl, yh, y0, bh, j)
                q = np.rint((lx * ly) * inv_q).astype(np.int64)
                ok &= (lx > 0) & (ly > 0) & (q > 0)
                np.add.at(counts[s], (j * nx + i)[ok], q[ok])
    dens = counts.astype(np.float64) * math.ldexp(1.0, -40)
    tq = target * math.ldexp(1.0, 40)
    over = np.zeros(S)
    for s in range(S):
        acc = 0.0
        for c in counts[s].astype(np.float64):
            if c > tq:
                acc += c - tq
        over[s] = acc / total if total > 0 else 0.0
    return counts.reshape(S, ny, nx), dens.reshape(S, ny, nx), over


def _csr_args(g: Graph):
    col = g.col if g.col.size else np.zeros(1, dtype=np.int32)
    val = g.val if g.val.size else np.zeros(1, dtype=np.float64)
    return g.row_ptr, np.ascontiguousarray(col), np.ascontiguousarray(val)


def apply(g: Graph, d: np.ndarray, sigma: float, x: np.ndarray, norm: str = "sym") -> np.ndarray:
    """One product y = A~_sigma x (Eq. 16; ``norm='rw'``: (D+sigma I)^-1 (A+sigma I) x)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = 1 if x.ndim == 1 else int(np.prod(x.shape[1:]))
    y = np.zeros_like(x)
    rp, col, val = _csr_args(g)
    lib().oracle_apply(g.n, K, _p(rp), _p(col), _p(val), _p(np.ascontiguousarray(d, dtype=np.float64)),
                       float(sigma), 0 if norm == "sym" else 1, _p(x), _p(y))
    return y


def _netlist_args(net_ptr, pin_cell):
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pin_cell = np.ascontiguousarray(pin_cell, dtype=np.int32)
    if pin_cell.size == 0:
        pin_cell = np.zeros(1, dtype=np.int32)
    return net_ptr, pin_cell


def apply_cut(g: Graph, d: np.ndarray, sigma: float, x: np.ndarray, net_ptr: np.ndarray, pin_cell: np.ndarray,
              cut: int, norm: str = "sym") -> np.ndarray:
    """One product y = A~_sigma x with the cliques of the nets of at least
    `cut` pins applied from the netlist (g holds the other nets, from
    build_graph(..., cut); d the degrees of the whole expansion)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = 1 if x.ndim == 1 else int(np.prod(x.shape[1:]))
    y = np.zeros_like(x)
    rp, col, val = _csr_args(g)
    npt, pc = _netlist_args(net_ptr, pin_cell)
    rc = lib().oracle_apply_cut(g.n, K, _p(rp), _p(col), _p(val), _p(np.ascontiguousarray(d, dtype=np.float64)),
                                float(sigma), 0 if norm == "sym" else 1, int(npt.size - 1), _p(npt), _p(pc), int(cut),
                                _p(x), _p(y))
    if rc != 0:
        raise MemoryError("oracle_apply_cut: out of memory")
    return y


def gift(g: Graph, d: np.ndarray, sig: np.ndarray, is_fixed: np.ndarray | None,
         terms=DEFAULT_TERMS, norm: str = "sym", reimpose: bool = True, implicit=None) -> np.ndarray:
    """GiFt (Eq. 15): sum_t alpha_t A~_{sigma_t}^{k_t} g, fixed rows reimposed.
    implicit = (net_ptr, pin_cell, cut): g holds the nets of fewer than cut
    pins and the larger nets' cliques are applied from the netlist."""
    x = np.ascontiguousarray(sig, dtype=np.float64)
    K = 1 if x.ndim == 1 else int(np.prod(x.shape[1:]))
    out = np.zeros_like(x)
    sg = np.array([t[0] for t in terms], dtype=np.float64)
    pw = np.array([t[1] for t in terms], dtype=np.int32)
    al = np.array([t[2] for t in terms], dtype=np.float64)
    fx = np.ascontiguousarray(is_fixed if is_fixed is not None else np.zeros(g.n), dtype=np.uint8)
    rp, col, val = _csr_args(g)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    if implicit is not None and implicit[2] > 0:
        npt, pc = _netlist_args(implicit[0], implicit[1])
        rc = lib().oracle_filter_cut(g.n, K, _p(rp), _p(col), _p(val), _p(dd), len(terms), _p(sg), _p(pw), _p(al),
                                     0 if norm == "sym" else 1, 1 if reimpose else 0, _p(fx), int(npt.size - 1),
                                     _p(npt), _p(pc), int(implicit[2]), _p(x), _p(out))
    else:
        rc = lib().oracle_filter(g.n, K, _p(rp), _p(col), _p(val), _p(dd), len(terms), _p(sg), _p(pw), _p(al),
                                 0 if norm == "sym" else 1, 1 if reimpose else 0, _p(fx), _p(x), _p(out))
    if rc != 0:
        raise MemoryError("oracle_filter: out of memory")
    return out


def hpwl(net_ptr: np.ndarray, pin_cell: np.ndarray, xy: np.ndarray) -> np.ndarray:
    """HPWL per signal of locations xy [N, S, 2]."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    S = xy.shape[1]
    out = np.zeros(S, dtype=np.float64)
    net_ptr = np.ascontiguousarray(net_ptr, dtype=np.int64)
    pc = np.ascontiguousarray(pin_cell, dtype=np.int32)
    if pc.size == 0:
        pc = np.zeros(1, dtype=np.int32)
    lib().oracle_hpwl(int(net_ptr.size - 1), _p(net_ptr), _p(pc), S, _p(xy), _p(out))
    return out


def run(nl, sig: np.ndarray, fmt: str = "f64", terms=DEFAULT_TERMS, norm: str = "sym",
        reimpose: bool = True, cut: int = 0):
    """Whole path for a netlist: (graph, degrees, filtered signal).

    ``fmt`` rounds the weights as the storage format would before the degrees
    are taken (degrees always over the stored weights).  ``cut`` > 0 applies
    the cliques of the nets of at least cut pins from the netlist (the same
    operator; for netlists whose full expansion is too large to form): the
    graph then holds the other nets, their weights rounded, and the degrees
    add the large nets' cliques exactly."""
    g = build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut)
    if fmt != "f64":
        g = stored(g, fmt)
    d = degrees(g)
    if cut > 0:
        d = implicit_degrees(d, nl.net_ptr, nl.pin_cell, cut)
    out = gift(g, d, sig, nl.is_fixed, terms, norm, reimpose,
               implicit=(nl.net_ptr, nl.pin_cell, cut) if cut > 0 else None)
    return g, d, out


def largest_component(g: Graph) -> np.ndarray:
    """Mask of the largest connected component of the graph (ties: the
    component holding the smallest cell id).  A library routine (scipy's
    breadth-first labelling) serves as the step."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    a = csr_matrix((np.ones(g.nnz), np.asarray(g.col, dtype=np.int64), g.row_ptr), shape=(g.n, g.n))
    ncomp, lab = connected_components(a, directed=False)
    sizes = np.bincount(lab, minlength=ncomp)
    first = np.full(ncomp, g.n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(g.n, dtype=np.int64))
    best = np.lexsort((first, -sizes))[0]
    return lab == best


def eigen_placement(g: Graph, d: np.ndarray):
    """Hall's eigenvector placement as the paper analyses it (Sec. 3.3.1,
    Eq. 23-24, an ideal low-pass filter keeping u_2 and u_3): the
    eigenvectors of the graph Laplacian L = D - A (Sec. 2.1, d_i the row sums
    of the stored weights) for its second and third smallest eigenvalues.

    The eigenvector placer assumes one connected graph; a netlist graph has
    cells without nets and small components, each adding an eigenvalue 0, so
    u_2 and u_3 are taken on the largest connected component and are 0 on
    every other cell.  Returns (u [n][2] FP64, unit 2-norm, sign arbitrary;
    (lambda_2, lambda_3); the component mask).  Dense symmetric
    eigendecomposition (numpy) for up to 2,000 component cells, else
    shift-invert Lanczos (scipy's ARPACK) around -1e-3 for the three
    eigenvalues nearest it (0, lambda_2, lambda_3)."""
    from scipy.sparse import csr_matrix, diags
    mask = largest_component(g)
    idx = np.flatnonzero(mask)
    m = idx.size
    if m < 3:
        raise ValueError("eigen_placement: the largest component has fewer than 3 cells")
    a = csr_matrix((np.asarray(g.val, dtype=np.float64), np.asarray(g.col, dtype=np.int64), g.row_ptr),
                   shape=(g.n, g.n))
    a = a[idx][:, idx]
    lap = (diags(np.asarray(d, dtype=np.float64)[idx]) - a).tocsc()
    if m <= 2000:
        w, v = np.linalg.eigh(lap.toarray())
    else:
        from scipy.sparse.linalg import eigsh
        w, v = eigsh(lap, k=3, sigma=-1e-3, which="LM", tol=0.0)
        order = np.argsort(w)
        w, v = w[order], v[:, order]
    u = np.zeros((g.n, 2), dtype=np.float64)
    u[idx, 0] = v[:, 1]
    u[idx, 1] = v[:, 2]
    return u, (float(w[1]), float(w[2])), mask
