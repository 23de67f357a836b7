"""Seeded synthetic netlists and location signals.

This module produces INPUTS only: netlists (net_ptr / pin_cell / is_fixed) and
initial (x, y) signals.  It holds none of the filter's arithmetic, so both the
CUDA path and the CPU oracle may consume what it generates.

Random numbers come from a counter-based SplitMix64 stream: output k of stream
``tag`` under ``seed`` is ``mix64(key(seed, tag) + (k + 1) * GAMMA)`` where
``mix64`` is the SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Every draw is addressed by an
explicit counter, so a netlist is a pure function of (law, sizes, seed).

Workload laws (the paper measures on ISPD2014, which is not available here; the
synthetic designs take its shapes: tens of thousands to millions of cells, about
one net per cell, mostly 2- and 3-pin nets):

* pin count ``"geom"``: 2 with probability 0.6, else ``min(2 + G, 50)`` with
  ``G ~ Geometric(p=0.35)`` on {1, 2, ...};
* pin count ``"zipf"``: ``min(1 + Z, cap)`` with ``Z ~ Zipf(s)`` on {1, 2, ...}
  (heavy-tailed clock/reset-like nets);
* the pins of one net sit on distinct cells drawn uniformly over all cells;
* fixed IO cells are the last ``num_fixed`` cells, uniform on the die perimeter;
* movable initial locations are uniform over the die (or, in the paper's own
  mode, ``N(0, 1)`` around the die centre, Algorithm 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags: one per kind of draw
T_PINCOUNT, T_GEOM, T_CELL, T_FIXPOS, T_SIGNAL, T_MISC = 1, 2, 3, 4, 5, 6
T_REDRAW = 100  # + round number


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
        t = _mix64(np.array([tag], dtype=np.uint64) + GAMMA)
        return _mix64(base ^ t)[0]


def u64(seed: int, tag: int, counters: np.ndarray) -> np.ndarray:
    """Output ``counters`` of stream ``tag`` (uint64)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, tag) + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, tag: int, counters: np.ndarray) -> np.ndarray:
    """Uniform float64 on [0, 1) with 53 random bits."""
    return (u64(seed, tag, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _zeta(s: float, k: int = 20000) -> float:
    # partial sum + Euler-Maclaurin tail
    n = np.arange(1, k, dtype=np.float64)
    head = float(np.sum(n ** -s))
    return head + k ** (1 - s) / (s - 1) + 0.5 * k ** -s + s * k ** (-s - 1) / 12.0


@dataclass
class Netlist:
    num_cells: int
    num_nets: int
    net_ptr: np.ndarray      # int64 [E+1]
    pin_cell: np.ndarray     # int32 [P]
    is_fixed: np.ndarray     # uint8 [N]
    fixed_xy: np.ndarray     # float32 [N, 2] (rows of movable cells are 0)
    die: float = 1000.0
    meta: dict = field(default_factory=dict)

    @property
    def num_pins(self) -> int:
        return int(self.net_ptr[-1])


def pin_counts(law: str, num_nets: int, seed: int, cap: int, zipf_s: float = 2.2) -> np.ndarray:
    idx = np.arange(num_nets, dtype=np.uint64)
    if law == "geom":
        u = uniform(seed, T_PINCOUNT, idx)
        v = uniform(seed, T_GEOM, idx)
        g = np.ceil(np.log1p(-v) / math.log1p(-0.35))
        g = np.maximum(g, 1.0)
        m = np.where(u < 0.6, 2.0, np.minimum(2.0 + g, float(cap)))
        return m.astype(np.int64)
    if law == "zipf":
        kmax = cap  # Z >= cap - 1 is capped anyway
        ks = np.arange(1, kmax, dtype=np.float64)
        p = ks ** -zipf_s / _zeta(zipf_s)
        cdf = np.cumsum(p)
        u = uniform(seed, T_PINCOUNT, idx)
        z = np.searchsorted(cdf, u, side="right") + 1  # in 1..kmax
        return np.minimum(1 + z, cap).astype(np.int64)
    raise ValueError(f"unknown pin-count law {law!r}")


def draw_cells(m: np.ndarray, num_cells: int, seed: int, distinct: bool = True) -> np.ndarray:
    """Uniform cells for every pin slot; with ``distinct`` a net never repeats a cell."""
    E = m.shape[0]
    P = int(m.sum())
    slots = np.arange(P, dtype=np.uint64)
    cells = np.floor(uniform(seed, T_CELL, slots) * num_cells).astype(np.int64)
    if not distinct or P == 0:
        return cells.astype(np.int32)
    if np.any(m > num_cells):
        raise ValueError("a net has more pins than there are cells")
    net_of = np.repeat(np.arange(E, dtype=np.int64), m)
    rnd = 0
    while True:
        order = np.lexsort((np.arange(P), cells, net_of))
        sc, sn = cells[order], net_of[order]
        dup = (sn[1:] == sn[:-1]) & (sc[1:] == sc[:-1])
        if not dup.any():
            break
        where = order[1:][dup]
        rnd += 1
        cells[where] = np.floor(
            uniform(seed, T_REDRAW + rnd, where.astype(np.uint64)) * num_cells).astype(np.int64)
    return cells.astype(np.int32)


def perimeter_xy(num: int, die: float, seed: int) -> np.ndarray:
    t = uniform(seed, T_FIXPOS, np.arange(num, dtype=np.uint64)) * 4.0 * die
    side = np.minimum(np.floor(t / die), 3).astype(np.int64)
    off = t - side * die
    x = np.select([side == 0, side == 1, side == 2], [off, np.full_like(off, die), die - off], 0.0)
    y = np.select([side == 0, side == 1, side == 2], [0.0, off, np.full_like(off, die)], die - off)
    return np.stack([x, y], axis=1)


def make_netlist(num_movable: int, num_fixed: int, num_nets: int, seed: int,
                 law: str = "geom", cap: int = 50, die: float = 1000.0,
                 zipf_s: float = 2.2) -> Netlist:
    N = num_movable + num_fixed
    m = pin_counts(law, num_nets, seed, min(cap, N), zipf_s)
    net_ptr = np.zeros(num_nets + 1, dtype=np.int64)
    np.cumsum(m, out=net_ptr[1:])
    pin_cell = draw_cells(m, N, seed)
    is_fixed = np.zeros(N, dtype=np.uint8)
    is_fixed[num_movable:] = 1
    fixed_xy = np.zeros((N, 2), dtype=np.float32)
    if num_fixed:
        fixed_xy[num_movable:] = perimeter_xy(num_fixed, die, seed).astype(np.float32)
    return Netlist(N, num_nets, net_ptr, pin_cell, is_fixed, fixed_xy, die,
                   dict(law=law, seed=seed, num_movable=num_movable, num_fixed=num_fixed))


def lattice_netlist(nx: int, ny: int, num_nets: int, seed: int, max_pins: int = 4, radius: int = 2) -> Netlist:
    """A netlist with locality: cells on an nx x ny lattice (cell r * nx + c),
    each net an anchor cell drawn uniformly plus 1..max_pins-1 cells at
    offsets drawn uniformly in [-radius, radius]^2 (clamped to the lattice;
    repeated cells dropped, so a net may shrink).  Placement-like structure:
    the graph's low Laplacian eigenvalues are separated, unlike a uniform
    random netlist's."""
    N = nx * ny
    idx = np.arange(num_nets, dtype=np.uint64)
    anchor = np.minimum(np.floor(uniform(seed, T_CELL, idx) * N), N - 1).astype(np.int64)
    extra = 1 + np.floor(uniform(seed, T_PINCOUNT, idx) * (max_pins - 1)).astype(np.int64)
    off = np.floor(uniform(seed, T_GEOM, np.arange(num_nets * (max_pins - 1) * 2, dtype=np.uint64))
                   * (2 * radius + 1)).astype(np.int64).reshape(num_nets, max_pins - 1, 2) - radius
    ar, ac = anchor // nx, anchor % nx
    rr = np.clip(ar[:, None] + off[:, :, 0], 0, ny - 1)
    cc = np.clip(ac[:, None] + off[:, :, 1], 0, nx - 1)
    others = rr * nx + cc
    nets = []
    for e in range(num_nets):
        cells = [int(anchor[e])]
        for c in others[e, :extra[e]]:
            if int(c) not in cells:
                cells.append(int(c))
        nets.append(cells)
    net_ptr = np.zeros(num_nets + 1, dtype=np.int64)
    np.cumsum([len(c) for c in nets], out=net_ptr[1:])
    pin_cell = np.array([c for n in nets for c in n], dtype=np.int32)
    return Netlist(N, num_nets, net_ptr, pin_cell, np.zeros(N, dtype=np.uint8), np.zeros((N, 2), np.float32),
                   1000.0, dict(law="lattice", seed=seed, nx=nx, ny=ny))


def make_signals(nl: Netlist, num_signals: int, seed: int, mode: str = "uniform") -> np.ndarray:
    """Initial locations g, float32 [N, S, 2]; fixed rows hold their positions."""
    N, S = nl.num_cells, num_signals
    cnt = np.arange(N * S * 2, dtype=np.uint64)
    if mode == "uniform":
        g = uniform(seed, T_SIGNAL, cnt) * nl.die
    elif mode == "centre":
        u1 = uniform(seed, T_SIGNAL, cnt)
        u2 = uniform(seed, T_MISC, cnt)
        g = nl.die / 2 + np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2 * np.pi * u2)
    else:
        raise ValueError(mode)
    g = g.reshape(N, S, 2).astype(np.float32)
    fx = nl.is_fixed.astype(bool)
    g[fx] = nl.fixed_xy[fx][:, None, :]
    return np.ascontiguousarray(g)


def random_small(seed: int, num_cells: int, num_nets: int, max_pins: int,
                 num_fixed: int = 0, allow_repeat: bool = False, min_pins: int = 0) -> Netlist:
    """Tiny irregular netlists for tests: nets of 0..max_pins pins, optionally
    with a cell repeated inside a net."""
    idx = np.arange(num_nets, dtype=np.uint64)
    span = max_pins - min_pins + 1
    m = (min_pins + np.floor(uniform(seed, T_PINCOUNT, idx) * span)).astype(np.int64)
    if not allow_repeat:
        m = np.minimum(m, num_cells)
    net_ptr = np.zeros(num_nets + 1, dtype=np.int64)
    np.cumsum(m, out=net_ptr[1:])
    pin_cell = draw_cells(m, num_cells, seed, distinct=not allow_repeat)
    is_fixed = np.zeros(num_cells, dtype=np.uint8)
    fixed_xy = np.zeros((num_cells, 2), dtype=np.float32)
    if num_fixed:
        is_fixed[num_cells - num_fixed:] = 1
        fixed_xy[num_cells - num_fixed:] = perimeter_xy(num_fixed, 1000.0, seed).astype(np.float32)
    return Netlist(num_cells, num_nets, net_ptr, pin_cell, is_fixed, fixed_xy, 1000.0,
                   dict(law="small", seed=seed))


# ----------------------------------------------------------------------------
# Named workloads.  Seeds: 2502176320 + k for workload k.
# ----------------------------------------------------------------------------
SEED0 = 2502176320

WORKLOADS = {
    "plain-10k": dict(num_movable=10_000, num_fixed=200, num_nets=12_000, S=1, law="geom", cap=50, seed=SEED0 + 1),
    "large-2.2m": dict(num_movable=2_200_000, num_fixed=2_000, num_nets=2_300_000, S=8, law="geom", cap=50, seed=SEED0 + 2),
    "fanout-1.3m": dict(num_movable=1_287_000, num_fixed=13_000, num_nets=1_400_000, S=4, law="zipf", cap=2000, seed=SEED0 + 5),
}


def workload(name: str, scale: float = 1.0) -> tuple[Netlist, np.ndarray]:
    """Netlist + signals of a named single-graph workload (``scale`` shrinks it)."""
    w = WORKLOADS[name]
    mv = max(2, int(round(w["num_movable"] * scale)))
    fx = int(round(w["num_fixed"] * scale))
    ne = max(1, int(round(w["num_nets"] * scale)))
    nl = make_netlist(mv, fx, ne, w["seed"], law=w["law"], cap=w["cap"])
    g = make_signals(nl, w["S"], w["seed"])
    return nl, g


def batch_workload(num_graphs: int = 64, seed: int = SEED0 + 3, lo: int = 5_000, hi: int = 300_000,
                   S: int = 4, fixed_frac: float = 0.01, scale: float = 1.0):
    """Many uneven graphs: cells log-uniform in [lo, hi], nets/cell uniform in [1.0, 1.2]."""
    u = uniform(seed, T_MISC, np.arange(2 * num_graphs, dtype=np.uint64)).reshape(num_graphs, 2)
    out = []
    for k in range(num_graphs):
        n = int(round(math.exp(math.log(lo) + u[k, 0] * (math.log(hi) - math.log(lo))) * scale))
        n = max(n, 8)
        e = max(1, int(round(n * (1.0 + 0.2 * u[k, 1]))))
        nf = int(round(n * fixed_frac))
        nl = make_netlist(n - nf, nf, e, seed * 1000 + k, law="geom", cap=50)
        out.append((nl, make_signals(nl, S, seed * 1000 + k)))
    return out


def arrival_times(num: int, rate: float, seed: int) -> np.ndarray:
    """Poisson arrivals: cumulative exponential gaps (seconds)."""
    u = uniform(seed, T_MISC, np.arange(num, dtype=np.uint64))
    return np.cumsum(-np.log1p(-u) / rate)
