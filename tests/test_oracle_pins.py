"""Pins that tie the FP64 oracle to the paper and to mathematics, not to itself.

Each check comes from a source independent of the oracle's code:
closed forms derived by hand (tests/golden), Theorem 1 and spectral facts,
a brute-force dense construction on tiny inputs, scipy's COO->CSR duplicate
summation, numpy's own float conversions, and hand-computed HPWL.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_f():
    out, ex = {}, None
    for line in open(os.path.join(GOLD, "single_net_filter.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "f":
            out[int(t[1])] = Fraction(int(t[2]), int(t[3]))
        elif t[0] == "example":
            ex = [float(v) for v in t[1:]]
    return out, ex


def _single_net(M, N=None):
    N = N or M
    net_ptr = np.array([0, M], dtype=np.int64)
    pin_cell = np.arange(M, dtype=np.int32)
    return N, net_ptr, pin_cell


# ---------------------------------------------------------------- closed forms
def test_single_net_closed_form():
    """GiFt on K_M equals mean + f_M (g - mean), f_M derived by hand."""
    fm, _ = _golden_f()
    for M, f in fm.items():
        N, rp, pc = _single_net(M)
        g = oracle.build_graph(N, rp, pc)
        d = oracle.degrees(g)
        assert np.allclose(d, 2.0 * (M - 1) / M, rtol=1e-13, atol=0)
        x = synth.uniform(7, 1, np.arange(M * 2, dtype=np.uint64)).reshape(M, 2) * 1000
        y = oracle.gift(g, d, x, None)
        mean = x.mean(axis=0)
        want = mean + float(f) * (x - mean)
        np.testing.assert_allclose(y, want, rtol=1e-13, atol=1e-11)


def test_golden_values_follow_their_derivation():
    """The fixture's rationals are the closed form its header derives, in
    exact arithmetic: r_s = (s - w) / (d + s), w = 2/M, d = w (M - 1),
    f_M = 0.1 r_2^2 + 0.7 r_4^2 + 0.2 r_4^4; the worked example is
    1/2 -+ f_2 / 2."""
    fm, ex = _golden_f()
    assert sorted(fm) == [2, 3, 4, 50]
    for M, f in fm.items():
        w = Fraction(2, M)
        d = w * (M - 1)
        r2, r4 = (2 - w) / (d + 2), (4 - w) / (d + 4)
        assert f == Fraction(1, 10) * r2 ** 2 + Fraction(7, 10) * r4 ** 2 + Fraction(2, 10) * r4 ** 4
    assert ex[:2] == [0.0, 1.0]
    assert ex[2] == pytest.approx(float(Fraction(1, 2) - fm[2] / 2), rel=0, abs=1e-16)
    assert ex[3] == pytest.approx(float(Fraction(1, 2) + fm[2] / 2), rel=0, abs=1e-16)


def test_worked_example_two_pin():
    _, ex = _golden_f()
    g = oracle.build_graph(2, np.array([0, 2]), np.array([0, 1], dtype=np.int32))
    y = oracle.gift(g, oracle.degrees(g), np.array([[ex[0]], [ex[1]]]), None)
    np.testing.assert_allclose(y[:, 0], ex[2:], rtol=0, atol=1e-15)


def test_no_edges_is_identity():
    """No net of >= 2 pins: A = 0, A~_s = I, and the alphas sum to 1."""
    rp = np.array([0, 0, 1, 2], dtype=np.int64)  # empty, 1-pin, 1-pin
    pc = np.array([3, 4], dtype=np.int32)
    g = oracle.build_graph(6, rp, pc)
    assert g.nnz == 0
    x = np.arange(12, dtype=np.float64).reshape(6, 2)
    np.testing.assert_allclose(oracle.gift(g, oracle.degrees(g), x, None), x, rtol=1e-15)


def test_single_net_per_term():
    """Each term alone on K_3: A~_s^k g = mean + r_s^k (g - mean)."""
    M = 3
    N, rp, pc = _single_net(M)
    g = oracle.build_graph(N, rp, pc)
    d = oracle.degrees(g)
    x = np.array([[1.0], [5.0], [9.0]])
    w = Fraction(2, M)
    dd = w * (M - 1)
    for s in (1, 2, 4, 7):
        for k in (1, 2, 3, 4):
            r = float(((s - w) / (dd + s)) ** k)
            y = oracle.gift(g, d, x, None, terms=((float(s), k, 1.0),))
            np.testing.assert_allclose(y[:, 0], 5.0 + r * (x[:, 0] - 5.0), rtol=1e-14)


# -------------------------------------------------------------- brute force
def _dense_reference(nl, x, terms=oracle.DEFAULT_TERMS, norm="sym", reimpose=True):
    """Independent dense construction: loops over nets and slot pairs, numpy powers."""
    N = nl.num_cells
    A = np.zeros((N, N))
    for e in range(nl.num_nets):
        cells = [int(c) for c in nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]]
        M = len(cells)
        if M < 2:
            continue
        for a in range(M):
            for b in range(M):
                if a != b and cells[a] != cells[b]:
                    A[cells[a], cells[b]] += 2.0 / M
    deg = A.sum(axis=1)
    out = np.zeros_like(x)
    for s, k, al in terms:
        if norm == "sym":
            S = np.diag(1.0 / np.sqrt(deg + s))
            T = S @ (A + s * np.eye(N)) @ S
        else:
            T = np.diag(1.0 / (deg + s)) @ (A + s * np.eye(N))
        out += al * (np.linalg.matrix_power(T, k) @ x)
    if reimpose:
        fx = nl.is_fixed.astype(bool)
        out[fx] = x[fx]
    return A, out


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_dense_brute_force(seed):
    rep = seed % 2 == 0
    nl = synth.random_small(seed, num_cells=24 + seed, num_nets=20 + 3 * seed, max_pins=7,
                            num_fixed=3, allow_repeat=rep)
    x = synth.uniform(seed, 9, np.arange(nl.num_cells * 4, dtype=np.uint64)).reshape(nl.num_cells, 4) * 1000
    A, want = _dense_reference(nl, x)
    g, d, got = oracle.run(nl, x)
    dense = np.zeros_like(A)
    for i in range(nl.num_cells):
        for k in range(g.row_ptr[i], g.row_ptr[i + 1]):
            dense[i, g.col[k]] = g.val[k]
    np.testing.assert_allclose(dense, A, rtol=1e-15, atol=0)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)
    # random-walk variant, no fixed rows
    _, want_rw = _dense_reference(nl, x, norm="rw", reimpose=False)
    got_rw = oracle.gift(g, d, x, nl.is_fixed, norm="rw", reimpose=False)
    np.testing.assert_allclose(got_rw, want_rw, rtol=1e-12, atol=1e-9)
    # arbitrary term list
    terms = ((1.0, 1, 0.25), (3.0, 3, 0.5), (0.5, 2, 0.25))
    _, want_t = _dense_reference(nl, x, terms=terms)
    np.testing.assert_allclose(oracle.gift(g, d, x, nl.is_fixed, terms=terms), want_t, rtol=1e-12, atol=1e-9)


def test_structure_matches_scipy_coo_sum_duplicates():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    nl = synth.random_small(11, num_cells=300, num_nets=400, max_pins=9, allow_repeat=True)
    rows, cols, ws = [], [], []
    for e in range(nl.num_nets):
        cells = nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]
        M = len(cells)
        if M < 2:
            continue
        for a in range(M):
            for b in range(M):
                if a != b and cells[a] != cells[b]:
                    rows.append(cells[a]); cols.append(cells[b]); ws.append(2.0 / M)
    ref = scipy_sparse.coo_matrix((ws, (rows, cols)), shape=(nl.num_cells,) * 2).tocsr()
    ref.sum_duplicates()
    ref.sort_indices()
    g = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell)
    np.testing.assert_array_equal(g.row_ptr, ref.indptr)
    np.testing.assert_array_equal(g.col, ref.indices)
    np.testing.assert_allclose(g.val, ref.data, rtol=1e-15)


# ------------------------------------------------------------ invariants
def _small_graph(seed=21, N=40, E=50):
    nl = synth.random_small(seed, num_cells=N, num_nets=E, max_pins=6, min_pins=2)
    g = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell)
    return nl, g, oracle.degrees(g)


def _dense_op(g, d, sigma, norm="sym"):
    return oracle.apply(g, d, sigma, np.eye(g.n), norm=norm)


def test_theorem1_top_eigenvector():
    """A~_s (d + s)^(1/2) = (d + s)^(1/2): eigenvalue 1 (Theorem 1 with self-loops)."""
    _, g, d = _small_graph()
    for s in (2.0, 4.0, 1.0):
        v = np.sqrt(d + s)
        np.testing.assert_allclose(oracle.apply(g, d, s, v), v, rtol=1e-13)
        y = v
        for _ in range(4):
            y = oracle.apply(g, d, s, y)
        np.testing.assert_allclose(y, v, rtol=1e-12)


def test_spectrum_bounds():
    """Eigenvalues of A~_s lie in [-1 + 2s/(d_max + s), 1] and the top one is 1."""
    _, g, d = _small_graph()
    for s in (2.0, 4.0):
        T = _dense_op(g, d, s)
        np.testing.assert_allclose(T, T.T, atol=1e-14)
        ev = np.linalg.eigvalsh(T)
        assert ev.max() == pytest.approx(1.0, abs=1e-12)
        assert ev.min() >= -1 + 2 * s / (d.max() + s) - 1e-12
        # Theorem 1: A~ = I - L~ with L~ the normalised Laplacian of the self-looped graph
        Aself = np.zeros((g.n, g.n))
        for i in range(g.n):
            Aself[i, g.col[g.row_ptr[i]:g.row_ptr[i + 1]]] = g.val[g.row_ptr[i]:g.row_ptr[i + 1]]
        Aself += s * np.eye(g.n)
        Dh = np.diag(1.0 / np.sqrt(Aself.sum(axis=1)))
        Lt = np.eye(g.n) - Dh @ Aself @ Dh
        np.testing.assert_allclose(np.sort(1.0 - np.linalg.eigvalsh(Lt)), np.sort(ev), atol=1e-12)


def test_gift_operator_symmetric_psd_contraction():
    _, g, d = _small_graph(seed=5)
    G = oracle.gift(g, d, np.eye(g.n), None, reimpose=False)
    np.testing.assert_allclose(G, G.T, atol=1e-14)
    ev = np.linalg.eigvalsh(G)
    assert ev.min() >= -1e-13
    assert ev.max() <= 1.0 + 1e-12
    assert ev.max() == pytest.approx(1.0, abs=1e-12)


def test_random_walk_keeps_constants():
    _, g, d = _small_graph(seed=8)
    c = np.full((g.n, 2), 3.25)
    np.testing.assert_allclose(oracle.gift(g, d, c, None, norm="rw", reimpose=False), c, rtol=1e-13)


def test_linearity_nonnegativity_columns():
    nl, g, d = _small_graph(seed=9)
    rng = synth.uniform(3, 3, np.arange(g.n * 4, dtype=np.uint64)).reshape(g.n, 4)
    a, b = rng[:, :2], rng[:, 2:]
    ga = oracle.gift(g, d, a, None, reimpose=False)
    gb = oracle.gift(g, d, b, None, reimpose=False)
    gab = oracle.gift(g, d, 2.0 * a - 3.0 * b, None, reimpose=False)
    np.testing.assert_allclose(gab, 2 * ga - 3 * gb, rtol=1e-11, atol=1e-12)
    assert (ga >= 0).all()
    # x and y columns are treated identically
    sw = oracle.gift(g, d, a[:, ::-1], None, reimpose=False)
    np.testing.assert_array_equal(sw, ga[:, ::-1])


def test_permutation_equivariance():
    nl = synth.random_small(13, num_cells=60, num_nets=70, max_pins=6, num_fixed=4)
    perm = (synth.u64(1, 1, np.arange(60, dtype=np.uint64)) % np.uint64(1 << 40)).argsort()
    inv = np.empty_like(perm); inv[perm] = np.arange(60)
    x = synth.uniform(2, 2, np.arange(120, dtype=np.uint64)).reshape(60, 2) * 100
    _, _, y = oracle.run(nl, x)
    nl2 = synth.Netlist(60, nl.num_nets, nl.net_ptr, inv[nl.pin_cell].astype(np.int32),
                        nl.is_fixed[perm], nl.fixed_xy[perm])
    _, _, y2 = oracle.run(nl2, x[perm])
    np.testing.assert_allclose(y2, y[perm], rtol=1e-12)


def test_fixed_rows_reimposed_exactly():
    nl = synth.random_small(17, num_cells=50, num_nets=60, max_pins=5, num_fixed=7)
    x = synth.uniform(4, 4, np.arange(100, dtype=np.uint64)).reshape(50, 2) * 1000
    g, d, y = oracle.run(nl, x)
    y0 = oracle.gift(g, d, x, nl.is_fixed, reimpose=False)
    fx = nl.is_fixed.astype(bool)
    np.testing.assert_array_equal(y[fx], x[fx])
    np.testing.assert_array_equal(y[~fx], y0[~fx])


def test_rejects_bad_netlists():
    with pytest.raises(ValueError):
        oracle.build_graph(3, np.array([0, 2]), np.array([0, 3], dtype=np.int32))
    with pytest.raises(ValueError):
        oracle.build_graph(3, np.array([0, 2, 1]), np.array([0, 1], dtype=np.int32))


# ---------------------------------------------------------- storage rounding
def test_round_f32_f16_match_numpy():
    v = np.concatenate([2.0 / np.arange(2, 3000), np.cumsum(2.0 / np.arange(2, 500)),
                        synth.uniform(5, 5, np.arange(5000, dtype=np.uint64)) * 7,
                        [1e-6, 3e-5, 6.1e-5, 65504.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11]])
    np.testing.assert_array_equal(oracle.round_values(v, "f32"), v.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(oracle.round_values(v, "f16"), v.astype(np.float16).astype(np.float64))


def _bf16_neighbours(v):
    f = np.float32(v)
    b = np.frombuffer(np.float32(f).tobytes(), dtype=np.uint32)[0] & np.uint32(0xFFFF0000)
    cands = []
    for k in (-1, 0, 1, 2):
        bits = np.uint32((int(b) + (k << 16)) & 0xFFFFFFFF)
        cands.append(float(np.frombuffer(bits.tobytes(), dtype=np.float32)[0]))
    return cands


def test_round_bf16_is_nearest_even():
    v = np.concatenate([2.0 / np.arange(2, 2001), np.cumsum(2.0 / np.arange(2, 300)),
                        synth.uniform(6, 6, np.arange(3000, dtype=np.uint64)) * 50,
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 0.6669921875]])
    got = oracle.round_values(v, "bf16")
    for x, r in zip(v, got):
        cands = _bf16_neighbours(x)
        fx = Fraction(x)
        best = min(abs(Fraction(c) - fx) for c in cands)
        near = [c for c in cands if abs(Fraction(c) - fx) == best]
        if len(near) == 1:
            assert r == near[0], (x, r, near)
        else:  # tie: even significand (low bf16 bit clear)
            even = [c for c in near if (np.frombuffer(np.float32(c).tobytes(), np.uint32)[0] >> 16) & 1 == 0]
            assert r == even[0]


def test_bf16_degrees_use_stored_weights():
    """With rounded weights the operator stays normalised (Theorem 1 holds exactly)."""
    nl = synth.random_small(19, num_cells=40, num_nets=50, max_pins=7, min_pins=2)
    g = oracle.stored(oracle.build_graph(40, nl.net_ptr, nl.pin_cell), "bf16")
    d = oracle.degrees(g)
    v = np.sqrt(d + 4.0)
    np.testing.assert_allclose(oracle.apply(g, d, 4.0, v), v, rtol=1e-13)
    # the whole path rounds before it takes the degrees: every weight is a
    # bf16 value and each degree is the plain sum of its row's stored weights
    x = synth.uniform(19, 19, np.arange(80, dtype=np.uint64)).reshape(40, 2)
    g2, d2, _ = oracle.run(nl, x, fmt="bf16")
    np.testing.assert_array_equal(g2.val, g.val)
    for i in range(40):
        assert d2[i] == pytest.approx(math.fsum(g2.val[g2.row_ptr[i]:g2.row_ptr[i + 1]]), rel=1e-15)
    assert any(abs(d2[i] - oracle.degrees(oracle.build_graph(40, nl.net_ptr, nl.pin_cell))[i]) > 1e-6
               for i in range(40))  # the rounding is visible in the degrees


# ------------------------------------------------------------------ HPWL
def test_hpwl_hand_example():
    cells, nets, want = {}, [], None
    for line in open(os.path.join(GOLD, "hpwl_hand.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "cell":
            cells[int(t[1])] = (float(t[2]), float(t[3]))
        elif t[0] == "net":
            nets.append([int(c) for c in t[1:]])
        elif t[0] == "hpwl":
            want = float(t[1])
    xy = np.array([cells[i] for i in range(len(cells))])[:, None, :]
    net_ptr = np.concatenate([[0], np.cumsum([len(n) for n in nets])])
    pc = np.array([c for n in nets for c in n], dtype=np.int32)
    assert oracle.hpwl(net_ptr, pc, xy)[0] == want


def test_hpwl_brute_force():
    nl = synth.random_small(23, num_cells=80, num_nets=90, max_pins=8)
    xy = synth.uniform(8, 8, np.arange(80 * 3 * 2, dtype=np.uint64)).reshape(80, 3, 2) * 1000
    got = oracle.hpwl(nl.net_ptr, nl.pin_cell, xy)
    for s in range(3):
        tot = 0.0
        for e in range(nl.num_nets):
            cs = nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]]
            if len(cs) == 0:
                continue
            p = xy[cs, s, :]
            tot += (p[:, 0].max() - p[:, 0].min()) + (p[:, 1].max() - p[:, 1].min())
        assert got[s] == pytest.approx(tot, rel=1e-14)


# ------------------------------------------------------------ implicit cliques
@pytest.mark.parametrize("cut", [2, 3, 4, 6, 50])
@pytest.mark.parametrize("repeat", [False, True])
def test_cut_graph_plus_implicit_degrees_equal_full_degrees(cut, repeat):
    """Leaving the nets of >= cut pins out of the expansion and adding their
    cliques' degrees gives the full clique's degrees (FP64 weights, sums in
    another order)."""
    nl = synth.random_small(41 + cut, 60, 90, 9, num_fixed=2, allow_repeat=repeat)
    full = oracle.degrees(oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell))
    G = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut)
    d = oracle.implicit_degrees(oracle.degrees(G), nl.net_ptr, nl.pin_cell, cut)
    np.testing.assert_allclose(d, full, rtol=1e-14, atol=1e-15)
    # the cut graph holds exactly the pairs of the smaller nets
    M = np.diff(nl.net_ptr)
    small = synth.Netlist(nl.num_cells, 0, np.array([0], dtype=np.int64), np.zeros(0, np.int32),
                          nl.is_fixed, nl.fixed_xy)
    keep = [e for e in range(nl.num_nets) if M[e] < cut]
    ptr = np.concatenate([[0], np.cumsum([M[e] for e in keep])]).astype(np.int64)
    pins = np.concatenate([nl.pin_cell[nl.net_ptr[e]:nl.net_ptr[e + 1]] for e in keep] or
                          [np.zeros(0, np.int32)]).astype(np.int32)
    Gs = oracle.build_graph(small.num_cells, ptr, pins)
    np.testing.assert_array_equal(G.row_ptr, Gs.row_ptr)
    np.testing.assert_array_equal(G.col, Gs.col)
    np.testing.assert_array_equal(G.val, Gs.val)


@pytest.mark.parametrize("M,k", [(2, 1), (5, 1), (5, 2), (7, 3), (9, 4)])
def test_implicit_degree_of_one_net_by_pair_count(M, k):
    """One net of M pins, k of them on cell 0 and the rest on distinct cells:
    cell 0 has k (M - k) ordered pairs with other cells, each of weight 2/M."""
    cells = [0] * k + list(range(1, M - k + 1))
    nl_ptr = np.array([0, M], dtype=np.int64)
    pins = np.array(cells, dtype=np.int32)
    n = M - k + 1
    d = oracle.implicit_degrees(np.zeros(n), nl_ptr, pins, cut=2)
    assert d[0] == (k * (2.0 / M)) * (M - k)
    for c in range(1, n):
        assert d[c] == (1 * (2.0 / M)) * (M - 1)
    G = oracle.build_graph(n, nl_ptr, pins, cut=2)
    assert G.nnz == 0


@pytest.mark.parametrize("cut", [2, 3, 5, 50])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_implicit_apply_matches_dense_brute_force(seed, cut):
    """The product with the large nets' cliques applied from the netlist
    equals the independent dense construction's product (repeated cells
    included), in both normalisations and for two sigmas, and so does the
    whole filter built that way."""
    nl = synth.random_small(seed + 60, num_cells=30 + seed, num_nets=26 + 4 * seed, max_pins=8, num_fixed=2,
                            allow_repeat=seed != 2)
    x = synth.uniform(seed, 9, np.arange(nl.num_cells * 4, dtype=np.uint64)).reshape(nl.num_cells, 4) * 1000
    A, want = _dense_reference(nl, x)
    deg = A.sum(axis=1)
    G = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell, cut=cut)
    d = oracle.implicit_degrees(oracle.degrees(G), nl.net_ptr, nl.pin_cell, cut)
    for sigma in (2.0, 4.0):
        S = np.diag(1.0 / np.sqrt(deg + sigma))
        ref_sym = S @ (A + sigma * np.eye(nl.num_cells)) @ S @ x
        ref_rw = np.diag(1.0 / (deg + sigma)) @ (A + sigma * np.eye(nl.num_cells)) @ x
        got_sym = oracle.apply_cut(G, d, sigma, x, nl.net_ptr, nl.pin_cell, cut)
        got_rw = oracle.apply_cut(G, d, sigma, x, nl.net_ptr, nl.pin_cell, cut, norm="rw")
        np.testing.assert_allclose(got_sym, ref_sym, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(got_rw, ref_rw, rtol=1e-12, atol=1e-9)
    _, _, got = oracle.run(nl, x, cut=cut)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)


def test_implicit_single_net_closed_form():
    """GiFt on K_M with the clique applied from the netlist (every net
    implicit) equals mean + f_M (g - mean), f_M derived by hand."""
    fm, _ = _golden_f()
    for M, f in fm.items():
        N, rp, pc = _single_net(M)
        nl = synth.Netlist(N, 1, rp, pc, np.zeros(N, np.uint8), np.zeros((N, 2), np.float32), 1000.0, {})
        x = synth.uniform(7, 1, np.arange(M * 2, dtype=np.uint64)).reshape(M, 2) * 1000
        G, d, y = oracle.run(nl, x, cut=2)
        assert G.nnz == 0
        np.testing.assert_allclose(d, 2.0 * (M - 1) / M, rtol=1e-13, atol=0)
        mean = x.mean(axis=0)
        np.testing.assert_allclose(y, mean + float(f) * (x - mean), rtol=1e-13, atol=1e-11)


# ------------------------------------------------------------ Tikhonov smoothing
@pytest.mark.parametrize("M", [2, 3, 7])
@pytest.mark.parametrize("sigma,lam", [(2.0, 1.0), (4.0, 0.5), (1.0, 3.0)])
def test_tikhonov_single_net_closed_form(M, sigma, lam):
    """One M-pin clique: A~_sigma keeps constants (eigenvalue 1) and scales the
    zero-mean part by r = (sigma - w) / (d + sigma), w = 2/M, d = (M - 1) w, so
    ((1 + lam) I - lam A~)^-1 g = mean + (g - mean) / (1 + lam (1 - r))."""
    N, ptr, pins = _single_net(M)
    G = oracle.build_graph(N, ptr, pins)
    d = oracle.degrees(G)
    g = np.linspace(0.0, 7.0, 2 * N).reshape(N, 2) ** 1.5
    got = oracle.tikhonov(G, d, g, sigma, lam, reimpose=False)
    w = 2.0 / M
    r = (sigma - w) / ((M - 1) * w + sigma)
    mean = g.mean(axis=0)
    np.testing.assert_allclose(got, mean + (g - mean) / (1.0 + lam * (1.0 - r)), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("sigma,lam", [(2.0, 1.0), (4.0, 2.0)])
def test_tikhonov_dense_brute_force(seed, sigma, lam):
    nl = synth.random_small(seed + 60, 30, 40, 6, num_fixed=3, allow_repeat=seed == 3)
    x = synth.make_signals(nl, 2, seed).reshape(nl.num_cells, -1).astype(np.float64)
    A, _ = _dense_reference(nl, x)
    deg = A.sum(axis=1)
    S = np.diag(1.0 / np.sqrt(deg + sigma))
    T = S @ (A + sigma * np.eye(nl.num_cells)) @ S
    want = np.linalg.solve((1.0 + lam) * np.eye(nl.num_cells) - lam * T, x)
    fx = nl.is_fixed.astype(bool)
    want[fx] = x[fx]
    G = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell)
    got = oracle.tikhonov(G, oracle.degrees(G), x, sigma, lam, nl.is_fixed)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10)


def test_tikhonov_without_smoothing_is_identity():
    nl = synth.random_small(71, 25, 30, 5)
    x = synth.make_signals(nl, 1, 3).reshape(nl.num_cells, -1).astype(np.float64)
    G = oracle.build_graph(nl.num_cells, nl.net_ptr, nl.pin_cell)
    np.testing.assert_allclose(oracle.tikhonov(G, oracle.degrees(G), x, 2.0, 0.0, reimpose=False), x, rtol=1e-14)


# ------------------------------------------------------------ bin density (Eq. 5)
def test_density_hand_cases():
    """4 x 4 bins of 10 x 10 on [0, 40)^2.  A 2 x 2 cell centred in bin (1, 2)
    puts its area 4 there (density 0.04); a 2 x 2 cell centred on the corner
    shared by bins (2,2), (3,2), (2,3), (3,3) puts 1 in each; a cell outside
    the die adds nothing."""
    xy = np.array([[[15.0, 25.0]], [[30.0, 30.0]], [[-50.0, 5.0]]], dtype=np.float32)  # [N=3][S=1][2]
    counts, dens, over = oracle.density(xy, (0, 0, 40, 40), 4, 4, target=1.0, unit=(2.0, 2.0))
    q = math.ldexp(1.0, 40) / 100.0  # quanta per unit area
    want = np.zeros((4, 4))
    want[2, 1] = 4.0
    for j, i in ((2, 2), (2, 3), (3, 2), (3, 3)):
        want[j, i] = 1.0
    np.testing.assert_array_equal(counts[0], np.rint(want * q).astype(np.int64))
    np.testing.assert_allclose(dens[0], want / 100.0, rtol=0, atol=math.ldexp(1.0, -40))  # one quantum
    assert over[0] == 0.0  # every bin far below its area


def test_density_conserves_area_and_counts_overflow():
    rng_xy = synth.uniform(5, synth.T_MISC, np.arange(2000, dtype=np.uint64)).reshape(1000, 1, 2) * 900.0 + 50.0
    xy = rng_xy.astype(np.float32)
    counts, dens, over = oracle.density(xy, (0, 0, 1000, 1000), 16, 16, target=0.0, unit=(3.0, 5.0))
    q = math.ldexp(1.0, 40) / (62.5 * 62.5)
    total = round(15.0 * q) * 1000
    # every cell lies inside the die: the pieces add up to the cells' area, up
    # to half a quantum per piece (at most 4 pieces per cell here)
    assert abs(int(counts.sum()) - total) <= 4 * 1000
    # target 0: every quantum is overflow
    assert abs(over[0] - counts.sum() / total) <= 1e-12
    # one cell per bin, each bin exactly half covered by a cell, target 0.5: no overflow
    c = (np.arange(4) + 0.5) * 25.0
    X, Y = np.meshgrid(c, c)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)[:, None, :].astype(np.float32)
    _, dens, over = oracle.density(xy, (0, 0, 100, 100), 4, 4, target=0.5, unit=(25.0, 12.5))
    np.testing.assert_allclose(dens[0], 0.5, rtol=0, atol=math.ldexp(1.0, -40))
    assert over[0] == 0.0


def test_density_overflow_hand_case():
    """Two bins of 10 x 10 on [0, 20) x [0, 10), target 0.5 (capacity 50 per
    bin).  Three 5 x 5 cells stacked in bin 0 (area 75) and one in bin 1
    (area 25): only bin 0 overflows, by 25, over a total cell area of 100.
    The same three cells alone in one bin overflow it by 25 of 75."""
    xy = np.array([[[5.0, 5.0]], [[5.0, 5.0]], [[5.0, 5.0]], [[15.0, 5.0]]], dtype=np.float32)
    counts, dens, over = oracle.density(xy, (0, 0, 20, 10), 2, 1, target=0.5, unit=(5.0, 5.0))
    np.testing.assert_array_equal(dens[0], [[0.75, 0.25]])
    assert over[0] == 0.25
    _, dens, over = oracle.density(xy[:3], (0, 0, 10, 10), 1, 1, target=0.5, unit=(5.0, 5.0))
    assert dens[0, 0, 0] == 0.75
    assert over[0] == 25.0 / 75.0
