"""Pins of the oracle's eigenvector placement (Sec. 3.3.1, Eq. 23-24: u_2 and
u_3 of L = D - A, Sec. 2.1) against closed forms, not against the oracle's own
library calls: the unit-weight path P_n (eigenvalues 2 - 2cos(k pi / n),
eigenvectors cos(k pi (2i + 1) / 2n)), products of paths (grid graphs, sums
of the path eigenvalues), the cycle (a double eigenvalue: compared as a
subspace), a single M-pin net (L = w (M I - J), w = 2/M) and the component
rule (largest component, ties to the smallest cell id, zeros elsewhere).
Two-pin nets have weight 2/2 = 1, so these netlists give unit-weight graphs.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def netlist(num_cells, edges):
    net_ptr = np.arange(0, 2 * len(edges) + 1, 2, dtype=np.int64)
    pin_cell = np.array([c for e in edges for c in e], dtype=np.int32)
    return num_cells, net_ptr, pin_cell


def path_edges(cells):
    return [(cells[i], cells[i + 1]) for i in range(len(cells) - 1)]


def grid_edges(a, b, base=0):
    e = []
    for r in range(a):
        for c in range(b):
            i = base + r * b + c
            if c + 1 < b:
                e.append((i, i + 1))
            if r + 1 < a:
                e.append((i, i + b))
    return e


def mu(k, n):  # eigenvalue k of the unit path Laplacian on n cells
    return 2.0 - 2.0 * math.cos(k * math.pi / n)


def vec(k, n):  # its eigenvector, unit norm
    v = np.cos(k * math.pi * (2 * np.arange(n) + 1) / (2 * n))
    return v / np.linalg.norm(v)


def run(num_cells, edges):
    n, net_ptr, pin_cell = netlist(num_cells, edges)
    g = oracle.build_graph(n, net_ptr, pin_cell)
    return oracle.eigen_placement(g, oracle.degrees(g))


def same_line(u, v, tol):
    """u = +-v for unit vectors."""
    assert abs(abs(float(np.dot(u, v))) - 1.0) <= tol, float(np.dot(u, v))


@pytest.mark.parametrize("n", [3, 7, 50, 300])
def test_path_closed_form(n):
    u, lam, mask = run(n, path_edges(list(range(n))))
    assert mask.all()
    assert lam[0] == pytest.approx(mu(1, n), rel=1e-10, abs=1e-13)
    assert lam[1] == pytest.approx(mu(2, n), rel=1e-10, abs=1e-13)
    same_line(u[:, 0], vec(1, n), 1e-10)
    same_line(u[:, 1], vec(2, n), 1e-10)


@pytest.mark.parametrize("a,b", [(6, 9), (40, 60)])  # 2,400 cells takes the shift-invert branch
def test_grid_closed_form(a, b):
    """Rows r, columns c, cell r * b + c.  With b > a: lambda_2 = mu_1(b)
    (cosine along the rows), lambda_3 = min(mu_2(b), mu_1(a))."""
    u, lam, _ = run(a * b, grid_edges(a, b))
    assert lam[0] == pytest.approx(mu(1, b), rel=1e-9)
    same_line(u[:, 0], np.kron(np.ones(a) / math.sqrt(a), vec(1, b)), 1e-9)
    third = sorted([(mu(2, b), np.kron(np.ones(a) / math.sqrt(a), vec(2, b))),
                    (mu(1, a), np.kron(vec(1, a), np.ones(b) / math.sqrt(b)))], key=lambda t: t[0])[0]
    assert lam[1] == pytest.approx(third[0], rel=1e-9)
    same_line(u[:, 1], third[1], 1e-9)


def test_largest_component_and_zeros_elsewhere():
    """Paths on cells 0..11 and 20..49, cells 12..19 and 50..54 without nets:
    the 30-cell path is the component; its u_2, u_3 are the path's, every
    other cell gets 0."""
    edges = path_edges(list(range(12))) + path_edges(list(range(20, 50)))
    u, lam, mask = run(55, edges)
    assert np.array_equal(np.flatnonzero(mask), np.arange(20, 50))
    assert lam == pytest.approx((mu(1, 30), mu(2, 30)), rel=1e-10)
    same_line(u[20:50, 0], vec(1, 30), 1e-10)
    same_line(u[20:50, 1], vec(2, 30), 1e-10)
    assert not u[:20].any() and not u[50:].any()


def test_component_tie_goes_to_the_smallest_cell_id():
    edges = path_edges(list(range(20, 35))) + path_edges(list(range(2, 17)))
    _, _, mask = run(40, edges)
    assert np.array_equal(np.flatnonzero(mask), np.arange(2, 17))


def test_cycle_double_eigenvalue_subspace():
    """C_n: lambda_2 = lambda_3 = 2 - 2cos(2 pi / n); span{u_2, u_3} is the span
    of cos and sin of 2 pi i / n (equal orthogonal projectors)."""
    n = 24
    u, lam, _ = run(n, path_edges(list(range(n))) + [(n - 1, 0)])
    want = 2.0 - 2.0 * math.cos(2 * math.pi / n)
    assert lam == pytest.approx((want, want), rel=1e-10)
    t = 2 * math.pi * np.arange(n) / n
    basis = np.stack([np.cos(t), np.sin(t)], axis=1) / math.sqrt(n / 2)
    np.testing.assert_allclose(u @ u.T, basis @ basis.T, atol=1e-10)


def test_single_net_clique():
    """One 5-pin net: w = 2/5, L = w (5 I - J), eigenvalues 0 and 5w = 2
    (four times): lambda_2 = lambda_3 = 2, u orthonormal and orthogonal to 1."""
    g = oracle.build_graph(5, np.array([0, 5], dtype=np.int64), np.arange(5, dtype=np.int32))
    u, lam, _ = oracle.eigen_placement(g, oracle.degrees(g))
    assert lam == pytest.approx((2.0, 2.0), rel=1e-12)
    np.testing.assert_allclose(u.T @ u, np.eye(2), atol=1e-12)
    np.testing.assert_allclose(u.sum(axis=0), 0.0, atol=1e-12)


def test_too_small_component_rejected():
    with pytest.raises(ValueError):
        run(4, [(0, 1)])
