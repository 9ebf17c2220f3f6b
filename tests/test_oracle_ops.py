"""Pins for the oracle's level operators: residual, colouring, smoother."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph

GRAPHS = [
    lambda: I.workload("C1"),
    lambda: I.grid3d(7, 6, 5, "checkerboard", block=2, xscale=100.0),
    lambda: random_graph(60, 0.08, 3),
    lambda: I.ring(50, 4),
]


@pytest.mark.parametrize("mk", GRAPHS)
def test_residual_matches_scipy(mk):
    g = mk()
    rng = np.random.default_rng(0)
    x, b = rng.standard_normal(g.n), rng.standard_normal(g.n)
    r = O.residual(g, x, b)
    ref = b - g.to_scipy() @ x
    assert np.allclose(r, ref, rtol=0, atol=1e-12 * (np.abs(g.val).max() * np.abs(x).max() * 8 + 1))


def test_laplacian_rows_sum_to_zero():
    # Section 2.2: A 1 = 0, off-diagonals <= 0, symmetric
    for mk in GRAPHS:
        A = mk().to_scipy()
        assert abs(A @ np.ones(A.shape[0])).max() < 1e-12 * abs(A).max() * 8
        off = A - sp.diags(A.diagonal())
        assert off.data.max() <= 0
        assert abs(A - A.T).max() == 0


def _greedy_colour_by_priority(g, seed):
    """Sequential greedy colouring visiting vertices in decreasing (priority, id)."""
    pri = [(O.splitmix64(seed ^ i), i) for i in range(g.n)]
    order = sorted(range(g.n), key=lambda i: pri[i], reverse=True)
    col = np.full(g.n, -1)
    for v in order:
        used = {col[u] for u in g.col[g.rowptr[v]:g.rowptr[v + 1]] if u != v and col[u] >= 0}
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return col


@pytest.mark.parametrize("mk", GRAPHS)
def test_colour_equals_priority_greedy(mk):
    # Jones-Plassmann rounds colour a vertex exactly when every higher-priority
    # neighbour is coloured, so the result equals the sequential greedy colouring
    # in decreasing priority order.
    g = mk()
    col, nc, rounds = O.colour(g, seed=77)
    assert np.array_equal(col, _greedy_colour_by_priority(g, 77))
    assert nc == col.max() + 1
    A = g.to_scipy().tocoo()
    m = A.row != A.col
    assert np.all(col[A.row[m]] != col[A.col[m]])


@pytest.mark.parametrize("mk", GRAPHS)
@pytest.mark.parametrize("forward", [True, False])
def test_mcgs_equals_triangular_solve_in_colour_order(mk, forward):
    # A forward GS sweep in a row order pi solves (D + L_pi) x_new = b - U_pi x_old
    # for the matrix permuted by pi; rows of one colour are independent so any
    # order inside a colour gives the same result.
    g = mk()
    col, nc, _ = O.colour(g, seed=5)
    rng = np.random.default_rng(1)
    b, x0 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    x = O.mcgs_sweep(g, col, nc, b, x0, forward=forward)
    key = col if forward else (nc - 1 - col)
    perm = np.lexsort((np.arange(g.n), key))
    A = g.to_scipy()[perm][:, perm].tocsr()
    lower = sp.tril(A, format="csr")
    upper = sp.triu(A, k=1, format="csr")
    xp = spla.spsolve_triangular(lower, b[perm] - upper @ x0[perm], lower=True)
    ref = np.empty(g.n); ref[perm] = xp
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # and it is the same as a plain GS sweep in that order
    assert np.allclose(O.gs_perm_sweep(g, perm, b, x0), x, rtol=0, atol=0)


@pytest.mark.parametrize("mk", GRAPHS)
def test_l1_jacobi_sweep(mk):
    # x_new = x + D^{-1} (b - A x) with D the diagonal of row l1 norms; the
    # l1 smoother never increases the energy norm of the error for SPD A
    # (2D - A is positive definite)
    g = mk()
    A = g.to_scipy()
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(g.n); xs -= xs.mean()
    b = A @ xs
    x0 = rng.standard_normal(g.n)
    x1 = O.l1jac_sweep(g, b, x0)
    d = np.asarray(abs(A).sum(axis=1)).ravel()
    assert np.allclose(x1, x0 + (b - A @ x0) / d, rtol=1e-13, atol=1e-13 * np.abs(x1).max())
    e0, e1 = xs - x0, xs - x1
    assert e1 @ (A @ e1) < e0 @ (A @ e0)


def test_smoother_colouring_rule():
    # connected bipartite graphs (grids): two colours, the parity of the
    # breadth-first distance from vertex 0, so every edge joins both colours
    import scipy.sparse.csgraph as csg
    for g in (I.grid2d(9, 7), I.grid3d(5, 4, 3, "unit"), I.workload("C2-small")):
        col, nc, levels = O.colour_smoother(g)
        A = g.to_scipy().tocoo()
        off = A.row != A.col
        d = csg.shortest_path(g.to_scipy().astype(bool).astype(float), unweighted=True, indices=0)
        assert nc == 2 and col[0] == 0
        assert np.array_equal(col, d.astype(np.int64) % 2)
        assert np.all(col[A.row[off]] != col[A.col[off]])
        assert levels == int(d.max()) + 1
    # an odd cycle (rings with k = 4 have triangles) or a disconnected graph:
    # the Jones-Plassmann colouring
    for g in (I.ring(40, 4), I.workload("C4-small"),
              I.laplacian_from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], [1.0] * 4)):
        col, nc, _ = O.colour_smoother(g, seed=77)
        ref, ncr, _ = O.colour(g, seed=77)
        assert nc == ncr and np.array_equal(col, ref)
