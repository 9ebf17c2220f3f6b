"""The seeded input recipes against what the configurations state: sizes,
weight laws, block structure, degree laws, connectivity, Laplacian form, and
right-hand sides orthogonal to the constants. The generators feed both the
oracle and the CUDA path, so a drift here would move both sides at once."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components
from scipy.stats import kstest

from paper_1806_07028_gb300 import inputs as I


def _offdiag_weights(g):
    A = g.to_scipy().tocoo()
    m = A.row != A.col
    return A.row[m], A.col[m], -A.data[m]


def _check_laplacian(g):
    A = g.to_scipy().tocsr()
    assert (A - A.T).count_nonzero() == 0 or abs(A - A.T).max() == 0.0
    d = A.diagonal()
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.all(np.abs(rs) <= 1e-12 * np.maximum(d, 1e-300))
    _, _, w = _offdiag_weights(g)
    assert np.all(w > 0)
    assert connected_components(A, directed=False)[0] == 1


def test_c1_grid_loguniform_weights():
    # 64 x 64 grid, 4-neighbour edges, weights log-uniform in [1e-3, 1]
    g = I.workload("C1")
    assert g.n == 4096 and g.nnz == 4096 + 2 * (2 * 64 * 63)
    _check_laplacian(g)
    i, j, w = _offdiag_weights(g)
    assert set(np.unique(np.abs(i - j))) == {1, 64}
    assert w.min() >= 1e-3 and w.max() <= 1.0
    lw = np.log10(w[i < j])
    assert kstest(lw, "uniform", args=(-3.0, 3.0)).pvalue > 1e-3


@pytest.fixture(scope="module")
def c2():
    return I.workload("C2")


def test_c2_sizes(c2):
    n = 128 ** 3
    assert c2.n == n and c2.nnz == n + 2 * 3 * 127 * 128 * 128 == 14_581_760


def test_c2_checkerboard_and_anisotropy(c2):
    # vertex coefficient 1 or 1e-4 on 8^3 checkerboard blocks; edge weight the
    # harmonic mean of its ends; x-edges (ids differ by 1) times 100
    i, j, w = _offdiag_weights(c2)
    up = i < j
    i, j, w = i[up], j[up], w[up]
    hm = 2e-4 / (1 + 1e-4)
    base = np.array([1.0, 1e-4, hm])
    xe = (j - i) == 1
    for sel, scale in ((xe, 100.0), (~xe, 1.0)):
        got = np.unique(w[sel] / scale)
        assert np.all(np.min(np.abs(got[:, None] - base[None, :]) / base[None, :], axis=1) < 1e-14)
    assert xe.sum() == 127 * 128 * 128
    # the coefficient of a vertex follows the parity of its block
    nx = 128
    v = i[~xe]
    x, y, z = v % nx, (v // nx) % nx, v // (nx * nx)
    u = j[~xe]
    xu, yu, zu = u % nx, (u // nx) % nx, u // (nx * nx)
    par_v = (x // 8 + y // 8 + z // 8) % 2
    par_u = (xu // 8 + yu // 8 + zu // 8) % 2
    same = par_v == par_u
    expect = np.where(par_v[same] == 0, 1.0, 1e-4)
    assert np.allclose(w[~xe][same], expect, rtol=1e-15, atol=0)   # 2ab/(a+b) at a = b
    assert np.allclose(w[~xe][~same], hm, rtol=1e-15, atol=0)


def test_c3_chung_lu_small():
    # Chung-Lu, degree exponent 2.1, mean degree 10, largest component,
    # weights uniform in (0, 1]
    g = I.workload("C3-small")
    _check_laplacian(g)
    A = g.to_scipy().tocsr()
    deg = np.diff(A.indptr) - 1
    assert 8.0 <= deg.mean() <= 10.5
    # discrete power-law tail, maximum-likelihood exponent (continuous
    # approximation with the half-integer shift) over degrees >= 10
    d = deg[deg >= 10]
    alpha = 1.0 + d.size / np.log(d / 9.5).sum()
    assert 1.9 <= alpha <= 2.4, alpha
    _, _, w = _offdiag_weights(g)
    assert w.min() > 0.0 and w.max() <= 1.0
    assert kstest(w, "uniform", args=(0.0, 1.0)).pvalue > 1e-3


def test_c4_random_geometric_small():
    # unit square, radius r with n pi r^2 = 12, weights 1/distance; the mean
    # degree of a unit-square RGG is (n - 1)(pi r^2 - 8 r^3 / 3 + r^4 / 2)
    n = 20_000
    g = I.workload("C4-small")
    _check_laplacian(g)
    r = np.sqrt(12.0 / (np.pi * n))
    expect = (n - 1) * (np.pi * r * r - 8.0 * r ** 3 / 3.0 + r ** 4 / 2.0)
    deg = np.diff(g.to_scipy().tocsr().indptr) - 1
    assert g.n == n
    assert abs(deg.mean() - expect) <= 0.02 * expect
    _, _, w = _offdiag_weights(g)
    assert w.min() * r >= 1.0 - 1e-12   # every edge is at most r long


def test_c5_sizes_and_block_coefficients():
    n = 256 ** 3
    E = 3 * 255 * 256 * 256
    assert E == 50_135_040 and n + 2 * E == 117_047_296
    g = I.workload("C5-small")   # 32^3 with 16^3 blocks: 8 block coefficients
    _check_laplacian(g)
    i, j, w = _offdiag_weights(g)
    nx = 32
    bid = lambda v: (v % nx) // 16 + 2 * (((v // nx) % nx) // 16) + 4 * ((v // (nx * nx)) // 16)
    same = bid(i) == bid(j)
    coef = {}
    for b, ww in zip(bid(i[same]), w[same]):
        coef.setdefault(int(b), set()).add(float(ww))
    assert sorted(coef) == list(range(8))
    assert all(len(s) == 1 for s in coef.values())
    c = np.array([next(iter(coef[b])) for b in range(8)])
    assert np.all((c >= 1e-6) & (c <= 1.0))


def test_right_hand_sides():
    b = I.rhs_normal(100_000, 7)
    assert abs(b.sum()) <= 1e-9 * np.linalg.norm(b)
    assert abs(b.std() - 1.0) < 0.02
    lf = I.rhs_lowfreq(1000)
    assert lf.sum() == 0.0 and lf[-1] == -999.0 and np.all(lf[:-1] == 1.0)


def test_workloads_are_reproducible():
    a, b = I.workload("C3-small"), I.workload("C3-small")
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val)
    c = I.workload("C3-small", seed=1)
    assert c.n != a.n or not np.array_equal(c.val[: min(c.nnz, a.nnz)], a.val[: min(c.nnz, a.nnz)])
    assert sp.issparse(a.to_scipy())
