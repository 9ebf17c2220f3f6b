"""Pins for the oracle's cycles and adaptive drivers (Alg. 2, Alg. 5, Alg. 6)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _exact(g, b):
    """Solution of A x = b with x orthogonal to 1 (dense, pinned last unknown)."""
    A = g.to_scipy().toarray()
    A[-1, :] = 0; A[:, -1] = 0; A[-1, -1] = 1
    bb = b.copy(); bb[-1] = 0
    x = np.linalg.solve(A, bb)
    return x - x.mean()


@pytest.mark.parametrize("gamma", ["v", "w"])
@pytest.mark.parametrize("mode", [O.P1_E_SCALED, O.P1_BOOLEAN])
def test_cycle_is_symmetric(gamma, mode):
    # forward pre-smoothing and backward post-smoothing make the cycle a
    # symmetric operator: <V r1, r2> = <r1, V r2>
    g = I.grid3d(9, 8, 7, "checkerboard", block=3, xscale=100.0)
    h = O.Hierarchy(g, O.start_vector(g), O.default_params(p1_mode=mode, n_min=30))
    rng = np.random.default_rng(0)
    r1, r2 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    f = h.vcycle if gamma == "v" else h.wcycle
    a, b = f(r1) @ r2, r1 @ f(r2)
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_cycle_is_linear():
    g = I.workload("C1")
    h = O.Hierarchy(g, O.start_vector(g))
    rng = np.random.default_rng(1)
    r1, r2 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    lhs = h.vcycle(2.0 * r1 + r2)
    rhs = 2.0 * h.vcycle(r1) + h.vcycle(r2)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


@pytest.mark.parametrize("mk", [lambda: I.grid2d(12, 12, "loguniform", seed=3),
                                lambda: random_graph(150, 0.03, 4),
                                lambda: I.ring(128, 4)])
def test_two_level_exact_when_error_spans_P1(mk):
    # Section 3.3 and Alg. 6: with e = the exact error, e is in Range(P_1), so
    # one coarse-grid correction with an exact coarse solve (no smoothing)
    # recovers the solution.
    g = mk()
    b = I.rhs_normal(g.n, 1)
    xs = _exact(g, b)
    x0 = np.random.default_rng(2).standard_normal(g.n); x0 -= x0.mean()
    err = xs - x0
    e = err / np.linalg.norm(err)
    p = O.default_params(max_levels=2, n_min=4, nu_pre=0, nu_post=0)
    h = O.Hierarchy(g, e, p)
    assert h.nlevels == 2
    x1 = x0 + h.vcycle(b - g.to_scipy() @ x0)
    x1 -= x1.mean()
    assert np.linalg.norm(x1 - xs) <= 1e-9 * np.linalg.norm(xs)


def test_smooth_error_pcg_reduces_energy_error():
    # Alg. 2: a few preconditioned CG steps on A e = r approximate the error
    g = I.grid2d(24, 24, "loguniform", seed=7)
    A = g.to_scipy()
    b = I.rhs_normal(g.n, 2)
    xs = _exact(g, b)
    x = np.zeros(g.n)
    r = b - A @ x
    h = O.Hierarchy(g, O.start_vector(g))
    e = O.smooth_error(g, r, [h])
    d0, d1 = xs - x, xs - x - e
    assert d1 @ (A @ d1) < 0.05 * (d0 @ (A @ d0))
    # composite branch (re > numW) on three hierarchies
    hs = [h, O.Hierarchy(g, O.start_vector(g, O.default_params(seed=2))),
          O.Hierarchy(g, O.start_vector(g, O.default_params(seed=3)))]
    e3 = O.smooth_error(g, r, hs)
    d3 = xs - x - e3
    assert d3 @ (A @ d3) < 0.05 * (d0 @ (A @ d0))


@pytest.mark.parametrize("name", ["C1", "C2-small", "C5-small", "C4-small", "C3-small"])
def test_solve_reaches_tolerance(name):
    g = I.workload(name)
    b = I.rhs_normal(g.n, 11)
    x, st, hist = O.solve(g, b)
    A = g.to_scipy()
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert st["status"] == "OK" and rel <= 1e-8, (st, rel)
    assert abs(x.mean()) < 1e-12 * np.abs(x).max()
    assert len(hist) == st["iters"] + 1 and hist[-1] <= 1e-8
    if g.n <= 5000:
        xs = _exact(g, b)
        kappa_bound = 1e-8 * np.linalg.cond(A.toarray() + np.ones((g.n, g.n)) / g.n)
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa_bound


def test_solve_low_frequency_rhs_and_variants():
    g = I.grid2d(32, 32)
    for b in (I.rhs_lowfreq(g.n), I.rhs_normal(g.n, 5)):
        for thr in (1e-6, 0.4):
            for mode in (O.P1_E_SCALED, O.P1_BOOLEAN):
                x, st, _ = O.solve(g, b, params=O.default_params(threshold=thr, p1_mode=mode))
                assert st["status"] == "OK", (thr, mode, st)


def test_solve_zero_rhs_alg6():
    g = I.grid2d(32, 32)
    x0 = np.random.default_rng(4).standard_normal(g.n)
    x, st, hist = O.solve_zero_rhs(g, x0)
    assert st["status"] == "OK"
    assert np.linalg.norm(g.to_scipy() @ x) <= 1e-8 * np.linalg.norm(g.to_scipy() @ (x0 - x0.mean()))


def test_paper_tables_context_grid_oc_and_iterations():
    # Tables 1-3 report OC between 2.07 and 2.17 on unweighted 2D grids and
    # 13-21 iterations for Alg. 5(2). Our smoother order and start vector differ
    # (iteration counts are context, not a pin); OC is the same quantity.
    with open(os.path.join(GOLDEN, "paper_tables_grid.json")) as f:
        ref = json.load(f)
    g = I.grid2d(64, 64)
    for b, key in ((I.rhs_lowfreq(g.n), "table1_lf"), (I.rhs_normal(g.n, 0), "table2_zs")):
        x, st, _ = O.solve(g, b)
        row = ref[key]["4096"]
        assert st["status"] == "OK"
        assert abs(st["oc_mean"] - row["alg5_2_oc"]) < 0.15
        assert st["iters"] <= 2 * row["alg5_2_iter"]


def test_paper_tables_context_zero_rhs_alg6():
    # Tables 3 and 6: Alg. 6 (b = 0) takes 16 iterations and 4 hierarchies on
    # grids, 15 and 4 on rings, at every size. Our start vector and smoother
    # order differ, so the counts are context (a band, not a pin); OC is the
    # same quantity.
    with open(os.path.join(GOLDEN, "paper_tables_grid.json")) as f:
        grid = json.load(f)["table3_zero"]["4096"]
    with open(os.path.join(GOLDEN, "paper_tables_ring.json")) as f:
        ring = json.load(f)["table6_zero"]["1024"]
    for g, row in ((I.grid2d(64, 64), grid), (I.ring(1024, 4), ring)):
        x0 = np.random.default_rng(4).standard_normal(g.n)
        x, st, _ = O.solve_zero_rhs(g, x0)
        assert st["status"] == "OK"
        assert row["alg6_iter"] / 2 <= st["iters"] <= 2 * row["alg6_iter"]
        assert st["resetups"] + 1 <= 2 * row["alg6_re"]
        assert abs(st["oc_mean"] - row["alg6_oc"]) < 0.15


def test_paper_tables_context_ring_alg5():
    # Tables 4 and 5 (rings, n = 2^10): Alg. 5(1) 7-8 iterations, Alg. 5(2)
    # 14 iterations with 6 hierarchies, OC 1.57-1.58
    with open(os.path.join(GOLDEN, "paper_tables_ring.json")) as f:
        ref = json.load(f)
    g = I.ring(1024, 4)
    for b, key in ((I.rhs_lowfreq(g.n), "table4_lf"), (I.rhs_normal(g.n, 0), "table5_zs")):
        row = ref[key]["1024"]
        for thr, it, oc in ((1e-6, "alg5_1_iter", "alg5_1_oc"), (0.4, "alg5_2_iter", "alg5_2_oc")):
            x, st, _ = O.solve(g, b, params=O.default_params(threshold=thr))
            assert st["status"] == "OK"
            assert st["iters"] <= 2 * row[it]
            assert abs(st["oc_mean"] - row[oc]) < 0.15


@pytest.mark.parametrize("name", ["C1", "C5-small", "C4-small"])
def test_fcg_outer_iteration(name):
    # flexible CG preconditioned by the adaptive V-cycle (not in the paper):
    # reaches the tolerance (checked with scipy), keeps x orthogonal to 1, and
    # its first step equals the stationary one scaled by the exact line search
    g = I.workload(name)
    A = g.to_scipy()
    b = I.rhs_normal(g.n, 11)
    x, st, hist = O.solve(g, b, params=O.default_params(outer=1))
    assert st["status"] == "OK"
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    assert abs(x.mean()) < 1e-12 * np.abs(x).max()
    # one step: x1 = alpha z, z = V b, alpha = b.z / z.Az (exact line search)
    x1, s1, h1 = O.solve(g, b, params=O.default_params(outer=1, max_iter=1, threshold=10.0))
    e = O.start_vector(g)
    z = O.Hierarchy(g, e).vcycle(b)
    alpha = (b @ z) / (z @ (A @ z))
    ref = alpha * z
    ref -= ref.mean()
    assert np.linalg.norm(x1 - ref) <= 1e-10 * np.linalg.norm(ref)
