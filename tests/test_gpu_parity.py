"""GPU path vs the CPU oracle, through the C ABI.

Integer and setup results (random numbers, colours, reweighted graph, path
cover, aggregates, coarse patterns and FP64 Galerkin values, P values) must
match bit for bit when both sides get the same smooth error. Floating-point
cycle results are compared with tolerances derived from the summation orders.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1806_07028_gb300.build import build
    build()
    import paper_1806_07028_gb300 as pkg
    return pkg


def _graphs():
    return {
        "C1": I.workload("C1"),
        "C2-small": I.workload("C2-small"),
        "C5-small": I.workload("C5-small"),
        "er": random_graph(3000, 0.002, 7),
        "ring": I.ring(2000, 4),
        "C4-small": I.workload("C4-small"),
    }


GRAPHS = _graphs()
NAMES = list(GRAPHS)


def _t(a, P, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0", dtype=dtype)


def test_uniform_bit_exact(P):
    for seed, n in ((0, 1), (7, 1001), (2**40 + 3, 123457)):
        g = P.uniform(seed, n).cpu().numpy()
        assert np.array_equal(g.view(np.uint64), O.uniform_pm1(seed, n).view(np.uint64))


@pytest.mark.parametrize("name", NAMES)
def test_colour_bit_exact(P, name):
    import torch
    g = GRAPHS[name]
    col, nc = P.colour(_t(g.rowptr, P, torch.int32), _t(g.col, P, torch.int32), 99)
    ref, ncr, _ = O.colour(g, seed=99)
    assert nc == ncr and np.array_equal(col.cpu().numpy(), ref)


@pytest.mark.parametrize("name", NAMES)
def test_residual_and_norm(P, name):
    import torch
    g = GRAPHS[name]
    rng = np.random.default_rng(3)
    x, b = rng.standard_normal(g.n), rng.standard_normal(g.n)
    r, nrm = P.residual(_t(g.rowptr, P, torch.int32), _t(g.col, P, torch.int32),
                        _t(g.val, P), _t(x, P), _t(b, P))
    ref = O.residual(g, x, b)
    rowabs = np.abs(g.to_scipy()) @ np.abs(x) + np.abs(b)
    assert np.all(np.abs(r.cpu().numpy() - ref) <= 32 * EPS * rowabs)
    assert abs(nrm.item() - ref @ ref) <= 1e-12 * (ref @ ref)
    # FP32 variant against the FP64 oracle: float rounding only
    r32 = P.residual_f32(_t(g.rowptr, P, torch.int32), _t(g.col, P, torch.int32),
                         _t(g.val, P, torch.float32), _t(x, P, torch.float32), _t(b, P, torch.float32))
    assert np.all(np.abs(r32.cpu().numpy() - ref) <= 64 * 2.0**-24 * rowabs)


def _compare_hierarchy(P, g, e, mode, precision=0):
    params = P.default_params(keep_setup=1, p1_mode=mode, precision=precision, n_min=64)
    s = P.Solver(g, params=params, e0=e)
    h = O.Hierarchy(g, e, O.default_params(p1_mode=mode, n_min=64))
    assert s.num_levels(0) == h.nlevels
    cp, cc, cw = s.reweighted(0, 0)
    rp, rc, rw = h.candidates()
    assert np.array_equal(cp, rp) and np.array_equal(cc, rc)
    assert np.array_equal(cw.view(np.uint64), rw.view(np.uint64))
    for lev in range(h.nlevels):
        G, R = s.level(0, lev, cover=True), h.level(lev)
        for k in ("n", "nnz", "nc", "ncolour", "leftover_rounds"):
            assert G[k] == R[k], (lev, k)
        if lev == 0:
            assert G["cover_rounds"] == R["cover_rounds"]
        assert np.array_equal(G["nbr0"], R["nbr0"]) and np.array_equal(G["nbr1"], R["nbr1"]), lev
        assert np.array_equal(G["rowptr"], R["rowptr"]) and np.array_equal(G["col"], R["col"]), lev
        assert np.array_equal(G["val"].view(np.uint64), R["val"].view(np.uint64)), lev
        if R["agg"] is not None:
            assert np.array_equal(G["agg"], R["agg"]), lev
        if R["pval"] is not None:
            assert np.array_equal(G["pval"].view(np.uint64), R["pval"].view(np.uint64))
        if lev + 1 < h.nlevels and R["ncolour"] > 0:
            assert np.array_equal(G["colour"], R["colour"]), lev
    assert s.sizes(0, 0)["pinned"] == h.sizes(0)["pinned"]
    return s, h


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("mode", [0, 1])
def test_setup_bit_exact_given_same_error(P, name, mode):
    g = GRAPHS[name]
    e = O.start_vector(g)          # same smooth error fed to both sides
    s, h = _compare_hierarchy(P, g, e, mode)
    s.close()


def test_setup_bit_exact_with_ties(P):
    # quantised error: many equal |e_i - e_j|, decided by the id tie-break
    g = I.grid2d(96, 80)
    e = np.round(np.random.default_rng(1).standard_normal(g.n), 1)
    _compare_hierarchy(P, g, e, 0)[0].close()
    _compare_hierarchy(P, g, np.zeros(g.n), 1)[0].close()


def test_setup_bit_exact_hub_rows(P):
    # scale-free graph (Chung-Lu, exponent 2.1, hubs of degree ~600): 1,805
    # rows of the A^2 product have more than 256 contributions and 227 more
    # than 2,048 (up to 15,792), so the block (shared memory) and global
    # row products, the long-row split and the per-block proposal ordering
    # all run, on the fine level and in the coarse Galerkin products
    g = I.chung_lu(3000, 2.1, 10.0, seed=1)
    e = O.start_vector(g)
    for mode in (0, 1):
        _compare_hierarchy(P, g, e, mode)[0].close()


@pytest.mark.parametrize("name", ["C1", "C2-small", "er"])
@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_matches_oracle(P, name, gamma):
    g = GRAPHS[name]
    e = O.start_vector(g)
    s, h = _compare_hierarchy(P, g, e, 0)
    r = I.rhs_normal(g.n, 5)
    c = s.cycle(r, hist=0, gamma=gamma).cpu().numpy()
    ref = h.vcycle(r) if gamma == 1 else h.wcycle(r)
    assert np.linalg.norm(c - ref) <= 1e-9 * np.linalg.norm(ref)
    s.close()
    # FP32 cycle inside FP64 refinement: same hierarchy, float arithmetic
    s32, _ = _compare_hierarchy(P, g, e, 0, precision=1)
    c32 = s32.cycle(r, hist=0, gamma=gamma).cpu().numpy()
    assert np.linalg.norm(c32 - ref) <= 2e-4 * np.linalg.norm(ref)
    s32.close()


def test_start_vector_and_smooth_error_match_oracle(P):
    g = GRAPHS["C2-small"]
    s = P.Solver(g)
    e_gpu = s.start_vector().cpu().numpy()
    e_orc = O.start_vector(g)
    assert np.linalg.norm(e_gpu - e_orc) <= 1e-10
    # Alg. 2 on the same hierarchies (W-cycle branch, then composite branch)
    e0 = e_orc
    s = P.Solver(g, e0=e0)
    hs = [O.Hierarchy(g, e0)]
    r = I.rhs_normal(g.n, 2)
    for k in range(3):
        eg = s.smooth_error(r).cpu().numpy()
        eo = O.smooth_error(g, r, hs)
        assert np.linalg.norm(eg - eo) <= 1e-7 * np.linalg.norm(eo), k
        ek = O.start_vector(g, O.default_params(seed=100 + k))
        s.adapt(ek)
        hs.append(O.Hierarchy(g, ek))


@pytest.mark.parametrize("name", NAMES + ["C3-small"])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_reaches_tolerance(P, name, precision):
    g = GRAPHS.get(name) or I.workload(name)
    b = I.rhs_normal(g.n, 11)
    s = P.Solver(g, params=P.default_params(precision=precision))
    x, st = s.solve(b)
    x = x.cpu().numpy()
    rel = np.linalg.norm(b - g.to_scipy() @ x) / np.linalg.norm(b)
    assert st["status"] == "OK" and rel <= 1e-8, (st, rel)
    s.close()


# graphs on which the FP64 GPU solve follows the oracle's trajectory step for
# step: same iterations, same re-setup steps, same residual history (up to the
# rounding that Alg. 2's PCG feeds into later covers)
TRAJ = {"C1": GRAPHS["C1"], "C2-small": GRAPHS["C2-small"], "C5-small": GRAPHS["C5-small"],
        "er": GRAPHS["er"], "ring": GRAPHS["ring"], "grid64u": I.grid2d(64, 64)}


@pytest.mark.parametrize("name", list(TRAJ))
def test_fp64_solve_follows_the_oracle(P, name):
    # same start vector on both sides, so the first hierarchy is the same bits
    g = TRAJ[name]
    b = I.rhs_normal(g.n, 11)
    e0 = O.start_vector(g)
    xo, so, ho = O.solve(g, b, e0=e0)
    s = P.Solver(g, params=P.default_params(precision=0), e0=e0)
    x, st = s.solve(b)
    s.close()
    x, hg = x.cpu().numpy(), st["res_hist"]
    assert so["status"] == "OK" and st["status"] == "OK"
    assert (st["iters"], st["resetups"], st["cycles"], st["wcycles"]) == \
        (so["iters"], so["resetups"], so["cycles"], so["wcycles"])
    assert st["rebuilt_after"] == so["rebuilt_after"]
    rel = np.abs(hg - ho) / ho
    # until the first re-setup both run the same hierarchy: rounding only
    k1 = so["rebuilt_after"][0] if so["rebuilt_after"] else len(ho) - 1
    assert np.all(rel[: k1 + 1] <= 1e-9), rel[: k1 + 1]
    # later hierarchies come from Alg. 2 errors that differ by rounding; the
    # histories stay close and the solutions agree far below the tolerance
    assert np.all(rel <= 0.2), rel
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


def test_fp64_solve_where_trajectories_part(P):
    # C4-small (random geometric graph): the PCG error of a later re-setup
    # differs from the oracle's by rounding, which reorders nearly equal
    # reweighted edges, so later covers differ. Up to the first re-setup the
    # histories agree to rounding; both solves reach the same solution.
    g = GRAPHS["C4-small"]
    b = I.rhs_normal(g.n, 11)
    e0 = O.start_vector(g)
    xo, so, ho = O.solve(g, b, e0=e0)
    s = P.Solver(g, params=P.default_params(precision=0), e0=e0)
    x, st = s.solve(b)
    s.close()
    x, hg = x.cpu().numpy(), st["res_hist"]
    k1 = so["rebuilt_after"][0]
    assert st["rebuilt_after"][0] == k1
    assert np.all(np.abs(hg[: k1 + 1] - ho[: k1 + 1]) <= 1e-9 * ho[: k1 + 1])
    assert abs(st["iters"] - so["iters"]) <= 2 and abs(st["resetups"] - so["resetups"]) <= 2
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("name", list(TRAJ) + ["C4-small"])
def test_alg6_follows_the_oracle(P, name):
    g = TRAJ.get(name) or GRAPHS[name]
    x0 = np.random.default_rng(4).standard_normal(g.n)
    e0 = O.start_vector(g)
    xo, so, ho = O.solve_zero_rhs(g, x0, e0=e0)
    s = P.Solver(g, params=P.default_params(precision=0, threshold=0.5), e0=e0)
    x, st = s.solve_zero_rhs(x0)
    s.close()
    assert so["status"] == "OK" and st["status"] == "OK"
    assert (st["iters"], st["resetups"]) == (so["iters"], so["resetups"])
    hg = st["res_hist"]
    # the rebuilds of Alg. 6 use the iterate itself, so rounding stays small
    tol = 0.05 if name == "C4-small" else 1e-11
    assert np.all(np.abs(hg - ho) <= tol * ho), np.abs(hg - ho) / ho


@pytest.mark.parametrize("name", ["C1", "C2-small", "C4-small"])
def test_two_runs_are_bit_identical(P, name):
    # every reduction and every integer round has a fixed order: the same
    # inputs give the same bits, in either precision
    g = GRAPHS[name]
    b = I.rhs_normal(g.n, 2)
    for prec in (0, 1):
        out = []
        for _ in range(2):
            s = P.Solver(g, params=P.default_params(precision=prec, keep_setup=1))
            x, st = s.solve(b)
            lv = s.level(s.num_hierarchies - 1, 0, cover=True)
            out.append((x.cpu().numpy(), st, lv))
            s.close()
        (xa, sa, la), (xb, sb, lb) = out
        assert np.array_equal(xa.view(np.uint64), xb.view(np.uint64))
        assert sa["iters"] == sb["iters"] and sa["rebuilt_after"] == sb["rebuilt_after"]
        for k in ("agg", "nbr0", "nbr1", "col"):
            assert np.array_equal(la[k], lb[k]), k


def test_solve_host_e2e(P):
    g = GRAPHS["C1"]
    b = I.rhs_normal(g.n, 1)
    x, st = P.solve_host(g, b)
    assert st["status"] == "OK"
    assert np.linalg.norm(b - g.to_scipy() @ x) <= 1e-8 * np.linalg.norm(b)


def test_invalid_inputs_return_status(P):
    from paper_1806_07028_gb300 import native as N
    g = I.grid2d(8, 8)
    bad = I.Graph(g.rowptr, g.col, g.val.copy())
    bad.val[1] = +1.0                       # positive off-diagonal (also asymmetric)
    with pytest.raises(N.PCAMGError) as ei:
        P.Solver(bad)
    assert ei.value.status == N.ERR_NOT_LAPLACIAN
    bad = I.Graph(g.rowptr, g.col[::-1].copy(), g.val)   # unsorted columns
    with pytest.raises(N.PCAMGError) as ei:
        P.Solver(bad)
    assert ei.value.status == N.ERR_INVALID
    s = P.Solver(g)
    b = np.ones(g.n); b[3] = np.nan
    with pytest.raises(N.PCAMGError) as ei:
        s.solve(b)
    assert ei.value.status == N.ERR_INVALID
    # max_iter hit: NOT_CONVERGED with stats filled
    g2 = I.grid2d(48, 48)
    s2 = P.Solver(g2, params=P.default_params(max_iter=1, threshold=10.0))
    x, st = s2.solve(I.rhs_normal(g2.n, 0))
    assert st["status"] == "NOT_CONVERGED" and st["iters"] == 1
    # a path cover that needs more rounds than allowed: ROUND_CAP, no handle
    with pytest.raises(N.PCAMGError) as ei:
        P.Solver(g2, params=P.default_params(max_cover_rounds=1))
    assert ei.value.status == N.ERR_ROUND_CAP
    # coarsening forbidden (one level) above the dense limit: COARSE_TOO_BIG
    with pytest.raises(N.PCAMGError) as ei:
        P.Solver(g2, params=P.default_params(max_levels=1, dense_max=100))
    assert ei.value.status == N.ERR_COARSE_TOO_BIG
    # invalid parameters are refused before any work
    for kw in (dict(update_mode=7), dict(max_cover_rounds=-1), dict(tol=0.0)):
        with pytest.raises(N.PCAMGError) as ei:
            P.Solver(g2, params=P.default_params(**kw))
        assert ei.value.status == N.ERR_INVALID


def test_fp64_is_scale_equivariant_and_fp32_range_gives_diverged(P):
    # A scaled by 2^-200 stays exact in FP64 (every entry is still a normal
    # number) and every step of Alg. 5 is then scaled exactly: the same
    # iterations and re-setups, x scaled by 2^200. In FP32 every entry of that
    # matrix underflows to zero, the first cycle divides by a zero diagonal and
    # the residual is no longer finite: DIVERGED, returned with the statistics.
    g = GRAPHS["C1"]
    s = 2.0 ** -200
    gs = I.Graph(g.rowptr, g.col, g.val * s)
    b = I.rhs_normal(g.n, 3)
    x0, st0 = P.Solver(g, params=P.default_params(precision=0)).solve(b)
    x1, st1 = P.Solver(gs, params=P.default_params(precision=0)).solve(b)
    assert st0["status"] == "OK" and st1["status"] == "OK"
    assert (st1["iters"], st1["resetups"]) == (st0["iters"], st0["resetups"])
    x0h, x1h = x0.cpu().numpy(), x1.cpu().numpy() * s
    assert np.linalg.norm(x1h - x0h) <= 1e-10 * np.linalg.norm(x0h)
    s2 = P.Solver(gs, params=P.default_params(precision=1))
    x2, st2 = s2.solve(b, raise_on_error=False)
    assert st2["status"] == "DIVERGED" and st2["iters"] == 0
    assert not np.isfinite(st2["rel_res"])


@pytest.mark.parametrize("name", ["C1", "C2-small", "C4-small"])
@pytest.mark.parametrize("precision", [0, 1])
def test_coarse_tail_block_matches_per_level_kernels(P, name, precision):
    # the single-block coarse tail runs the same steps as the per-level kernels:
    # no tail, a partial tail and an all-levels tail give the same correction;
    # so does the tail applied as its dense operator (one visit from zero is a
    # linear map), for V- and W-cycles, on the first and on repeated visits
    g = GRAPHS[name]
    e = O.start_vector(g)
    h = O.Hierarchy(g, e)
    r = I.rhs_normal(g.n, 8)
    tol = 1e-9 if precision == 0 else 2e-4
    for gamma in (1, 2):
        ref = h.vcycle(r) if gamma == 1 else h.wcycle(r)
        for tail in (0, 2000, 10**9):
            for dense in ((0,) if tail == 0 else (0, 3)):
                s = P.Solver(g, params=P.default_params(precision=precision, tail_rows=tail,
                                                        tail_dense=dense), e0=e)
                for _ in range(2):   # the second call replays the captured graph
                    c = s.cycle(r, hist=0, gamma=gamma).cpu().numpy()
                    assert np.linalg.norm(c - ref) <= tol * np.linalg.norm(ref), (tail, dense, gamma)
                s.close()


# ---- MWM_setup (Section 2.1) ---------------------------------------------------
@pytest.mark.parametrize("name", NAMES)
def test_mwm_hierarchy_bit_exact(P, name):
    # heaviest-first matching, attachment, numbering, boolean Galerkin products
    # and colours: the same bits as the oracle's MWM_setup
    g = GRAPHS[name]
    s = P.Solver(g, params=P.default_params(start=3, n_min=64))
    h = O.Hierarchy(g, None, O.default_params(n_min=64))
    assert s.num_levels(0) == h.nlevels
    for lev in range(h.nlevels):
        G, R = s.level(0, lev), h.level(lev)
        for k in ("n", "nnz", "nc", "ncolour"):
            assert G[k] == R[k], (lev, k)
        if lev == 0:
            assert G["cover_rounds"] == R["cover_rounds"]
        assert np.array_equal(G["rowptr"], R["rowptr"]) and np.array_equal(G["col"], R["col"]), lev
        assert np.array_equal(G["val"].view(np.uint64), R["val"].view(np.uint64)), lev
        if R["agg"] is not None:
            assert np.array_equal(G["agg"], R["agg"]), lev
        assert G["pval"] is None
        if lev + 1 < h.nlevels and R["ncolour"] > 0:
            assert np.array_equal(G["colour"], R["colour"]), lev
    assert s.sizes(0, 0)["pinned"] == h.sizes(0)["pinned"] == 1
    s.close()


@pytest.mark.parametrize("name,nmin", [("grid64u", 2), ("ring", 64)])
def test_mwm_comparator_and_mwm_start_follow_the_oracle(P, name, nmin):
    # UA-AMG w/MWM (never re-set up) and Alg. 5(2) from the MWM hierarchy, FP64:
    # the same iterations and re-setup steps as the oracle
    g = TRAJ.get(name) or GRAPHS[name]
    b = I.rhs_lowfreq(g.n)
    for thr in (1e9, 0.4):
        xo, so, ho = O.solve(g, b, params=O.default_params(init_mwm=1, threshold=thr, n_min=nmin,
                                                           max_iter=2500))
        s = P.Solver(g, params=P.default_params(start=3, threshold=thr, n_min=nmin, max_iter=2500,
                                                precision=0))
        x, st = s.solve(b)
        s.close()
        assert so["status"] == "OK" and st["status"] == "OK"
        assert (st["iters"], st["resetups"]) == (so["iters"], so["resetups"]), (thr, st, so)
        assert st["rebuilt_after"] == so["rebuilt_after"]
        # the same hierarchy until the first re-setup: rounding only (it grows
        # slowly over the comparator's many iterations)
        k1 = min(so["rebuilt_after"][0] if so["rebuilt_after"] else len(ho) - 1, 10)
        hg = st["res_hist"]
        assert np.all(np.abs(hg[: k1 + 1] - ho[: k1 + 1]) <= 1e-9 * ho[: k1 + 1])
        assert np.all(np.abs(hg - ho) <= 1e-3 * ho)


# ---- flexible-CG outer iteration (not in the paper) ------------------------------
@pytest.mark.parametrize("name", ["C1", "C5-small", "er"])
def test_fcg_outer_follows_the_oracle(P, name):
    g = TRAJ.get(name) or GRAPHS[name]
    b = I.rhs_normal(g.n, 11)
    e0 = O.start_vector(g)
    xo, so, ho = O.solve(g, b, e0=e0, params=O.default_params(outer=1))
    for prec in (0, 1):
        s = P.Solver(g, params=P.default_params(precision=prec, outer=1), e0=e0)
        x, st = s.solve(b)
        s.close()
        x = x.cpu().numpy()
        rel = np.linalg.norm(b - g.to_scipy() @ x) / np.linalg.norm(b)
        assert st["status"] == "OK" and rel <= 1e-8, (st, rel)
        if prec == 0:
            assert (st["iters"], st["resetups"]) == (so["iters"], so["resetups"])
            assert st["rebuilt_after"] == so["rebuilt_after"]
            # CG's inner products differ in summation order: rounding compounds
            # through alpha and beta, so the histories agree to 1e-7 relative
            k1 = so["rebuilt_after"][0] if so["rebuilt_after"] else len(ho) - 1
            hg = st["res_hist"]
            assert np.all(np.abs(hg[: k1 + 1] - ho[: k1 + 1]) <= 1e-7 * ho[: k1 + 1])
            assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
