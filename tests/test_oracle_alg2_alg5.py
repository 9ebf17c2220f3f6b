"""Pins for the oracle's Alg. 2 preconditioner, its PCG iterate and the Alg. 5
re-setup trigger, each against something assembled independently of the oracle.

- The preconditioner (Alg. 2, Section 3.2): every hierarchy's cycle is
  assembled as an explicit matrix with numpy from the exported level matrices,
  aggregates, prolongation values and colours (textbook two-grid recursion:
  pre-smoother, coarse correction, post-smoother; dense coarsest solve), then
  composed into the W-cycle (Re <= numW) or the palindrome
  B_1 ... B_Re B_Re ... B_1 of V-cycles.
- The PCG iterate: with a fixed symmetric positive definite preconditioner Z,
  k steps of preconditioned CG from zero give the A-orthogonal projection of
  the solution onto the Krylov space span{Zr, (ZA)Zr, ...} (a closed form that
  does not use the CG recurrences).
- The Alg. 5 trigger: the printed order (the smooth error drives the rebuild
  only) gives Re = Iter - 1 when every step re-sets up (threshold ~ 0, the
  paper's Alg. 5(1)), never re-sets up above the largest possible factor, and
  the recorded rebuild steps follow from the residual history by the rule
  "mean factor since the last rebuild exceeds the threshold".
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ assembled cycles
def _dense(rowptr, col, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i, col[k]] += val[k]
    return A


def _levels(h, params):
    """Per level: dense A, dense P (n x nc), smoother kind and colours."""
    out = []
    for lev in range(h.nlevels):
        L = h.level(lev)
        n = L["n"]
        A = _dense(L["rowptr"], L["col"], L["val"], n)
        d = dict(A=A, n=n, colour=L["colour"])
        d["jac"] = lev >= 1 and n <= params.l1jac_rows
        if L["agg"] is not None:
            nc = int(L["agg"].max()) + 1
            P = np.zeros((n, nc))
            pv = L["pval"] if L["pval"] is not None else np.ones(n)
            P[np.arange(n), L["agg"]] = pv
            d["P"] = P
        d["pinned"] = L["pinned"]
        out.append(d)
    return out


def _smoother_matrices(d):
    """M_pre, M_post with x <- x + M^{-1}(b - A x) for one sweep.

    Multicolour Gauss-Seidel visits colour 0..C-1 (forward) or C-1..0
    (backward); rows of one colour are independent. A forward sweep is the
    lower-triangular solve in colour order: M[i, j] = a_ij when colour(j) <=
    colour(i), else 0 (within one colour only the diagonal is nonzero).
    l1-Jacobi: M = diag(sum_j |a_ij|)."""
    A = d["A"]
    if d["jac"]:
        M = np.diag(np.abs(A).sum(axis=1))
        return M, M
    c = d["colour"]
    lower = c[None, :] <= c[:, None]
    upper = c[None, :] >= c[:, None]
    return np.where(lower, A, 0.0), np.where(upper, A, 0.0)


def _coarse_inverse(d, boolean_chain):
    A = d["A"]
    m = d["n"]
    if boolean_chain:
        # constant null space kept exactly: the last unknown is pinned
        assert d["pinned"] == 1
        X = np.zeros((m, m))
        X[:-1, :-1] = np.linalg.inv(A[:-1, :-1])
        return X
    assert d["pinned"] == 0
    return np.linalg.inv(A)


def _cycle_matrix(levels, gamma, boolean_chain, nu_pre=1, nu_post=1):
    """The linear map r -> c of one cycle from a zero start, as a matrix."""
    def rec(l):
        d = levels[l]
        if l == len(levels) - 1:
            return _coarse_inverse(d, boolean_chain)
        A, P = d["A"], d["P"]
        n = d["n"]
        Mf, Mb = _smoother_matrices(d)
        I_n = np.eye(n)
        Bc1 = rec(l + 1)
        Ac = levels[l + 1]["A"]
        Bc = Bc1.copy()
        for _ in range(gamma - 1):      # further coarse visits from the current iterate
            Bc = Bc + Bc1 @ (np.eye(Ac.shape[0]) - Ac @ Bc)
        T = np.zeros((n, n))
        for _ in range(nu_pre):
            T = T + np.linalg.solve(Mf, I_n - A @ T)
        T = T + P @ Bc @ P.T @ (I_n - A @ T)
        for _ in range(nu_post):
            T = T + np.linalg.solve(Mb, I_n - A @ T)
        return T
    return rec(0)


def _small_graphs():
    return [("grid", I.grid2d(9, 7, "loguniform", seed=5)),
            ("er", random_graph(60, 0.06, 3))]


def _hist(g, params, k):
    hs = []
    for s in range(k):
        e = O.start_vector(g, O.default_params(seed=100 + s, relax_sweeps=2 + s))
        hs.append(O.Hierarchy(g, e, params))
    return hs


@pytest.mark.parametrize("gname,g", _small_graphs())
@pytest.mark.parametrize("p1", [O.P1_E_SCALED, O.P1_BOOLEAN])
@pytest.mark.parametrize("l1jac", [2147483647, 0])
def test_cycles_equal_assembled_matrices(gname, g, p1, l1jac):
    params = O.default_params(n_min=4, p1_mode=p1, l1jac_rows=l1jac)
    h = O.Hierarchy(g, O.start_vector(g), params)
    assert h.nlevels >= 3
    levels = _levels(h, params)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(g.n)
    for gamma, f in ((1, h.vcycle), (2, h.wcycle)):
        B = _cycle_matrix(levels, gamma, p1 == O.P1_BOOLEAN)
        c = f(r)
        assert np.linalg.norm(c - B @ r) <= 1e-12 * np.linalg.norm(B @ r), (gamma,)


@pytest.mark.parametrize("gname,g", _small_graphs())
@pytest.mark.parametrize("p1", [O.P1_E_SCALED, O.P1_BOOLEAN])
def test_precond_is_w_cycle_then_palindrome(gname, g, p1):
    # Alg. 2: W-cycle on the newest hierarchy while Re <= numW, else the
    # symmetric composite z = sum of B_j applied in the order j = 1..Re, Re..1
    params = O.default_params(n_min=4, p1_mode=p1)
    hs = _hist(g, params, 4)
    mats_v = [_cycle_matrix(_levels(h, params), 1, p1 == O.P1_BOOLEAN) for h in hs]
    mats_w = [_cycle_matrix(_levels(h, params), 2, p1 == O.P1_BOOLEAN) for h in hs]
    A = g.to_scipy().toarray()
    rng = np.random.default_rng(11)
    r = rng.standard_normal(g.n)
    r -= r.mean()
    for re in range(1, 5):
        z = O.precond(g, r, hs[:re], params)
        if re <= params.numW:
            Z = mats_w[re - 1]
        else:
            E = np.eye(g.n)
            order = list(range(re)) + list(range(re - 1, -1, -1))
            for j in order:                   # error propagation, first factor applied first
                E = (np.eye(g.n) - mats_v[j] @ A) @ E
            # z = Z r with I - Z A = E on the range of A: build Z by the same
            # accumulation, z_{s+1} = z_s + B_j (r - A z_s)
            Z = np.zeros((g.n, g.n))
            for j in order:
                Z = Z + mats_v[j] @ (np.eye(g.n) - A @ Z)
            assert np.allclose(np.eye(g.n) - Z @ A, E, atol=1e-10)
            # the palindrome is symmetric; a repeated order (1..Re, 1..Re) is not
            assert np.allclose(Z, Z.T, atol=1e-10 * np.abs(Z).max())
        ref = Z @ r
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref), re
    # a wrong hierarchy or order is detected by the same comparison
    z3 = O.precond(g, r, hs[:3], params)
    Zbad = np.zeros((g.n, g.n))
    for j in [0, 1, 2, 0, 1, 2]:
        Zbad = Zbad + mats_v[j] @ (np.eye(g.n) - A @ Zbad)
    assert np.linalg.norm(z3 - Zbad @ r) > 1e-6 * np.linalg.norm(z3)


@pytest.mark.parametrize("re", [1, 3])
def test_pcg_iterate_is_krylov_projection(re):
    # k PCG steps from 0 with a fixed SPD preconditioner Z give
    # e_k = V (V^T A V)^{-1} V^T r, V a basis of span{Zr, (ZA)Zr, ..., (ZA)^{k-1} Zr}
    g = I.grid2d(9, 7, "loguniform", seed=5)
    params = O.default_params(n_min=4)
    hs = _hist(g, params, re)
    A = g.to_scipy().toarray()
    r = I.rhs_normal(g.n, 3)
    k = params.iterW if re <= params.numW else params.iterV
    cols = [O.precond(g, r, hs, params)]
    for _ in range(k - 1):
        cols.append(O.precond(g, A @ cols[-1], hs, params))
    V, _ = np.linalg.qr(np.array(cols).T)
    ek = V @ np.linalg.solve(V.T @ A @ V, V.T @ r)
    e = O.smooth_error(g, r, hs, params)
    assert np.linalg.norm(e - ek) <= 1e-7 * np.linalg.norm(ek)


# ------------------------------------------------------------- Alg. 5 trigger
def _trigger_steps(hist, thr):
    """Rebuild steps implied by a residual history when the smooth error only
    drives the rebuild: after step k rebuild iff the mean of ||r_j||/||r_{j-1}||
    over the steps since the last rebuild exceeds thr (and step k has not
    reached the tolerance)."""
    out, win = [], []
    for k in range(1, len(hist)):
        win.append(hist[k] / hist[k - 1])
        if k == len(hist) - 1:
            break
        if np.mean(win) > thr:
            out.append(k)
            win = []
    return out


def test_trigger_rule_on_hand_built_history():
    # factors 0.9 | 0.1 0.5 0.7 | 0.3 0.2 ... : the window mean passes 0.4 after
    # step 1 (0.9), then after step 4 (mean of 0.1, 0.5, 0.7 = 0.433)
    f = [0.9, 0.1, 0.5, 0.7, 0.3, 0.2, 0.1]
    hist = np.cumprod([1.0] + f)
    assert _trigger_steps(hist, 0.4) == [1, 4]


@pytest.mark.parametrize("mk", [lambda: I.grid2d(32, 32), lambda: I.ring(512, 4),
                                lambda: I.grid2d(20, 20, "loguniform", seed=2)])
def test_alg5_trigger_follows_the_window_mean(mk):
    g = mk()
    for b in (I.rhs_lowfreq(g.n), I.rhs_normal(g.n, 1)):
        for thr in (0.4, 0.25, 0.6):
            _, st, hist = O.solve(g, b, params=O.default_params(threshold=thr))
            assert st["status"] == "OK"
            assert st["rebuilt_after"] == _trigger_steps(hist, thr)
            assert st["resetups"] == len(st["rebuilt_after"])


def test_alg5_1_resetups_every_step():
    # Section 4: with threshold 1e-6 Alg. 5 re-sets up after every iteration
    # but the last, so Re = Iter - 1
    for g in (I.grid2d(32, 32), I.ring(512, 4)):
        for b in (I.rhs_lowfreq(g.n), I.rhs_normal(g.n, 0)):
            _, st, _ = O.solve(g, b, params=O.default_params(threshold=1e-6))
            assert st["status"] == "OK"
            assert st["resetups"] == st["iters"] - 1
            assert st["rebuilt_after"] == list(range(1, st["iters"]))


def test_no_resetup_above_any_factor():
    # the V-cycle is a contraction here, so a threshold of 1 never triggers;
    # the solve is the plain V-cycle iteration on the first hierarchy
    g = I.grid2d(16, 16)
    b = I.rhs_normal(g.n, 0)
    _, st, hist = O.solve(g, b, params=O.default_params(threshold=1.0, max_iter=2000))
    assert st["resetups"] == 0 and st["rebuilt_after"] == []
    assert np.all(hist[1:] < hist[:-1])


def test_alg5_2_resetups_match_paper_tables():
    # Tables 1, 2 (grids) and 4, 5 (rings), Alg. 5(2): the number of re-setups
    # is within 2 of the paper's on every row we run (n = 2^12, 2^14 grids;
    # 2^10, 2^12 rings; low-frequency and zero-sum random b). The paper's start
    # is a matching and its smoother lexicographic Gauss-Seidel, so iteration
    # counts differ more (within a factor 1.6 here).
    with open(os.path.join(GOLDEN, "paper_tables_grid.json")) as f:
        grid = json.load(f)
    with open(os.path.join(GOLDEN, "paper_tables_ring.json")) as f:
        ring = json.load(f)
    rows = [(I.grid2d(64, 64), grid, "4096"), (I.grid2d(128, 128), grid, "16384"),
            (I.ring(1024, 4), ring, "1024"), (I.ring(4096, 4), ring, "4096")]
    for g, ref, key in rows:
        keys = ("table1_lf", "table2_zs") if ref is grid else ("table4_lf", "table5_zs")
        for b, t in ((I.rhs_lowfreq(g.n), keys[0]), (I.rhs_normal(g.n, 0), keys[1])):
            row = ref[t][key]
            _, st, _ = O.solve(g, b)
            assert st["status"] == "OK"
            assert abs(st["resetups"] - row["alg5_2_re"]) <= 2, (t, key, st)
            assert st["iters"] <= 1.6 * row["alg5_2_iter"], (t, key, st)


# ------------------------------------------- round leftovers vs the paper's loop
def _vcycle_factor(g, h, b, iters=20):
    """Mean contraction of the residual over the last 10 of `iters` stationary
    V-cycles with hierarchy h (geometric mean of the step factors)."""
    A = g.to_scipy()
    x = np.zeros(g.n)
    r = b.copy()
    res = [np.linalg.norm(r)]
    for _ in range(iters):
        x += h.vcycle(r)
        x -= x.mean()
        r = b - A @ x
        res.append(np.linalg.norm(r))
    res = np.array(res)
    return float(np.exp(np.mean(np.log(res[-10:] / res[-11:-1]))))


@pytest.mark.parametrize("mk", [lambda: I.workload("C1"), lambda: I.workload("C5-small"),
                                lambda: I.workload("C4-small"), lambda: random_graph(1500, 0.004, 3)])
def test_round_leftovers_match_the_sequential_loop_in_quality(mk):
    # The path cover of the round variant is Alg. 1's greedy cover exactly; the
    # leftovers (Alg. 3 cases 1-3) are handled in rounds instead of the paper's
    # ascending loop. Compared on quality: the V-cycle convergence factor of
    # hierarchies built both ways from the same error vectors agrees to 0.01.
    g = mk()
    b = I.rhs_normal(g.n, 1)
    e1 = O.start_vector(g)
    h0 = O.Hierarchy(g, e1)
    e2 = O.smooth_error(g, b, [h0])
    e2 = (e2 - e2.mean()) / np.linalg.norm(e2 - e2.mean())
    for e in (e1, e2):
        f = [_vcycle_factor(g, O.Hierarchy(g, e, O.default_params(leftover_mode=m)), b)
             for m in (O.LEFT_ROUNDS, O.LEFT_SEQUENTIAL)]
        assert abs(f[0] - f[1]) <= 0.01, f
