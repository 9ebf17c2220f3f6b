"""Pins for the oracle's setup (Alg. 4): reweighting, path cover (Alg. 1),
path-cover aggregation (Alg. 3), prolongation and Galerkin products."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import (cover_edges, edges_of, is_path_cover, max_path_cover_weight,
                           nbr_lists, random_graph)


def _pattern(g):
    return sp.csr_matrix((np.ones(g.nnz), g.col, g.rowptr), shape=(g.n, g.n))


# ---------------------------------------------------------------- reweighting
def _hub_graph():
    # scale-free (Chung-Lu, exponent 2.1): hub rows of the A^2 product reach
    # 15,792 contributions, the case of the GPU's long-row paths
    return I.chung_lu(3000, 2.1, 10.0, seed=1)


@pytest.mark.parametrize("mk", [lambda: I.workload("C1"), lambda: random_graph(80, 0.05, 1),
                                lambda: I.grid3d(5, 4, 6, "unit"), _hub_graph])
def test_candidates_are_the_A2_pattern(mk):
    # Alg. 4 step 2: the reweighted graph lives on the pattern of A^2 (no diagonal)
    g = mk()
    e = np.random.default_rng(2).standard_normal(g.n)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    A2 = (_pattern(g) @ _pattern(g)).tocsr()
    A2.setdiag(0); A2.eliminate_zeros(); A2.sort_indices()
    assert np.array_equal(cp, A2.indptr) and np.array_equal(cc, A2.indices)
    # symmetric weights, bit for bit, and heavier exactly when |e_u - e_v| is smaller
    W = sp.csr_matrix((cw, cc, cp), shape=(g.n, g.n))
    assert (W != W.T).nnz == 0
    u = np.repeat(np.arange(g.n), np.diff(cp))
    d = np.abs(e[u] - e[cc])
    order = np.argsort(d, kind="stable")
    assert np.all(np.diff(cw[order]) <= 0)
    assert np.allclose(cw * d, 1.0, rtol=4e-16 * 4)


def test_candidates_zero_error_gives_unit_weights():
    g = I.grid2d(5, 4)
    cp, cc, cw = O.candidates(g.rowptr, g.col, np.zeros(g.n))
    assert np.all(cw == 1.0)


def test_candidates_equal_values_are_capped():
    # |e_u - e_v| = 0 is capped at delta = 2^-52 max|e|
    g = I.grid2d(4, 4)
    e = np.repeat([1.0, 2.0, 3.0, 4.0], 4)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    assert cw.max() == 1.0 / (4.0 * 2.0**-52)


# ---------------------------------------------------------------- path cover
def _cover_graphs():
    out = []
    for s in range(6):
        g = random_graph(40 + 10 * s, 0.06, s)
        e = np.random.default_rng(100 + s).standard_normal(g.n)
        out.append((g, e))
    g = I.grid2d(12, 9)
    out.append((g, np.round(np.random.default_rng(5).standard_normal(g.n), 1)))  # many ties
    out.append((g, np.zeros(g.n)))                                                # all tied
    g = I.ring(64, 4)
    out.append((g, np.sin(np.arange(64) * 2 * np.pi / 64)))
    g = I.workload("C1")
    out.append((g, O.start_vector(g)))
    return out


@pytest.mark.parametrize("case", range(10))
def test_cover_ld_rounds_equal_greedy_alg1(case):
    g, e = _cover_graphs()[case]
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    g0, g1 = O.cover_greedy(cp, cc, cw)
    l0, l1, rounds = O.cover_ld(cp, cc, cw)
    assert np.array_equal(g0, l0) and np.array_equal(g1, l1)
    es = cover_edges(l0, l1)
    assert is_path_cover(g.n, es)
    cand = edges_of(cp, cc, cw)
    assert es <= set(cand)
    # maximal: every other candidate edge touches a degree-2 vertex or joins
    # the two ends of one path (Alg. 1 keeps every edge it can)
    deg = np.array([len(x) for x in nbr_lists(l0, l1)])
    comp = _path_ids(g.n, es)
    for (a, b) in cand:
        if (a, b) in es:
            continue
        assert deg[a] == 2 or deg[b] == 2 or comp[a] == comp[b]


def _path_ids(n, es):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b in es:
        parent[find(a)] = find(b)
    return [find(x) for x in range(n)]


@pytest.mark.parametrize("seed", range(12))
def test_cover_half_approximation_brute_force(seed):
    # Section 2.2 (Moran et al.): the greedy cover weighs at least half of the
    # best path cover. Checked exhaustively on tiny weighted graphs.
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 9))
    ei, ej = [], []
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.4:
                ei.append(a); ej.append(b)
    if len(ei) > 13:
        ei, ej = ei[:13], ej[:13]
    if not ei:
        ei, ej = [0], [1]
    w = rng.uniform(0.1, 1.0, len(ei))
    W = sp.coo_matrix((np.r_[w, w], (np.r_[ei, ej], np.r_[ej, ei])), shape=(n, n)).tocsr()
    W.sort_indices()
    cp, cc, cw = W.indptr.astype(np.int32), W.indices.astype(np.int32), W.data.copy()
    n0, n1 = O.cover_greedy(cp, cc, cw)
    l0, l1, _ = O.cover_ld(cp, cc, cw)
    assert np.array_equal(n0, l0) and np.array_equal(n1, l1)
    es = cover_edges(n0, n1)
    cand = edges_of(cp, cc, cw)
    got = sum(cand[x] for x in es)
    best = max_path_cover_weight(n, cand)
    assert got >= 0.5 * best - 1e-12
    assert got <= best + 1e-12


@pytest.mark.parametrize("f", [lambda i: i, lambda i: i**2, lambda i: np.sqrt(i + 1.0),
                               lambda i: -np.exp(i / 7.0)])
def test_cover_of_path_graph_with_monotone_error_is_the_path(f):
    # along a path graph with strictly monotone e, every distance-2 edge of the
    # A^2 pattern is lighter than the two path edges it spans
    n = 30
    g = I.laplacian_from_edges(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1))
    e = np.array([f(i) for i in range(n)], dtype=float)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, _ = O.cover_ld(cp, cc, cw)
    assert cover_edges(n0, n1) == {(i, i + 1) for i in range(n - 1)}


def test_cover_follows_level_sets_of_linear_error():
    # Fig. 3: on a grid with e linear in x, the level sets are the columns;
    # every column is one consecutive piece of a path
    nx, ny = 10, 8
    g = I.grid2d(nx, ny)
    e = np.tile(np.arange(nx, dtype=float), ny)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, _ = O.cover_ld(cp, cc, cw)
    es = cover_edges(n0, n1)
    for x in range(nx):
        inside = [(a, b) for (a, b) in es if a % nx == x and b % nx == x]
        assert len(inside) == ny - 1


# ---------------------------------------------------------------- aggregation
def _tilde(edges, n):
    i = np.array([a for a, b in edges]); j = np.array([b for a, b in edges])
    w = np.array([edges[k] for k in edges], dtype=float)
    W = sp.coo_matrix((np.r_[w, w], (np.r_[i, j], np.r_[j, i])), shape=(n, n)).tocsr()
    W.sort_indices()
    return W.indptr.astype(np.int32), W.indices.astype(np.int32), W.data.copy()


def test_aggregate_hand_example_cases_1_2_3():
    # Alg. 3 worked by hand. Cover: path 0-1-2-3-4 and singletons 5, 6, 7.
    # Pairing along the path: {0,1}, {2,3}; 4 is left over (odd tail).
    # Best neighbours in the reweighted graph: 4->3, 5->3, 6->7, 7->6.
    # Round 1: 6,7 are mutual (case 1) -> {6,7}. Joiners of {2,3}: 4 then 5.
    #   4: aggregate of 3 has size 2 -> {2,3,4} (case 2)
    #   5: aggregate of 3 has size 3 -> 3 leaves, {3,5} is new (case 3)
    # Aggregates by smallest member: {0,1}=0, {2,4}=1, {3,5}=2, {6,7}=3.
    # Shortened cover: the path's two matched aggregates 0 and 1 stay joined.
    n = 8
    nbr0 = np.array([1, 0, 1, 2, 3, -1, -1, -1], np.int32)
    nbr1 = np.array([-1, 2, 3, 4, -1, -1, -1, -1], np.int32)
    tp, tc, tw = _tilde({(0, 1): 9, (1, 2): 9, (2, 3): 9, (3, 4): 5, (3, 5): 4, (4, 5): 1,
                         (6, 7): 3, (0, 6): 1, (1, 7): 2}, n)
    for mode in (O.LEFT_ROUNDS, O.LEFT_SEQUENTIAL):
        agg, nc, cn0, cn1, rounds = O.aggregate(nbr0, nbr1, tp, tc, tw, leftover_mode=mode)
        assert nc == 4
        assert agg.tolist() == [0, 0, 1, 2, 1, 2, 3, 3]
        assert cn0.tolist() == [1, 0, -1, -1] and cn1.tolist() == [-1, -1, -1, -1]


def test_aggregate_hand_example_rounds_vs_sequential():
    # Leftovers a=0,b=1,c=2 (all singletons in the cover), plus pair {3,4}.
    # best: 0->1, 1->2, 2->1, and 5 (singleton) -> 0.
    # Rounds: round 1: 1,2 mutual -> {1,2}; 0 waits (best 1 unaggregated, not
    #   mutual); 5 waits. Round 2: 0 joins {1,2} -> {0,1,2}; 5's best 0 was
    #   unaggregated at the start of round 2 -> waits. Round 3: 5 -> aggregate
    #   of 0 has size 3 -> 0 leaves: {1,2}, {0,5}.
    #   Result by smallest member: {0,5}=0, {1,2}=1, {3,4}=2.
    # Paper's sequential loop (u ascending): 0 pairs with unaggregated 1 ->
    #   {0,1}; 1 done; 2 -> best 1 in a pair -> {0,1,2}; 5 -> best 0 in a
    #   triple -> {1,2}, {0,5}. Same aggregates here, different route.
    n = 6
    nbr0 = np.array([-1, -1, -1, 4, 3, -1], np.int32)
    nbr1 = np.full(n, -1, np.int32)
    tp, tc, tw = _tilde({(0, 1): 2, (1, 2): 5, (0, 5): 1, (2, 3): 0.5, (3, 4): 7}, n)
    agg, nc, cn0, cn1, rounds = O.aggregate(nbr0, nbr1, tp, tc, tw)
    assert (agg.tolist(), nc, rounds) == ([0, 1, 1, 2, 2, 0], 3, 3)
    agg2, nc2, _, _, _ = O.aggregate(nbr0, nbr1, tp, tc, tw, leftover_mode=O.LEFT_SEQUENTIAL)
    assert agg2.tolist() == [0, 1, 1, 2, 2, 0]


def test_aggregate_sequential_tail_after_round_cap():
    # With a round cap of 0 the rounds variant is the paper's sequential loop.
    g = random_graph(70, 0.05, 9)
    e = np.random.default_rng(3).standard_normal(g.n)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, _ = O.cover_ld(cp, cc, cw)
    a1 = O.aggregate(n0, n1, cp, cc, cw, round_cap=0)[0]
    a2 = O.aggregate(n0, n1, cp, cc, cw, leftover_mode=O.LEFT_SEQUENTIAL)[0]
    assert np.array_equal(a1, a2)


def _check_aggregation(g, e, mode=O.LEFT_ROUNDS):
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, _ = O.cover_ld(cp, cc, cw)
    agg, nc, cn0, cn1, rounds = O.aggregate(n0, n1, cp, cc, cw, leftover_mode=mode)
    sizes = np.bincount(agg, minlength=nc)
    assert agg.min() == 0 and agg.max() == nc - 1
    assert set(np.unique(sizes)) <= {2, 3}           # sizes 2 or 3 (Section 3.3)
    first = np.array([np.flatnonzero(agg == k)[0] for k in range(nc)])
    assert np.all(np.diff(first) > 0)                  # numbered by smallest member
    assert is_path_cover(nc, cover_edges(cn0, cn1))    # shortened paths stay a cover
    # every matched pair along a fine path is one aggregate
    return agg, nc, cn0, cn1


@pytest.mark.parametrize("seed", range(5))
def test_aggregation_invariants(seed):
    g = random_graph(120, 0.03, 20 + seed)
    e = np.random.default_rng(seed).standard_normal(g.n)
    _check_aggregation(g, e)
    _check_aggregation(g, e, O.LEFT_SEQUENTIAL)


def test_aggregation_invariants_grid_and_ring():
    for g in (I.workload("C1"), I.ring(200, 4), I.grid3d(9, 8, 7, "checkerboard", block=3), _hub_graph()):
        _check_aggregation(g, O.start_vector(g))


# ---------------------------------------------------------------- P and Galerkin
def _P(agg, nc, pval=None):
    n = agg.size
    v = np.ones(n) if pval is None else pval
    return sp.csr_matrix((v, (np.arange(n), agg)), shape=(n, nc))


@pytest.mark.parametrize("hub", [False, True])
@pytest.mark.parametrize("mode", [O.P1_E_SCALED, O.P1_BOOLEAN])
def test_hierarchy_galerkin_matches_dense_product(mode, hub):
    g = _hub_graph() if hub else I.grid3d(10, 9, 8, "checkerboard", block=3, xscale=100.0)
    e = O.start_vector(g)
    h = O.Hierarchy(g, e, O.default_params(p1_mode=mode, n_min=20))
    assert h.nlevels >= 3
    for lev in range(h.nlevels - 1):
        L, Cl = h.level(lev), h.level(lev + 1)
        A = sp.csr_matrix((L["val"], L["col"], L["rowptr"]), shape=(L["n"], L["n"]))
        P = _P(L["agg"], L["nc"], L["pval"])
        ref = (P.T @ A @ P).toarray()
        got = sp.csr_matrix((Cl["val"], Cl["col"], Cl["rowptr"]), shape=(Cl["n"], Cl["n"])).toarray()
        scale = np.abs(ref).max()
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * scale)
        # pattern: the boolean product of the patterns (cancellations kept)
        B = _P(L["agg"], L["nc"])
        pat = (B.T @ (abs(A) > 0).astype(float) @ B).tocsr()
        pat.sort_indices()
        assert np.array_equal(pat.indptr, Cl["rowptr"]) and np.array_equal(pat.indices, Cl["col"])
        if lev == 0 and mode == O.P1_E_SCALED:
            # P_1 1 = e (Section 3.3: e lies in the range of P_1)
            assert np.array_equal(P @ np.ones(L["nc"]), e)
            # row sums of A_2 = B^T (e * A e) and x^T A_2 x = (Px)^T A (Px)
            assert np.allclose(got.sum(axis=1), B.T @ (e * (A @ e)), atol=1e-12 * scale)
            x = np.random.default_rng(0).standard_normal(L["nc"])
            assert np.isclose(x @ got @ x, (P @ x) @ A @ (P @ x), rtol=1e-10)
            assert np.linalg.eigvalsh(got).min() > 0
        if mode == O.P1_BOOLEAN or lev > 0:
            Acs = sp.csr_matrix(got)
            if mode == O.P1_BOOLEAN:
                # a Laplacian stays a Laplacian: zero row sums, off-diagonals <= 0
                assert np.abs(got.sum(axis=1)).max() < 1e-12 * scale
                off = got - np.diag(np.diag(got))
                assert off.max() <= 1e-12 * scale
            assert np.allclose(got, got.T, rtol=0, atol=1e-14 * scale)
            del Acs


def test_coarse_reweighted_graph_is_boolean_coarsening():
    g = I.workload("C1")
    e = O.start_vector(g)
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, _ = O.cover_ld(cp, cc, cw)
    agg, nc, _, _, _ = O.aggregate(n0, n1, cp, cc, cw)
    tp, tc, tw = O.galerkin(cp, cc, cw, agg, nc, drop_diag=True)
    W = sp.csr_matrix((cw, cc, cp), shape=(g.n, g.n))
    B = _P(agg, nc)
    ref = (B.T @ W @ B).toarray()
    np.fill_diagonal(ref, 0)
    got = sp.csr_matrix((tw, tc, tp), shape=(nc, nc)).toarray()
    assert np.allclose(got, ref, rtol=1e-14, atol=0)
    assert np.all(tw > 0)


def test_coarse_solve_pinned_cholesky():
    for mode in (O.P1_E_SCALED, O.P1_BOOLEAN):
        g = I.grid2d(20, 20, "loguniform", seed=4)
        h = O.Hierarchy(g, O.start_vector(g), O.default_params(p1_mode=mode, n_min=100))
        L = h.level(h.nlevels - 1)
        A = sp.csr_matrix((L["val"], L["col"], L["rowptr"]), shape=(L["n"], L["n"])).toarray()
        r = np.random.default_rng(1).standard_normal(L["n"])
        if mode == O.P1_BOOLEAN:
            r -= r.mean()
            x = h.coarse_solve(r)
            ref = np.linalg.lstsq(A, r, rcond=None)[0]
            assert np.allclose(x - x.mean(), ref - ref.mean(), atol=1e-9 * np.abs(ref).max())
            assert x[-1] == 0.0 and h.sizes(0)["pinned"] == 1
        else:
            x = h.coarse_solve(r)
            assert np.allclose(x, np.linalg.solve(A, r), rtol=1e-8, atol=1e-10 * np.abs(x).max())
