"""The full C2 workload (128^3 grid, n = 2,097,152, high-contrast weights) in
the benchmark's configuration (FP32 cycles in FP64 refinement, default
parameters): the first hierarchy against the oracle, bit for bit on the
levels the oracle exports (fed the same smooth error), the properties of every
level that hold at any size, and a complete solve checked on the host."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1806_07028_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1806_07028_gb300.build import build
    build()
    import paper_1806_07028_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def C2():
    return I.workload("C2")


def _cover_is_path_cover(n, nbr0, nbr1):
    # degree <= 2, symmetric, no cycles (Alg. 1 keeps only paths)
    for a, b in ((nbr0, nbr1), (nbr1, nbr0)):
        m = a >= 0
        u, v = np.flatnonzero(m), a[m]
        assert np.all(v != u)
        assert np.all((nbr0[v] == u) | (nbr1[v] == u))
    assert np.all((nbr0 != nbr1) | (nbr0 < 0))
    i = np.concatenate([np.flatnonzero(nbr0 >= 0), np.flatnonzero(nbr1 >= 0)])
    j = np.concatenate([nbr0[nbr0 >= 0], nbr1[nbr1 >= 0]])
    E = sp.csr_matrix((np.ones(i.size), (i, j)), shape=(n, n))
    ncomp, lab = sp.csgraph.connected_components(E, directed=False)
    edges = i.size // 2
    assert edges == n - ncomp          # a forest: every component is a path


def test_fullsize_first_hierarchy(P, C2):
    g = C2
    e = O.start_vector(g)
    s = P.Solver(g, params=P.default_params(keep_setup=1, precision=1), e0=e)
    h = O.Hierarchy(g, e)
    assert s.num_levels(0) == h.nlevels
    # level 0: the reweighted A^2 graph, the path cover, the aggregates and P,
    # and level 1's Galerkin matrix, bit for bit
    cp, cc, cw = s.reweighted(0, 0)
    rp, rc, rw = h.candidates()
    assert np.array_equal(cp, rp) and np.array_equal(cc, rc)
    assert np.array_equal(cw.view(np.uint64), rw.view(np.uint64))
    del cp, cc, cw, rp, rc, rw
    prev = None
    for lev in range(h.nlevels):
        G, R = s.level(0, lev, cover=(lev == 0)), h.level(lev)
        for k in ("n", "nnz", "nc", "leftover_rounds"):
            assert G[k] == R[k], (lev, k)
        if lev == 0:
            assert G["cover_rounds"] == R["cover_rounds"]
            assert np.array_equal(G["nbr0"], R["nbr0"]) and np.array_equal(G["nbr1"], R["nbr1"])
            _cover_is_path_cover(G["n"], G["nbr0"], G["nbr1"])
            assert np.array_equal(G["pval"].view(np.uint64), R["pval"].view(np.uint64))
        if lev <= 2:
            assert np.array_equal(G["rowptr"], R["rowptr"]) and np.array_equal(G["col"], R["col"]), lev
            assert np.array_equal(G["val"].view(np.uint64), R["val"].view(np.uint64)), lev
            if R["agg"] is not None:
                assert np.array_equal(G["agg"], R["agg"]), lev
        # every level: P has one nonzero per row (aggregates cover all rows)
        # and the matrix is symmetric
        if G["agg"] is not None:
            cnt = np.bincount(G["agg"], minlength=G["nc"])
            assert G["agg"].min() >= 0 and cnt.min() >= 1
        A = sp.csr_matrix((G["val"], G["col"], G["rowptr"]), shape=(G["n"], G["n"]))
        assert abs(A - A.T).max() <= 1e-15 * abs(A).max(), lev
        # row sums through the levels: P_1 carries e (Section 3.3), so with
        # p = P_1 1 (its values) A_1 1 = P_1^T (A p); below it P is boolean and
        # A_{l+1} 1 = B^T (A_l 1)
        rs = np.asarray(A.sum(axis=1)).ravel()
        if lev == 1:
            want = np.bincount(prev["agg"], weights=prev["pval"] * (prev["A"] @ prev["pval"]), minlength=G["n"])
            assert np.abs(rs - want).max() <= 1e-10 * np.abs(A).sum(axis=1).max(), lev
        elif lev >= 2:
            want = np.bincount(prev["agg"], weights=prev["rs"], minlength=G["n"])
            assert np.abs(rs - want).max() <= 1e-10 * np.abs(A).sum(axis=1).max(), lev
        prev = dict(agg=G["agg"], pval=G["pval"], A=A, rs=rs)
    s.close()


def test_fullsize_cycles_and_start_match_oracle(P, C2):
    # at this size the cycles keep the finest level in colour order (its
    # colours fill the streaming smoother): the start vector's relaxation in
    # that order, and V- and W-cycles through it, against the oracle
    g = C2
    s = P.Solver(g)
    e_gpu = s.start_vector().cpu().numpy()
    s.close()
    e = O.start_vector(g)
    assert np.linalg.norm(e_gpu - e) <= 1e-10 * np.linalg.norm(e)
    h = O.Hierarchy(g, e)
    r = I.rhs_normal(g.n, 6)
    for gamma in (1, 2):
        ref = h.vcycle(r) if gamma == 1 else h.wcycle(r)
        for precision, tol in ((0, 1e-9), (1, 2e-4)):
            s = P.Solver(g, params=P.default_params(precision=precision), e0=e)
            for _ in range(2):   # capture, then replay
                c = s.cycle(r, hist=0, gamma=gamma).cpu().numpy()
                assert np.linalg.norm(c - ref) <= tol * np.linalg.norm(ref), (gamma, precision)
            s.close()


def test_fullsize_boolean_hierarchy_is_laplacian(P, C2):
    # with a boolean P_1 every coarse matrix is a weighted graph Laplacian:
    # symmetric, nonpositive off-diagonals, zero row sums
    s = P.Solver(C2, params=P.default_params(keep_setup=1, precision=1, p1_mode=1))
    for lev in range(s.num_levels(0)):
        G = s.level(0, lev)
        A = sp.csr_matrix((G["val"], G["col"], G["rowptr"]), shape=(G["n"], G["n"]))
        off = A - sp.diags(A.diagonal())
        assert off.data.max(initial=0.0) <= 0.0, lev
        rows = np.asarray(abs(A).sum(axis=1)).ravel()
        assert np.all(np.abs(np.asarray(A.sum(axis=1)).ravel()) <= 1e-12 * rows), lev
        assert abs(A - A.T).max() <= 1e-15 * abs(A).max(), lev
    s.close()


def test_fullsize_solve_reaches_tolerance(P, C2):
    g = C2
    b = I.rhs_normal(g.n, 11)
    s = P.Solver(g, params=P.default_params(precision=1))
    x, st = s.solve(b)
    s.close()
    assert st["status"] == "OK"
    xh = x.cpu().numpy()
    rel = np.linalg.norm(b - g.to_scipy() @ xh) / np.linalg.norm(b)
    assert rel <= 1e-8 and abs(rel - st["rel_res"]) <= 1e-12
    assert abs(xh.sum()) <= 1e-8 * np.abs(xh).sum()     # x orthogonal to the constants


# ---- the full C5 workload: 256^3 grid, n = 16,777,216, jump coefficients on
# 16^3 blocks; the benchmark's headline form (FP32 cycles in FP64 refinement,
# learned start)

@pytest.fixture(scope="module")
def C5():
    return I.workload("C5")


def test_fullsize_C5_first_level_matches_oracle(P, C5):
    # Alg. 4 at level 0 against the oracle's level-wise routines fed the same
    # smooth error (the oracle's relaxed random start): A^2 reweighting (step 2),
    # the path cover in rounds (Alg. 1), aggregates (Alg. 3), P_1 carrying e
    # (Section 3.3) and level 1's Galerkin matrix P_1^T A P_1, bit for bit
    g = C5
    e = O.start_vector(g)
    s = P.Solver(g, params=P.default_params(precision=1))
    e_gpu = s.start_vector().cpu().numpy()
    s.close()
    assert np.linalg.norm(e_gpu - e) <= 1e-10 * np.linalg.norm(e)
    del e_gpu
    s = P.Solver(g, params=P.default_params(keep_setup=1, precision=1), e0=e)
    G0 = s.level(0, 0, cover=True)
    G1 = s.level(0, 1)
    s.close()
    del G0["rowptr"], G0["col"], G0["val"]
    cp, cc, cw = O.candidates(g.rowptr, g.col, e)
    n0, n1, rounds = O.cover_ld(cp, cc, cw)
    assert G0["cover_rounds"] == rounds
    assert np.array_equal(G0["nbr0"], n0) and np.array_equal(G0["nbr1"], n1)
    agg, nc, _, _, lrounds = O.aggregate(n0, n1, cp, cc, cw)
    del cp, cc, cw
    assert (G0["nc"], G0["leftover_rounds"]) == (nc, lrounds)
    assert np.array_equal(G0["agg"], agg)
    _cover_is_path_cover(g.n, G0["nbr0"], G0["nbr1"])
    assert np.bincount(agg, minlength=nc).min() >= 1     # one nonzero per row of P, no empty aggregate
    # (P_1)_ui = e_u, or 1 on an aggregate where e vanishes entirely
    vanish = np.bincount(agg, weights=(e != 0.0).astype(np.float64), minlength=nc) == 0.0
    pval = np.where(vanish[agg], 1.0, e)
    assert np.array_equal(G0["pval"].view(np.uint64), pval.view(np.uint64))
    rp, ci, va = O.galerkin(g.rowptr, g.col, g.val, agg, nc, pval)
    assert G1["n"] == nc and G1["nnz"] == ci.size
    assert np.array_equal(G1["rowptr"], rp) and np.array_equal(G1["col"], ci)
    assert np.array_equal(G1["val"].view(np.uint64), va.view(np.uint64))


def test_fullsize_C5_learned_fp32ir_solve_reaches_tolerance(P, C5):
    # the benchmark's headline form end to end: the shipped network's start
    # vector, FP32 hierarchy and cycles inside FP64 refinement, to 1e-8
    # checked on the host
    g = C5
    b = I.rhs_normal(g.n, 11)
    s = P.Solver(g, params=P.default_params(precision=1), mpnn=P.Mpnn.pretrained())
    x, st = s.solve(b)
    s.close()
    assert st["status"] == "OK"
    xh = x.cpu().numpy()
    rel = np.linalg.norm(b - g.to_scipy() @ xh) / np.linalg.norm(b)
    assert rel <= 1e-8 and abs(rel - st["rel_res"]) <= 1e-12
    assert abs(xh.sum()) <= 1e-8 * np.abs(xh).sum()
