"""The oracle's several-right-hand-side solve (orc_solve_multi): the outer
iteration of Alg. 5 without re-setup, one column at a time, preconditioned by
Alg. 2's composite product of V-cycles over the given hierarchies. Pinned to
the composite preconditioner (itself pinned against assembled V-cycle
matrices), to flexible CG written out here from its recurrence, and to the
residual computed with scipy."""
import numpy as np
import pytest

import oracle as O
from paper_1806_07028_gb300 import inputs as I


@pytest.fixture(scope="module")
def case():
    g = I.grid2d(24, 20)
    e1 = O.start_vector(g)
    e2 = O.start_vector(g, O.default_params(seed=77))
    hs = [O.Hierarchy(g, e1), O.Hierarchy(g, e2)]
    B = np.stack([I.rhs_normal(g.n, 10 + c) for c in range(3)], axis=1)
    return g, hs, B


def _composite(g, hs, r):
    return O.precond(g, r, hs, O.default_params(numW=0))


def test_first_stationary_step_is_the_composite(case):
    g, hs, B = case
    X, it, rel, st = O.solve_multi(g, B, hs, params=O.default_params(outer=0, max_iter=1))
    assert st == "NOT_CONVERGED" and list(it) == [1, 1, 1]
    for c in range(3):
        z = _composite(g, hs, B[:, c])
        z -= z.mean()
        assert np.allclose(X[:, c], z, rtol=0, atol=1e-13 * np.abs(z).max())


def test_two_flexible_cg_steps(case):
    # flexible CG from x = 0 with the composite z = M(r): p0 = z0, alpha =
    # r.z / p.Ap, then beta = z1.(r1 - r0) / (z0.r0), p1 = z1 + beta p0
    g, hs, B = case
    A = g.to_scipy()
    X, it, rel, st = O.solve_multi(g, B, hs, params=O.default_params(outer=1, max_iter=2))
    for c in range(3):
        b = B[:, c]
        x = np.zeros(g.n)
        r = b.copy()
        p = zold = rold = None
        for k in range(2):
            z = _composite(g, hs, r)
            if k == 0:
                p = z.copy()
            else:
                beta = z @ (r - rold) / (zold @ rold)
                p = z + beta * p
            alpha = (r @ z) / (p @ (A @ p))
            x = x + alpha * p
            rold, zold = r, z
            x -= x.mean()
            r = b - A @ x
        assert np.linalg.norm(X[:, c] - x) <= 1e-11 * np.linalg.norm(x), c
        assert abs(rel[c] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-12


def test_columns_are_independent_and_converge(case):
    g, hs, B = case
    A = g.to_scipy()
    X, it, rel, st = O.solve_multi(g, B, hs, params=O.default_params(outer=1))
    assert st == "OK"
    for c in range(3):
        x1, it1, rel1, st1 = O.solve_multi(g, B[:, c:c + 1], hs, params=O.default_params(outer=1))
        assert np.array_equal(X[:, c], x1[:, 0]) and it[c] == it1[0]
        res = np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c])
        assert res <= 1e-8 and abs(res - rel[c]) <= 1e-14
        assert abs(X[:, c].sum()) <= 1e-10 * np.abs(X[:, c]).sum()
    # the stationary form also converges with both hierarchies
    X0, it0, rel0, st0 = O.solve_multi(g, B, hs, params=O.default_params(outer=0))
    assert st0 == "OK" and np.all(it0 >= it)


def test_invalid(case):
    g, hs, B = case
    Z = B.copy()
    Z[:, 1] = 0.0
    assert O.solve_multi(g, Z, hs)[3] == "INVALID"
