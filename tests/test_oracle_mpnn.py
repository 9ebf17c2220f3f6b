"""Pins for the oracle of the learned start-vector network (oracle/mpnn.py)."""
import math

import numpy as np
import pytest

import oracle.mpnn as M
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph


def _unit(v):
    v = v - v.mean()
    return v / np.linalg.norm(v)


@pytest.fixture(scope="module")
def case():
    g = random_graph(30, 0.15, 3)
    rng = np.random.default_rng(0)
    u = _unit(rng.standard_normal(g.n))
    e = _unit(rng.standard_normal(g.n))
    th = M.bf16_round(I.mpnn_init_params(1).astype(np.float64))
    th[M.n_params() - 1] = 0.3           # nonzero output bias
    return g, u, e, th, M.candidate_pattern(g)


def test_gelu_closed_values():
    # GELU(x) = x Phi(x): Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1)
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(np.array(-1.0)) + 0.15865525393145707) < 1e-15
    assert abs(M.gelu(np.array(3.0)) - 3.0 * 0.9986501019683699) < 1e-14
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(x), fd, rtol=0, atol=1e-9)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).standard_normal(10000) * np.logspace(-20, 20, 10000)
    x = np.concatenate([x, [1.0, 1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-8), 0.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)
    # ties go to the even mantissa
    assert M.bf16_round(np.array([1 + 2**-8]))[0] == 1.0
    assert M.bf16_round(np.array([1 + 3 * 2**-8]))[0] == 1 + 2**-6


def test_neighbour_mean_path_and_constant():
    # path 0 -(2)- 1 -(3)- 2: m_0 = h_1, m_1 = (2 h_0 + 3 h_2) / 5, m_2 = h_1
    g = I.laplacian_from_edges(3, np.array([0, 1]), np.array([1, 2]), np.array([2.0, 3.0]), "p3")
    h = np.array([[1.0, -2.0], [4.0, 0.5], [-3.0, 7.0]])
    m = M.neighbour_mean(g, h)
    assert np.allclose(m[0], h[1]) and np.allclose(m[2], h[1])
    assert np.allclose(m[1], (2 * h[0] + 3 * h[2]) / 5)
    gg = random_graph(40, 0.1, 1)
    c = np.tile(np.arange(5.0), (gg.n, 1))
    assert np.allclose(M.neighbour_mean(gg, c), c, rtol=0, atol=1e-14)


def test_forward_normalised_and_permutation_equivariant(case):
    g, u, e, th, _ = case
    y = M.forward(g, u, th)
    assert abs(y.sum()) < 1e-12 and abs(np.linalg.norm(y) - 1) < 1e-12
    perm = np.random.default_rng(2).permutation(g.n)
    inv = np.argsort(perm)
    A = g.to_scipy()[perm][:, perm].tocoo()
    m = A.row < A.col
    gp = I.laplacian_from_edges(g.n, A.row[m], A.col[m], -A.data[m], "perm")
    yp = M.forward(gp, u[perm], th)
    assert np.allclose(yp, y[perm], rtol=0, atol=1e-12)
    Lp, gradp = M.backward(gp, u[perm], th, e[perm])
    L, grad = M.backward(g, u, th, e)
    assert abs(L - Lp) < 1e-12 and np.allclose(grad, gradp, rtol=1e-10, atol=1e-12)
    assert inv.size == g.n


def test_loss_minimum_at_target(case):
    # Gibbs: the cross-entropy of p against q is smallest (the entropy of p)
    # when q = p, i.e. at y-hat = e; there the gradient vanishes
    g, u, e, th, cand = case
    L0, g0 = M.loss_and_grad(cand, e, e)
    assert np.all(g0 == 0.0)
    ptr, col = cand
    ent = 0.0
    for i in range(g.n):
        t = np.abs(e[i] - e[col[ptr[i]:ptr[i + 1]]])
        tau = t.std()
        p = np.exp(-t / tau) / np.exp(-t / tau).sum()
        ent -= (p * np.log(p)).sum()
    assert abs(L0 - ent / g.n) < 1e-12
    rng = np.random.default_rng(4)
    for _ in range(5):
        L1, _ = M.loss_and_grad(cand, _unit(rng.standard_normal(g.n)), e)
        assert L1 > L0
    # shift of y-hat and a joint sign flip leave the loss unchanged
    L2, _ = M.loss_and_grad(cand, e + 0.7, e)
    L3, _ = M.loss_and_grad(cand, -e, -e)
    assert abs(L2 - L0) < 1e-12 and abs(L3 - L0) < 1e-12


@pytest.mark.parametrize("group", [s[0] for s in M.param_shapes()])
def test_backward_matches_central_differences(case, group):
    g, u, e, th, cand = case
    L, grad = M.backward(g, u, th, e, cand)
    off = 0
    for name, s in M.param_shapes():
        sz = int(np.prod(s))
        if name == group:
            break
        off += sz
    idx = off + np.random.default_rng(7).choice(sz, size=min(sz, 24), replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss(g, u, tp, e, cand) - M.loss(g, u, tm, e, cand)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1e-3, np.abs(grad).max()), (name, k, fd, grad[k])


def test_adam_first_step_is_signed_lr():
    # bias-corrected first step: m_hat = g, v_hat = g^2, so the step is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15, atol=0)
    th2, m2, v2 = M.adam_step(th, g, m, v, 2, lr=0.01)
    assert np.allclose(m2, (0.9 * 0.1 + 0.1) * g) and np.allclose(v2, (0.999 * 0.001 + 0.001) * g * g)


def test_init_and_layout():
    th = I.mpnn_init_params(3).astype(np.float64)
    assert th.size == M.n_params() == 33345
    assert np.array_equal(th.astype(np.float32).astype(np.float64), th)
    P = M.unflatten(th)
    assert P["W0"].shape == (64, 128) and np.all(P["b0"] == 0)
    assert np.all(np.abs(P["W0"]) <= 1 / math.sqrt(128))
