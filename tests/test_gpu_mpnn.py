"""Learned start vector on the GPU vs the FP64 oracle (oracle/mpnn.py).

The GPU stages the layer operands in bfloat16 and accumulates the
tensor-core products in FP32; the oracle runs in FP64 from the same
bfloat16-rounded weights. The tolerances allow a few bfloat16 roundings
(2^-9 relative each) per layer over five layers.
"""
import numpy as np
import pytest

import oracle.mpnn as M
from paper_1806_07028_gb300 import inputs as I
from tests.helpers import random_graph

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


def _params(seed=1):
    w = I.mpnn_init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    off = 0
    for name, s in M.param_shapes():
        sz = int(np.prod(s))
        if name.startswith("b"):
            w[off:off + sz] = rng.uniform(-0.2, 0.2, sz)   # exercise the bias paths
        off += sz
    return w.astype(np.float32)


def _case(P, g, seed=1):
    w = _params(seed)
    net = P.Mpnn(w)
    s = P.Solver(g)
    u = s.start_vector()
    th = M.bf16_round(w.astype(np.float64))
    return net, s, u, th


GRAPHS = {
    "rgg": lambda: I.rgg(3000, 12.0, seed=11),
    "er": lambda: random_graph(700, 0.01, 5),
}


def _smooth_target(g, seed=9):
    t = np.random.default_rng(seed).standard_normal(g.n)
    A = g.to_scipy()
    d = A.diagonal()
    for _ in range(20):                      # a few damped Jacobi steps on noise
        t = t - 0.6 * (A @ t) / d
    t -= t.mean()
    return t / np.linalg.norm(t)


@pytest.mark.parametrize("name", ["rgg", "er"])
def test_forward_matches_oracle(P, name):
    g = GRAPHS[name]()
    net, s, u, th = _case(P, g)
    y = net.forward(s, u).cpu().numpy()
    ref, C = M.forward(g, u.cpu().numpy(), th, keep=True)
    err = np.linalg.norm(y - ref)
    assert abs(y.sum()) < 1e-9 and abs(np.linalg.norm(y) - 1) < 1e-9
    # bfloat16 operands: relative error ~2^-9 per rounding in w_out . h, magnified
    # by removing the mean of y (b_out only shifts y and drops out)
    amp = np.linalg.norm(C["y"] - th[-1]) / C["nrm"]
    tol = 16 * 2.0**-9 * amp
    print(f"forward {name}: err {err:.3e}, mean-removal gain {amp:.2f}, tol {tol:.3e}")
    assert err <= tol, (err, tol)
    s.close()
    net.close()


@pytest.mark.parametrize("name", ["rgg", "er"])
@pytest.mark.parametrize("seed", [2, 4])
def test_loss_and_gradient_match_oracle(P, name, seed):
    # The loss gradient with respect to the output is a steep function of the
    # output (softmax of |y_i - y_j| / tau_i), so the forward pass's bfloat16
    # error alone moves it by a few per cent. The backward pass is therefore
    # checked from the GPU's own output: the oracle evaluates the loss gradient
    # at the GPU's y-hat and carries it back through its FP64 network. What is
    # left is the backward pass's own rounding: every product it forms has its
    # two factors staged in bfloat16 (relative 2^-9 each), so each gradient
    # entry may move by at most about 2^-8 times the sum of the absolute values
    # of its terms (oracle.mpnn.backward_magnitude), whatever cancellation the
    # signed sum has. Each parameter group must also agree to 5 % in 2-norm.
    g = GRAPHS[name]()
    net, s, u, th = _case(P, g, seed=seed)
    t = _smooth_target(g)
    y_gpu = net.forward(s, u).cpu().numpy()
    L = net.loss_grad(s, u, t)
    gg = net.grad().astype(np.float64)
    uu = u.cpu().numpy()
    Lr, _ = M.backward(g, uu, th, t)
    assert abs(L - Lr) <= 2e-2 * abs(Lr), (L, Lr)
    cand = M.candidate_pattern(g)
    y_orc, C = M.forward(g, uu, th, keep=True)
    _, gy_at_gpu = M.loss_and_grad(cand, y_gpu, t)
    ref = M.backward_from(C, y_orc, gy_at_gpu)
    mag = M.backward_magnitude(g, uu, th, t)
    off = 0
    for name_, sh in M.param_shapes():
        sz = int(np.prod(sh))
        a, b, m = gg[off:off + sz], ref[off:off + sz], mag[off:off + sz]
        off += sz
        if name_ == "b_out":
            # y-hat does not depend on b_out: its gradient is zero up to rounding
            assert np.abs(a).max() <= 1e-4 * np.abs(gg).max()
            continue
        assert np.all(np.abs(a - b) <= 2.0**-8 * m), (name_, (np.abs(a - b) / (2.0**-8 * m)).max())
        assert np.linalg.norm(a - b) <= 0.05 * np.linalg.norm(b), (name_, np.linalg.norm(a - b) / np.linalg.norm(b))
    s.close()
    net.close()


def test_adam_step_matches_oracle(P):
    g = GRAPHS["er"]()
    net, s, u, th = _case(P, g, seed=3)
    t = _smooth_target(g, 1)
    w0 = net.params.astype(np.float64)
    net.loss_grad(s, u, t)
    gg = net.grad().astype(np.float64)
    net.adam_step(0.01)
    w1 = net.params.astype(np.float64)
    ref, _, _ = M.adam_step(w0, gg, np.zeros_like(w0), np.zeros_like(w0), 1, lr=0.01)
    assert np.allclose(w1, ref, rtol=1e-5, atol=1e-7)
    s.close()
    net.close()


def test_save_load_roundtrip(P, tmp_path):
    w = _params(4)
    net = P.Mpnn(w)
    f = tmp_path / "net.mpnn"
    net.save(f)
    net2 = P.Mpnn.load(f)
    assert np.array_equal(net2.params, w)
    net.close()
    net2.close()


def test_learned_start_solves(P):
    g = I.rgg(4000, 12.0, seed=21)
    net = P.Mpnn(_params(5))
    s = P.Solver(g, mpnn=net)
    x, st = s.solve(I.rhs_normal(g.n, 2))
    assert st["status"] == "OK" and st["rel_res"] <= 1e-8
    s.close()
    net.close()


def test_training_example_and_loss_decrease(P):
    # the target of a training example is the first Alg. 2 smooth error of a
    # plain run; Adam steps on one graph lower its loss
    g = I.rgg(3000, 12.0, seed=31)
    ex = P.training_example(g, seed=0)
    assert ex is not None
    s, u, t = ex
    tt = t.cpu().numpy()
    assert abs(tt.sum()) < 1e-8 and abs(np.linalg.norm(tt) - 1) < 1e-8
    net = P.Mpnn(seed=0)
    hist = P.train(net, [ex], epochs=30, lr=3e-3)
    assert hist[-1] < hist[0]
    s.close()
    net.close()


def test_trained_network_gain(P):
    # what the shipped network (trained on 200 seeded random geometric graphs)
    # gains over the relaxed random start on held-out graphs of the same kind:
    # the first hierarchy's convergence factor, the re-setups and the solve time
    from paper_1806_07028_gb300 import train_mpnn as T
    net = P.Mpnn.pretrained()
    rows = T.evaluate(net, T.rgg_set(3, 20_000, 40_000, seed=424242))
    m = T.summarise(rows)
    print("held-out means:", m)
    for r in rows:
        assert r["random"]["status"] == "OK" and r["learned"]["status"] == "OK"
    assert m["learned"]["resetups"] <= m["random"]["resetups"]
    assert m["learned"]["conv"] <= m["random"]["conv"] + 0.005
    net.close()
