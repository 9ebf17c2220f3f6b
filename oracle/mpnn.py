"""Oracle of the learned start-vector network -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatement of the message-passing network that proposes the
first test vector of the adaptive method, its training loss, the analytic
backward pass and the Adam update. The paper has no learned component (its
first hierarchy comes from a matching, Section 4); this network is the
project's own definition and is written out here as that definition:

* input features per vertex i: ``u_i sqrt(n)``, ``log max(deg_i, 1)`` and
  ``log max(D_i, tiny)``, the last two minus their means over the vertices;
  u is the relaxed random start vector (unit norm, zero mean), deg_i the
  number of off-diagonal neighbours and D_i = sum_{j != i} |a_ij|;
* input head ``h0 = C(GELU(W_in f + b_in))`` (3 -> 64);
* four layers ``h' = C(GELU(W_l [h ; m] + b_l))`` with the weighted neighbour
  mean ``m_i = sum_{j != i} |a_ij| h_j / D_i`` (128 -> 64);
* C subtracts from every channel its mean over the vertices, so activations
  carry the variation between vertices rather than a common offset (which
  bfloat16 activations would otherwise resolve poorly);
* output head ``y = w_out . h + b_out`` (64 -> 1), then y minus its mean,
  divided by its 2-norm;
* loss: for every vertex i over its candidate set C(i) (the pattern of A^2
  without i, the pairs the reweighting of Alg. 4 scores), the softmax of
  ``-|e_i - e_j| / tau_i`` of the target e is compared with the softmax of
  ``-|y_i - y_j| / tau_i`` of the prediction by cross-entropy; tau_i is the
  standard deviation of ``|e_i - e_j|`` over C(i) (rows with tau_i = 0 are
  skipped); the loss is the sum over rows divided by n. ``sign(0) = 0`` in
  the gradient.

Pins (tests/test_oracle_mpnn.py): central finite differences for every
parameter group, the constant-input and permutation invariants of the forward
pass, the Gibbs minimum of the loss at y = e, and closed values of GELU.
The quality of the learned vector is parity unpinned: it is judged by the
measured convergence of the method, not by a reference value.

Only the tests, the smoke check and the benchmark's baseline legs may import
this module.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.special import erf

HIDDEN = 64
LAYERS = 4
NFEAT = 3
TINY = 1e-300


def param_shapes():
    """Parameter groups in the order of the flat parameter vector."""
    shapes = [("W_in", (HIDDEN, NFEAT)), ("b_in", (HIDDEN,))]
    for l in range(LAYERS):
        shapes += [(f"W{l}", (HIDDEN, 2 * HIDDEN)), (f"b{l}", (HIDDEN,))]
    shapes += [("w_out", (HIDDEN,)), ("b_out", (1,))]
    return shapes


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(theta):
    out, k = {}, 0
    for name, s in param_shapes():
        sz = int(np.prod(s))
        out[name] = np.asarray(theta[k:k + sz], dtype=np.float64).reshape(s)
        k += sz
    return out


def flatten(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def graph_terms(g):
    """Off-diagonal |a_ij| as CSR, its row sums D and degrees."""
    A = sp.csr_matrix((np.asarray(g.val, np.float64), np.asarray(g.col), np.asarray(g.rowptr)),
                      shape=(g.n, g.n))
    W = abs(A - sp.diags(A.diagonal())).tocsr()
    W.eliminate_zeros()
    D = np.asarray(W.sum(axis=1)).ravel()
    deg = np.diff(W.indptr)
    return W, D, deg


def features(g, u):
    _, D, deg = graph_terms(g)
    n = g.n
    f1 = np.log(np.maximum(deg, 1).astype(np.float64))
    f2 = np.log(np.maximum(D, TINY))
    return np.stack([np.asarray(u, np.float64) * math.sqrt(n), f1 - f1.mean(), f2 - f2.mean()], axis=1)


def centre(h):
    """Subtract every channel's mean over the vertices."""
    return h - h.mean(axis=0)


def neighbour_mean(g, h):
    """m_i = sum_{j != i} |a_ij| h_j / D_i."""
    W, D, _ = graph_terms(g)
    return (W @ h) / np.maximum(D, TINY)[:, None]


def forward(g, u, theta, keep=False):
    """The network's output y-hat (zero mean, unit norm); with keep=True also
    the intermediate values the backward pass needs."""
    P = unflatten(theta)
    W, D, _ = graph_terms(g)
    Dinv = 1.0 / np.maximum(D, TINY)
    F = features(g, u)
    z_in = F @ P["W_in"].T + P["b_in"]
    h = centre(gelu(z_in))
    hs, ms, zs = [h], [], []
    for l in range(LAYERS):
        m = (W @ h) * Dinv[:, None]
        z = np.concatenate([h, m], axis=1) @ P[f"W{l}"].T + P[f"b{l}"]
        h = centre(gelu(z))
        ms.append(m); zs.append(z); hs.append(h)
    y = h @ P["w_out"] + P["b_out"][0]
    zc = y - y.mean()
    nrm = np.linalg.norm(zc)
    yhat = zc / nrm
    if not keep:
        return yhat
    return yhat, dict(F=F, z_in=z_in, hs=hs, ms=ms, zs=zs, y=y, nrm=nrm, W=W, Dinv=Dinv, P=P)


def candidate_pattern(g):
    """Pattern of A^2 without the diagonal (sorted CSR): the candidate pairs."""
    A = sp.csr_matrix((np.ones(len(g.col)), np.asarray(g.col), np.asarray(g.rowptr)), shape=(g.n, g.n))
    A2 = (A @ A + A).tocsr()
    A2.setdiag(0)
    A2.eliminate_zeros()
    A2.sort_indices()
    return A2.indptr.astype(np.int64), A2.indices.astype(np.int64)


def _row_softmax(ptr, x):
    """Row-wise softmax and log-sum-exp of x over the CSR segments."""
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    mx = np.full(n, -np.inf)
    np.maximum.at(mx, rows, x)
    ex = np.exp(x - mx[rows])
    s = np.bincount(rows, weights=ex, minlength=n)
    lse = mx + np.log(s)
    return ex / s[rows], lse, rows


def loss_and_grad(cand, yhat, ehat):
    """Level-set cross-entropy loss and its gradient with respect to y-hat."""
    ptr, col = cand
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    t = np.abs(ehat[rows] - ehat[col])
    cnt = np.maximum(np.diff(ptr), 1)
    mean_t = np.bincount(rows, weights=t, minlength=n) / cnt
    var_t = np.bincount(rows, weights=(t - mean_t[rows]) ** 2, minlength=n) / cnt
    tau = np.sqrt(var_t)
    ok = tau > 0.0
    keep = ok[rows]
    tau_safe = np.where(ok, tau, 1.0)
    p, _, _ = _row_softmax(ptr, -t / tau_safe[rows])
    d = yhat[rows] - yhat[col]
    q, lse, _ = _row_softmax(ptr, -np.abs(d) / tau_safe[rows])
    logq = -np.abs(d) / tau_safe[rows] - lse[rows]
    L = -np.sum(np.where(keep, p * logq, 0.0)) / n
    coef = np.where(keep, (q - p) / tau_safe[rows], 0.0) / n
    sg = np.sign(d)
    g = np.bincount(rows, weights=-sg * coef, minlength=n) + np.bincount(col, weights=sg * coef, minlength=n)
    return L, g


def backward(g, u, theta, ehat, cand=None):
    """Loss and its gradient with respect to the flat parameter vector."""
    if cand is None:
        cand = candidate_pattern(g)
    yhat, C = forward(g, u, theta, keep=True)
    L, gy = loss_and_grad(cand, yhat, ehat)
    return L, backward_from(C, yhat, gy)


def backward_from(C, yhat, gy):
    """The gradient with respect to the parameters given the network's kept
    values C (forward(..., keep=True)), its output y-hat and the loss gradient
    gy with respect to y-hat."""
    P, W, Dinv = C["P"], C["W"], C["Dinv"]
    # y-hat = (y - mean y) / ||y - mean y||
    gz = (gy - yhat * (yhat @ gy)) / C["nrm"]
    dy = gz - gz.mean()
    grads = {}
    hL = C["hs"][-1]
    grads["w_out"] = hL.T @ dy
    grads["b_out"] = np.array([dy.sum()])
    dh = np.outer(dy, P["w_out"])
    WT = W.T.tocsr()
    for l in reversed(range(LAYERS)):
        z, h, m = C["zs"][l], C["hs"][l], C["ms"][l]
        dz = centre(dh) * gelu_grad(z)
        X = np.concatenate([h, m], axis=1)
        grads[f"W{l}"] = dz.T @ X
        grads[f"b{l}"] = dz.sum(axis=0)
        dX = dz @ P[f"W{l}"]
        dm = dX[:, HIDDEN:]
        dh = dX[:, :HIDDEN] + WT @ (dm * Dinv[:, None])
    dz_in = centre(dh) * gelu_grad(C["z_in"])
    grads["W_in"] = dz_in.T @ C["F"]
    grads["b_in"] = dz_in.sum(axis=0)
    return flatten(grads)


def backward_magnitude(g, u, theta, ehat, cand=None):
    """Per parameter, the sum of the absolute values of the terms whose sum the
    backward pass forms for it: every product and sum of the backward pass of
    `backward` taken over absolute values (|dy|, |W|, |X|, |gelu'|, ...). A
    rounding of relative size u in any operand of those terms moves the
    gradient entry by at most about u times this magnitude, whatever
    cancellation the signed sum has."""
    if cand is None:
        cand = candidate_pattern(g)
    yhat, C = forward(g, u, theta, keep=True)
    P, W, Dinv = C["P"], C["W"], C["Dinv"]
    _, gy = loss_and_grad(cand, yhat, ehat)
    gz = (np.abs(gy) + np.abs(yhat) * (np.abs(yhat) @ np.abs(gy))) / C["nrm"]
    dy = gz + gz.mean()
    grads = {}
    hL = np.abs(C["hs"][-1])
    grads["w_out"] = hL.T @ dy
    grads["b_out"] = np.array([dy.sum()])
    dh = np.outer(dy, np.abs(P["w_out"]))
    WT = W.T.tocsr()
    for l in reversed(range(LAYERS)):
        z, h, m = C["zs"][l], C["hs"][l], C["ms"][l]
        dz = (dh + dh.mean(axis=0)) * np.abs(gelu_grad(z))
        X = np.abs(np.concatenate([h, m], axis=1))
        grads[f"W{l}"] = dz.T @ X
        grads[f"b{l}"] = dz.sum(axis=0)
        dX = dz @ np.abs(P[f"W{l}"])
        dm = dX[:, HIDDEN:]
        dh = dX[:, :HIDDEN] + WT @ (dm * Dinv[:, None])
    dz_in = (dh + dh.mean(axis=0)) * np.abs(gelu_grad(C["z_in"]))
    grads["W_in"] = dz_in.T @ np.abs(C["F"])
    grads["b_in"] = dz_in.sum(axis=0)
    return flatten(grads)


def loss(g, u, theta, ehat, cand=None):
    if cand is None:
        cand = candidate_pattern(g)
    return loss_and_grad(cand, forward(g, u, theta), ehat)[0]


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns the new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
