"""Python binding of the PC-alphaAMG library: torch supplies device memory and the
stream; every step of the method runs in the library's CUDA kernels.

>>> from paper_1806_07028_gb300 import Solver, inputs
>>> g = inputs.workload("C1")
>>> s = Solver(g)                       # validates A, builds the first hierarchy
>>> x, st = s.solve(inputs.rhs_normal(g.n))
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import native as N


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(a, dtype, device):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


# ---- device memory through PyTorch -------------------------------------------
# The library allocates every device buffer through callbacks when they are
# installed (pcamg_set_allocator); these route them to PyTorch's caching
# allocator, so that the library and torch share one pool of device memory.
_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_allocator = {"kind": None, "fns": None, "calls": [0, 0]}


def _torch_alloc(nbytes, stream, ctx):
    torch = _torch()
    _allocator["calls"][0] += 1
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                  stream=int(stream or 0))
    except Exception:
        return None


def _torch_free(ptr, stream, ctx):
    _allocator["calls"][1] += 1
    _torch().cuda.caching_allocator_delete(int(ptr))


def use_allocator(kind="torch"):
    """Where the library's device memory comes from from now on: "torch" (the
    PyTorch caching allocator, the default of this binding) or "library" (the
    library's own cached pool). Handles and networks made earlier keep theirs."""
    if kind == _allocator["kind"]:
        return
    if kind == "torch":
        fns = (_ALLOC_T(_torch_alloc), _FREE_T(_torch_free))
        N.check(N.lib().pcamg_set_allocator(C.cast(fns[0], C.c_void_p), C.cast(fns[1], C.c_void_p), None))
        _allocator["fns"] = fns   # the callbacks must outlive every handle made with them
    elif kind == "library":
        N.check(N.lib().pcamg_set_allocator(None, None, None))
    else:
        raise ValueError(kind)
    _allocator["kind"] = kind


def allocator_calls():
    """(allocations, frees) made through the torch callbacks so far."""
    return tuple(_allocator["calls"])


def _ensure_allocator():
    if _allocator["kind"] is None:
        import os
        use_allocator(os.environ.get("PCAMG_ALLOCATOR", "torch"))


def default_params(**kw) -> N.Params:
    p = N.Params()
    N.check(N.lib().pcamg_default_params(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _stats_dict(st, hist, rebuilt=None):
    d = {f: getattr(st, f) for f, _ in N.Stats._fields_ if f not in ("res_hist", "rebuilt")}
    d["status"] = N.status_name(st.status)
    d["res_hist"] = hist[: st.res_hist_len].copy() if hist is not None else None
    if rebuilt is not None:
        d["rebuilt_after"] = [int(k) for k in np.nonzero(rebuilt[: max(st.res_hist_len, 1)])[0]]
    return d


class Solver:
    """A handle of the library bound to one CSR Laplacian on one GPU."""

    def __init__(self, graph, params: N.Params | None = None, e0=None, device="cuda:0",
                 stream=None, mpnn=None):
        torch = _torch()
        _ensure_allocator()
        self.device = torch.device(device)
        self.params = params if params is not None else default_params()
        if e0 is not None:
            self.params.start = N.START_USER
        if mpnn is not None:           # learned start vector
            self.params.start = N.START_LEARNED
            self.params.mpnn = mpnn._h
        self.n = int(graph.n)
        self.nnz = int(graph.nnz)
        with torch.cuda.device(self.device):
            self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            rp = _dev(graph.rowptr, torch.int32, self.device)
            ci = _dev(graph.col, torch.int32, self.device)
            va = _dev(graph.val, torch.float64, self.device)
            e = _dev(e0, torch.float64, self.device) if e0 is not None else None
            h = C.c_void_p()
            st = N.lib().pcamg_setup(C.byref(h), C.byref(self.params), self.n, self.nnz, _ptr(rp),
                                     _ptr(ci), _ptr(va), _ptr(e) if e is not None else None,
                                     _stream_ptr(self._stream))
            N.check(st, None)
            self._h = h

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            N.lib().pcamg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- method steps -------------------------------------------------------
    def adapt(self, e):
        """Alg. 4 from smooth error e (used as given); the new hierarchy becomes current."""
        torch = _torch()
        with torch.cuda.device(self.device):
            et = _dev(e, torch.float64, self.device)
            N.check(N.lib().pcamg_adapt(self._h, _ptr(et)), self._h)

    def solve(self, b, x0=None, hist_cap=4096, raise_on_error=True):
        """Alg. 5. Returns (x as a torch tensor on the device, stats dict)."""
        torch = _torch()
        with torch.cuda.device(self.device):
            bt = _dev(b, torch.float64, self.device)
            xt = (torch.zeros(self.n, dtype=torch.float64, device=self.device) if x0 is None
                  else _dev(x0, torch.float64, self.device).clone())
            hist = np.zeros(hist_cap)
            reb = np.zeros(hist_cap, np.int32)
            st = N.Stats()
            st.res_hist = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.rebuilt = reb.ctypes.data_as(C.POINTER(C.c_int32))
            st.res_hist_cap = hist_cap
            status = N.lib().pcamg_solve(self._h, _ptr(bt), _ptr(xt), C.byref(st))
            if raise_on_error and status not in (N.OK, N.ERR_NOT_CONVERGED):
                N.check(status, self._h)
            return xt, _stats_dict(st, hist, reb)

    def solve_zero_rhs(self, x0, hist_cap=4096):
        """Alg. 6 (b = 0) from initial guess x0."""
        torch = _torch()
        with torch.cuda.device(self.device):
            xt = _dev(x0, torch.float64, self.device).clone()
            hist = np.zeros(hist_cap)
            reb = np.zeros(hist_cap, np.int32)
            st = N.Stats()
            st.res_hist = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.rebuilt = reb.ctypes.data_as(C.POINTER(C.c_int32))
            st.res_hist_cap = hist_cap
            status = N.lib().pcamg_solve_zero_rhs(self._h, _ptr(xt), C.byref(st))
            if status not in (N.OK, N.ERR_NOT_CONVERGED):
                N.check(status, self._h)
            return xt, _stats_dict(st, hist, reb)

    def solve_multi(self, B, X0=None, raise_on_error=True):
        """Several right-hand sides at once (the columns of B, shape n x k):
        each column's outer iteration (params.outer) without re-setup,
        preconditioned by Alg. 2's symmetric composite of V-cycles over every
        hierarchy the handle holds, up to 8 columns per batched cycle. Returns (X, n x k torch tensor on the device, and a
        dict with per-column "iters", "rel_res" and the "status")."""
        torch = _torch()
        with torch.cuda.device(self.device):
            Bt = torch.as_tensor(B, dtype=torch.float64)
            if Bt.dim() == 1:
                Bt = Bt[:, None]
            if Bt.dim() != 2 or Bt.shape[0] != self.n:
                raise ValueError("B must be n x k")
            k = int(Bt.shape[1])
            # column-major n x k: column c at offset c * n
            Bc = Bt.t().contiguous().to(self.device)
            Xc = (torch.zeros((k, self.n), dtype=torch.float64, device=self.device) if X0 is None else
                  torch.as_tensor(X0, dtype=torch.float64).reshape(self.n, k).t().contiguous().to(self.device))
            iters = np.zeros(k, np.int32)
            rel = np.zeros(k)
            status = N.lib().pcamg_solve_multi(self._h, k, _ptr(Bc), _ptr(Xc),
                                               iters.ctypes.data_as(C.c_void_p), rel.ctypes.data_as(C.c_void_p))
            if raise_on_error and status not in (N.OK, N.ERR_NOT_CONVERGED):
                N.check(status, self._h)
            return Xc.t(), {"iters": iters, "rel_res": rel, "status": N.status_name(status)}

    def cycle(self, r, hist=-1, gamma=1):
        """One V- (gamma=1) or W-cycle (gamma=2) correction of hierarchy `hist`."""
        torch = _torch()
        if hist < 0:
            hist = self.num_hierarchies + hist
        with torch.cuda.device(self.device):
            rt = _dev(r, torch.float64, self.device)
            ct = torch.empty(self.n, dtype=torch.float64, device=self.device)
            N.check(N.lib().pcamg_cycle(self._h, hist, gamma, _ptr(rt), _ptr(ct)), self._h)
            return ct

    def smooth_error(self, r):
        """Alg. 2 on the current history; returns the raw PCG iterate."""
        torch = _torch()
        with torch.cuda.device(self.device):
            rt = _dev(r, torch.float64, self.device)
            et = torch.empty(self.n, dtype=torch.float64, device=self.device)
            N.check(N.lib().pcamg_smooth_error(self._h, _ptr(rt), _ptr(et)), self._h)
            return et

    def start_vector(self):
        torch = _torch()
        with torch.cuda.device(self.device):
            et = torch.empty(self.n, dtype=torch.float64, device=self.device)
            N.check(N.lib().pcamg_start_vector(self._h, _ptr(et)), self._h)
            return et

    def last_smooth_error(self):
        """The normalised error the newest hierarchy was built from."""
        torch = _torch()
        with torch.cuda.device(self.device):
            et = torch.empty(self.n, dtype=torch.float64, device=self.device)
            N.check(N.lib().pcamg_last_smooth_error(self._h, _ptr(et)), self._h)
            return et

    # -- inspection -----------------------------------------------------------
    @property
    def num_hierarchies(self):
        return int(N.lib().pcamg_num_hierarchies(self._h))

    def num_levels(self, hist=-1):
        if hist < 0:
            hist = self.num_hierarchies + hist
        return int(N.lib().pcamg_num_levels(self._h, hist))

    def sizes(self, hist, lev):
        s = np.zeros(8, np.int64)
        N.check(N.lib().pcamg_level_sizes(self._h, hist, lev, s.ctypes.data_as(C.c_void_p)), self._h)
        return dict(n=int(s[0]), nnz=int(s[1]), nc=int(s[2]), ncolour=int(s[3]),
                    cover_rounds=int(s[4]), leftover_rounds=int(s[5]), pinned=int(s[6]),
                    tnnz=int(s[7]))

    def level(self, hist, lev, cover=False):
        """One level copied to host numpy arrays."""
        if hist < 0:
            hist = self.num_hierarchies + hist
        s = self.sizes(hist, lev)
        n, nnz, nc = s["n"], s["nnz"], s["nc"]
        agg = np.full(n, -1, np.int32)
        n0 = np.full(n, -1, np.int32); n1 = np.full(n, -1, np.int32)
        rp = np.empty(n + 1, np.int32); ci = np.empty(nnz, np.int32); va = np.empty(nnz)
        pv = np.full(n, np.nan); co = np.full(n, -1, np.int32)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        N.check(N.lib().pcamg_export_level(self._h, hist, lev, p(agg) if nc else None,
                                           p(n0) if cover else None, p(n1) if cover else None,
                                           p(rp), p(ci), p(va), p(pv), p(co)), self._h)
        out = dict(s)
        out.update(rowptr=rp, col=ci, val=va, colour=co if s["ncolour"] else None,
                   agg=agg if nc else None,
                   pval=pv if (lev == 0 and nc and not np.isnan(pv).all()) else None)
        if cover:
            out.update(nbr0=n0, nbr1=n1)
        return out

    def reweighted(self, hist, lev):
        s = self.sizes(hist, lev)
        ptr = np.empty(s["n"] + 1, np.int32); col = np.empty(s["tnnz"], np.int32)
        w = np.empty(s["tnnz"])
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        N.check(N.lib().pcamg_export_reweighted(self._h, hist, lev, p(ptr), p(col), p(w)), self._h)
        return ptr, col, w


# ---- single kernels ---------------------------------------------------------
def residual(rowptr, col, val, x, b, want_norm=True, stream=None):
    """r = b - A x and ||r||^2 on the device (torch tensors in, tensors out)."""
    torch = _torch()
    _ensure_allocator()
    n = rowptr.numel() - 1
    r = torch.empty(n, dtype=torch.float64, device=x.device)
    nrm = torch.zeros(1, dtype=torch.float64, device=x.device) if want_norm else None
    N.check(N.lib().pcamg_residual(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(b), _ptr(r),
                                   _ptr(nrm) if nrm is not None else None, _stream_ptr(stream)))
    return r, nrm


def residual_f32(rowptr, col, val32, x32, b32, stream=None):
    torch = _torch()
    n = rowptr.numel() - 1
    r = torch.empty(n, dtype=torch.float32, device=x32.device)
    N.check(N.lib().pcamg_residual_f32(n, _ptr(rowptr), _ptr(col), _ptr(val32), _ptr(x32),
                                       _ptr(b32), _ptr(r), _stream_ptr(stream)))
    return r


def uniform(seed, n, device="cuda:0", stream=None):
    torch = _torch()
    out = torch.empty(n, dtype=torch.float64, device=device)
    N.check(N.lib().pcamg_uniform(seed, n, _ptr(out), _stream_ptr(stream)))
    return out


def colour(rowptr, col, seed, stream=None):
    torch = _torch()
    n = rowptr.numel() - 1
    out = torch.empty(n, dtype=torch.int32, device=rowptr.device)
    nc = C.c_int32(0)
    N.check(N.lib().pcamg_colour(n, _ptr(rowptr), _ptr(col), seed, _ptr(out), C.byref(nc),
                                 _stream_ptr(stream)))
    return out, int(nc.value)


def solve_host(graph, b, x0=None, params=None):
    """End-to-end call on host numpy buffers (copies happen inside the library)."""
    _ensure_allocator()
    p = params if params is not None else default_params()
    rp = np.ascontiguousarray(graph.rowptr, np.int32)
    ci = np.ascontiguousarray(graph.col, np.int32)
    va = np.ascontiguousarray(graph.val, np.float64)
    bb = np.ascontiguousarray(b, np.float64)
    x = np.zeros(graph.n) if x0 is None else np.array(x0, dtype=np.float64)
    st = N.Stats()
    q = lambda a: a.ctypes.data_as(C.c_void_p)
    status = N.lib().pcamg_solve_host(C.byref(p), graph.n, graph.nnz, q(rp), q(ci), q(va), q(bb),
                                      q(x), C.byref(st), _stream_ptr())
    if status not in (N.OK, N.ERR_NOT_CONVERGED):
        N.check(status)
    return x, _stats_dict(st, None)


class Mpnn:
    """The learned start-vector network (see include/pcamg.h): parameters live
    on the GPU; forward, loss gradient and Adam run in the library's kernels."""

    def __init__(self, params=None, seed=0, _handle=None):
        if _handle is not None:
            self._h = _handle
            return
        if params is None:
            from .inputs import mpnn_init_params
            params = mpnn_init_params(seed)
        w = np.ascontiguousarray(params, dtype=np.float32)
        if w.size != self.num_params():
            raise ValueError(f"expected {self.num_params()} parameters, got {w.size}")
        _ensure_allocator()
        h = C.c_void_p()
        N.check(N.lib().pcamg_mpnn_create(C.byref(h), w.ctypes.data_as(C.c_void_p)))
        self._h = h

    @staticmethod
    def num_params():
        return int(N.lib().pcamg_mpnn_num_params())

    @classmethod
    def pretrained(cls):
        """The network shipped with the package: trained by train_mpnn on 200
        seeded random geometric graphs (n 10k-100k), 30 epochs."""
        import os
        return cls.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                     "mpnn_rgg200.mpnn"))

    @classmethod
    def load(cls, path):
        _ensure_allocator()
        h = C.c_void_p()
        N.check(N.lib().pcamg_mpnn_load(C.byref(h), str(path).encode()))
        return cls(_handle=h)

    def save(self, path):
        N.check(N.lib().pcamg_mpnn_save(self._h, str(path).encode()))

    def close(self):
        if getattr(self, "_h", None):
            N.lib().pcamg_mpnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self):
        w = np.empty(self.num_params(), dtype=np.float32)
        N.check(N.lib().pcamg_mpnn_get_params(self._h, w.ctypes.data_as(C.c_void_p)))
        return w

    @params.setter
    def params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        N.check(N.lib().pcamg_mpnn_set_params(self._h, w.ctypes.data_as(C.c_void_p)))

    def grad(self):
        g = np.empty(self.num_params(), dtype=np.float32)
        N.check(N.lib().pcamg_mpnn_get_grad(self._h, g.ctypes.data_as(C.c_void_p)))
        return g

    def forward(self, solver, u):
        """The network's start vector on solver's graph from the relaxed random start u."""
        torch = _torch()
        with torch.cuda.device(solver.device):
            ut = _dev(u, torch.float64, solver.device)
            yt = torch.empty(solver.n, dtype=torch.float64, device=solver.device)
            N.check(N.lib().pcamg_mpnn_forward(self._h, solver._h, _ptr(ut), _ptr(yt)), solver._h)
            return yt

    def loss_grad(self, solver, u, target):
        """Loss against the target smooth error; the gradient stays in the network."""
        torch = _torch()
        with torch.cuda.device(solver.device):
            ut = _dev(u, torch.float64, solver.device)
            tt = _dev(target, torch.float64, solver.device)
            L = C.c_double(0.0)
            N.check(N.lib().pcamg_mpnn_loss_grad(self._h, solver._h, _ptr(ut), _ptr(tt), C.byref(L)),
                    solver._h)
            return float(L.value)

    def adam_step(self, lr=1e-3):
        N.check(N.lib().pcamg_mpnn_adam_step(self._h, C.c_float(lr)))


def training_example(graph, seed=0, params=None):
    """One training example of the learned start: a solver bound to the graph
    (kept for the loss's A^2 pattern), the relaxed random start u, and the
    target -- the first Alg. 2 smooth error of a plain run (right-hand side
    N(0,1) minus its mean, stopped right after the first re-setup). Returns
    None when the plain run converged without a re-setup."""
    from .inputs import rhs_normal
    p = params if params is not None else default_params()
    p.max_resetups = 1
    s = Solver(graph, params=p)
    _, st = s.solve(rhs_normal(graph.n, seed), raise_on_error=False)
    if st["resetups"] < 1:
        s.close()
        return None
    return s, s.start_vector(), s.last_smooth_error()


def train(net, examples, epochs=10, lr=1e-3):
    """Adam over the examples, one step per example per epoch; returns the mean
    loss of every epoch."""
    hist = []
    for _ in range(epochs):
        tot = 0.0
        for s, u, t in examples:
            tot += net.loss_grad(s, u, t)
            net.adam_step(lr)
        hist.append(tot / max(1, len(examples)))
    return hist


def first_cycles(graph, mpnn=None, e0=None, cycles=5, seed=0, params=None):
    """Convergence factors ||r_k|| / ||r_{k-1}|| of the first V-cycles on the
    first hierarchy (no re-setup), from the relaxed random start, the learned
    start (mpnn) or a given start vector (e0)."""
    from .inputs import rhs_normal
    p = params if params is not None else default_params()
    p.threshold = 1e30
    p.max_iter = cycles
    p.tol = 1e-300
    s = Solver(graph, params=p, mpnn=mpnn, e0=e0)
    _, st = s.solve(rhs_normal(graph.n, seed), raise_on_error=False)
    s.close()
    h = st["res_hist"]
    return h[1:] / h[:-1]
