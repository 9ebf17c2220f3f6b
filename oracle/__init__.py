"""CPU oracle for PC-alphaAMG (arXiv 1806.07028) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 C restatement of the method (Alg. 1-6 of the
paper), loaded through ctypes. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the CUDA library never
does, and the two share no code.

Every function mirrors one in ``oracle.h``; arrays are numpy and are copied to
contiguous int32 / float64 first.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = ["orc_core.c", "orc_setup.c", "orc_solve.c"]
_lock = threading.Lock()
_lib = None

P1_E_SCALED, P1_BOOLEAN = 0, 1
LEFT_ROUNDS, LEFT_SEQUENTIAL = 0, 1
COVER_LD, COVER_GREEDY = 0, 1
UPD_REBUILD_ONLY, UPD_ADD_CORRECTION = 0, 1
OUTER_STATIONARY, OUTER_FCG = 0, 1
ERR = {0: "OK", 1: "INVALID", 2: "NOT_LAPLACIAN", 3: "OOM", 5: "ROUND_CAP", 6: "SINGULAR",
       7: "NOT_CONVERGED", 8: "DIVERGED", 9: "COARSE_TOO_BIG"}


def build(force=False):
    """Compile the oracle with gcc (-O2, no FMA contraction) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdrs = [os.path.join(_HERE, h) for h in ("oracle.h", "orc_internal.h")]
    if not force and os.path.exists(_SO):
        t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= t for s in srcs + hdrs):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("threshold", C.c_double),
                ("numW", C.c_int32), ("iterW", C.c_int32), ("iterV", C.c_int32),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("relax_sweeps", C.c_int32),
                ("seed", C.c_uint64), ("n_min", C.c_int32), ("max_levels", C.c_int32),
                ("round_cap", C.c_int32), ("p1_mode", C.c_int32), ("leftover_mode", C.c_int32),
                ("cover_mode", C.c_int32), ("dense_max", C.c_int32), ("l1jac_rows", C.c_int32),
                ("update_mode", C.c_int32), ("keep_setup", C.c_int32), ("init_mwm", C.c_int32),
                ("outer", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("resetups", C.c_int32), ("levels", C.c_int32),
                ("status", C.c_int32), ("rel_res", C.c_double), ("oc_mean", C.c_double),
                ("cycles", C.c_int64), ("wcycles", C.c_int64)]


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_PI = C.POINTER(C.c_int32)
_PD = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_default_params.argtypes = [C.POINTER(Params)]
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
            L.orc_splitmix64.argtypes = [C.c_uint64]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_uniform_pm1.argtypes = [C.c_uint64, C.c_int64, _f64p]
            L.orc_residual.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
            L.orc_colour.argtypes = [C.c_int32, _i32p, _i32p, C.c_uint64, _i32p, _PI]
            L.orc_colour.restype = C.c_int32
            L.orc_colour_smoother.argtypes = [C.c_int32, _i32p, _i32p, C.c_uint64, _i32p, _PI]
            L.orc_colour_smoother.restype = C.c_int32
            L.orc_mcgs_sweep.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, C.c_int32,
                                         _f64p, _f64p, C.c_int32]
            L.orc_l1jac_sweep.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.orc_gs_perm_sweep.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, _f64p, _f64p]
            L.orc_candidates.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.POINTER(_PI),
                                         C.POINTER(_PI), C.POINTER(_PD)]
            L.orc_candidates.restype = C.c_int32
            for f in (L.orc_cover_greedy,):
                f.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p]
                f.restype = C.c_int32
            L.orc_cover_ld.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _PI]
            L.orc_cover_ld.restype = C.c_int32
            L.orc_aggregate.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _i32p, _f64p, C.c_int32,
                                        C.c_int32, _i32p, _PI, _i32p, _i32p, _PI]
            L.orc_aggregate.restype = C.c_int32
            L.orc_galerkin.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, C.c_int32,
                                       C.c_void_p, C.c_int32, C.POINTER(_PI), C.POINTER(_PI),
                                       C.POINTER(_PD), C.POINTER(C.c_int64)]
            L.orc_galerkin.restype = C.c_int32
            L.orc_build.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, C.POINTER(Params), _PI]
            L.orc_build.restype = C.c_void_p
            L.orc_build_mwm.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.POINTER(Params), _PI]
            L.orc_build_mwm.restype = C.c_void_p
            L.orc_mwm_aggregate.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _i32p, _PI, _PI]
            L.orc_mwm_aggregate.restype = C.c_int32
            L.orc_hier_free.argtypes = [C.c_void_p]
            L.orc_hier_nlevels.argtypes = [C.c_void_p]
            L.orc_hier_nlevels.restype = C.c_int32
            L.orc_hier_sizes.argtypes = [C.c_void_p, C.c_int32, _i64p]
            L.orc_hier_export.argtypes = [C.c_void_p, C.c_int32] + [C.c_void_p] * 8
            L.orc_hier_export_candidates.argtypes = [C.c_void_p, _i32p, _i32p, _f64p]
            L.orc_hier_oc.argtypes = [C.c_void_p]
            L.orc_hier_oc.restype = C.c_double
            for f in (L.orc_vcycle, L.orc_wcycle, L.orc_coarse_solve):
                f.argtypes = [C.c_void_p, _f64p, _f64p]
            L.orc_start_vector.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.POINTER(Params), _f64p]
            L.orc_start_vector.restype = C.c_int32
            L.orc_smooth_error.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p,
                                           C.POINTER(C.c_void_p), C.c_int32, C.POINTER(Params), _f64p]
            L.orc_smooth_error.restype = C.c_int32
            L.orc_solve.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.POINTER(Params),
                                    C.c_void_p, C.POINTER(Stats), C.c_void_p, C.c_int32, C.c_void_p]
            L.orc_precond.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.POINTER(C.c_void_p),
                                      C.c_int32, C.POINTER(Params), _f64p, _f64p]
            L.orc_solve.restype = C.c_int32
            L.orc_solve_zero_rhs.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, C.POINTER(Params),
                                             C.c_void_p, C.POINTER(Stats), C.c_void_p, C.c_int32]
            L.orc_solve_zero_rhs.restype = C.c_int32
            L.orc_solve_multi.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _f64p, _f64p,
                                          C.POINTER(Params), C.POINTER(C.c_void_p), C.c_int32, C.c_void_p,
                                          C.c_void_p]
            L.orc_solve_multi.restype = C.c_int32
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _csr(g):
    return _i32(g.rowptr), _i32(g.col), _f64(g.val)


def default_params(**kw):
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _take(ptr, n, dtype):
    if n == 0:
        out = np.zeros(0, dtype=dtype)
    else:
        out = np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)
    lib().orc_free(C.cast(ptr, C.c_void_p))
    return out


# ---- random numbers --------------------------------------------------------
def philox4x64_10(ctr, key):
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(np.asarray(ctr, dtype=np.uint64), np.asarray(key, dtype=np.uint64), out)
    return out


def splitmix64(x):
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def uniform_pm1(seed, n):
    out = np.empty(n, dtype=np.float64)
    lib().orc_uniform_pm1(seed, n, out)
    return out


# ---- level operators ---------------------------------------------------------
def residual(g, x, b):
    rp, ci, v = _csr(g)
    r = np.empty(g.n)
    lib().orc_residual(g.n, rp, ci, v, _f64(x), _f64(b), r)
    return r


def colour(g, seed=12345, rowptr=None, col=None, n=None):
    if g is not None:
        rowptr, col, n = g.rowptr, g.col, g.n
    out = np.empty(n, dtype=np.int32)
    rounds = C.c_int32(0)
    nc = lib().orc_colour(n, _i32(rowptr), _i32(col), seed, out, C.byref(rounds))
    if nc < 0:
        raise RuntimeError(ERR.get(-nc))
    return out, int(nc), int(rounds.value)


def colour_smoother(g, seed=12345):
    """The smoother's colouring: BFS parity on connected bipartite graphs, else JP."""
    out = np.empty(g.n, dtype=np.int32)
    rounds = C.c_int32(0)
    nc = lib().orc_colour_smoother(g.n, _i32(g.rowptr), _i32(g.col), seed, out, C.byref(rounds))
    if nc < 0:
        raise RuntimeError(ERR.get(-nc))
    return out, int(nc), int(rounds.value)


def mcgs_sweep(g, colours, ncolour, b, x, forward=True):
    rp, ci, v = _csr(g)
    x = _f64(x).copy()
    lib().orc_mcgs_sweep(g.n, rp, ci, v, _i32(colours), ncolour, _f64(b), x, 1 if forward else 0)
    return x


def l1jac_sweep(g, b, x):
    rp, ci, v = _csr(g)
    x = _f64(x).copy()
    lib().orc_l1jac_sweep(g.n, rp, ci, v, _f64(b), x)
    return x


def gs_perm_sweep(g, perm, b, x):
    rp, ci, v = _csr(g)
    x = _f64(x).copy()
    lib().orc_gs_perm_sweep(g.n, rp, ci, v, _i32(perm), _f64(b), x)
    return x


# ---- setup pieces -------------------------------------------------------------
def candidates(rowptr, col, e):
    n = len(rowptr) - 1
    cp, cc, cw = _PI(), _PI(), _PD()
    st = lib().orc_candidates(n, _i32(rowptr), _i32(col), _f64(e), C.byref(cp), C.byref(cc), C.byref(cw))
    if st:
        raise RuntimeError(ERR.get(st))
    ptr = _take(cp, n + 1, np.int32)
    nn = int(ptr[-1])
    return ptr, _take(cc, nn, np.int32), _take(cw, nn, np.float64)


def cover_greedy(cptr, ccol, cw):
    n = len(cptr) - 1
    n0 = np.empty(n, np.int32); n1 = np.empty(n, np.int32)
    st = lib().orc_cover_greedy(n, _i32(cptr), _i32(ccol), _f64(cw), n0, n1)
    if st:
        raise RuntimeError(ERR.get(st))
    return n0, n1


def cover_ld(cptr, ccol, cw):
    n = len(cptr) - 1
    n0 = np.empty(n, np.int32); n1 = np.empty(n, np.int32)
    rounds = C.c_int32(0)
    st = lib().orc_cover_ld(n, _i32(cptr), _i32(ccol), _f64(cw), n0, n1, C.byref(rounds))
    if st:
        raise RuntimeError(ERR.get(st))
    return n0, n1, int(rounds.value)


def aggregate(nbr0, nbr1, tptr, tcol, tw, round_cap=64, leftover_mode=LEFT_ROUNDS):
    n = len(nbr0)
    agg = np.empty(n, np.int32)
    cn0 = np.empty(max(n, 1), np.int32); cn1 = np.empty(max(n, 1), np.int32)
    nc = C.c_int32(0); rounds = C.c_int32(0)
    st = lib().orc_aggregate(n, _i32(nbr0), _i32(nbr1), _i32(tptr), _i32(tcol), _f64(tw),
                             round_cap, leftover_mode, agg, C.byref(nc), cn0, cn1, C.byref(rounds))
    if st:
        raise RuntimeError(ERR.get(st))
    k = int(nc.value)
    return agg, k, cn0[:k].copy(), cn1[:k].copy(), int(rounds.value)


def galerkin(rowptr, col, val, agg, nc, pval=None, drop_diag=False):
    n = len(rowptr) - 1
    op, oc, ov = _PI(), _PI(), _PD()
    nnz = C.c_int64(0)
    pv = None if pval is None else _f64(pval)
    st = lib().orc_galerkin(n, _i32(rowptr), _i32(col), _f64(val), _i32(agg), nc,
                            None if pv is None else pv.ctypes.data_as(C.c_void_p),
                            1 if drop_diag else 0, C.byref(op), C.byref(oc), C.byref(ov), C.byref(nnz))
    if st:
        raise RuntimeError(ERR.get(st))
    k = int(nnz.value)
    return _take(op, nc + 1, np.int32), _take(oc, k, np.int32), _take(ov, k, np.float64)


# ---- hierarchy --------------------------------------------------------------------
def mwm_aggregate(g, ld=True):
    """MWM aggregation of one level (Section 2.1): (agg, nc, rounds)."""
    rp, ci, v = _csr(g)
    agg = np.empty(g.n, np.int32)
    nc, rounds = C.c_int32(0), C.c_int32(0)
    st = lib().orc_mwm_aggregate(g.n, rp, ci, v, 1 if ld else 0, agg, C.byref(nc), C.byref(rounds))
    if st:
        raise RuntimeError(ERR.get(st))
    return agg, int(nc.value), int(rounds.value)


class Hierarchy:
    """An oracle hierarchy built from smooth error e (Alg. 4), or, with
    e = None, by MWM_setup (Section 2.1)."""

    def __init__(self, g, e, params=None):
        self.g = g
        p = params if params is not None else default_params()
        self._p = p
        rp, ci, v = _csr(g)
        self._keep = (rp, ci, v)
        st = C.c_int32(0)
        if e is None:
            h = lib().orc_build_mwm(g.n, rp, ci, v, C.byref(p), C.byref(st))
        else:
            h = lib().orc_build(g.n, rp, ci, v, _f64(e), C.byref(p), C.byref(st))
        if not h:
            raise RuntimeError(f"orc_build failed: {ERR.get(st.value, st.value)}")
        self._h = h

    def close(self):
        if self._h:
            lib().orc_hier_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlevels(self):
        return int(lib().orc_hier_nlevels(self._h))

    def sizes(self, lev):
        s = np.zeros(8, np.int64)
        lib().orc_hier_sizes(self._h, lev, s)
        return dict(n=int(s[0]), nnz=int(s[1]), nc=int(s[2]), ncolour=int(s[3]),
                    cover_rounds=int(s[4]), leftover_rounds=int(s[5]), pinned=int(s[6]),
                    cand_nnz=int(s[7]))

    def level(self, lev):
        s = self.sizes(lev)
        n, nnz, nc = s["n"], s["nnz"], s["nc"]
        agg = np.full(n, -1, np.int32); n0 = np.full(n, -1, np.int32); n1 = np.full(n, -1, np.int32)
        rp = np.empty(n + 1, np.int32); ci = np.empty(nnz, np.int32); v = np.empty(nnz, np.float64)
        pv = np.full(n, np.nan); colr = np.full(n, -1, np.int32)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        lib().orc_hier_export(self._h, lev, ptr(agg), ptr(n0), ptr(n1), ptr(rp), ptr(ci), ptr(v),
                              ptr(pv), ptr(colr))
        out = dict(s)
        out.update(rowptr=rp, col=ci, val=v, nbr0=n0, nbr1=n1, colour=colr)
        out["agg"] = agg if nc > 0 else None
        out["pval"] = pv if (lev == 0 and nc > 0 and not np.isnan(pv).all()) else None
        return out

    def candidates(self):
        s = self.sizes(0)
        cp = np.empty(s["n"] + 1, np.int32); cc = np.empty(s["cand_nnz"], np.int32)
        cw = np.empty(s["cand_nnz"], np.float64)
        lib().orc_hier_export_candidates(self._h, cp, cc, cw)
        return cp, cc, cw

    def oc(self):
        return float(lib().orc_hier_oc(self._h))

    def vcycle(self, r):
        c = np.empty(self.g.n)
        lib().orc_vcycle(self._h, _f64(r), c)
        return c

    def wcycle(self, r):
        c = np.empty(self.g.n)
        lib().orc_wcycle(self._h, _f64(r), c)
        return c

    def coarse_solve(self, r):
        x = np.empty(len(r))
        lib().orc_coarse_solve(self._h, _f64(r), x)
        return x


def start_vector(g, params=None):
    p = params if params is not None else default_params()
    rp, ci, v = _csr(g)
    e = np.empty(g.n)
    st = lib().orc_start_vector(g.n, rp, ci, v, C.byref(p), e)
    if st:
        raise RuntimeError(ERR.get(st))
    return e


def smooth_error(g, r, hiers, params=None):
    p = params if params is not None else default_params()
    rp, ci, v = _csr(g)
    arr = (C.c_void_p * len(hiers))(*[h._h for h in hiers])
    e = np.empty(g.n)
    st = lib().orc_smooth_error(g.n, rp, ci, v, _f64(r), arr, len(hiers), C.byref(p), e)
    if st:
        raise RuntimeError(ERR.get(st))
    return e


def precond(g, r, hiers, params=None):
    """The preconditioner of Alg. 2's PCG for a history of len(hiers) hierarchies."""
    p = params if params is not None else default_params()
    rp, ci, v = _csr(g)
    arr = (C.c_void_p * len(hiers))(*[h._h for h in hiers])
    z = np.empty(g.n)
    lib().orc_precond(g.n, rp, ci, v, arr, len(hiers), C.byref(p), _f64(r), z)
    return z


def solve_multi(g, B, hiers, X0=None, params=None):
    """Several right-hand sides (the columns of B, n x k): each column's outer
    iteration of Alg. 5 without re-setup, preconditioned by the composite of
    V-cycles over hiers. Returns (X n x k, iters, rel_res, status)."""
    p = params if params is not None else default_params()
    rp, ci, v = _csr(g)
    Bc = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(g.n, -1).T)   # k x n: column-major
    k = Bc.shape[0]
    Xc = (np.zeros_like(Bc) if X0 is None else
          np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(g.n, k).T))
    arr = (C.c_void_p * len(hiers))(*[h._h for h in hiers])
    iters = np.zeros(k, np.int32)
    rel = np.zeros(k)
    st = lib().orc_solve_multi(g.n, rp, ci, v, k, Bc, Xc, C.byref(p), arr, len(hiers),
                               iters.ctypes.data_as(C.c_void_p), rel.ctypes.data_as(C.c_void_p))
    return Xc.T.copy(), iters, rel, ERR.get(st, st)


def solve(g, b, x0=None, params=None, e0=None, hist_cap=4096):
    """Alg. 5. Returns (x, stats dict, residual history). stats["rebuilt_after"]
    lists the steps k after whose V-cycle a re-setup ran."""
    p = params if params is not None else default_params()
    rp, ci, v = _csr(g)
    x = np.zeros(g.n) if x0 is None else _f64(x0).copy()
    st = Stats()
    hist = np.full(hist_cap, np.nan)
    reb = np.zeros(hist_cap, np.int32)
    ee = None if e0 is None else _f64(e0)
    lib().orc_solve(g.n, rp, ci, v, _f64(b), x, C.byref(p),
                    None if ee is None else ee.ctypes.data_as(C.c_void_p), C.byref(st),
                    hist.ctypes.data_as(C.c_void_p), hist_cap, reb.ctypes.data_as(C.c_void_p))
    s = dict(iters=st.iters, resetups=st.resetups, levels=st.levels, status=ERR.get(st.status, st.status),
             rel_res=st.rel_res, oc_mean=st.oc_mean, cycles=st.cycles, wcycles=st.wcycles,
             rebuilt_after=[int(k) for k in np.nonzero(reb[: st.iters + 1])[0]])
    return x, s, hist[: st.iters + 1]


def solve_zero_rhs(g, x0, params=None, e0=None, hist_cap=4096):
    """Alg. 6 (b = 0)."""
    p = params if params is not None else default_params(threshold=0.5)
    rp, ci, v = _csr(g)
    x = _f64(x0).copy()
    st = Stats()
    hist = np.full(hist_cap, np.nan)
    ee = None if e0 is None else _f64(e0)
    lib().orc_solve_zero_rhs(g.n, rp, ci, v, x, C.byref(p),
                             None if ee is None else ee.ctypes.data_as(C.c_void_p), C.byref(st),
                             hist.ctypes.data_as(C.c_void_p), hist_cap)
    s = dict(iters=st.iters, resetups=st.resetups, levels=st.levels, status=ERR.get(st.status, st.status),
             rel_res=st.rel_res, oc_mean=st.oc_mean, cycles=st.cycles)
    return x, s, hist[: st.iters + 1]
