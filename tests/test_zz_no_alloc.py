"""The allocation-free residual entry point, for callers that cannot allocate
device memory (allocation-free hot loops, memory fully owned by a pool). It
must give the same r and ||r||^2 as the ordinary entry point and as the CPU
oracle, including on a second call that reuses its fixed scratch array.

This file is collected last on purpose, and also runs alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1806_07028_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1806_07028_gb300.build import build
    build()
    from paper_1806_07028_gb300 import native as N
    return N


def _p(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("name", ["C1", "C4-small", "C2-small"])
def test_noalloc_residual_matches_allocating_entry_point(lib, name):
    import torch
    N = lib
    g = I.workload(name)
    dev = torch.device("cuda:0")
    rp = torch.as_tensor(g.rowptr, device=dev)
    ci = torch.as_tensor(g.col, device=dev)
    va = torch.as_tensor(g.val, device=dev)
    rowabs = np.abs(g.to_scipy())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):          # two calls in a row share the fixed scratch
        rng = np.random.default_rng(10 + call)
        x = torch.as_tensor(rng.standard_normal(g.n), device=dev)
        b = torch.as_tensor(rng.standard_normal(g.n), device=dev)
        r_ref = torch.empty(g.n, dtype=torch.float64, device=dev)
        n_ref = torch.zeros(1, dtype=torch.float64, device=dev)
        N.check(N.lib().pcamg_residual(g.n, _p(rp), _p(ci), _p(va), _p(x), _p(b), _p(r_ref),
                                       _p(n_ref), stream))
        r = torch.full((g.n,), np.nan, dtype=torch.float64, device=dev)
        nr = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        N.check(N.lib().pcamg_residual_noalloc(g.n, _p(rp), _p(ci), _p(va), _p(x), _p(b), _p(r),
                                               _p(nr), stream))
        torch.cuda.synchronize()
        tol = 32 * EPS * (rowabs @ np.abs(x.cpu().numpy()) + np.abs(b.cpu().numpy()))
        assert np.all(np.abs(r.cpu().numpy() - r_ref.cpu().numpy()) <= tol)
        assert abs(nr.item() - n_ref.item()) <= 1e-12 * n_ref.item()
        ro = O.residual(g, x.cpu().numpy(), b.cpu().numpy())     # the oracle's r = b - A x
        assert np.all(np.abs(r.cpu().numpy() - ro) <= tol)
        assert abs(nr.item() - ro @ ro) <= 1e-12 * (ro @ ro)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    N = lib
    one = C.c_void_p(1)   # never dereferenced: the size check comes first
    st = N.lib().pcamg_residual_noalloc(67_108_865, one, one, one, one, one, one, one, None)
    assert st == N.ERR_INVALID          # null d_norm2 is rejected first
    st = N.lib().pcamg_residual_noalloc(67_108_865, one, one, one, one, one, one, one, one)
    assert st == N.ERR_INVALID
    assert b"67,108,864" in N.lib().pcamg_last_error(None)
