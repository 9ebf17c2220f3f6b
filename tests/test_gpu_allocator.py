"""Device memory through the caller's allocator (pcamg_set_allocator): every
buffer of a handle and of a network comes from the installed callbacks and is
returned through them; the results do not depend on where the memory came from."""
import ctypes as C

import numpy as np
import pytest

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


def test_every_buffer_goes_through_the_callbacks(P):
    import torch
    P.use_allocator("torch")
    g = I.workload("C2-small")
    b = I.rhs_normal(g.n, 3)
    a0, f0 = P.allocator_calls()
    s = P.Solver(g, params=P.default_params(precision=1))
    x_t, st = s.solve(b)
    x_t = x_t.cpu().numpy()
    a1, f1 = P.allocator_calls()
    assert a1 - a0 > 50          # hierarchies, work vectors, setup scratch
    s.close()
    torch.cuda.synchronize()
    a2, f2 = P.allocator_calls()
    assert a2 - a0 == f2 - f0    # everything allocated was returned
    # the same solve from the library's own pool gives the same bits
    P.use_allocator("library")
    try:
        s = P.Solver(g, params=P.default_params(precision=1))
        x_l, st_l = s.solve(b)
        s.close()
        a3, _ = P.allocator_calls()
        assert a3 == a2          # no callback while the library pool is in use
    finally:
        P.use_allocator("torch")
    assert st["iters"] == st_l["iters"] and st["resetups"] == st_l["resetups"]
    assert np.array_equal(x_t, x_l.cpu().numpy())


def test_network_memory_through_the_callbacks(P):
    import torch
    P.use_allocator("torch")
    a0, f0 = P.allocator_calls()
    net = P.Mpnn(seed=1)
    a1, _ = P.allocator_calls()
    assert a1 - a0 >= 6          # weights, Adam moments, gradient, rounded copies
    net.close()
    torch.cuda.synchronize()
    a2, f2 = P.allocator_calls()
    assert a2 - a0 == f2 - f0


def test_half_an_allocator_is_rejected(P):
    from paper_1806_07028_gb300 import native as N
    fn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)(lambda n, s, c: None)
    assert N.lib().pcamg_set_allocator(C.cast(fn, C.c_void_p), None, None) == N.ERR_INVALID


def test_failed_allocation_is_an_oom_status(P):
    # an allocator that refuses: the handle is not created and the status says why
    from paper_1806_07028_gb300 import native as N
    refuse = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)(lambda n, s, c: None)
    nofree = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)(lambda p, s, c: None)
    L = N.lib()
    assert L.pcamg_set_allocator(C.cast(refuse, C.c_void_p), C.cast(nofree, C.c_void_p), None) == N.OK
    try:
        g = I.grid2d(16, 16)
        with pytest.raises(N.PCAMGError) as ei:
            P.Solver(g)
        assert ei.value.status == N.ERR_OOM
    finally:
        import paper_1806_07028_gb300.solver as S
        S._allocator["kind"] = None
        P.use_allocator("torch")
