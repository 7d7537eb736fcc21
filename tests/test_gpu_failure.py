"""Failure paths without a GPU fault: an injected allocation failure gives
EIG_ERR_NOMEM (solve and server request) and leaves the handle usable, and a
queued server request can be cancelled (status EIG_CANCELLED) while a running
one is left to finish.
"""
import numpy as np
import pytest

from paper_1011_3077_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    from paper_1011_3077_gb300 import build, eigdc
    build.build()
    yield eigdc, torch
    eigdc.eig_debug_fail_allocations(0)
    torch.cuda.synchronize()


def test_injected_allocation_failure_then_recovery(E):
    eigdc, torch = E
    A, lam = workloads.symmetric_uniform(120, seed=3)
    h = eigdc.Handle(0)
    eigdc.eig_debug_fail_allocations(1)
    rc, w, U, info = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=1))
    assert rc == eigdc.EIG_ERR_NOMEM
    assert "allocation" in h.last_error()
    rc, w, U, info = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=1))
    assert rc == eigdc.EIG_OK
    assert np.abs(np.sort(w) - lam).max() <= 1e-12
    h.close()


def _sym_request(torch, eigdc, srv, n, seed, params):
    A, _ = workloads.symmetric_uniform(n, seed=seed)
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    dA = eigdc.to_device(A)
    dw, dU = z(n), z(n, n)
    torch.cuda.synchronize()
    return srv.submit(eigdc.EIG_KIND_SYM, dA, dw, None, dU, params), A, dw


def test_server_request_with_injected_failure(E):
    eigdc, torch = E
    srv = eigdc.Server(0, 1, 60.0)
    params = eigdc.default_params(seed=2)
    eigdc.eig_debug_fail_allocations(1)
    t1, _, _ = _sym_request(torch, eigdc, srv, 200, 5, params)
    rc, st = srv.wait(t1, 300.0)
    assert rc == 0 and st == eigdc.EIG_ERR_NOMEM
    t2, A, dw = _sym_request(torch, eigdc, srv, 200, 6, params)
    rc, st = srv.wait(t2, 300.0)
    assert rc == 0 and st == eigdc.EIG_OK
    srv.close()


def test_cancel_queued_request(E):
    eigdc, torch = E
    srv = eigdc.Server(0, 1, 60.0)
    params = eigdc.default_params(seed=3)
    t_big, _, _ = _sym_request(torch, eigdc, srv, 1500, 7, params)   # holds the one worker
    queued = [_sym_request(torch, eigdc, srv, 100, 8 + i, params)[0] for i in range(3)]
    got = srv.cancel(queued[-1])
    rc, st = srv.wait(queued[-1], 300.0)
    assert rc == 0
    if got == 1:
        assert st == eigdc.EIG_CANCELLED
    else:
        assert got == 0 and st == eigdc.EIG_OK
    for t in [t_big] + queued[:-1]:
        rc, st = srv.wait(t, 600.0)
        assert rc == 0 and st == eigdc.EIG_OK
        assert srv.cancel(t) == 0          # finished: nothing to cancel
    assert eigdc.lib().eig_server_cancel(srv._s, 10 ** 9) == eigdc.EIG_ERR_ARG
    srv.close()
