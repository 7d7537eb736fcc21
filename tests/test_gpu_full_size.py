"""GPU checks at the benchmarked sizes, in the launch configuration bench.py
times, through the C-ABI.

The oracle cannot solve these sizes on the host in test time.  Each check is a
property that holds at any size: the construction prescribes the spectrum
(A = Q diag(lambda) Q^T with Haar Q), so the sorted eigenvalues must match
lambda within 1e-10 ||A||_2; U must be orthogonal, ||U^T U - I||_2 <= 1e-12
(power iteration on the symmetric residual); and the backward error
||A - U diag(w) U^T||_F / ||A||_F must stay <= 1e-12.  The whole-solve parity
with the oracle's tree and eigenvalues is checked at n = 1024 in
test_gpu_parity_large.py.

  * the symmetric semicircle workload at n = 8192 in EIG_FP64_TC, 8 node
    workers (the Sec. 3.4 recursion with median shifts, Algorithm 6);
  * the batched workload, 2000 symmetric problems with n log-uniform in
    [32, 512] and lambda ~ U[-1, 1], in one persistent fused launch.
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
    h = eigdc.Handle(0)
    yield eigdc, h, torch
    torch.cuda.synchronize()
    h.close()


def _orth_2norm(torch, U, iters=40):
    n = U.shape[0]
    R = U.t() @ U - torch.eye(n, dtype=U.dtype, device=U.device)
    v = torch.ones(n, dtype=U.dtype, device=U.device) / np.sqrt(n)
    est = 0.0
    for _ in range(iters):
        y = R @ v
        est = float(torch.linalg.norm(y))
        if est == 0.0:
            break
        v = y / est
    return est


def _check_sym(torch, dA0, w, dU, lam):
    """Prescribed spectrum, orthogonality and backward error on the device.
    dA0 and dU hold column-major matrices as torch (n, n) tensors (their
    transposes); A is symmetric, so the residual's norm is the same."""
    nA = float(np.max(np.abs(lam)))
    assert np.max(np.abs(np.sort(w) - lam)) <= 1e-10 * nA
    U = dU.t()
    assert _orth_2norm(torch, U) <= 1e-12
    A = dA0.t()
    res = A - (U * torch.from_numpy(w).to(U.device)) @ U.t()
    assert float(torch.linalg.norm(res)) <= 1e-12 * float(torch.linalg.norm(A))


def test_config3_symmetric_8192_fp64tc(E):
    eigdc, h, torch = E
    n = 8192
    A, lam = workloads.symmetric_semicircle(n, seed=3)
    dA0 = eigdc.to_device(A)
    del A
    dA = dA0.clone()
    dw = torch.zeros(n, dtype=torch.float64, device="cuda")
    dU = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    p = eigdc.default_params(seed=0, leaf_size=64, workers=8, prec=eigdc.EIG_FP64_TC)
    rc, info = eigdc.eig_solve(h, eigdc.EIG_KIND_SYM, n, dA, n, dw, None, dU, n, p)
    assert rc == eigdc.EIG_OK, h.last_error()
    # a binary recursion tree: every split adds two nodes and one leaf
    assert info.nodes == 2 * info.splits + 1 and info.leaves == info.splits + 1
    _check_sym(torch, dA0, dw.cpu().numpy(), dU, lam)


def test_config4_batched_2000_fused(E):
    eigdc, h, torch = E
    mats, lams = workloads.batched_symmetric(count=2000, seed=4)
    ns = [A.shape[0] for A in mats]
    dA0 = [eigdc.to_device(A) for A in mats]
    dAs = [a.clone() for a in dA0]
    dws = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    dUs = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for n in ns]
    p = eigdc.default_params(seed=0, leaf_size=64)
    rc, st, infos = eigdc.eig_solve_batched_fused(h, ns, dAs, ns, dws, dUs, ns, p)
    assert rc == eigdc.EIG_OK, h.last_error()
    assert all(s == eigdc.EIG_OK for s in st)
    for a0, w, U, lam in zip(dA0, dws, dUs, lams):
        _check_sym(torch, a0, w.cpu().numpy(), U, lam)
