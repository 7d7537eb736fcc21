"""Node-parallel and batched execution (GPU).

The recursion's nodes and independent problems run on host workers with their
own CUDA streams.  Every node's arithmetic depends only on its own data and
its path-based Philox stream, so results must not depend on the schedule:
bitwise equal between 1 and 8 workers, and between a batched call and
separate calls.
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


def test_parallel_recursion_is_schedule_independent_sym(E):
    eigdc, h, torch = E
    A, lam = workloads.symmetric_uniform(420, seed=11)
    r1 = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=4, workers=1, leaf_size=48))
    r8 = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=4, workers=8, leaf_size=48))
    assert r1[0] == r8[0] == eigdc.EIG_OK
    assert np.array_equal(r1[1], r8[1]) and np.array_equal(r1[2], r8[2])
    assert r1[3].splits == r8[3].splits and r1[3].total_iters == r8[3].total_iters
    assert np.max(np.abs(r8[1] - lam)) <= 1e-10


def test_parallel_recursion_is_schedule_independent_nonsym(E):
    eigdc, h, torch = E
    A, d, _ = workloads.nonsymmetric_schur(300, seed=5, offdiag_scale=0.1 / np.sqrt(300))
    a = eigdc.schur_nonsymmetric(h, A, eigdc.default_params(seed=2, workers=1, leaf_size=40))
    b = eigdc.schur_nonsymmetric(h, A, eigdc.default_params(seed=2, workers=8, leaf_size=40))
    assert a[0] == b[0] == eigdc.EIG_OK
    for x, y in zip(a[1:5], b[1:5]):
        assert np.array_equal(x, y)
    assert np.linalg.norm(A - b[2] @ b[1] @ b[2].T) / np.linalg.norm(A) <= 1e-12


def test_batched_equals_separate_calls(E):
    eigdc, h, torch = E
    mats, spectra = workloads.batched_symmetric(count=24, seed=9, nmin=8, nmax=220)
    p = eigdc.default_params(seed=3, workers=6)
    dAs = [eigdc.to_device(A) for A in mats]
    dws = [torch.zeros(A.shape[0], dtype=torch.float64, device="cuda") for A in mats]
    dUs = [torch.zeros(A.shape, dtype=torch.float64, device="cuda") for A in mats]
    ns = [A.shape[0] for A in mats]
    rc, st, infos = eigdc.eig_solve_batched(h, eigdc.EIG_KIND_SYM, ns, dAs, ns, dws, None, dUs, ns, p)
    assert rc == eigdc.EIG_OK and all(x == 0 for x in st)
    for A, lam, dw, dU in zip(mats, spectra, dws, dUs):
        rc1, w1, U1, _ = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=3, workers=1))
        w = dw.cpu().numpy()
        U = eigdc.to_host(dU)
        assert np.array_equal(w, w1) and np.array_equal(U, U1)
        n = A.shape[0]
        assert np.max(np.abs(w - lam)) <= 1e-10
        assert np.linalg.norm(A - (U * w) @ U.T) <= 1e-12 * np.linalg.norm(A)


def test_batched_nonsymmetric_and_errors(E):
    eigdc, h, torch = E
    probs = [workloads.nonsymmetric_schur(n, seed=n, offdiag_scale=0.1 / np.sqrt(n))[0]
             for n in (70, 130, 33)]
    bad = np.eye(40)
    bad[1, 2] = np.inf
    probs.append(bad)
    ns = [A.shape[0] for A in probs]
    dAs = [eigdc.to_device(A) for A in probs]
    dwr = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    dwi = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    dUs = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for n in ns]
    rc, st, infos = eigdc.eig_solve_batched(h, eigdc.EIG_KIND_NONSYM, ns, dAs, ns, dwr, dwi, dUs,
                                            ns, eigdc.default_params(seed=1, workers=3))
    assert rc == eigdc.EIG_OK
    assert st[:3] == [0, 0, 0] and st[3] == eigdc.EIG_NONFINITE
    for A, dA, dU in zip(probs[:3], dAs, dUs):
        T, U = eigdc.to_host(dA), eigdc.to_host(dU)
        assert np.linalg.norm(A - U @ T @ U.T) / np.linalg.norm(A) <= 1e-12
