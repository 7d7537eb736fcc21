"""GPU parity of the fused batched symmetric solver (eig_solve_batched_fused):
one persistent launch, every problem's whole recursion inside one CTA.

Each problem must take the oracle's recursion tree (equal split, node and
failed-attempt counts: the Philox draws, node ids and decisions are shared)
and meet the FP64 targets of the whole-solve parity tests: eigenvalues within
1e-12 ||A|| of the oracle's and within 1e-10 ||A|| of the prescribed spectrum,
||U^T U - I||_2 <= 1e-12, ||A - U L U^T||_F / ||A||_F <= 1e-12.  Against the
host-driven eig_solve_batched the trees are equal and the eigenvalues agree
to 1e-12 ||A|| (the two paths block their products differently).  The same
kernel finishes the small nodes of eig_solve (fused_tail), continuing each
node's id, interval and depth: the tree must not change.
"""
import numpy as np
import pytest

from oracle.solve import eig_sym as oeig_sym
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


def _fused(eigdc, torch, h, mats, params):
    ns = [A.shape[0] for A in mats]
    dAs = [eigdc.to_device(A) for A in mats]
    dws = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    dUs = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for n in ns]
    rc, st, infos = eigdc.eig_solve_batched_fused(h, ns, dAs, ns, dws, dUs, ns, params)
    return rc, st, infos, [w.cpu().numpy() for w in dws], [eigdc.to_host(U) for U in dUs]


def _targets(A, w, U, lam):
    n = A.shape[0]
    nA = max(np.max(np.abs(lam)), 1e-300)
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert np.linalg.norm(U.T @ U - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(A - (U * w) @ U.T) <= 1e-12 * max(np.linalg.norm(A), 1e-300)


@pytest.mark.parametrize("leaf", [64, 32])
def test_fused_matches_oracle(E, leaf):
    eigdc, h, torch = E
    sizes = [1, 2, 7, 64, 65, 100, 150, 201] if leaf == 64 else [33, 97, 150]
    cases = [workloads.symmetric_uniform(n, seed=n + leaf) for n in sizes]
    p = eigdc.default_params(seed=5, leaf_size=leaf)
    rc, st, infos, ws, Us = _fused(eigdc, torch, h, [A for A, _ in cases], p)
    assert rc == eigdc.EIG_OK and st == [0] * len(sizes), h.last_error()
    for (A, lam), w, U, inf in zip(cases, ws, Us, infos):
        _targets(A, w, U, lam)
        wo, Uo, io = oeig_sym(A, seed=5, leaf_size=leaf)
        assert io.status == 0
        assert (inf.splits, inf.nodes, inf.failed_attempts) == (io.splits, io.nodes,
                                                                io.failed_attempts)
        assert np.max(np.abs(w - wo)) <= 1e-12 * max(np.max(np.abs(lam)), 1e-300)


def test_fused_matches_host_batched_on_the_batched_workload(E):
    """A slice of the batched workload (n log-uniform in [32, 512], lambda ~
    U[-1, 1]) through both batched paths; repeated fused calls are bit-identical."""
    eigdc, h, torch = E
    mats, lams = workloads.batched_symmetric(count=16, seed=4)
    p = eigdc.default_params(seed=0, leaf_size=64, workers=8)
    rc, st, infos, ws, Us = _fused(eigdc, torch, h, mats, p)
    assert rc == eigdc.EIG_OK and all(s == 0 for s in st), h.last_error()
    ns = [A.shape[0] for A in mats]
    dAs = [eigdc.to_device(A) for A in mats]
    dws = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    dUs = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for n in ns]
    rc2, st2, inf2 = eigdc.eig_solve_batched(h, eigdc.EIG_KIND_SYM, ns, dAs, ns, dws, None, dUs,
                                             ns, p)
    assert rc2 == eigdc.EIG_OK and all(s == 0 for s in st2)
    for A, lam, w, U, a, b, w2 in zip(mats, lams, ws, Us, infos, inf2, dws):
        _targets(A, w, U, lam)
        assert (a.splits, a.nodes, a.failed_attempts) == (b.splits, b.nodes, b.failed_attempts)
        assert np.max(np.abs(w - w2.cpu().numpy())) <= 1e-12 * np.max(np.abs(lam))
    rc3, st3, inf3, ws3, Us3 = _fused(eigdc, torch, h, mats, p)
    assert rc3 == eigdc.EIG_OK
    for w, U, w3, U3 in zip(ws, Us, ws3, Us3):
        assert np.array_equal(w, w3) and np.array_equal(U, U3)


def test_fused_errors_and_edge_cases(E):
    eigdc, h, torch = E
    p = eigdc.default_params(seed=1)
    rc, st, _, _, _ = _fused(eigdc, torch, h, [np.eye(513)], p)
    assert rc == eigdc.EIG_ERR_ARG and "512" in h.last_error()
    bad = np.eye(80)
    bad[3, 5] = np.nan
    good, lam = workloads.symmetric_uniform(90, seed=2)
    rc, st, infos, ws, Us = _fused(eigdc, torch, h, [bad, good, np.zeros((70, 70)),
                                                     2.5 * np.eye(100)], p)
    assert rc == eigdc.EIG_OK
    assert st[0] == eigdc.EIG_NONFINITE and st[1] == eigdc.EIG_OK
    _targets(good, ws[1], Us[1], lam)
    assert st[2] in (eigdc.EIG_OK, eigdc.EIG_NO_SPLIT) and st[3] in (eigdc.EIG_OK, eigdc.EIG_NO_SPLIT)
    rc, st, _, _, _ = _fused(eigdc, torch, h, [], p)
    assert rc == eigdc.EIG_OK and st == []


def test_fused_autotune_then_solve(E):
    eigdc, h, torch = E
    rc, best, cands = eigdc.eig_fused_autotune(h, 40, 32, 256, seed=3)
    assert rc == eigdc.EIG_OK, h.last_error()
    assert 2 <= len(cands) <= 6 and all(ms > 0 for _, _, ms in cands)
    assert best[2] == min(ms for _, _, ms in cands) and best[0] in (16, 32)
    mats, lams = workloads.batched_symmetric(count=6, seed=9, nmax=300)
    rc, st, infos, ws, Us = _fused(eigdc, torch, h, mats, eigdc.default_params(seed=2))
    assert rc == eigdc.EIG_OK and all(s == 0 for s in st)
    for A, lam, w, U in zip(mats, lams, ws, Us):
        _targets(A, w, U, lam)


@pytest.mark.parametrize("n,tail,prec", [(300, 128, 0), (700, 200, 0), (700, 160, 2)])
def test_fused_tail_takes_the_same_tree(E, n, tail, prec):
    """eig_solve with fused_tail: the nodes of at most `tail` rows finish in one
    launch of the fused solver, continuing their node ids and intervals.  The
    recursion must be the one without the tail (and, at n = 300, the
    oracle's): equal split, node and failed-attempt counts and depth;
    eigenvalues within 1e-12 ||A|| of the tail-free solve; FP64 targets."""
    eigdc, h, torch = E
    A, lam = workloads.symmetric_semicircle(n, seed=n + tail)
    out = {}
    for t in (0, tail):
        p = eigdc.default_params(seed=4, prec=prec, fused_tail=t)
        rc, w, U, info = eigdc.solve_symmetric(h, A, p)
        assert rc == eigdc.EIG_OK, h.last_error()
        _targets(A, w, U, lam)
        out[t] = (w, info)
    (w0, i0), (w1, i1) = out[0], out[tail]
    key = lambda i: (i.splits, i.nodes, i.failed_attempts, i.max_depth, i.leaves)
    assert key(i1) == key(i0)
    assert np.max(np.abs(w1 - w0)) <= 1e-12 * np.max(np.abs(lam))
    if n <= 300:
        wo, Uo, io = oeig_sym(A, seed=4)
        assert (i1.splits, i1.nodes, i1.failed_attempts) == (io.splits, io.nodes,
                                                             io.failed_attempts)
        assert np.max(np.abs(w1 - wo)) <= 1e-12 * np.max(np.abs(lam))


def test_fused_tail_argument_check(E):
    eigdc, h, torch = E
    A, lam = workloads.symmetric_uniform(100, seed=1)
    rc, w, U, info = eigdc.solve_symmetric(h, A, eigdc.default_params(fused_tail=-1))
    assert rc == eigdc.EIG_ERR_ARG
    # a tail at or below the leaf size has no node to take: the plain solve
    rc, w, U, info = eigdc.solve_symmetric(h, A, eigdc.default_params(fused_tail=64))
    assert rc == eigdc.EIG_OK
    _targets(A, w, U, lam)
