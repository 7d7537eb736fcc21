"""GPU parity of whole solves at n = 1024 against the oracle (slow: the
oracle's unblocked FP64 solve at this size takes a few minutes of host time,
computed once per module and shared by the precision forms).

Symmetric: the semicircle construction of the full-recursion workload
(lambda = sqrt(u1) cos(2 pi u2) on [-1, 1], Q Haar, median-shift recursion,
Sec. 3.4 and Algorithm 6).  Nonsymmetric: the triangular construction of the
real Schur workload (diagonal half |z| in [0.2, 0.9], half in [1.1, 3], random
signs; strict upper part N(0, (c/sqrt(n))^2)), unit-circle root split then
real Moebius lines (Sec. 3.3).

Checks, in the plain FP64 path and in the FP64-accurate tensor-core form:
  * the recursion takes the oracle's tree: equal split, node and
    failed-attempt counts (Philox draws are shared, and every decision is a
    comparison of well-separated FP64 scores);
  * sorted eigenvalues agree elementwise with the oracle's within
    1e-10 ||A||_2 (symmetric), and within the first-order bound
    1e-13 n kappa_i ||A||_2 of each eigenvalue's condition number kappa_i
    (nonsymmetric; both sides are backward stable);
  * ||U^T U - I||_2 <= 1e-12 and ||A - U T U^T||_F / ||A||_F <= 1e-12.
"""
import numpy as np
import pytest

from oracle.solve import eig_sym as oeig_sym, schur_nonsym as oschur
from oracle import trevc as otrevc
from paper_1011_3077_gb300 import workloads

pytestmark = pytest.mark.gpu

N = 1024
_cache = {}


@pytest.fixture(scope="module")
def E():
    import torch
    from paper_1011_3077_gb300 import build, eigdc
    build.build()
    h = eigdc.Handle(0)
    yield eigdc, h, torch
    torch.cuda.synchronize()
    h.close()


def _sym_case():
    if "sym" not in _cache:
        A, lam = workloads.symmetric_semicircle(N, seed=3)
        wo, Uo, io = oeig_sym(A, seed=5)
        assert io.status == 0
        _cache["sym"] = (A, lam, wo, io)
    return _cache["sym"]


def _orth2(U):
    return np.linalg.norm(U.T @ U - np.eye(U.shape[0]), 2)


@pytest.mark.parametrize("prec", [0, 2])
def test_symmetric_semicircle_n1024_matches_oracle(E, prec):
    eigdc, h, torch = E
    A, lam, wo, io = _sym_case()
    rc, w, Uv, info = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=5, prec=prec))
    assert rc == eigdc.EIG_OK, h.last_error()
    assert (info.splits, info.nodes, info.failed_attempts) == (io.splits, io.nodes,
                                                               io.failed_attempts)
    nA = np.max(np.abs(lam))
    assert np.max(np.abs(w - wo)) <= 1e-10 * nA
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert _orth2(Uv) <= 1e-12
    assert np.linalg.norm(A - (Uv * w) @ Uv.T) <= 1e-12 * np.linalg.norm(A)
