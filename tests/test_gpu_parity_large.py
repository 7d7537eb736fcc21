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


def _eig_condition(T):
    """kappa_i = ||y_i|| ||x_i|| / |y_i^T x_i| of the triangular T from the
    oracle's eigenvector recurrence (right vectors of T, left vectors as the
    right vectors of the reversed transpose, which is again upper triangular)."""
    n = T.shape[0]
    X = otrevc.triangular_eigenvectors(T)
    J = np.arange(n)[::-1]
    Yr = otrevc.triangular_eigenvectors(T.T[J][:, J])
    Y = Yr[J][:, J]
    num = np.linalg.norm(X, axis=0) * np.linalg.norm(Y, axis=0)
    return num / np.abs(np.sum(Y * X, axis=0))


def _nonsym_case():
    if "nonsym" not in _cache:
        # strict-upper scale 0.1/sqrt(n): at 1/sqrt(n) the oracle itself stops
        # with NO_SPLIT at n = 1024 (13 splits, then a node whose
        # pseudospectrum reaches every line tried)
        A, d, T0 = workloads.nonsymmetric_schur(N, seed=2, offdiag_scale=0.1 / np.sqrt(N))
        To, Qo, wro, wio, io = oschur(A, seed=2)
        assert io.status == 0
        _cache["nonsym"] = (A, d, T0, wro, io, _eig_condition(T0))
    return _cache["nonsym"]


@pytest.mark.parametrize("prec", [0, 2])
def test_nonsymmetric_n1024_matches_oracle(E, prec):
    eigdc, h, torch = E
    A, d, T0, wro, io, kappa = _nonsym_case()
    rc, T, Us, wr, wi, info = eigdc.schur_nonsymmetric(h, A, eigdc.default_params(seed=2, prec=prec))
    assert rc == eigdc.EIG_OK, h.last_error()
    assert (info.splits, info.nodes, info.failed_attempts) == (io.splits, io.nodes,
                                                               io.failed_attempts)
    assert np.all(wi == 0.0)
    nA = np.linalg.norm(A, 2)
    order = np.argsort(d)
    tol = 1e-13 * N * kappa[order] * nA + 1e-12
    assert np.all(np.abs(np.sort(wr) - d[order]) <= tol)
    assert np.all(np.abs(np.sort(wr) - np.sort(wro)) <= 2 * tol)
    assert _orth2(Us) <= 1e-12
    assert np.linalg.norm(A - Us @ T @ Us.T) <= 1e-12 * np.linalg.norm(A)
