"""Pins for the oracle's generator, Householder QR/RQ and split test."""
import os

import numpy as np
import pytest

from oracle import philox
from oracle.householder import house, qr_factor, qr_explicit, rq_explicit
from oracle.split import split_scores, split_test, choose_k
from tests.pinlib import cholesky_upper

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        ctr, key, want = vals[:4], vals[4:6], vals[6:10]
        got = philox.philox4x32_10(*[np.array([c]) for c in ctr], *key)
        assert [int(g[0]) for g in got] == want


def test_splitmix64_known_answer():
    for row in _rows("splitmix64_kat.txt"):
        assert philox.splitmix64(int(row[0], 16)) == int(row[1], 16)


def test_uniforms_range_and_exactness():
    u1, u2 = philox.uniform_pairs(100000, seed=123, purpose=4, stream=99)
    assert np.all(u1 > 0.0) and np.all(u1 < 1.0)
    assert np.all(u2 >= 0.0) and np.all(u2 < 1.0)
    # both are integer multiples of 2^-53
    assert np.all(np.floor(u1 * 2.0 ** 53) == u1 * 2.0 ** 53)
    assert np.all(np.floor(u2 * 2.0 ** 53) == u2 * 2.0 ** 53)
    assert abs(np.mean(u2) - 0.5) < 0.005


def test_gaussian_moments_and_streams():
    z = philox.gaussian_matrix(400, 500, seed=7, purpose=4, stream=5)
    assert z.shape == (400, 500)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05
    # column-major element order: element e = i + j*rows is pair e//2
    flat = z.T.reshape(-1)
    w = philox.gaussian_matrix(1, 400 * 500, seed=7, purpose=4, stream=5).reshape(-1)
    assert np.array_equal(flat, w)
    other = philox.gaussian_matrix(400, 500, seed=7, purpose=4, stream=6)
    assert abs(np.corrcoef(z.ravel(), other.ravel())[0, 1]) < 0.01
    att = philox.gaussian_matrix(400, 500, seed=7, purpose=4, stream=5, attempt=1)
    assert not np.array_equal(att, z)


def test_child_ids_distinct():
    seen = {philox.ROOT_NODE}
    frontier = [philox.ROOT_NODE]
    for _ in range(10):
        nxt = []
        for p in frontier:
            for side in (0, 1):
                c = philox.child_node(p, side)
                assert c not in seen
                seen.add(c)
                nxt.append(c)
        frontier = nxt


# ---------------------------------------------------------------- Householder

@pytest.mark.parametrize("x", [
    np.array([3.0, 4.0]), np.array([-3.0, 4.0, 1.0]), np.array([2.0, 0.0, 0.0]),
    np.array([-2.0, 0.0]), np.array([0.0, 0.0, 0.0]), np.array([1e-150, 1e-150]),
    np.array([0.0, -5.0, 2.0]),
])
def test_house_maps_to_positive_e1(x):
    v, beta, mu = house(x)
    P = np.eye(len(x)) - beta * np.outer(v, v)
    y = P @ x
    assert v[0] == 1.0
    assert mu >= 0.0
    assert np.allclose(y[0], np.linalg.norm(x), rtol=1e-14, atol=0)
    assert np.allclose(y[1:], 0.0, atol=1e-15 * max(1.0, np.linalg.norm(x)))
    assert np.allclose(P @ P.T, np.eye(len(x)), atol=1e-15)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (40, 40), (64, 17), (130, 65)])
def test_qr_identities(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    X = rng.standard_normal((m, n))
    Q, R = qr_explicit(X)
    assert np.allclose(Q @ R, X, atol=1e-13 * np.linalg.norm(X))
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-14 * max(n, 1))
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    # uniqueness: R is the Cholesky factor of X^T X
    Rc = cholesky_upper(X.T @ X)
    assert np.allclose(R, Rc, atol=1e-10 * np.linalg.norm(X))
    # Q^T X = [R; 0] through the reflectors directly
    f = qr_factor(X)
    QtX = f.qt_times(X)
    assert np.allclose(QtX[:n], R, atol=1e-13 * np.linalg.norm(X))
    assert np.allclose(QtX[n:], 0.0, atol=1e-13 * np.linalg.norm(X))
    # library QR with the same sign convention gives the same factors
    Ql, Rl = np.linalg.qr(X)
    s = np.sign(np.diag(Rl))
    s[s == 0] = 1
    assert np.allclose(Q, Ql * s, atol=1e-12)


def test_qr_full_q_orthogonal_and_rank_deficient():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30, 10))
    X[:, 4] = X[:, 1] * 2.0           # exact rank deficiency
    f = qr_factor(X)
    Qfull = f.q_times(np.eye(30))
    assert np.allclose(Qfull.T @ Qfull, np.eye(30), atol=1e-13)
    assert np.allclose(Qfull[:, :10] @ f.R, X, atol=1e-12)
    assert abs(f.R[4, 4]) < 1e-13


def test_rq_identity():
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 33):
        Y = rng.standard_normal((n, n))
        R, Q = rq_explicit(Y)
        assert np.allclose(R @ Q, Y, atol=1e-13 * max(1, n))
        assert np.allclose(Q @ Q.T, np.eye(n), atol=1e-13 * max(1, n))
        assert np.all(np.tril(R, -1) == 0.0)
        assert np.all(np.diag(R) >= 0.0)


# ---------------------------------------------------------------- split test

def _brute_scores(A):
    n = A.shape[0]
    return np.array([np.max(np.sum(np.abs(A[k:, :k]), axis=0)) for k in range(1, n)])


@pytest.mark.parametrize("n", [2, 3, 9, 40])
def test_split_scores_brute_force(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    assert np.allclose(split_scores(A), _brute_scores(A), rtol=1e-14, atol=0)


def test_split_finds_block_triangular_k():
    rng = np.random.default_rng(2)
    n, k = 30, 11
    A = rng.standard_normal((n, n))
    A[k:, :k] = 0.0
    kk, e, _ = split_test(A)
    assert kk == k and e == 0.0


def test_split_tie_breaks():
    # all-zero scores: closest to n/2, then smaller
    assert choose_k(np.zeros(9), 10) == 5
    assert choose_k(np.zeros(8), 9) == 4
    assert choose_k(np.array([3.0, 1.0, 1.0, 2.0]), 5) == 2
    D = np.diag(np.arange(1.0, 8.0))
    assert split_test(D)[0] == 3


def test_split_pencil_sum():
    rng = np.random.default_rng(5)
    n = 12
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    k, e, es = split_test(A, B)
    nA = np.max(np.sum(np.abs(A), 0))
    nB = np.max(np.sum(np.abs(B), 0))
    want = _brute_scores(A) / nA + _brute_scores(B) / nB
    assert np.allclose(es, want, rtol=1e-14)
    assert k == int(np.argmin(want)) + 1
