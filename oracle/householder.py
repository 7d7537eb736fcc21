"""Householder QR with explicit Q, and RQ by index reversal (oracle side).

The paper uses QR, RQ, QL and LQ as black-box routines with explicit
orthogonal factors (Sec. 3 intro; Sec. 4.2.1 notes that the orthogonal factor
can be formed explicitly at a constant-factor extra cost and that RQ, QL and LQ
have identical cost).  It fixes no sign convention.  Reading used throughout
this project: every factorization returns a triangular factor with a
non-negative diagonal, which makes QR of a full-column-rank matrix unique
(R is then the Cholesky factor of X^T X).

The reflector of a vector x is the textbook one that maps x to +||x|| e1
(Golub and Van Loan, Matrix Computations, Sec. 5.1: the first component of v
is chosen by the cancellation-free formula -sigma / (x1 + mu) when x1 > 0):
    P = I - beta v v^T,  v[0] = 1,  P x = mu e1,  mu = ||x||_2 >= 0.

Unblocked, one column at a time, no reordering.  Pinned by
tests/test_oracle_basics.py: Q R = X, Q^T Q = I, triangularity, R equal
to the Cholesky factor of X^T X computed by an independent textbook Cholesky,
and the RQ identity Y = R Q.
"""
import numpy as np


def house(x):
    """Return (v, beta, mu) with (I - beta v v^T) x = mu e1, v[0] = 1, mu >= 0."""
    x = np.asarray(x, dtype=np.float64)
    v = x.copy()
    v[0] = 1.0
    sigma = float(x[1:] @ x[1:]) if x.shape[0] > 1 else 0.0
    x0 = float(x[0])
    if sigma == 0.0:
        if x0 >= 0.0:
            return v, 0.0, x0
        # x = x0 e1 with x0 < 0: reflect through e1^perp
        return v, 2.0, -x0
    mu = np.sqrt(x0 * x0 + sigma)
    if x0 <= 0.0:
        v0 = x0 - mu
    else:
        v0 = -sigma / (x0 + mu)
    beta = 2.0 * v0 * v0 / (sigma + v0 * v0)
    v = x / v0
    v[0] = 1.0
    return v, float(beta), float(mu)


class QRFactors:
    """Householder vectors, scalars and R of X = Q R (X is m x n, m >= n)."""

    def __init__(self, vs, betas, R, m):
        self.vs = vs          # vs[j] has length m - j, vs[j][0] = 1
        self.betas = betas
        self.R = R            # n x n upper triangular, diag >= 0
        self.m = m

    def q_times(self, E):
        """Q E for an m x c matrix E: apply H_0 H_1 ... H_{n-1} (last one first)."""
        Y = np.array(E, dtype=np.float64, copy=True)
        for j in range(len(self.vs) - 1, -1, -1):
            v, beta = self.vs[j], self.betas[j]
            if beta == 0.0:
                continue
            Y[j:, :] -= beta * np.outer(v, v @ Y[j:, :])
        return Y

    def qt_times(self, E):
        """Q^T E: apply H_{n-1} ... H_0 (first one first)."""
        Y = np.array(E, dtype=np.float64, copy=True)
        for j in range(len(self.vs)):
            v, beta = self.vs[j], self.betas[j]
            if beta == 0.0:
                continue
            Y[j:, :] -= beta * np.outer(v, v @ Y[j:, :])
        return Y


def qr_factor(X):
    """Householder QR of X (m x n, m >= n), one column at a time."""
    W = np.array(X, dtype=np.float64, copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("qr_factor needs m >= n")
    vs, betas = [], []
    R = np.zeros((n, n))
    for j in range(n):
        v, beta, mu = house(W[j:, j])
        if beta != 0.0 and j + 1 < n:
            W[j:, j + 1:] -= beta * np.outer(v, v @ W[j:, j + 1:])
        W[j, j] = mu
        W[j + 1:, j] = 0.0
        vs.append(v)
        betas.append(beta)
        R[j, j:] = W[j, j:]
    return QRFactors(vs, betas, R, m)


def qr_explicit(X):
    """(Q, R) with Q m x n having orthonormal columns, X = Q R, diag(R) >= 0."""
    f = qr_factor(X)
    m, n = np.asarray(X).shape
    E = np.zeros((m, n))
    E[:n, :n] = np.eye(n)
    return f.q_times(E), f.R


def rq_explicit(Y):
    """(R, Q) with Y = R Q for square Y, R upper triangular with diag >= 0.

    Index reversal J: QR of Z = (J Y)^T = Z~ R~ gives
        Y = (J R~^T J)(J Q~^T),
    where J R~^T J is upper triangular with the diagonal of R~ reversed.
    """
    Y = np.asarray(Y, dtype=np.float64)
    Z = Y[::-1, :].T
    Qt, Rt = qr_explicit(Z)
    R = Rt.T[::-1, ::-1].copy()
    Q = Qt.T[::-1, :].copy()
    return R, Q
