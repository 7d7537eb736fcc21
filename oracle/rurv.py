"""Haar matrix, RURV (Algorithm 1) and GRURV (Algorithm 2), oracle side.

Algorithm 1 (RURV): draw B with i.i.d. N(0,1) entries, [V, R^] = QR(B),
A^ = A V^H, [U, R] = QR(A^); then A = U R V.  Sec. 2 states that the Q factor
of a Gaussian matrix is Haar distributed; that holds with the Q factor whose
R has a non-negative diagonal (the convention of householder.py), so no
further sign fix is needed.

Algorithm 2 (GRURV) for k = 2 and exponents (m1, m2):
  m2 = +1: [U, R2, V] = RURV(A2);  m2 = -1: [U, L2, V] = RULV(A2^H), R2 = L2^H
  then for i = 1: m1 = +1: [U, R1] = QR(A1 U_cur), U_cur = U
                  m1 = -1: [U, R1] = RQ(U_cur^H A1), U_cur = U^H
and M = A1^{m1} A2^{m2} = U_cur R1^{m1} R2^{m2} V (the Lemma after Algorithm 2).
The splitter of Algorithms 4-6 is GRURV(2, A_p + B_p, A_p, -1, +1): its U_cur
spans, in its leading columns, the range of (A_p + B_p)^{-1} A_p, which tends
to the projector onto the deflating subspace outside the unit circle (Sec. 3.2).

RULV (QL-based) is used for the left deflating subspace of pencils
(Algorithm 4, line 4): QL of X is obtained from QR of X with reversed
columns: X J = Q~ R~  gives  X = (Q~ J)(J R~ J), J R~ J lower triangular.

Pinned by tests/test_oracle_method.py: the GRURV lemma identity with inverses
done by long-double Gaussian elimination, the subspace of U_cur against the
exact projector of a small diagonalisable pencil, and Haar moments.
"""
import numpy as np

from .householder import qr_explicit, rq_explicit
from .philox import gaussian_matrix, PURPOSE_HAAR


def haar(n, seed, stream, attempt=0, purpose=PURPOSE_HAAR):
    """n x n Haar orthogonal V from the Philox Gaussian draw of this stream."""
    G = gaussian_matrix(n, n, seed, purpose, stream, attempt)
    V, _ = qr_explicit(G)
    return V


def rurv(A, V):
    """Algorithm 1 with a given Haar V: returns (U, R) with A = U R V."""
    U, R = qr_explicit(np.asarray(A) @ V.T)
    return U, R


def ql_explicit(X):
    """(Q, L) with X = Q L, L lower triangular with non-negative diagonal."""
    X = np.asarray(X, dtype=np.float64)
    Qt, Rt = qr_explicit(X[:, ::-1])
    return Qt[:, ::-1].copy(), Rt[::-1, ::-1].copy()


def rulv(A, V):
    """RURV with QL: A V^T = U L; returns (U, L) with A = U L V."""
    return ql_explicit(np.asarray(A) @ V.T)


def grurv2(A1, A2, m1, m2, V):
    """GRURV(2; A1, A2; m1, m2) with the Haar matrix V given.

    Returns (U_cur, R1, R2) with A1^{m1} A2^{m2} = U_cur R1^{m1} R2^{m2} V.
    """
    if m2 == 1:
        U, R2 = rurv(A2, V)
    else:
        U, L2 = rulv(np.asarray(A2).T, V)
        R2 = L2.T
    U_cur = U
    if m1 == 1:
        U, R1 = qr_explicit(np.asarray(A1) @ U_cur)
        U_cur = U
    else:
        R1, Q = rq_explicit(U_cur.T @ np.asarray(A1))
        U_cur = Q.T
    return U_cur, R1, R2


def splitter_right(Ap, Bp, V):
    """Q_R = GRURV(2, A_p + B_p, A_p, -1, +1) (Algorithms 4-6, line 2)."""
    U_cur, R1, R2 = grurv2(Ap + Bp, Ap, -1, 1, V)
    return U_cur, R1, R2


def splitter_left(Ap, Bp, V):
    """Q_L = GRURV(2, A_p^H, (A_p + B_p)^H, +1, -1) (Algorithm 4, line 4)."""
    U_cur, R1, R2 = grurv2(Ap.T, (Ap + Bp).T, 1, -1, V)
    return U_cur, R1, R2


def numerical_rank(R2, R1, rel_tol=1e-8):
    """RURV rank decision: #{|R2_ii| > rel_tol * max_i |R1_ii|}.

    R2 is the triangular factor of RURV(A_p) and R1 that of the RQ step on
    A_p + B_p.  The splitter's matrix is (A_p + B_p)^{-1} A_p (Sec. 3.2), so
    A_p's singular values are measured against the size of A_p + B_p, of which
    max |R1_ii| is the scale (reading; the paper leaves the rank decision
    implicit).  A_p negligible next to B_p (every eigenvalue inside) gives 0.
    """
    d2 = np.abs(np.diag(R2))
    scale = float(np.max(np.abs(np.diag(R1)))) if R1.size else 0.0
    if d2.size == 0 or scale == 0.0:
        return 0
    return int(np.sum(d2 > rel_tol * scale))
