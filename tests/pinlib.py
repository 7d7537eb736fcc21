"""Independent reference routines used only to pin the oracle in tests.

These are different algorithms from the ones the oracle implements, so that a
mistake in the oracle cannot be repeated here: a textbook Cholesky
factorization, Gaussian elimination with partial pivoting in long double,
closed forms for 2x2 / 3x3 symmetric eigenvalues.
"""
import numpy as np


def cholesky_upper(M):
    """Upper-triangular R with R^T R = M (textbook inner-product Cholesky)."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    R = np.zeros((n, n))
    for j in range(n):
        s = M[j, j] - R[:j, j] @ R[:j, j]
        R[j, j] = np.sqrt(s)
        for k in range(j + 1, n):
            R[j, k] = (M[j, k] - R[:j, j] @ R[:j, k]) / R[j, j]
    return R


def ld_solve(A, B):
    """A^{-1} B by Gaussian elimination with partial pivoting in long double."""
    A = np.array(A, dtype=np.longdouble)
    B = np.array(B, dtype=np.longdouble)
    if B.ndim == 1:
        B = B[:, None]
    n = A.shape[0]
    M = np.concatenate([A, B], axis=1)
    for k in range(n):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if p != k:
            M[[k, p]] = M[[p, k]]
        for i in range(k + 1, n):
            f = M[i, k] / M[k, k]
            M[i, k:] -= f * M[k, k:]
    X = np.zeros((n, B.shape[1]), dtype=np.longdouble)
    for i in range(n - 1, -1, -1):
        X[i] = (M[i, n:] - M[i, i + 1:n] @ X[i + 1:]) / M[i, i]
    return X


def ld_inv(A):
    return ld_solve(A, np.eye(A.shape[0]))


def eig2_sym(a, b, d):
    """Eigenvalues of [[a, b], [b, d]] ascending, closed form."""
    m = 0.5 * (a + d)
    r = np.hypot(0.5 * (a - d), b)
    return np.array([m - r, m + r])


def eig3_sym(A):
    """Eigenvalues of a 3x3 symmetric matrix by the trigonometric cubic formula."""
    A = np.asarray(A, dtype=np.float64)
    q = np.trace(A) / 3.0
    p1 = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
    p2 = (A[0, 0] - q) ** 2 + (A[1, 1] - q) ** 2 + (A[2, 2] - q) ** 2 + 2 * p1
    p = np.sqrt(p2 / 6.0)
    if p == 0.0:
        return np.array([q, q, q])
    Bm = (A - q * np.eye(3)) / p
    r = np.linalg.det(Bm) / 2.0
    r = min(1.0, max(-1.0, r))
    phi = np.arccos(r) / 3.0
    e1 = q + 2 * p * np.cos(phi)
    e3 = q + 2 * p * np.cos(phi + 2 * np.pi / 3)
    e2 = 3 * q - e1 - e3
    return np.sort(np.array([e1, e2, e3]))


def subspace_residual(U1, X):
    """||(I - U1 U1^T) X||_2 / ||X||_2 for U1 with orthonormal columns."""
    P = X - U1 @ (U1.T @ X)
    return np.linalg.norm(P, 2) / np.linalg.norm(X, 2)


def cholesky_upper_c(M):
    """Upper-triangular R, real positive diagonal, R^H R = M (Hermitian M)."""
    M = np.asarray(M, dtype=np.complex128)
    n = M.shape[0]
    R = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        s = (M[j, j] - np.vdot(R[:j, j], R[:j, j])).real
        R[j, j] = np.sqrt(s)
        for k in range(j + 1, n):
            R[j, k] = (M[j, k] - np.vdot(R[:j, j], R[:j, k])) / R[j, j]
    return R


def ld_solve_c(A, B):
    """A^{-1} B over C by Gaussian elimination with partial pivoting in long double."""
    A = np.array(A, dtype=np.clongdouble)
    B = np.array(B, dtype=np.clongdouble)
    if B.ndim == 1:
        B = B[:, None]
    n = A.shape[0]
    M = np.concatenate([A, B], axis=1)
    for k in range(n):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if p != k:
            M[[k, p]] = M[[p, k]]
        for i in range(k + 1, n):
            f = M[i, k] / M[k, k]
            M[i, k:] -= f * M[k, k:]
    X = np.zeros((n, B.shape[1]), dtype=np.clongdouble)
    for i in range(n - 1, -1, -1):
        X[i] = (M[i, n:] - M[i, i + 1:n] @ X[i + 1:]) / M[i, i]
    return X


def subspace_residual_c(U1, X):
    """||(I - U1 U1^H) X||_2 / ||X||_2 for U1 with orthonormal columns (complex)."""
    P = X - U1 @ (U1.conj().T @ X)
    return np.linalg.norm(P, 2) / np.linalg.norm(X, 2)
