"""Singular values through the symmetric eigensolver (RSVD, Sec. 3.2), oracle side.

Test infrastructure only.  The paper reduces the SVD of A (m x n) to the
symmetric eigenproblem of the embedding H = [[0, A], [A^T, 0]] of order
m + n: its eigenvalues are +-sigma_i (and |m - n| zeros) and the eigenvector
of +sigma_i is [u_i; v_i] / sqrt(2) for the singular pair (u_i, v_i).  Here
H goes through the RSEP recursion (solve.eig_sym), the min(m, n) largest
eigenvalues are the singular values (descending), and u_i, v_i are the two
halves of their eigenvectors scaled by sqrt(2) (reading: for sigma_i > 0 each
half has norm 1/sqrt(2) exactly in exact arithmetic; zero singular values do
not determine their vectors and are returned with whatever the halves hold).

Pinned by tests/test_oracle_method.py: prescribed singular values of
A = U diag(s) V^T, agreement with the library SVD, A = U S V^T and the
orthogonality of U and V.
"""
import numpy as np

from .solve import eig_sym


def embed(A):
    """H = [[0, A], [A^T, 0]]."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    H = np.zeros((m + n, m + n))
    H[:m, m:] = A
    H[m:, :m] = A.T
    return H


def svd(A, seed=0, leaf_size=64, split_tol=None):
    """(s descending, U (m x r), V (n x r), info), r = min(m, n)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    r = min(m, n)
    w, W, info = eig_sym(embed(A), seed=seed, leaf_size=leaf_size, split_tol=split_tol)
    idx = np.arange(m + n - 1, m + n - 1 - r, -1)     # the r largest, descending
    s = w[idx]
    U = np.sqrt(2.0) * W[:m, idx]
    V = np.sqrt(2.0) * W[m:, idx]
    return s, U, V, info
