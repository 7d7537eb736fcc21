"""Similarity and block-size choice (Algorithms 4-6, Sec. 4.2.1), oracle side.

After the splitter U (Algorithms 5/6, line 2) the step forms A^ = U^H A U
(RSEP also symmetrises, A^ := (A^ + A^^H)/2) and chooses the block size k that
minimises ||E21||_1 / ||A||_1 (plus ||F21||_1 / ||B||_1 for pencils,
Algorithm 4), where E21 = A^(k+1:n, 1:k) in 1-based indexing.

Sec. 4.2.1 computes the n-1 candidates with a column-wise prefix (here:
suffix) sum and a row-wise max reduction:
    S[k][j] = sum_{i >= k} |A^_ij|,   f(k) = max_{j < k} S[k][j]  (0-based k),
    e(k) = f(k) / ||A^||_1 for k = 1 .. n-1.
This oracle evaluates exactly that definition.

Readings (paper silent): the winner is the smallest e(k); exact ties go to the
k closest to n/2, then the smaller k.  Acceptance threshold split_tol is a
parameter (1e-12 by default in FP64).

Pinned by tests/test_oracle_basics.py: brute-force slicing of every E21 block.
"""
import numpy as np


def similarity(A, QL, QR):
    """Q_L^H A Q_R."""
    return QL.T @ np.asarray(A) @ QR


def symmetrise(A):
    return 0.5 * (A + A.T)


def _norm1(X):
    return float(np.max(np.sum(np.abs(X), axis=0))) if X.size else 0.0


def split_scores(Ahat):
    """e(k)*||A^||_1 for k = 1..n-1 via column suffix sums and prefix max."""
    n = Ahat.shape[0]
    absA = np.abs(Ahat)
    S = np.zeros((n + 1, n))
    for i in range(n - 1, -1, -1):         # column-wise suffix sums
        S[i] = S[i + 1] + absA[i]
    f = np.zeros(n)
    for k in range(1, n):                   # row-wise prefix max over j < k
        f[k] = np.max(S[k, :k])
    return f[1:]


def choose_k(scores, n):
    """Index k (1..n-1) of the smallest score; ties -> closest to n/2, then smaller."""
    best = None
    for idx, val in enumerate(scores):
        k = idx + 1
        key = (val, abs(2 * k - n), k)
        if best is None or key < best[0]:
            best = (key, k)
    return best[1]


def split_test(Ahat, Bhat=None, normA=None, normB=None):
    """Return (k, e(k), all e values) for A^ (and B^ for a pencil)."""
    Ahat = np.asarray(Ahat)
    n = Ahat.shape[0]
    if n < 2:
        return 0, 0.0, np.zeros(0)
    nA = _norm1(Ahat) if normA is None else normA
    e = split_scores(Ahat) / (nA if nA > 0 else 1.0)
    if Bhat is not None:
        nB = _norm1(Bhat) if normB is None else normB
        e = e + split_scores(np.asarray(Bhat)) / (nB if nB > 0 else 1.0)
    k = choose_k(e, n)
    return k, float(e[k - 1]), e
