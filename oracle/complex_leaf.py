"""Complex Schur form of a small matrix, for the leaves of the complex-plane
recursion (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.6 solves a small enough subproblem by the standard algorithm.  Once
the splitting lines of Sec. 3.3 are drawn at random angles the blocks are
complex, and the standard algorithm is then the complex QR iteration
(Golub and Van Loan, Matrix Computations, Ch. 7): Householder reduction to
upper Hessenberg form, then single-shift QR steps done implicitly with
Givens rotations (bulge chasing), with
  * deflation when |h_{k,k-1}| <= u (|h_{k-1,k-1}| + |h_kk|), u = 2^-53;
  * the Wilkinson shift: the eigenvalue of the trailing 2 x 2 block of the
    active window closer to its last diagonal entry;
  * an exceptional shift h_kk + 0.75 |h_{k,k-1}| (an ad hoc value, reading)
    every 10th step without a deflation.
The complex Givens rotation of (a, b) is G = [[conj a, conj b], [-b, a]] / rho,
rho = sqrt(|a|^2 + |b|^2), so G (a, b)^T = (rho, 0)^T.

Pinned by tests/test_oracle_complex.py: the 2 x 2 closed form of the
eigenvalues, prescribed spectra, unitarity and backward error, triangular
structure, and the library eigenvalues as a special-case check.
"""
import numpy as np

from .complex_qr import chouse, _reflect_rows, _reflect_cols

U_ROUND = 2.0 ** -53


def chessenberg(A):
    """(H, Z) with A = Z H Z^H, H upper Hessenberg (complex Householder)."""
    H = np.array(A, dtype=np.complex128, copy=True)
    n = H.shape[0]
    Z = np.eye(n, dtype=np.complex128)
    for k in range(n - 2):
        v, _ = chouse(H[k + 1:, k])
        if v is None:
            continue
        H[k + 1:, :] = _reflect_rows(v, H[k + 1:, :])
        H[:, k + 1:] = _reflect_cols(H[:, k + 1:], v)
        Z[:, k + 1:] = _reflect_cols(Z[:, k + 1:], v)
        H[k + 2:, k] = 0.0
    return H, Z


def givens(a, b):
    """2 x 2 unitary G with G (a, b)^T = (rho, 0)^T, rho >= 0."""
    rho = float(np.sqrt(abs(a) ** 2 + abs(b) ** 2))
    if rho == 0.0:
        return np.eye(2, dtype=np.complex128)
    G = np.array([[np.conj(a), np.conj(b)], [-b, a]], dtype=np.complex128)
    return G.real / rho + 1j * (G.imag / rho)   # no reciprocal of a subnormal rho


def _apply(H, Z, k, G):
    """H <- G_k H G_k^H, Z <- Z G_k^H, G acting on indices (k, k+1)."""
    H[k:k + 2, :] = G @ H[k:k + 2, :]
    H[:, k:k + 2] = H[:, k:k + 2] @ G.conj().T
    Z[:, k:k + 2] = Z[:, k:k + 2] @ G.conj().T


def wilkinson_shift(a, b, c, d):
    """Eigenvalue of [[a, b], [c, d]] closer to d."""
    tr2 = 0.5 * (a + d)
    disc = np.sqrt((0.5 * (a - d)) ** 2 + b * c + 0j)
    l1, l2 = tr2 + disc, tr2 - disc
    return l1 if abs(l1 - d) <= abs(l2 - d) else l2


def _qr_step(H, Z, lo, hi, mu):
    """One implicit single-shift step on the active window lo..hi."""
    G = givens(H[lo, lo] - mu, H[lo + 1, lo])
    _apply(H, Z, lo, G)
    for k in range(lo + 1, hi):
        G = givens(H[k, k - 1], H[k + 1, k - 1])
        _apply(H, Z, k, G)
        H[k + 1, k - 1] = 0.0


def complex_schur(A, max_iter_per_eig=40):
    """(T, Z, w, ok): A = Z T Z^H, T upper triangular, w = diag(T)."""
    H, Z = chessenberg(A)
    n = H.shape[0]
    hi = n - 1
    its = 0
    budget = max_iter_per_eig * max(n, 1)
    while hi > 0:
        lo = hi
        while lo > 0:
            scale = abs(H[lo - 1, lo - 1]) + abs(H[lo, lo])
            if scale == 0.0:
                scale = float(np.sum(np.abs(H[lo - 1:hi + 1, lo - 1:hi + 1])))
            if abs(H[lo, lo - 1]) <= U_ROUND * scale:
                H[lo, lo - 1] = 0.0
                break
            lo -= 1
        if lo == hi:
            hi -= 1
            its = 0
            continue
        its += 1
        budget -= 1
        if budget < 0:
            return H, Z, np.diag(H).copy(), False
        if its % 10 == 0:
            mu = H[hi, hi] + 0.75 * abs(H[hi, hi - 1])
        else:
            mu = wilkinson_shift(H[hi - 1, hi - 1], H[hi - 1, hi], H[hi, hi - 1], H[hi, hi])
        _qr_step(H, Z, lo, hi, mu)
    T = np.triu(H)
    return T, Z, np.diag(T).copy(), True
