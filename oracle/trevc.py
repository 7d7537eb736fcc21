"""Eigenvectors from the Schur form (TREVC, the eigenvector section), oracle side.

Test infrastructure only.  For A = Q T Q^H with T upper triangular and
distinct eigenvalues, the eigenvector matrix of T is the upper triangular X
with T X = X D, D = diag(T); column j follows from X_jj (chosen 1 here) by
    X_ij = (T_ij X_jj + sum_{k=i+1}^{j-1} T_ik X_kj) / (T_jj - T_ii),  i < j,
and the eigenvectors of A are the columns of Q X (normalised to unit 2-norm).

The nonsymmetric solver returns the real Schur form, quasi-upper-triangular
with a 2 x 2 block [[a, b], [c, d]] per complex pair.  Reading: such a block
is first made triangular in complex arithmetic by the unitary G whose first
column is the block's eigenvector (mu - d, c) / ||.|| for the eigenvalue mu of
positive imaginary part; G^H acts on the block's two rows of T, G on its two
columns of T and Q.  The result is a complex Schur form to which the
recurrence applies.

Pinned by tests/test_oracle_method.py: the 2 x 2 triangular closed form
X = [[1, b / (d - a)], [0, 1]], the residual ||A V - V L|| against ||A|| ||V||
on prescribed spectra with real and complex eigenvalues, and agreement (up
to scaling) with the library eigenvectors.
"""
import numpy as np


def real_to_complex_schur(T, Q, wi):
    """(Tc, Qc): a complex Schur form A = Qc Tc Qc^H from the real one (T, Q, wi)."""
    Tc = np.array(T, dtype=np.complex128)
    Qc = np.array(Q, dtype=np.complex128)
    n = Tc.shape[0]
    i = 0
    while i < n - 1:
        if wi[i] > 0.0 and wi[i + 1] == -wi[i]:
            a, b, c, d = Tc[i, i], Tc[i, i + 1], Tc[i + 1, i], Tc[i + 1, i + 1]
            tr, det = a + d, a * d - b * c
            disc = np.sqrt(tr * tr / 4.0 - det + 0j)
            mu = tr / 2.0 + disc
            if mu.imag < 0:
                mu = tr / 2.0 - disc
            v = np.array([mu - d, c])
            v = v / np.linalg.norm(v)
            G = np.array([[v[0], -np.conj(v[1])], [v[1], np.conj(v[0])]])
            Tc[i:i + 2, :] = G.conj().T @ Tc[i:i + 2, :]
            Tc[:, i:i + 2] = Tc[:, i:i + 2] @ G
            Qc[:, i:i + 2] = Qc[:, i:i + 2] @ G
            Tc[i + 1, i] = 0.0
            i += 2
        else:
            i += 1
    return Tc, Qc


def small_pivot(T):
    """smin = u max_i |T_ii| (u = 2^-53; 2^-1022 if T's diagonal is zero)."""
    d = np.abs(np.diag(np.asarray(T)))
    top = float(np.max(d)) if d.size else 0.0
    return max(2.0 ** -53 * top, 2.0 ** -1022)


def triangular_eigenvectors(T):
    """Upper triangular X with T X = X diag(T), X_jj = 1.

    A denominator T_jj - T_ii of modulus below small_pivot(T) is replaced by
    small_pivot(T) (reading: the paper divides by it directly; an exact double
    eigenvalue would give an infinite vector, and the standard triangular
    eigenvector solvers perturb such pivots to the rounding level instead).
    Distinct eigenvalues separated by more than that are unaffected."""
    T = np.asarray(T)
    n = T.shape[0]
    smin = small_pivot(T)
    X = np.zeros((n, n), dtype=np.result_type(T.dtype, np.float64))
    for j in range(n):
        X[j, j] = 1.0
        for i in range(j - 1, -1, -1):
            s = T[i, j] * X[j, j] + T[i, i + 1:j] @ X[i + 1:j, j]
            den = T[j, j] - T[i, i]
            if abs(den) < smin:
                den = smin
            X[i, j] = s / den
    return X


def eigenvectors(T, Q, wi):
    """(lam, V): eigenvalues diag(Tc) and unit eigenvectors V = Qc X of A = Q T Q^T."""
    Tc, Qc = real_to_complex_schur(T, Q, wi)
    X = triangular_eigenvectors(Tc)
    V = Qc @ X
    V = V / np.linalg.norm(V, axis=0)
    return np.diag(Tc).copy(), V
