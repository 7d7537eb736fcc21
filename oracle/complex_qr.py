"""Complex Householder QR, RQ by index reversal and the Haar unitary (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The complex-plane strategy of Sec. 3.3 draws splitting lines at a random
angle, so the deflating subspaces, the splitter and the blocks are complex;
the factorizations of Sec. 3 (QR, RQ with explicit unitary factors) and the
Gaussian matrix of Algorithm 1 are then taken over C.

Conventions (readings; the paper fixes none):
  * reflector of x (Golub and Van Loan, Matrix Computations, Sec. 5.1, the
    complex case): with x0 = |x0| e^{i phi} (phi = 0 when x0 = 0),
    v = x + e^{i phi} ||x|| e1 and P = I - 2 v v^H / (v^H v), so that
    P x = -e^{i phi} ||x|| e1.  P is Hermitian and unitary;
  * after the n reflectors the diagonal of R is made real and non-negative
    by a diagonal unitary D: Q <- Q D, R <- D^H R.  That makes the QR of a
    full-column-rank X unique (R is the Cholesky factor of X^H X), so the
    result does not depend on the reflector convention;
  * RQ of a square Y: QR of Z = (J Y)^H = Z~ R~ gives
    Y = (J R~^H J)(J Z~^H), J the index reversal; J R~^H J is upper
    triangular with a real non-negative diagonal;
  * Haar unitary: the Q factor of a complex Ginibre matrix G = X + i Y, with
    X and Y independent N(0,1) draws, under the non-negative diagonal
    convention (F. Mezzadri, "How to generate random matrices from the
    classical compact groups", Notices AMS 54 (2007)).  X comes from the
    Philox stream of purpose PURPOSE_HAAR, Y from PURPOSE_HAAR_IMAG, same
    seed, node and attempt word.

Pinned by tests/test_oracle_complex.py: Q^H Q = I, Q R = X, R against an
independent complex Cholesky of X^H X, the RQ identity, and the Haar moments
E|V_ij|^2 = 1/n, E V_ij^2 = 0, E|tr V|^2 = 1 (a real or sign-biased Q fails
the last two).
"""
import numpy as np

from .philox import gaussian_matrix, PURPOSE_HAAR

PURPOSE_HAAR_IMAG = 7


def chouse(x):
    """(v, mu) with (I - 2 v v^H / v^H v) x = mu e1, mu = -e^{i phi} ||x||.

    v is None when x is already a multiple of e1 with nothing to do (x = 0).
    """
    x = np.asarray(x, dtype=np.complex128)
    nrm = float(np.sqrt(np.sum(np.abs(x) ** 2)))
    if nrm == 0.0:
        return None, 0.0 + 0.0j
    x0 = x[0]
    a0 = abs(x0)
    # real and imaginary parts divided separately: numpy's complex-by-real
    # division goes through a reciprocal that overflows for a subnormal |x0|
    ph = complex(x0.real / a0, x0.imag / a0) if a0 > 0 else 1.0 + 0.0j
    v = x.copy()
    v[0] = x0 + ph * nrm
    return v, -ph * nrm


def _reflect_rows(v, W):
    """(I - 2 v v^H / v^H v) W."""
    return W - np.outer(v, (2.0 / np.vdot(v, v).real) * (v.conj() @ W))


def _reflect_cols(W, v):
    """W (I - 2 v v^H / v^H v)."""
    return W - np.outer((2.0 / np.vdot(v, v).real) * (W @ v), v.conj())


class CQRFactors:
    """Reflectors, phases and R of X = Q R (X is m x n, m >= n)."""

    def __init__(self, vs, phases, R, m):
        self.vs = vs            # vs[j] acts on rows j.., None for an identity
        self.phases = phases    # D = diag(phases): Q = H_0 ... H_{n-1} diag(D, I)
        self.R = R
        self.m = m

    def q_times(self, E):
        """Q E for an m x c matrix E (the phases act on the first n rows of E)."""
        Y = np.array(E, dtype=np.complex128, copy=True)
        n = len(self.vs)
        Y[:n, :] *= self.phases[:, None]
        for j in range(n - 1, -1, -1):
            v = self.vs[j]
            if v is not None:
                Y[j:, :] = _reflect_rows(v, Y[j:, :])
        return Y


def cqr_factor(X):
    """Complex Householder QR, one column at a time, R with real diag >= 0."""
    W = np.array(X, dtype=np.complex128, copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("cqr_factor needs m >= n")
    vs = []
    for j in range(n):
        v, mu = chouse(W[j:, j])
        if v is not None:
            W[j:, j:] = _reflect_rows(v, W[j:, j:])
            W[j, j] = mu
            W[j + 1:, j] = 0.0
        vs.append(v)
    R = np.triu(W[:n, :n])
    d = np.diag(R).copy()
    phases = np.ones(n, dtype=np.complex128)
    nz = np.abs(d) > 0.0
    ad = np.abs(d[nz])
    phases[nz] = d[nz].real / ad + 1j * (d[nz].imag / ad)
    R = phases.conj()[:, None] * R
    R[np.arange(n), np.arange(n)] = np.abs(d)
    return CQRFactors(vs, phases, R, m)


def cqr_explicit(X):
    """(Q, R): Q m x n with orthonormal columns, X = Q R, diag(R) real >= 0."""
    f = cqr_factor(X)
    m, n = np.asarray(X).shape
    E = np.zeros((m, n), dtype=np.complex128)
    E[:n, :n] = np.eye(n)
    return f.q_times(E), f.R


def crq_explicit(Y):
    """(R, Q) with Y = R Q, Q unitary, R upper triangular with real diag >= 0."""
    Y = np.asarray(Y, dtype=np.complex128)
    Z = Y[::-1, :].conj().T
    Qt, Rt = cqr_explicit(Z)
    R = Rt.conj().T[::-1, ::-1].copy()
    Q = Qt.conj().T[::-1, :].copy()
    return R, Q


def chaar(n, seed, stream, attempt=0, purpose=PURPOSE_HAAR, purpose_imag=PURPOSE_HAAR_IMAG):
    """n x n Haar unitary from the Philox Ginibre draw of this stream."""
    G = (gaussian_matrix(n, n, seed, purpose, stream, attempt)
         + 1j * gaussian_matrix(n, n, seed, purpose_imag, stream, attempt))
    V, _ = cqr_explicit(G)
    return V
