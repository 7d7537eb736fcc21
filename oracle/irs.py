"""Implicit repeated squaring (Algorithm 3) and the region maps (oracle side).

Algorithm 3 (Sec. 3.1): with A_0 = A, B_0 = B, repeat
    [B_j; -A_j] = Q [R_j; 0]          (QR of the stacked 2n x n matrix)
    A_{j+1} = Q12^T A_j,  B_{j+1} = Q22^T B_j
until ||R_j - R_{j-1}||_1 <= tau ||R_{j-1}||_1 (then p = j + 1) or j > maxit.
Q12 and Q22 are the top and bottom n x n blocks of the last n columns of the
2n x 2n orthogonal factor; here they are formed by applying the reflectors to
[0; I] (Sec. 3.2 shows A_{j+1}^{-1} B_{j+1} = (A_j^{-1} B_j)^2).

Readings where the paper is silent:
  * the test needs R_{j-1}, so it is first evaluated at j = 1;
  * R_j is made unique by a non-negative diagonal (householder.py);
  * the loop runs j = 0, 1, ..., maxit (the paper's "until j > maxit");
    on exit without convergence the last iterate is returned with
    converged = False.

Region maps (eigenvalues are those of det(A - z B) = 0):
  * unit circle: (A, B) unchanged (Sec. 3.1);
  * circle |z - c| = r, real c: (A - c B, r B) (Sec. 3.5 uses circles of
    radius 2^(-+2^k) about the origin);
  * line Re z = sigma with scale s: the Moebius map f(z) = (z-sigma+s)/(z-sigma-s)
    of Sec. 3.3 (s = 1 there) sends (A, B) to (A - (sigma-s) B, A - (sigma+s) B).
After the map, eigenvalues outside the unit circle are those outside the
circle / right of the line.

Pinned by tests/test_oracle_method.py: the diagonal closed form of one step,
R_j against an independent Cholesky of A_j^T A_j + B_j^T B_j, and
A_p^{-1} B_p = (A^{-1} B)^(2^p) by long-double Gaussian elimination.
"""
import numpy as np

from .householder import qr_factor

REGION_UNIT_CIRCLE = 0
REGION_CIRCLE = 1
REGION_LINE = 2


def region_map(A, B, kind, c_or_sigma=0.0, r_or_s=1.0):
    """Pencil (A', B') whose unit-circle split is the requested region's split."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    B = np.eye(n) if B is None else np.asarray(B, dtype=np.float64)
    if kind == REGION_UNIT_CIRCLE:
        return A.copy(), B.copy()
    if kind == REGION_CIRCLE:
        return A - c_or_sigma * B, r_or_s * B
    if kind == REGION_LINE:
        sigma, s = c_or_sigma, r_or_s
        return A - (sigma - s) * B, A - (sigma + s) * B
    raise ValueError("unknown region kind %r" % (kind,))


def norm1(X):
    """Matrix 1-norm: the largest column sum of absolute values."""
    X = np.asarray(X)
    if X.size == 0:
        return 0.0
    return float(np.max(np.sum(np.abs(X), axis=0)))


def default_tau(n):
    """Reading: tau = max(1e-14, 4 sqrt(n) u) with u = 2^-53 (paper silent)."""
    return max(1e-14, 4.0 * np.sqrt(n) * 2.0 ** -53)


class IRSResult:
    def __init__(self, Ap, Bp, iters, converged, ratios, Rs):
        self.Ap = Ap
        self.Bp = Bp
        self.iters = iters          # p: number of squarings performed
        self.converged = converged
        self.ratios = ratios        # ratio at j = 1, 2, ...
        self.Rs = Rs                # R_j for j = 0, 1, ... (if recorded)


def irs_step(Aj, Bj):
    """One squaring: returns (A_{j+1}, B_{j+1}, R_j)."""
    n = Aj.shape[0]
    W = np.vstack([Bj, -Aj])
    f = qr_factor(W)
    E = np.zeros((2 * n, n))
    E[n:, :] = np.eye(n)
    Y = f.q_times(E)                   # last n columns of Q: [Q12; Q22]
    Q12, Q22 = Y[:n, :], Y[n:, :]
    return Q12.T @ Aj, Q22.T @ Bj, f.R


def irs(A, B, tau=None, maxit=60, record_R=False):
    """Algorithm 3 on the pencil (A, B); B = None means the identity."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    B = np.eye(n) if B is None else np.array(B, dtype=np.float64, copy=True)
    if tau is None:
        tau = default_tau(n)
    Aj, Bj = A, B
    R_prev = None
    ratios, Rs = [], []
    j = 0
    while True:
        A_next, B_next, R = irs_step(Aj, Bj)
        if record_R:
            Rs.append(R.copy())
        if R_prev is not None:
            den = norm1(R_prev)
            num = norm1(R - R_prev)
            ratio = num / den if den > 0.0 else (0.0 if num == 0.0 else np.inf)
            ratios.append(ratio)
            if ratio <= tau:
                return IRSResult(A_next, B_next, j + 1, True, ratios, Rs)
        R_prev = R
        Aj, Bj = A_next, B_next
        j += 1
        if j > maxit:
            return IRSResult(Aj, Bj, j, False, ratios, Rs)
