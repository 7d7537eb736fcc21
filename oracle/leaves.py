"""Small-problem solvers for the leaves of the recursion (oracle side).

Sec. 3.6 ("Our algorithm") says a subproblem small enough is solved by the
standard algorithm and its eigenvalues returned.  The paper names no
particular one; readings used here (textbook algorithms, Golub and Van Loan,
Matrix Computations, Ch. 7-8):

  * symmetric: cyclic-by-row Jacobi with the symmetric 2x2 Schur rotation,
    sweeps until off(A) <= n u ||A||_F (u = 2^-53);
  * nonsymmetric: Householder reduction to Hessenberg form, then Francis
    double-shift QR with deflation on |h_{i+1,i}| <= u (|h_ii| + |h_{i+1,i+1}|),
    each remaining 2x2 block put in standard form (upper triangular when its
    eigenvalues are real, equal diagonal entries when complex).

Pinned by tests/test_oracle_method.py: 2x2 / 3x3 closed forms, prescribed
spectra, orthogonality and backward error, quasi-triangular structure.
"""
import numpy as np

from .householder import house

U_ROUND = 2.0 ** -53


# ---------------------------------------------------------------- Jacobi

def _sym_schur2(a_pp, a_qq, a_pq):
    """(c, s) of the rotation that zeroes a_pq (symmetric 2x2 Schur)."""
    if a_pq == 0.0:
        return 1.0, 0.0
    tau = (a_qq - a_pp) / (2.0 * a_pq)
    if tau >= 0.0:
        t = 1.0 / (tau + np.sqrt(1.0 + tau * tau))
    else:
        t = -1.0 / (-tau + np.sqrt(1.0 + tau * tau))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, t * c


def _off(A):
    """Frobenius norm of the off-diagonal part, summed directly."""
    D = A - np.diag(np.diag(A))
    return float(np.sqrt(np.sum(D * D)))


def jacobi_eig(A, max_sweeps=40):
    """(w, V) with A V = V diag(w), w ascending, by cyclic-by-row Jacobi."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    if n == 0:
        return np.zeros(0), V
    fro = float(np.sqrt(np.sum(A * A)))
    tol = n * U_ROUND * fro
    for _ in range(max_sweeps):
        if _off(A) <= tol:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                c, s = _sym_schur2(A[p, p], A[q, q], A[p, q])
                if s == 0.0:
                    continue
                cp, cq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * cp - s * cq
                A[:, q] = s * cp + c * cq
                rp, rq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * rp - s * rq
                A[q, :] = s * rp + c * rq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


# ------------------------------------------------------ Hessenberg + Francis

def hessenberg(A):
    """(H, Z) with A = Z H Z^T, H upper Hessenberg."""
    H = np.array(A, dtype=np.float64, copy=True)
    n = H.shape[0]
    Z = np.eye(n)
    for k in range(n - 2):
        v, beta, _ = house(H[k + 1:, k])
        if beta == 0.0:
            continue
        H[k + 1:, k:] -= beta * np.outer(v, v @ H[k + 1:, k:])
        H[:, k + 1:] -= beta * np.outer(H[:, k + 1:] @ v, v)
        Z[:, k + 1:] -= beta * np.outer(Z[:, k + 1:] @ v, v)
        H[k + 2:, k] = 0.0
    return H, Z


def _rot_rows_cols(H, Z, k, c, s):
    """H <- G^T H G, Z <- Z G for G = [[c, -s], [s, c]] acting on (k, k+1)."""
    r0, r1 = H[k, :].copy(), H[k + 1, :].copy()
    H[k, :] = c * r0 + s * r1
    H[k + 1, :] = -s * r0 + c * r1
    c0, c1 = H[:, k].copy(), H[:, k + 1].copy()
    H[:, k] = c * c0 + s * c1
    H[:, k + 1] = -s * c0 + c * c1
    z0, z1 = Z[:, k].copy(), Z[:, k + 1].copy()
    Z[:, k] = c * z0 + s * z1
    Z[:, k + 1] = -s * z0 + c * z1


def standardize_2x2(H, Z, k):
    """Put the 2x2 diagonal block at (k, k+1) in standard form; return its eigenvalues."""
    a, b = H[k, k], H[k, k + 1]
    c, d = H[k + 1, k], H[k + 1, k + 1]
    if c == 0.0:
        return (a, 0.0), (d, 0.0)
    p = 0.5 * (a - d)
    disc = p * p + b * c
    if disc >= 0.0:
        # real pair: rotate an eigenvector of eigenvalue d + z onto e1
        z = p + np.copysign(np.sqrt(disc), p)
        nrm = np.hypot(z, c)
        cs, sn = z / nrm, c / nrm
        _rot_rows_cols(H, Z, k, cs, sn)
        H[k + 1, k] = 0.0
        return (H[k, k], 0.0), (H[k + 1, k + 1], 0.0)
    # complex pair: rotation angle theta with tan(2 theta) = -(a - d) / (b + c)
    theta = 0.5 * np.arctan2(-(a - d), (b + c))
    _rot_rows_cols(H, Z, k, np.cos(theta), np.sin(theta))
    mid = 0.5 * (H[k, k] + H[k + 1, k + 1])
    H[k, k] = mid
    H[k + 1, k + 1] = mid
    im = np.sqrt(abs(H[k, k + 1] * H[k + 1, k]))
    return (mid, im), (mid, -im)


def _francis_step(H, Z, lo, hi, exceptional=False):
    """One implicit double-shift step on the active block lo..hi (size >= 3)."""
    n = H.shape[0]
    m = hi
    if exceptional:
        w = abs(H[m, m - 1]) + abs(H[m - 1, m - 2])
        s = 1.5 * w + H[m, m]
        t = w * w
    else:
        s = H[m - 1, m - 1] + H[m, m]
        t = H[m - 1, m - 1] * H[m, m] - H[m - 1, m] * H[m, m - 1]
    x = H[lo, lo] * H[lo, lo] + H[lo, lo + 1] * H[lo + 1, lo] - s * H[lo, lo] + t
    y = H[lo + 1, lo] * (H[lo, lo] + H[lo + 1, lo + 1] - s)
    z = H[lo + 1, lo] * H[lo + 2, lo + 1]
    for k in range(lo, hi - 1):
        v, beta, _ = house(np.array([x, y, z]))
        q = max(lo, k - 1)
        H[k:k + 3, q:n] -= beta * np.outer(v, v @ H[k:k + 3, q:n])
        r = min(k + 3, hi)
        H[0:r + 1, k:k + 3] -= beta * np.outer(H[0:r + 1, k:k + 3] @ v, v)
        Z[:, k:k + 3] -= beta * np.outer(Z[:, k:k + 3] @ v, v)
        if k > lo:
            H[k + 1, k - 1] = 0.0
            H[k + 2, k - 1] = 0.0
        x = H[k + 1, k]
        y = H[k + 2, k]
        if k < hi - 2:
            z = H[k + 3, k]
    v, beta, _ = house(np.array([x, y]))
    H[hi - 1:hi + 1, hi - 2:n] -= beta * np.outer(v, v @ H[hi - 1:hi + 1, hi - 2:n])
    H[0:hi + 1, hi - 1:hi + 1] -= beta * np.outer(H[0:hi + 1, hi - 1:hi + 1] @ v, v)
    Z[:, hi - 1:hi + 1] -= beta * np.outer(Z[:, hi - 1:hi + 1] @ v, v)
    H[hi, hi - 2] = 0.0


def real_schur(A, max_iter_per_eig=40):
    """(T, Z, wr, wi, ok): A = Z T Z^T, T quasi-upper-triangular in standard form."""
    H, Z = hessenberg(A)
    n = H.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    hi = n - 1
    its = 0
    total_budget = max_iter_per_eig * max(n, 1)
    while hi >= 0:
        if hi == 0:
            wr[0], wi[0] = H[0, 0], 0.0
            hi -= 1
            continue
        lo = hi
        while lo > 0:
            scale = abs(H[lo - 1, lo - 1]) + abs(H[lo, lo])
            if scale == 0.0:
                scale = float(np.sum(np.abs(H[max(0, lo - 1):hi + 1, max(0, lo - 1):hi + 1])))
            if abs(H[lo, lo - 1]) <= U_ROUND * scale:
                H[lo, lo - 1] = 0.0
                break
            lo -= 1
        if lo == hi:
            wr[hi], wi[hi] = H[hi, hi], 0.0
            hi -= 1
            its = 0
            continue
        if lo == hi - 1:
            (r0, i0), (r1, i1) = standardize_2x2(H, Z, hi - 1)
            wr[hi - 1], wi[hi - 1], wr[hi], wi[hi] = r0, i0, r1, i1
            hi -= 2
            its = 0
            continue
        its += 1
        total_budget -= 1
        if total_budget < 0:
            return H, Z, wr, wi, False
        _francis_step(H, Z, lo, hi, exceptional=(its % 11 == 10))
    return H, Z, wr, wi, True


# ------------------------------------------------------ pencil leaves

def _back_solve_right(A, R):
    """X with X R = A for upper-triangular R (column-by-column substitution)."""
    n = R.shape[0]
    X = np.zeros_like(A)
    for j in range(n):
        X[:, j] = (A[:, j] - X[:, :j] @ R[:j, j]) / R[j, j]
    return X


def _upper_rotation(b10, b11):
    """2x2 orthogonal Z with [b10, b11] Z = [0, r], r = hypot(b10, b11) >= 0."""
    r = float(np.hypot(b10, b11))
    if r == 0.0:
        return np.eye(2)
    return np.array([[b11, b10], [-b10, b11]]) / r


def pencil_schur_leaf(A, B, cond_limit=1e8, swapped=False):
    """Generalized real Schur form of a small regular pencil (A, B).

    Reading for the leaves of the pencil recursion (the paper leaves small
    subproblems to "the standard algorithm"): with B well conditioned,
    M = A B^{-1} has the eigenvalues of the pencil; its real Schur form
    M = QL TM QL^T and the RQ factorisation QL^T B = R Z give
        QL^T A Z^T = TM R (quasi-upper-triangular),  QL^T B Z^T = R (upper),
    i.e. QR_ = Z^T.  B^{-1} is applied through its QR factors and a triangular
    substitution.

    swapped: the leaf comes from the group the recursion handles as (B, A)
    (eigenvalues outside the unit circle, Sec. 3.5), where A, not B, is the
    well-conditioned matrix (B may be singular: infinite eigenvalues).  The
    same construction is then run on (B, A); it leaves B's blocks of complex
    pairs 2x2 and A's triangular, so each such block of Q_L^T B Q_R is made
    upper triangular by one rotation of its two columns of Q_R (A's block
    becomes a full 2x2 block).

    Returns (S, T, QL, QR_, wi, ok) with S = QL^T A QR_ quasi-upper-triangular
    and T = QL^T B QR_ upper triangular (up to rounding); wi marks the 2x2
    blocks (wi[i] > 0, wi[i+1] = -wi[i]).  ok is False when max|R_ii| /
    min|R_ii| of the factorised matrix's QR exceeds cond_limit.
    """
    from .householder import qr_explicit, rq_explicit
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    P, Qm = (B, A) if swapped else (A, B)
    QB, RB = qr_explicit(Qm)
    d = np.abs(np.diag(RB))
    if d.size and (d.min() == 0.0 or d.max() / d.min() > cond_limit):
        return None, None, None, None, None, False
    X = _back_solve_right(P, RB)          # P Qm^{-1} = P R^{-1} QB^T
    M = X @ QB.T
    TM, QL, wr, wi, ok = real_schur(M)
    R, Qrq = rq_explicit(QL.T @ Qm)
    QR_ = Qrq.T
    if swapped:
        m = A.shape[0]
        i = 0
        while i < m - 1:
            if wi[i] > 0.0 and wi[i + 1] == -wi[i]:
                blk = QL[:, i:i + 2].T @ B @ QR_[:, i:i + 2]
                QR_[:, i:i + 2] = QR_[:, i:i + 2] @ _upper_rotation(blk[1, 0], blk[1, 1])
                i += 2
            else:
                i += 1
    S = QL.T @ A @ QR_
    T = QL.T @ B @ QR_
    return S, T, QL, QR_, wi, ok
