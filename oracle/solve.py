"""One divide step (RSEP / RNEP / RGNEP) and the recursive drivers (oracle).

One step (Algorithms 4-6): map the region to the unit circle, run IRS
(Algorithm 3), take the splitter U = GRURV(2, A_p + B_p, A_p, -1, +1), form
A^ = U^T A U (symmetrised for RSEP), choose k minimising ||E21||_1 / ||A||_1.
The leading k columns of U span the (right) deflating subspace of the
eigenvalues outside the unit circle, so A11 = A^(1:k, 1:k) holds the
eigenvalues outside the circle / right of the line (Sec. 3.1, Sec. 3.2).

Recursive strategy, symmetric (Sec. 3.4): keep an interval [lo, hi] that
contains the node's eigenvalues, split at a point x and, if no split happens
but one side is empty, shrink the interval and redraw.
Readings (paper silent or other sources):
  * root interval of a symmetric matrix: [c - rho, c + rho] intersected with
    Gershgorin, c = tr(A)/n, rho = 1.1 x the power-iteration estimate of
    ||A - cI||_2 (16 steps from a Philox Gaussian vector, purpose 9).  Every
    eigenvalue lies within ||A - cI||_2 of c; Gershgorin alone overstates that
    radius by about sqrt(n) for dense matrices (19 vs 1 at n = 2048 on the
    semicircle), and the line scale s below is the interval's half-width, so
    the Moebius distances d / s of Sec. 3.3 (and with them the squaring count
    and the subspace conditioning) follow the true spread.  An estimate that
    falls short of the extreme eigenvalue still gives valid splits (the lines
    only need to lie inside the spectrum's hull);
  * first attempt: x = median(diag A_node) + 0.01 R (2 xi - 1), later attempts
    x uniform in [c - R/2, c + R/2] (the paper's rule), with c, R the centre
    and half-width of [lo, hi] and xi a Philox uniform of the node;
  * line scale s = R (the paper assumes ||A|| = O(1), Sec. 3.3);
  * the side of an unsplit node is read from the numerical rank of R2 in
    RURV(A_p), measured against |A_p + B_p| (rurv.numerical_rank): rank 0
    means no eigenvalue right of x, rank n none left of it;
  * split_tol None means max(1e-12, 16 n u): the rounding floor of
    ||E21||_1 / ||A||_1 after an FP64 step grows about like n u (measured
    4-5 n u at n = 2048 and 4096); for pencils max(1e-10, 16 n u)
    (default_split_tol);
  * a split is accepted when 0 < k < n and e(k) <= split_tol; after max_fail
    unproductive attempts the solve stops with status NO_SPLIT;
  * Theorem 2.1 holds with high probability only: when IRS converged and the
    rank is strictly between 0 and n but e(k) > split_tol, the step redraws V
    (up to v_draws times) and reuses A_p, B_p before giving up on the shift;
  * nonsymmetric nodes use real lines only (angle 0 in Sec. 3.3's strategy)
    on the Gershgorin interval of the real parts, optionally the unit circle
    at the root; complex pairs end in 2x2 blocks of the leaf solver.

Parity: one step is pinned through its parts (IRS, GRURV, split test); the
drivers are pinned by prescribed spectra, closed forms and backward error in
tests/test_oracle_method.py.
"""
import numpy as np

from .irs import (irs, region_map, norm1, default_tau, REGION_LINE, REGION_UNIT_CIRCLE,
                  REGION_CIRCLE)
from .rurv import haar, splitter_right, splitter_left, numerical_rank
from .split import split_test, symmetrise
from .leaves import jacobi_eig, real_schur, pencil_schur_leaf
from .philox import (uniform_scalar, attempt_code, gaussian_matrix, PURPOSE_SHIFT,
                     PURPOSE_HAAR, PURPOSE_HAAR_LEFT, PURPOSE_POWER, ROOT_NODE, child_node)

STATUS_OK = 0
STATUS_NO_CONVERGENCE = 1
STATUS_NO_SPLIT = 2


class StepResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def split_from_irs(A, B, res, res_t, seed, stream, attempt, draw, symmetric):
    """Splitter, similarity and split test for one Haar draw (Algorithms 4-6)."""
    n = A.shape[0]
    V = haar(n, seed, stream, attempt_code(attempt, draw), PURPOSE_HAAR)
    QR_, R1, R2 = splitter_right(res.Ap, res.Bp, V)
    rank = numerical_rank(R2, R1)
    out = dict(QR=QR_, rank=rank, R1=R1, R2=R2, draw=draw)
    if B is None:
        Ahat = QR_.T @ A @ QR_
        if symmetric:
            Ahat = symmetrise(Ahat)
        k, e, es = split_test(Ahat, normA=norm1(A))
        out.update(Ahat=Ahat, Bhat=None, QL=QR_, k=k, e=e, scores=es)
    else:
        VL = haar(n, seed, stream, attempt_code(attempt, draw), PURPOSE_HAAR_LEFT)
        QL, _, _ = splitter_left(res_t.Ap, res_t.Bp, VL)
        Ahat = QL.T @ A @ QR_
        Bhat = QL.T @ B @ QR_
        k, e, es = split_test(Ahat, Bhat, normA=norm1(A), normB=norm1(B))
        out.update(Ahat=Ahat, Bhat=Bhat, QL=QL, k=k, e=e, scores=es)
    return out


def default_split_tol(n, pencil=False):
    """max(1e-12, 16 n u), u = 2^-53 (see the module docstring); pencils
    max(1e-10, 16 n u).  Reading for pencils (Algorithm 4 only asks for
    "small enough"): Q_L and Q_R come from two independent IRS + GRURV runs,
    so ||F21|| carries their mutual error (about u / Dif each) with no
    cancellation, concentrated in the few columns of ill-separated
    directions; the 1-norm score, a column maximum, then overstates the
    backward error ||A - Q_L S Q_R^T||_F / ||A||_F of the finished solve by
    10-50x (measured at n = 2048-4096), so 1e-10 keeps that backward error
    near 1e-11."""
    return max(1e-10 if pencil else 1e-12, 16.0 * n * 2.0 ** -53)


def divide_step(A, B=None, region=(REGION_UNIT_CIRCLE, 0.0, 1.0), seed=0,
                stream=ROOT_NODE, attempt=0, tau=None, maxit=60,
                symmetric=False, split_tol=None, record_R=False, v_draws=4):
    """One step of RSEP (symmetric) / RNEP (B None) / RGNEP (B given)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if split_tol is None:
        split_tol = default_split_tol(n, pencil=B is not None)
    kind, c, r = region
    Am, Bm = region_map(A, B, kind, c, r)
    res = irs(Am, Bm, tau=tau, maxit=maxit, record_R=record_R)
    res_t = None
    if B is not None:
        B = np.asarray(B, dtype=np.float64)
        AmT, BmT = region_map(A.T, B.T, kind, c, r)
        res_t = irs(AmT, BmT, tau=tau, maxit=maxit)
    out = None
    for draw in range(v_draws):
        out = split_from_irs(A, B, res, res_t, seed, stream, attempt, draw, symmetric)
        k, e = out["k"], out["e"]
        out["accepted"] = bool(res.converged and (res_t is None or res_t.converged)
                               and 0 < k < n and e <= split_tol)
        if out["accepted"] or not res.converged or out["rank"] in (0, n):
            break
    out["irs"] = res
    out["irs_left"] = res_t
    return StepResult(**out)


def gershgorin_interval(A):
    """[lo, hi] containing the real parts of all eigenvalues (row discs)."""
    A = np.asarray(A)
    d = np.diag(A)
    rad = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - rad)), float(np.max(d + rad))


POWER_STEPS = 16


def spectral_interval(A, seed):
    """Root interval of a symmetric A (reading in the module docstring)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    glo, ghi = gershgorin_interval(A)
    c = float(np.sum(np.diag(A))) / n
    x = gaussian_matrix(n, 1, seed, PURPOSE_POWER, ROOT_NODE)[:, 0]
    x = x / np.sqrt(x @ x)
    est = 0.0
    for _ in range(POWER_STEPS):
        y = A @ x - c * x
        est = float(np.sqrt(y @ y))
        if est == 0.0:
            break
        x = y / est
    rho = 1.1 * est
    lo, hi = max(glo, c - rho), min(ghi, c + rho)
    if not lo < hi:
        return glo, ghi
    return lo, hi


def choose_shift(A_node, lo, hi, seed, node, attempt):
    """(sigma, s) for the node's attempt (reading in the module docstring)."""
    c = 0.5 * (lo + hi)
    R = 0.5 * (hi - lo)
    if R <= 0.0:
        R = max(abs(c), 1.0) * 1e-3
    xi = uniform_scalar(seed, PURPOSE_SHIFT, node, attempt)
    if attempt == 0:
        sigma = float(np.median(np.diag(A_node))) + 0.01 * R * (2.0 * xi - 1.0)
    else:
        sigma = c + R * (xi - 0.5)
    sigma = min(max(sigma, lo + 1e-3 * R), hi - 1e-3 * R)
    return sigma, R


class SolveInfo:
    def __init__(self):
        self.status = STATUS_OK
        self.nodes = 0
        self.splits = 0
        self.iters = []
        self.depth = 0
        self.failed_attempts = 0


def _recurse(A, seed, leaf_size, tau, maxit, split_tol, max_fail, symmetric,
             root_unit_circle, info):
    # split_tol None: automatic per node size (default_split_tol)
    """Shared recursion; returns (Q, blocks) with A = Q T Q^T block structure."""
    n = A.shape[0]
    Q = np.eye(n)
    leaves = []       # (offset, size, node matrix)
    lo0, hi0 = spectral_interval(A, seed) if symmetric and n > leaf_size else gershgorin_interval(A)
    work = [(0, n, np.array(A, dtype=np.float64), lo0, hi0, ROOT_NODE, 0)]
    while work:
        off, m, An, lo, hi, node, depth = work.pop()
        info.nodes += 1
        info.depth = max(info.depth, depth)
        if m <= leaf_size:
            leaves.append((off, m, An))
            continue
        attempt = 0
        fails = 0
        done = False
        while not done:
            if root_unit_circle and node == ROOT_NODE and attempt == 0:
                region = (REGION_UNIT_CIRCLE, 0.0, 1.0)
            else:
                sigma, s = choose_shift(An, lo, hi, seed, node, attempt)
                region = (REGION_LINE, sigma, s)
            st = divide_step(An, None, region, seed, node, attempt, tau, maxit,
                             symmetric=symmetric, split_tol=split_tol)
            info.iters.append(st.irs.iters)
            if st.accepted:
                k = st.k
                Q[:, off:off + m] = Q[:, off:off + m] @ st.QR
                A11 = st.Ahat[:k, :k].copy()
                A22 = st.Ahat[k:, k:].copy()
                if region[0] == REGION_LINE:
                    sig = region[1]
                    lo1, hi1 = sig, hi
                    lo2, hi2 = lo, sig
                else:
                    lo1, hi1 = gershgorin_interval(A11)
                    lo2, hi2 = gershgorin_interval(A22)
                if not symmetric:
                    g1 = gershgorin_interval(A11)
                    g2 = gershgorin_interval(A22)
                    lo1, hi1 = max(lo1, g1[0]), min(hi1, g1[1])
                    lo2, hi2 = max(lo2, g2[0]), min(hi2, g2[1])
                    if lo1 >= hi1:
                        lo1, hi1 = g1
                    if lo2 >= hi2:
                        lo2, hi2 = g2
                info.splits += 1
                work.append((off + k, m - k, A22, lo2, hi2, child_node(node, 1), depth + 1))
                work.append((off, k, A11, lo1, hi1, child_node(node, 0), depth + 1))
                done = True
                continue
            info.failed_attempts += 1
            if region[0] == REGION_LINE and st.irs.converged:
                if st.rank == 0:
                    hi = region[1]       # nothing right of the line
                elif st.rank == m:
                    lo = region[1]       # nothing left of the line
                else:
                    fails += 1
            else:
                fails += 1
            attempt += 1
            if fails > max_fail or attempt > 250:
                info.status = STATUS_NO_SPLIT
                return Q, leaves, False
    return Q, leaves, True


def eig_sym(A, seed=0, leaf_size=64, tau=None, maxit=60, split_tol=None, max_fail=8):
    """(w ascending, U, info) for symmetric A by RSEP recursion + Jacobi leaves."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    info = SolveInfo()
    Q, leaves, ok = _recurse(A, seed, leaf_size, tau, maxit, split_tol, max_fail,
                             True, False, info)
    w = np.zeros(n)
    if not ok:
        return w, Q, info
    for off, m, An in leaves:
        wl, Vl = jacobi_eig(An)
        Q[:, off:off + m] = Q[:, off:off + m] @ Vl
        w[off:off + m] = wl
    order = np.argsort(w, kind="stable")
    return w[order], Q[:, order], info


def schur_nonsym(A, seed=0, leaf_size=64, tau=None, maxit=60, split_tol=None,
                 max_fail=8, root_unit_circle=True):
    """(T, Q, wr, wi, info): A = Q T Q^T, T quasi-triangular (RNEP + Francis)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    info = SolveInfo()
    Q, leaves, ok = _recurse(A, seed, leaf_size, tau, maxit, split_tol, max_fail,
                             False, root_unit_circle, info)
    wr = np.zeros(n)
    wi = np.zeros(n)
    if not ok:
        return None, Q, wr, wi, info
    for off, m, An in leaves:
        _, Zl, wrl, wil, good = real_schur(An)
        if not good:
            info.status = STATUS_NO_CONVERGENCE
        Q[:, off:off + m] = Q[:, off:off + m] @ Zl
        wr[off:off + m] = wrl
        wi[off:off + m] = wil
    T = Q.T @ A @ Q
    T = quasi_triangular_part(T, wi)
    return T, Q, wr, wi, info


RADIUS_EXP_LIMIT = 512.0     # 2^(+-512): the circle search stops there


def _circle_region(r):
    if r == 1.0:
        return (REGION_UNIT_CIRCLE, 0.0, 1.0)
    return (REGION_CIRCLE, 0.0, r)


def pencil_schur(A, B, seed=0, leaf_size=64, tau=None, maxit=60, split_tol=None, max_fail=8):
    """Generalized real Schur form of a regular pencil by RGNEP recursion.

    Strategy (Sec. 3.5): the root first divides on circles |z| = r about the
    origin: r = 1; if every eigenvalue is inside, r = 1/2, 1/4, 1/16, ...
    (r <- r^2); if every one is outside, r = 2, 4, 16, ...  A circle that
    divides splits the node: the inside group keeps the orientation and lies
    in |z| < r, the outside group continues as the swapped pencil (B, A),
    whose eigenvalues 1/lambda lie in |z| < 1/r.  If the search runs past the
    last circle holding everything inside (outside), that circle bounds the
    spectrum (the node is swapped in the second case) and the node goes on
    with real lines.  Below the root: real lines Re z = sigma over [-b, b], b
    the bound of the node, sigma uniform in the middle half of [lo, hi], with
    the empty-side rule of the symmetric strategy (reading: real lines, as
    for RNEP).  Readings where the paper is silent: a circle whose IRS does
    not converge, or that splits but fails the split test, is retried with
    its radius times 2^((2 xi - 1)/4) (xi the node's Philox uniform for the
    attempt) and counts as a failure; the search stops at 2^(+-512).
    Leaves by pencil_schur_leaf in the node's orientation (a swapped leaf
    factorises A, which is well conditioned there, so infinite eigenvalues are
    allowed).  Returns (S, T, QL, QR, alpha_re, alpha_im, beta, info) with
    QL^T A QR = S quasi-upper-triangular and QL^T B QR = T upper.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n = A.shape[0]
    info = SolveInfo()
    QL = np.eye(n)
    QRm = np.eye(n)
    leaves = []
    work = [(0, n, A.copy(), B.copy(), -1.0, 1.0, False, ROOT_NODE, 0)]
    while work:
        off, m, An, Bn, lo, hi, swapped, node, depth = work.pop()
        info.nodes += 1
        info.depth = max(info.depth, depth)
        if m <= leaf_size:
            leaves.append((off, m, An, Bn, swapped))
            continue
        attempt = 0
        fails = 0
        circle = node == ROOT_NODE      # circle search phase
        r, r_prev, direction = 1.0, None, 0
        r_try = r
        while True:
            P, Qm = (Bn, An) if swapped else (An, Bn)
            if circle:
                region = _circle_region(r_try)
            else:
                c = 0.5 * (lo + hi)
                R = 0.5 * (hi - lo)
                xi = uniform_scalar(seed, PURPOSE_SHIFT, node, attempt)
                sigma = c + R * (xi - 0.5)
                region = (REGION_LINE, sigma, R)
            st = divide_step(P, Qm, region, seed, node, attempt, tau, maxit,
                             symmetric=False, split_tol=split_tol)
            info.iters.append(st.irs.iters)
            if st.accepted:
                k = st.k
                QL[:, off:off + m] = QL[:, off:off + m] @ st.QL
                QRm[:, off:off + m] = QRm[:, off:off + m] @ st.QR
                Ah = st.QL.T @ An @ st.QR
                Bh = st.QL.T @ Bn @ st.QR
                if circle:
                    # outside group (leading k) continues swapped, |1/z| < 1/r
                    rr = region[2]
                    c1 = (-1.0 / rr, 1.0 / rr, not swapped)
                    c2 = (-rr, rr, swapped)
                else:
                    c1 = (region[1], hi, swapped)
                    c2 = (lo, region[1], swapped)
                info.splits += 1
                work.append((off + k, m - k, Ah[k:, k:].copy(), Bh[k:, k:].copy(), c2[0], c2[1],
                             c2[2], child_node(node, 1), depth + 1))
                work.append((off, k, Ah[:k, :k].copy(), Bh[:k, :k].copy(), c1[0], c1[1], c1[2],
                             child_node(node, 0), depth + 1))
                break
            info.failed_attempts += 1
            empty = st.irs.converged and st.rank in (0, m)
            if circle and empty:
                inside = st.rank == 0
                if inside and direction > 0:
                    # all outside r_prev, all inside r: bounded after the swap
                    swapped, lo, hi, circle = not swapped, -1.0 / r_prev, 1.0 / r_prev, False
                elif not inside and direction < 0:
                    # all inside r_prev, all outside r: r_prev bounds them
                    lo, hi, circle = -r_prev, r_prev, False
                else:
                    direction = -1 if inside else 1
                    r_prev = r
                    r = (0.5 if inside else 2.0) if r == 1.0 else r * r
                    if abs(np.log2(r)) > RADIUS_EXP_LIMIT:
                        if inside:
                            lo, hi = -r_prev, r_prev
                        else:
                            swapped, lo, hi = not swapped, -1.0 / r_prev, 1.0 / r_prev
                        circle = False
                r_try = r
            elif circle:
                fails += 1
                xi = uniform_scalar(seed, PURPOSE_SHIFT, node, attempt)
                r_try = r * 2.0 ** (0.25 * (2.0 * xi - 1.0))
            elif region[0] == REGION_LINE and empty:
                if st.rank == 0:
                    hi = region[1]
                else:
                    lo = region[1]
            else:
                fails += 1
            attempt += 1
            if fails > max_fail or attempt > 250:
                info.status = STATUS_NO_SPLIT
                return None, None, QL, QRm, None, None, None, info
    wi_pattern = np.zeros(n)
    for off, m, An, Bn, sw in leaves:
        S, T, ZL, ZR, wil, ok = pencil_schur_leaf(An, Bn, swapped=sw)
        if S is None or not ok:
            info.status = STATUS_NO_CONVERGENCE
            return None, None, QL, QRm, None, None, None, info
        QL[:, off:off + m] = QL[:, off:off + m] @ ZL
        QRm[:, off:off + m] = QRm[:, off:off + m] @ ZR
        wi_pattern[off:off + m] = np.asarray(wil, dtype=np.float64)
    Sf = QL.T @ A @ QRm
    Tf = QL.T @ B @ QRm
    if split_real_pairs(Sf, Tf, QL, QRm, wi_pattern):
        Sf = QL.T @ A @ QRm
        Tf = QL.T @ B @ QRm
    S = quasi_triangular_part(Sf, wi_pattern)
    T = np.triu(Tf)
    ar, ai, be = pencil_eigenvalues(S, T, wi_pattern)
    return S, T, QL, QRm, ar, ai, be, info


def pair_quadratic(s, t):
    """Coefficients (a, b, c) of det(s - z t) = a z^2 + b z + c for a 2 x 2
    block s and an upper triangular t; the reversed polynomial c w^2 + b w + a
    has the roots w = 1/z (the swapped block (t, s))."""
    a = t[0, 0] * t[1, 1]
    b = -(s[0, 0] * t[1, 1] + s[1, 1] * t[0, 0] - s[1, 0] * t[0, 1])
    c = s[0, 0] * s[1, 1] - s[0, 1] * s[1, 0]
    return a, b, c


def _rotation_from(vec):
    """2 x 2 rotation whose first column is vec / |vec| (identity for vec = 0)."""
    r = float(np.hypot(vec[0], vec[1]))
    if r == 0.0:
        return np.eye(2)
    x0, x1 = vec[0] / r, vec[1] / r
    return np.array([[x0, -x1], [x1, x0]])


def split_real_pairs(S, T, QL, QR, wi):
    """Split the 2 x 2 blocks marked as complex pairs (wi[i] > 0, wi[i+1] =
    -wi[i]) whose generalized eigenvalues are real, in place on QL, QR, wi.

    A leaf's Francis iteration can leave two nearly equal real eigenvalues of
    M (for instance a multiple eigenvalue at infinity seen as mu = 0 in a
    swapped leaf) as a 2 x 2 block with a tiny imaginary part; in the (S, T)
    frame that block may have real eigenvalues, which a generalized real Schur
    form keeps in 1 x 1 blocks.  For a real eigenvalue alpha/beta (taken in
    the orientation with the larger leading coefficient), x spans the null
    space of beta S2 - alpha T2 (orthogonal to its larger row), Z rotates e1
    onto x and Q rotates e1 onto S2 x (or T2 x): Q^T S2 Z and Q^T T2 Z are then
    upper triangular.  Returns True if a block was split."""
    n = S.shape[0]
    changed = False
    i = 0
    while i < n - 1:
        if not (wi[i] > 0.0 and wi[i + 1] == -wi[i]):
            i += 1
            continue
        s = S[i:i + 2, i:i + 2]
        t = np.triu(T[i:i + 2, i:i + 2])
        a, b, c = pair_quadratic(s, t)
        disc = b * b - 4.0 * a * c
        if disc < 0.0 or (a == 0.0 and c == 0.0):
            i += 2
            continue
        r = np.sqrt(disc)
        q = -0.5 * (b + (r if b >= 0.0 else -r))     # the larger-magnitude root term
        if abs(a) >= abs(c):
            alpha, beta = (q / a if q != 0.0 else 0.0), 1.0
        else:
            alpha, beta = 1.0, (q / c if q != 0.0 else 0.0)
        N = beta * s - alpha * t
        row = N[0] if np.hypot(*N[0]) >= np.hypot(*N[1]) else N[1]
        Z = _rotation_from(np.array([-row[1], row[0]]))
        x = Z[:, 0]
        u, v = s @ x, t @ x
        Q = _rotation_from(u if np.hypot(*u) >= np.hypot(*v) else v)
        QR[:, i:i + 2] = QR[:, i:i + 2] @ Z
        QL[:, i:i + 2] = QL[:, i:i + 2] @ Q
        wi[i] = wi[i + 1] = 0.0
        changed = True
        i += 2
    return changed


def pencil_eigenvalues(S, T, wi):
    """(alpha_re, alpha_im, beta) from a quasi-triangular S and triangular T:
    1x1 blocks give (s_ii, 0, t_ii); a 2x2 block (marked by wi[i] > 0 and
    wi[i+1] = -wi[i]) gives its roots of det(S_blk - z T_blk) = 0, solved in
    the orientation with the larger leading coefficient: z = alpha with
    beta = 1 if |det T_blk| >= |det S_blk|, else the roots w = p +- i q of the
    swapped block give alpha = p -+ i q, beta = p^2 + q^2 (z = alpha / beta).
    The first index of a pair carries the positive imaginary part."""
    n = S.shape[0]
    ar, ai, be = np.zeros(n), np.zeros(n), np.zeros(n)
    i = 0
    while i < n:
        if i + 1 < n and wi[i] > 0.0 and wi[i + 1] == -wi[i]:
            s = S[i:i + 2, i:i + 2]
            t = np.triu(T[i:i + 2, i:i + 2])
            a, b, c = pair_quadratic(s, t)
            disc = b * b - 4 * a * c
            lead, const = (a, c) if abs(a) >= abs(c) else (c, a)
            if disc < 0:
                re = -b / (2 * lead)
                im = np.sqrt(-disc) / (2 * abs(lead))
                if abs(a) >= abs(c):
                    vals = [(re, im, 1.0), (re, -im, 1.0)]
                else:
                    m2 = re * re + im * im
                    vals = [(re, im, m2), (re, -im, m2)]
            else:
                r = np.sqrt(disc)
                w1 = (-b + r) / (2 * lead)
                w2 = (-b - r) / (2 * lead)
                if abs(a) >= abs(c):
                    vals = [(w1, 0.0, 1.0), (w2, 0.0, 1.0)]
                else:
                    vals = [(1.0, 0.0, w1), (1.0, 0.0, w2)]
            (ar[i], ai[i], be[i]), (ar[i + 1], ai[i + 1], be[i + 1]) = vals
            i += 2
        else:
            ar[i], ai[i], be[i] = S[i, i], 0.0, T[i, i]
            i += 1
    return ar, ai, be


def quasi_triangular_part(T, wi):
    """Zero everything below the diagonal except the 2x2 blocks of complex pairs."""
    n = T.shape[0]
    out = np.triu(T)
    i = 0
    while i < n - 1:
        if wi[i] != 0.0 and wi[i + 1] == -wi[i]:
            out[i + 1, i] = T[i + 1, i]
            i += 2
        else:
            i += 1
    return out
