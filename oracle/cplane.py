"""Complex-plane strategy for the nonsymmetric problem (Sec. 3.3), oracle side.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.3 (B = I): find a disk of radius R holding every eigenvalue (Gershgorin),
draw an angle theta uniformly in [0, 2 pi), the radial line at that angle
meets the concentric circle of radius R/2 in a diameter, pick a point a
uniformly on that diameter and split along the line L through a perpendicular
to it.  A step makes progress when it splits, or when it shows that one side
of L holds no eigenvalue (that part of the disk is chopped off).  After one
such chop the next line is drawn perpendicular to the first chord, again at
most R/2 from the centre; a second chop leaves a region that fits in a circle
of radius at most sin(5 pi/12) R, on which the search restarts (the 2-step
radius shrink).  After a split each block takes the Gershgorin disk of its
own matrix.  A cluster that no line splits is, per the remarks of Sec. 3.3,
returned with a convex enclosure: the disk cut by the half-planes found empty.

One step on a line: write the line as {z : Re(conj(w) z) = t}, |w| = 1,
w = e^{i theta}, t = a + Re(conj(w) c) for a disk centred at c.  The Moebius
map of Sec. 3.3, rotated by w, sends (A, I) to
    A_0 = A - w (t - s) I,   B_0 = A - w (t + s) I,
whose eigenvalue f(z) = (z - w(t - s)) / (z - w(t + s)) lies outside the
unit circle exactly when Re(conj(w) z) > t (scale s = R, as for real lines).
Then IRS (Algorithm 3, conjugate transposes), the splitter
Q = GRURV(2, A_p + B_p, A_p, -1, +1) with a Haar unitary V (Algorithm 2),
A^ = Q^H A Q and the block size k minimising ||E21||_1 / ||A||_1
(Algorithm 5).  The leading k columns of Q span the invariant subspace of the
eigenvalues with Re(conj(w) z) > t.

Readings (paper silent):
  * root: the Gershgorin disk about the mean eigenvalue c = tr(A)/n, radius
    the smaller of the row and the column bound of A - c I.  After a split a
    child takes the smaller of the disk |z - c| <= ||A_ii - c I||_F (c its
    mean eigenvalue) and the smallest circle enclosing the parent region cut
    by the child's side of the line.  Sec. 3.3 names Gershgorin bounds there;
    but the splitter's trailing columns span the complementary invariant
    subspace in a basis that rounding picks (A_p is numerically rank
    deficient, so the QR of A_p V^H fixes only its leading columns), and a
    Gershgorin radius changes with that basis while the Frobenius norm and the
    trace do not;
  * draws: u1, u2 of the Philox pair of purpose PURPOSE_LINE for the node
    and attempt; theta = 2 pi u2, a = R (u1 - 1/2); the perpendicular line
    of the 2-step rule uses w' = i w and the same a rule;
  * side of an unsplit node: the numerical rank of the RURV factor as for
    real lines (rank 0: nothing right of L, rank n: nothing left of it);
  * recentering: the enclosing circle of the region (disk cut by the chopped
    half-planes) is the smallest one through the region's corner points, used
    when it also holds the region's arcs (otherwise the disk is kept).  The
    search moves to it after one chop when its radius is at most
    sin(5 pi/12) R (a small cap kept), else after the second chop, the one
    on the perpendicular line (the 2-step rule);
  * a step that converges to 0 < k < n with e(k) > split_tol, or does not
    converge, is a failed attempt; after max_fail of them the node is a
    cluster: with enclose=True it is reported with its region and put in
    Schur form by the leaf solver, otherwise the solve stops with NO_SPLIT;
  * A^ is not symmetrised; the leaves use the complex QR iteration
    (complex_leaf.complex_schur).

IRS on a pencil (A_j, B_j): the last n columns of the 2n x 2n unitary of the
QR of [B_j; -A_j] form Q12, Q22.  They are unique only up to a right unitary
factor, so A_p and B_p depend on the reflector convention while R_j and the
splitter Q do not (Q R_j and (A_p + B_p)^{-1} A_p are invariant).

Pinned by tests/test_oracle_complex.py: A_p^{-1} B_p = (A^{-1} B)^(2^p) by
long-double complex elimination, R_j against an independent Cholesky, the line
map's side count on prescribed spectra, the splitter's subspace against the
exact invariant subspace, the enclosing-circle geometry (sin(5 pi/12) R for
the worst 2-step case, R / sqrt(2) for a quarter disk, the half-chord for a
cap) and the drivers on prescribed spectra, the near-axis and the Jordan
examples of Sec. 3.3.1.
"""
import numpy as np

from .complex_qr import cqr_factor, cqr_explicit, crq_explicit, chaar
from .complex_leaf import complex_schur
from .irs import default_tau
from .philox import uniform_pairs, attempt_code, ROOT_NODE, child_node
from .solve import default_split_tol, STATUS_OK, STATUS_NO_SPLIT, STATUS_NO_CONVERGENCE

PURPOSE_LINE = 8
SHRINK = float(np.sin(5.0 * np.pi / 12.0))    # the 2-step bound on the new radius


# ----------------------------------------------------------- one step

def norm1(X):
    X = np.asarray(X)
    if X.size == 0:
        return 0.0
    return float(np.max(np.sum(np.abs(X), axis=0)))


def line_map(A, w, t, s):
    """(A_0, B_0) = (A - w (t - s) I, A - w (t + s) I) (rotated Moebius map)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    I = np.eye(n, dtype=np.complex128)
    return A - w * (t - s) * I, A - w * (t + s) * I


class CIRSResult:
    def __init__(self, Ap, Bp, iters, converged, ratios, Rs):
        self.Ap = Ap
        self.Bp = Bp
        self.iters = iters
        self.converged = converged
        self.ratios = ratios
        self.Rs = Rs


def cirs_step(Aj, Bj):
    """One squaring over C: returns (A_{j+1}, B_{j+1}, R_j)."""
    n = Aj.shape[0]
    f = cqr_factor(np.vstack([Bj, -Aj]))
    E = np.zeros((2 * n, n), dtype=np.complex128)
    E[n:, :] = np.eye(n)
    Y = f.q_times(E)
    Q12, Q22 = Y[:n, :], Y[n:, :]
    return Q12.conj().T @ Aj, Q22.conj().T @ Bj, f.R


def cirs(A, B, tau=None, maxit=60, record_R=False):
    """Algorithm 3 over C, same stopping rule as the real oracle (irs.irs)."""
    Aj = np.array(A, dtype=np.complex128, copy=True)
    Bj = np.array(B, dtype=np.complex128, copy=True)
    n = Aj.shape[0]
    if tau is None:
        tau = default_tau(n)
    R_prev = None
    ratios, Rs = [], []
    j = 0
    while True:
        A_next, B_next, R = cirs_step(Aj, Bj)
        if record_R:
            Rs.append(R.copy())
        if R_prev is not None:
            den = norm1(R_prev)
            num = norm1(R - R_prev)
            ratio = num / den if den > 0.0 else (0.0 if num == 0.0 else np.inf)
            ratios.append(ratio)
            if ratio <= tau:
                return CIRSResult(A_next, B_next, j + 1, True, ratios, Rs)
        R_prev = R
        Aj, Bj = A_next, B_next
        j += 1
        if j > maxit:
            return CIRSResult(Aj, Bj, j, False, ratios, Rs)


def csplitter(Ap, Bp, V):
    """Q = GRURV(2, A_p + B_p, A_p, -1, +1) over C: (Q, R1, R2).

    RURV(A_p): A_p V^H = U R2; then RQ: U^H (A_p + B_p) = R1 Q1, Q = Q1^H, so
    (A_p + B_p)^{-1} A_p = Q R1^{-1} R2 V (the lemma after Algorithm 2).
    """
    U, R2 = cqr_explicit(np.asarray(Ap) @ V.conj().T)
    R1, Q1 = crq_explicit(U.conj().T @ (np.asarray(Ap) + np.asarray(Bp)))
    return Q1.conj().T, R1, R2


def numerical_rank(R2, R1, rel_tol=1e-8):
    """#{|R2_ii| > rel_tol max_i |R1_ii|} (the real oracle's rule, over C)."""
    d2 = np.abs(np.diag(R2))
    scale = float(np.max(np.abs(np.diag(R1)))) if R1.size else 0.0
    if d2.size == 0 or scale == 0.0:
        return 0
    return int(np.sum(d2 > rel_tol * scale))


def split_scores(Ahat):
    """||E21(k)||_1 for k = 1..n-1: column suffix sums, prefix max (Sec. 4.2.1)."""
    n = Ahat.shape[0]
    absA = np.abs(Ahat)
    S = np.zeros((n + 1, n))
    for i in range(n - 1, -1, -1):
        S[i] = S[i + 1] + absA[i]
    f = np.zeros(n)
    for k in range(1, n):
        f[k] = np.max(S[k, :k])
    return f[1:]


def choose_k(scores, n):
    """Smallest score; ties to the k closest to n/2, then the smaller k."""
    best = None
    for idx, val in enumerate(scores):
        k = idx + 1
        key = (val, abs(2 * k - n), k)
        if best is None or key < best[0]:
            best = (key, k)
    return best[1]


class CStep:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def line_step(A, w, t, s, seed, stream, attempt, tau=None, maxit=60, split_tol=None,
              v_draws=4):
    """One RNEP step on the line Re(conj(w) z) = t with scale s (Algorithm 5)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    if split_tol is None:
        split_tol = default_split_tol(n)
    A0, B0 = line_map(A, w, t, s)
    res = cirs(A0, B0, tau=tau, maxit=maxit)
    normA = norm1(A)
    out = None
    for draw in range(v_draws):
        V = chaar(n, seed, stream, attempt_code(attempt, draw))
        Q, R1, R2 = csplitter(res.Ap, res.Bp, V)
        rank = numerical_rank(R2, R1)
        Ahat = Q.conj().T @ A @ Q
        e_all = split_scores(Ahat) / (normA if normA > 0 else 1.0)
        k = choose_k(e_all, n) if n >= 2 else 0
        e = float(e_all[k - 1]) if n >= 2 else 0.0
        accepted = bool(res.converged and 0 < k < n and e <= split_tol)
        out = CStep(Q=Q, R1=R1, R2=R2, rank=rank, Ahat=Ahat, k=k, e=e, scores=e_all,
                    accepted=accepted, draw=draw, irs=res)
        if accepted or not res.converged or rank in (0, n):
            break
    return out


# ----------------------------------------------------------- geometry

class Region:
    """Disk |z - c| <= R cut by half-planes Re(conj(w) z) >= t, each (w, t)."""

    def __init__(self, c, R, halfplanes=()):
        self.c = complex(c)
        self.R = float(R)
        self.halfplanes = list(halfplanes)

    def contains(self, z, slack=1e-12):
        tol = slack * max(self.R, abs(self.c), 1e-300)
        if abs(z - self.c) > self.R + tol:
            return False
        return all((np.conj(w) * z).real >= t - tol for (w, t) in self.halfplanes)

    def copy(self):
        return Region(self.c, self.R, self.halfplanes)


def _line_circle(c, R, w, t):
    """Points of the circle |z - c| = R on the line Re(conj(w) z) = t."""
    d = t - (np.conj(w) * c).real        # signed distance of the line from c
    if abs(d) > R:
        return []
    h = np.sqrt(max(R * R - d * d, 0.0))
    foot = c + w * d
    return [foot + 1j * w * h, foot - 1j * w * h]


def _line_line(w1, t1, w2, t2):
    """Intersection of Re(conj(w1) z) = t1 and Re(conj(w2) z) = t2 (None if parallel)."""
    a11, a12 = w1.real, w1.imag
    a21, a22 = w2.real, w2.imag
    det = a11 * a22 - a12 * a21
    if abs(det) < 1e-14:
        return None
    x = (t1 * a22 - a12 * t2) / det
    y = (a11 * t2 - t1 * a21) / det
    return complex(x, y)


def _circle_2(p, q):
    return 0.5 * (p + q), 0.5 * abs(p - q)


def _circle_3(p, q, r):
    """Circumcircle of three points (None when collinear)."""
    ax, ay = p.real, p.imag
    bx, by = q.real, q.imag
    cx, cy = r.real, r.imag
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    if abs(d) < 1e-300:
        return None
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay)
          + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx)
          + (cx * cx + cy * cy) * (bx - ax)) / d
    m = complex(ux, uy)
    return m, abs(p - m)


def min_circle_points(pts):
    """Smallest circle holding a few points: brute force over pairs and triples."""
    pts = list(pts)
    if not pts:
        return None
    if len(pts) == 1:
        return pts[0], 0.0
    cands = []
    for i in range(len(pts)):
        for j in range(i + 1, len(pts)):
            cands.append(_circle_2(pts[i], pts[j]))
            for k in range(j + 1, len(pts)):
                c3 = _circle_3(pts[i], pts[j], pts[k])
                if c3 is not None:
                    cands.append(c3)
    best = None
    for m, r in cands:
        tol = 1e-12 * max(r, 1e-300)
        if all(abs(p - m) <= r + tol for p in pts):
            if best is None or r < best[1]:
                best = (m, r)
    return best


def enclosing_circle(region):
    """(centre, radius) of a circle holding the region; the disk if no smaller one.

    Corners: the chord ends inside the other half-planes and the pairwise
    line intersections inside the disk.  The smallest circle through them
    holds the region when it also holds the farthest point of the boundary
    circle (the point opposite its centre), if that point is in the region.
    """
    c, R = region.c, region.R
    if not region.halfplanes:
        return c, R
    corners = []
    for i, (w, t) in enumerate(region.halfplanes):
        for z in _line_circle(c, R, w, t):
            if region.contains(z):
                corners.append(z)
        for (w2, t2) in region.halfplanes[i + 1:]:
            z = _line_line(w, t, w2, t2)
            if z is not None and region.contains(z):
                corners.append(z)
    best = min_circle_points(corners)
    if best is None:
        return c, R
    m, r = best
    if r >= R or m == c:
        # a circle centred at c holding a point of the boundary circle is the disk
        return c, R
    # the distance from m to a point of the boundary circle grows monotonically
    # towards the point opposite m; if that point is in the region it is the
    # farthest one, otherwise the farthest region point on an arc is an arc end
    dm = m - c
    far = c - R * complex(dm.real / abs(dm), dm.imag / abs(dm))
    if region.contains(far) and abs(far - m) > r * (1.0 + 1e-12):
        return c, R
    return m, r


def gershgorin_disk(A):
    """(c, R): c = tr(A)/n, R the smaller of the row and column bounds of A - cI."""
    A = np.asarray(A)
    n = A.shape[0]
    c = complex(np.trace(A) / n)
    D = A - c * np.eye(n)
    absD = np.abs(D)
    diag = np.abs(np.diag(D))
    off = absD - np.diag(np.diag(absD))
    row = float(np.max(diag + np.sum(off, axis=1)))
    col = float(np.max(diag + np.sum(off, axis=0)))
    return c, min(row, col)


def frobenius_disk(A):
    """(c, R): c = tr(A)/n, R = ||A - c I||_F, a disk holding the spectrum.

    Unlike the Gershgorin radius, R does not change under a unitary change of
    basis, so it does not depend on which orthonormal basis of its invariant
    subspace a block was computed in (see the module docstring)."""
    A = np.asarray(A)
    n = A.shape[0]
    c = complex(np.trace(A) / n)
    D = A - c * np.eye(n)
    return c, float(np.sqrt(np.sum(np.abs(D) ** 2)))


# ----------------------------------------------------------- driver

class CInfo:
    def __init__(self):
        self.status = STATUS_OK
        self.nodes = 0
        self.splits = 0
        self.iters = []
        self.depth = 0
        self.failed_attempts = 0   # attempts that did not split (chops included)
        self.chops = 0
        self.recenters = []        # (node, old radius, new radius, "one chop" | "two chops")
        self.lines = []            # (node, attempt, w, t, outcome, disk centre, disk radius, rank)
        self.clusters = []         # (offset, size, Region)
        self.split_regions = []    # (node, Region, (w, t), [own disks], [child Regions])


def draw_line(region, seed, node, attempt, perpendicular_to=None):
    """(w, t) of the attempt's line: random angle, or perpendicular to a chord."""
    u1, u2 = uniform_pairs(1, seed, PURPOSE_LINE, node, attempt)
    u1, u2 = float(u1[0]), float(u2[0])
    if perpendicular_to is None:
        w = complex(np.cos(2.0 * np.pi * u2), np.sin(2.0 * np.pi * u2))
    else:
        w = 1j * perpendicular_to
    a = region.R * (u1 - 0.5)
    t = a + (np.conj(w) * region.c).real
    return w, t


def schur_complex_plane(A, seed=0, leaf_size=64, tau=None, maxit=60, split_tol=None,
                        max_fail=8, enclose=False, max_attempts=250):
    """(T, U, lam, info): A = U T U^H with T upper triangular, lam = diag(T).

    The recursion of Sec. 3.3 with lines at random angles; the readings are in
    the module docstring.  On NO_SPLIT, T is None.
    """
    A = np.asarray(A)
    n = A.shape[0]
    Ac = np.array(A, dtype=np.complex128)
    info = CInfo()
    U = np.eye(n, dtype=np.complex128)
    leaves = []
    c0, R0 = gershgorin_disk(Ac) if n else (0j, 0.0)
    work = [(0, n, Ac, Region(c0, R0), ROOT_NODE, 0)]
    while work:
        off, m, An, region, node, depth = work.pop()
        info.nodes += 1
        info.depth = max(info.depth, depth)
        if m <= leaf_size:
            leaves.append((off, m, An))
            continue
        attempt = 0
        fails = 0
        pending = None            # normal of the chord chopped since the last recentering
        while True:
            if region.R <= 0.0:
                # every Gershgorin disk is a point: A_node = c I
                leaves.append((off, m, An))
                break
            w, t = draw_line(region, seed, node, attempt, pending)
            st = line_step(An, w, t, region.R, seed, node, attempt, tau, maxit, split_tol)
            info.iters.append(st.irs.iters)
            if st.accepted:
                k = st.k
                U[:, off:off + m] = U[:, off:off + m] @ st.Q
                A11 = st.Ahat[:k, :k].copy()
                A22 = st.Ahat[k:, k:].copy()
                r1 = region.copy()
                r1.halfplanes.append((w, t))
                r2 = region.copy()
                r2.halfplanes.append((-w, -t))
                kids, own = [], []
                for Ab, rr in ((A11, r1), (A22, r2)):
                    cg, Rg = frobenius_disk(Ab)
                    own.append((cg, Rg))
                    ce, Re = enclosing_circle(rr)
                    kids.append(Region(cg, Rg) if Rg <= Re else Region(ce, Re))
                info.split_regions.append((node, region.copy(), (w, t), own, kids))
                info.splits += 1
                info.lines.append((node, attempt, w, t, "split", region.c, region.R, st.rank))
                work.append((off + k, m - k, A22, kids[1], child_node(node, 1), depth + 1))
                work.append((off, k, A11, kids[0], child_node(node, 0), depth + 1))
                break
            info.failed_attempts += 1
            if st.irs.converged and st.rank in (0, m):
                # nothing on one side of the line: chop it off
                info.chops += 1
                info.lines.append((node, attempt, w, t, "chop", region.c, region.R, st.rank))
                keep = (w, t) if st.rank == m else (-w, -t)
                region.halfplanes.append(keep)
                cn, rn = enclosing_circle(region)
                if rn <= SHRINK * region.R:
                    info.recenters.append((node, region.R, rn, "one chop"))
                    region = Region(cn, rn)
                    pending = None
                elif pending is None:
                    pending = w
                else:
                    if rn < region.R:
                        info.recenters.append((node, region.R, rn, "two chops"))
                        region = Region(cn, rn)
                    pending = None
            else:
                fails += 1
                info.lines.append((node, attempt, w, t, "fail", region.c, region.R, st.rank))
                pending = None
            attempt += 1
            if fails > max_fail or attempt > max_attempts:
                if enclose:
                    info.clusters.append((off, m, region.copy()))
                    leaves.append((off, m, An))
                    break
                info.status = STATUS_NO_SPLIT
                return None, U, np.zeros(n, dtype=np.complex128), info
    lam = np.zeros(n, dtype=np.complex128)
    for off, m, An in leaves:
        _, Zl, wl, good = complex_schur(An)
        if not good:
            info.status = STATUS_NO_CONVERGENCE
        U[:, off:off + m] = U[:, off:off + m] @ Zl
        lam[off:off + m] = wl
    T = np.triu(U.conj().T @ Ac @ U)
    return T, U, np.diag(T).copy(), info
