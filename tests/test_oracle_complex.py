"""Pins for the complex-plane oracle: complex QR / RQ, the Haar unitary, IRS over
C, the rotated line map, the splitter, the complex Schur leaf, the enclosing
circles of the 2-step rule and the driver of Sec. 3.3.

Each pin checks the oracle against something other than itself: a textbook
complex Cholesky, long-double complex elimination, closed forms, prescribed
spectra, Haar moments, plane geometry with known answers, and the Sec. 3.3.1
examples (eigenvalues near the imaginary axis, a Jordan block).
"""
import numpy as np
import pytest

from oracle.complex_qr import chouse, cqr_explicit, crq_explicit, chaar
from oracle.complex_leaf import complex_schur, chessenberg, wilkinson_shift
from oracle.cplane import (cirs, cirs_step, line_map, line_step, Region, enclosing_circle,
                           gershgorin_disk, schur_complex_plane, SHRINK)
from oracle import cplane
from oracle.irs import irs
from oracle.solve import STATUS_OK, STATUS_NO_SPLIT
from paper_1011_3077_gb300 import workloads
from tests.pinlib import cholesky_upper_c, ld_solve_c, subspace_residual_c

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _prescribed(lam, rng, coupling=0.25):
    """A = S diag(lam) S^-1 with a well-conditioned complex S."""
    n = len(lam)
    S = np.eye(n) + coupling * _crandn(rng, n, n) / np.sqrt(2 * n)
    Sinv = np.array(ld_solve_c(S, np.eye(n)), dtype=np.complex128)
    return S @ np.diag(lam) @ Sinv, S


def _match(got, want):
    """Largest distance after greedy nearest matching of two multisets."""
    got = list(np.asarray(got, dtype=np.complex128))
    worst = 0.0
    for z in want:
        i = int(np.argmin([abs(g - z) for g in got]))
        worst = max(worst, abs(got[i] - z))
        got.pop(i)
    return worst


# ------------------------------------------------------------ QR / RQ / Haar

@pytest.mark.parametrize("m,n", [(9, 6), (6, 6), (12, 1)])
def test_cqr_is_unique_cholesky_factor(m, n):
    rng = np.random.default_rng(11 + m)
    X = _crandn(rng, m, n)
    Q, R = cqr_explicit(X)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < 1e-14
    assert np.abs(Q @ R - X).max() < 1e-13 * np.abs(X).max() * m
    assert np.abs(np.tril(R, -1)).max() == 0.0
    assert np.all(np.diag(R).real >= 0.0) and np.all(np.diag(R).imag == 0.0)
    Rc = cholesky_upper_c(X.conj().T @ X)
    assert np.abs(R - Rc).max() < 1e-12 * np.abs(Rc).max()


def test_cqr_phase_of_a_multiple_of_e1():
    X = np.zeros((4, 2), dtype=np.complex128)
    X[0, 0] = 3j
    X[:, 1] = [1.0, 2.0j, 0.0, -1.0]
    Q, R = cqr_explicit(X)
    assert abs(R[0, 0] - 3.0) < 1e-15
    assert np.abs(Q[:, 0] - np.array([1j, 0, 0, 0])).max() < 1e-15
    v, mu = chouse(np.zeros(3))
    assert v is None and mu == 0.0


def test_crq_identity():
    rng = np.random.default_rng(5)
    Y = _crandn(rng, 7, 7)
    R, Q = crq_explicit(Y)
    assert np.abs(R @ Q - Y).max() < 1e-13 * np.abs(Y).max() * 7
    assert np.abs(Q @ Q.conj().T - np.eye(7)).max() < 1e-14
    assert np.abs(np.tril(R, -1)).max() == 0.0
    assert np.all(np.diag(R).real >= 0.0) and np.all(np.diag(R).imag == 0.0)


def test_chaar_moments():
    # Haar on U(n): E|V_ij|^2 = 1/n, E V_ij^2 = 0, E|tr V|^2 = 1
    n, draws = 3, 1500
    sq, sq2, tr2 = 0.0, 0.0 + 0.0j, 0.0
    for d in range(draws):
        V = chaar(n, seed=77, stream=1000 + d)
        assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-14
        sq += float(np.mean(np.abs(V) ** 2))
        sq2 += complex(np.mean(V * V))
        tr2 += abs(np.trace(V)) ** 2
    assert abs(sq / draws - 1.0 / n) < 1e-12      # rows are unit vectors
    assert abs(sq2 / draws) < 0.05
    assert abs(tr2 / draws - 1.0) < 0.12


# ------------------------------------------------------------ IRS over C

def _pencil_with_quotient(rng, n, mu):
    """(A, B) with A^{-1} B = M, M = S diag(mu) S^{-1}."""
    A = _crandn(rng, n, n) + 2.0 * np.eye(n)
    M, _ = _prescribed(mu, rng)
    return A, A @ M, M


def test_cirs_squares_the_quotient():
    rng = np.random.default_rng(21)
    n = 5
    mu = np.array([0.5, 1.4j, -1.2, 0.7 - 0.6j, 1.3 + 0.2j])
    A, B, M = _pencil_with_quotient(rng, n, mu)
    Aj, Bj = A, B
    for j in range(3):
        An, Bn, R = cirs_step(Aj, Bj)
        Rc = cholesky_upper_c(Aj.conj().T @ Aj + Bj.conj().T @ Bj)
        assert np.abs(R - Rc).max() < 1e-11 * np.abs(Rc).max()
        Aj, Bj = An, Bn
    got = np.array(ld_solve_c(Aj, Bj), dtype=np.complex128)
    M8 = np.linalg.matrix_power(M, 8)
    assert np.linalg.norm(got - M8) < 1e-10 * np.linalg.norm(M8)


def test_cirs_on_a_real_pencil_matches_the_real_oracle():
    rng = np.random.default_rng(22)
    n = 6
    A = rng.standard_normal((n, n)) + 3.0 * np.eye(n)
    B = rng.standard_normal((n, n))
    rc = cirs(A, B, maxit=6, record_R=True)
    rr = irs(A, B, maxit=6, record_R=True)
    assert rc.iters == rr.iters and rc.converged == rr.converged
    for Rcj, Rrj in zip(rc.Rs, rr.Rs):
        assert np.abs(Rcj - Rrj).max() < 1e-12 * max(1.0, np.abs(Rrj).max())


# ------------------------------------------------------------ line map, splitter

def test_line_map_sends_the_half_plane_outside_the_unit_circle():
    rng = np.random.default_rng(31)
    lam = _crandn(rng, 40)
    for _ in range(20):
        w = np.exp(2j * np.pi * rng.uniform())
        t = rng.uniform(-1, 1)
        s = rng.uniform(0.5, 3.0)
        A0, B0 = line_map(np.diag(lam), w, t, s)
        mu = np.diag(A0) / np.diag(B0)
        right = (np.conj(w) * lam).real > t
        assert np.array_equal(np.abs(mu) > 1.0, right)
        # a point on the line maps onto the unit circle
        z = w * (t + 1j * rng.uniform(-2, 2))
        A1, B1 = line_map(np.array([[z]]), w, t, s)
        assert abs(abs(A1[0, 0] / B1[0, 0]) - 1.0) < 1e-12


def test_splitter_spans_the_invariant_subspace_right_of_the_line():
    rng = np.random.default_rng(41)
    w = np.exp(0.7j)
    t = 0.2
    n = 10
    # four eigenvalues right of Re(conj(w) z) = t, six left, margin >= 0.3
    along = np.array([0.9, 1.2, 0.6, 1.5, -0.4, -0.9, -0.2, -1.3, -0.6, -0.1])
    across = rng.uniform(-1.0, 1.0, n)
    lam = w * (along + 1j * across)
    A, S = _prescribed(lam, rng)
    st = line_step(A, w, t, 2.0, seed=5, stream=1, attempt=0)
    assert st.accepted and st.k == 4 and st.rank == 4
    right = (np.conj(w) * lam).real > t
    assert subspace_residual_c(st.Q[:, :4], S[:, right]) < 1e-10
    assert np.abs(st.Ahat[4:, :4]).max() < 1e-12 * np.abs(A).max()
    _, _, w11, ok = complex_schur(st.Ahat[:4, :4])
    assert ok and _match(w11, lam[right]) < 1e-10


# ------------------------------------------------------------ complex Schur leaf

def test_complex_schur_2x2_closed_form():
    rng = np.random.default_rng(51)
    for _ in range(10):
        A = _crandn(rng, 2, 2)
        tr = A[0, 0] + A[1, 1]
        det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
        r = np.sqrt(tr * tr / 4.0 - det + 0j)
        T, Z, w, ok = complex_schur(A)
        assert ok and T[1, 0] == 0.0
        assert _match(w, [tr / 2 + r, tr / 2 - r]) < 1e-13 * (1 + abs(tr))
        assert np.abs(Z @ T @ Z.conj().T - A).max() < 1e-14 * 4


def test_chessenberg_structure():
    rng = np.random.default_rng(52)
    A = _crandn(rng, 9, 9)
    H, Z = chessenberg(A)
    assert np.abs(np.tril(H, -2)).max() == 0.0
    assert np.abs(Z.conj().T @ Z - np.eye(9)).max() < 1e-14
    assert np.abs(Z @ H @ Z.conj().T - A).max() < 1e-13


def test_wilkinson_shift_is_the_closer_eigenvalue():
    a, b, c, d = 1.0, 2.0, 0.5, 3.0          # eigenvalues 2 +- sqrt(2)
    assert abs(wilkinson_shift(a, b, c, d) - (2 + np.sqrt(2))) < 1e-15


@pytest.mark.parametrize("n", [7, 24])
def test_complex_schur_prescribed_spectrum(n):
    rng = np.random.default_rng(53 + n)
    lam = _crandn(rng, n)
    A, _ = _prescribed(lam, rng)
    T, Z, w, ok = complex_schur(A)
    assert ok
    assert np.abs(np.tril(T, -1)).max() == 0.0
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() < 1e-13
    assert np.linalg.norm(Z @ T @ Z.conj().T - A) < 1e-14 * n * np.linalg.norm(A)
    assert _match(w, lam) < 1e-11


def test_complex_schur_of_a_real_matrix_with_pairs():
    A, _ = workloads.normal_complex(20, seed=3)
    T, Z, w, ok = complex_schur(A)
    assert ok
    assert _match(w, np.linalg.eigvals(A)) < 1e-12
    assert np.linalg.norm(Z @ T @ Z.conj().T - A) < 1e-13 * np.linalg.norm(A)


# ------------------------------------------------------------ geometry

def test_two_step_worst_case_radius_is_sin_5pi_12():
    # chord at distance R/2 keeps Re z >= -R/2, perpendicular chord keeps Im z <= R/2
    for R, c in [(1.0, 0j), (3.0, 1.0 - 2.0j)]:
        reg = Region(c, R, [(1.0 + 0j, c.real - R / 2), (-1j, -c.imag - R / 2)])
        m, r = enclosing_circle(reg)
        assert abs(r - np.sin(5 * np.pi / 12) * R) < 1e-12 * R
        # centre: midpoint of the arc ends at angles 30 and 240 degrees
        p1 = c + R * np.exp(1j * np.pi / 6)
        p2 = c + R * np.exp(1j * 4 * np.pi / 3)
        assert abs(m - 0.5 * (p1 + p2)) < 1e-12 * R
    assert abs(SHRINK - 0.9659258262890683) < 1e-15


def test_quarter_disk_and_caps():
    m, r = enclosing_circle(Region(0, 2.0, [(1.0 + 0j, 0.0), (-1j, 0.0)]))
    assert abs(r - 2.0 / np.sqrt(2)) < 1e-12 and abs(m - (1.0 - 1.0j)) < 1e-12
    d = 0.6
    m, r = enclosing_circle(Region(0, 1.0, [(1.0 + 0j, d)]))        # small cap kept
    assert abs(r - np.sqrt(1 - d * d)) < 1e-12 and abs(m - d) < 1e-12
    m, r = enclosing_circle(Region(0, 1.0, [(1.0 + 0j, -d)]))       # large side kept
    assert r == 1.0 and m == 0


def _sample_region(reg, rng, count):
    pts = []
    for _ in range(10000 * count):
        if len(pts) == count:
            break
        z = reg.c + reg.R * np.sqrt(rng.uniform()) * np.exp(2j * np.pi * rng.uniform())
        if reg.contains(z, slack=0.0):
            pts.append(z)
    return np.array(pts)


def test_enclosing_circle_holds_random_regions():
    rng = np.random.default_rng(61)
    for trial in range(60):
        c = complex(*rng.uniform(-1, 1, 2))
        R = rng.uniform(0.5, 2.0)
        anchor = c + 0.3 * R * np.exp(2j * np.pi * rng.uniform())   # kept by every cut
        hps = []
        for _ in range(int(rng.integers(1, 4))):
            w = np.exp(2j * np.pi * rng.uniform())
            t = (np.conj(w) * c).real + R * rng.uniform(-0.5, 0.5)
            hps.append((w, t) if (np.conj(w) * anchor).real >= t else (-w, -t))
        reg = Region(c, R, hps)
        m, r = enclosing_circle(reg)
        assert r <= R
        pts = _sample_region(reg, rng, 300)
        assert np.all(np.abs(pts - m) <= r * (1 + 1e-12))
        # the region's arc points too: the boundary circle inside the half-planes
        phi = np.linspace(0, 2 * np.pi, 2000, endpoint=False)
        arc = [z for z in c + R * np.exp(1j * phi) if reg.contains(z, slack=0.0)]
        assert all(abs(z - m) <= r * (1 + 1e-12) for z in arc)


def test_two_perpendicular_chops_always_shrink():
    rng = np.random.default_rng(62)
    for _ in range(200):
        R = 1.0
        w = np.exp(2j * np.pi * rng.uniform())
        s1 = 1 if rng.uniform() < 0.5 else -1
        s2 = 1 if rng.uniform() < 0.5 else -1
        a1, a2 = rng.uniform(-0.5, 0.5, 2)
        reg = Region(0, R, [(s1 * w, s1 * a1), (s2 * 1j * w, s2 * a2)])
        _, r = enclosing_circle(reg)
        assert r <= SHRINK * R + 1e-12


def test_gershgorin_disk_holds_the_spectrum():
    rng = np.random.default_rng(63)
    for n in (3, 8, 20):
        lam = _crandn(rng, n)
        A, _ = _prescribed(lam, rng, coupling=0.6)
        c, R = gershgorin_disk(A)
        assert abs(c - np.mean(lam)) < 1e-12 * n
        assert np.all(np.abs(lam - c) <= R * (1 + 1e-12))


def test_frobenius_disk_holds_the_spectrum_and_ignores_the_basis():
    rng = np.random.default_rng(64)
    for n in (2, 9, 30):
        lam = _crandn(rng, n)
        A, _ = _prescribed(lam, rng, coupling=0.6)
        c, R = cplane.frobenius_disk(A)
        assert abs(c - np.mean(lam)) < 1e-12 * n
        assert np.all(np.abs(lam - c) <= R * (1 + 1e-12))
        W = cqr_explicit(_crandn(rng, n, n))[0]
        c2, R2 = cplane.frobenius_disk(W.conj().T @ A @ W)
        assert abs(c2 - c) < 1e-12 * n and abs(R2 - R) < 1e-12 * R
        cg, Rg = gershgorin_disk(W.conj().T @ A @ W)
        assert abs(Rg - gershgorin_disk(A)[1]) > 1e-6      # the Gershgorin radius does move


# ------------------------------------------------------------ driver

def _check_schur(A, T, U, tol):
    n = A.shape[0]
    assert np.abs(np.tril(T, -1)).max() == 0.0
    assert np.abs(U.conj().T @ U - np.eye(n)).max() < 1e-12
    assert np.linalg.norm(U @ T @ U.conj().T - A) < tol * np.linalg.norm(A)


def test_driver_prescribed_complex_spectrum():
    rng = np.random.default_rng(71)
    n = 40
    lam = _crandn(rng, n)
    A, _ = _prescribed(lam, rng)
    T, U, w, info = schur_complex_plane(A, seed=2, leaf_size=8)
    assert info.status == STATUS_OK and info.splits >= 4
    _check_schur(A, T, U, 1e-13)
    assert _match(w, lam) < 1e-10
    # every line lies at most R/2 from the centre of its disk
    for (_, _, wl, t, _, c, R, _) in info.lines:
        assert abs(t - (np.conj(wl) * c).real) <= 0.5 * R * (1 + 1e-12)


def test_driver_eigenvalues_near_the_imaginary_axis():
    # Sec. 3.3.1: real parts +-1e-10, imaginary parts in [-1.5, 1.5]
    A = workloads.near_axis(25)
    T, U, w, info = schur_complex_plane(A, seed=3, leaf_size=4)
    assert info.status == STATUS_OK and info.splits >= 3
    _check_schur(A, T, U, 1e-13)
    assert _match(w, np.linalg.eigvals(A)) < 1e-12


def test_driver_reports_the_jordan_cluster_with_an_enclosure():
    # Sec. 3.3.1: a 16 x 16 Jordan block at 0.1 next to 16 eigenvalues with
    # negative real part; no line splits the block's pseudospectrum
    A = workloads.jordan_hard(32)
    T, U, w, info = schur_complex_plane(A, seed=1, leaf_size=4, enclose=True)
    assert info.status == STATUS_OK
    _check_schur(A, T, U, 1e-12)
    clusters = [(off, m, reg) for off, m, reg in info.clusters if reg.contains(0.1)]
    assert len(clusters) == 1
    off, m, reg = clusters[0]
    assert m >= 16
    assert all(reg.contains(z) for z in w[off:off + m])
    # the eigenvalues outside the cluster are the well-conditioned negative ones
    rest = np.concatenate([w[:off], w[off + m:]])
    assert len(rest) == 32 - m
    ev = np.linalg.eigvals(A)
    neg = ev[ev.real < -0.01]
    for z in rest:
        assert np.min(np.abs(neg - z)) < 1e-9
    _, _, _, info2 = schur_complex_plane(A, seed=1, leaf_size=4, enclose=False)
    assert info2.status == STATUS_NO_SPLIT


def test_driver_two_step_rule_on_a_loose_disk():
    # a strongly non-normal matrix: the Gershgorin disk is far larger than
    # the spectrum, so lines chop empty parts and the disk shrinks
    rng = np.random.default_rng(81)
    n = 24
    lam = 0.05 * _crandn(rng, n)
    N = np.triu(_crandn(rng, n, n), 1)
    Qh = cqr_explicit(_crandn(rng, n, n))[0]
    A = Qh @ (np.diag(lam) + 0.3 * N) @ Qh.conj().T
    T, U, w, info = schur_complex_plane(A, seed=4, leaf_size=6, enclose=True)
    assert info.status == STATUS_OK
    _check_schur(A, T, U, 1e-12)
    assert info.chops >= 2 and len(info.recenters) >= 1
    for (_, old, new, why) in info.recenters:
        assert new <= SHRINK * old * (1 + 1e-12) or why == "two chops"
        assert new < old
    # after a chop that did not move the disk, the next line of the node is perpendicular
    lines = info.lines
    for i in range(len(lines) - 1):
        node, att, wl, _, outcome, c, R, _ = lines[i]
        nn, natt, wn, _, _, cn, Rn, _ = lines[i + 1]
        if outcome == "chop" and nn == node and cn == c and Rn == R:
            prev_perp = i > 0 and lines[i - 1][0] == node and lines[i - 1][4] == "chop" \
                and lines[i - 1][5] == c and lines[i - 1][6] == R
            if not prev_perp:
                assert abs(wn - 1j * wl) < 1e-15


def test_rotating_the_plane_leaves_the_step_unchanged():
    # (e^{i phi} A, line e^{i phi} w) maps to e^{i phi} times the same pencil:
    # the R_j of IRS (non-negative diagonal) and the step's decisions agree
    rng = np.random.default_rng(91)
    n = 30
    lam = 1.5 * _crandn(rng, n)
    A, _ = _prescribed(lam, rng)
    w, t, s = np.exp(0.3j), 0.1, 3.0
    phi = np.exp(1.1j)
    r0 = cirs(*line_map(A, w, t, s), record_R=True)
    r1 = cirs(*line_map(phi * A, phi * w, t, s), record_R=True)
    assert r0.iters == r1.iters and r0.converged and r1.converged
    for R0, R1 in zip(r0.Rs, r1.Rs):
        assert np.abs(R0 - R1).max() <= 1e-12 * np.abs(R0).max()
    s0 = line_step(A, w, t, s, seed=4, stream=9, attempt=0)
    s1 = line_step(phi * A, phi * w, t, s, seed=4, stream=9, attempt=0)
    assert (s0.k, s0.rank, s0.accepted) == (s1.k, s1.rank, s1.accepted)


def test_squarings_follow_the_distance_to_a_rotated_line():
    # Sec. 3.3.1, Fig. 1 with the line at an angle: normal matrices whose
    # nearest eigenvalue sits 4e-3 from the line take the same number of
    # squarings at n = 60 and n = 200
    w, t = np.exp(0.8j), 0.05
    counts = []
    for n, seed in ((60, 1), (200, 2)):
        rng = np.random.default_rng(seed)
        along = rng.uniform(-1.5, 1.5, n)
        along = np.where(np.abs(along - t) < 4e-3, t + 4e-3 * np.sign(along - t + 1e-300), along)
        along[np.argmin(np.abs(along - t))] = t + 4e-3
        lam = w * (along + 1j * rng.uniform(-1.5, 1.5, n))
        W = cqr_explicit(_crandn(rng, n, n))[0]
        A = W @ np.diag(lam) @ W.conj().T
        res = cirs(*line_map(A, w, t, 3.0))
        assert res.converged
        counts.append(res.iters)
    assert abs(counts[0] - counts[1]) <= 1


@pytest.mark.parametrize("field", ["real", "complex"])
def test_rurv_is_rank_revealing(field):
    # Theorem 2.1 (RURV is a strong rank-revealing factorisation w.h.p.):
    # sigma_max(R22) >= sigma_{r+1} always (interlacing); with high probability
    # sigma_min(R11) is within sqrt(r (n-r)) of sigma_r, ||R11^-1 R12|| = O(sqrt(r (n-r)))
    # and sigma_max(R22) is a small multiple of sigma_{r+1}.  The constants are
    # not stated; loose ones are checked on the median of 40 Haar draws.
    from oracle.rurv import haar, rurv
    from oracle.householder import qr_explicit
    rng = np.random.default_rng(93)
    n, r = 40, 10
    sig = np.concatenate([rng.uniform(1.0, 2.0, r), 1e-8 * rng.uniform(0.5, 1.0, n - r)])
    sig = -np.sort(-sig)
    if field == "real":
        P = qr_explicit(rng.standard_normal((n, n)))[0]
        Q = qr_explicit(rng.standard_normal((n, n)))[0]
    else:
        P = cqr_explicit(_crandn(rng, n, n))[0]
        Q = cqr_explicit(_crandn(rng, n, n))[0]
    A = (P * sig) @ Q.conj().T
    lo, hi, cross = [], [], []
    for d in range(40):
        if field == "real":
            V = haar(n, 5, 100 + d)
            _, R = rurv(A, V)
        else:
            V = chaar(n, 5, 100 + d)
            _, R = cqr_explicit(A @ V.conj().T)
        R11, R12, R22 = R[:r, :r], R[:r, r:], R[r:, r:]
        s11 = np.linalg.svd(R11, compute_uv=False)
        s22 = np.linalg.svd(R22, compute_uv=False)
        assert s22[0] >= sig[r] * (1 - 1e-6)
        assert s11[-1] <= np.sqrt(2) * sig[r - 1] * (1 + 1e-12)
        lo.append(s11[-1] * np.sqrt(r * (n - r)) / sig[r - 1])
        hi.append(s22[0] / sig[r])
        cross.append(np.linalg.norm(np.linalg.solve(R11, R12), 2) / np.sqrt(r * (n - r)))
    assert np.median(lo) >= 0.05
    assert np.median(hi) <= 1e3
    assert np.median(cross) <= 10.0


def test_squaring_count_follows_the_papers_distance_formula():
    # Sec. 3.3 (eqs. p-eq and d1): with d_L(A, I) the distance to the line,
    #   d_L = 2 min_theta sigma_min(sin(theta)(A - aI) + i cos(theta) I),
    # and n_a = ||(A - aI + I, A - aI - I)||, about log2(n_a/d_L - 1) +
    # log2 log2(1/eps) squarings reach relative error eps.  For a normal A,
    # d_L = 2 min_lambda |delta| / sqrt(1 + gamma^2) (delta + i gamma = lambda - a);
    # that closed form is checked against a grid over theta, then the squaring
    # counts of the rotated, scaled problem against the bound.
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = 40
        w = np.exp(2j * np.pi * rng.uniform())
        t = rng.uniform(-0.3, 0.3)
        s = 3.0
        lam = 1.5 * _crandn(rng, n)
        dist = 10.0 ** rng.uniform(-6, -1)
        lam[0] = w * (t + dist + 1j * rng.uniform(-1, 1))
        W = cqr_explicit(_crandn(rng, n, n))[0]
        A = W @ np.diag(lam) @ W.conj().T
        res = cirs(*line_map(A, w, t, s))
        assert res.converged
        zp = (np.conj(w) * lam - t) / s                  # the line becomes Re z = 0
        dL = 2.0 * np.min(np.abs(zp.real) / np.sqrt(1.0 + zp.imag ** 2))
        Ap = (np.conj(w) * A - t * np.eye(n)) / s
        if trial == 0:
            smin = lambda th: np.linalg.svd(np.sin(th) * Ap + 1j * np.cos(th) * np.eye(n),
                                            compute_uv=False)[-1]
            # the minimiser: sin(theta) gamma + cos(theta) = 0 for the nearest eigenvalue
            i = int(np.argmin(np.abs(zp.real) / np.sqrt(1.0 + zp.imag ** 2)))
            th_star = np.arctan2(1.0, -zp.imag[i])
            assert abs(2.0 * smin(th_star) - dL) <= 1e-8 * dL
            grid = min(smin(th) for th in np.linspace(0.0, np.pi, 4001))
            assert 2.0 * grid >= dL * (1.0 - 1e-9)            # nothing smaller elsewhere
        na = np.linalg.norm(np.vstack([Ap + np.eye(n), Ap - np.eye(n)]), 2)
        eps = 4.0 * np.sqrt(n) * 2.0 ** -53              # the stopping tolerance tau
        bound = np.log2(na / dL - 1.0) + np.log2(np.log2(1.0 / eps))
        assert bound - 2.0 <= res.iters <= bound + 1.0
