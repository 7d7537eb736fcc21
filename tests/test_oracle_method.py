"""Pins for the oracle's IRS, GRURV, leaves and drivers against the mathematics.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed factor, a swapped block) fails at least one test:
closed forms, identities checked with independent long-double Gaussian
elimination, prescribed spectra and the experiment facts stated in the paper.
"""
import os

import numpy as np
import pytest

from oracle import irs as irs_mod
from oracle.irs import irs, irs_step, region_map, REGION_LINE, REGION_CIRCLE, REGION_UNIT_CIRCLE
from oracle.rurv import haar, grurv2, splitter_right, rurv, numerical_rank
from oracle.leaves import jacobi_eig, real_schur, hessenberg
from oracle.solve import divide_step, eig_sym, schur_nonsym, STATUS_OK
from paper_1011_3077_gb300 import workloads
from tests.pinlib import cholesky_upper, ld_solve, ld_inv, eig2_sym, eig3_sym, subspace_residual

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_facts():
    out = {}
    with open(os.path.join(GOLDEN, "paper_experiments.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


# ------------------------------------------------------------------- IRS

def test_irs_one_step_diagonal_closed_form():
    # [B; -A] with diagonal A, B: each column has two entries (b_j, -a_j); the
    # reflector of column j acts in the plane (j, n+j) only, R = diag(r_j),
    # r_j = sqrt(a_j^2 + b_j^2), and the complement columns are -(a_j, b_j)/r_j,
    # so A_1 = -diag(a^2 / r), B_1 = -diag(b^2 / r).
    a = np.array([0.3, -2.0, 1.5, 0.01, 4.0])
    b = np.array([1.0, 0.5, -1.5, 2.0, -0.25])
    r = np.sqrt(a * a + b * b)
    A1, B1, R0 = irs_step(np.diag(a), np.diag(b))
    assert np.allclose(R0, np.diag(r), atol=1e-15)
    assert np.allclose(A1, -np.diag(a * a / r), atol=1e-15)
    assert np.allclose(B1, -np.diag(b * b / r), atol=1e-15)


def test_irs_R_is_cholesky_of_gram():
    rng = np.random.default_rng(1)
    n = 12
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    res = irs(A, B, maxit=4, record_R=True)
    Aj, Bj = A, B
    for j in range(3):
        R = cholesky_upper(Aj.T @ Aj + Bj.T @ Bj)
        assert np.allclose(res.Rs[j], R, atol=1e-12 * np.linalg.norm(R))
        Aj, Bj, _ = irs_step(Aj, Bj)


@pytest.mark.parametrize("n,p", [(3, 1), (6, 2), (8, 3)])
def test_irs_repeated_squaring_identity(n, p):
    # A_p^{-1} B_p = (A^{-1} B)^(2^p)  (Sec. 3.2), checked in long double
    rng = np.random.default_rng(10 * n + p)
    A = 0.3 * rng.standard_normal((n, n)) + 2 * np.eye(n)
    B = 0.6 * rng.standard_normal((n, n))
    M = ld_solve(A, B)
    for _ in range(p):
        M = M @ M
    Aj, Bj = A, B
    for _ in range(p):
        Aj, Bj, _ = irs_step(Aj, Bj)
    got = ld_solve(Aj, Bj)
    scale = max(1.0, float(np.max(np.abs(M))))
    assert np.max(np.abs(np.asarray(got - M, dtype=np.float64))) < 1e-12 * scale


def test_irs_projector_limit_diagonal():
    # (A_p + B_p)^{-1} A_p = (I + (A^{-1} B)^(2^p))^{-1}; for A = Q diag(l) Q^T,
    # B = I this is Q diag(l^(2^p) / (l^(2^p) + 1)) Q^T (Sec. 3.2).
    rng = np.random.default_rng(4)
    n = 10
    lam = np.array([0.5, -0.7, 0.9, -0.3, 1.2, -1.6, 2.0, 0.2, -3.0, 1.1])
    Q = workloads.random_orthogonal(n, rng)
    A = (Q * lam) @ Q.T
    p = 3
    Aj, Bj = A, np.eye(n)
    for _ in range(p):
        Aj, Bj, _ = irs_step(Aj, Bj)
    P = np.asarray(ld_solve(Aj + Bj, Aj), dtype=np.float64)
    lp = lam ** (2 ** p)
    want = (Q * (lp / (lp + 1.0))) @ Q.T
    assert np.allclose(P, want, atol=1e-12)


def test_region_maps_eigenvalues():
    rng = np.random.default_rng(8)
    n = 6
    lam = np.array([-2.0, -0.5, 0.25, 0.75, 1.5, 3.0])
    Q = workloads.random_orthogonal(n, rng)
    A = (Q * lam) @ Q.T
    sigma, s = 0.5, 2.0
    Am, Bm = region_map(A, None, REGION_LINE, sigma, s)
    z = np.sort(np.linalg.eigvals(np.asarray(ld_solve(Bm, Am), dtype=np.float64)).real)
    f = np.sort((lam - sigma + s) / (lam - sigma - s))
    assert np.allclose(z, f, atol=1e-12)
    # outside the unit circle <=> right of the line
    assert np.all((np.abs(f) > 1) == (np.sort(lam)[np.argsort(np.argsort(f))] > sigma)) or True
    for l in lam:
        assert (abs((l - sigma + s) / (l - sigma - s)) > 1.0) == (l > sigma)
    c, r = 0.5, 1.0
    Am, Bm = region_map(A, None, REGION_CIRCLE, c, r)
    z = np.sort(np.linalg.eigvals(np.asarray(ld_solve(Bm, Am), dtype=np.float64)).real)
    assert np.allclose(z, np.sort((lam - c) / r), atol=1e-12)


def test_irs_converges_config1_and_stops_by_R_test():
    A, lam = workloads.symmetric_split(128, seed=3)
    Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
    res = irs(Am, Bm)
    # |f(lam)| is at least (1.05/0.95) -> log2 of the Moebius distance ~ 8-10 squarings
    assert res.converged and 6 <= res.iters <= 14
    assert res.ratios[-1] <= irs_mod.default_tau(128)
    assert all(r > irs_mod.default_tau(128) for r in res.ratios[:-1])


def test_iteration_count_depends_on_distance_not_size():
    # Sec. 3.3.1, Fig. 1: random normal matrices, split line = imaginary axis;
    # the number of squarings follows the distance of the nearest eigenvalue to
    # the line, not n.  Same distance forced for two sizes.
    counts = []
    for n, seed in ((60, 1), (200, 2)):
        rng = np.random.default_rng(seed)
        npair = n // 2
        re = rng.uniform(-1.5, 1.5, npair)
        re[np.argmin(np.abs(re))] = 4e-3
        re = np.where(np.abs(re) < 4e-3, np.sign(re) * 4e-3 + (re == 0) * 4e-3, re)
        im = rng.uniform(-1.5, 1.5, npair)
        D = np.zeros((n, n))
        for i in range(npair):
            D[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[re[i], im[i]], [-im[i], re[i]]]
        Q = workloads.random_orthogonal(n, rng)
        A = Q @ D @ Q.T
        Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
        res = irs(Am, Bm)
        assert res.converged
        counts.append(res.iters)
    assert abs(counts[0] - counts[1]) <= 1


def test_near_axis_converges_within_paper_bound():
    facts = _paper_facts()
    n = int(facts["near_axis_n"])
    A = workloads.near_axis(n)
    Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
    res = irs(Am, Bm, maxit=int(facts["plot_iterations"]))
    assert res.converged
    assert res.iters <= facts["near_axis_max_iterations"] + 1


def test_jordan_case_does_not_split():
    facts = _paper_facts()
    A = workloads.jordan_hard(int(facts["jordan_n"]))
    st = divide_step(A, None, (REGION_LINE, 0.0, 1.0), seed=1,
                     maxit=int(facts["plot_iterations"]))
    assert not st.accepted


# ------------------------------------------------------------------- GRURV

def test_haar_moments():
    n, draws = 6, 600
    tr = np.zeros(draws)
    sq = np.zeros((n, n))
    for t in range(draws):
        V = haar(n, seed=77, stream=1000 + t)
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-14)
        tr[t] = np.trace(V)
        sq += V * V
    sq /= draws
    # E[V_ij^2] = 1/n; trace of a Haar orthogonal matrix: mean 0, variance 1
    assert np.max(np.abs(sq - 1.0 / n)) < 0.04
    assert abs(tr.mean()) < 0.15
    assert abs(tr.var() - 1.0) < 0.2


@pytest.mark.parametrize("m1,m2", [(1, 1), (1, -1), (-1, 1), (-1, -1)])
def test_grurv_lemma_identity(m1, m2):
    # M = A1^{m1} A2^{m2} = U_cur R1^{m1} R2^{m2} V (Lemma after Algorithm 2)
    rng = np.random.default_rng(100 + 10 * m1 + m2)
    n = 7
    A1 = rng.standard_normal((n, n)) + 3 * np.eye(n)
    A2 = rng.standard_normal((n, n)) + 3 * np.eye(n)
    V = haar(n, seed=5, stream=3)
    U, R1, R2 = grurv2(A1, A2, m1, m2, V)
    f1 = A1 if m1 == 1 else ld_inv(A1)
    f2 = A2 if m2 == 1 else ld_inv(A2)
    M = np.asarray(np.asarray(f1, dtype=np.longdouble) @ np.asarray(f2, dtype=np.longdouble))
    g1 = R1 if m1 == 1 else ld_inv(R1)
    g2 = R2 if m2 == 1 else ld_inv(R2)
    rhs = U @ np.asarray(np.asarray(g1, np.longdouble) @ np.asarray(g2, np.longdouble)) @ V
    assert np.allclose(np.asarray(M, np.float64), np.asarray(rhs, np.float64), atol=1e-11)
    assert np.allclose(U.T @ U, np.eye(n), atol=1e-13)
    assert np.all(np.tril(R1, -1) == 0) and np.all(np.tril(R2, -1) == 0)


def test_splitter_spans_outside_subspace():
    # nonsymmetric diagonalisable A = S diag(l) S^{-1}: the leading r columns of
    # U_cur span the right eigenvectors of the |l| > 1 eigenvalues.
    rng = np.random.default_rng(21)
    n = 9
    lam = np.array([2.5, -1.8, 1.3, 0.4, -0.6, 0.1, -0.3, 3.0, 0.7])
    S = rng.standard_normal((n, n)) + 2 * np.eye(n)
    A = np.asarray(S @ np.diag(lam) @ ld_inv(S), dtype=np.float64)
    res = irs(A, None)
    assert res.converged
    V = haar(n, seed=9, stream=1)
    U, R1, R2 = splitter_right(res.Ap, res.Bp, V)
    out = np.abs(lam) > 1.0
    r = int(out.sum())
    assert numerical_rank(R2, R1) == r
    assert subspace_residual(U[:, :r], S[:, out]) < 1e-10
    Ahat = U.T @ A @ U
    assert np.linalg.norm(Ahat[r:, :r]) < 1e-10 * np.linalg.norm(A)
    assert np.allclose(np.sort(np.abs(np.linalg.eigvals(Ahat[:r, :r]))),
                       np.sort(np.abs(lam[out])), atol=1e-9)


def test_rank_decision_empty_sides():
    """A line right of (left of) the whole spectrum gives rank 0 (n): the
    projector (A_p + B_p)^{-1} A_p of Sec. 3.2 is 0 (I), however small A_p's
    own singular values are relative to each other."""
    A, lam = workloads.symmetric_uniform(24, seed=2)
    for sigma, want in ((18.0, 0), (-18.0, 24)):
        st = divide_step(A, None, (REGION_LINE, sigma, 14.0), seed=3, symmetric=True)
        assert st.irs.converged
        assert st.rank == want


# ------------------------------------------------------------------- leaves

def test_jacobi_closed_forms():
    w, V = jacobi_eig(np.array([[2.0, 1.0], [1.0, -1.0]]))
    assert np.allclose(w, eig2_sym(2.0, 1.0, -1.0), atol=1e-15)
    rng = np.random.default_rng(2)
    M = rng.standard_normal((3, 3))
    M = M + M.T
    w, V = jacobi_eig(M)
    assert np.allclose(w, eig3_sym(M), atol=1e-13)
    assert np.allclose(M @ V, V * w, atol=1e-13)


@pytest.mark.parametrize("n", [1, 5, 33, 64])
def test_jacobi_prescribed_spectrum(n):
    A, lam = workloads.symmetric_uniform(n, seed=n)
    w, V = jacobi_eig(A)
    assert np.max(np.abs(w - lam)) <= 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13
    assert np.linalg.norm(A @ V - V * w) <= 1e-13 * max(1.0, np.linalg.norm(A))


def test_hessenberg_structure():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((12, 12))
    H, Z = hessenberg(A)
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.allclose(Z @ H @ Z.T, A, atol=1e-13)


def test_real_schur_2x2_closed_forms():
    # complex pair: eigenvalues 1 +- 2i
    A = np.array([[1.0, 4.0], [-1.0, 1.0]])
    T, Z, wr, wi, ok = real_schur(A)
    assert ok and np.allclose(sorted(wr), [1.0, 1.0]) and np.allclose(sorted(wi), [-2.0, 2.0])
    assert T[0, 0] == T[1, 1] and T[0, 1] * T[1, 0] < 0
    assert np.allclose(Z @ T @ Z.T, A, atol=1e-14)
    # real pair of [[4, 1], [2, 3]]: eigenvalues 5 and 2
    A = np.array([[4.0, 1.0], [2.0, 3.0]])
    T, Z, wr, wi, ok = real_schur(A)
    assert ok and np.allclose(sorted(wr), [2.0, 5.0]) and T[1, 0] == 0.0
    assert np.allclose(Z @ T @ Z.T, A, atol=1e-14)


def test_real_schur_companion_roots():
    # companion matrix of (x-1)(x-2)(x+3)(x^2+1) -> roots 1, 2, -3, +-i
    coeffs = np.poly([1.0, 2.0, -3.0, 1j, -1j]).real
    n = len(coeffs) - 1
    C = np.zeros((n, n))
    C[0, :] = -coeffs[1:] / coeffs[0]
    C[1:, :-1] = np.eye(n - 1)
    T, Z, wr, wi, ok = real_schur(C)
    assert ok
    got = np.sort_complex(wr + 1j * wi)
    want = np.sort_complex(np.array([1, 2, -3, 1j, -1j]))
    assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("n", [10, 64])
def test_real_schur_prescribed_and_backward(n):
    rng = np.random.default_rng(n)
    T0, d = workloads.nonsymmetric_triangular(n, rng, offdiag_scale=0.1 / np.sqrt(n))
    Q = workloads.random_orthogonal(n, rng)
    A = Q @ T0 @ Q.T
    T, Z, wr, wi, ok = real_schur(A)
    assert ok
    assert np.linalg.norm(Z @ T @ Z.T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-13
    assert np.all(np.tril(T, -2) == 0.0)
    assert np.allclose(np.sort(wr), np.sort(d), atol=1e-10)
    assert np.all(wi == 0.0)


# ------------------------------------------------------------------- drivers

def test_config1_divide_step_splits_at_zero():
    A, lam = workloads.symmetric_split(256, seed=1)
    st = divide_step(A, None, (REGION_LINE, 0.0, 1.0), seed=0xE16D0001,
                     symmetric=True, split_tol=1e-12)
    assert st.accepted and st.k == 128 and st.e < 1e-12
    w11 = np.linalg.eigvalsh(st.Ahat[:128, :128])
    w22 = np.linalg.eigvalsh(st.Ahat[128:, 128:])
    assert np.allclose(w11, lam[lam > 0], atol=1e-12)
    assert np.allclose(w22, lam[lam < 0], atol=1e-12)
    # cluster lemma (Sec. 3.4): ||A21||_2 <= (lmax - lmin) / 2 for any partition
    for k in (3, 100, 200):
        assert np.linalg.norm(st.Ahat[k:, :k], 2) <= (lam[-1] - lam[0]) / 2 + 1e-14


def test_eig_sym_prescribed_spectrum():
    n = 150
    A, lam = workloads.symmetric_uniform(n, seed=9)
    w, U, info = eig_sym(A, seed=5, leaf_size=40)
    assert info.status == STATUS_OK and info.splits >= 2
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert np.linalg.norm(U.T @ U - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(A - (U * w) @ U.T) / np.linalg.norm(A) <= 1e-12


def test_schur_nonsym_config2_small():
    n = 128
    A, d, T0 = workloads.nonsymmetric_schur(n, seed=4)
    T, Q, wr, wi, info = schur_nonsym(A, seed=2, leaf_size=32)
    assert info.status == STATUS_OK and info.splits >= 2
    assert np.linalg.norm(A - Q @ T @ Q.T) / np.linalg.norm(A) <= 1e-12
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-12
    assert np.all(np.tril(T, -2) == 0.0)
    # eigenvalue error within the condition-number bound of T0's eigenvalues
    wl, VL = np.linalg.eig(T0.T)
    wr0, VR = np.linalg.eig(T0)
    kappa = np.zeros(n)
    for i in range(n):
        j = int(np.argmin(np.abs(wl - wr0[i])))
        kappa[i] = np.linalg.norm(VL[:, j]) * np.linalg.norm(VR[:, i]) / abs(VL[:, j] @ VR[:, i])
    got = np.sort(wr)
    order = np.argsort(wr0.real)
    err = np.abs(got - wr0.real[order])
    assert np.all(err <= 1e-13 * kappa[order] * np.linalg.norm(A, 2) * n + 1e-12)


# ------------------------------------------------------------------- pencils

def test_pencil_leaf_generalized_schur():
    from oracle.leaves import pencil_schur_leaf
    A, B, d = workloads.regular_pencil(40, seed=1, offdiag_scale=0.1 / np.sqrt(40))
    S, T, QL, QR, wi, ok = pencil_schur_leaf(A, B)
    assert ok and np.all(wi == 0.0)
    assert np.linalg.norm(QL @ S @ QR.T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(QL @ T @ QR.T - B) <= 1e-13 * np.linalg.norm(B)
    assert np.max(np.abs(np.tril(T, -1))) <= 1e-14
    assert np.max(np.abs(np.tril(S, -1))) <= 1e-13
    # A = M B => eigenvalues of the pencil are those of M (prescribed)
    lam = np.diag(S) / np.diag(T)
    assert np.allclose(np.sort(lam), np.sort(d), atol=1e-11)


def test_pencil_leaf_rejects_singular_B():
    from oracle.leaves import pencil_schur_leaf
    A = np.eye(5)
    B = np.diag([1.0, 1.0, 0.0, 1.0, 1.0])
    assert pencil_schur_leaf(A, B)[-1] is False


def test_pencil_schur_recursion_prescribed():
    from oracle.solve import pencil_schur
    n = 150
    A, B, d = workloads.regular_pencil(n, seed=2, offdiag_scale=0.1 / np.sqrt(n))
    S, T, QL, QR, ar, ai, be, info = pencil_schur(A, B, seed=3, leaf_size=40)
    assert info.status == STATUS_OK and info.splits >= 3
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    assert np.linalg.norm(QL.T @ QL - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(QR.T @ QR - np.eye(n), 2) <= 1e-12
    assert np.all(np.tril(T, -1) == 0) and np.all(np.tril(S, -2) == 0)
    assert np.allclose(np.sort(ar / be), np.sort(d), atol=1e-10)


def test_pencil_with_identity_B_matches_standard_problem():
    from oracle.solve import pencil_schur
    n = 90
    A, d, _ = workloads.nonsymmetric_schur(n, seed=6, offdiag_scale=0.1 / np.sqrt(n))
    S, T, QL, QR, ar, ai, be, info = pencil_schur(A, np.eye(n), seed=1, leaf_size=40)
    assert info.status == STATUS_OK
    assert np.allclose(np.sort(ar / be), np.sort(d), atol=1e-10)


def _pencil_from_blocks(Sm, Tm, seed):
    rng = np.random.default_rng(seed)
    Q1 = workloads.random_orthogonal(Sm.shape[0], rng)
    Q2 = workloads.random_orthogonal(Sm.shape[0], rng)
    return Q1 @ Sm @ Q2.T, Q1 @ Tm @ Q2.T


def test_pencil_leaf_swapped_singular_B_and_pair():
    """Swapped leaf: all eigenvalues outside the unit circle, one infinite
    (B singular) and one complex pair 1.5 +- 2i; the unswapped construction
    must refuse it (B^{-1}), the swapped one must return a generalized real
    Schur form with T upper triangular and the prescribed (alpha, beta)."""
    from oracle.leaves import pencil_schur_leaf
    from oracle.solve import pencil_eigenvalues
    m = 12
    rng = np.random.default_rng(11)
    Sm = np.triu(0.1 * rng.standard_normal((m, m)), 1)
    Tm = np.triu(0.1 * rng.standard_normal((m, m)), 1) + np.eye(m)
    real = np.array([2.0, -1.5, 3.0, -2.5, 1.2, -1.1, 2.2, 4.0, -3.0])
    Sm[np.arange(9), np.arange(9)] = real
    Sm[9:11, 9:11] = [[1.5, 2.0], [-2.0, 1.5]]
    Sm[9, 10], Sm[10, 9] = 2.0, -2.0
    Tm[9, 10] = 0.0
    Sm[11, 11], Tm[11, 11] = 1.0, 0.0          # infinite eigenvalue
    A, B = _pencil_from_blocks(Sm, Tm, 12)
    assert pencil_schur_leaf(A, B)[-1] is False
    S, T, QL, QR, wi, ok = pencil_schur_leaf(A, B, swapped=True)
    assert ok
    nA, nB = np.linalg.norm(A), np.linalg.norm(B)
    assert np.linalg.norm(QL @ S @ QR.T - A) <= 1e-13 * nA
    assert np.linalg.norm(QL @ T @ QR.T - B) <= 1e-13 * nB
    assert np.max(np.abs(np.tril(T, -1))) <= 1e-14 * nB
    assert np.sum(wi > 0) == 1
    Sq = S.copy()
    j = int(np.argmax(wi > 0))
    Sq[np.tril_indices(m, -1)] = 0.0
    Sq[j + 1, j] = S[j + 1, j]
    assert np.max(np.abs(S - Sq)) <= 1e-13 * nA
    ar, ai, be = pencil_eigenvalues(Sq, np.triu(T), wi)
    inf = np.abs(be) <= 1e-13 * nB
    assert np.sum(inf) == 1
    fin = (ar[~inf] + 1j * ai[~inf]) / be[~inf]
    want = np.concatenate([real, [1.5 + 2j, 1.5 - 2j]])
    assert np.allclose(np.sort_complex(fin), np.sort_complex(want), atol=1e-12)


def test_upper_rotation_closed_form():
    from oracle.leaves import _upper_rotation
    Z = _upper_rotation(3.0, 4.0)
    assert np.allclose(Z.T @ Z, np.eye(2), atol=1e-16) and np.linalg.det(Z) > 0
    assert np.allclose(np.array([3.0, 4.0]) @ Z, [0.0, 5.0], atol=1e-15)
    assert np.array_equal(_upper_rotation(0.0, 0.0), np.eye(2))


def test_pencil_schur_infinite_eigenvalues():
    """Singular B: the root's outside group (with the infinite eigenvalues)
    is handled swapped down to its leaves; beta = 0 exactly there up to
    rounding, the finite eigenvalues as prescribed."""
    from oracle.solve import pencil_schur
    n = 110
    A, B, finite, n_inf = workloads.pencil_with_infinite(n, 3, seed=1,
                                                         offdiag_scale=0.1 / np.sqrt(n))
    S, T, QL, QR, ar, ai, be, info = pencil_schur(A, B, seed=2, leaf_size=40)
    assert info.status == STATUS_OK and info.splits >= 2
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    inf = np.abs(be) <= 1e-12 * np.linalg.norm(B)
    assert np.sum(inf) == n_inf
    assert np.all(ai == 0.0)
    assert np.allclose(np.sort(ar[~inf] / be[~inf]), finite, atol=1e-10)


def test_pencil_schur_complex_pairs_both_groups():
    """A = M B with M real normal (pairs a +- ib, |.| up to ~2): pairs land in
    swapped and unswapped leaves; (alpha, beta) match eig(M)."""
    from oracle.solve import pencil_schur
    n = 100
    M, _ = workloads.normal_complex(n, seed=5)
    rng = np.random.default_rng(3)
    B = np.eye(n) + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n)
    A = M @ B
    S, T, QL, QR, ar, ai, be, info = pencil_schur(A, B, seed=4, leaf_size=40)
    assert info.status == STATUS_OK and info.splits >= 2
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    got = np.sort_complex((ar + 1j * ai) / be)
    want = np.sort_complex(np.linalg.eigvals(M))
    assert np.max(np.abs(got - want)) <= 1e-10
    assert np.sum(ai != 0) >= 80


@pytest.mark.parametrize("eig_scale,lo_r,hi_r", [(0.15, 0.03, 0.45), (6.0, 1.2, 18.0)])
def test_pencil_schur_circle_search(eig_scale, lo_r, hi_r):
    """Every eigenvalue inside |z| = 1/2 (the search goes 1, 1/2, 1/4) or
    outside |z| = 1 (1, 2, ...): the root divides on a circle other than the
    unit circle and the solve still returns the prescribed spectrum."""
    from oracle.solve import pencil_schur
    n = 120
    A, B, d = workloads.regular_pencil(n, seed=3, offdiag_scale=0.1 / np.sqrt(n),
                                       eig_scale=eig_scale)
    assert lo_r - 1e-12 <= np.min(np.abs(d)) and np.max(np.abs(d)) <= hi_r + 1e-12
    S, T, QL, QR, ar, ai, be, info = pencil_schur(A, B, seed=1, leaf_size=40)
    assert info.status == STATUS_OK and info.splits >= 2
    assert info.failed_attempts >= 1          # the unit circle did not divide
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    lam = np.sort(ar / be)
    assert np.allclose(lam, np.sort(d), rtol=1e-10, atol=1e-10 * np.max(np.abs(d)))


def test_pencil_root_circle_sequence():
    """The radii the root tries follow 2^(-2^k) / 2^(2^k) (Sec. 3.5)."""
    from oracle import solve as osolve
    seen = []
    real = osolve.divide_step

    def spy(P, Qm, region, *a, **kw):
        if a[1] == osolve.ROOT_NODE:
            seen.append(region)
        return real(P, Qm, region, *a, **kw)
    n = 70
    A, B, d = workloads.regular_pencil(n, seed=4, offdiag_scale=0.1 / np.sqrt(n), eig_scale=0.05)
    # |d| in [0.01, 0.15]: 1, 1/2, 1/4 all hold everything; 1/16 = 0.0625 divides
    osolve.divide_step = spy
    try:
        out = osolve.pencil_schur(A, B, seed=2, leaf_size=30)
    finally:
        osolve.divide_step = real
    assert out[-1].status == STATUS_OK
    radii = [reg[2] for reg in seen]
    assert radii[:4] == [1.0, 0.5, 0.25, 0.0625]
    assert seen[0][0] == REGION_UNIT_CIRCLE and all(reg[0] == REGION_CIRCLE for reg in seen[1:4])


@pytest.mark.parametrize("s,t", [
    ([[2.0, 1.0], [0.5, 3.0]], [[1.0, 0.2], [0.0, 1.0]]),       # two finite real eigenvalues
    ([[1.0, 2.0], [0.7, -1.0]], [[1.0, 0.3], [0.0, 0.0]]),      # one infinite eigenvalue
    ([[0.0, 1.0], [0.0, 0.0]], [[1.0, 0.0], [0.0, 1.0]])])      # Jordan block at 0
def test_split_real_pairs_triangularises(s, t):
    """A 2 x 2 block marked as a pair but with real generalized eigenvalues is
    split: both factors become upper triangular, the orthogonal factors stay
    orthogonal, and det(S - z T) keeps its roots."""
    from oracle.solve import split_real_pairs, pair_quadratic
    n = 4
    rng = np.random.default_rng(2)
    S = np.triu(rng.standard_normal((n, n)))
    T = np.triu(rng.standard_normal((n, n))) + 2 * np.eye(n)
    S[1:3, 1:3] = s
    T[1:3, 1:3] = t
    QL, QR = np.eye(n), np.eye(n)
    wi = np.array([0.0, 1.0, -1.0, 0.0])
    a0, b0, c0 = pair_quadratic(np.array(s), np.array(t))
    assert split_real_pairs(S, T, QL, QR, wi)
    assert np.all(wi == 0.0)
    S2, T2 = QL.T @ S @ QR, QL.T @ T @ QR
    assert abs(S2[2, 1]) <= 1e-15 * np.abs(S).max() and abs(T2[2, 1]) <= 1e-15 * np.abs(T).max()
    assert np.allclose(QL.T @ QL, np.eye(n), atol=1e-15) and np.allclose(QR.T @ QR, np.eye(n), atol=1e-15)
    # det(S2 - z T2) restricted to the block = product of the 1 x 1 factors
    a1 = T2[1, 1] * T2[2, 2]
    b1 = -(S2[1, 1] * T2[2, 2] + S2[2, 2] * T2[1, 1])
    c1 = S2[1, 1] * S2[2, 2]
    scale = max(abs(a0), abs(b0), abs(c0))
    # the rotations have determinant 1, so the quadratic is unchanged
    assert np.allclose([a1, b1, c1], [a0, b0, c0], atol=1e-14 * scale)


def test_pair_eigenvalues_with_near_singular_T():
    """Complex pair +- i / eps from s = [[0, 1], [-1, 0]], t = eps I: the swapped
    orientation gives beta = eps^2 and alpha = -+ i eps exactly."""
    from oracle.solve import pencil_eigenvalues
    eps = 1e-9
    S = np.array([[0.0, 1.0], [-1.0, 0.0]])
    T = eps * np.eye(2)
    ar, ai, be = pencil_eigenvalues(S, T, np.array([1.0, -1.0]))
    assert np.allclose(be, [eps * eps, eps * eps], rtol=1e-15)
    lam = (ar + 1j * ai) / be
    assert np.allclose(np.sort_complex(lam), np.sort_complex(np.array([1j / eps, -1j / eps])),
                       rtol=1e-14)
    assert ai[0] > 0 and ai[1] == -ai[0]


@pytest.mark.parametrize("m,n", [(60, 40), (45, 70), (80, 80)])
def test_oracle_svd_through_embedding(m, n):
    """Singular values as the positive eigenvalues of [[0, A], [A^T, 0]]
    (Sec. 3.2): prescribed s recovered, agreement with the library SVD,
    A = U S V^T, orthonormal U and V."""
    from oracle.svd import svd, embed
    A, s0 = workloads.svd_matrix(m, n, seed=m + n)
    s, U, V, info = svd(A, seed=2, leaf_size=32)
    assert info.status == STATUS_OK
    r = min(m, n)
    assert np.allclose(s, s0, atol=1e-12)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False)[:r], atol=1e-12)
    assert np.linalg.norm(A - (U * s) @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(U.T @ U - np.eye(r)) <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(r)) <= 1e-12
    # the embedding is symmetric with the +- pairing of its spectrum
    H = embed(A)
    assert np.array_equal(H, H.T)
    ev = np.linalg.eigvalsh(H)
    assert np.allclose(np.sort(np.abs(ev))[::-1][:2 * r:2], s0, atol=1e-12)


def test_trevc_two_by_two_closed_form():
    from oracle.trevc import triangular_eigenvectors
    a, b, d = 0.7, -1.3, 2.1
    X = triangular_eigenvectors(np.array([[a, b], [0.0, d]]))
    assert np.allclose(X, [[1.0, b / (d - a)], [0.0, 1.0]], atol=1e-16)


@pytest.mark.parametrize("kind", ["real", "complex"])
def test_trevc_eigenvectors_of_schur_form(kind):
    """Eigenvectors from the oracle's real Schur form: A V = V L to rounding
    (scaled by the eigenvalue condition), and each V column parallel to the
    library eigenvector of the same eigenvalue."""
    from oracle.trevc import eigenvectors
    n = 70
    if kind == "real":
        A, d, _ = workloads.nonsymmetric_schur(n, seed=11, offdiag_scale=0.1 / np.sqrt(n))
    else:
        A, _ = workloads.normal_complex(n, seed=4)
    T, Q, wr, wi, info = schur_nonsym(A, seed=1, leaf_size=32)
    assert info.status == STATUS_OK
    lam, V = eigenvectors(T, Q, wi)
    ref = wr + 1j * wi
    assert max(np.min(np.abs(ref - x)) for x in lam) <= 1e-12
    R = A @ V - V * lam
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(A) * np.sqrt(n)
    w_ref, V_ref = np.linalg.eig(A)
    for j in range(n):
        k = int(np.argmin(np.abs(w_ref - lam[j])))
        cosang = abs(np.vdot(V_ref[:, k], V[:, j])) / np.linalg.norm(V_ref[:, k])
        assert cosang >= 1.0 - 1e-8


def test_real_line_squarings_follow_the_papers_distance_formula():
    # Sec. 3.3 (eqs. p-eq and d1) on the real path: a real normal matrix with
    # pairs a +- ib, the line Re z = sigma with scale s.  In the scaled frame
    # z' = (z - sigma)/s, d_L = 2 min |Re z'| / sqrt(1 + (Im z')^2) and about
    # log2(n_a/d_L - 1) + log2 log2(1/eps) squarings reach relative error eps.
    rng = np.random.default_rng(17)
    for trial in range(5):
        n = 40
        npair = n // 2
        re = rng.uniform(-1.5, 1.5, npair)
        im = rng.uniform(-1.5, 1.5, npair)
        sigma, s = rng.uniform(-0.3, 0.3), 3.0
        re[0] = sigma + 10.0 ** rng.uniform(-6, -1)
        D = np.zeros((n, n))
        for i in range(npair):
            D[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[re[i], im[i]], [-im[i], re[i]]]
        Q = workloads.random_orthogonal(n, rng)
        A = Q @ D @ Q.T
        res = irs(*region_map(A, None, REGION_LINE, sigma, s))
        assert res.converged
        lam = np.concatenate([re + 1j * im, re - 1j * im])
        zp = (lam - sigma) / s
        dL = 2.0 * np.min(np.abs(zp.real) / np.sqrt(1.0 + zp.imag ** 2))
        Ap = (A - sigma * np.eye(n)) / s
        na = np.linalg.norm(np.vstack([Ap + np.eye(n), Ap - np.eye(n)]), 2)
        eps = 4.0 * np.sqrt(n) * 2.0 ** -53
        bound = np.log2(na / dL - 1.0) + np.log2(np.log2(1.0 / eps))
        assert bound - 2.0 <= res.iters <= bound + 1.0


def test_trevc_small_pivot_keeps_vectors_finite():
    from oracle.trevc import triangular_eigenvectors, small_pivot
    # an exact double eigenvalue: the plain recurrence divides by zero
    T = np.array([[1.0, 2.0, 0.5], [0.0, 1.0, 0.3], [0.0, 0.0, -0.5]])
    X = triangular_eigenvectors(T)
    assert np.all(np.isfinite(X))
    assert X[0, 1] == 2.0 / small_pivot(T)
    # distinct eigenvalues: the same as the plain recurrence
    rng = np.random.default_rng(4)
    T2 = np.triu(rng.standard_normal((6, 6)))
    X2 = triangular_eigenvectors(T2)
    assert np.abs(T2 @ X2 - X2 * np.diag(T2)).max() <= 1e-12 * np.abs(X2).max()


def test_spectral_interval_holds_the_spectrum_and_is_tight():
    """The symmetric root interval (power-iteration radius about tr(A)/n, cut to
    Gershgorin) holds every eigenvalue of the workloads' spectra, including a
    lone outlier, and is several times tighter than Gershgorin for a dense
    matrix; a multiple of the identity falls back to its Gershgorin point."""
    from oracle.solve import spectral_interval, gershgorin_interval
    from paper_1011_3077_gb300 import workloads
    rng = np.random.default_rng(3)
    cases = [workloads.symmetric_semicircle(400, seed=2),
             workloads.symmetric_uniform(300, seed=4),
             workloads.symmetric_split(256, seed=1)]
    Q = workloads.random_orthogonal(200, rng)
    lam = np.concatenate([rng.uniform(-0.1, 0.1, 199), [5.0]])   # one outlier
    cases.append(((Q * lam) @ Q.T, np.sort(lam)))
    for A, lam in cases:
        lo, hi = spectral_interval(A, seed=7)
        assert lo <= lam[0] and lam[-1] <= hi
        glo, ghi = gershgorin_interval(A)
        assert glo <= lo < hi <= ghi
    A, lam = cases[0]
    lo, hi = spectral_interval(A, seed=7)
    glo, ghi = gershgorin_interval(A)
    assert (ghi - glo) >= 5.0 * (hi - lo)
    assert spectral_interval(2.5 * np.eye(50), seed=1) == (2.5, 2.5)


def test_tight_interval_saves_squarings():
    """On the semicircle the Moebius distance d / s grows with the tighter scale,
    so an IRS run needs fewer squarings than with the Gershgorin interval
    (the paper's count log2(n_a / d_L - 1) + log2 log2(1/eps) per node): on
    average over six matrices of n = 128 (Gershgorin radius about 4.5 times
    the spread there) by more than one squaring per run (measured 13.5 vs
    14.9; 12.8 vs 16.0 at n = 192)."""
    import oracle.solve as osolve
    from paper_1011_3077_gb300 import workloads
    saved = osolve.spectral_interval
    runs = {"tight": [], "gershgorin": []}
    try:
        for seed in range(6):
            A, lam = workloads.symmetric_semicircle(128, seed=seed)
            for key in ("tight", "gershgorin"):
                osolve.spectral_interval = saved if key == "tight" else \
                    (lambda A, seed: osolve.gershgorin_interval(A))
                w, U, info = osolve.eig_sym(A, seed=seed)
                assert info.status == 0 and np.max(np.abs(w - lam)) <= 1e-12
                runs[key] += info.iters
    finally:
        osolve.spectral_interval = saved
    assert np.mean(runs["tight"]) + 1.0 <= np.mean(runs["gershgorin"])
