"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Tolerances (derived from FP64 rounding, u = 2^-53 ~ 1.1e-16):
  * GEMM: |C - C_ref| <= 8 k u max|A| max|B| elementwise (k-term dot products);
  * QR factors, Haar V, iterates: 1e-11 relative to the norm of the matrix
    (a few hundred u times n for n <= 520, with margin for the different
    blocking / summation order of the GPU reductions);
  * Gaussian draws: 1e-13 absolute (log / sincospi vs libm, same 52-bit
    uniforms bit for bit);
  * split residuals and integers (k, rank, iteration count) must agree exactly
    where the value is well separated from its decision threshold;
  * whole solves: the stated targets -- eigenvalue error <= 1e-10 ||A||,
    ||U^T U - I||_2 <= 1e-12, ||A - U L U^T||_F / ||A||_F <= 1e-12.
"""
import numpy as np
import pytest

from oracle import philox as ophilox
from oracle.householder import qr_explicit as oqr
from oracle.irs import irs as oirs, region_map, REGION_LINE, REGION_UNIT_CIRCLE, norm1
from oracle.rurv import haar as ohaar
from oracle.split import split_scores as osplit_scores, choose_k as ochoose_k
from oracle.solve import divide_step as odivide_step, eig_sym as oeig_sym, schur_nonsym as oschur
from paper_1011_3077_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def E():
    import torch
    from paper_1011_3077_gb300 import build, eigdc
    build.build()
    h = eigdc.Handle(0)
    yield eigdc, h, torch
    torch.cuda.synchronize()
    h.close()


# ------------------------------------------------------------------ GEMM
@pytest.mark.parametrize("m,n,k,ta,tb", [
    (1, 1, 1, 0, 0), (63, 65, 17, 0, 0), (130, 70, 300, 1, 0), (64, 130, 33, 0, 1),
    (100, 100, 100, 1, 1), (32, 1000, 4000, 1, 0), (300, 257, 5, 0, 0)])
def test_gemm_matches_reference(E, m, n, k, ta, tb):
    eigdc, h, torch = E
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    alpha, beta = 0.7, -1.3
    ref = alpha * ((A.T if ta else A) @ (B.T if tb else B)) + beta * C
    dA, dB, dC = eigdc.to_device(A), eigdc.to_device(B), eigdc.to_device(C)
    eigdc.eig_gemm(h, ta, tb, m, n, k, alpha, dA, eigdc.ld(dA), dB, eigdc.ld(dB), beta, dC, eigdc.ld(dC))
    got = eigdc.to_host(dC)
    tol = 8 * k * U * np.abs(A).max() * np.abs(B).max() + 4 * U * np.abs(C).max()
    assert np.max(np.abs(got - ref)) <= tol


# ------------------------------------------------------------------ Philox / Haar
@pytest.mark.parametrize("rows,cols,stream,attempt", [(1, 1, 1, 0), (37, 29, 99, 3), (256, 256, 12345678901, 200)])
def test_gaussian_matches_oracle(E, rows, cols, stream, attempt):
    eigdc, h, torch = E
    seed = 0xE16D0001
    dG = torch.zeros((cols, rows), dtype=torch.float64, device="cuda")
    eigdc.eig_gaussian(h, rows, cols, seed, 4, stream, attempt, dG, rows)
    got = eigdc.to_host(dG)
    want = ophilox.gaussian_matrix(rows, cols, seed, 4, stream, attempt)
    assert np.max(np.abs(got - want)) <= 1e-13


@pytest.mark.parametrize("n", [1, 7, 64, 130])
def test_haar_matches_oracle(E, n):
    eigdc, h, torch = E
    dV = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eigdc.eig_haar(h, n, 77, 4, 5, 2, dV, n)
    got = eigdc.to_host(dV)
    want = ohaar(n, 77, 5, 2)
    assert np.max(np.abs(got - want)) <= 1e-11
    assert np.max(np.abs(got.T @ got - np.eye(n))) <= 1e-13 * max(n, 8)


# ------------------------------------------------------------------ QR
@pytest.mark.parametrize("m,n", [(1, 1), (8, 3), (64, 32), (130, 97), (520, 260), (1000, 500), (2050, 1025)])
def test_qr_matches_oracle(E, m, n):
    eigdc, h, torch = E
    rng = np.random.default_rng(m * 7 + n)
    X = rng.standard_normal((m, n))
    dX = eigdc.to_device(X)
    dQ = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    dR = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eigdc.eig_qr(h, m, n, dX, m, dQ, m, dR, n)
    Q, R = eigdc.to_host(dQ), eigdc.to_host(dR)
    nx = np.linalg.norm(X, 2)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)
    assert np.linalg.norm(Q @ R - X) <= 1e-13 * np.sqrt(m) * nx * max(1, np.sqrt(n))
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 1e-14 * m
    if m <= 1000:
        Qo, Ro = oqr(X)
        assert np.max(np.abs(R - Ro)) <= 1e-11 * nx
        assert np.max(np.abs(Q - Qo)) <= 1e-10


def test_qr_special_columns(E):
    """Zero columns, a negative pivot with nothing below it, rank deficiency."""
    eigdc, h, torch = E
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 12))
    X[:, 2] = 0.0
    X[:, 5] = X[:, 1] * 3.0
    X[5:, 7] = 0.0
    Y = np.zeros((6, 3))
    Y[0, 0] = -2.0
    Y[:, 1] = rng.standard_normal(6)
    Y[1, 2] = 1.0
    # X: column 5 depends on column 1, so the reflectors from column 5 on act
    # on rounding noise and are not unique; rows 0..4 of R are.
    for M, rows in ((X, 5), (Y, 3)):
        m, n = M.shape
        dX = eigdc.to_device(M)
        dQ = torch.zeros((n, m), dtype=torch.float64, device="cuda")
        dR = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        eigdc.eig_qr(h, m, n, dX, m, dQ, m, dR, n)
        Q, R = eigdc.to_host(dQ), eigdc.to_host(dR)
        Qo, Ro = oqr(M)
        assert np.max(np.abs(R[:rows] - Ro[:rows])) <= 1e-12 * max(1, np.abs(M).max())
        assert R[2, 2] == 0.0 or M is Y
        assert np.allclose(Q @ R, M, atol=1e-13)
        assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-14)
        assert np.all(np.diag(R) >= 0)


# ------------------------------------------------------------------ split test
@pytest.mark.parametrize("n", [2, 3, 33, 100, 257])
def test_split_test_matches_oracle(E, n):
    eigdc, h, torch = E
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A[n // 3:, : n // 3] *= 1e-9
    dA = eigdc.to_device(A)
    nA = norm1(A)
    k, e, scores = eigdc.eig_split_test(h, n, dA, n, nA, want_scores=True)
    want = osplit_scores(A) / nA
    assert np.allclose(scores, want, rtol=1e-13, atol=0)
    assert k == ochoose_k(want, n)


def test_split_test_pencil_and_ties(E):
    eigdc, h, torch = E
    n = 10
    D = np.diag(np.arange(1.0, n + 1))
    dD = eigdc.to_device(D)
    k, e, _ = eigdc.eig_split_test(h, n, dD, n, norm1(D))
    assert k == n // 2 and e == 0.0
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    k, e, sc = eigdc.eig_split_test(h, n, eigdc.to_device(A), n, norm1(A), eigdc.to_device(B), n,
                                    norm1(B), want_scores=True)
    want = osplit_scores(A) / norm1(A) + osplit_scores(B) / norm1(B)
    assert np.allclose(sc, want, rtol=1e-13) and k == ochoose_k(want, n)


# ------------------------------------------------------------------ IRS
def _dev_pair(eigdc, torch, A, B):
    dA = eigdc.to_device(A)
    dB = eigdc.to_device(B) if B is not None else None
    return dA, dB


@pytest.mark.parametrize("n,sq", [(1, 2), (5, 1), (33, 3), (100, 4), (161, 2)])
def test_irs_iterates_match_oracle(E, n, sq):
    """Exactly `sq` squarings (R-test disabled): A_p, B_p, R_{p-1} elementwise."""
    eigdc, h, torch = E
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n)) + 2 * np.eye(n)
    dA, dB = _dev_pair(eigdc, torch, A, B)
    reg = eigdc.Region(REGION_UNIT_CIRCLE, 0.0, 1.0)
    p = eigdc.default_params(tau=-1.0, maxit=sq - 1)
    rc, info = eigdc.eig_divide_step(h, n, dA, n, dB, n, reg, p)
    assert rc == eigdc.EIG_NO_CONVERGENCE and info.iters == sq
    res = oirs(A, B, tau=-1.0, maxit=sq - 1, record_R=True)
    Ap, Bp = eigdc.to_host(dA), eigdc.to_host(dB)
    scale = np.linalg.norm(np.vstack([A, B]), 2)
    assert np.max(np.abs(Ap - res.Ap)) <= 1e-11 * scale
    assert np.max(np.abs(Bp - res.Bp)) <= 1e-11 * scale
    dR = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eigdc.eig_last_R(h, n, dR, n)
    assert np.max(np.abs(eigdc.to_host(dR) - res.Rs[-1])) <= 1e-11 * scale


def test_config1_divide_step_matches_oracle(E):
    """Symmetric n = 256, line Re z = 0: iteration count, R_{p-1}, A_p, B_p."""
    eigdc, h, torch = E
    A, lam = workloads.symmetric_split(256, seed=1)
    n = 256
    dA = eigdc.to_device(A)
    dB = None
    reg = eigdc.Region(eigdc.EIG_REGION_LINE, 0.0, 1.0)
    p = eigdc.default_params()
    rc, info = eigdc.eig_divide_step(h, n, dA, n, dB, 0, reg, p)
    assert rc == eigdc.EIG_OK and info.converged == 1
    Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
    res = oirs(Am, Bm, record_R=True)
    assert info.iters == res.iters
    dR = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eigdc.eig_last_R(h, n, dR, n)
    assert np.max(np.abs(eigdc.to_host(dR) - res.Rs[-1])) <= 1e-11 * norm1(res.Rs[-1])
    assert np.max(np.abs(eigdc.to_host(dA) - res.Ap)) <= 1e-10


def test_config1_split_matches_oracle(E):
    """GRURV + similarity + split test on config 1: k, A11 elementwise (Sec. 3.1)."""
    eigdc, h, torch = E
    A, lam = workloads.symmetric_split(256, seed=1)
    n = 256
    seed = 0xE16D0001
    st = odivide_step(A, None, (REGION_LINE, 0.0, 1.0), seed=seed, stream=1, attempt=0,
                      symmetric=True)
    Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
    dAp, dBp = eigdc.to_device(Am), eigdc.to_device(Bm)
    rc, info = eigdc.eig_divide_step(h, n, dAp, n, dBp, n, eigdc.Region(0, 0.0, 1.0),
                                     eigdc.default_params())
    assert rc == 0
    dA = eigdc.to_device(A)
    dQ = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    p = eigdc.default_params(seed=seed)
    rc, sinfo = eigdc.eig_split(h, n, dAp, dBp, n, dA, n, dQ, n, 1, 1, 0, p)
    assert rc == eigdc.EIG_OK and st.accepted
    assert sinfo.k == st.k == 128
    assert sinfo.rank == st.rank == 128
    assert sinfo.draw == st.draw
    assert sinfo.split_residual <= 1e-12
    Ahat = eigdc.to_host(dA)
    k = sinfo.k
    assert np.max(np.abs(Ahat[:k, :k] - st.Ahat[:k, :k])) <= 1e-10
    assert np.allclose(np.linalg.eigvalsh(Ahat[:k, :k]), lam[lam > 0], atol=1e-11)
    assert np.allclose(np.linalg.eigvalsh(Ahat[k:, k:]), lam[lam < 0], atol=1e-11)
    Q = eigdc.to_host(dQ)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 1e-13


def test_rank_decision_empty_sides_gpu(E):
    """A line beyond the spectrum: rank 0 (right of everything) or n (left),
    measured against |A_p + B_p|, as in the oracle."""
    eigdc, h, torch = E
    from oracle.solve import divide_step as ods
    A, lam = workloads.symmetric_uniform(40, seed=2)
    n = 40
    for sigma, want in ((18.0, 0), (-18.0, n)):
        Am, Bm = region_map(A, None, REGION_LINE, sigma, 14.0)
        dAp, dBp = eigdc.to_device(Am), eigdc.to_device(Bm)
        rc, info = eigdc.eig_divide_step(h, n, dAp, n, dBp, n, eigdc.Region(0, 0.0, 1.0),
                                         eigdc.default_params())
        assert rc == eigdc.EIG_OK
        dQ = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        rc, si = eigdc.eig_split(h, n, dAp, dBp, n, eigdc.to_device(A), n, dQ, n, 1, 1, 0,
                                 eigdc.default_params(seed=3))
        st = ods(A, None, (REGION_LINE, sigma, 14.0), seed=3, stream=1, symmetric=True)
        assert si.rank == want == st.rank


# ------------------------------------------------------------------ whole solves
@pytest.mark.parametrize("n,leaf", [(1, 64), (2, 64), (64, 64), (150, 40), (300, 64)])
def test_eig_solve_symmetric(E, n, leaf):
    eigdc, h, torch = E
    A, lam = workloads.symmetric_uniform(n, seed=n)
    p = eigdc.default_params(seed=5, leaf_size=leaf)
    rc, w, Uv, info = eigdc.solve_symmetric(h, A, p)
    assert rc == eigdc.EIG_OK
    nA = max(np.linalg.norm(A, 2), 1e-300)
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert np.linalg.norm(Uv.T @ Uv - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(A - (Uv * w) @ Uv.T) <= 1e-12 * np.linalg.norm(A)
    if 2 < n <= 150:
        # the trees may differ where a split score sits near its threshold;
        # the eigenvalues are unique
        wo, Uo, io = oeig_sym(A, seed=5, leaf_size=leaf)
        assert io.status == 0
        assert np.max(np.abs(w - wo)) <= 1e-12 * nA


def test_eig_solve_symmetric_degenerate(E):
    """Zero matrix, identity multiple, a 2-value spectrum (clusters)."""
    eigdc, h, torch = E
    for A in (np.zeros((70, 70)), 3.0 * np.eye(90)):
        rc, w, Uv, info = eigdc.solve_symmetric(h, A, eigdc.default_params(leaf_size=64))
        assert rc in (eigdc.EIG_OK, eigdc.EIG_NO_SPLIT)
    rng = np.random.default_rng(2)
    n = 130
    lam = np.where(np.arange(n) < 60, -0.5, 0.5)
    Q = workloads.random_orthogonal(n, rng)
    A = (Q * lam) @ Q.T
    rc, w, Uv, info = eigdc.solve_symmetric(h, A, eigdc.default_params(seed=3))
    assert rc == eigdc.EIG_OK
    assert np.max(np.abs(w - np.sort(lam))) <= 1e-10
    assert np.linalg.norm(A - (Uv * w) @ Uv.T) <= 1e-12 * np.linalg.norm(A)


def test_nonfinite_input_rejected(E):
    eigdc, h, torch = E
    A = np.eye(80)
    A[3, 4] = np.nan
    rc, w, Uv, info = eigdc.solve_symmetric(h, A)
    assert rc == eigdc.EIG_NONFINITE


def test_argument_errors(E):
    eigdc, h, torch = E
    reg = eigdc.Region(7, 0.0, 1.0)
    dA = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    rc, _ = eigdc.eig_divide_step(h, 4, dA, 4, None, 0, reg, eigdc.default_params())
    assert rc == eigdc.EIG_ERR_ARG and "region" in h.last_error()
    rc, _ = eigdc.eig_divide_step(h, 4, dA, 2, None, 0, eigdc.Region(0, 0, 1), eigdc.default_params())
    assert rc == eigdc.EIG_ERR_ARG


def test_jordan_case_reports_no_split(E):
    """Sec. 3.3.1, Fig. 2(b): the line Re z = 0 meets the pseudospectrum."""
    eigdc, h, torch = E
    A = workloads.jordan_hard(32)
    n = 32
    dA = eigdc.to_device(A)
    rc, info = eigdc.eig_divide_step(h, n, dA, n, None, 0, eigdc.Region(2, 0.0, 1.0),
                                     eigdc.default_params(maxit=60))
    st = odivide_step(A, None, (REGION_LINE, 0.0, 1.0), seed=1, maxit=60)
    assert not st.accepted
    if rc == eigdc.EIG_OK:
        # converged R-test: the split must still be rejected
        Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
        dAp, dBp = eigdc.to_device(Am), eigdc.to_device(Bm)
        eigdc.eig_divide_step(h, n, dAp, n, dBp, n, eigdc.Region(0, 0.0, 1.0), eigdc.default_params())
        dQ = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        rc2, si = eigdc.eig_split(h, n, dAp, dBp, n, eigdc.to_device(A), n, dQ, n, 0, 1, 0,
                                  eigdc.default_params(seed=1))
        assert rc2 == eigdc.EIG_NO_SPLIT
    else:
        assert rc == eigdc.EIG_NO_CONVERGENCE and info.iters == 61


def _eig_condition(T):
    """kappa_i = ||y_i|| ||x_i|| / |y_i^H x_i| from left/right eigenvectors (test side)."""
    wr0, VR = np.linalg.eig(T)
    wl, VL = np.linalg.eig(T.T)
    kap = np.zeros(T.shape[0])
    for i in range(T.shape[0]):
        j = int(np.argmin(np.abs(wl - wr0[i])))
        kap[i] = np.linalg.norm(VL[:, j]) * np.linalg.norm(VR[:, i]) / abs(VL[:, j] @ VR[:, i])
    # reorder to match the diagonal of the (triangular) T
    out = np.zeros_like(kap)
    d = np.diag(T)
    for i in range(len(d)):
        out[i] = kap[int(np.argmin(np.abs(wr0 - d[i])))]
    return out


@pytest.mark.parametrize("n,leaf", [(40, 64), (128, 32), (200, 64)])
def test_schur_nonsymmetric(E, n, leaf):
    eigdc, h, torch = E
    A, d, T0 = workloads.nonsymmetric_schur(n, seed=4)
    p = eigdc.default_params(seed=2, leaf_size=leaf)
    rc, T, Us, wr, wi, info = eigdc.schur_nonsymmetric(h, A, p)
    assert rc == eigdc.EIG_OK
    assert np.linalg.norm(A - Us @ T @ Us.T) / np.linalg.norm(A) <= 1e-12
    assert np.linalg.norm(Us.T @ Us - np.eye(n), 2) <= 1e-12
    assert np.all(np.tril(T, -2) == 0.0)
    To, Qo, wro, wio, io = oschur(A, seed=2, leaf_size=leaf)
    assert io.status == 0
    # eigenvalues of the non-normal T0 are sensitive: compare within the
    # condition-number bound |dl_i| <= c n u kappa_i ||A||_2 (both sides are
    # backward stable to ~1e-13)
    assert np.all(wi == 0.0)
    kappa = _eig_condition(T0)
    order = np.argsort(d)
    nA = np.linalg.norm(A, 2)
    tol = 1e-13 * n * kappa[order] * nA + 1e-12
    assert np.all(np.abs(np.sort(wr) - d[order]) <= tol)
    assert np.all(np.abs(np.sort(wr) - np.sort(wro)) <= 2 * tol)


def test_schur_complex_pairs(E):
    """Real normal matrix with conjugate pairs: 2x2 blocks in standard form."""
    eigdc, h, torch = E
    A, _ = workloads.normal_complex(90, seed=3)
    rc, T, Us, wr, wi, info = eigdc.schur_nonsymmetric(h, A, eigdc.default_params(seed=1))
    assert rc == eigdc.EIG_OK
    assert np.linalg.norm(A - Us @ T @ Us.T) / np.linalg.norm(A) <= 1e-12
    ev = np.sort_complex(np.linalg.eigvals(A))
    got = np.sort_complex(wr + 1j * wi)
    assert np.max(np.abs(ev - got)) <= 1e-10
    assert np.sum(wi != 0) >= 80
