"""FP64-accurate tensor-core contractions (EIG_FP64_TC) on the GPU.

The error-free split cuts every row of op(A) and column of op(B) into nine
signed 6-bit digits in balanced form (|digit| <= 32, 53 bits below a
power-of-two scale 2^e, the last digit rounded) and keeps the digit-pair
levels 0..9, each accumulated exactly in FP32 over 1792-wide K chunks.  Error
model per element, with a = max |row of op(A)|, b = max |column of op(B)|:
digit rounding <= 2 * 2^-53 a b per term, dropped levels <= 2^-59 a b per
term, FP64 drain rounding ~ 10 u |c| per chunk.  Tests use
|C - C_ref| <= 16 k u a b (u = 2^-53), which also covers the FP64 rounding of
the reference; an inexact FP32 accumulation would break it by ~2^29.  Shapes
with k > 1792 (up to 4100 here) span several exact chunks.
Integer operands whose digits are exact give an exactly integer product: that
pins the exactness of the tensor-core accumulation bit for bit.
Whole solves in EIG_FP64_TC meet the FP64 targets (eigenvalue error
<= 1e-10 ||A||, orthogonality and backward error <= 1e-12) and take the same
recursion (splits) as the FP64 path, whose kernels are pinned to the oracle.
"""
import numpy as np
import pytest

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


def _op(X, t):
    return X.T if t else X


def _run(eigdc, h, torch, A, B, ta, tb, alpha=1.0, beta=0.0, C0=None):
    m = _op(A, ta).shape[0]
    n = _op(B, tb).shape[1]
    k = _op(A, ta).shape[1]
    dA, dB = eigdc.to_device(A), eigdc.to_device(B)
    dC = eigdc.to_device(C0 if C0 is not None else np.zeros((m, n)))
    eigdc.eig_gemm_fp64tc(h, ta, tb, m, n, k, alpha, dA, A.shape[0], dB, B.shape[0], beta, dC,
                          m)
    return eigdc.to_host(dC)


@pytest.mark.parametrize("m,n,k,ta,tb", [
    (1, 1, 1, 0, 0), (63, 65, 17, 0, 0), (130, 70, 300, 1, 0), (128, 48, 448, 0, 0),
    (200, 100, 1000, 0, 1), (257, 129, 2048, 1, 0), (64, 130, 33, 1, 1), (700, 500, 4100, 0, 0),
    (128, 48, 1792, 0, 0), (96, 60, 3585, 1, 1)])
def test_fp64tc_gemm_accuracy(E, m, n, k, ta, tb):
    eigdc, h, torch = E
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    # rows / columns of very different magnitude exercise the per-row scale
    oA, oB = _op(A, ta), _op(B, tb)
    oA *= np.exp2(rng.integers(-40, 40, size=(m, 1)))
    oB *= np.exp2(rng.integers(-40, 40, size=(1, n)))
    C0 = rng.standard_normal((m, n))
    got = _run(eigdc, h, torch, A, B, ta, tb, alpha=1.5, beta=-0.5, C0=C0)
    ref = 1.5 * (oA @ oB) - 0.5 * C0
    a = np.max(np.abs(oA), axis=1)[:, None]
    b = np.max(np.abs(oB), axis=0)[None, :]
    tol = 16 * k * U * 1.5 * a * b + 4 * U * np.abs(C0)
    assert np.all(np.abs(got - ref) <= tol)


def test_fp64tc_integer_product_is_exact(E):
    """Integer operands below 2^10: two digits hold each entry exactly, every
    level sum is an exact integer, so C must equal the int64 product."""
    eigdc, h, torch = E
    rng = np.random.default_rng(5)
    m, n, k = 300, 200, 4096
    Ai = rng.integers(-1000, 1001, size=(m, k))
    Bi = rng.integers(-1000, 1001, size=(k, n))
    got = _run(eigdc, h, torch, Ai.astype(np.float64), Bi.astype(np.float64), 0, 0)
    exact = Ai @ Bi
    assert np.array_equal(got, exact.astype(np.float64))


def test_fp64tc_zero_and_special_rows(E):
    eigdc, h, torch = E
    rng = np.random.default_rng(9)
    m, n, k = 150, 90, 700
    A = rng.standard_normal((m, k))
    A[3] = 0.0
    A[7] = 1e-300 * rng.standard_normal(k)   # near the bottom of the range
    B = rng.standard_normal((k, n))
    B[:, 4] = 0.0
    got = _run(eigdc, h, torch, A, B, 0, 0)
    ref = A @ B
    assert np.all(got[3] == 0.0) and np.all(got[:, 4] == 0.0)
    a = np.max(np.abs(A), axis=1)[:, None]
    b = np.max(np.abs(B), axis=0)[None, :]
    assert np.all(np.abs(got - ref) <= 16 * k * U * a * b)


def _solve_pair(eigdc, h, kind, A, seed, leaf=64):
    out = {}
    for prec in (eigdc.EIG_FP64, eigdc.EIG_FP64_TC):
        p = eigdc.default_params(seed=seed, leaf_size=leaf, prec=prec)
        if kind == eigdc.EIG_KIND_SYM:
            out[prec] = eigdc.solve_symmetric(h, A, p)
        else:
            out[prec] = eigdc.schur_nonsymmetric(h, A, p)
    return out


@pytest.mark.parametrize("n", [400, 700])
def test_fp64tc_symmetric_solve(E, n):
    eigdc, h, torch = E
    A, lam = workloads.symmetric_uniform(n, seed=n)
    out = _solve_pair(eigdc, h, eigdc.EIG_KIND_SYM, A, seed=3)
    rc, w, Us, info = out[eigdc.EIG_FP64_TC]
    assert rc == eigdc.EIG_OK
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert np.linalg.norm(Us.T @ Us - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(A - (Us * w) @ Us.T) / np.linalg.norm(A) <= 1e-12
    assert info.splits == out[eigdc.EIG_FP64][3].splits


def test_fp64tc_nonsymmetric_solve(E):
    eigdc, h, torch = E
    n = 500
    A, d, _ = workloads.nonsymmetric_schur(n, seed=4, offdiag_scale=0.1 / np.sqrt(n))
    out = _solve_pair(eigdc, h, eigdc.EIG_KIND_NONSYM, A, seed=2)
    rc, T, Us, wr, wi, info = out[eigdc.EIG_FP64_TC]
    assert rc == eigdc.EIG_OK
    assert np.linalg.norm(A - Us @ T @ Us.T) / np.linalg.norm(A) <= 1e-12
    assert np.linalg.norm(Us.T @ Us - np.eye(n), 2) <= 1e-12
    assert np.all(np.tril(T, -2) == 0.0)
    assert np.max(np.abs(np.sort(wr) - np.sort(d))) <= 1e-9
    assert info.splits == out[eigdc.EIG_FP64][5].splits


def test_fp64tc_pencil_solve(E):
    eigdc, h, torch = E
    n = 450
    A, B, d = workloads.regular_pencil(n, seed=2, offdiag_scale=0.1 / np.sqrt(n))
    res = {}
    for prec in (eigdc.EIG_FP64, eigdc.EIG_FP64_TC):
        res[prec] = eigdc.pencil_schur(h, A, B, eigdc.default_params(seed=3, prec=prec))
    rc, S, T, QL, QR, ar, ai, be, info = res[eigdc.EIG_FP64_TC]
    assert rc == eigdc.EIG_OK
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    assert np.linalg.norm(QL.T @ QL - np.eye(n), 2) <= 1e-12
    assert np.max(np.abs(np.sort(ar / be) - np.sort(d))) <= 1e-9
    assert info.splits == res[eigdc.EIG_FP64][-1].splits


@pytest.mark.parametrize("n,sq", [(600, 2), (777, 1)])
def test_fp64tc_two_level_irs_iterates_match_oracle(E, n, sq):
    """At these sizes the QR of the stacked 2n x n matrix and the complement
    Q [0; I] run in the two-level form (256-column outer blocks whose
    aggregated reflectors update the trailing matrix on the tensor cores):
    exactly `sq` squarings (R-test off) give the oracle's A_p, B_p and
    R_{p-1} elementwise (tolerance of the FP64 iterate tests, the error-free
    split keeping FP64 accuracy)."""
    eigdc, h, torch = E
    from oracle.irs import irs as oirs
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n)) + 2 * np.eye(n)
    dA, dB = eigdc.to_device(A), eigdc.to_device(B)
    reg = eigdc.Region(0, 0.0, 1.0)
    p = eigdc.default_params(tau=-1.0, maxit=sq - 1, prec=eigdc.EIG_FP64_TC)
    rc, info = eigdc.eig_divide_step(h, n, dA, n, dB, n, reg, p)
    assert rc == eigdc.EIG_NO_CONVERGENCE and info.iters == sq
    res = oirs(A, B, tau=-1.0, maxit=sq - 1, record_R=True)
    scale = np.linalg.norm(np.vstack([A, B]), 2)
    assert np.max(np.abs(eigdc.to_host(dA) - res.Ap)) <= 1e-11 * scale
    assert np.max(np.abs(eigdc.to_host(dB) - res.Bp)) <= 1e-11 * scale
    dR = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eigdc.eig_last_R(h, n, dR, n)
    assert np.max(np.abs(eigdc.to_host(dR) - res.Rs[-1])) <= 1e-11 * scale


def test_irs_floor_stop_in_fp64tc(E):
    """R-test with tau far below the rounding floor of the ratio (1e-18):
    plain FP64 keeps the oracle's test and runs into maxit (j = 0..maxit), the
    FP64-accurate tensor-core form also stops once the ratio is <= 1e-10 and
    falls less than 4x over a squaring (the floor), well before maxit."""
    eigdc, h, torch = E
    n = 300
    rng = np.random.default_rng(11)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n)) + 2 * np.eye(n)
    reg = eigdc.Region(0, 0.0, 1.0)
    out = {}
    for prec in (eigdc.EIG_FP64, eigdc.EIG_FP64_TC):
        dA, dB = eigdc.to_device(A), eigdc.to_device(B)
        p = eigdc.default_params(tau=1e-18, maxit=40, prec=prec)
        rc, info = eigdc.eig_divide_step(h, n, dA, n, dB, n, reg, p)
        out[prec] = (rc, info, eigdc.to_host(dA))
    rc0, i0, A0 = out[eigdc.EIG_FP64]
    rc1, i1, A1 = out[eigdc.EIG_FP64_TC]
    assert rc0 == eigdc.EIG_NO_CONVERGENCE and i0.iters == 41 and i0.converged == 0
    assert rc1 == eigdc.EIG_OK and i1.converged == 1 and i1.iters < 41
    assert 0.0 <= i1.last_ratio <= 1e-10
    assert np.all(np.isfinite(A1))
