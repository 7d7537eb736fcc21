"""Split-precision (BF16 x 3 on tcgen05) contractions against FP64 references (GPU).

Error model of the three-term split: each FP64 entry x = hi + mid + lo with
|x - (hi + mid + lo)| <= 2^-24 |x|; the six kept products drop terms of size
<= 3 * 2^-24 |a||b|, and FP32 accumulation over k terms adds at most about
k * 2^-24 sum |a_i b_i| (typically sqrt(k) * 2^-24).  Tests use
|C - C_ref| <= 2^-20 * sum_i |a_i||b_i| elementwise, a loose form of that bound
that still fails by orders of magnitude on a wrong plane, sign or transpose.
Measured on GB300: 5e-7 (k = 64) to 2.6e-6 (k = 4096) relative to
sum |a_i||b_i|; the tensor cores' FP32 accumulation grows with k, so the
bound is 2^-16 (and a plain single-plane BF16 product would sit near 2^-9).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    from paper_1011_3077_gb300 import build, eigdc
    build.build()
    h = eigdc.Handle(0)
    yield eigdc, h, torch
    torch.cuda.synchronize()
    h.close()


@pytest.mark.parametrize("m,n,k,ta,tb", [
    (128, 128, 64, 1, 0), (128, 128, 64, 0, 0), (130, 70, 300, 1, 0), (1, 1, 1, 0, 0),
    (64, 200, 129, 0, 1), (257, 129, 1000, 1, 1), (512, 512, 2048, 1, 0), (300, 32, 4096, 1, 0),
    (100, 90, 0, 0, 0)])
def test_split_gemm_matches_fp64(E, m, n, k, ta, tb):
    eigdc, h, torch = E
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    alpha, beta = 1.25, -0.5
    opA = A.T if ta else A
    opB = B.T if tb else B
    ref = alpha * (opA @ opB) + beta * C
    dA, dB, dC = eigdc.to_device(A), eigdc.to_device(B), eigdc.to_device(C)
    lda = max(1, A.shape[0])
    ldb = max(1, B.shape[0])
    eigdc.eig_gemm_split(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, eigdc.ld(dC))
    got = eigdc.to_host(dC)
    scale = abs(alpha) * (np.abs(opA) @ np.abs(opB)) + 1e-300
    err = np.abs(got - ref)
    rel = float(np.max(err / scale)) if k > 0 else float(np.max(err))
    print("m=%d n=%d k=%d ta=%d tb=%d: max err / sum|a||b| = %.3e" % (m, n, k, ta, tb, rel))
    if k == 0:
        assert np.allclose(got, beta * C, atol=1e-15)
    else:
        assert rel <= 2.0 ** -16


# ------------------------------------------------------------------ the path in split precision
def test_split_divide_step_config1(E):
    """IRS with split-precision products: iterates at equal squaring counts match
    the FP64 oracle to the FP32 level, and the R-test (or its stagnation) fires."""
    eigdc, h, torch = E
    from paper_1011_3077_gb300 import workloads
    from oracle.irs import irs as oirs, region_map, REGION_LINE
    A, lam = workloads.symmetric_split(256, seed=1)
    n = 256
    Am, Bm = region_map(A, None, REGION_LINE, 0.0, 1.0)
    for sq in (1, 3, 6):
        dA, dB = eigdc.to_device(Am), eigdc.to_device(Bm)
        rc, info = eigdc.eig_divide_step(h, n, dA, n, dB, n, eigdc.Region(0, 0.0, 1.0),
                                         eigdc.default_params(prec=eigdc.EIG_SPLIT_BF16X3,
                                                              tau=-1.0, maxit=sq - 1))
        res = oirs(Am, Bm, tau=-1.0, maxit=sq - 1)
        scale = np.linalg.norm(np.vstack([Am, Bm]), 2)
        err = max(np.max(np.abs(eigdc.to_host(dA) - res.Ap)), np.max(np.abs(eigdc.to_host(dB) - res.Bp)))
        print("split IRS %d squarings: max iterate difference %.2e (relative)" % (sq, err / scale))
        assert err <= 1e-4 * scale
    dA = eigdc.to_device(A)
    rc, info = eigdc.eig_divide_step(h, n, dA, n, None, 0, eigdc.Region(2, 0.0, 1.0),
                                     eigdc.default_params(prec=eigdc.EIG_SPLIT_BF16X3))
    assert rc == eigdc.EIG_OK and info.converged and info.iters <= 14


@pytest.mark.parametrize("n", [200, 400])
def test_split_symmetric_solve_refined(E, n):
    """Split-precision recursion + FP64 refinement meets the FP64 targets."""
    eigdc, h, torch = E
    from paper_1011_3077_gb300 import workloads
    from oracle.solve import eig_sym
    A, lam = workloads.symmetric_uniform(n, seed=n + 1)
    p = eigdc.default_params(seed=7, prec=eigdc.EIG_SPLIT_BF16X3)
    rc, w, Uv, info = eigdc.solve_symmetric(h, A, p)
    assert rc == eigdc.EIG_OK
    nA = np.linalg.norm(A, 2)
    ev_err = np.max(np.abs(w - lam)) / nA
    orth = np.linalg.norm(Uv.T @ Uv - np.eye(n), 2)
    bwd = np.linalg.norm(A - (Uv * w) @ Uv.T) / np.linalg.norm(A)
    msg = "split n=%d: eig err %.2e, orth %.2e, bwd %.2e, splits %d" % (n, ev_err, orth, bwd, info.splits)
    if n <= 200:
        # error against the FP64 oracle's eigenvalues (unique; the trees may differ)
        wo, Uo, io = eig_sym(A, seed=7)
        gap = np.max(np.abs(w - wo)) / nA
        msg += ", |w - w_oracle|/|A| = %.2e" % gap
        assert io.status == 0 and gap <= 1e-10
    print(msg)
    assert ev_err <= 1e-10
    assert orth <= 1e-12
    assert bwd <= 1e-12


# ------------------------------------------------------------------ unbiased FP32-level form
@pytest.mark.parametrize("m,n,k,ta,tb", [
    (128, 96, 64, 1, 0), (130, 70, 300, 0, 1), (257, 129, 1000, 1, 1), (64, 200, 4100, 0, 0),
    (300, 48, 16384, 1, 0), (5, 3, 7, 0, 0)])
def test_fp32tc_gemm_bound(E, m, n, k, ta, tb):
    """Four-digit error-free split: every product term is off by at most about
    2^-24 of its row / column maxima (truncated digits, the last rounded, and
    the dropped weight levels), accumulation exact; bound 8 k 2^-24 rowmax colmax."""
    eigdc, h, torch = E
    rng = np.random.default_rng(m + 3 * n + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = 0.5 * (opA @ opB) - 2.0 * C
    dA, dB, dC = eigdc.to_device(A), eigdc.to_device(B), eigdc.to_device(C)
    eigdc.eig_gemm_fp32tc(h, ta, tb, m, n, k, 0.5, dA, max(1, A.shape[0]), dB,
                          max(1, B.shape[0]), -2.0, dC, eigdc.ld(dC))
    got = eigdc.to_host(dC)
    bound = 0.5 * 8 * k * 2.0 ** -24 * np.abs(opA).max(axis=1)[:, None] * \
        np.abs(opB).max(axis=0)[None, :] + 4 * 2.0 ** -53 * np.abs(2.0 * C)
    assert np.all(np.abs(got - ref) <= bound)


def test_fp32tc_has_no_accumulation_bias(E):
    """Positive data: BF16 x 3 drifts by about -6e-9 k relative (its FP32
    accumulator truncates every addition: -1e-4 at k = 16384 measured).  The
    exact chunked form keeps only the K-independent offset of the dropped
    weight levels 4.. (all of one sign for positive data): at most about
    5 x 2^-24 relative (measured -1.8e-7), the same at k = 512 and 16384."""
    eigdc, h, torch = E
    m = n = 256
    means = []
    for k in (512, 16384):
        rng = np.random.default_rng(5 + k)
        A = rng.uniform(0, 1, (m, k))
        B = rng.uniform(0, 1, (k, n))
        ref = A @ B
        dA, dB = eigdc.to_device(A), eigdc.to_device(B)
        dC = eigdc.to_device(np.zeros((m, n)))
        eigdc.eig_gemm_fp32tc(h, 0, 0, m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m)
        rel = (eigdc.to_host(dC) - ref) / ref
        assert abs(rel.mean()) <= 2.0 ** -21 and np.abs(rel).max() <= 2.0 ** -20
        means.append(rel.mean())
    assert abs(means[1]) <= 2.0 * abs(means[0]) + 2.0 ** -24


@pytest.mark.parametrize("n", [300, 700])
def test_split_fp32_symmetric_solve(E, n):
    """EIG_SPLIT_FP32 recursion + FP64 refinement meets the FP64 targets and
    the FP64 oracle's eigenvalues."""
    eigdc, h, torch = E
    from paper_1011_3077_gb300 import workloads
    from oracle.solve import eig_sym
    A, lam = workloads.symmetric_semicircle(n, seed=n + 3)
    rc, w, Uv, info = eigdc.solve_symmetric(h, A, eigdc.default_params(
        seed=7, prec=eigdc.EIG_SPLIT_FP32))
    assert rc == eigdc.EIG_OK, h.last_error()
    nA = np.max(np.abs(lam))
    assert np.max(np.abs(w - lam)) <= 1e-10 * nA
    assert np.linalg.norm(Uv.T @ Uv - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(A - (Uv * w) @ Uv.T) <= 1e-12 * np.linalg.norm(A)
    if n <= 300:
        wo, Uo, io = eig_sym(A, seed=7)
        assert io.status == 0 and np.max(np.abs(w - wo)) <= 1e-10 * nA
