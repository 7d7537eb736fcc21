"""eig_gemm_noalloc against eig_gemm (GPU).

The no-allocation GEMM is for callers that cannot call cudaMalloc (device
memory reserved by another allocator's pool, or loops that cannot take an
allocation's device synchronisation).  It keeps its split-K scratch in a
static device array, so these checks call it twice in a row (the second call
reuses the array the first one left behind) and compare each result with the
workspace-based eig_gemm, within the GEMM tolerance of the parity tests:
|C - C_ref| <= 8 k u max|A| max|B| + 4 u max|C|.  This file sorts last so a
run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1011_3077_gb300 import build, eigdc
    build.build()
    h = eigdc.Handle(0)
    yield eigdc, h, torch
    torch.cuda.synchronize()
    h.close()


def _splits(m, n, k):
    """K-chunk count the library's split-K chooser picks for an m x n x k
    product: whole waves of two CTAs per SM on 152 SMs, chunks of at least
    128, at most 32 (restated here so each case can assert which path, the
    static scratch or none, it exercises)."""
    bm, bn = (32, 128) if m <= 32 else (64, 64)
    tiles = -(-m // bm) * -(-n // bn)
    wave = 2 * 152
    if tiles >= wave:
        return 1
    best, best_eff = 1, 0.0
    for s in range(1, max(1, min(32, k // 128)) + 1):
        ctas = tiles * s
        waves = -(-ctas // wave)
        eff = ctas / (waves * wave) - 0.002 * s
        if eff > best_eff:
            best, best_eff = s, eff
    return best


SCRATCH = 1 << 20   # doubles in the library's static split-K array


def _case(rng, m, n, k, ta, tb):
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    return A, B, C


@pytest.mark.parametrize("m,n,k,ta,tb,split", [
    (64, 64, 4096, 1, 0, True),     # many K-chunks in the static scratch
    (130, 70, 1300, 0, 1, True),    # a few K-chunks, ragged tiles
    (256, 256, 2048, 0, 0, True),   # splits * m * n exactly fills the scratch
    (300, 257, 5, 0, 0, False),     # no split: the scratch is not touched
])
def test_noalloc_matches_eig_gemm_twice(env, m, n, k, ta, tb, split):
    eigdc, h, torch = env
    s = _splits(m, n, k)
    assert (s > 1) == split and s * m * n <= SCRATCH
    if (m, n, k) == (256, 256, 2048):
        assert s * m * n == SCRATCH
    rng = np.random.default_rng(m * 31 + k)
    stream = torch.cuda.current_stream()
    for call in range(2):
        A, B, C = _case(rng, m, n, k, ta, tb)
        alpha, beta = 0.75, -0.5 + call
        dA, dB = eigdc.to_device(A), eigdc.to_device(B)
        dC1, dC2 = eigdc.to_device(C), eigdc.to_device(C)
        eigdc.eig_gemm(h, ta, tb, m, n, k, alpha, dA, eigdc.ld(dA), dB, eigdc.ld(dB), beta,
                       dC1, eigdc.ld(dC1))
        rc = eigdc.eig_gemm_noalloc(stream, ta, tb, m, n, k, alpha, dA, eigdc.ld(dA), dB,
                                    eigdc.ld(dB), beta, dC2, eigdc.ld(dC2))
        assert rc == eigdc.EIG_OK
        torch.cuda.synchronize()
        got, ref = eigdc.to_host(dC2), eigdc.to_host(dC1)
        tol = 8 * k * U * np.abs(A).max() * np.abs(B).max() + 4 * U * np.abs(C).max()
        assert np.max(np.abs(got - ref)) <= tol
        exact = alpha * ((A.T if ta else A) @ (B.T if tb else B)) + beta * C
        assert np.max(np.abs(got - exact)) <= tol


@pytest.mark.parametrize("m,n,k", [
    (512, 512, 8192),    # splits * m * n far above 2^20 doubles
    (256, 256, 2176),    # one K-chunk more than the exact fit above
])
def test_noalloc_rejects_oversized_scratch(env, m, n, k):
    eigdc, h, torch = env
    assert _splits(m, n, k) * m * n > SCRATCH
    dA = torch.zeros((k, m), dtype=torch.float64, device="cuda")
    dB = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    rc = eigdc.eig_gemm_noalloc(torch.cuda.current_stream(), 0, 0, m, n, k, 1.0, dA, m, dB, k,
                                0.0, dC, m)
    assert rc == eigdc.EIG_ERR_SCRATCH
