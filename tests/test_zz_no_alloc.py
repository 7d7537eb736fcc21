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


def _case(rng, m, n, k, ta, tb):
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    return A, B, C


@pytest.mark.parametrize("m,n,k,ta,tb", [
    (64, 64, 4096, 1, 0),     # 16 K-chunks: uses the static scratch
    (130, 70, 1300, 0, 1),    # a few K-chunks, ragged tiles
    (300, 257, 5, 0, 0),      # no split: the scratch is not touched
])
def test_noalloc_matches_eig_gemm_twice(env, m, n, k, ta, tb):
    eigdc, h, torch = env
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


def test_noalloc_rejects_oversized_scratch(env):
    eigdc, h, torch = env
    m = n = 512
    k = 8192              # 5 K-chunks of 512 x 512 > 2^20 doubles
    dA = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    dB = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    dC = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    rc = eigdc.eig_gemm_noalloc(torch.cuda.current_stream(), 0, 0, m, n, k, 1.0, dA, m, dB, k,
                                0.0, dC, m)
    assert rc == eigdc.EIG_ERR_SCRATCH
