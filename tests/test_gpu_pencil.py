"""GPU parity of the pencil path (RGNEP, Algorithm 4, Sec. 3.5) against the oracle.

Tolerances (FP64, u = 2^-53):
  * one step: k and the RURV rank must agree exactly; the leading blocks
    A^11 = Q_L(:, :k)^T A Q_R(:, :k) and B^11 are determined by stable
    subspaces and their Gram-Schmidt bases (positive-diagonal QR convention),
    so they agree elementwise to 1e-10 ||(A, B)||; the trailing blocks carry
    bases chosen by rounding, so only their generalized eigenvalues are
    compared;
  * whole solves: backward errors ||A - Q_L S Q_R^T||_F <= 1e-12 ||A||_F (and
    for B), orthogonality <= 1e-12, exact zero patterns, eigenvalues within
    1e-10 of the prescribed ones and of the oracle's; the recursion tree (number
    of splits and leaves) equals the oracle's, since every decision (k, rank,
    swap) is a well-separated integer.
"""
import numpy as np
import pytest

from oracle.irs import REGION_UNIT_CIRCLE, REGION_LINE, region_map
from oracle.solve import divide_step as odivide_step, pencil_schur as opencil
from paper_1011_3077_gb300 import workloads

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


def _gen_eigs(A, B):
    from scipy.linalg import eigvals
    return eigvals(A, B)


def _gpu_pencil_step(eigdc, h, torch, A, B, region, seed, stream, attempt):
    n = A.shape[0]
    kind, c, r = region
    reg = eigdc.Region(kind, c, r)
    p = eigdc.default_params(seed=seed)
    dAR, dBR = eigdc.to_device(A), eigdc.to_device(B)
    rc1, i1 = eigdc.eig_divide_step(h, n, dAR, n, dBR, n, reg, p)
    dAL, dBL = eigdc.to_device(A.T.copy()), eigdc.to_device(B.T.copy())
    rc2, i2 = eigdc.eig_divide_step(h, n, dAL, n, dBL, n, reg, p)
    assert rc1 == eigdc.EIG_OK and rc2 == eigdc.EIG_OK
    dA, dB = eigdc.to_device(A), eigdc.to_device(B)
    z = lambda: torch.zeros((n, n), dtype=torch.float64, device="cuda")
    dQL, dQR = z(), z()
    rc, si = eigdc.eig_split_pencil(h, n, dAR, dBR, dAL, dBL, n, dA, n, dB, n, dQL, n, dQR, n,
                                    stream, attempt, p)
    return (rc, si, i1, i2, eigdc.to_host(dAR), eigdc.to_host(dAL), eigdc.to_host(dA),
            eigdc.to_host(dB), eigdc.to_host(dQL), eigdc.to_host(dQR))


@pytest.mark.parametrize("n,region", [(150, (REGION_UNIT_CIRCLE, 0.0, 1.0)),
                                      (97, (REGION_LINE, 0.3, 1.0))])
def test_pencil_step_matches_oracle(E, n, region):
    eigdc, h, torch = E
    A, B, d = workloads.regular_pencil(n, seed=2, offdiag_scale=0.1 / np.sqrt(n))
    seed, stream = 77, 1
    st = odivide_step(A, B, region, seed=seed, stream=stream, attempt=0)
    assert st.accepted
    rc, si, i1, i2, ApR, ApL, Ah, Bh, QL, QR = _gpu_pencil_step(eigdc, h, torch, A, B, region,
                                                               seed, stream, 0)
    assert rc == eigdc.EIG_OK
    assert i1.iters == st.irs.iters and i2.iters == st.irs_left.iters
    scale = np.linalg.norm(np.vstack(region_map(A, B, *region)), 2)
    assert np.max(np.abs(ApR - st.irs.Ap)) <= 1e-10 * scale
    assert np.max(np.abs(ApL - st.irs_left.Ap)) <= 1e-10 * scale
    k = si.k
    assert k == st.k and si.rank == st.rank and si.draw == st.draw
    # the pencil score is rounding-dominated (two independently computed
    # subspaces); its floor depends on the summation order, so 1e-11, ten
    # times below the pencil acceptance threshold
    assert si.split_residual <= 1e-11
    sAB = max(np.linalg.norm(A, 2), np.linalg.norm(B, 2))
    assert np.max(np.abs(Ah[:k, :k] - st.Ahat[:k, :k])) <= 1e-10 * sAB
    assert np.max(np.abs(Bh[:k, :k] - st.Bhat[:k, :k])) <= 1e-10 * sAB
    assert np.max(np.abs(QL.T @ QL - np.eye(n))) <= 1e-13
    assert np.max(np.abs(QR.T @ QR - np.eye(n))) <= 1e-13
    # the split itself: Q_L^T (A, B) Q_R and the blocks' spectra
    assert np.max(np.abs(QL.T @ A @ QR - Ah)) <= 1e-12 * sAB
    if region[0] == REGION_UNIT_CIRCLE:
        outside = np.sort(d[np.abs(d) > 1.0])
        inside = np.sort(d[np.abs(d) < 1.0])
    else:
        outside = np.sort(d[d > region[1]])
        inside = np.sort(d[d < region[1]])
    assert k == len(outside)
    assert np.allclose(np.sort(_gen_eigs(Ah[:k, :k], Bh[:k, :k]).real), outside, atol=1e-9)
    assert np.allclose(np.sort(_gen_eigs(Ah[k:, k:], Bh[k:, k:]).real), inside, atol=1e-9)


def _check_form(A, B, S, T, QL, QR, ar, ai, be):
    n = A.shape[0]
    assert np.linalg.norm(A - QL @ S @ QR.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(B - QL @ T @ QR.T) <= 1e-12 * np.linalg.norm(B)
    assert np.linalg.norm(QL.T @ QL - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(QR.T @ QR - np.eye(n), 2) <= 1e-12
    assert np.all(np.tril(T, -1) == 0.0) and np.all(np.tril(S, -2) == 0.0)
    # a nonzero subdiagonal of S only inside a marked complex pair
    for i in range(n - 1):
        if S[i + 1, i] != 0.0:
            assert ai[i] > 0 and ai[i + 1] == -ai[i]


@pytest.mark.parametrize("n,leaf,workers", [(150, 40, 1), (200, 64, 8), (60, 64, 1)])
def test_pencil_schur_matches_oracle(E, n, leaf, workers):
    eigdc, h, torch = E
    A, B, d = workloads.regular_pencil(n, seed=2, offdiag_scale=0.1 / np.sqrt(n))
    p = eigdc.default_params(seed=3, leaf_size=leaf, workers=workers)
    rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(h, A, B, p)
    assert rc == eigdc.EIG_OK
    _check_form(A, B, S, T, QL, QR, ar, ai, be)
    So, To, QLo, QRo, aro, aio, beo, io = opencil(A, B, seed=3, leaf_size=leaf)
    assert io.status == 0
    assert info.splits == io.splits and info.nodes == io.nodes
    assert np.all(ai == 0.0)
    got = np.sort(ar / be)
    assert np.allclose(got, np.sort(d), atol=1e-10)
    assert np.allclose(got, np.sort(aro / beo), atol=1e-10)


def test_pencil_schur_complex_pairs(E):
    eigdc, h, torch = E
    n = 100
    M, _ = workloads.normal_complex(n, seed=5)
    rng = np.random.default_rng(3)
    B = np.eye(n) + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n)
    A = M @ B
    rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(
        h, A, B, eigdc.default_params(seed=4, leaf_size=40))
    assert rc == eigdc.EIG_OK
    _check_form(A, B, S, T, QL, QR, ar, ai, be)
    So, To, QLo, QRo, aro, aio, beo, io = opencil(A, B, seed=4, leaf_size=40)
    assert info.splits == io.splits
    got = np.sort_complex((ar + 1j * ai) / be)
    assert np.max(np.abs(got - np.sort_complex(np.linalg.eigvals(M)))) <= 1e-10
    assert np.max(np.abs(got - np.sort_complex((aro + 1j * aio) / beo))) <= 1e-10
    assert np.sum(ai != 0) >= 80


def test_pencil_schur_infinite_eigenvalues(E):
    """Singular B: three semisimple infinite eigenvalues (beta ~ 0)."""
    eigdc, h, torch = E
    n = 110
    A, B, finite, n_inf = workloads.pencil_with_infinite(n, 3, seed=1,
                                                         offdiag_scale=0.1 / np.sqrt(n))
    rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(
        h, A, B, eigdc.default_params(seed=2, leaf_size=40))
    assert rc == eigdc.EIG_OK
    _check_form(A, B, S, T, QL, QR, ar, ai, be)
    inf = np.abs(be) <= 1e-12 * np.linalg.norm(B)
    assert np.sum(inf) == n_inf
    assert np.allclose(np.sort(ar[~inf] / be[~inf]), finite, atol=1e-10)


@pytest.mark.parametrize("eig_scale", [0.15, 6.0, 0.05])
def test_pencil_circle_search_matches_oracle(E, eig_scale):
    """Spectra entirely inside |z| = 1/2 or outside |z| = 1: the root's circle
    search (Sec. 3.5) takes the same radii, splits and failed attempts as the
    oracle."""
    eigdc, h, torch = E
    n = 120
    A, B, d = workloads.regular_pencil(n, seed=3, offdiag_scale=0.1 / np.sqrt(n),
                                       eig_scale=eig_scale)
    rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(
        h, A, B, eigdc.default_params(seed=1, leaf_size=40))
    assert rc == eigdc.EIG_OK
    _check_form(A, B, S, T, QL, QR, ar, ai, be)
    So, To, QLo, QRo, aro, aio, beo, io = opencil(A, B, seed=1, leaf_size=40)
    assert io.status == 0
    assert info.splits == io.splits and info.nodes == io.nodes
    assert info.failed_attempts == io.failed_attempts >= 1
    lam = np.sort(ar / be)
    assert np.allclose(lam, np.sort(d), rtol=1e-10, atol=1e-10 * np.max(np.abs(d)))


def test_pencil_identity_B_matches_standard(E):
    eigdc, h, torch = E
    n = 90
    A, d, _ = workloads.nonsymmetric_schur(n, seed=6, offdiag_scale=0.1 / np.sqrt(n))
    rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(
        h, A, np.eye(n), eigdc.default_params(seed=1, leaf_size=40))
    assert rc == eigdc.EIG_OK
    assert np.allclose(np.sort(ar / be), np.sort(d), atol=1e-10)


def test_pencil_schedule_independent(E):
    """1 worker and 8 workers give bit-identical factors."""
    eigdc, h, torch = E
    n = 180
    A, B, d = workloads.regular_pencil(n, seed=4, offdiag_scale=0.1 / np.sqrt(n))
    r1 = eigdc.pencil_schur(h, A, B, eigdc.default_params(seed=5, leaf_size=32, workers=1))
    r8 = eigdc.pencil_schur(h, A, B, eigdc.default_params(seed=5, leaf_size=32, workers=8))
    assert r1[0] == r8[0] == eigdc.EIG_OK
    for a, b in zip(r1[1:8], r8[1:8]):
        assert np.array_equal(a, b)


def test_pencil_small_and_leaf_only(E):
    """n <= leaf_size: no split, a single leaf (n = 1 included)."""
    eigdc, h, torch = E
    for n in (1, 2, 7, 64):
        A, B, d = workloads.regular_pencil(n, seed=n, offdiag_scale=0.1)
        rc, S, T, QL, QR, ar, ai, be, info = eigdc.pencil_schur(h, A, B, eigdc.default_params())
        assert rc == eigdc.EIG_OK and info.splits == 0 and info.leaves == 1
        _check_form(A, B, S, T, QL, QR, ar, ai, be)
        assert np.allclose(np.sort(ar / be), np.sort(d), atol=1e-10)


def test_pencil_argument_errors(E):
    eigdc, h, torch = E
    n = 8
    A, B, d = workloads.regular_pencil(n, seed=1)
    dA, dB = eigdc.to_device(A), eigdc.to_device(B)
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    p = eigdc.default_params(prec=eigdc.EIG_SPLIT_BF16X3)
    rc, _ = eigdc.eig_pencil_schur(h, n, dA, n, dB, n, z(n, n), n, z(n, n), n, z(n), z(n), z(n), p)
    assert rc == eigdc.EIG_ERR_ARG
    rc, _ = eigdc.eig_pencil_schur(h, n, dA, n - 1, dB, n, z(n, n), n, z(n, n), n, z(n), z(n),
                                   z(n), eigdc.default_params())
    assert rc == eigdc.EIG_ERR_ARG
    B2 = B.copy()
    B2[0, 0] = np.nan
    rc, *_ = eigdc.pencil_schur(h, A, B2)
    assert rc == eigdc.EIG_NONFINITE
