"""Seeded synthetic inputs for the eigensolver (tests, bench, smoke).

This module holds no arithmetic of the method itself: it only builds test
matrices with prescribed spectra.  It uses numpy's own generator and a library
QR to draw random orthogonal similarity matrices.  Both the CUDA path and the
CPU oracle receive the same arrays from here.

Workloads (sizes are parameters; the defaults follow the stated configurations):
  * symmetric_split(n=256): A = Q diag(lam) Q^T, half of lam uniform in
    [-1, -0.05], half in [0.05, 1], randomly permuted; one split at 0.
  * nonsymmetric_schur(n=2048): A = Q T Q^T, T upper triangular, diagonal half
    |z| ~ U[0.2, 0.9], half |z| ~ U[1.1, 3] with random sign (positions
    permuted), strict upper part N(0, 1/n).
  * symmetric_semicircle(n=8192): lam from the Wigner semicircle on [-1, 1]
    (x = sqrt(u1) cos(2 pi u2)), Q Haar.
  * batched_symmetric(count=2000): n log-uniform in [32, 512], lam ~ U[-1, 1].
  * regular_pencil(n): B = I + 0.1 G / sqrt(n), A = (Q T Q^T) B.
  * svd_matrix(m, n): A = U diag(s) V^T, s ~ U[0.05, 1], U and V random
    orthonormal.
  * pencil_with_infinite(n, n_inf): A = Q1 S Q2^T, B = Q1 T Q2^T with S, T
    upper triangular; n_inf diagonal pairs (s, t) = (1, 0) with those rows of
    T zero (a semisimple infinite eigenvalue, singular B), the others (d_i, 1)
    with d_i as in nonsymmetric_triangular.
  * normal_complex(n): real normal matrix with conjugate pairs a +- ib,
    a, b ~ U[-1.5, 1.5] (the random normal examples of Sec. 3.3.1).
  * near_axis(n=25): real parts +-1e-10, imaginary parts U[-1.5, 1.5].
  * jordan_hard(n=32): half the eigenvalues with negative real part, half a
    single Jordan block at 0.1.
"""
import numpy as np

MASTER_SEED = 0xE16D0000


def rng_for(config_id, extra=0):
    return np.random.default_rng([MASTER_SEED + config_id, extra])


def random_orthogonal(n, rng):
    """Haar orthogonal matrix from a library QR of a Gaussian draw, sign-fixed."""
    if n == 0:
        return np.zeros((0, 0))
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def _sym_from_spectrum(lam, rng):
    Q = random_orthogonal(len(lam), rng)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


def symmetric_split(n=256, seed=1):
    rng = rng_for(1, seed)
    h = n // 2
    lam = np.concatenate([rng.uniform(-1.0, -0.05, h), rng.uniform(0.05, 1.0, n - h)])
    rng.shuffle(lam)
    return _sym_from_spectrum(lam, rng), np.sort(lam)


def symmetric_uniform(n, seed=0, lo=-1.0, hi=1.0):
    rng = rng_for(4, seed)
    lam = rng.uniform(lo, hi, n)
    return _sym_from_spectrum(lam, rng), np.sort(lam)


def symmetric_semicircle(n=8192, seed=3):
    rng = rng_for(3, seed)
    u1 = rng.uniform(0.0, 1.0, n)
    u2 = rng.uniform(0.0, 1.0, n)
    lam = np.sqrt(u1) * np.cos(2.0 * np.pi * u2)
    return _sym_from_spectrum(lam, rng), np.sort(lam)


def nonsymmetric_triangular(n, rng, offdiag_scale=None):
    h = n // 2
    mags = np.concatenate([rng.uniform(0.2, 0.9, h), rng.uniform(1.1, 3.0, n - h)])
    signs = rng.choice(np.array([-1.0, 1.0]), n)
    d = mags * signs
    rng.shuffle(d)
    scale = (1.0 / np.sqrt(n)) if offdiag_scale is None else offdiag_scale
    T = np.triu(rng.standard_normal((n, n)) * scale, 1) + np.diag(d)
    return T, d


def nonsymmetric_schur(n=2048, seed=2, offdiag_scale=None):
    rng = rng_for(2, seed)
    T, d = nonsymmetric_triangular(n, rng, offdiag_scale)
    Q = random_orthogonal(n, rng)
    return Q @ T @ Q.T, d, T


def batched_symmetric(count=2000, seed=4, nmin=32, nmax=512):
    rng = rng_for(4, seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))).astype(int)
    mats, spectra = [], []
    for n in sizes:
        lam = rng.uniform(-1.0, 1.0, n)
        mats.append(_sym_from_spectrum(lam, rng))
        spectra.append(np.sort(lam))
    return mats, spectra


def regular_pencil(n, seed=5, offdiag_scale=None, eig_scale=1.0):
    """(A, B, eigenvalues) with A = (Q T Q^T) B; eig_scale multiplies T (its
    spectrum and its coupling, so relative conditioning is unchanged), e.g.
    0.15: every eigenvalue inside |z| < 1/2; 6: every one outside |z| = 1."""
    rng = rng_for(5, seed)
    T, d = nonsymmetric_triangular(n, rng, offdiag_scale)
    if eig_scale != 1.0:
        T = T * eig_scale
        d = d * eig_scale
    Q = random_orthogonal(n, rng)
    M = Q @ T @ Q.T
    B = np.eye(n) + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n)
    return M @ B, B, d


def svd_matrix(m, n, seed=10, lo=0.05, hi=1.0):
    """(A, singular values descending): A = U diag(s) V^T with U, V random
    orthonormal (m x r, n x r), r = min(m, n), s ~ U[lo, hi]."""
    rng = rng_for(10, seed)
    r = min(m, n)
    s = np.sort(rng.uniform(lo, hi, r))[::-1]
    U = random_orthogonal(m, rng)[:, :r]
    V = random_orthogonal(n, rng)[:, :r]
    return (U * s) @ V.T, s


def pencil_with_infinite(n, n_inf=2, seed=9, offdiag_scale=None):
    """(A, B, finite eigenvalues sorted, n_inf) of a regular pencil whose B is
    singular: det(A - z B) = prod (s_ii - z t_ii) with t_ii = 0 at n_inf
    positions."""
    rng = rng_for(9, seed)
    S, d = nonsymmetric_triangular(n, rng, offdiag_scale)
    scale = (1.0 / np.sqrt(n)) if offdiag_scale is None else offdiag_scale
    T = np.triu(rng.standard_normal((n, n)) * scale, 1) + np.eye(n)
    idx = rng.choice(n, n_inf, replace=False)
    S[idx, idx] = 1.0
    T[idx, :] = 0.0       # rank(T) = n - n_inf: the infinite eigenvalue is semisimple
    finite = np.sort(np.delete(d, idx))
    Q1 = random_orthogonal(n, rng)
    Q2 = random_orthogonal(n, rng)
    return Q1 @ S @ Q2.T, Q1 @ T @ Q2.T, finite, n_inf


def _real_normal_from_pairs(re, im, real_eigs, rng):
    blocks = []
    for a, b in zip(re, im):
        blocks.append(np.array([[a, b], [-b, a]]))
    n = 2 * len(re) + len(real_eigs)
    D = np.zeros((n, n))
    i = 0
    for blk in blocks:
        D[i:i + 2, i:i + 2] = blk
        i += 2
    for x in real_eigs:
        D[i, i] = x
        i += 1
    Q = random_orthogonal(n, rng)
    return Q @ D @ Q.T


def normal_complex(n, seed=6):
    rng = rng_for(6, seed)
    npair = n // 2
    re = rng.uniform(-1.5, 1.5, npair)
    im = rng.uniform(-1.5, 1.5, npair)
    real_eigs = rng.uniform(-1.5, 1.5, n - 2 * npair)
    A = _real_normal_from_pairs(re, im, real_eigs, rng)
    dist = float(np.min(np.abs(np.concatenate([re, real_eigs]))))
    return A, dist


def near_axis(n=25, seed=7):
    rng = rng_for(7, seed)
    npair = n // 2
    re = rng.choice(np.array([-1e-10, 1e-10]), npair)
    im = rng.uniform(-1.5, 1.5, npair)
    real_eigs = rng.choice(np.array([-1e-10, 1e-10]), n - 2 * npair)
    return _real_normal_from_pairs(re, im, real_eigs, rng)


def jordan_hard(n=32, seed=8):
    rng = rng_for(8, seed)
    h = n // 2
    D = np.zeros((n, n))
    neg = -rng.uniform(0.05, 1.5, h)
    D[:h, :h] = np.diag(neg)
    J = 0.1 * np.eye(n - h) + np.diag(np.ones(n - h - 1), 1)
    D[h:, h:] = J
    Q = random_orthogonal(n, rng)
    return Q @ D @ Q.T
