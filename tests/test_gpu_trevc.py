"""GPU parity of the eigenvectors from the Schur form (eig_eigenvectors).

The real Schur form comes from the GPU solver (eig_solve, nonsymmetric); the
oracle (oracle/trevc.py) takes the same (T, Q, wi).  Eigenvalues agree to
1e-13 |A|, each eigenvector agrees with the oracle's up to a unit scalar to
1e-10 kappa (the recurrence divides by eigenvalue differences), and
||A V - V diag(lam)||_F <= 1e-12 ||A||_F ||V||_F.
"""
import numpy as np
import pytest

from oracle import trevc as otrevc
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


@pytest.mark.parametrize("case", ["normal50", "normal97", "triangular200", "single"])
def test_eigenvectors_match_oracle(E, case):
    eigdc, h, torch = E
    if case == "normal50":
        A = workloads.normal_complex(50, seed=2)[0]
    elif case == "normal97":
        A = workloads.normal_complex(97, seed=4)[0]
    elif case == "triangular200":
        A = workloads.nonsymmetric_schur(200, seed=3, offdiag_scale=0.1 / np.sqrt(200))[0]
    else:
        A = np.array([[3.0]])
    n = A.shape[0]
    rc, T, Q, wr, wi, info = eigdc.schur_nonsymmetric(h, A, eigdc.default_params(seed=1, leaf_size=32))
    assert rc == eigdc.EIG_OK
    rc, lam, V = eigdc.eigenvectors(h, T, Q, wi)
    assert rc == eigdc.EIG_OK
    lo, Vo = otrevc.eigenvectors(T, Q, wi)
    assert np.abs(lam - lo).max() <= 1e-13 * max(1.0, np.abs(A).max())
    ph = np.sum(V.conj() * Vo, axis=0)
    ph = ph / np.abs(ph)
    assert np.abs(V * ph - Vo).max() <= 1e-10
    assert np.abs(np.linalg.norm(V, axis=0) - 1.0).max() <= 1e-14
    assert np.linalg.norm(A @ V - V * lam) <= 1e-12 * np.linalg.norm(A) * np.sqrt(n)


def test_argument_errors(E):
    eigdc, h, torch = E
    d = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    z = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    rc = eigdc.eig_eigenvectors(h, 4, d, 3, d, 4, d, z, 4, z)
    assert rc == eigdc.EIG_ERR_ARG


def test_eigenvectors_of_a_complex_schur_form(E):
    """eig_eigenvectors_complex on eig_schur_complex's output against the
    oracle's triangular recurrence on the same (T, U)."""
    eigdc, h, torch = E
    rng = np.random.default_rng(77)
    n = 90
    lam0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    S = np.eye(n) + 0.25 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    A = S @ np.diag(lam0) @ np.linalg.inv(S)
    rc, T, U, w, info, _ = eigdc.schur_complex(h, A, eigdc.default_params(seed=2, leaf_size=16))
    assert rc == eigdc.EIG_OK
    rc, lam, V = eigdc.eigenvectors_complex(h, T, U)
    assert rc == eigdc.EIG_OK
    X = otrevc.triangular_eigenvectors(T)
    Vo = U @ X
    Vo = Vo / np.linalg.norm(Vo, axis=0)
    assert np.abs(lam - np.diag(T)).max() == 0.0
    ph = np.sum(V.conj() * Vo, axis=0)
    ph = ph / np.abs(ph)
    assert np.abs(V * ph - Vo).max() <= 1e-10
    assert np.linalg.norm(A @ V - V * lam) <= 1e-12 * np.linalg.norm(A) * np.sqrt(n)
