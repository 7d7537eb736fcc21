"""Host-side pieces of the serving loop on the CPU (torch CPU tensors).

The complex-plane request construction must have its prescribed spectrum, and
the backward-error formula (column-major tensors hold the transposes) must
return rounding-level values for an exact Schur form and a large value for a
wrong one.
"""
import numpy as np
import pytest


def test_complex_request_construction_and_backward_error():
    torch = pytest.importorskip("torch")
    from paper_1011_3077_gb300 import eigdc, serving
    n = 40
    dA, d = serving.synthesize_complex(n, seed=7, device="cpu")
    A = dA.numpy().T                        # column-major storage holds A^T
    lam = np.linalg.eigvals(A)
    dd = d.numpy()
    assert max(np.min(np.abs(lam - z)) for z in dd) <= 1e-10
    # an exact complex Schur form of A from the library QR of the
    # eigenvector matrix (test input only)
    Q, _ = np.linalg.qr(np.linalg.eig(A)[1])
    T = Q.conj().T @ A @ Q
    T = np.triu(T)
    o = {"A0": dA.clone(), "dU": torch.from_numpy(np.ascontiguousarray(Q.T)),
         "dT": torch.from_numpy(np.ascontiguousarray(T.T))}
    bwd = serving.backward_error(eigdc.EIG_KIND_CPLANE, dA, o)
    assert bwd <= 1e-12
    o_bad = dict(o, dU=torch.from_numpy(np.ascontiguousarray(Q)))   # transposed by mistake
    assert serving.backward_error(eigdc.EIG_KIND_CPLANE, dA, o_bad) > 1e-3

