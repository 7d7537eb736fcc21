"""Serving (GPU): continuous batching under an HBM budget, and every result
identical alone and in the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    import torch
    from paper_1011_3077_gb300 import build, eigdc, serving
    build.build()
    rng = np.random.default_rng(3)
    kinds = [(eigdc.EIG_KIND_SYM, eigdc.EIG_KIND_NONSYM, eigdc.EIG_KIND_PENCIL)[i % 3]
             for i in range(16)]
    sizes = rng.integers(24, 180, size=16)
    inputs = [serving.synthesize(k, int(n), 100 + i) for i, (k, n) in enumerate(zip(kinds, sizes))]
    torch.cuda.synchronize()
    params = eigdc.default_params(seed=9)
    # in the mix: all submitted at once, a budget that admits only a few at a
    # time (three of the largest footprints; eig_workspace_size bounds each)
    import ctypes
    h0 = eigdc.Handle(0)
    need = 0
    for k, n in zip(kinds, sizes):
        b = ctypes.c_size_t()
        assert eigdc.lib().eig_workspace_size(h0.ptr, int(n), int(k), ctypes.byref(b)) == 0
        need = max(need, b.value)
    h0.close()
    budget_gb = 3 * need * 1e-9
    srv = eigdc.Server(0, 6, budget_gb)
    bufs, tickets = [], []
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    for (dA0, dB0, ref), k in zip(inputs, kinds):
        n = dA0.shape[0]
        dA = dA0.clone()
        dwr, dwi, dU = z(n), z(n), z(n, n)
        if k == eigdc.EIG_KIND_PENCIL:
            dB, dQR, dbe = dB0.clone(), z(n, n), z(n)
            torch.cuda.synchronize()
            bufs.append((dA, dwr, dwi, dU, dB, dQR, dbe))
            tickets.append(srv.submit_pencil(dA, dB, dU, dQR, dwr, dwi, dbe, params))
            continue
        torch.cuda.synchronize()
        bufs.append((dA, dwr, dwi, dU))
        tickets.append(srv.submit(k, dA, dwr, dwi, dU, params))
    for t in tickets:
        rc, st = srv.wait(t, 600.0)
        assert rc == 0 and st == 0
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == 16 and stats["pending"] == 0
    assert stats["peak_reserved_gb"] <= budget_gb + 1e-12
    # alone: the same request through eig_solve with one worker
    h = eigdc.Handle(0)
    p1 = eigdc.default_params(seed=9, workers=1)
    for (dA0, dB0, ref), k, got in zip(inputs, kinds, bufs):
        n = dA0.shape[0]
        a = dA0.clone()
        wr, wi, U = z(n), z(n), z(n, n)
        if k == eigdc.EIG_KIND_PENCIL:
            b, QR, be = dB0.clone(), z(n, n), z(n)
            rc, info = eigdc.eig_pencil_schur(h, n, a, n, b, n, U, n, QR, n, wr, wi, be, p1)
            assert rc == 0
            for mine, theirs in zip((a, wr, wi, U, b, QR, be), got):
                assert torch.equal(mine, theirs)
            lam = torch.sort(wr / be).values
        else:
            rc, info = eigdc.eig_solve(h, k, n, a, n, wr, wi, U, n, p1)
            assert rc == 0
            dA, dwr, dwi, dU = got
            assert torch.equal(a, dA) and torch.equal(wr, dwr) and torch.equal(U, dU)
            lam = torch.sort(wr).values
        A_host = dA0.cpu().numpy().T
        B_host = dB0.cpu().numpy().T if k == eigdc.EIG_KIND_PENCIL else None
        tol = 1e-10 * float(torch.max(torch.abs(ref))) * _kappa(k, A_host, B_host)
        assert float(torch.max(torch.abs(lam - ref))) <= tol
    h.close()


def _kappa(kind, A, B=None):
    """Relative condition of the spectrum (1 for symmetric A): the largest
    ||y|| ||x|| (||A|| + |l| ||B||) / (|y^H B x| max|l|) over the eigenvalues l
    of (A, B) (B = I for one matrix), from the library's left and right
    eigenvectors (test side): a backward error eps moves l by at most about
    eps max|l| times it."""
    from paper_1011_3077_gb300 import eigdc
    if kind == eigdc.EIG_KIND_SYM:
        return 1.0
    import scipy.linalg as sla
    Bm = np.eye(A.shape[0]) if B is None else B
    w, VL, VR = sla.eig(A, Bm, left=True, right=True)
    num = np.linalg.norm(VL, axis=0) * np.linalg.norm(VR, axis=0)
    den = np.abs(np.sum(VL.conj() * (Bm @ VR), axis=0))
    scale = (np.linalg.norm(A, 2) + np.abs(w) * np.linalg.norm(Bm, 2)) / np.abs(w).max()
    return float(np.max(num / den * scale))


def test_served_results_match_the_oracle():
    """Requests of every kind served together (n up to 180): each result takes
    the oracle's recursion tree and its eigenvalues agree with the oracle's
    within 1e-10 ||A|| (times the eigenvalue condition number for the
    nonsymmetric and pencil kinds, both sides being backward stable)."""
    import torch
    from paper_1011_3077_gb300 import build, eigdc, serving
    from oracle.solve import eig_sym, schur_nonsym, pencil_schur
    build.build()
    kinds = [eigdc.EIG_KIND_SYM, eigdc.EIG_KIND_NONSYM, eigdc.EIG_KIND_PENCIL] * 3
    sizes = [60, 72, 66, 120, 150, 101, 180, 171, 140]
    inputs = [serving.synthesize(k, n, 500 + i) for i, (k, n) in enumerate(zip(kinds, sizes))]
    torch.cuda.synchronize()
    params = eigdc.default_params(seed=4)
    srv = eigdc.Server(0, 4, 4.0)
    z = lambda *s_: torch.zeros(s_, dtype=torch.float64, device="cuda")
    bufs, tickets = [], []
    for (dA0, dB0, ref), k in zip(inputs, kinds):
        n = dA0.shape[0]
        dA, dwr, dwi, dU = dA0.clone(), z(n), z(n), z(n, n)
        if k == eigdc.EIG_KIND_PENCIL:
            dB, dQR, dbe = dB0.clone(), z(n, n), z(n)
            torch.cuda.synchronize()
            bufs.append((dwr, dbe))
            tickets.append(srv.submit_pencil(dA, dB, dU, dQR, dwr, dwi, dbe, params))
        else:
            torch.cuda.synchronize()
            bufs.append((dwr, None))
            tickets.append(srv.submit(k, dA, dwr, dwi, dU, params))
    infos = []
    for t in tickets:
        rc, st = srv.wait(t, 600.0)
        assert rc == 0 and st == 0
        infos.append(srv.poll(t)[2])
    srv.close()
    for (dA0, dB0, ref), k, (dwr, dbe), info in zip(inputs, kinds, bufs, infos):
        A = dA0.cpu().numpy().T
        if k == eigdc.EIG_KIND_SYM:
            wo, _, io = eig_sym(A, seed=4)
            got, want = dwr.cpu().numpy(), wo
        elif k == eigdc.EIG_KIND_NONSYM:
            To, Qo, wro, wio, io = schur_nonsym(A, seed=4)
            assert np.all(wio == 0.0)
            got, want = np.sort(dwr.cpu().numpy()), np.sort(wro)
        else:
            B = dB0.cpu().numpy().T
            So, To, QLo, QRo, aro, aio, beo, io = pencil_schur(A, B, seed=4)
            got = np.sort((dwr / dbe).cpu().numpy())
            want = np.sort(aro / beo)
        assert io.status == 0
        assert (info.splits, info.nodes, info.failed_attempts) == (io.splits, io.nodes,
                                                                   io.failed_attempts)
        B_host = dB0.cpu().numpy().T if k == eigdc.EIG_KIND_PENCIL else None
        tol = 1e-10 * float(torch.max(torch.abs(ref))) * _kappa(k, A, B_host)
        assert np.max(np.abs(got - want)) <= tol


def test_serving_loop_reports_latency():
    from paper_1011_3077_gb300 import build, eigdc, serving
    build.build()
    out = serving.run(rate=400.0, count=12, nmin=32, nmax=256, workers=4, budget_gb=8.0, seed=2)
    assert out["ok"] == 12 and out["mix"]["pencil"] >= 1
    assert out["latency_s"]["p99"] >= out["latency_s"]["p50"] > 0
    assert out["max_eigenvalue_error"] <= 1e-9      # pencils: kappa-limited, up to ~1e-10 here
    assert out["max_backward_error"] <= 1e-12
