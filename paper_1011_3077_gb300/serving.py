"""Serving loop: Poisson arrivals of mixed eigenproblems on one GPU.

Requests (symmetric eigendecomposition, nonsymmetric real Schur form,
generalized real Schur form of a regular pencil, and with a fourth --mix share
the complex Schur form by lines at random angles) of log-uniform size arrive
as a Poisson stream and are submitted to the native request server
(include/eigdc.h, eig_server_*), which admits them under an HBM budget as
workers free up and overlaps their work on the device.  The loop reports
throughput and p50/p99 latency (arrival to completion).

Inputs are synthesised on the device before the clock starts (random
orthogonal similarity of a prescribed spectrum; a library QR draws the
orthogonal factor -- input generation, not the method).  Nonsymmetric
requests use the triangular construction with strict-upper scale 0.1/sqrt(n)
(the reduced-coupling reading of the nonsymmetric workload); pencils are
A = (Q T Q^T) B with that T and B = I + 0.1 G / sqrt(n).  By default every
request runs in EIG_FP64_TC (FP64 in and out, the large products on the
tensor cores through the error-free split); symmetric requests can take a
split-precision form instead (prec_sym: EIG_SPLIT_FP32 or EIG_SPLIT_BF16X3,
FP32-level products refined to FP64 at the end); nonsymmetric, pencil and
complex-plane requests run in EIG_FP64_TC or EIG_FP64.

Usage: python -m paper_1011_3077_gb300.serving --rate 200 --count 40
"""
import argparse
import json
import math
import time

import numpy as np

from . import eigdc


def _orthogonal(n, gen, device):
    """Haar orthogonal factor (sign-fixed QR of a Gaussian; the QR runs on the
    host, which keeps input generation off the device's linear-algebra
    library)."""
    import torch
    G = torch.randn((n, n), generator=gen, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(G.cpu())
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    return (Q * s).to(device)


def synthesize_complex(n, seed, device="cuda"):
    """Complex-plane request: A = Q T Q^H with Q unitary (library QR of a complex
    Gaussian) and T upper triangular, diagonal uniform in the disk of radius
    1.5, strict upper part N(0, (0.1/sqrt(n))^2); returns (dA column-major
    complex128, the prescribed eigenvalues)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    G = torch.complex(torch.randn((n, n), generator=gen, dtype=torch.float64, device=device),
                      torch.randn((n, n), generator=gen, dtype=torch.float64, device=device))
    Q, R = torch.linalg.qr(G.cpu())
    ph = torch.diagonal(R) / torch.abs(torch.diagonal(R))
    Q = (Q * ph).to(device)
    rad = 1.5 * torch.sqrt(torch.rand(n, generator=gen, dtype=torch.float64, device=device))
    ang = 2.0 * math.pi * torch.rand(n, generator=gen, dtype=torch.float64, device=device)
    d = torch.polar(rad, ang)
    N = torch.complex(torch.randn((n, n), generator=gen, dtype=torch.float64, device=device),
                      torch.randn((n, n), generator=gen, dtype=torch.float64, device=device))
    T = torch.triu(N * (0.1 / math.sqrt(2.0 * n)), 1) + torch.diag(d)
    A = Q @ T @ Q.conj().T
    return A.T.contiguous(), d


def synthesize(kind, n, seed, device="cuda"):
    """(dA column-major, dB column-major or None, reference spectrum) for one request."""
    import torch
    if kind == eigdc.EIG_KIND_CPLANE:
        dA, d = synthesize_complex(n, seed, device)
        return dA, None, d
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    Q = _orthogonal(n, gen, device)
    dB = None
    if kind == eigdc.EIG_KIND_SYM:
        lam = torch.rand(n, generator=gen, dtype=torch.float64, device=device) * 2.0 - 1.0
        A = (Q * lam) @ Q.T
        A = 0.5 * (A + A.T)
        ref = torch.sort(lam).values
    else:
        h = n // 2
        mags = torch.cat([0.2 + 0.7 * torch.rand(h, generator=gen, dtype=torch.float64, device=device),
                          1.1 + 1.9 * torch.rand(n - h, generator=gen, dtype=torch.float64, device=device)])
        sgn = torch.where(torch.rand(n, generator=gen, device=device) < 0.5, -1.0, 1.0).to(torch.float64)
        d = (mags * sgn)[torch.randperm(n, generator=gen, device=device)]
        T = torch.triu(torch.randn((n, n), generator=gen, dtype=torch.float64, device=device)
                       * (0.1 / math.sqrt(n)), 1) + torch.diag(d)
        A = Q @ T @ Q.T
        ref = torch.sort(d).values
        if kind == eigdc.EIG_KIND_PENCIL:
            G = torch.randn((n, n), generator=gen, dtype=torch.float64, device=device)
            B = torch.eye(n, dtype=torch.float64, device=device) + G * (0.1 / math.sqrt(n))
            A = A @ B
            dB = B.T.contiguous()
    # column-major storage of A is the row-major storage of A^T
    return A.T.contiguous(), dB, ref


def backward_error(kind, dA, o):
    """||A - U L U^T||_F / ||A||_F (symmetric), ||A - U T U^T|| / ||A||
    (Schur), max over A and B of ||X - Q_L X^ Q_R^T|| / ||X|| (pencil).
    Tensors hold column-major matrices, i.e. the row-major transposes."""
    import torch
    A0 = o["A0"]
    if kind == eigdc.EIG_KIND_CPLANE:
        Ut, Tt = o["dU"], o["dT"]   # transposes of U and T
        rec = (Ut.T @ Tt.T @ Ut.T.conj().T).T
        return float(torch.linalg.norm(A0 - rec) / torch.linalg.norm(A0))
    if kind == eigdc.EIG_KIND_SYM:
        Ut = o["dU"]
        rec = Ut.T @ torch.diag(o["dwr"]) @ Ut
        return float(torch.linalg.norm(A0 - rec) / torch.linalg.norm(A0))
    if kind == eigdc.EIG_KIND_NONSYM:
        Ut = o["dU"]
        return float(torch.linalg.norm(A0 - Ut.T @ dA @ Ut) / torch.linalg.norm(A0))
    QLt, QRt = o["dU"], o["dQR"]
    rA = torch.linalg.norm(A0 - QRt.T @ dA @ QLt) / torch.linalg.norm(A0)
    rB = torch.linalg.norm(o["B0"] - QRt.T @ o["dB"] @ QLt) / torch.linalg.norm(o["B0"])
    return float(max(rA, rB))


def trace(count, rate=200.0, nmin=64, nmax=4096, mix=(0.5, 0.3, 0.2), seed=5):
    """(arrival times in s, kinds, sizes) of a seeded Poisson stream: exponential
    gaps of mean 1/rate, kinds drawn with the shares `mix` (symmetric,
    nonsymmetric, pencil and an optional fourth complex-plane share), sizes
    log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    arrivals = np.cumsum(gaps) - gaps[0]
    kinds = rng.choice([eigdc.EIG_KIND_SYM, eigdc.EIG_KIND_NONSYM, eigdc.EIG_KIND_PENCIL,
                        eigdc.EIG_KIND_CPLANE][:len(mix)],
                       size=count, p=np.asarray(mix) / np.sum(mix))
    sizes = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))).astype(int)
    return arrivals, kinds, sizes


def run(rate=200.0, count=40, nmin=64, nmax=4096, mix=(0.5, 0.3, 0.2), workers=8,
        budget_gb=120.0, prec=eigdc.EIG_FP64_TC, seed=5, device="cuda", verbose=False,
        details=False, prec_sym=None, host_io=False, sym_split_max_n=1024, fused_tail=0):
    """Serve one seeded trace; returns throughput, latency percentiles and the
    accuracy of every result.

    prec: arithmetic of the nonsymmetric, pencil and complex-plane requests
    (EIG_FP64 or EIG_FP64_TC); prec_sym: that of the symmetric requests of
    order up to sym_split_max_n (default prec; the split-precision forms apply
    to them: above about n = 1000 the FP32-level iterates no longer separate
    the closest eigenvalues at the median shift, so larger symmetric requests
    run in `prec`).  host_io: the
    inputs start in pinned host memory; each request's input is copied to the
    device when it arrives and its outputs are read back when it completes,
    both inside the timed region (the end-to-end form); the byte counts are
    returned.  fused_tail: the symmetric requests' nodes of at most this many
    rows finish in one launch of the fused batched solver (eig_params_t).
    The makespan is the CUDA-event time from the first arrival to
    the last completion, with the device synchronised on both sides."""
    import torch
    arrivals, kinds, sizes = trace(count, rate, nmin, nmax, mix, seed)
    reqs = []
    for i in range(count):
        n = int(sizes[i])
        kind = int(kinds[i])
        dA, dB, ref = synthesize(kind, n, seed * 1000003 + i, device)
        z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=device)
        zc = lambda *shape: torch.zeros(shape, dtype=torch.complex128, device=device)
        if kind == eigdc.EIG_KIND_CPLANE:
            out = dict(dw=zc(n), dU=zc(n, n), dT=zc(n, n), A0=dA.clone())
        else:
            out = dict(dwr=z(n), dwi=z(n), dU=z(n, n), A0=dA.clone())
            if kind == eigdc.EIG_KIND_PENCIL:
                out.update(dB=dB, dQR=z(n, n), dbe=z(n), B0=dB.clone())
        if host_io:
            out["hA"] = dA.cpu().pin_memory()
            if kind == eigdc.EIG_KIND_PENCIL:
                out["hB"] = dB.cpu().pin_memory()
            # pinned host destinations of the outputs
            out["host_out"] = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory()
                               for k, v in out.items()
                               if k in ("dw", "dU", "dT", "dwr", "dwi", "dQR", "dbe") or
                               (k == "dB" and kind == eigdc.EIG_KIND_PENCIL)}
            dA.zero_()
            if kind == eigdc.EIG_KIND_PENCIL:
                dB.zero_()
        reqs.append((kind, n, dA, out, ref))
    torch.cuda.synchronize()
    srv = eigdc.Server(0, workers, budget_gb)
    # fused_tail applies to the symmetric requests only (their small nodes
    # finish in one launch of the fused batched solver)
    params = eigdc.default_params(seed=seed, prec=prec, fused_tail=fused_tail)
    params_sym = eigdc.default_params(seed=seed, prec=prec if prec_sym is None else prec_sym,
                                      fused_tail=fused_tail)
    copy_stream = torch.cuda.Stream(device=device)
    h2d = d2h = 0
    tickets = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    t0 = time.perf_counter()
    for i, (kind, n, dA, o, ref) in enumerate(reqs):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if host_io:
            with torch.cuda.stream(copy_stream):
                dA.copy_(o["hA"], non_blocking=True)
                h2d += o["hA"].numel() * o["hA"].element_size()
                if kind == eigdc.EIG_KIND_PENCIL:
                    o["dB"].copy_(o["hB"], non_blocking=True)
                    h2d += o["hB"].numel() * o["hB"].element_size()
            copy_stream.synchronize()
        if kind == eigdc.EIG_KIND_PENCIL:
            tickets.append(srv.submit_pencil(dA, o["dB"], o["dU"], o["dQR"], o["dwr"], o["dwi"],
                                             o["dbe"], params))
        elif kind == eigdc.EIG_KIND_CPLANE:
            tickets.append(srv.submit_complex(dA, o["dT"], o["dU"], o["dw"], params))
        elif kind == eigdc.EIG_KIND_SYM:
            tickets.append(srv.submit(kind, dA, o["dwr"], o["dwi"], o["dU"],
                                      params_sym if n <= sym_split_max_n else params))
        else:
            tickets.append(srv.submit(kind, dA, o["dwr"], o["dwi"], o["dU"], params))
    statuses, lat, wait, service, flops, trees = [], [], [], [], 0.0, []
    for t, (kind, n, dA, o, ref) in zip(tickets, reqs):
        srv.wait(t, 3600.0)
        st, times, info = srv.poll(t)
        statuses.append(st)
        trees.append({"splits": info.splits, "nodes": info.nodes,
                      "failed_attempts": info.failed_attempts, "squarings": info.total_iters})
        wait.append(times[0])
        service.append(times[1])
        lat.append(times[2])
        flops += info.flops
        if host_io:
            with torch.cuda.stream(copy_stream):
                for k, hbuf in o["host_out"].items():
                    hbuf.copy_(o[k], non_blocking=True)
                    d2h += hbuf.numel() * hbuf.element_size()
                if kind in (eigdc.EIG_KIND_NONSYM, eigdc.EIG_KIND_PENCIL):
                    # the Schur / generalized Schur form is returned in dA
                    o.setdefault("host_T", torch.empty(dA.shape, dtype=dA.dtype).pin_memory())
                    o["host_T"].copy_(dA, non_blocking=True)
                    d2h += dA.numel() * dA.element_size()
            copy_stream.synchronize()
    torch.cuda.synchronize()
    e1.record()
    e1.synchronize()
    makespan = e0.elapsed_time(e1) / 1e3
    stats = srv.stats()
    srv.close()
    errs, bwds, records = [], [], []
    by_kind = {}
    for i, ((kind, n, dA, o, ref), st) in enumerate(zip(reqs, statuses)):
        err = bwd = None
        if st == 0 and kind == eigdc.EIG_KIND_CPLANE:
            # distance of each prescribed eigenvalue to the nearest computed one
            err = float(torch.max(torch.min(torch.abs(ref[:, None] - o["dw"][None, :]), dim=1).values))
            bwd = backward_error(kind, dA, o)
        elif st == 0:
            w = o["dwr"] / o["dbe"] if kind == eigdc.EIG_KIND_PENCIL else o["dwr"]
            err = float(torch.max(torch.abs(torch.sort(w).values - ref)))
            bwd = backward_error(kind, dA, o)
        if err is not None:
            errs.append(err)
            bwds.append(bwd)
            k = by_kind.setdefault(int(kind), {"count": 0, "max_eig_err": 0.0, "max_bwd": 0.0})
            k["count"] += 1
            k["max_eig_err"] = max(k["max_eig_err"], err)
            k["max_bwd"] = max(k["max_bwd"], bwd)
        rec = {"kind": kind, "n": n, "status": st, "wait_s": wait[i],
               "service_s": service[i], "latency_s": lat[i], "eig_err": err,
               "backward_err": bwd}
        rec.update(trees[i])
        records.append(rec)
    names = {eigdc.EIG_KIND_SYM: "sym", eigdc.EIG_KIND_NONSYM: "nonsym",
             eigdc.EIG_KIND_PENCIL: "pencil", eigdc.EIG_KIND_CPLANE: "complex_plane"}
    pnames = {eigdc.EIG_FP64: "fp64", eigdc.EIG_SPLIT_BF16X3: "bf16x3 split",
              eigdc.EIG_FP64_TC: "fp64 (tensor-core error-free split)",
              eigdc.EIG_SPLIT_FP32: "fp32-level split (unbiased four-digit tensor-core products, "
                                    "FP64 refinement)"}
    ok = sum(1 for s_ in statuses if s_ == 0)
    out = {
        "requests": count, "ok": ok, "offered_rate_per_s": rate,
        "solves_per_s": ok / makespan, "makespan_s": makespan, "flops": flops,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "service_s": {"p50": float(np.percentile(service, 50)), "p99": float(np.percentile(service, 99))},
        "sizes": {"min": int(sizes.min()), "max": int(sizes.max())},
        "max_backward_error": max(bwds) if bwds else None,
        "max_eigenvalue_error": max(errs) if errs else None,
        "by_kind": {names[k]: v for k, v in by_kind.items()},
        "peak_reserved_gb": stats["peak_reserved_gb"], "budget_gb": budget_gb,
        "workers": workers,
        "precision": pnames[prec],
        "precision_sym": pnames[prec if prec_sym is None else prec_sym],
        "mix": {"sym": int(np.sum(kinds == eigdc.EIG_KIND_SYM)),
                "nonsym": int(np.sum(kinds == eigdc.EIG_KIND_NONSYM)),
                "pencil": int(np.sum(kinds == eigdc.EIG_KIND_PENCIL)),
                "complex_plane": int(np.sum(kinds == eigdc.EIG_KIND_CPLANE))},
    }
    if host_io:
        out["h2d_bytes"] = h2d
        out["d2h_bytes"] = d2h
    if verbose:
        print(json.dumps(out))
    if details:
        out["requests_detail"] = records
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--count", type=int, default=40)
    ap.add_argument("--nmin", type=int, default=64)
    ap.add_argument("--nmax", type=int, default=4096)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--prec", type=int, default=2)
    ap.add_argument("--prec-sym", type=int, default=None)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--mix", default="0.5,0.3,0.2",
                    help="shares of symmetric, nonsymmetric, pencil and (optional fourth) "
                         "complex-plane requests")
    a = ap.parse_args()
    from . import build
    build.build()
    mix = tuple(float(x) for x in a.mix.split(","))
    run(a.rate, a.count, a.nmin, a.nmax, mix=mix, workers=a.workers, budget_gb=a.budget_gb,
        prec=a.prec, seed=a.seed, verbose=True, prec_sym=a.prec_sym)


if __name__ == "__main__":
    main()
