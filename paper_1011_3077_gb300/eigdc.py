"""ctypes binding of libeigdc (include/eigdc.h): same entry-point names,
argument marshalling only.

Every numerical step runs in the CUDA library; this module only converts
Python values and torch tensors (device memory, stream) to the C-ABI's plain
pointers and sizes.  If the shared library is missing or cannot be loaded the
import of :func:`lib` raises: there is no CPU fallback.

Matrices cross the boundary column-major.  :func:`to_device` stores a numpy
matrix A as the row-major torch tensor A^T (whose memory is A column-major)
and :func:`to_host` undoes it.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeigdc.so")

EIG_OK = 0
EIG_ERR_ARG = -1
EIG_ERR_CUDA = -2
EIG_ERR_NOMEM = -3
EIG_ERR_SCRATCH = -4
EIG_NO_CONVERGENCE = 1
EIG_NO_SPLIT = 2
EIG_NEAR_SINGULAR_PENCIL = 3
EIG_NONFINITE = 4
EIG_TIMEOUT = 5
EIG_CANCELLED = 6

EIG_REGION_UNIT_CIRCLE = 0
EIG_REGION_CIRCLE = 1
EIG_REGION_LINE = 2
EIG_FP64 = 0
EIG_SPLIT_BF16X3 = 1
EIG_FP64_TC = 2
EIG_SPLIT_FP32 = 3
EIG_KIND_SYM = 0
EIG_KIND_NONSYM = 1
EIG_KIND_PENCIL = 2
EIG_KIND_CPLANE = 3
PURPOSE_HAAR = 4
PURPOSE_SHIFT = 5
PURPOSE_HAAR_LEFT = 6
PURPOSE_HAAR_IMAG = 7
PURPOSE_LINE = 8
ROOT_NODE = 1
EIG_MAX_HALFPLANES = 8


class Region(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c_or_sigma", ctypes.c_double),
                ("r_or_s", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("maxit", ctypes.c_int),
                ("split_tol", ctypes.c_double), ("leaf_size", ctypes.c_int),
                ("prec", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("max_fail", ctypes.c_int), ("nb", ctypes.c_int),
                ("v_draws", ctypes.c_int), ("root_unit_circle", ctypes.c_int),
                ("workers", ctypes.c_int), ("graphs", ctypes.c_int),
                ("fused_tail", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("last_ratio", ctypes.c_double),
                ("converged", ctypes.c_int), ("k", ctypes.c_int),
                ("split_residual", ctypes.c_double), ("rank", ctypes.c_int),
                ("draw", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nodes", ctypes.c_int), ("splits", ctypes.c_int),
                ("max_depth", ctypes.c_int), ("total_iters", ctypes.c_int),
                ("failed_attempts", ctypes.c_int), ("leaves", ctypes.c_int),
                ("flops", ctypes.c_double)]


class Enclosure(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int), ("size", ctypes.c_int),
                ("c_re", ctypes.c_double), ("c_im", ctypes.c_double), ("R", ctypes.c_double),
                ("nhp", ctypes.c_int),
                ("w_re", ctypes.c_double * EIG_MAX_HALFPLANES),
                ("w_im", ctypes.c_double * EIG_MAX_HALFPLANES),
                ("t", ctypes.c_double * EIG_MAX_HALFPLANES)]

    def region(self):
        """(centre, radius, [(w, t), ...]) with complex centre and normals."""
        hps = [(complex(self.w_re[i], self.w_im[i]), self.t[i]) for i in range(self.nhp)]
        return complex(self.c_re, self.c_im), self.R, hps


class FusedConfig(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U64 = ctypes.c_uint64

_SIGNATURES = {
    "eig_default_params": (None, [ctypes.POINTER(Params)]),
    "eig_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "eig_destroy": (_I, [_P]),
    "eig_last_error": (ctypes.c_char_p, [_P]),
    "eig_kernel_launches": (ctypes.c_ulonglong, []),
    "eig_gemm_timing": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_ulonglong),
                             ctypes.POINTER(_D)]),
    "eig_kernel_timing": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_ulonglong),
                               ctypes.POINTER(_D)]),
    "eig_workspace_size": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "eig_divide_step": (_I, [_P, _I, _P, _I, _P, _I, ctypes.POINTER(Region),
                             ctypes.POINTER(Params), ctypes.POINTER(StepInfo)]),
    "eig_last_R": (_I, [_P, _I, _P, _I]),
    "eig_split": (_I, [_P, _I, _P, _P, _I, _P, _I, _P, _I, _I, _U64, _I,
                       ctypes.POINTER(Params), ctypes.POINTER(StepInfo)]),
    "eig_split_pencil": (_I, [_P, _I, _P, _P, _P, _P, _I, _P, _I, _P, _I, _P, _I, _P, _I,
                              _U64, _I, ctypes.POINTER(Params), ctypes.POINTER(StepInfo)]),
    "eig_pencil_schur": (_I, [_P, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P,
                              ctypes.POINTER(Params), ctypes.POINTER(SolveInfo)]),
    "eig_solve": (_I, [_P, _I, _I, _P, _I, _P, _P, _P, _I, ctypes.POINTER(Params),
                       ctypes.POINTER(SolveInfo)]),
    "eig_svd": (_I, [_P, _I, _I, _P, _I, _P, _P, _I, _P, _I, ctypes.POINTER(Params),
                     ctypes.POINTER(SolveInfo)]),
    "eig_solve_batched": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Params),
                               _P, _P]),
    "eig_solve_batched_fused": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Params),
                                     _P, _P]),
    "eig_fused_autotune": (_I, [_P, _I, _I, _I, _U64, ctypes.POINTER(FusedConfig), _I,
                                ctypes.POINTER(_I), ctypes.POINTER(FusedConfig)]),
    "eig_server_create": (_I, [ctypes.POINTER(_P), _I, _I, _D]),
    "eig_server_submit": (_I, [_P, _I, _I, _P, _I, _P, _P, _P, _I, ctypes.POINTER(Params),
                               ctypes.POINTER(_U64)]),
    "eig_server_submit_pencil": (_I, [_P, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P,
                                      ctypes.POINTER(Params), ctypes.POINTER(_U64)]),
    "eig_server_submit_complex": (_I, [_P, _I, _P, _I, _P, _I, _P, _I, _P, ctypes.POINTER(Params),
                                       _I, ctypes.POINTER(_U64)]),
    "eig_server_poll": (_I, [_P, _U64, ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(_D), ctypes.POINTER(SolveInfo)]),
    "eig_server_wait": (_I, [_P, _U64, _D, ctypes.POINTER(_I)]),
    "eig_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_ulonglong),
                              ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(_D),
                              ctypes.POINTER(_D)]),
    "eig_server_destroy": (_I, [_P]),
    "eig_server_cancel": (_I, [_P, _U64]),
    "eig_debug_fail_allocations": (_I, [_I]),
    "eig_qr": (_I, [_P, _I, _I, _P, _I, _P, _I, _P, _I]),
    "eig_gaussian": (_I, [_P, _I, _I, _U64, _I, _U64, _I, _P, _I]),
    "eig_haar": (_I, [_P, _I, _U64, _I, _U64, _I, _P, _I]),
    "eig_split_test": (_I, [_P, _I, _P, _I, _D, _P, _I, _D, ctypes.POINTER(_I),
                            ctypes.POINTER(_D), _P]),
    "eig_gemm": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P, _I]),
    "eig_gemm_split": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P, _I]),
    "eig_gemm_fp64tc": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P, _I]),
    "eig_gemm_fp32tc": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P, _I]),
    "eig_gemm_noalloc": (_I, [_P, _I, _I, _I, _I, _I, _D, _P, _I, _P, _I, _D, _P, _I]),
    "eig_eigenvectors": (_I, [_P, _I, _P, _I, _P, _I, _P, _P, _I, _P]),
    "eig_eigenvectors_complex": (_I, [_P, _I, _P, _I, _P, _I, _P, _I, _P]),
    "eig_zgemm": (_I, [_P, _I, _I, _I, _I, _I, _D, _D, _P, _I, _P, _I, _D, _D, _P, _I]),
    "eig_zqr": (_I, [_P, _I, _I, _P, _I, _P, _I, _P, _I]),
    "eig_zhaar": (_I, [_P, _I, _U64, _U64, _I, _P, _I]),
    "eig_zline_step": (_I, [_P, _I, _P, _I, _D, _D, _D, _D, _U64, _I, ctypes.POINTER(Params),
                            _P, _I, _P, _I, ctypes.POINTER(StepInfo)]),
    "eig_schur_complex": (_I, [_P, _I, _P, _I, _P, _I, _P, _I, _P, ctypes.POINTER(Params), _I,
                               ctypes.POINTER(Enclosure), _I, ctypes.POINTER(_I),
                               ctypes.POINTER(SolveInfo)]),
    "eig_cplane_enclosing_circle": (_I, [_D, _D, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                         ctypes.POINTER(_D), ctypes.POINTER(_D),
                                         ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "eig_cplane_draw_line": (_I, [_U64, _U64, _I, _D, _D, _D, _I, _D, _D, ctypes.POINTER(_D),
                                  ctypes.POINTER(_D), ctypes.POINTER(_D)]),
}

EXPORTED = tuple(_SIGNATURES)


def lib():
    """The loaded libeigdc (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libeigdc.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class EigError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("eigdc error %d: %s" % (code, msg))
        self.code = code


def default_params(**kw):
    p = Params()
    lib().eig_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Handle:
    """eig_create / eig_destroy around a torch CUDA stream."""

    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self._h = ctypes.c_void_p()
        rc = lib().eig_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(stream.cuda_stream))
        if rc != EIG_OK:
            raise EigError(rc, "eig_create failed")

    @property
    def ptr(self):
        return self._h

    def last_error(self):
        return lib().eig_last_error(self._h).decode()

    def check(self, rc, allow=()):
        if rc != EIG_OK and rc not in allow:
            raise EigError(rc, self.last_error())
        return rc

    def close(self):
        if self._h:
            lib().eig_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- layout

def to_device(A, device="cuda"):
    """numpy (rows x cols) -> torch float64 tensor holding A column-major."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).to(device)


def to_host(t):
    """Inverse of to_device."""
    return t.detach().cpu().numpy().T.copy()


def ld(t):
    """Leading dimension of a to_device() tensor (its row stride)."""
    return int(t.stride(0)) if t.dim() == 2 else int(t.shape[0])


# ----------------------------------------------------------------- entry points

def eig_kernel_launches():
    return int(lib().eig_kernel_launches())


def eig_gemm_timing_start():
    rc = lib().eig_gemm_timing(1, None, None, None)
    if rc != EIG_OK:
        raise EigError(rc, "eig_gemm_timing start failed")


TIMING_FAMILIES = {0: "dgemm_kernel", 1: "tcx_gemm_kernel<9>", 2: "tcx_gemm_kernel<4>/<5>",
                   3: "fused_batched_kernel"}


def eig_kernel_timing(family):
    """(total ms, launches, work) of a timed kernel family of the last timed region."""
    ms, cnt, work = ctypes.c_double(), ctypes.c_ulonglong(), ctypes.c_double()
    rc = lib().eig_kernel_timing(family, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(work))
    if rc != EIG_OK:
        raise EigError(rc, "eig_kernel_timing: unknown family")
    return ms.value, cnt.value, work.value


def eig_gemm_timing_stop():
    """(summed launch ms, launches, summed flops) of the FP64 GEMMs since start."""
    ms, cnt, fl = ctypes.c_double(), ctypes.c_ulonglong(), ctypes.c_double()
    rc = lib().eig_gemm_timing(0, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(fl))
    if rc != EIG_OK:
        raise EigError(rc, "eig_gemm_timing stop failed")
    return ms.value, int(cnt.value), fl.value


def eig_divide_step(h, n, dA, lda, dB, ldb, region, params):
    info = StepInfo()
    rc = lib().eig_divide_step(h.ptr, n, _ptr(dA), lda, _ptr(dB), ldb, ctypes.byref(region),
                               ctypes.byref(params), ctypes.byref(info))
    return rc, info


def eig_last_R(h, n, dR, ldr):
    return h.check(lib().eig_last_R(h.ptr, n, _ptr(dR), ldr))


def eig_split(h, n, dAp, dBp, ldp, dA, lda, dQ, ldq, symmetric, stream, attempt, params):
    info = StepInfo()
    rc = lib().eig_split(h.ptr, n, _ptr(dAp), _ptr(dBp), ldp, _ptr(dA), lda, _ptr(dQ), ldq,
                         int(symmetric), int(stream), int(attempt), ctypes.byref(params),
                         ctypes.byref(info))
    return rc, info


def eig_split_pencil(h, n, dApR, dBpR, dApL, dBpL, ldp, dA, lda, dB, ldb, dQL, ldql, dQR, ldqr,
                     stream, attempt, params):
    info = StepInfo()
    rc = lib().eig_split_pencil(h.ptr, n, _ptr(dApR), _ptr(dBpR), _ptr(dApL), _ptr(dBpL), ldp,
                                _ptr(dA), lda, _ptr(dB), ldb, _ptr(dQL), ldql, _ptr(dQR), ldqr,
                                int(stream), int(attempt), ctypes.byref(params),
                                ctypes.byref(info))
    return rc, info


def eig_pencil_schur(h, n, dA, lda, dB, ldb, dQL, ldql, dQR, ldqr, dar, dai, dbe, params):
    info = SolveInfo()
    rc = lib().eig_pencil_schur(h.ptr, n, _ptr(dA), lda, _ptr(dB), ldb, _ptr(dQL), ldql,
                                _ptr(dQR), ldqr, _ptr(dar), _ptr(dai), _ptr(dbe),
                                ctypes.byref(params), ctypes.byref(info))
    return rc, info


def eig_solve(h, kind, n, dA, lda, dwr, dwi, dU, ldu, params):
    info = SolveInfo()
    rc = lib().eig_solve(h.ptr, kind, n, _ptr(dA), lda, _ptr(dwr), _ptr(dwi), _ptr(dU), ldu,
                         ctypes.byref(params), ctypes.byref(info))
    return rc, info


def eig_solve_batched(h, kind, ns, dAs, ldas, dwrs, dwis, dUs, ldus, params):
    """Host arrays built here from Python lists; returns (rc, status array, infos)."""
    count = len(ns)
    I = ctypes.c_int * max(count, 1)
    Pp = ctypes.c_void_p * max(count, 1)
    n_a = I(*ns)
    lda_a = I(*ldas)
    ldu_a = I(*ldus)
    A_a = Pp(*[t.data_ptr() for t in dAs])
    wr_a = Pp(*[t.data_ptr() for t in dwrs])
    wi_a = Pp(*[t.data_ptr() for t in dwis]) if dwis is not None else None
    U_a = Pp(*[t.data_ptr() for t in dUs])
    st = I()
    infos = (SolveInfo * max(count, 1))()
    rc = lib().eig_solve_batched(h.ptr, kind, count, ctypes.cast(n_a, _P), ctypes.cast(A_a, _P),
                                 ctypes.cast(lda_a, _P), ctypes.cast(wr_a, _P),
                                 ctypes.cast(wi_a, _P) if wi_a is not None else None,
                                 ctypes.cast(U_a, _P), ctypes.cast(ldu_a, _P),
                                 ctypes.byref(params), ctypes.cast(st, _P), ctypes.cast(infos, _P))
    return rc, [st[i] for i in range(count)], [infos[i] for i in range(count)]


def eig_solve_batched_fused(h, ns, dAs, ldas, dws, dUs, ldus, params):
    """One persistent fused launch over symmetric problems (n <= 512); returns
    (rc, status list, infos)."""
    count = len(ns)
    I = ctypes.c_int * max(count, 1)
    Pp = ctypes.c_void_p * max(count, 1)
    n_a, lda_a, ldu_a = I(*ns), I(*ldas), I(*ldus)
    A_a = Pp(*[t.data_ptr() for t in dAs])
    w_a = Pp(*[t.data_ptr() for t in dws])
    U_a = Pp(*[t.data_ptr() for t in dUs])
    st = I()
    infos = (SolveInfo * max(count, 1))()
    rc = lib().eig_solve_batched_fused(h.ptr, count, ctypes.cast(n_a, _P), ctypes.cast(A_a, _P),
                                       ctypes.cast(lda_a, _P), ctypes.cast(w_a, _P),
                                       ctypes.cast(U_a, _P), ctypes.cast(ldu_a, _P),
                                       ctypes.byref(params), ctypes.cast(st, _P),
                                       ctypes.cast(infos, _P))
    return rc, [st[i] for i in range(count)], [infos[i] for i in range(count)]


def eig_fused_autotune(h, samples, nmin, nmax, seed=0):
    """Times the fused solver's launch shapes on a synthetic batch and keeps the
    fastest on the handle; returns (rc, best, [candidates])."""
    cap = 16
    table = (FusedConfig * cap)()
    nt = ctypes.c_int(0)
    best = FusedConfig()
    rc = lib().eig_fused_autotune(h.ptr, samples, nmin, nmax, int(seed), table, cap,
                                  ctypes.byref(nt), ctypes.byref(best))
    cands = [(table[i].nb, table[i].ctas_per_sm, table[i].ms) for i in range(min(nt.value, cap))]
    return rc, (best.nb, best.ctas_per_sm, best.ms), cands


class Server:
    """eig_server_* wrapper: submit device buffers, poll or wait for completion."""

    def __init__(self, device=0, workers=8, hbm_budget_gb=120.0):
        self._s = ctypes.c_void_p()
        rc = lib().eig_server_create(ctypes.byref(self._s), device, workers, hbm_budget_gb)
        if rc != EIG_OK:
            raise EigError(rc, "eig_server_create failed")
        self._keep = {}

    def submit(self, kind, dA, dwr, dwi, dU, params=None):
        n = int(dA.shape[0])
        t = ctypes.c_uint64()
        p = params or default_params()
        rc = lib().eig_server_submit(self._s, kind, n, _ptr(dA), n, _ptr(dwr), _ptr(dwi),
                                     _ptr(dU), n, ctypes.byref(p), ctypes.byref(t))
        if rc != EIG_OK:
            raise EigError(rc, "eig_server_submit failed")
        self._keep[t.value] = (dA, dwr, dwi, dU)     # buffers live until done
        return t.value

    def submit_pencil(self, dA, dB, dQL, dQR, dar, dai, dbe, params=None):
        n = int(dA.shape[0])
        t = ctypes.c_uint64()
        p = params or default_params()
        rc = lib().eig_server_submit_pencil(self._s, n, _ptr(dA), n, _ptr(dB), n, _ptr(dQL), n,
                                            _ptr(dQR), n, _ptr(dar), _ptr(dai), _ptr(dbe),
                                            ctypes.byref(p), ctypes.byref(t))
        if rc != EIG_OK:
            raise EigError(rc, "eig_server_submit_pencil failed")
        self._keep[t.value] = (dA, dB, dQL, dQR, dar, dai, dbe)
        return t.value

    def poll(self, ticket):
        done = ctypes.c_int()
        st = ctypes.c_int()
        times = (ctypes.c_double * 3)()
        info = SolveInfo()
        lib().eig_server_poll(self._s, ticket, ctypes.byref(done), ctypes.byref(st), times,
                              ctypes.byref(info))
        if not done.value:
            return None
        return st.value, (times[0], times[1], times[2]), info

    def wait(self, ticket, timeout_s=600.0):
        st = ctypes.c_int()
        rc = lib().eig_server_wait(self._s, ticket, timeout_s, ctypes.byref(st))
        return rc, st.value

    def submit_complex(self, dA, dT, dU, dw, params=None, enclose=False):
        """Complex-plane request on complex128 device tensors (column-major)."""
        n = int(dA.shape[0])
        t = ctypes.c_uint64()
        p = params or default_params()
        rc = lib().eig_server_submit_complex(self._s, n, _ptr(dA), n, _ptr(dT), n, _ptr(dU), n,
                                             _ptr(dw), ctypes.byref(p), 1 if enclose else 0,
                                             ctypes.byref(t))
        if rc != EIG_OK:
            raise EigError(rc, "eig_server_submit_complex failed")
        self._keep[t.value] = (dA, dT, dU, dw)
        return t.value

    def cancel(self, ticket):
        """1 if the queued request was removed (status EIG_CANCELLED), 0 if it
        had already started or finished."""
        return lib().eig_server_cancel(self._s, ticket)

    def stats(self):
        c = ctypes.c_ulonglong()
        q = ctypes.c_ulonglong()
        r = ctypes.c_double()
        pk = ctypes.c_double()
        lib().eig_server_stats(self._s, ctypes.byref(c), ctypes.byref(q), ctypes.byref(r),
                               ctypes.byref(pk))
        return {"completed": c.value, "pending": q.value, "reserved_gb": r.value,
                "peak_reserved_gb": pk.value}

    def close(self):
        if self._s:
            lib().eig_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eig_qr(h, m, n, dX, ldx, dQ, ldq, dR, ldr):
    return h.check(lib().eig_qr(h.ptr, m, n, _ptr(dX), ldx, _ptr(dQ), ldq, _ptr(dR), ldr))


def eig_gaussian(h, rows, cols, seed, purpose, stream, attempt, dG, ldg):
    return h.check(lib().eig_gaussian(h.ptr, rows, cols, seed, purpose, stream, attempt,
                                      _ptr(dG), ldg))


def eig_haar(h, n, seed, purpose, stream, attempt, dV, ldv):
    return h.check(lib().eig_haar(h.ptr, n, seed, purpose, stream, attempt, _ptr(dV), ldv))


def eig_split_test(h, n, dA, lda, normA, dB=None, ldb=0, normB=0.0, want_scores=False):
    k = ctypes.c_int()
    e = ctypes.c_double()
    scores = np.zeros(max(n - 1, 1)) if want_scores else None
    sp = scores.ctypes.data_as(ctypes.c_void_p) if want_scores else ctypes.c_void_p(0)
    h.check(lib().eig_split_test(h.ptr, n, _ptr(dA), lda, normA, _ptr(dB), ldb, normB,
                                 ctypes.byref(k), ctypes.byref(e), sp))
    return k.value, e.value, (scores[:n - 1] if want_scores else None)


def eig_gemm(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    return h.check(lib().eig_gemm(h.ptr, int(ta), int(tb), m, n, k, alpha, _ptr(dA), lda,
                                  _ptr(dB), ldb, beta, _ptr(dC), ldc))


def eig_gemm_split(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    return h.check(lib().eig_gemm_split(h.ptr, int(ta), int(tb), m, n, k, alpha, _ptr(dA), lda,
                                        _ptr(dB), ldb, beta, _ptr(dC), ldc))


def eig_gemm_fp64tc(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    return h.check(lib().eig_gemm_fp64tc(h.ptr, int(ta), int(tb), m, n, k, alpha, _ptr(dA), lda,
                                        _ptr(dB), ldb, beta, _ptr(dC), ldc))


def eig_gemm_fp32tc(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    return h.check(lib().eig_gemm_fp32tc(h.ptr, int(ta), int(tb), m, n, k, alpha, _ptr(dA), lda,
                                        _ptr(dB), ldb, beta, _ptr(dC), ldc))


def eig_gemm_noalloc(stream, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    """Returns the status code (no handle: EIG_ERR_SCRATCH for shapes whose
    split-K partials exceed the static scratch)."""
    return lib().eig_gemm_noalloc(ctypes.c_void_p(stream.cuda_stream), int(ta), int(tb), m, n, k,
                                  alpha, _ptr(dA), lda, _ptr(dB), ldb, beta, _ptr(dC), ldc)


# ----------------------------------------------------------------- convenience

def solve_symmetric(h, A, params=None):
    """(w ascending, U, info) for a symmetric numpy matrix, through eig_solve."""
    import torch
    n = A.shape[0]
    params = params or default_params()
    dA = to_device(A)
    dw = torch.zeros(n, dtype=torch.float64, device=dA.device)
    dU = torch.zeros((n, n), dtype=torch.float64, device=dA.device)
    rc, info = eig_solve(h, EIG_KIND_SYM, n, dA, n, dw, None, dU, n, params)
    return rc, dw.cpu().numpy(), to_host(dU), info


def schur_nonsymmetric(h, A, params=None):
    """(T, U, wr, wi, info) for a real numpy matrix, through eig_solve."""
    import torch
    n = A.shape[0]
    params = params or default_params()
    dA = to_device(A)
    dwr = torch.zeros(n, dtype=torch.float64, device=dA.device)
    dwi = torch.zeros(n, dtype=torch.float64, device=dA.device)
    dU = torch.zeros((n, n), dtype=torch.float64, device=dA.device)
    rc, info = eig_solve(h, EIG_KIND_NONSYM, n, dA, n, dwr, dwi, dU, n, params)
    return rc, to_host(dA), to_host(dU), dwr.cpu().numpy(), dwi.cpu().numpy(), info


def pencil_schur(h, A, B, params=None):
    """(rc, S, T, QL, QR, alphar, alphai, beta, info) for a real numpy pencil,
    through eig_pencil_schur."""
    import torch
    n = A.shape[0]
    params = params or default_params()
    dA = to_device(A)
    dB = to_device(B)
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=dA.device)
    dQL, dQR = z(n, n), z(n, n)
    dar, dai, dbe = z(n), z(n), z(n)
    rc, info = eig_pencil_schur(h, n, dA, n, dB, n, dQL, n, dQR, n, dar, dai, dbe, params)
    return (rc, to_host(dA), to_host(dB), to_host(dQL), to_host(dQR), dar.cpu().numpy(),
            dai.cpu().numpy(), dbe.cpu().numpy(), info)


def eig_svd(h, m, n, dA, lda, dS, dU, ldu, dV, ldv, params):
    info = SolveInfo()
    rc = lib().eig_svd(h.ptr, m, n, _ptr(dA), lda, _ptr(dS), _ptr(dU), ldu, _ptr(dV), ldv,
                       ctypes.byref(params), ctypes.byref(info))
    return rc, info


def svd(h, A, params=None):
    """(rc, s descending, U, V, info) for a real numpy matrix, through eig_svd."""
    import torch
    m, n = A.shape
    r = min(m, n)
    params = params or default_params()
    dA = to_device(A)
    dS = torch.zeros(r, dtype=torch.float64, device=dA.device)
    dU = torch.zeros((r, m), dtype=torch.float64, device=dA.device)   # column-major m x r
    dV = torch.zeros((r, n), dtype=torch.float64, device=dA.device)
    rc, info = eig_svd(h, m, n, dA, m, dS, dU, m, dV, n, params)
    return rc, dS.cpu().numpy(), dU.cpu().numpy().T.copy(), dV.cpu().numpy().T.copy(), info


# ----------------------------------------------------------------- eigenvectors

def eig_eigenvectors(h, n, dT, ldt, dQ, ldq, dwi, dV, ldv, dlam):
    return lib().eig_eigenvectors(h.ptr, n, _ptr(dT), ldt, _ptr(dQ), ldq, _ptr(dwi), _ptr(dV),
                                  ldv, _ptr(dlam))


def eigenvectors(h, T, Q, wi):
    """(rc, lam, V) for a real Schur form (T, Q, wi) as schur_nonsymmetric returns it."""
    import torch
    n = T.shape[0]
    dT, dQ = to_device(T), to_device(Q)
    dwi = torch.from_numpy(np.ascontiguousarray(wi, dtype=np.float64)).to(dT.device)
    dV = torch.zeros((n, n), dtype=torch.complex128, device=dT.device)
    dlam = torch.zeros(n, dtype=torch.complex128, device=dT.device)
    rc = eig_eigenvectors(h, n, dT, n, dQ, n, dwi, dV, n, dlam)
    return rc, dlam.cpu().numpy(), dV.cpu().numpy().T.copy()


def eigenvectors_complex(h, T, U):
    """(rc, lam, V) for a complex Schur form (T, U) as schur_complex returns it."""
    import torch
    n = T.shape[0]
    dT, dU = to_device_complex(T), to_device_complex(U)
    dV = torch.zeros((n, n), dtype=torch.complex128, device=dT.device)
    dlam = torch.zeros(n, dtype=torch.complex128, device=dT.device)
    rc = lib().eig_eigenvectors_complex(h.ptr, n, _ptr(dT), n, _ptr(dU), n, _ptr(dV), n,
                                        _ptr(dlam))
    return rc, dlam.cpu().numpy(), dV.cpu().numpy().T.copy()


# ----------------------------------------------------------------- complex-plane strategy

def to_device_complex(A, device="cuda"):
    """numpy (rows x cols) -> torch complex128 tensor holding A column-major (interleaved)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.complex128).T)).to(device)


def eig_schur_complex(h, n, dA, lda, dT, ldt, dU, ldu, dw, params, enclose=False, enc_cap=16):
    """Complex Schur form through the C-ABI; returns (rc, info, enclosures)."""
    info = SolveInfo()
    enc = (Enclosure * max(enc_cap, 1))()
    n_enc = ctypes.c_int(0)
    rc = lib().eig_schur_complex(h.ptr, n, _ptr(dA), lda, _ptr(dT), ldt, _ptr(dU), ldu, _ptr(dw),
                                 ctypes.byref(params), 1 if enclose else 0, enc, enc_cap,
                                 ctypes.byref(n_enc), ctypes.byref(info))
    return rc, info, [enc[i] for i in range(min(n_enc.value, enc_cap))]


def eig_zgemm(h, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc):
    alpha, beta = complex(alpha), complex(beta)
    return lib().eig_zgemm(h.ptr, int(ta), int(tb), m, n, k, alpha.real, alpha.imag, _ptr(dA), lda,
                           _ptr(dB), ldb, beta.real, beta.imag, _ptr(dC), ldc)


def eig_zqr(h, m, n, dX, ldx, dQ, ldq, dR=None, ldr=0):
    return lib().eig_zqr(h.ptr, m, n, _ptr(dX), ldx, _ptr(dQ), ldq, _ptr(dR), ldr)


def eig_zhaar(h, n, seed, stream, attempt, dV, ldv):
    return lib().eig_zhaar(h.ptr, n, int(seed), int(stream), int(attempt), _ptr(dV), ldv)


def eig_zline_step(h, n, dA, lda, w, t, s, stream, attempt, params, dQ=None, ldq=0, dAhat=None,
                   ldah=0):
    """One complex-plane step; returns (rc, StepInfo)."""
    info = StepInfo()
    w = complex(w)
    rc = lib().eig_zline_step(h.ptr, n, _ptr(dA), lda, w.real, w.imag, float(t), float(s),
                              int(stream), int(attempt), ctypes.byref(params), _ptr(dQ), ldq,
                              _ptr(dAhat), ldah, ctypes.byref(info))
    return rc, info


def schur_complex(h, A, params=None, enclose=False):
    """(rc, T, U, w, info, enclosures) for a numpy matrix: A = U T U^H (Sec. 3.3)."""
    import torch
    n = A.shape[0]
    params = params or default_params()
    dA = to_device_complex(A)
    z = lambda *shape: torch.zeros(shape, dtype=torch.complex128, device=dA.device)
    dT, dU, dw = z(n, n), z(n, n), z(n)
    rc, info, enc = eig_schur_complex(h, n, dA, n, dT, n, dU, n, dw, params, enclose)
    return (rc, dT.cpu().numpy().T.copy(), dU.cpu().numpy().T.copy(), dw.cpu().numpy(), info,
            enc)


def cplane_enclosing_circle(c, R, halfplanes):
    """Host-only: (centre, radius) of a circle holding {|z - c| <= R} cut by the
    half-planes Re(conj(w) z) >= t given as [(w, t), ...]."""
    k = len(halfplanes)
    arr = ctypes.c_double * max(k, 1)
    wr = arr(*[complex(w).real for w, _ in halfplanes])
    wi = arr(*[complex(w).imag for w, _ in halfplanes])
    tt = arr(*[float(t) for _, t in halfplanes])
    mr, mi, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().eig_cplane_enclosing_circle(complex(c).real, complex(c).imag, float(R), k, wr, wi,
                                           tt, ctypes.byref(mr), ctypes.byref(mi),
                                           ctypes.byref(r))
    if rc != EIG_OK:
        raise EigError(rc, "eig_cplane_enclosing_circle: invalid argument")
    return complex(mr.value, mi.value), r.value


def cplane_draw_line(seed, node, attempt, c, R, perpendicular_to=None):
    """Host-only: the (w, t) of the strategy's line for (seed, node, attempt)."""
    pw = complex(perpendicular_to) if perpendicular_to is not None else 0j
    wr, wi, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().eig_cplane_draw_line(int(seed), int(node), int(attempt), complex(c).real,
                                    complex(c).imag, float(R),
                                    0 if perpendicular_to is None else 1, pw.real, pw.imag,
                                    ctypes.byref(wr), ctypes.byref(wi), ctypes.byref(t))
    if rc != EIG_OK:
        raise EigError(rc, "eig_cplane_draw_line: invalid argument")
    return complex(wr.value, wi.value), t.value


def eig_debug_fail_allocations(count):
    """Host-side fault injection: the next `count` workspace allocations fail
    (EIG_ERR_NOMEM).  Returns the previous pending count."""
    return int(lib().eig_debug_fail_allocations(int(count)))
