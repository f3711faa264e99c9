"""Thin ctypes binding to libzolo.so (the C ABI declared in include/zolo.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
library.  Matrices are torch tensors in column-major layout (stride(0) == 1),
FP64, on the handle's device; PyTorch supplies device memory and the stream.
If the shared library is missing this module raises at import time: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libzolo.so")

ZOLO_MAX_R = 8
ZOLO_MAX_ITERS = 8
ZOLO_FP64 = 0
ZOLO_SPLIT_BF16 = 1
ZOLO_SPLIT_FP16 = 2
ZOLO_SPLIT_FP8 = 3
ZOLO_R_TUNED = -1

ERRORS = {1: "ZOLO_ENONFINITE", 2: "ZOLO_ECHOL", 3: "ZOLO_ENOTCONV", 4: "ZOLO_ECUDA",
          5: "ZOLO_ENOMEM", 6: "ZOLO_EEIG", 7: "ZOLO_ETIMEOUT", 8: "ZOLO_EIO", 9: "ZOLO_EINVAL",
          10: "ZOLO_ECOMM", 11: "ZOLO_EPENDING", 12: "ZOLO_EGUARD"}
ZOLO_EPENDING = 11
ZOLO_PHASES = 8
PHASE_NAMES = ["bounds", "qr", "chol", "newton_schulz", "H", "estimates", "eig", "U"]

# int (*)(double* buf, int64_t count, void* stream, void* ctx)
SUM_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                          ctypes.c_void_p)


class ZoloOpts(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("posteriori", ctypes.c_int),
                ("ns_steps", ctypes.c_int), ("prec", ctypes.c_int), ("force_qr", ctypes.c_int),
                ("chol_form", ctypes.c_int), ("estimate", ctypes.c_int)]


class ZoloInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("r", ctypes.c_int),
                ("used_qr", ctypes.c_int * ZOLO_MAX_ITERS),
                ("ell", ctypes.c_double * (ZOLO_MAX_ITERS + 1)),
                ("delta", ctypes.c_double * ZOLO_MAX_ITERS),
                ("chol_fallbacks", ctypes.c_int), ("eig_sweeps", ctypes.c_int),
                ("ms", ctypes.c_double), ("chol_form", ctypes.c_int),
                ("bwd_est", ctypes.c_double), ("orth_est", ctypes.c_double),
                ("ms_phase", ctypes.c_float * ZOLO_PHASES)]


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("sm_ms", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libzolo.so is not built ({LIB_PATH}); run "
                          "`python -m paper_1806_06204_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    DP = ctypes.POINTER(ctypes.c_double)
    lib.zolo_opts_default.argtypes = [ctypes.POINTER(ZoloOpts)]
    lib.zolo_opts_default.restype = None
    lib.zolo_create.argtypes = [ctypes.POINTER(P), I]
    lib.zolo_create.restype = I
    lib.zolo_destroy.argtypes = [P]
    lib.zolo_destroy.restype = I
    lib.zolo_coefficients.argtypes = [D, I, DP, DP, DP, DP]
    lib.zolo_coefficients.restype = I
    lib.zolo_schedule.argtypes = [D, I, I, DP, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.zolo_schedule.restype = I
    pd_args = [P, P, I64, I64, I64, P, I64, P, I64, ctypes.POINTER(ZoloOpts),
               ctypes.POINTER(ZoloInfo), P]
    svd_args = [P, P, I64, I64, I64, P, I64, P, P, I64, ctypes.POINTER(ZoloOpts),
                ctypes.POINTER(ZoloInfo), P]
    for name, args in (("zolo_pd", pd_args), ("zolo_pd_host", pd_args), ("zolo_pd_async", pd_args),
                       ("zolo_svd", svd_args), ("zolo_svd_host", svd_args)):
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.zolo_strerror.argtypes = [I]
    lib.zolo_strerror.restype = ctypes.c_char_p
    lib.zolo_dgemm.argtypes = [P, I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64, I, I, P]
    lib.zolo_dgemm.restype = I
    lib.zolo_dgemm_noalloc.argtypes = [I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64, I, P]
    lib.zolo_dgemm_noalloc.restype = I
    lib.zolo_pd_batched.argtypes = [P, I, P, P, P, P, P, P, P, P, ctypes.POINTER(ZoloOpts),
                                    ctypes.POINTER(ZoloInfo), P]
    lib.zolo_pd_batched.restype = I
    lib.zolo_workspace_bytes.argtypes = [I64, I64, I, I, I, ctypes.POINTER(ctypes.c_uint64)]
    lib.zolo_workspace_bytes.restype = I
    lib.zolo_shift_range.argtypes = [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.zolo_shift_range.restype = I
    lib.zolo_pd_sharded.argtypes = pd_args + [I, I, SUM_FN, P]
    lib.zolo_pd_sharded.restype = I
    lib.zolo_debug_guards.argtypes = [P, I]
    lib.zolo_debug_guards.restype = I
    lib.zolo_batch_graphs.argtypes = [P, I]
    lib.zolo_batch_graphs.restype = I
    lib.zolo_debug_stall.argtypes = [P, I, I64]
    lib.zolo_debug_stall.restype = I
    lib.zolo_autotune.argtypes = [P, I]
    lib.zolo_autotune.restype = I
    lib.zolo_tuned_r.argtypes = [P, I64, I64, I, D]
    lib.zolo_tuned_r.restype = I
    for f in (lib.zolo_tune_save, lib.zolo_tune_load):
        f.argtypes = [P, ctypes.c_char_p]
        f.restype = I
    lib.zolo_kernel_launches.argtypes = []
    lib.zolo_kernel_launches.restype = ctypes.c_uint64
    lib.zolo_profile.argtypes = [I]
    lib.zolo_profile.restype = I
    lib.zolo_profile_read.argtypes = [ctypes.POINTER(KStat), I]
    lib.zolo_profile_read.restype = I
    return lib


LIB = _load()

EXPORTED = ["zolo_opts_default", "zolo_create", "zolo_destroy", "zolo_coefficients",
            "zolo_schedule", "zolo_pd", "zolo_svd", "zolo_pd_host", "zolo_svd_host",
            "zolo_strerror", "zolo_kernel_launches", "zolo_profile", "zolo_profile_read",
            "zolo_dgemm", "zolo_dgemm_noalloc", "zolo_pd_batched", "zolo_tuned_r",
            "zolo_tune_save", "zolo_tune_load", "zolo_autotune",
            "zolo_workspace_bytes", "zolo_debug_stall", "zolo_shift_range",
            "zolo_pd_sharded", "zolo_pd_async", "zolo_batch_graphs", "zolo_debug_guards"]


def kernel_launches() -> int:
    return int(LIB.zolo_kernel_launches())


def profile(enable: bool) -> None:
    LIB.zolo_profile(int(enable))


def profile_read() -> dict:
    """{class name: dict(launches, ms, flops, bytes, sm_ms)} accumulated since profile(True)."""
    buf = (KStat * 16)()
    k = LIB.zolo_profile_read(buf, 16)
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, flops=buf[i].flops,
                                       bytes=buf[i].bytes, sm_ms=buf[i].sm_ms)
            for i in range(min(k, 16))}


class ZoloError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = LIB.zolo_strerror(code).decode()
        super().__init__(f"{where} returned {code} ({ERRORS.get(code, 'argument')}: {msg})")


@dataclass
class Info:
    status: int
    iters: int
    r: int
    used_qr: list
    ell: list
    delta: list
    chol_fallbacks: int
    eig_sweeps: int
    ms: float
    chol_form: int
    bwd_est: float = 0.0
    orth_est: float = 0.0
    ms_phase: dict = field(default_factory=dict)

    @staticmethod
    def from_c(ci: ZoloInfo) -> "Info":
        k = ci.iters
        return Info(ci.status, k, ci.r, [bool(x) for x in ci.used_qr[:k]], list(ci.ell[:k + 1]),
                    list(ci.delta[:k]), ci.chol_fallbacks, ci.eig_sweeps, ci.ms, ci.chol_form,
                    ci.bwd_est, ci.orth_est,
                    {nm: float(ci.ms_phase[i]) for i, nm in enumerate(PHASE_NAMES)})


def opts(beta: float, alpha: float = 1.0, r: int = 0, max_iter: int = 6, posteriori: bool = False,
         ns_steps: int = 0, prec: int = ZOLO_FP64, force_qr: int = -1,
         chol_form: int = 0, estimate: bool = False) -> ZoloOpts:
    o = ZoloOpts()
    LIB.zolo_opts_default(ctypes.byref(o))
    o.r, o.alpha, o.beta, o.max_iter = r, alpha, beta, max_iter
    o.posteriori, o.ns_steps, o.prec, o.force_qr = int(posteriori), ns_steps, prec, force_qr
    o.chol_form = chol_form
    o.estimate = int(estimate)
    return o


def coefficients(ell: float, r: int):
    c = (ctypes.c_double * (2 * r))()
    a = (ctypes.c_double * r)()
    mh, gap = ctypes.c_double(), ctypes.c_double()
    e = LIB.zolo_coefficients(ell, r, c, a, ctypes.byref(mh), ctypes.byref(gap))
    if e:
        raise ZoloError(e, "zolo_coefficients")
    return list(c), list(a), mh.value, gap.value


def schedule(ell0: float, r: int = 0, max_iter: int = 8):
    ells = (ctypes.c_double * (ZOLO_MAX_ITERS + 1))()
    qr = (ctypes.c_int * ZOLO_MAX_ITERS)()
    ru = ctypes.c_int()
    k = LIB.zolo_schedule(ell0, r, max_iter, ells, qr, ctypes.byref(ru))
    if k < 0:
        raise ZoloError(k, "zolo_schedule")
    return list(ells[:k + 1]), [bool(x) for x in qr[:k]], ru.value


def workspace_bytes(m: int, n: int, r: int = 0, prec: int = ZOLO_FP64, svd: bool = False) -> int:
    """Device bytes a zolo_pd / zolo_svd call keeps in its handle (host-only query)."""
    out = ctypes.c_uint64()
    e = LIB.zolo_workspace_bytes(m, n, r, prec, int(svd), ctypes.byref(out))
    if e:
        raise ZoloError(e, "zolo_workspace_bytes")
    return int(out.value)


def autotune(handle, enable: bool) -> None:
    """Measure the contraction kernels of shapes met from now on (see zolo.h)."""
    e = LIB.zolo_autotune(handle.ptr, int(enable))
    if e:
        raise ZoloError(e, "zolo_autotune")


ZOLO_STALL_SPLIT_GEMM = 1
ZOLO_STALL_JACOBI32 = 2
ZOLO_STALL_JACOBI64 = 3


def debug_guards(handle, enable: bool) -> None:
    """Guard zones around the workspace's buffers, checked after each call (zolo.h)."""
    e = LIB.zolo_debug_guards(handle.ptr, int(enable))
    if e:
        raise ZoloError(e, "zolo_debug_guards")


def batch_graphs(handle, enable: bool) -> None:
    """zolo_pd_batched: record and replay a CUDA graph (True, default) or queue directly."""
    e = LIB.zolo_batch_graphs(handle.ptr, int(enable))
    if e:
        raise ZoloError(e, "zolo_batch_graphs")


def debug_stall(handle, where: int, ns: int = 0) -> None:
    """Test hook: make a kernel's first wait one that nothing completes (see zolo.h)."""
    e = LIB.zolo_debug_stall(handle.ptr, where, ns)
    if e:
        raise ZoloError(e, "zolo_debug_stall")


def tuned_r(handle, m: int, n: int, prec: int, ell0: float) -> int:
    """The r the handle has measured fastest for (m, n, prec, l_0), or 0."""
    return int(LIB.zolo_tuned_r(handle.ptr, m, n, prec, ell0))


def tune_save(handle, path: str) -> None:
    e = LIB.zolo_tune_save(handle.ptr, path.encode())
    if e:
        raise ZoloError(e, "zolo_tune_save")


def tune_load(handle, path: str) -> int:
    """Merge a saved tuning cache into the handle; returns the status (0 or ZOLO_E*)."""
    return int(LIB.zolo_tune_load(handle.ptr, path.encode()))


class Handle:
    """Owns a libzolo handle (device binding and workspace cache)."""

    def __init__(self, device: int = -1):
        self._h = ctypes.c_void_p()
        e = LIB.zolo_create(ctypes.byref(self._h), device)
        if e:
            raise ZoloError(e, "zolo_create")

    def close(self):
        if self._h:
            LIB.zolo_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._h


def _colmajor(t, name):
    import torch
    if t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 tensor")
    # strides of size-1 dimensions carry no information (torch may normalise them)
    if (t.shape[0] > 1 and t.stride(0) != 1) or _ld(t) < max(1, t.shape[0]):
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return t


def _ld(t) -> int:
    """Leading dimension of a column-major matrix view."""
    return t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])


def empty_colmajor(m: int, n: int, device="cuda"):
    import torch
    return torch.empty((n, m), dtype=torch.float64, device=device).t()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def zolo_pd(handle: Handle, A, o: ZoloOpts, Qp=None, H=None, stream=None, check=True):
    """Polar decomposition of the device tensor A (m x n, column-major)."""
    _colmajor(A, "A")
    m, n = A.shape
    Qp = empty_colmajor(m, n, A.device) if Qp is None else _colmajor(Qp, "Qp")
    H = empty_colmajor(n, n, A.device) if H is None else _colmajor(H, "H")
    info = ZoloInfo()
    e = LIB.zolo_pd(handle.ptr, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A),
                    ctypes.c_void_p(Qp.data_ptr()), _ld(Qp), ctypes.c_void_p(H.data_ptr()),
                    _ld(H), ctypes.byref(o), ctypes.byref(info), _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_pd")
    return Qp, H, Info.from_c(info)


def zolo_pd_async(handle: Handle, A, o: ZoloOpts, Qp=None, H=None, stream=None):
    """Queue a polar decomposition without host synchronisation.

    Returns (Qp, H, pending): Qp and H are written when the stream gets there,
    and pending() -> Info reads the status the library's host function leaves
    once the stream has been synchronised (ZOLO_EPENDING before that)."""
    _colmajor(A, "A")
    m, n = A.shape
    Qp = empty_colmajor(m, n, A.device) if Qp is None else _colmajor(Qp, "Qp")
    H = empty_colmajor(n, n, A.device) if H is None else _colmajor(H, "H")
    info = ZoloInfo()   # filled by the library's host function; kept alive by the closure
    e = LIB.zolo_pd_async(handle.ptr, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A),
                          ctypes.c_void_p(Qp.data_ptr()), _ld(Qp), ctypes.c_void_p(H.data_ptr()),
                          _ld(H), ctypes.byref(o), ctypes.byref(info), _stream(stream))
    if e:
        raise ZoloError(e, "zolo_pd_async")
    return Qp, H, lambda: Info.from_c(info)


def zolo_svd(handle: Handle, A, o: ZoloOpts, stream=None, check=True):
    """SVD of the device tensor A (m x n, column-major): (U, S, V, info)."""
    import torch
    _colmajor(A, "A")
    m, n = A.shape
    U = empty_colmajor(m, n, A.device)
    V = empty_colmajor(n, n, A.device)
    S = torch.empty(n, dtype=torch.float64, device=A.device)
    info = ZoloInfo()
    e = LIB.zolo_svd(handle.ptr, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A),
                     ctypes.c_void_p(U.data_ptr()), _ld(U), ctypes.c_void_p(S.data_ptr()),
                     ctypes.c_void_p(V.data_ptr()), _ld(V), ctypes.byref(o),
                     ctypes.byref(info), _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_svd")
    return U, S, V, Info.from_c(info)


def zolo_pd_batched(handle: Handle, As, os, Qps=None, Hs=None, stream=None, check=True):
    """Polar decompositions of a list of device tensors in one call.

    `os` is one ZoloOpts for all matrices or a list with one per matrix.
    Returns (Qps, Hs, infos, status)."""
    n_mat = len(As)
    if isinstance(os, ZoloOpts):
        os = [os] * n_mat
    if len(os) != n_mat:
        raise ValueError("one option set per matrix")
    for a in As:
        _colmajor(a, "A")
    Qps = [empty_colmajor(a.shape[0], a.shape[1], a.device) for a in As] if Qps is None else Qps
    Hs = [empty_colmajor(a.shape[1], a.shape[1], a.device) for a in As] if Hs is None else Hs
    for q, h in zip(Qps, Hs):
        _colmajor(q, "Qp")
        _colmajor(h, "H")
    PA = ctypes.c_void_p * max(n_mat, 1)
    LA = ctypes.c_int64 * max(n_mat, 1)
    a_p = PA(*[a.data_ptr() for a in As])
    q_p = PA(*[q.data_ptr() for q in Qps])
    h_p = PA(*[h.data_ptr() for h in Hs])
    m_a = LA(*[a.shape[0] for a in As])
    n_a = LA(*[a.shape[1] for a in As])
    lda = LA(*[_ld(a) for a in As])
    ldq = LA(*[_ld(q) for q in Qps])
    ldh = LA(*[_ld(h) for h in Hs])
    o_a = (ZoloOpts * max(n_mat, 1))(*os)
    i_a = (ZoloInfo * max(n_mat, 1))()
    e = LIB.zolo_pd_batched(handle.ptr, n_mat, ctypes.cast(a_p, ctypes.c_void_p),
                            ctypes.cast(m_a, ctypes.c_void_p), ctypes.cast(n_a, ctypes.c_void_p),
                            ctypes.cast(lda, ctypes.c_void_p), ctypes.cast(q_p, ctypes.c_void_p),
                            ctypes.cast(ldq, ctypes.c_void_p), ctypes.cast(h_p, ctypes.c_void_p),
                            ctypes.cast(ldh, ctypes.c_void_p), o_a, i_a, _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_pd_batched")
    return Qps, Hs, [Info.from_c(i_a[i]) for i in range(n_mat)], e


def shift_range(r: int, rank: int, nranks: int):
    """The shifts [j0, j1) rank `rank` of `nranks` takes (host only, no device)."""
    j0, j1 = ctypes.c_int(), ctypes.c_int()
    e = LIB.zolo_shift_range(r, rank, nranks, ctypes.byref(j0), ctypes.byref(j1))
    if e:
        raise ZoloError(e, "zolo_shift_range")
    return j0.value, j1.value


def torch_allreduce(group=None):
    """A sum over the ranks of a torch.distributed process group, in place:
    the function zolo_pd_sharded expects (NCCL on GPUs, gloo on CPUs)."""
    import torch.distributed as dist

    def f(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return f


class _DeviceArray:
    """`count` doubles of device memory at `ptr`, exposed to torch without a copy."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8",
                                         "data": (ptr, False), "version": 3, "strides": None}


def zolo_pd_sharded(handle: Handle, A, o: ZoloOpts, rank: int, nranks: int, allreduce,
                    Qp=None, H=None, stream=None, check=True):
    """Polar decomposition with the r shifts of every iteration shared out over
    `nranks` ranks (each rank calls this with the same A and options).
    allreduce(t) must sum the 1-D float64 device tensor t over all ranks in
    place, ordered on torch's current stream (torch_allreduce(group) does)."""
    import torch
    _colmajor(A, "A")
    m, n = A.shape
    Qp = empty_colmajor(m, n, A.device) if Qp is None else _colmajor(Qp, "Qp")
    H = empty_colmajor(n, n, A.device) if H is None else _colmajor(H, "H")
    info = ZoloInfo()
    st = _stream(stream)

    def cb(buf, count, stream_ptr, ctx):
        try:
            t = torch.as_tensor(_DeviceArray(buf, count), device=A.device)
            s = (torch.cuda.ExternalStream(stream_ptr, device=A.device) if stream_ptr
                 else torch.cuda.default_stream(A.device))
            with torch.cuda.stream(s):
                allreduce(t)
            return 0
        except Exception:   # reported to the library as a failed sum (ZOLO_ECOMM)
            import traceback
            traceback.print_exc()
            return 1

    fn = SUM_FN(cb)
    e = LIB.zolo_pd_sharded(handle.ptr, ctypes.c_void_p(A.data_ptr()), m, n, _ld(A),
                            ctypes.c_void_p(Qp.data_ptr()), _ld(Qp), ctypes.c_void_p(H.data_ptr()),
                            _ld(H), ctypes.byref(o), ctypes.byref(info), st, rank, nranks, fn,
                            None)
    if e and check:
        raise ZoloError(e, "zolo_pd_sharded")
    return Qp, H, Info.from_c(info)


def _host_ptr(a):
    import numpy as np
    if a.dtype != np.float64 or not a.flags.f_contiguous:
        raise ValueError("host matrices must be float64, Fortran (column-major) order")
    return ctypes.c_void_p(a.ctypes.data)


def zolo_pd_host(handle: Handle, A, o: ZoloOpts, Qp, H, stream=None, check=True):
    """Polar decomposition with host (numpy, Fortran-order) buffers; copies inside the call."""
    m, n = A.shape
    info = ZoloInfo()
    e = LIB.zolo_pd_host(handle.ptr, _host_ptr(A), m, n, m, _host_ptr(Qp), m, _host_ptr(H), n,
                         ctypes.byref(o), ctypes.byref(info), _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_pd_host")
    return Info.from_c(info)


def zolo_svd_host(handle: Handle, A, o: ZoloOpts, U, S, V, stream=None, check=True):
    """SVD with host (numpy, Fortran-order) buffers; copies inside the call."""
    m, n = A.shape
    info = ZoloInfo()
    e = LIB.zolo_svd_host(handle.ptr, _host_ptr(A), m, n, m, _host_ptr(U), m,
                          ctypes.c_void_p(S.ctypes.data), _host_ptr(V), n, ctypes.byref(o),
                          ctypes.byref(info), _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_svd_host")
    return Info.from_c(info)


def _gemm_shape(A, B, transA, transB):
    """(m, n, k) of op(A) op(B); raises unless op(B)'s rows match op(A)'s columns."""
    m = A.shape[1] if transA else A.shape[0]
    k = A.shape[0] if transA else A.shape[1]
    kb = B.shape[1] if transB else B.shape[0]
    n = B.shape[0] if transB else B.shape[1]
    if kb != k:
        raise ValueError(f"op(A) is {m} x {k} but op(B) has {kb} rows")
    return m, n, k


def _check_c(C, m, n):
    if tuple(C.shape) != (m, n):
        raise ValueError(f"C must be {m} x {n}, got {tuple(C.shape)}")


def zolo_dgemm(handle: Handle, A, B, C=None, alpha=1.0, beta=0.0, transA=False, transB=False,
               prec: int = ZOLO_FP64, slices: int = 0, stream=None, check=True):
    """C = alpha op(A) op(B) + beta C on the device (column-major float64 tensors)."""
    _colmajor(A, "A")
    _colmajor(B, "B")
    m, n, k = _gemm_shape(A, B, transA, transB)
    if C is None:
        C = empty_colmajor(m, n, A.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
    _colmajor(C, "C")
    _check_c(C, m, n)
    e = LIB.zolo_dgemm(handle.ptr, int(transA), int(transB), m, n, k, alpha,
                       ctypes.c_void_p(A.data_ptr()), _ld(A), ctypes.c_void_p(B.data_ptr()), _ld(B),
                       beta, ctypes.c_void_p(C.data_ptr()), _ld(C), prec, slices, _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_dgemm")
    return C


def zolo_dgemm_noalloc(A, B, C, alpha=1.0, beta=0.0, transA=False, transB=False, slices: int = 0,
                       stream=None, check=True):
    """Split-precision C = alpha op(A) op(B) + beta C using only the library's fixed
    device scratch (no allocation inside the call); C must be given."""
    _colmajor(A, "A")
    _colmajor(B, "B")
    _colmajor(C, "C")
    m, n, k = _gemm_shape(A, B, transA, transB)
    _check_c(C, m, n)
    e = LIB.zolo_dgemm_noalloc(int(transA), int(transB), m, n, k, alpha,
                               ctypes.c_void_p(A.data_ptr()), _ld(A), ctypes.c_void_p(B.data_ptr()),
                               _ld(B), beta, ctypes.c_void_p(C.data_ptr()), _ld(C), slices,
                               _stream(stream))
    if e and check:
        raise ZoloError(e, "zolo_dgemm_noalloc")
    return e
