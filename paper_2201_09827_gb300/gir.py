"""Thin ctypes binding of ``libgir.so`` (include/gir.h): argument marshalling only.

Every step of the solver runs in the CUDA library. Torch is used only to own device memory
and to supply the current CUDA stream; tensors are passed as raw device pointers. If the
library is missing the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, replace

import torch

from . import build as _build

GIR_FP64, GIR_FP32, GIR_FP16, GIR_BF16, GIR_FP8_E4M3, GIR_DD = range(6)
PREC = {"fp64": GIR_FP64, "fp32": GIR_FP32, "fp16": GIR_FP16, "bf16": GIR_BF16, "e4m3": GIR_FP8_E4M3,
        "dd": GIR_DD}
STATUS = ["GIR_OK", "GIR_NOT_CONVERGED", "GIR_SINGULAR", "GIR_NONFINITE", "GIR_INVALID_ARG", "GIR_TIMEOUT",
          "GIR_CUDA_ERROR", "GIR_OOM", "GIR_UNSUPPORTED"]
GIR_OK, GIR_NOT_CONVERGED, GIR_SINGULAR, GIR_NONFINITE, GIR_INVALID_ARG, GIR_TIMEOUT, GIR_CUDA_ERROR, GIR_OOM, \
    GIR_UNSUPPORTED = range(9)
GIR_MAX_M = 112
GIR_MAX_K = 64
GIR_MAX_IR = 64


class CParams(C.Structure):
    _fields_ = [("uf", C.c_int), ("u", C.c_int), ("ur", C.c_int), ("ua", C.c_int), ("m", C.c_int), ("k", C.c_int),
                ("tau", C.c_double), ("imax", C.c_int), ("target_berr", C.c_double), ("carry_mode", C.c_int),
                ("max_its", C.c_int), ("lu_nb", C.c_int), ("flags", C.c_uint)]


class CInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("ir_steps", C.c_int), ("total_its", C.c_int), ("its", C.c_int * GIR_MAX_IR),
                ("carry_applies", C.c_int * GIR_MAX_IR), ("berr", C.c_double * (GIR_MAX_IR + 1)),
                ("final_berr", C.c_double), ("cycles", C.c_int), ("k_eff", C.c_int), ("ms_factor", C.c_float),
                ("ms_solve", C.c_float), ("cw_berr", C.c_double * (GIR_MAX_IR + 1)), ("final_cw_berr", C.c_double)]


SYMBOLS = {
    "gir_factor": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(CParams), C.c_void_p, C.POINTER(C.c_void_p)]),
    "gir_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(CInfo), C.c_void_p]),
    "gir_solve_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(CInfo),
                                    C.c_void_p]),
    "gir_batch_solve": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(CParams), C.POINTER(CInfo),
                                  C.c_void_p]),
    "gir_autotune": (C.c_int, [C.POINTER(C.c_int64), C.c_int, C.c_void_p]),
    "gir_batch_engine": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(CParams)]),
    "gir_tune_report": (C.c_int, [C.c_char_p, C.c_int]),
    "gir_adjoint_grad_a": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "gir_free": (None, [C.c_void_p]),
    "gir_status_string": (C.c_char_p, [C.c_int]),
    "gir_handle_n": (C.c_int64, [C.c_void_p]),
    "gir_residual": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                               C.c_void_p]),
    "gir_backward_errors": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "gir_selftest_wait_timeout": (C.c_int, [C.c_longlong, C.c_void_p]),
    "gir_gemv": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gir_export_factors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double), C.c_void_p]),
    "gir_apply_minv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gir_apply_atilde": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gir_gcrodr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_int),
                             C.c_void_p]),
    "gir_export_recycle": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                     C.c_void_p]),
    "gir_reset_recycle": (C.c_int, [C.c_void_p]),
    "gir_lu_panel": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "gir_lu_update": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "gir_gemv_t_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gir_trace_enable": (None, [C.c_int]),
    "gir_trace_report": (C.c_int, [C.c_char_p, C.c_int]),
    "gir_trace_select": (None, [C.c_char_p]),
    "gir_launch_count": (C.c_ulonglong, []),
    "gir_small_eig": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int, C.POINTER(C.c_int), C.c_int]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgir.so (raises if it is missing and ``build_if_missing`` is false)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
        _build.build_library()
    lib = C.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GirError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS[status] if 0 <= status < len(STATUS) else status}")


@dataclass
class Params:
    """Arguments of Algorithm 4: precisions (u_f, u, u_r, u_a), restart m, recycle k, tau, i_max."""
    uf: str = "bf16"
    u: str = "fp64"
    ur: str = "fp64"
    ua: str = "fp64"
    m: int = 30
    k: int = 10
    tau: float = 1e-8
    imax: int = 10
    target_berr: float = -1.0
    carry_mode: int = 1
    max_its: int = 0
    lu_nb: int = 0
    flags: int = 0

    def c(self) -> CParams:
        return CParams(PREC[self.uf], PREC[self.u], PREC[self.ur], PREC[self.ua], self.m, self.k, self.tau, self.imax,
                       self.target_berr, self.carry_mode, self.max_its, self.lu_nb, self.flags)


GIR_FLAG_AUTOTUNE = 0x1
GIR_FLAG_CW_BERR = 0x2   # also compute the componentwise backward error and stop on both
GIR_FLAG_SIR = 0x4       # Algorithm 1 comparator: correction by substitution, no GCRO-DR
GIR_FLAG_ADAPTIVE_K = 0x8  # k = its_1 - 1 from the first refinement step (Section 5)
GIR_FLAG_EIG_FP64 = 0x10  # harmonic Ritz eigenvalues by FP64 Hessenberg QR (default FP32)
GIR_FLAG_BASIS_FP32 = 0x20  # Krylov and recycle basis vectors rounded to FP32 when stored
GIR_FLAG_BATCH_STREAMS = 0x40  # batch_solve on the worker-stream pool instead of the persistent kernel
GIR_FLAG_BATCH_PERSISTENT = 0x80  # batch_solve as the persistent kernel whatever the cost model prefers


@dataclass
class Info:
    status: int
    ir_steps: int
    total_its: int
    its: list
    carry_applies: list
    berr: list
    final_berr: float
    cycles: int
    k_eff: int
    ms_factor: float
    ms_solve: float
    cw_berr: list = field(default_factory=list)
    final_cw_berr: float = -1.0

    @classmethod
    def from_c(cls, ci: CInfo):
        s = ci.ir_steps
        nb = s + 1
        return cls(ci.status, s, ci.total_its, list(ci.its[:s]), list(ci.carry_applies[:s]), list(ci.berr[:nb]),
                   ci.final_berr, ci.cycles, ci.k_eff, ci.ms_factor, ci.ms_solve, list(ci.cw_berr[:nb]),
                   ci.final_cw_berr)

    @property
    def converged(self):
        return self.status == GIR_OK

    def paper_format(self):
        if not self.converged:
            return "-"
        return f"{self.total_its} ({','.join(str(i) for i in self.its)})"


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check_matrix(A: torch.Tensor):
    if not A.is_cuda or A.dtype != torch.float64 or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square FP64 CUDA tensor")
    if A.stride(1) != 1:
        raise ValueError("A must be row-major (stride(1) == 1)")
    return A.shape[0], A.stride(0)


def _check_vec(v: torch.Tensor, n: int):
    if not v.is_cuda or v.dtype != torch.float64 or v.numel() != n or not v.is_contiguous():
        raise ValueError("vectors must be contiguous FP64 CUDA tensors of length n")


class Factorization:
    """A gir_handle: the u_f LU factors of A plus the recycle spaces (Algorithm 4, the factorization step)."""

    def __init__(self, A: torch.Tensor, params: Params, stream=None):
        lib = load()
        self.n, self.lda = _check_matrix(A)
        self.params = params
        self._cp = params.c()
        h = C.c_void_p()
        st = lib.gir_factor(_ptr(A), self.n, self.lda, C.byref(self._cp), _stream(stream), C.byref(h))
        if st != GIR_OK:
            raise GirError(st, "gir_factor")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().gir_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, A, b, x=None, stream=None, raise_on_error=False):
        n = self.n
        _check_vec(b, n)
        if x is None:
            x = torch.empty_like(b)
        ci = CInfo()
        st = load().gir_solve(self._h, _ptr(A), A.stride(0), _ptr(b), _ptr(x), C.byref(ci), _stream(stream))
        info = Info.from_c(ci)
        info.status = st
        if raise_on_error and st not in (GIR_OK, GIR_NOT_CONVERGED):
            raise GirError(st, "gir_solve")
        return x, info

    def solve_adjoint(self, A, g, lam=None, stream=None):
        _check_vec(g, self.n)
        if lam is None:
            lam = torch.empty_like(g)
        ci = CInfo()
        st = load().gir_solve_adjoint(self._h, _ptr(A), A.stride(0), _ptr(g), _ptr(lam), C.byref(ci), _stream(stream))
        info = Info.from_c(ci)
        info.status = st
        return lam, info

    def export_factors(self, stream=None):
        n = self.n
        LU = torch.empty(n, n, dtype=torch.float32, device="cuda")
        ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
        R = torch.empty(n, dtype=torch.float64, device="cuda")
        S = torch.empty(n, dtype=torch.float64, device="cuda")
        mu = C.c_double()
        st = load().gir_export_factors(self._h, _ptr(LU), _ptr(ipiv), _ptr(R), _ptr(S), C.byref(mu), _stream(stream))
        if st != GIR_OK:
            raise GirError(st, "gir_export_factors")
        return LU, ipiv, R, S, mu.value

    def apply_minv(self, v, trans=False, stream=None):
        w = torch.empty_like(v)
        st = load().gir_apply_minv(self._h, _ptr(v), _ptr(w), int(trans), _stream(stream))
        if st != GIR_OK:
            raise GirError(st, "gir_apply_minv")
        return w

    def apply_atilde(self, A, v, trans=False, stream=None):
        w = torch.empty_like(v)
        st = load().gir_apply_atilde(self._h, _ptr(A), A.stride(0), _ptr(v), _ptr(w), int(trans), _stream(stream))
        if st != GIR_OK:
            raise GirError(st, "gir_apply_atilde")
        return w

    def gcrodr(self, A, c, stream=None):
        d = torch.empty_like(c)
        its = C.c_int()
        st = load().gir_gcrodr(self._h, _ptr(A), A.stride(0), _ptr(c), _ptr(d), C.byref(its), _stream(stream))
        if st not in (GIR_OK, GIR_NOT_CONVERGED):
            raise GirError(st, "gir_gcrodr")
        return d, its.value, st

    def export_recycle(self, adjoint=False, kcap=GIR_MAX_K, stream=None):
        U = torch.zeros(kcap, self.n, dtype=torch.float64, device="cuda")
        Cm = torch.zeros(kcap, self.n, dtype=torch.float64, device="cuda")
        k = C.c_int()
        st = load().gir_export_recycle(self._h, int(adjoint), _ptr(U), _ptr(Cm), kcap, C.byref(k), _stream(stream))
        if st != GIR_OK:
            raise GirError(st, "gir_export_recycle")
        return U[:k.value].T.contiguous(), Cm[:k.value].T.contiguous()

    def reset_recycle(self):
        load().gir_reset_recycle(self._h)


def residual(A, x, b, prec="fp64", stream=None):
    n, lda = _check_matrix(A)
    r = torch.empty_like(b)
    st = load().gir_residual(_ptr(A), n, lda, _ptr(x), _ptr(b), _ptr(r), PREC[prec], _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_residual")
    return r


def backward_errors(A, x, b, prec="fp64", stream=None):
    """(eta, omega): normwise and componentwise backward errors of x (Table 2's two columns)."""
    n, lda = _check_matrix(A)
    eta, om = C.c_double(0.0), C.c_double(0.0)
    st = load().gir_backward_errors(_ptr(A), n, lda, _ptr(x), _ptr(b), PREC[prec], C.byref(eta), C.byref(om),
                                    _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_backward_errors")
    return eta.value, om.value


def selftest_wait_timeout(spin_limit=100000, stream=None):
    """Status of a device wait made to run out (GIR_TIMEOUT is the expected answer)."""
    return load().gir_selftest_wait_timeout(int(spin_limit), _stream(stream))


def gemv(A, v, trans=False, stream=None):
    n, lda = _check_matrix(A)
    w = torch.empty_like(v)
    st = load().gir_gemv(_ptr(A), n, lda, _ptr(v), _ptr(w), int(trans), _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_gemv")
    return w


def small_eig(M, k, largest, mcap, eig_prec="fp32"):
    """GPU single-warp eigen-solver of the harmonic Ritz step on a host numpy matrix (testing).

    ``eig_prec`` is the precision of the Hessenberg QR that gives the eigenvalues: "fp32" (the
    solver's default) or "fp64"."""
    import numpy as np
    M = np.asarray(M, dtype=np.float64)
    d = M.shape[0]
    Mc = np.asfortranarray(M)
    wr = np.zeros(d)
    wi = np.zeros(d)
    kcap = min(d, k + 2)
    P = np.zeros((d, kcap), order="F")
    kout = C.c_int()
    st = load().gir_small_eig(Mc.ctypes.data_as(C.c_void_p), d, k, int(largest), mcap,
                              wr.ctypes.data_as(C.c_void_p), wi.ctypes.data_as(C.c_void_p),
                              P.ctypes.data_as(C.c_void_p), kcap, C.byref(kout), PREC[eig_prec])
    if st != GIR_OK:
        raise GirError(st, "gir_small_eig")
    kk = kout.value
    failed = kk < 0
    cols = -kk - 1 if failed else kk
    return wr, wi, P[:, :cols], failed


def lu_panel(W: torch.Tensor, cluster: int = 0, stream=None):
    """GEPP of one FP32 panel (m x w, w <= 32) in place on the GPU; returns the pivot rows."""
    if not W.is_cuda or W.dtype != torch.float32 or W.dim() != 2 or W.stride(1) != 1:
        raise ValueError("W must be a row-major FP32 CUDA matrix")
    m, w = W.shape
    ipiv = torch.empty(w, dtype=torch.int32, device=W.device)
    st = load().gir_lu_panel(_ptr(W), W.stride(0), m, w, _ptr(ipiv), cluster, _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_lu_panel")
    return ipiv


def lu_update(Cm: torch.Tensor, A16: torch.Tensor, B16: torch.Tensor, fmt="bf16", use_tc=True, stream=None):
    """Cm -= A16 @ B16 (16-bit operands stored as int16 bit patterns) on the tensor-core or CUDA-core path."""
    M, K = A16.shape
    N = B16.shape[1]
    Bt = B16.t().contiguous()
    st = load().gir_lu_update(_ptr(Cm), Cm.stride(0), _ptr(A16), A16.stride(0), _ptr(B16), B16.stride(0), _ptr(Bt),
                              Bt.stride(0), M, N, K, PREC[fmt], int(use_tc), _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_lu_update")
    return Cm


def trace_enable(on=True):
    load().gir_trace_enable(int(on))


def trace_select(names=None):
    """Time only the named phases (None: all)."""
    load().gir_trace_select(None if not names else ",".join(names).encode())


def trace_report():
    """{phase: (ms, calls)} accumulated since the last report (resolves pending events)."""
    lib = load()
    n = lib.gir_trace_report(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib.gir_trace_report(buf, n + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        name, ms, cnt = line.split("\t")
        out[name] = (float(ms), int(cnt))
    return out


def launch_count() -> int:
    return int(load().gir_launch_count())


def solve(A, b, params: Params | None = None, stream=None):
    """x = A^-1 b by RGMRES-IR (Algorithm 4) on one system.

    A and b may be CUDA tensors (the solve runs in place on the device) or CPU tensors: then
    they are staged through pinned host buffers, copied to the current device on the solve's
    stream, and x is copied back to a CPU tensor (the host <-> device copies are part of the
    call). Returns (x, Info)."""
    params = params or Params()
    host = not A.is_cuda
    if host:
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            Ah = A if A.is_pinned() else A.pin_memory()
            bh = b if b.is_pinned() else b.pin_memory()
            Ad = Ah.to("cuda", non_blocking=True)
            bd = bh.to("cuda", non_blocking=True)
            F = Factorization(Ad, params, stream=s)
            xd, info = F.solve(Ad, bd, stream=s)
            F.close()
            xh = torch.empty(xd.shape, dtype=xd.dtype, pin_memory=True)
            xh.copy_(xd, non_blocking=True)
        s.synchronize()
        return xh, info
    F = Factorization(A, params, stream=stream)
    x, info = F.solve(A, b, stream=stream)
    F.close()
    return x, info


def autotune(sizes, stream=None):
    """Measure LU block widths for the size classes of `sizes` and the batch worker count."""
    sizes = [int(v) for v in sizes]
    arr = (C.c_int64 * len(sizes))(*sizes)
    st = load().gir_autotune(arr, len(sizes), _stream(stream))
    if st != GIR_OK:
        raise GirError(st, "gir_autotune")


def tune_report() -> str:
    lib = load()
    need = lib.gir_tune_report(None, 0)
    buf = C.create_string_buffer(need)
    lib.gir_tune_report(buf, need)
    return buf.value.decode()


def batch_engine(sizes, params: Params, ldas=None) -> str:
    """'persistent' or 'streams': the engine gir_batch_solve picks for these orders and parameters."""
    sizes = [int(v) for v in sizes]
    ldas = [int(v) for v in (ldas or sizes)]
    ns = (C.c_int64 * len(sizes))(*sizes)
    ls = (C.c_int64 * len(ldas))(*ldas)
    cp = params.c()
    r = load().gir_batch_engine(len(sizes), ns, ls, C.byref(cp))
    if r < 0:
        raise GirError(GIR_INVALID_ARG, "gir_batch_engine")
    return "persistent" if r == 1 else "streams"


def batch_solve(As, bs, params: Params, stream=None, autotune: bool = False, engine: str = "auto"):
    """Solve independent systems A_i x_i = b_i (gir_batch_solve).

    engine="auto": one persistent kernel launch for the whole batch where it applies (u_f bf16 or
    fp16, ua fp64, no CW_BERR / SIR flag, n <= 8192, m <= 100) and the cost model prefers it (many
    systems), else the worker-stream pool; engine="persistent" forces the kernel
    (GIR_FLAG_BATCH_PERSISTENT; GirError if it cannot take the batch), engine="streams" the pool
    (GIR_FLAG_BATCH_STREAMS). autotune=True measures missing size classes of the pool first
    (GIR_FLAG_AUTOTUNE)."""
    if engine not in ("auto", "persistent", "streams"):
        raise ValueError(f"engine must be 'auto', 'persistent' or 'streams', not {engine!r}")
    if autotune:
        params = replace(params, flags=params.flags | GIR_FLAG_AUTOTUNE)
    if engine == "streams":
        params = replace(params, flags=params.flags | GIR_FLAG_BATCH_STREAMS)
    elif engine == "persistent":
        params = replace(params, flags=params.flags | GIR_FLAG_BATCH_PERSISTENT)
    lib = load()
    nsys = len(As)
    ns = (C.c_int64 * nsys)(*[A.shape[0] for A in As])
    ldas = (C.c_int64 * nsys)(*[A.stride(0) for A in As])
    xs = [torch.empty_like(b) for b in bs]
    Ap = (C.c_void_p * nsys)(*[A.data_ptr() for A in As])
    bp = (C.c_void_p * nsys)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * nsys)(*[x.data_ptr() for x in xs])
    infos = (CInfo * nsys)()
    cp = params.c()
    st = lib.gir_batch_solve(nsys, ns, Ap, ldas, bp, xp, C.byref(cp), infos, _stream(stream))
    if engine == "persistent" and st == GIR_UNSUPPORTED:
        raise GirError(st, "gir_batch_solve: the persistent kernel cannot take this batch")
    return xs, [Info.from_c(infos[i]) for i in range(nsys)], st


class GirSolve(torch.autograd.Function):
    """x = A^-1 b by RGMRES-IR; backward solves A^T lambda = g with the same factors.

    Gradients: db = lambda, dA = -lambda x^T, both computed by the library (the adjoint solve
    and gir_adjoint_grad_a).
    """

    @staticmethod
    def forward(ctx, A, b, params: Params):
        F = Factorization(A, params)
        x, info = F.solve(A, b, raise_on_error=True)
        ctx.F = F
        ctx.save_for_backward(A, x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, g):
        A, x = ctx.saved_tensors
        lam, info = ctx.F.solve_adjoint(A, g.contiguous())
        if info.status not in (GIR_OK, GIR_NOT_CONVERGED):
            raise GirError(info.status, "gir_solve_adjoint")
        dA = None
        if ctx.needs_input_grad[0]:
            n = x.shape[0]
            dA = torch.empty((n, n), dtype=torch.float64, device=x.device)
            st = load().gir_adjoint_grad_a(_ptr(lam), _ptr(x), n, _ptr(dA), n, _stream(None))
            if st != GIR_OK:
                raise GirError(st, "gir_adjoint_grad_a")
        return dA, lam, None
