"""ctypes binding of libtprod (include/tprod.h).

Argument marshalling only: every step of every call runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (float32 or float64,
contiguous); the current torch stream is used; workspaces come from torch's
caching allocator.  There is no CPU path: a missing library or a non-CUDA
tensor raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libtprod.so")

TP_OK, TP_ERR_ARG, TP_ERR_CUDA, TP_ERR_WORKSPACE = 0, -1, -2, -3
TP_ERR_BREAKDOWN, TP_ERR_NOT_CONVERGED, TP_ERR_TIMEOUT, TP_ERR_UNSUPPORTED = -4, -5, -6, -7
TP_ERR_NONFINITE = -8
TP_FP32, TP_FP64, TP_TF32, TP_BF16 = 0, 1, 2, 3


class TpInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("k", ctypes.c_int), ("r", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("residual", ctypes.c_double), ("tau_delta", ctypes.c_double), ("eta", ctypes.c_double),
                ("mu", ctypes.c_double), ("margin", ctypes.c_double), ("norm_a2", ctypes.c_double)]


class RtsvdParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_double), ("eps", ctypes.c_double),
                ("eps_rel", ctypes.c_double), ("p_over", ctypes.c_int), ("q_power", ctypes.c_int),
                ("block", ctypes.c_int), ("r_max", ctypes.c_int), ("res_hist", ctypes.c_void_p)]


class TtsvdParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_double), ("res_hist", ctypes.c_void_p)]


class TgkbParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_double), ("k_max", ctypes.c_int),
                ("res_hist", ctypes.c_void_p), ("delta_p", ctypes.c_void_p)]


class TikParams(ctypes.Structure):
    _fields_ = [("gkb", TgkbParams), ("mu_lo", ctypes.c_double), ("mu_hi", ctypes.c_double),
                ("log_tol", ctypes.c_double)]


# every symbol include/tprod.h declares
EXPORTS = ("tprod_fft", "tprod_ifft", "tprod_gemm_workspace_bytes", "tprod_gemm", "rtsvd_workspace_bytes",
           "rtsvd_truncated_solve", "tgkb_workspace_bytes", "tgkb_solve", "tgkb_tikhonov_workspace_bytes",
           "tgkb_tikhonov_solve", "tp_status_string", "tp_version", "tp_kernel_launches", "tp_timing_enable",
           "tp_timing_read", "tp_wait_budget", "tp_wait_stall", "tprod_gemm_noalloc", "rtsvd_adjoint", "nested_tgkb_workspace_bytes",
           "nested_tgkb_solve", "ttsvd_workspace_bytes", "ttsvd_solve", "tgkb_triplets_workspace_bytes",
           "tgkb_triplets", "sep_grad_c_workspace_bytes", "sep_grad_c", "tgkb_tikhonov_grad_c_workspace_bytes",
           "tgkb_tikhonov_grad_c", "sep_operator", "ttsvd_adjoint",
           "rtsvd_truncated_solve_hat", "tgkb_solve_hat", "tgkb_tikhonov_solve_hat",
           "tgkb_tikhonov_adjoint_workspace_bytes", "tgkb_tikhonov_adjoint", "tgkb_adjoint_workspace_bytes",
           "tgkb_adjoint", "rtsvd_autotune", "tp_autotune_table", "tp_autotune_clear", "tp_autotune_set")

KERNEL_CLASSES = ("dft", "gemm", "orth", "svd", "gkb", "dp", "tik", "misc")

_lib = None


class TprodError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {status_string(status)} ({status})")
        self.status = status


def load(path: str | None = None):
    """Load libtprod.so (built by paper_2110_02485_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libtprod.so not built ({p}); run `python -m paper_2110_02485_gb300.build`")
    L = ctypes.CDLL(p)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.tprod_fft.argtypes = [vp, i, i, i, vp, i, vp]
    L.tprod_ifft.argtypes = [vp, i, i, i, vp, i, vp]
    L.tprod_gemm_workspace_bytes.argtypes = [i, i, i, i, i]
    L.tprod_gemm_workspace_bytes.restype = sz
    L.tprod_gemm.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp, sz, vp]
    L.rtsvd_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(RtsvdParams), i]
    L.rtsvd_workspace_bytes.restype = sz
    L.rtsvd_truncated_solve.argtypes = [vp, vp, vp, i, i, i, i, ctypes.POINTER(RtsvdParams), vp, vp, i, vp, sz, vp]
    L.rtsvd_adjoint.argtypes = [vp, i, i, i, i, ctypes.POINTER(RtsvdParams), vp, i, vp, sz, vp]
    L.ttsvd_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(TtsvdParams), i]
    L.ttsvd_workspace_bytes.restype = sz
    L.ttsvd_solve.argtypes = [vp, vp, i, i, i, i, ctypes.POINTER(TtsvdParams), vp, vp, i, vp, sz, vp]
    L.tgkb_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(TgkbParams), i]
    L.tgkb_workspace_bytes.restype = sz
    L.tgkb_solve.argtypes = [vp, vp, i, i, i, i, ctypes.POINTER(TgkbParams), vp, vp, i, vp, sz, vp]
    L.nested_tgkb_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(TgkbParams), i]
    L.nested_tgkb_workspace_bytes.restype = sz
    L.nested_tgkb_solve.argtypes = [vp, vp, i, i, i, i, ctypes.POINTER(TgkbParams), vp, vp, i, vp, sz, vp]
    L.tgkb_triplets_workspace_bytes.argtypes = [i, i, i, i, i]
    L.tgkb_triplets_workspace_bytes.restype = sz
    L.tgkb_triplets.argtypes = [vp, vp, i, i, i, i, vp, vp, vp, i, vp, sz, vp]
    L.tgkb_tikhonov_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(TikParams), i]
    L.tgkb_tikhonov_workspace_bytes.restype = sz
    L.tgkb_tikhonov_solve.argtypes = [vp, vp, i, i, i, i, ctypes.POINTER(TikParams), vp, vp, i, vp, sz, vp]
    L.tgkb_tikhonov_solve_hat.argtypes = L.tgkb_tikhonov_solve.argtypes
    L.rtsvd_truncated_solve_hat.argtypes = L.rtsvd_truncated_solve.argtypes
    L.tgkb_solve_hat.argtypes = L.tgkb_solve.argtypes
    L.tp_status_string.argtypes = [i]
    L.tp_status_string.restype = ctypes.c_char_p
    L.tp_version.restype = i
    L.tp_kernel_launches.restype = i
    L.tp_timing_enable.argtypes = [i]
    L.tp_wait_budget.argtypes = [ctypes.c_longlong]
    L.tp_wait_budget.restype = i
    L.tp_wait_stall.argtypes = [i]
    L.tp_wait_stall.restype = i
    L.tp_timing_enable.restype = i
    L.tp_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), i]
    L.tp_timing_read.restype = i
    L.tprod_gemm_noalloc.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp]
    L.sep_operator.argtypes = [vp, vp, i, i, i, vp, i, vp]
    L.ttsvd_adjoint.argtypes = [vp, i, i, i, i, ctypes.POINTER(TtsvdParams), vp, i, vp, sz, vp]
    L.sep_grad_c_workspace_bytes.argtypes = [i, i, i, i]
    L.sep_grad_c_workspace_bytes.restype = sz
    L.sep_grad_c.argtypes = [vp, vp, vp, i, i, i, vp, i, vp, sz, vp]
    L.tgkb_tikhonov_grad_c_workspace_bytes.argtypes = [i, i, i, ctypes.POINTER(TikParams), i]
    L.tgkb_tikhonov_grad_c_workspace_bytes.restype = sz
    L.tgkb_tikhonov_grad_c.argtypes = [vp, vp, i, i, i, ctypes.POINTER(TikParams), vp, sz, vp, i, vp, sz, vp]
    L.tgkb_tikhonov_adjoint_workspace_bytes.argtypes = [i, i, i, ctypes.POINTER(TikParams), i]
    L.tgkb_tikhonov_adjoint_workspace_bytes.restype = sz
    L.tgkb_tikhonov_adjoint.argtypes = [vp, i, i, i, ctypes.POINTER(TikParams), vp, sz, vp, vp, i, vp, sz, vp]
    L.rtsvd_autotune.argtypes = [i, i, i, i, ctypes.POINTER(RtsvdParams), i, vp, sz, vp]
    L.tp_autotune_table.argtypes = [vp, vp, i]
    L.tp_autotune_table.restype = i
    L.tp_autotune_clear.argtypes = []
    L.tp_autotune_clear.restype = None
    L.tp_autotune_set.argtypes = [i, i, i, i, i, i, i]
    L.tp_autotune_set.restype = i
    L.tgkb_adjoint_workspace_bytes.argtypes = [i, i, i, ctypes.POINTER(TgkbParams), i]
    L.tgkb_adjoint_workspace_bytes.restype = sz
    L.tgkb_adjoint.argtypes = [vp, i, i, i, ctypes.POINTER(TgkbParams), vp, sz, vp, vp, i, vp, sz, vp]
    for f in ("tprod_fft", "tprod_ifft", "tprod_gemm", "rtsvd_truncated_solve", "tgkb_solve",
              "tgkb_tikhonov_solve", "rtsvd_truncated_solve_hat", "tgkb_solve_hat", "tgkb_tikhonov_solve_hat", "tprod_gemm_noalloc", "sep_grad_c", "tgkb_tikhonov_grad_c", "sep_operator",
              "ttsvd_adjoint", "tgkb_tikhonov_adjoint", "tgkb_adjoint", "rtsvd_autotune"):
        getattr(L, f).restype = i
    _lib = L
    return L


def status_string(st: int) -> str:
    return load().tp_status_string(int(st)).decode()


def kernel_launches() -> int:
    return int(load().tp_kernel_launches())


def wait_budget(cycles: int) -> None:
    """Bound (SM clock cycles) of the device-side waits for progress in later
    launches; 0 restores the defaults (about 1-2 s).  For failure-detection
    tests: a budget of a few cycles makes those waits run out on purpose."""
    _check("tp_wait_budget", load().tp_wait_budget(int(cycles)))


def wait_stall(on: bool) -> None:
    """With on, the grid-wide waits of the persistent tGKB kernels wait for an
    arrival that nothing makes, so each runs out after its budget
    (failure-detection tests; pair with a short wait_budget)."""
    _check("tp_wait_stall", load().tp_wait_stall(1 if on else 0))


def timing_enable(classes) -> None:
    """Bracket every later launch of the named kernel classes with CUDA events."""
    mask = 0
    for c in classes:
        mask |= 1 << KERNEL_CLASSES.index(c)
    load().tp_timing_enable(mask)


def timing_read() -> dict:
    """{class: (total device ms, launches)} since the last read; clears the record."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    rc = load().tp_timing_read(ms, cnt, n)
    if rc < 0:
        raise TprodError("tp_timing_read", rc)
    return {c: (ms[i], cnt[i]) for i, c in enumerate(KERNEL_CLASSES)}


def _check(fn: str, st: int):
    if st != TP_OK:
        raise TprodError(fn, st)


def _prec(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return TP_FP32
    if t.dtype == torch.float64:
        return TP_FP64
    raise TypeError(f"unsupported dtype {t.dtype} (float32 or float64)")


def _dev(*ts: torch.Tensor):
    for t in ts:
        if not t.is_cuda:
            raise TypeError("tprod works on CUDA tensors only (no CPU path)")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


class _Op:
    """The operator of a solve: the real tensor A (n, l, m) or its half
    spectrum A-hat (n/2+1, l, m) complex with n given (the *_hat entry
    points).  Shape, dtype and device as the solve needs them."""

    def __init__(self, A, Ahat, n):
        if (A is None) == (Ahat is None):
            raise ValueError("give exactly one of A and Ahat")
        if A is not None:
            _dev(A)
            self.t, self.hat = A, False
            self.n, self.l, self.m = A.shape
            self.dtype = A.dtype
        else:
            _dev(Ahat)
            if n is None or Ahat.shape[0] != int(n) // 2 + 1:
                raise ValueError("Ahat needs n with Ahat.shape[0] == n // 2 + 1")
            if Ahat.dtype not in (torch.complex64, torch.complex128):
                raise TypeError("Ahat must be complex64 or complex128")
            self.t, self.hat = Ahat, True
            self.n, (self.l, self.m) = int(n), Ahat.shape[1:]
            self.dtype = torch.float32 if Ahat.dtype == torch.complex64 else torch.float64
        self.device = self.t.device
        self.prec = TP_FP32 if self.dtype == torch.float32 else TP_FP64

    def entry(self, L, name):
        return getattr(L, name + "_hat") if self.hat else getattr(L, name)


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)


def _aligned(ws: torch.Tensor) -> tuple[ctypes.c_void_p, int]:
    p = ws.data_ptr()
    a = (p + 255) & ~255
    return ctypes.c_void_p(a), ws.numel() - (a - p)


def _cplx_dtype(t: torch.Tensor):
    return torch.complex64 if t.dtype == torch.float32 else torch.complex128


def fft(A: torch.Tensor) -> torch.Tensor:
    """Half-spectrum mode-3 DFT: A (n, l, m) real -> (n//2+1, l, m) complex."""
    _dev(A)
    n, l, m = A.shape
    out = torch.empty((n // 2 + 1, l, m), dtype=_cplx_dtype(A), device=A.device)
    _check("tprod_fft", load().tprod_fft(_ptr(A), l, m, n, _ptr(out), _prec(A), _stream()))
    return out


def ifft(Xh: torch.Tensor, n: int) -> torch.Tensor:
    """Inverse of fft: (n//2+1, l, m) complex -> (n, l, m) real."""
    _dev(Xh)
    h, l, m = Xh.shape
    if h != n // 2 + 1:
        raise ValueError("spectrum has the wrong number of slices for n")
    real = torch.float32 if Xh.dtype == torch.complex64 else torch.float64
    out = torch.empty((n, l, m), dtype=real, device=Xh.device)
    prec = TP_FP32 if real == torch.float32 else TP_FP64
    _check("tprod_ifft", load().tprod_ifft(_ptr(Xh), l, m, n, _ptr(out), prec, _stream()))
    return out


def tprod(A: torch.Tensor, B: torch.Tensor, transA: bool = False, tf32: bool = False,
          transB: bool = False) -> torch.Tensor:
    """t-product op(A) * op(B), op = the t-transpose when asked.  A (n, l, kk)
    [or (n, kk, l) with transA], B (n, kk, m) [or (n, m, kk) with transB].

    tf32=True (float32 only): the TP_TF32 precision form (one tf32 product on
    the tensor cores instead of the float32-accurate split)."""
    _dev(A, B)
    if A.dtype != B.dtype:
        raise TypeError("A and B must share a dtype")
    n, a1, a2 = A.shape
    nb, b1, b2 = B.shape
    l = a2 if transA else a1
    kk, m = (b2, b1) if transB else (b1, b2)
    if nb != n or (a1 if transA else a2) != kk:
        raise ValueError("shape mismatch")
    prec = _prec(A)
    if tf32:
        if prec != TP_FP32:
            raise TypeError("tf32 needs float32 tensors")
        prec = TP_TF32
    C = torch.empty((n, l, m), dtype=A.dtype, device=A.device)
    L = load()
    ws = _workspace(L.tprod_gemm_workspace_bytes(l, kk, m, n, prec), A.device)
    wp, wn = _aligned(ws)
    trans = int(bool(transA)) | (2 if transB else 0)
    _check("tprod_gemm", L.tprod_gemm(_ptr(A), _ptr(B), _ptr(C), l, kk, m, n, trans, prec, wp, wn, _stream()))
    return C


class Captured:
    """A sequence of this library's calls recorded once as a CUDA graph and
    replayed: the same kernels on the same buffers, without the per-launch
    host work and with shorter gaps between dependent kernels.  `fn` must
    enqueue only (sync=False calls) on fixed tensors; `outputs` holds what it
    returned during capture, rewritten by every replay.  Workspaces are
    allocated during capture from the graph's private pool and stay with it."""

    def __init__(self, fn, warmup: int = 2):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        n0 = kernel_launches()
        with torch.cuda.graph(self.graph):
            self.outputs = fn()
        self.launches = kernel_launches() - n0  # kernels of this library in one replay

    def replay(self):
        self.graph.replay()
        return self.outputs


class TProd(torch.autograd.Function):
    """C = A * B with the adjoint of the t-product as its backward:
    dL/dA = G * B^T and dL/dB = A^T * G (Section 2's t-transpose), both on the
    GPU through tprod_gemm."""

    @staticmethod
    def forward(ctx, A, B):
        ctx.save_for_backward(A, B)
        return tprod(A, B)

    @staticmethod
    def backward(ctx, G):
        A, B = ctx.saved_tensors
        G = G.contiguous()
        dA = tprod(G, B, transB=True) if ctx.needs_input_grad[0] else None
        dB = tprod(A, G, transA=True) if ctx.needs_input_grad[1] else None
        return dA, dB


def tprod_ad(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Differentiable t-product (torch.autograd)."""
    return TProd.apply(A, B)


def tprod_noalloc(A: torch.Tensor, B: torch.Tensor, transA: bool = False) -> torch.Tensor:
    """t-product computed in the library's fixed 16 MiB scratch (no workspace).

    For callers that cannot allocate device memory for a workspace; the output
    tensor is still the caller's.  Raises TprodError(TP_ERR_WORKSPACE) when
    the problem does not fit the scratch.
    """
    _dev(A, B)
    n, a1, a2 = A.shape
    nb, kk, m = B.shape
    l = a2 if transA else a1
    if nb != n or (a1 if transA else a2) != kk or A.dtype != B.dtype:
        raise ValueError("shape or dtype mismatch")
    C = torch.empty((n, l, m), dtype=A.dtype, device=A.device)
    _check("tprod_gemm_noalloc", load().tprod_gemm_noalloc(_ptr(A), _ptr(B), _ptr(C), l, kk, m, n, int(transA),
                                                           _prec(A), _stream()))
    return C


def _info_dict(buf: torch.Tensor) -> dict:
    raw = bytes(buf.cpu().numpy().tobytes())
    o = TpInfo.from_buffer_copy(raw[:ctypes.sizeof(TpInfo)])
    return {f: getattr(o, f) for f, _ in TpInfo._fields_}


def _info_list(buf: torch.Tensor, p: int) -> list:
    raw = bytes(buf.cpu().numpy().tobytes())
    sz = ctypes.sizeof(TpInfo)
    recs = [TpInfo.from_buffer_copy(raw[j * sz:(j + 1) * sz]) for j in range(p)]
    return [{f: getattr(o, f) for f, _ in TpInfo._fields_} for o in recs]


def _info_buf(device, count=1):
    return torch.zeros(count * ctypes.sizeof(TpInfo), dtype=torch.uint8, device=device)


class RtsvdFactor:
    """What rtsvd_solve(..., keep=True) leaves for rtsvd_adjoint: the solve's
    own workspace (factorisation and k) and its arguments."""

    def __init__(self, ws, P, hist, l, m, n, p, prec, device, dtype):
        self.ws, self.P, self.hist = ws, P, hist
        self.l, self.m, self.n, self.p = l, m, n, p
        self.prec, self.device, self.dtype = prec, device, dtype


def rtsvd_adjoint(fac: RtsvdFactor, G: torch.Tensor) -> torch.Tensor:
    """dL/dB = U_k S_k^{-1} V_k^T * G for the solve that made `fac` (k fixed)."""
    _dev(G)
    if tuple(G.shape) != (fac.n, fac.m, fac.p) or G.dtype != fac.dtype:
        raise ValueError("G must match the solution X of the solve")
    dB = torch.empty((fac.n, fac.l, fac.p), dtype=fac.dtype, device=fac.device)
    wp, wn = _aligned(fac.ws)
    _check("rtsvd_adjoint", load().rtsvd_adjoint(_ptr(G), fac.l, fac.m, fac.n, fac.p, ctypes.byref(fac.P), _ptr(dB),
                                                 fac.prec, wp, wn, _stream()))
    return dB


def rtsvd_solve(A, B, Omega, delta, tau, p_over, block=16, q_power=1, r_max=None, eps=0.0, eps_rel=0.0,
                res_hist=False, sync=True, tf32=False, keep=False, Ahat=None, n=None, bf16=False):
    """RT-tSVD method (Section 4.2).  Returns (X, info[, res_hist][, factor]).

    B is (n, l, p): p > 1 lateral slices share one factorisation and one k
    (problem (I6)).  tf32=True (float32 only): the TP_TF32 precision form of
    the block sketch and projection products.  keep=True also returns an
    RtsvdFactor for rtsvd_adjoint.  With A=None, Ahat (the half spectrum
    from fft(A)) and n: the rtsvd_truncated_solve_hat entry point.
    bf16=True (float32 only): the TP_BF16 form (sketch and power products on
    bfloat16 copies of A-hat)."""
    op = _Op(A, Ahat, n)
    _dev(B, Omega)
    n, l, m = op.n, op.l, op.m
    p = B.shape[2]
    r_max = min(l, m) if r_max is None else r_max
    prec = op.prec
    if tf32 and bf16:
        raise ValueError("tf32 and bf16 are two different forms")
    if tf32 or bf16:
        if prec != TP_FP32:
            raise TypeError("tf32 and bf16 need float32 tensors")
        prec = TP_TF32 if tf32 else TP_BF16
    X = torch.empty((n, m, p), dtype=op.dtype, device=op.device)
    hist = torch.empty(r_max + 1, dtype=torch.float64, device=op.device) if res_hist else None
    P = RtsvdParams(float(delta), float(tau), float(eps), float(eps_rel), int(p_over), int(q_power), int(block),
                    int(r_max), hist.data_ptr() if hist is not None else None)
    L = load()
    nb = L.rtsvd_workspace_bytes(l, m, n, p, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("rtsvd_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, op.device)
    wp, wn = _aligned(ws)
    info = _info_buf(op.device)
    _check("rtsvd_truncated_solve", op.entry(L, "rtsvd_truncated_solve")(
        _ptr(op.t), _ptr(B), _ptr(Omega), l, m, n, p, ctypes.byref(P), _ptr(X), _ptr(info), prec, wp, wn, _stream()))
    fac = (RtsvdFactor(ws, P, hist, l, m, n, p, prec, op.device, op.dtype),) if keep else ()
    if not sync:
        return (X, info, hist) + fac
    out = (X, _info_dict(info))
    return out + ((hist.cpu().numpy(),) if res_hist else ()) + fac


class RtsvdSolve(torch.autograd.Function):
    """X_k = RT-tSVD solution of A * X = B, differentiable in B with k held at
    the value the discrepancy principle chose (the adjoint is rtsvd_adjoint)."""

    @staticmethod
    def forward(ctx, B, A, Omega, kw):
        X, _, _, fac = rtsvd_solve(A, B, Omega, sync=False, keep=True, **kw)
        ctx.fac = fac
        return X

    @staticmethod
    def backward(ctx, G):
        return rtsvd_adjoint(ctx.fac, G.contiguous()), None, None, None


def rtsvd_solve_ad(A, B, Omega, delta, tau, p_over, **kw):
    """Differentiable (in B) RT-tSVD solve: returns X only."""
    return RtsvdSolve.apply(B, A, Omega, dict(delta=delta, tau=tau, p_over=p_over, **kw))


class TtsvdFactor:
    """What ttsvd_solve(..., keep=True) leaves for ttsvd_adjoint."""

    def __init__(self, ws, P, hist, l, m, n, p, prec, device, dtype):
        self.ws, self.P, self.hist = ws, P, hist
        self.l, self.m, self.n, self.p = l, m, n, p
        self.prec, self.device, self.dtype = prec, device, dtype


def ttsvd_adjoint(fac: TtsvdFactor, G: torch.Tensor) -> torch.Tensor:
    """dL/dB = U_s S_s^{-1} V_s^T * G for the T-tSVD solve that made `fac` (s fixed)."""
    _dev(G)
    if tuple(G.shape) != (fac.n, fac.m, fac.p) or G.dtype != fac.dtype:
        raise ValueError("G must match the solution X of the solve")
    dB = torch.empty((fac.n, fac.l, fac.p), dtype=fac.dtype, device=fac.device)
    wp, wn = _aligned(fac.ws)
    _check("ttsvd_adjoint", load().ttsvd_adjoint(_ptr(G), fac.l, fac.m, fac.n, fac.p, ctypes.byref(fac.P), _ptr(dB),
                                                 fac.prec, wp, wn, _stream()))
    return dB


def ttsvd_solve(A, B, delta, tau, res_hist=False, sync=True, keep=False):
    """T-tSVD method (Section 4.1).  Returns (X, info[, res_hist][, factor])."""
    _dev(A, B)
    n, l, m = A.shape
    p = B.shape[2]
    prec = _prec(A)
    X = torch.empty((n, m, p), dtype=A.dtype, device=A.device)
    hist = torch.empty(min(l, m) + 1, dtype=torch.float64, device=A.device) if res_hist else None
    P = TtsvdParams(float(delta), float(tau), hist.data_ptr() if hist is not None else None)
    L = load()
    nb = L.ttsvd_workspace_bytes(l, m, n, p, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("ttsvd_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, A.device)
    wp, wn = _aligned(ws)
    info = _info_buf(A.device)
    _check("ttsvd_solve", L.ttsvd_solve(_ptr(A), _ptr(B), l, m, n, p, ctypes.byref(P), _ptr(X), _ptr(info), prec, wp,
                                        wn, _stream()))
    fac = (TtsvdFactor(ws, P, hist, l, m, n, p, prec, A.device, A.dtype),) if keep else ()
    if not sync:
        return (X, info, hist) + fac
    out = (X, _info_dict(info))
    return out + ((hist.cpu().numpy(),) if res_hist else ()) + fac


def tgkb_solve(A, B, delta, tau, k_max, res_hist=False, sync=True, deltas=None, Ahat=None, n=None, keep=False):
    """tGKB method (Algorithm 4 + Eq. (solgkb)).  Returns (X, info[, res_hist][, factor]).

    B is (n, l, p); p > 1 is the tGKB_p method: every lateral slice j is
    solved on its own with bound deltas[j] (default: delta for all) and its own
    k_j; info is then a list of p records and res_hist a (p, k_max+1) array.
    With A=None, Ahat and n: the tgkb_solve_hat entry point.  keep=True (p = 1)
    also returns the solve's workspace for tgkb_adjoint."""
    op = _Op(A, Ahat, n)
    _dev(B)
    n, l, m = op.n, op.l, op.m
    p = B.shape[2]
    prec = op.prec
    X = torch.empty((n, m, p), dtype=op.dtype, device=op.device)
    hist = torch.empty((p, k_max + 1), dtype=torch.float64, device=op.device) if res_hist else None
    dp = None
    if deltas is not None:
        dl = [float(d) for d in deltas]
        if len(dl) != p:
            raise ValueError("deltas needs one bound per lateral slice")
        dp = (ctypes.c_double * p)(*dl)
    P = TgkbParams(float(delta), float(tau), int(k_max), hist.data_ptr() if hist is not None else None,
                   ctypes.cast(dp, ctypes.c_void_p) if dp is not None else None)
    L = load()
    nb = L.tgkb_workspace_bytes(l, m, n, p, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("tgkb_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, op.device)
    wp, wn = _aligned(ws)
    info = _info_buf(op.device, p)
    _check("tgkb_solve", op.entry(L, "tgkb_solve")(_ptr(op.t), _ptr(B), l, m, n, p, ctypes.byref(P), _ptr(X),
                                                   _ptr(info), prec, wp, wn, _stream()))
    if p == 1 and hist is not None:
        hist = hist[0]
    if keep and p != 1:
        raise ValueError("keep=True needs one lateral slice (tgkb_adjoint)")
    fac = (TgktFactor(ws, P, l, m, n, prec, op.device, op.dtype, op.t if op.hat else None),) if keep else ()
    if not sync:
        return (X, info, hist) + fac
    out = (X, _info_dict(info) if p == 1 else _info_list(info, p))
    return out + ((hist.cpu().numpy(),) if res_hist else ()) + fac


def nested_tgkb_solve(A, B, deltas, eta, k_max, res_hist=False, sync=True):
    """nested_tGKB_p (Algorithm 6): one Krylov basis from B[:, :, 0] serves
    every lateral slice in turn.  Returns (X, infos[, res_hist (p, k_max+1)])."""
    _dev(A, B)
    n, l, m = A.shape
    p = B.shape[2]
    prec = _prec(A)
    X = torch.empty((n, m, p), dtype=A.dtype, device=A.device)
    hist = torch.empty((p, k_max + 1), dtype=torch.float64, device=A.device) if res_hist else None
    dl = [float(d) for d in deltas]
    if len(dl) != p:
        raise ValueError("deltas needs one bound per lateral slice")
    dp = (ctypes.c_double * p)(*dl)
    P = TgkbParams(0.0, float(eta), int(k_max), hist.data_ptr() if hist is not None else None,
                   ctypes.cast(dp, ctypes.c_void_p))
    L = load()
    nb = L.nested_tgkb_workspace_bytes(l, m, n, p, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("nested_tgkb_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, A.device)
    wp, wn = _aligned(ws)
    info = _info_buf(A.device, p)
    _check("nested_tgkb_solve", L.nested_tgkb_solve(_ptr(A), _ptr(B), l, m, n, p, ctypes.byref(P), _ptr(X),
                                                    _ptr(info), prec, wp, wn, _stream()))
    if not sync:
        return X, info, hist
    out = (X, _info_list(info, p))
    return out + ((hist.cpu().numpy(),) if res_hist else ())


def tgkb_triplets(A, B, k):
    """t-singular triplets from k tGKB steps (Section 4.3): returns U (n, l, k),
    S (n, k) (tube i in column i), V (n, m, k)."""
    _dev(A, B)
    n, l, m = A.shape
    prec = _prec(A)
    U = torch.empty((n, l, k), dtype=A.dtype, device=A.device)
    S = torch.empty((n, k), dtype=A.dtype, device=A.device)
    V = torch.empty((n, m, k), dtype=A.dtype, device=A.device)
    L = load()
    nb = L.tgkb_triplets_workspace_bytes(l, m, n, int(k), prec)
    if nb == 0:
        raise TprodError("tgkb_triplets_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, A.device)
    wp, wn = _aligned(ws)
    _check("tgkb_triplets", L.tgkb_triplets(_ptr(A), _ptr(B), l, m, n, int(k), _ptr(U), _ptr(S), _ptr(V), prec, wp,
                                            wn, _stream()))
    return U, S, V


class TgktFactor:
    """What tgkt_solve(..., keep=True) leaves for tgkt_grad_c and
    tgkt_adjoint: the solve's workspace (A-hat, B-hat, basis, bidiagonal, k,
    mu, X-hat), its arguments, and the caller's A-hat when the solve was
    given one (None otherwise)."""

    def __init__(self, ws, P, l, m, n, prec, device, dtype, ahat=None):
        self.ws, self.P = ws, P
        self.l, self.m, self.n = l, m, n
        self.prec, self.device, self.dtype = prec, device, dtype
        self.ahat = ahat


def sep_operator(T: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """A(:,:,k) = c_k T, formed on the device: T (l, m) in the working
    precision, c float64 (n,).  Returns A (n, l, m)."""
    _dev(T, c)
    if T.dim() != 2 or c.dim() != 1 or c.dtype != torch.float64:
        raise ValueError("T must be (l, m) and c a float64 vector")
    l, m = T.shape
    n = c.shape[0]
    A = torch.empty((n, l, m), dtype=T.dtype, device=T.device)
    _check("sep_operator", load().sep_operator(_ptr(T), _ptr(c), l, m, n, _ptr(A), _prec(T), _stream()))
    return A


class SepRtsvdSolve(torch.autograd.Function):
    """X_k = RT-tSVD solution for the separable operator A(:,:,k) = c_k T,
    differentiable in B (rtsvd_adjoint) and in c (sep_grad_c), with k and the
    sketch rank held at the values the solve chose."""

    @staticmethod
    def forward(ctx, B, c, T, Omega, kw):
        A = sep_operator(T, c.detach())
        X, _, _, fac = rtsvd_solve(A, B, Omega, sync=False, keep=True, **kw)
        ctx.fac = fac
        ctx.save_for_backward(X, c)
        return X

    @staticmethod
    def backward(ctx, G):
        if ctx.needs_input_grad[2]:
            raise NotImplementedError("dL/dT is not provided")
        X, c = ctx.saved_tensors
        G = G.contiguous()
        dB = rtsvd_adjoint(ctx.fac, G) if ctx.needs_input_grad[0] else None
        dc = sep_grad_c(X, G, c.detach().contiguous()) if ctx.needs_input_grad[1] else None
        return dB, dc, None, None, None


def rtsvd_solve_sep_ad(c, T, B, Omega, delta, tau, p_over, **kw):
    """Differentiable (in B and c) RT-tSVD solve for A(:,:,k) = c_k T: returns X."""
    return SepRtsvdSolve.apply(B, c, T, Omega, dict(delta=delta, tau=tau, p_over=p_over, **kw))


class SepTgktSolve(torch.autograd.Function):
    """Tikhonov-tGKB solution for A(:,:,k) = c_k T, differentiable in B
    (tgkt_adjoint: the Krylov space moves with B) and in c (tgkt_grad_c),
    with k and mu held at the values the solve chose."""

    @staticmethod
    def forward(ctx, B, c, T, kw):
        A = sep_operator(T, c.detach())
        X, _, fac = tgkt_solve(A, B, sync=False, keep=True, **kw)
        ctx.fac = fac
        ctx.save_for_backward(c)
        return X

    @staticmethod
    def backward(ctx, G):
        if ctx.needs_input_grad[2]:
            raise NotImplementedError("dL/dT is not provided")
        (c,) = ctx.saved_tensors
        G = G.contiguous()
        dB = tgkt_adjoint(ctx.fac, G) if ctx.needs_input_grad[0] else None
        dc = tgkt_grad_c(ctx.fac, G, c.detach().contiguous()) if ctx.needs_input_grad[1] else None
        return dB, dc, None, None


def tgkt_solve_sep_ad(c, T, B, delta, tau, k_max, mu_lo, mu_hi, log_tol=1e-12):
    """Differentiable (in B and c) Tikhonov-tGKB solve for A(:,:,k) = c_k T: returns X."""
    return SepTgktSolve.apply(B, c, T, dict(delta=delta, tau=tau, k_max=k_max, mu_lo=mu_lo, mu_hi=mu_hi,
                                            log_tol=log_tol))


def sep_grad_c(X: torch.Tensor, G: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """dL/dc for a solution X (n, m, p) of a truncated solve (T-tSVD, RT-tSVD,
    tGKB, nested tGKB) with the separable operator A(:,:,k) = c_k T, at the
    solve's k, for G = dL/dX.  c: float64 CUDA tensor (n,).  Returns dc
    (float64, n)."""
    _dev(X, G, c)
    if tuple(G.shape) != tuple(X.shape) or G.dtype != X.dtype or c.dtype != torch.float64:
        raise ValueError("G must match X; c must be float64")
    n, m, p = X.shape
    if tuple(c.shape) != (n,):
        raise ValueError("c must hold n tube weights")
    prec = _prec(X)
    L = load()
    nb = L.sep_grad_c_workspace_bytes(m, n, p, prec)
    if nb == 0:
        raise TprodError("sep_grad_c_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, X.device)
    wp, wn = _aligned(ws)
    dc = torch.empty(n, dtype=torch.float64, device=X.device)
    _check("sep_grad_c", L.sep_grad_c(_ptr(X), _ptr(G), _ptr(c), m, n, p, _ptr(dc), prec, wp, wn, _stream()))
    return dc


def tgkt_grad_c(fac: "TgktFactor", G: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """dL/dc for the Tikhonov-tGKB solution that made `fac` (k and mu fixed),
    operator A(:,:,k) = c_k T, for G = dL/dX (n, m, 1).  Returns dc (float64, n)."""
    _dev(G, c)
    if tuple(G.shape) != (fac.n, fac.m, 1) or G.dtype != fac.dtype or c.dtype != torch.float64:
        raise ValueError("G must match the solution X of the solve; c must be float64")
    if tuple(c.shape) != (fac.n,):
        raise ValueError("c must hold n tube weights")
    L = load()
    nb = L.tgkb_tikhonov_grad_c_workspace_bytes(fac.l, fac.m, fac.n, ctypes.byref(fac.P), fac.prec)
    if nb == 0:
        raise TprodError("tgkb_tikhonov_grad_c_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, G.device)
    wp, wn = _aligned(ws)
    sp, sn = _aligned(fac.ws)
    dc = torch.empty(fac.n, dtype=torch.float64, device=G.device)
    _check("tgkb_tikhonov_grad_c", L.tgkb_tikhonov_grad_c(_ptr(G), _ptr(c), fac.l, fac.m, fac.n, ctypes.byref(fac.P),
                                                          sp, sn, _ptr(dc), fac.prec, wp, wn, _stream()))
    return dc


def tgkt_adjoint(fac: "TgktFactor", G: torch.Tensor) -> torch.Tensor:
    """dL/dB of the Tikhonov-tGKB solution that made `fac` (k and mu held at
    the solve's values; the Krylov space moves with B) for G = dL/dX (n, m,
    1): the reverse sweep through the solve's tGKB steps.  Returns dB (n, l, 1)."""
    _dev(G)
    if tuple(G.shape) != (fac.n, fac.m, 1) or G.dtype != fac.dtype:
        raise ValueError("G must match the solution X of the solve")
    G = G.contiguous()
    L = load()
    nb = L.tgkb_tikhonov_adjoint_workspace_bytes(fac.l, fac.m, fac.n, ctypes.byref(fac.P), fac.prec)
    if nb == 0:
        raise TprodError("tgkb_tikhonov_adjoint_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, G.device)
    wp, wn = _aligned(ws)
    sp, sn = _aligned(fac.ws)
    dB = torch.empty((fac.n, fac.l, 1), dtype=fac.dtype, device=G.device)
    _check("tgkb_tikhonov_adjoint", L.tgkb_tikhonov_adjoint(_ptr(G), fac.l, fac.m, fac.n, ctypes.byref(fac.P), sp, sn,
                                                            _ptr(fac.ahat), _ptr(dB), fac.prec, wp, wn, _stream()))
    return dB


_FORMS = {"fp32": TP_FP32, "tf32": TP_TF32, "bf16": TP_BF16, "fp64": TP_FP64}


def rtsvd_autotune(n, l, m, p=1, block=16, r_max=160, form="fp32", device="cuda") -> list:
    """Pick the stage counts of the tensor-core products that an rtsvd_solve
    of these sizes and form (fp32, tf32, bf16; fp64 tunes nothing) launches,
    by timing each candidate (rtsvd_autotune; synchronises the stream).  Later
    solves of these shapes use the choices; results do not change.  Returns
    the whole table (autotune_table)."""
    prec = _FORMS[form]
    P = RtsvdParams(1.0, 1.1, 0.1, 0.0, 1, 1, int(block), int(r_max), None)
    L = load()
    nb = L.rtsvd_workspace_bytes(l, m, n, p, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("rtsvd_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, torch.device(device))
    wp, wn = _aligned(ws)
    _check("rtsvd_autotune", L.rtsvd_autotune(l, m, n, p, ctypes.byref(P), prec, wp, wn, _stream()))
    return autotune_table()


def autotune_table() -> list:
    """The tuner's table: one dict per tuned product shape."""
    L = load()
    cap = 256
    ints = (ctypes.c_int * (8 * cap))()
    flts = (ctypes.c_float * (2 * cap))()
    cnt = L.tp_autotune_table(ctypes.cast(ints, ctypes.c_void_p), ctypes.cast(flts, ctypes.c_void_p), cap)
    ops = {0: "A", 2: "conj(A)", 3: "A^H"}
    forms = {3: "fp32", 1: "tf32", 0: "bf16"}
    return [{"op": ops.get(ints[8 * k], ints[8 * k]), "form": forms.get(ints[8 * k + 1], ints[8 * k + 1]),
             "columns": ints[8 * k + 2], "M": ints[8 * k + 3], "K": ints[8 * k + 4], "batch": ints[8 * k + 5],
             "stages": ints[8 * k + 6], "stages_default": ints[8 * k + 7], "ms": flts[2 * k],
             "ms_default": flts[2 * k + 1]} for k in range(cnt)]


def autotune_clear() -> None:
    """Every product shape back to the built-in stage-count rule."""
    load().tp_autotune_clear()


def autotune_set(op: int, form: str, columns: int, M: int, K: int, batch: int, stages: int) -> None:
    """Put one product shape's stage count into the table (op 0: A, 2: conj(A)
    from the transposed copy, 3: A^H)."""
    passes = {"fp32": 3, "tf32": 1, "bf16": 0}[form]
    _check("tp_autotune_set", load().tp_autotune_set(op, passes, columns, M, K, batch, stages))


def tgkb_adjoint(fac: "TgktFactor", G: torch.Tensor) -> torch.Tensor:
    """dL/dB of the single-slice tGKB solution that made `fac` (k held at the
    solve's value; the Krylov space moves with B) for G = dL/dX (n, m, 1).
    Returns dB (n, l, 1)."""
    _dev(G)
    if tuple(G.shape) != (fac.n, fac.m, 1) or G.dtype != fac.dtype:
        raise ValueError("G must match the solution X of the solve")
    G = G.contiguous()
    L = load()
    nb = L.tgkb_adjoint_workspace_bytes(fac.l, fac.m, fac.n, ctypes.byref(fac.P), fac.prec)
    if nb == 0:
        raise TprodError("tgkb_adjoint_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, G.device)
    wp, wn = _aligned(ws)
    sp, sn = _aligned(fac.ws)
    dB = torch.empty((fac.n, fac.l, 1), dtype=fac.dtype, device=G.device)
    _check("tgkb_adjoint", L.tgkb_adjoint(_ptr(G), fac.l, fac.m, fac.n, ctypes.byref(fac.P), sp, sn, _ptr(fac.ahat),
                                          _ptr(dB), fac.prec, wp, wn, _stream()))
    return dB


class TgkbSolve(torch.autograd.Function):
    """X = tGKB solution (one lateral slice), differentiable in B with k held
    at the value the solve chose (tgkb_adjoint); A is a constant."""

    @staticmethod
    def forward(ctx, B, A, kw):
        X, _, _, fac = tgkb_solve(A, B, sync=False, keep=True, **kw)
        ctx.fac = fac
        return X

    @staticmethod
    def backward(ctx, G):
        if ctx.needs_input_grad[1]:
            raise NotImplementedError("dL/dA is not provided")
        return tgkb_adjoint(ctx.fac, G.contiguous()), None, None


class TgktSolve(torch.autograd.Function):
    """X = Tikhonov-tGKB solution, differentiable in B with k and mu held at
    the values the solve chose (tgkt_adjoint); A is a constant."""

    @staticmethod
    def forward(ctx, B, A, kw):
        X, _, fac = tgkt_solve(A, B, sync=False, keep=True, **kw)
        ctx.fac = fac
        return X

    @staticmethod
    def backward(ctx, G):
        if ctx.needs_input_grad[1]:
            raise NotImplementedError("dL/dA is not provided")
        return tgkt_adjoint(ctx.fac, G.contiguous()), None, None


def tgkb_solve_ad(A, B, delta, tau, k_max):
    """Differentiable (in B) tGKB solve of one lateral slice: returns X."""
    return TgkbSolve.apply(B, A, dict(delta=delta, tau=tau, k_max=k_max))


def tgkt_solve_ad(A, B, delta, tau, k_max, mu_lo, mu_hi, log_tol=1e-12):
    """Differentiable (in B) Tikhonov-tGKB solve: returns X."""
    return TgktSolve.apply(B, A, dict(delta=delta, tau=tau, k_max=k_max, mu_lo=mu_lo, mu_hi=mu_hi, log_tol=log_tol))


def tgkt_solve(A, B, delta, tau, k_max, mu_lo, mu_hi, log_tol=1e-12, sync=True, keep=False, Ahat=None, n=None):
    """Tikhonov-tGKB (Section 5).  Returns (X, info[, factor]); keep=True also
    returns the solve's workspace for tgkt_grad_c.  With A=None, Ahat and n:
    the tgkb_tikhonov_solve_hat entry point."""
    op = _Op(A, Ahat, n)
    _dev(B)
    n, l, m = op.n, op.l, op.m
    prec = op.prec
    X = torch.empty((n, m, 1), dtype=op.dtype, device=op.device)
    P = TikParams(TgkbParams(float(delta), float(tau), int(k_max), None), float(mu_lo), float(mu_hi),
                  float(log_tol))
    L = load()
    nb = L.tgkb_tikhonov_workspace_bytes(l, m, n, 1, ctypes.byref(P), prec)
    if nb == 0:
        raise TprodError("tgkb_tikhonov_workspace_bytes", TP_ERR_ARG)
    ws = _workspace(nb, op.device)
    wp, wn = _aligned(ws)
    info = _info_buf(op.device)
    _check("tgkb_tikhonov_solve", op.entry(L, "tgkb_tikhonov_solve")(
        _ptr(op.t), _ptr(B), l, m, n, 1, ctypes.byref(P), _ptr(X), _ptr(info), prec, wp, wn, _stream()))
    if keep:
        fac = TgktFactor(ws, P, l, m, n, prec, op.device, op.dtype, op.t if op.hat else None)
        return (X, info, fac) if not sync else (X, _info_dict(info), fac)
    if not sync:
        return X, info
    return X, _info_dict(info)
