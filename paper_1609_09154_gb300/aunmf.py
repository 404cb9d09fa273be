"""Thin ctypes binding of libaunmf (include/aunmf.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device pointers and the
current torch CUDA stream is passed as the library's stream.  Every step of
the method runs in the library's CUDA kernels; there is no Python or CPU
fallback -- if the shared library is missing or fails to load, import-time
use raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MU, HALS, ABPP = 0, 1, 2
FP32, TF32, BF16 = 0, 1, 2
ALGOS = {"mu": MU, "hals": HALS, "abpp": ABPP}
PRECS = {"fp32": FP32, "tf32": TF32, "bf16": BF16}
K_MAX, BPP_K_MAX = 512, 64

OK, E_INVAL, E_NOMEM, E_CUDA, E_NUMERIC, E_NOCONVERGE, E_TIMEOUT, E_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
INJECT_NONE, INJECT_TC_WAIT, INJECT_GRID_BARRIER, INJECT_NOMEM, INJECT_SIMT_WAIT = 0, 1, 2, 3, 4


class AunmfError(RuntimeError):
    """A non-zero status.  For whole runs (run, run_batched) the library has
    still written its outputs; they are attached as `result`
    (W, H, relres, info) when available."""

    def __init__(self, code, msg, result=None):
        super().__init__(msg)
        self.code = code
        self.result = result


class Matrix(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64),
        ("dense", ctypes.c_void_p), ("lda", ctypes.c_int64),
        ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p),
        ("nnz", ctypes.c_int64),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int), ("mu_eps", ctypes.c_double), ("bpp_max_pivots", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("profile", ctypes.c_int),
        ("hals_variant", ctypes.c_int), ("stop_tol", ctypes.c_double),
        ("validate", ctypes.c_int), ("bpp_cold_start", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("bpp_pivots", ctypes.c_int64), ("bpp_nonconverged", ctypes.c_int64),
        ("bpp_numeric", ctypes.c_int64), ("iters_done", ctypes.c_int),
        ("ms_total", ctypes.c_float),
        ("ms_aht", ctypes.c_float), ("ms_wta", ctypes.c_float), ("ms_update", ctypes.c_float),
        ("ms_gram", ctypes.c_float), ("ms_other", ctypes.c_float),
        ("n_aht", ctypes.c_int), ("n_wta", ctypes.c_int), ("launches", ctypes.c_int64),
        ("tuned_bpp_warps", ctypes.c_int), ("tuned_bpp_rows", ctypes.c_int),
        ("bpp_redone", ctypes.c_int64),
        ("pgrad_first", ctypes.c_double), ("pgrad_last", ctypes.c_double),
        ("tuned_gemm_stages_aht", ctypes.c_int), ("tuned_gemm_stages_wta", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P, _I64, _I, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_MP, _OP, _IP = ctypes.POINTER(Matrix), ctypes.POINTER(Options), ctypes.POINTER(Info)

# name -> argtypes (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "aunmf_create": [ctypes.POINTER(_P), _P],
    "aunmf_set_stream": [_P, _P],
    "aunmf_destroy": [_P],
    "aunmf_strerror": [_I],
    "aunmf_last_cuda_error": [_P],
    "aunmf_run": [_P, _MP, _I, _I, _I, _P, _P, _P, _P, _P, _OP, _IP],
    "aunmf_run_host": [_P, _P, _I64, _I64, _I64, _I, _I, _I, _P, _P, _P, _P, _P, _OP, _IP],
    "aunmf_gram_w": [_P, _P, _I64, _I, _P],
    "aunmf_gram_h": [_P, _P, _I, _I64, _P],
    "aunmf_aht": [_P, _MP, _P, _I, _I, _P],
    "aunmf_wta": [_P, _MP, _P, _I, _I, _P],
    "aunmf_update_w": [_P, _I, _P, _P, _P, _I64, _I, _P, _I64, _D],
    "aunmf_update_h": [_P, _I, _P, _P, _P, _I, _I64, _D],
    "aunmf_nls_bpp": [_P, _P, _P, _I64, _I, _P, _I, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "aunmf_relres": [_P, _MP, _P, _P, _I, ctypes.POINTER(_D)],
    "aunmf_gram_w_noalloc": [_P, _I64, _I, _P, _P],
    "aunmf_test_inject": [_I, _D],
    "aunmf_check_status": [_P],
    "aunmf_probe_gather": [_P, _I64, _P, _I64, _I, _I64, _P, _P],
    "aunmf_loss_fwd": [_P, _MP, _I, _P, _P, _I, _P, _P],
    "aunmf_run_batched": [_P, _I, _MP, _P, _I, _I, _P, _P, _P, _P, _P, _OP, _IP],
    "aunmf_loss_bwd": [_P, _MP, _I, _P, _P, _I, _P, _P, _P, _P],
}
_RESTYPE = {"aunmf_strerror": ctypes.c_char_p, "aunmf_last_cuda_error": ctypes.c_char_p}

_libs = {}


def lib_path(checked: bool = False) -> str:
    return _build.LIB_CHECK if checked else _build.LIB


def load(build_if_missing: bool = True, checked: bool = False):
    """Load libaunmf.so, or with checked=True the bounds-checked variant
    libaunmf_check.so (building it first if allowed and missing)."""
    if checked in _libs:
        return _libs[checked]
    path = lib_path(checked)
    if build_if_missing and not _build.up_to_date(checked):
        _build.build(check=checked)
    if not os.path.exists(path):
        raise RuntimeError(f"libaunmf not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _RESTYPE.get(name, ctypes.c_int)
    _libs[checked] = L
    return L


def check_status(checked: bool = True) -> int:
    """aunmf_check_status of the given library: the first bounds-check site
    recorded since the last call (0 = none; -1 = a build without checks)."""
    site = ctypes.c_int(0)
    rc = load(checked=checked).aunmf_check_status(ctypes.byref(site))
    if rc != OK:
        raise AunmfError(rc, strerror(rc))
    return site.value


def strerror(code: int) -> str:
    return load().aunmf_strerror(code).decode()


def probe_gather(idx, X, k, sink, stream=None):
    """aunmf_probe_gather (a measurement, not a step of the method): enqueue
    the gather-roof kernel that loads row idx[e] of X for every e, on
    `stream` (default: torch's current stream).  idx: int32 CUDA tensor; X:
    rows x ld float32 CUDA tensor (ld % 4 == 0) whose first k columns are the
    factor; sink: one float32 on the device."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = load().aunmf_probe_gather(_ptr(idx), idx.numel(), _ptr(X), X.shape[0], k, X.stride(0),
                                   _ptr(sink), ctypes.c_void_p(s.cuda_stream))
    if rc != OK:
        raise AunmfError(rc, strerror(rc))


def test_inject(site: int, wait_ms: float = 0.0) -> int:
    """aunmf_test_inject: make one kind of bounded device wait run out (test
    support; INJECT_NONE restores normal operation).  Returns the status."""
    return load().aunmf_test_inject(site, wait_ms)


# ---------------------------------------------------------------- helpers
def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_dev(*ts):
    torch = _torch()
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("libaunmf entry points take CUDA tensors")
        if t.dtype != torch.float32 and t.dtype not in (torch.int64, torch.int32):
            raise ValueError(f"unexpected dtype {t.dtype}")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def dense_matrix(A) -> Matrix:
    _check_dev(A)
    m, n = A.shape
    return Matrix(m, n, A.data_ptr(), A.stride(0), None, None, None, 0)


def csr_matrix(rowptr, colidx, val, shape) -> Matrix:
    _check_dev(rowptr, colidx, val)
    m, n = shape
    return Matrix(m, n, None, 0, rowptr.data_ptr(), colidx.data_ptr(), val.data_ptr(),
                  int(val.numel()))


class Handle:
    """Owns an aunmf_handle bound to torch's current CUDA stream."""

    def __init__(self, stream=None, checked=False):
        torch = _torch()
        self._lib = load(checked=checked)
        s = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        self._check(self._lib.aunmf_create(ctypes.byref(self._h), ctypes.c_void_p(s.cuda_stream)))

    def _check(self, rc, allow=(), result=None):
        if rc != OK and rc not in allow:
            msg = strerror(rc)
            if rc == E_CUDA and getattr(self, "_h", None):
                msg += ": " + self._lib.aunmf_last_cuda_error(self._h).decode()
            raise AunmfError(rc, msg, result)
        return rc

    def set_stream(self, stream):
        self._check(self._lib.aunmf_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.aunmf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- whole runs
    def run(self, A, k, algo, iters, W0, H0, *, prec="fp32", mu_eps=0.0, bpp_max_pivots=0,
            use_graph=True, profile=False, out=None, allow_noconverge=False, hals_variant=0,
            stop_tol=0.0, validate=False, bpp_cold_start=False):
        """Alg. 1 on device tensors.  A: dense (m x n) tensor or a Matrix
        (e.g. from csr_matrix).  hals_variant 1: Eq. halsupdate as printed;
        stop_tol > 0: stop on the projected gradient; validate: check A, W0,
        H0 (and a CSR's structure) first; bpp_cold_start: every BPP solve
        from x = 0.  Returns (W, H, relres ndarray of info["iters_done"]
        entries, info dict)."""
        torch = _torch()
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        algo = ALGOS[algo] if isinstance(algo, str) else algo
        prec = PRECS[prec] if isinstance(prec, str) else prec
        _check_dev(W0, H0)
        dev = H0.device
        if out is None:
            W = torch.empty((M.m, k), device=dev, dtype=torch.float32)
            H = torch.empty((k, M.n), device=dev, dtype=torch.float32)
        else:
            W, H = out
        rel = np.zeros(max(iters, 1), dtype=np.float64)
        opt = Options(prec, mu_eps, bpp_max_pivots, int(use_graph), int(profile),
                      int(hals_variant), float(stop_tol), int(validate), int(bpp_cold_start))
        info = Info()
        rc = self._lib.aunmf_run(self._h, ctypes.byref(M), k, algo, iters, _ptr(W0), _ptr(H0),
                                 _ptr(W), _ptr(H), rel.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(opt), ctypes.byref(info))
        done = info.iters_done if rc in (OK, E_NOCONVERGE) else iters
        result = (W, H, rel[:done], info.as_dict())
        self._check(rc, allow=(E_NOCONVERGE,) if allow_noconverge else (), result=result)
        return result

    def run_batched(self, As, ks, iters, H0s, *, prec="tf32", use_graph=True, bpp_max_pivots=0,
                    allow_noconverge=False, validate=False, bpp_cold_start=False):
        """ABPP on many problems at once (lists of dense CUDA tensors A_p, ranks
        k_p, initial H0_p).  Returns (Ws, Hs, relres ndarray count x iters, info)."""
        torch = _torch()
        count = len(As)
        mats = (Matrix * count)(*[dense_matrix(A) for A in As])
        karr = (ctypes.c_int * count)(*ks)
        Ws = [torch.empty((A.shape[0], k), device=A.device, dtype=torch.float32)
              for A, k in zip(As, ks)]
        Hs = [torch.empty((k, A.shape[1]), device=A.device, dtype=torch.float32)
              for A, k in zip(As, ks)]
        _check_dev(*H0s)
        parr = lambda ts: (ctypes.c_void_p * count)(*[t.data_ptr() for t in ts])  # noqa: E731
        rel = np.zeros((count, max(iters, 1)), dtype=np.float64)
        prec = PRECS[prec] if isinstance(prec, str) else prec
        opt = Options(prec, 0.0, bpp_max_pivots, int(use_graph), 0, 0, 0.0, int(validate),
                      int(bpp_cold_start))
        info = Info()
        rc = self._lib.aunmf_run_batched(self._h, count, mats, karr, ABPP, iters, None,
                                         parr(H0s), parr(Ws), parr(Hs),
                                         rel.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opt),
                                         ctypes.byref(info))
        result = (Ws, Hs, rel[:, :iters], info.as_dict())
        self._check(rc, allow=(E_NOCONVERGE,) if allow_noconverge else (), result=result)
        return result

    def run_host(self, A, k, algo, iters, W0, H0, *, prec="fp32", use_graph=True,
                 profile=False, W=None, H=None, validate=False):
        """Alg. 1 with host (numpy float32) arrays; copies happen inside."""
        A = np.ascontiguousarray(A, dtype=np.float32) if not isinstance(A, np.ndarray) else A
        m, n = A.shape
        algo = ALGOS[algo] if isinstance(algo, str) else algo
        prec = PRECS[prec] if isinstance(prec, str) else prec
        W = np.empty((m, k), np.float32) if W is None else W
        H = np.empty((k, n), np.float32) if H is None else H
        rel = np.zeros(max(iters, 1), dtype=np.float64)
        opt = Options(prec, 0.0, 0, int(use_graph), int(profile), 0, 0.0, int(validate))
        info = Info()
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None  # noqa: E731
        rc = self._lib.aunmf_run_host(self._h, vp(A), m, n, A.strides[0] // 4, k, algo, iters,
                                      vp(W0), vp(H0), vp(W), vp(H), vp(rel), ctypes.byref(opt),
                                      ctypes.byref(info))
        self._check(rc)
        return W, H, rel[:iters], info.as_dict()

    # ---------------------------------------------------------- single steps
    def gram_w(self, W):
        torch = _torch()
        _check_dev(W)
        m, k = W.shape
        G = torch.empty((k, k), device=W.device, dtype=torch.float32)
        self._check(self._lib.aunmf_gram_w(self._h, _ptr(W), m, k, _ptr(G)))
        return G

    def gram_h(self, H):
        torch = _torch()
        _check_dev(H)
        k, n = H.shape
        G = torch.empty((k, k), device=H.device, dtype=torch.float32)
        self._check(self._lib.aunmf_gram_h(self._h, _ptr(H), k, n, _ptr(G)))
        return G

    def aht(self, A, H, prec="fp32"):
        torch = _torch()
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        _check_dev(H)
        k = H.shape[0]
        P = torch.empty((M.m, k), device=H.device, dtype=torch.float32)
        prec = PRECS[prec] if isinstance(prec, str) else prec
        self._check(self._lib.aunmf_aht(self._h, ctypes.byref(M), _ptr(H), k, prec, _ptr(P)))
        return P

    def wta(self, A, W, prec="fp32"):
        torch = _torch()
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        _check_dev(W)
        k = W.shape[1]
        P = torch.empty((k, M.n), device=W.device, dtype=torch.float32)
        prec = PRECS[prec] if isinstance(prec, str) else prec
        self._check(self._lib.aunmf_wta(self._h, ctypes.byref(M), _ptr(W), k, prec, _ptr(P)))
        return P

    def update_w(self, algo, W, PW, GH, H=None, eps=0.0):
        """In place on W (and H's rows for HALS)."""
        _check_dev(W, PW, GH, H)
        algo = ALGOS[algo] if isinstance(algo, str) else algo
        m, k = W.shape
        n = H.shape[1] if H is not None else 0
        self._check(self._lib.aunmf_update_w(self._h, algo, _ptr(W), _ptr(PW), _ptr(GH), m, k,
                                             _ptr(H), n, eps))
        return W, H

    def update_h(self, algo, H, PH, GW, eps=0.0):
        _check_dev(H, PH, GW)
        algo = ALGOS[algo] if isinstance(algo, str) else algo
        k, n = H.shape
        self._check(self._lib.aunmf_update_h(self._h, algo, _ptr(H), _ptr(PH), _ptr(GW), k, n,
                                             eps))
        return H

    def nls_bpp(self, G, R, max_pivots=0):
        """Rows of R (nrhs x k) against G (k x k).  Returns (X, pivots, nonconv)."""
        torch = _torch()
        _check_dev(G, R)
        nrhs, k = R.shape
        X = torch.empty_like(R)
        piv, nc = ctypes.c_int64(0), ctypes.c_int64(0)
        rc = self._lib.aunmf_nls_bpp(self._h, _ptr(G), _ptr(R), nrhs, k, _ptr(X), max_pivots,
                                     ctypes.byref(piv), ctypes.byref(nc))
        self._check(rc, allow=(E_NOCONVERGE,))
        return X, piv.value, nc.value

    def loss_fwd(self, A, W, H, prec="fp32", save_wta=True):
        """Returns (loss as a 0-dim float64 CUDA tensor, W^T A or None)."""
        torch = _torch()
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        _check_dev(W, H)
        k = W.shape[1]
        prec = PRECS[prec] if isinstance(prec, str) else prec
        loss = torch.empty((), device=W.device, dtype=torch.float64)
        wta = torch.empty((k, M.n), device=W.device, dtype=torch.float32) if save_wta else None
        self._check(self._lib.aunmf_loss_fwd(self._h, ctypes.byref(M), k, _ptr(W), _ptr(H), prec,
                                             _ptr(loss), _ptr(wta)))
        return loss, wta

    def loss_bwd(self, A, W, H, grad_out=None, wta=None, prec="fp32", need_w=True, need_h=True):
        """Returns (dW, dH); grad_out is a 1-element float32 CUDA tensor or None."""
        torch = _torch()
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        _check_dev(W, H, wta, grad_out)
        k = W.shape[1]
        prec = PRECS[prec] if isinstance(prec, str) else prec
        dW = torch.empty_like(W) if need_w else None
        dH = torch.empty_like(H) if need_h else None
        self._check(self._lib.aunmf_loss_bwd(self._h, ctypes.byref(M), k, _ptr(W), _ptr(H), prec,
                                             _ptr(wta), _ptr(grad_out), _ptr(dW), _ptr(dH)))
        return dW, dH

    def relres(self, A, W, H):
        M = A if isinstance(A, Matrix) else dense_matrix(A)
        _check_dev(W, H)
        out = ctypes.c_double(0.0)
        self._check(self._lib.aunmf_relres(self._h, ctypes.byref(M), _ptr(W), _ptr(H),
                                           W.shape[1], ctypes.byref(out)))
        return out.value
