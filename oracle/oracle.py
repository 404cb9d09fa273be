"""FP64 CPU oracle for alternating-updating NMF -- Python wrapper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It loads ``aunmf_oracle.c`` (plain C, double precision, built with
gcc) and shares nothing with the CUDA library: no code, no header, no helper.

Function map (paper sections / equations):
  gram_w, gram_h              Alg. 1 lines 3-4 (Gram matrices W^T W, H H^T)
  aht, wta                    Alg. 1 lines 3-4 (products A H^T, W^T A; dense or CSR)
  mu_update_w, mu_update_h    Sec. 4.1, Eq. (muupdate)
  hals_update_w, hals_update_h  Sec. 4.2, Eq. (halsupdate), readings R2/R3
  hals_update_w_printed, hals_update_h_printed  Eq. (halsupdate) as printed, R9
  pgrad                       Sec. 6.2, projected gradient norm, reading R10
  bpp_solve, bpp_update_w/h   Sec. 4.3, Eqs. (single NLS), (KKT); SolveBPP
  relres_direct, relres_trace Sec. 6.2 (relative error ||A-WH||/||A||)
  loss_grad                   0.5||A-WH||^2 and its gradient from R = WH - A
  nmf_run                     Alg. 1 driver (HALS variant, projected-gradient stop)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

MU, HALS, ABPP = 0, 1, 2
ALGOS = {"mu": MU, "hals": HALS, "abpp": ABPP}

OK, E_INVAL, E_NOMEM, E_NUMERIC, E_NOCONVERGE = 0, -1, -2, -4, -5

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aunmf_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile aunmf_oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _OUT)
    return _OUT


class _Mat(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("dense", ctypes.c_void_p),
        ("rowptr", ctypes.c_void_p),
        ("colidx", ctypes.c_void_p),
        ("val", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "or_num_threads": (I, []),
                "or_gram_w": (None, [P, I64, I, P]),
                "or_gram_h": (None, [P, I, I64, P]),
                "or_aht": (None, [P, P, I, P]),
                "or_wta": (None, [P, P, I, P]),
                "or_mu_update_w": (None, [P, P, P, I64, I, D]),
                "or_mu_update_h": (None, [P, P, P, I, I64, D]),
                "or_hals_update_w": (None, [P, P, P, I64, I, P, I64]),
                "or_hals_update_h": (None, [P, P, P, I, I64]),
                "or_hals_update_w_printed": (None, [P, P, P, I64, I]),
                "or_hals_update_h_printed": (None, [P, P, P, I, I64]),
                "or_pgrad2": (D, [P, P, P, P, P, P, I64, I64, I]),
                "or_bpp_solve": (I, [P, P, I, P, I]),
                "or_bpp_update_w": (I64, [P, P, P, I64, I, I]),
                "or_bpp_update_h": (I64, [P, P, P, I, I64, I]),
                "or_norm2_a": (D, [P]),
                "or_resid2_direct": (D, [P, P, P, I]),
                "or_relres_direct": (D, [P, P, P, I]),
                "or_relres_trace": (D, [D, P, P, P, P, I, I64]),
                "or_loss_grad": (D, [P, P, P, I, P, P]),
                "or_grad_w_row": (None, [P, P, P, I, I64, P]),
                "or_grad_h_col": (None, [P, P, P, I, I64, P]),
                "or_nmf_run": (I, [P, I, I, I, P, P, P, P, P, D, I, P]),
                "or_nmf_run_ex": (I, [P, I, I, I, P, P, P, P, P, D, I, P, I, D, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def _d(a) -> np.ndarray:
    """C-contiguous float64 copy/view."""
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class Matrix:
    """Dense (m x n ndarray) or CSR (indptr, indices, data, shape) input in FP64.

    Holds references to the arrays so the C side sees live memory."""

    def __init__(self, A=None, *, csr=None, shape=None):
        if A is not None:
            self.dense = _d(A)
            self.m, self.n = self.dense.shape
            self._keep = [self.dense]
            self.s = _Mat(self.m, self.n, _p(self.dense), None, None, None)
            self.sparse = False
        else:
            indptr, indices, data = csr
            self.rowptr = np.ascontiguousarray(indptr, dtype=np.int64)
            self.colidx = np.ascontiguousarray(indices, dtype=np.int32)
            self.val = _d(data)
            self.m, self.n = shape
            self._keep = [self.rowptr, self.colidx, self.val]
            self.s = _Mat(self.m, self.n, None, _p(self.rowptr), _p(self.colidx), _p(self.val))
            self.sparse = True

    @property
    def ptr(self):
        return ctypes.byref(self.s)


def as_matrix(A) -> Matrix:
    if isinstance(A, Matrix):
        return A
    if hasattr(A, "indptr"):  # scipy.sparse csr
        return Matrix(csr=(A.indptr, A.indices, A.data), shape=A.shape)
    return Matrix(A)


# ---------------------------------------------------------------- kernels
def gram_w(W):
    W = _d(W)
    m, k = W.shape
    G = np.empty((k, k))
    lib().or_gram_w(_p(W), m, k, _p(G))
    return G


def gram_h(H):
    H = _d(H)
    k, n = H.shape
    G = np.empty((k, k))
    lib().or_gram_h(_p(H), k, n, _p(G))
    return G


def aht(A, H):
    A = as_matrix(A)
    H = _d(H)
    k = H.shape[0]
    P = np.empty((A.m, k))
    lib().or_aht(A.ptr, _p(H), k, _p(P))
    return P


def wta(A, W):
    A = as_matrix(A)
    W = _d(W)
    k = W.shape[1]
    P = np.empty((k, A.n))
    lib().or_wta(A.ptr, _p(W), k, _p(P))
    return P


def mu_update_w(W, PW, GH, eps=1e-16):
    W = _d(W).copy()
    m, k = W.shape
    lib().or_mu_update_w(_p(W), _p(_d(PW)), _p(_d(GH)), m, k, eps)
    return W


def mu_update_h(H, PH, GW, eps=1e-16):
    H = _d(H).copy()
    k, n = H.shape
    lib().or_mu_update_h(_p(H), _p(_d(PH)), _p(_d(GW)), k, n, eps)
    return H


def hals_update_w(W, PW, GH, H=None):
    """Returns (W', H') -- H' is H with rows scaled by the column norms of W'
    (reading R3), or None when H is None."""
    W = _d(W).copy()
    m, k = W.shape
    if H is not None:
        H = _d(H).copy()
        lib().or_hals_update_w(_p(W), _p(_d(PW)), _p(_d(GH)), m, k, _p(H), H.shape[1])
    else:
        lib().or_hals_update_w(_p(W), _p(_d(PW)), _p(_d(GH)), m, k, None, 0)
    return W, H


def hals_update_h(H, PH, GW):
    H = _d(H).copy()
    k, n = H.shape
    lib().or_hals_update_h(_p(H), _p(_d(PH)), _p(_d(GW)), k, n)
    return H


def hals_update_w_printed(W, PW, GH):
    """Eq. (halsupdate) as printed (reading R9): no division by (H H^T)_ii,
    each column normalised before the next is updated, H untouched."""
    W = _d(W).copy()
    m, k = W.shape
    lib().or_hals_update_w_printed(_p(W), _p(_d(PW)), _p(_d(GH)), m, k)
    return W


def hals_update_h_printed(H, PH, GW):
    H = _d(H).copy()
    k, n = H.shape
    lib().or_hals_update_h_printed(_p(H), _p(_d(PH)), _p(_d(GW)), k, n)
    return H


def pgrad(W, H, GH, PW, GW, PH):
    """Norm of the projected gradient of 0.5 ||A - WH||^2 at (W, H) from its
    four products (reading R10)."""
    W, H = _d(W), _d(H)
    m, k = W.shape
    n = H.shape[1]
    return float(np.sqrt(lib().or_pgrad2(_p(W), _p(H), _p(_d(GH)), _p(_d(PW)), _p(_d(GW)),
                                         _p(_d(PH)), m, n, k)))


def bpp_solve(G, r, max_iter=None):
    """x = argmin_{x>=0} ||Cx - b|| from G = C^T C, r = C^T b.  Returns (x, rc)
    where rc >= 0 is the number of exchanges, < 0 an error code."""
    G = _d(G)
    r = _d(r)
    k = r.shape[0]
    x = np.empty(k)
    rc = lib().or_bpp_solve(_p(G), _p(r), k, _p(x), 10 * k if max_iter is None else max_iter)
    return x, rc


def bpp_update_w(PW, GH, max_iter=None):
    PW = _d(PW)
    m, k = PW.shape
    W = np.empty((m, k))
    rc = lib().or_bpp_update_w(_p(W), _p(PW), _p(_d(GH)), m, k, 10 * k if max_iter is None else max_iter)
    return W, rc


def bpp_update_h(PH, GW, max_iter=None):
    PH = _d(PH)
    k, n = PH.shape
    H = np.empty((k, n))
    rc = lib().or_bpp_update_h(_p(H), _p(PH), _p(_d(GW)), k, n, 10 * k if max_iter is None else max_iter)
    return H, rc


def norm2_a(A):
    return float(lib().or_norm2_a(as_matrix(A).ptr))


def relres_direct(A, W, H):
    W, H = _d(W), _d(H)
    return float(lib().or_relres_direct(as_matrix(A).ptr, _p(W), _p(H), W.shape[1]))


def relres_trace(norm2a, PH, H, GW, GH):
    PH, H, GW, GH = _d(PH), _d(H), _d(GW), _d(GH)
    k, n = H.shape
    return float(lib().or_relres_trace(norm2a, _p(PH), _p(H), _p(GW), _p(GH), k, n))


def loss_grad(A, W, H):
    A = as_matrix(A)
    W, H = _d(W), _d(H)
    k = W.shape[1]
    dW = np.empty_like(W)
    dH = np.empty_like(H)
    loss = lib().or_loss_grad(A.ptr, _p(W), _p(H), k, _p(dW), _p(dH))
    return float(loss), dW, dH


def grad_w_rows(A, W, H, rows):
    """Rows `rows` of dL/dW for dense A (large-matrix checks)."""
    A = as_matrix(A)
    W, H = _d(W), _d(H)
    k = W.shape[1]
    out = np.empty((len(rows), k))
    for t, r in enumerate(rows):
        row = np.empty(k)
        lib().or_grad_w_row(A.ptr, _p(W), _p(H), k, int(r), _p(row))
        out[t] = row
    return out


def grad_h_cols(A, W, H, cols):
    """Columns `cols` of dL/dH (as rows of the result) for dense A."""
    A = as_matrix(A)
    W, H = _d(W), _d(H)
    k = W.shape[1]
    out = np.empty((len(cols), k))
    for t, c in enumerate(cols):
        col = np.empty(k)
        lib().or_grad_h_col(A.ptr, _p(W), _p(H), k, int(c), _p(col))
        out[t] = col
    return out


def resid2(A, W, H):
    """||A - W H||_F^2 entry by entry."""
    W, H = _d(W), _d(H)
    return float(lib().or_resid2_direct(as_matrix(A).ptr, _p(W), _p(H), W.shape[1]))


def nmf_run(A, k, algo, iters, W0, H0, mu_eps=1e-16, bpp_max_iter=None, hals_variant=0,
            stop_tol=0.0, track_pgrad=False):
    """Alg. 1 from (W0, H0).  Returns dict(W, H, relres, rc, pivots, iters_done,
    pgrad); relres and pgrad hold iters_done entries (pgrad None unless
    tracked: track_pgrad or stop_tol > 0)."""
    A = as_matrix(A)
    algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    W0 = _d(W0) if W0 is not None else np.zeros((A.m, k))
    H0 = _d(H0)
    W = np.empty((A.m, k))
    H = np.empty((k, A.n))
    rel = np.zeros(iters)
    pg = np.zeros(iters) if (track_pgrad or stop_tol > 0) else None
    piv = ctypes.c_int64(0)
    done = ctypes.c_int(0)
    rc = lib().or_nmf_run_ex(
        A.ptr, k, algo, iters, _p(W0), _p(H0), _p(W), _p(H), _p(rel), mu_eps,
        10 * k if bpp_max_iter is None else bpp_max_iter, ctypes.byref(piv), int(hals_variant),
        float(stop_tol), _p(pg) if pg is not None else None, ctypes.byref(done),
    )
    d = int(done.value)
    return {"W": W, "H": H, "relres": rel[:d], "rc": int(rc), "pivots": int(piv.value),
            "iters_done": d, "pgrad": pg[:d] if pg is not None else None}
