"""CPU oracle for the mixed precision Gram-matrix thin SVD (arXiv 2603.11953).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only code
allowed to import this package.  It shares nothing with the CUDA path.

The arithmetic lives in ``tsvd_oracle.c`` (plain C, single thread, built with
gcc); this module only compiles it and marshals numpy arrays through ctypes.

Functions (all matrices column-major, numpy ``order='F'``):
  gram(A)                        -> (G_hi, G_lo, G_abs)   exact A^T A (Alg. 1 l.1-2)
  jacobi_fp64(M, tol, sweeps)    -> (lam, V, sweeps, status)   (Alg. 1 l.3, FP64)
  jacobi_dd(M_hi, M_lo, ...)     -> (lam_hi, lam_lo, V_hi, V_lo, sweeps, status)
  sort_sign(lam_hi, lam_lo, V_hi, V_lo) -> (sig_hi, sig_lo, V_hi, V_lo, status)
  svd(A, higher)                 -> dict with sigma_h, V_h, sigma_w, V_w, W_w, status
  rows_times(A, W, rows, p)      -> RN_p of exact A[rows] @ W        (Alg. 1 l.6)
  rows_explicit_u(A, V_hi, V_lo, sig_hi, sig_lo, rows) -> exact A V_h / sigma_h (DD)
  round_dd(hi, lo, p)            -> RN_p(hi + lo) by one exact rounding (Alg. 1 l.4-5)
  alg2(M, working)               -> Algorithm 2: FP64 Cholesky, cast R, SVD of R (sigma, V)
  cholesky(M)                    -> R, plain FP64 Cholesky M = R^T R (Cholesky QR, step 2)
  cholqr_rows(A, Rw, rows, p)    -> RN_p of the solutions q of q Rw = a for the given rows (step 3)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsvd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtsvd_oracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_FULL_RANK, NO_CONVERGENCE, BAD_ARG, NONFINITE = 0, 1, 2, 3, 4
U_H_FP64 = 2.0 ** -53
U_H_DD = 2.0 ** -104


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_gram.argtypes = [P, I64, I64, I64, I, P, P, P]
            lib.oracle_rows_times.argtypes = [P, I64, I64, I64, I, P, I64, P, I64, I, P]
            lib.oracle_rows_explicit_u.argtypes = [P, I64, I64, I64, I, P, P, P, P, P, I64, P, P]
            lib.oracle_jacobi_fp64.argtypes = [P, I, D, I, P, P, P]
            lib.oracle_jacobi_dd.argtypes = [P, P, I, D, I, P, P, P, P, P]
            lib.oracle_sort_sign.argtypes = [I, P, P, P, P, P, P]
            lib.oracle_svd.argtypes = [P, I64, I64, I64, I, I, D, I, P, P, P, P, P, P, P, P]
            lib.oracle_round_dd.argtypes = [P, P, I64, I, P]
            lib.oracle_alg2.argtypes = [P, I, I, D, I, P, P, P]
            lib.oracle_cholesky.argtypes = [P, I, P]
            lib.oracle_cholqr_rows.argtypes = [P, I64, I64, I64, I, P, P, I64, I, P]
            for f in (lib.oracle_gram, lib.oracle_rows_times, lib.oracle_rows_explicit_u,
                      lib.oracle_jacobi_fp64, lib.oracle_jacobi_dd, lib.oracle_sort_sign,
                      lib.oracle_svd, lib.oracle_round_dd, lib.oracle_alg2, lib.oracle_cholesky,
                      lib.oracle_cholqr_rows):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _as_input(A):
    A = np.asarray(A)
    if A.dtype == np.float32:
        working = 0
    elif A.dtype == np.float64:
        working = 1
    else:
        raise TypeError("A must be float32 or float64")
    A = np.asfortranarray(A)
    m, n = A.shape
    return A, m, n, max(m, 1), working


def gram(A):
    """Exact Gram M = A^T A: (G_hi, G_lo, G_abs), each n x n float64."""
    lib = _load()
    A, m, n, lda, working = _as_input(A)
    Gh = np.zeros((n, n), order="F")
    Gl = np.zeros((n, n), order="F")
    Ga = np.zeros((n, n), order="F")
    st = lib.oracle_gram(_ptr(A), m, n, lda, working, _ptr(Gh), _ptr(Gl), _ptr(Ga))
    if st != OK:
        raise ValueError(f"oracle_gram status {st}")
    return Gh, Gl, Ga


def rows_times(A, W, rows, p):
    """RN_p(exact A[rows, :] @ W) with p significant bits (24: FP32, 53: FP64)."""
    lib = _load()
    A, m, n, lda, working = _as_input(A)
    W = np.asfortranarray(np.asarray(W, dtype=np.float64))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), n), order="F")
    st = lib.oracle_rows_times(_ptr(A), m, n, lda, working, _ptr(W), W.shape[0], _ptr(rows),
                               len(rows), int(p), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_rows_times status {st}")
    return out


def rows_explicit_u(A, V_hi, V_lo, sig_hi, sig_lo, rows):
    """Explicit U rows = (exact A[rows] V_h) / sigma_h, as double-double (hi, lo)."""
    lib = _load()
    A, m, n, lda, working = _as_input(A)
    V_hi = np.asfortranarray(np.asarray(V_hi, dtype=np.float64))
    V_lo = None if V_lo is None else np.asfortranarray(np.asarray(V_lo, dtype=np.float64))
    sig_hi = np.ascontiguousarray(np.asarray(sig_hi, dtype=np.float64))
    sig_lo = None if sig_lo is None else np.ascontiguousarray(np.asarray(sig_lo, dtype=np.float64))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    oh = np.zeros((len(rows), n), order="F")
    ol = np.zeros((len(rows), n), order="F")
    st = lib.oracle_rows_explicit_u(_ptr(A), m, n, lda, working, _ptr(V_hi), _ptr(V_lo),
                                    _ptr(sig_hi), _ptr(sig_lo), _ptr(rows), len(rows),
                                    _ptr(oh), _ptr(ol))
    if st != OK:
        raise ValueError(f"oracle_rows_explicit_u status {st}")
    return oh, ol


def round_dd(hi, lo, p):
    """RN-even of the exact values hi + lo to p significant bits (p <= 53), one rounding."""
    lib = _load()
    hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float64)).ravel()
    lo = None if lo is None else np.ascontiguousarray(np.asarray(lo, dtype=np.float64)).ravel()
    out = np.zeros_like(hi)
    st = lib.oracle_round_dd(_ptr(hi), _ptr(lo), hi.size, int(p), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_round_dd status {st}")
    return out


def alg2(M, working=0, tol=None, max_sweeps=100):
    """Algorithm 2 on M (n x n): FP64 Cholesky M = R^T R, R cast to the working precision
    (working 0: FP32, 1: FP64), SVD of that R to FP64 accuracy.  Returns dict(sigma, V, status,
    sweeps), sigma descending, V with the sign rule.  tol defaults to n 2^-53: a one-sided Jacobi
    recomputes x_p^T x_q from the columns, whose rounding (~sqrt(n) 2^-53 of ||x_p|| ||x_q||)
    a smaller skip threshold could never get below."""
    lib = _load()
    M = np.array(M, dtype=np.float64, order="F", copy=True)
    n = M.shape[0]
    if tol is None:
        tol = n * U_H_FP64
    sig = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sw = ctypes.c_int(0)
    st = lib.oracle_alg2(_ptr(M), n, int(working), float(tol), int(max_sweeps), _ptr(sig), _ptr(V),
                         ctypes.byref(sw))
    return dict(sigma=sig, V=V, status=st, sweeps=sw.value)


def cholesky(M):
    """Plain FP64 Cholesky M = R^T R: (R upper triangular, status)."""
    lib = _load()
    M = np.array(M, dtype=np.float64, order="F", copy=True)
    n = M.shape[0]
    R = np.zeros((n, n), order="F")
    st = lib.oracle_cholesky(_ptr(M), n, _ptr(R))
    return R, st


def cholqr_rows(A, Rw, rows, p):
    """RN_p of q = a Rw^-1 for the given rows a of A (double-double forward substitution)."""
    lib = _load()
    A, m, n, lda, working = _as_input(A)
    Rw = np.asfortranarray(np.asarray(Rw, dtype=np.float64))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), n), order="F")
    st = lib.oracle_cholqr_rows(_ptr(A), m, n, lda, working, _ptr(Rw), _ptr(rows), len(rows), int(p), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_cholqr_rows status {st}")
    return out


def jacobi_fp64(M, tol=U_H_FP64, max_sweeps=100):
    """Two-sided cyclic Jacobi on symmetric M (FP64).  Returns lam, V, sweeps, status."""
    lib = _load()
    M = np.array(M, dtype=np.float64, order="F", copy=True)
    n = M.shape[0]
    lam = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sw = ctypes.c_int(0)
    st = lib.oracle_jacobi_fp64(_ptr(M), n, float(tol), int(max_sweeps), _ptr(lam), _ptr(V),
                                ctypes.byref(sw))
    return lam, V, sw.value, st


def jacobi_dd(M_hi, M_lo, tol=U_H_DD, max_sweeps=100):
    """Two-sided cyclic Jacobi in double-double.  Returns lam_hi, lam_lo, V_hi, V_lo, sweeps, status."""
    lib = _load()
    Mh = np.array(M_hi, dtype=np.float64, order="F", copy=True)
    Ml = np.array(M_lo, dtype=np.float64, order="F", copy=True)
    n = Mh.shape[0]
    lh, ll = np.zeros(n), np.zeros(n)
    Vh = np.zeros((n, n), order="F")
    Vl = np.zeros((n, n), order="F")
    sw = ctypes.c_int(0)
    st = lib.oracle_jacobi_dd(_ptr(Mh), _ptr(Ml), n, float(tol), int(max_sweeps), _ptr(lh), _ptr(ll),
                              _ptr(Vh), _ptr(Vl), ctypes.byref(sw))
    return lh, ll, Vh, Vl, sw.value, st


def sort_sign(lam_hi, lam_lo, V_hi, V_lo):
    lib = _load()
    lh = np.array(lam_hi, dtype=np.float64, copy=True)
    n = lh.shape[0]
    ll = np.zeros(n) if lam_lo is None else np.array(lam_lo, dtype=np.float64, copy=True)
    Vh = np.array(V_hi, dtype=np.float64, order="F", copy=True)
    Vl = np.zeros((n, n), order="F") if V_lo is None else np.array(V_lo, dtype=np.float64, order="F", copy=True)
    sh, sl = np.zeros(n), np.zeros(n)
    st = lib.oracle_sort_sign(n, _ptr(lh), _ptr(ll), _ptr(Vh), _ptr(Vl), _ptr(sh), _ptr(sl))
    return sh, sl, Vh, Vl, st


def svd(A, higher=1, tol=None, max_sweeps=100):
    """Algorithm 1 end to end (without U).  higher: 1 = FP64, 2 = double-double.

    Returns dict(status, sweeps, sigma_h, sigma_h_lo, V_h, V_h_lo, sigma_w, V_w, W_w)
    where *_w are rounded to A's precision (returned as float64 arrays holding
    working-precision values) and W_w = RN_w(V_w / sigma_w) column by column.
    """
    lib = _load()
    A, m, n, lda, working = _as_input(A)
    if tol is None:
        tol = U_H_FP64 if higher == 1 else U_H_DD
    sh, sl, sw_, = np.zeros(n), np.zeros(n), np.zeros(n)
    Vh = np.zeros((n, n), order="F")
    Vl = np.zeros((n, n), order="F")
    Vw = np.zeros((n, n), order="F")
    Ww = np.zeros((n, n), order="F")
    sweeps = ctypes.c_int(0)
    st = lib.oracle_svd(_ptr(A), m, n, lda, working, int(higher), float(tol), int(max_sweeps),
                        _ptr(sh), _ptr(sl), _ptr(Vh), _ptr(Vl), _ptr(sw_), _ptr(Vw), _ptr(Ww),
                        ctypes.byref(sweeps))
    return dict(status=st, sweeps=sweeps.value, sigma_h=sh, sigma_h_lo=sl, V_h=Vh, V_h_lo=Vl,
                sigma_w=sw_, V_w=Vw, W_w=Ww, working=working)
