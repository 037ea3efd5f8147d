"""GB300 (sm_103a) mixed precision Gram-matrix thin SVD -- Python binding.

A thin ctypes layer over ``libtsvd.so`` (the C ABI in ``include/tsvd.h``):
the functions below have the C names and only marshal arguments.  Every step
of the method runs in the library's CUDA kernels; there is no CPU fallback,
and importing a function fails loudly if the library has not been built
(``python -m paper_2603_11953_gb300.build``).

Pointers may be given as torch tensors (their ``data_ptr()`` is used), as
integers, or as None for optional outputs.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsvd.so")

TSVD_FP32, TSVD_FP64, TSVD_DD = 0, 1, 2
(TSVD_OK, TSVD_ERR_ARG, TSVD_ERR_ALIGN, TSVD_ERR_NONFINITE, TSVD_ERR_NOT_FULL_RANK,
 TSVD_ERR_NO_CONVERGENCE, TSVD_ERR_TIMEOUT, TSVD_ERR_UNSUPPORTED, TSVD_ERR_CUDA,
 TSVD_ERR_ALLOC) = range(10)

EXPORTED = ["tsvd_create", "tsvd_destroy", "tsvd_status_string", "tsvd_gram", "tsvd_eig",
            "tsvd_solve", "tsvd_batch_solve", "tsvd_sync_status", "tsvd_last_stage_ms",
            "tsvd_stage_ms_mean", "tsvd_gram_static", "tsvd_gram_colexp", "tsvd_gram_partial",
            "tsvd_gram_finish", "tsvd_solve_gram", "tsvd_cholqr", "tsvd_autotune_choice"]


class tsvd_opts(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int), ("chunk_rows", ctypes.c_int), ("split_k", ctypes.c_int),
                ("jacobi_tol", ctypes.c_double), ("max_sweeps", ctypes.c_int),
                ("eig_variant", ctypes.c_int), ("autotune", ctypes.c_int),
                ("timeout_cycles", ctypes.c_longlong), ("gram_variant", ctypes.c_int),
                ("timing", ctypes.c_int), ("u_variant", ctypes.c_int), ("fixed_scale", ctypes.c_int)]


class tsvd_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_int), ("off_norm", ctypes.c_double),
                ("kappa_B", ctypes.c_double)]


class TsvdError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {tsvd_status_string(status)} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtsvd.so (raises OSError if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise OSError(f"libtsvd.so not built at {path}; run python -m paper_2603_11953_gb300.build")
        lib = ctypes.CDLL(path)
        P, I64, I32, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_double
        lib.tsvd_create.argtypes = [ctypes.POINTER(P), I, P, ctypes.POINTER(tsvd_opts)]
        lib.tsvd_destroy.argtypes = [P]
        lib.tsvd_status_string.argtypes = [I]
        lib.tsvd_status_string.restype = ctypes.c_char_p
        lib.tsvd_gram.argtypes = [P, P, I64, I64, I64, I, I, P, I64]
        lib.tsvd_eig.argtypes = [P, P, I64, I64, P, P, I64, P]
        lib.tsvd_solve.argtypes = [P, P, I64, I64, I64, I, I, P, P, I64, P, I64, P]
        lib.tsvd_batch_solve.argtypes = [P, I32, P, P, P, P, I, I, P, P, P, P, P, P]
        lib.tsvd_sync_status.argtypes = [P]
        lib.tsvd_last_stage_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
        lib.tsvd_gram_static.argtypes = [P, I64, I64, I64, I, I, P, I64, P, P]
        lib.tsvd_gram_colexp.argtypes = [P, P, I64, I64, I64, I, P]
        lib.tsvd_gram_partial.argtypes = [P, P, I64, I64, I64, I, P, P]
        lib.tsvd_gram_finish.argtypes = [P, P, P, I64, I, P, I64]
        lib.tsvd_solve_gram.argtypes = [P, P, I64, P, I64, I64, I64, I, I, P, P, I64, P, I64, P]
        lib.tsvd_cholqr.argtypes = [P, P, I64, I64, I64, I, I, P, I64, P, I64, P]
        for name in EXPORTED:
            if name != "tsvd_status_string":
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _p(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, ctypes.Array) or isinstance(x, ctypes.Structure):
        return ctypes.cast(ctypes.pointer(x), ctypes.c_void_p)
    return ctypes.c_void_p(int(x))


def _check(fn, status):
    if status != TSVD_OK:
        raise TsvdError(fn, status)
    return status


def tsvd_status_string(status: int) -> str:
    return load_library().tsvd_status_string(int(status)).decode()


def tsvd_create(device: int = 0, stream=None, opts: tsvd_opts | None = None, check=True):
    """Returns (handle, status).  stream: a cudaStream_t as int (e.g.
    torch.cuda.current_stream().cuda_stream) or None for the default stream."""
    lib = load_library()
    h = ctypes.c_void_p()
    st = lib.tsvd_create(ctypes.byref(h), int(device), None if stream is None else ctypes.c_void_p(int(stream)),
                         None if opts is None else ctypes.byref(opts))
    if check:
        _check("tsvd_create", st)
    return h, st


def tsvd_destroy(h):
    return load_library().tsvd_destroy(h)


def tsvd_gram(h, A, m, n, lda, working, higher, G, ldg, check=True):
    st = load_library().tsvd_gram(h, _p(A), int(m), int(n), int(lda), int(working), int(higher), _p(G), int(ldg))
    return _check("tsvd_gram", st) if check else st


def tsvd_eig(h, M, n, ldm, lam, V, ldv, info=None, check=True):
    st = load_library().tsvd_eig(h, _p(M), int(n), int(ldm), _p(lam), _p(V), int(ldv), _p(info))
    return _check("tsvd_eig", st) if check else st


def tsvd_solve(h, A, m, n, lda, working, higher, sigma, V, ldv, U=None, ldu=0, info=None, check=True):
    st = load_library().tsvd_solve(h, _p(A), int(m), int(n), int(lda), int(working), int(higher), _p(sigma),
                                   _p(V), int(ldv), _p(U), int(ldu), _p(info))
    return _check("tsvd_solve", st) if check else st


def tsvd_batch_solve(h, count, A, m, n, lda, working, higher, sigma, V, ldv, U=None, ldu=None,
                     info=None, check=True):
    """A, sigma, V, U: sequences of device pointers (tensors or ints); m, n,
    lda, ldv, ldu: sequences of ints (marshalled into host arrays)."""
    def ptrs(seq):
        if seq is None:
            return None
        arr = (ctypes.c_void_p * count)(*[None if x is None else (x.data_ptr() if hasattr(x, "data_ptr") else int(x))
                                          for x in seq])
        return arr

    def ints(seq):
        return None if seq is None else (ctypes.c_int64 * count)(*[int(v) for v in seq])

    arrs = [ptrs(A), ints(m), ints(n), ints(lda), ptrs(sigma), ptrs(V), ints(ldv), ptrs(U), ints(ldu)]
    cast = [None if a is None else ctypes.cast(a, ctypes.c_void_p) for a in arrs]
    st = load_library().tsvd_batch_solve(h, int(count), cast[0], cast[1], cast[2], cast[3], int(working),
                                         int(higher), cast[4], cast[5], cast[6], cast[7], cast[8], _p(info))
    return _check("tsvd_batch_solve", st) if check else st


def tsvd_gram_static(A, m, n, lda, working, higher, G, ldg, info=None, stream=None, check=True):
    """Allocation-free Gram (no handle): see include/tsvd.h."""
    st = load_library().tsvd_gram_static(_p(A), int(m), int(n), int(lda), int(working), int(higher), _p(G),
                                         int(ldg), _p(info), None if stream is None else ctypes.c_void_p(int(stream)))
    return _check("tsvd_gram_static", st) if check else st


def tsvd_sync_status(h) -> int:
    return load_library().tsvd_sync_status(h)


def tsvd_last_stage_ms(h):
    out = (ctypes.c_float * 4)()
    _check("tsvd_last_stage_ms", load_library().tsvd_last_stage_ms(h, out))
    return list(out)


def tsvd_stage_ms_mean(h, last):
    out = (ctypes.c_float * 4)()
    _check("tsvd_stage_ms_mean", load_library().tsvd_stage_ms_mean(h, int(last), out))
    return list(out)


def tsvd_gram_colexp(h, A, m, n, lda, working, E, check=True):
    """Row-sharded Gram, step 1: E[j] = least e with max |a_rj| < 2^e over these rows."""
    st = load_library().tsvd_gram_colexp(h, _p(A), int(m), int(n), int(lda), int(working), _p(E))
    return _check("tsvd_gram_colexp", st) if check else st


def tsvd_gram_partial(h, A, m, n, lda, working, E, limbs, check=True):
    """Row-sharded Gram, step 3: these rows' exact part of A^T A as 4 x n x n int64 limbs."""
    st = load_library().tsvd_gram_partial(h, _p(A), int(m), int(n), int(lda), int(working), _p(E), _p(limbs))
    return _check("tsvd_gram_partial", st) if check else st


def tsvd_gram_finish(h, limbs, E, n, higher, G, ldg, check=True):
    """Row-sharded Gram, step 5: the (rank-summed) limbs rounded once to G."""
    st = load_library().tsvd_gram_finish(h, _p(limbs), _p(E), int(n), int(higher), _p(G), int(ldg))
    return _check("tsvd_gram_finish", st) if check else st


def tsvd_solve_gram(h, G, ldg, A, m, n, lda, working, higher, sigma, V, ldv, U=None, ldu=0, info=None, check=True):
    """Alg. 1 lines 3-6 on a given Gram matrix G, with U for the given rows of A."""
    st = load_library().tsvd_solve_gram(h, _p(G), int(ldg), _p(A), int(m), int(n), int(lda), int(working),
                                        int(higher), _p(sigma), _p(V), int(ldv), _p(U), int(ldu), _p(info))
    return _check("tsvd_solve_gram", st) if check else st


def tsvd_cholqr(h, A, m, n, lda, working, higher, Q, ldq, R=None, ldr=0, info=None, check=True):
    """Mixed precision Cholesky QR: A = Q R (Gram and Cholesky in FP64, Q R = A solved in FP32)."""
    st = load_library().tsvd_cholqr(h, _p(A), int(m), int(n), int(lda), int(working), int(higher), _p(Q), int(ldq),
                                    _p(R), int(ldr), _p(info))
    return _check("tsvd_cholqr", st) if check else st


def tsvd_autotune_choice(h, m, n, working):
    """The autotuner's choice for a shape: (split_k, u_variant, gram_ms, u_ms), or None."""
    sk, uv = ctypes.c_int32(0), ctypes.c_int32(0)
    gm, um = ctypes.c_float(0.0), ctypes.c_float(0.0)
    st = load_library().tsvd_autotune_choice(h, int(m), int(n), int(working), ctypes.byref(sk), ctypes.byref(uv),
                                             ctypes.byref(gm), ctypes.byref(um))
    return (sk.value, uv.value, gm.value, um.value) if st == TSVD_OK else None
