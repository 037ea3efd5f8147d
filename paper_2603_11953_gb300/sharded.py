"""Row-sharded Algorithm 1 over ``torch.distributed`` (Sec. 4.2.1 of the paper).

The rows of A are split over the ranks (one GPU each).  Every rank forms its
part of A^T A, one global reduction combines the parts, every rank then runs
the n x n stage on the same Gram matrix and computes its own rows of U.  Here
the reduction is made exact and order-free (include/tsvd.h, "Row-sharded
Gram"): an all-reduce MAX of the column exponents, then an all-reduce SUM of
each rank's Gram as 32-bit integer limbs, rounded once at the end; the result
is bitwise the same for any number of ranks and any split of the rows.

Only the steps' plumbing lives here; every step of the arithmetic runs in the
library's kernels (``LibraryOps``).  ``ops`` can be replaced (tests do, with a
CPU model of the integer arithmetic) to exercise the exchange on CPU ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import (TSVD_FP32, TSVD_FP64, tsvd_gram_colexp, tsvd_gram_finish, tsvd_gram_partial, tsvd_solve_gram,
               tsvd_sync_status, TSVD_OK, TsvdError)


class LibraryOps:
    """The per-rank steps on the library's kernels (handle h, FP32 working precision).  With
    check=False nothing synchronises the host: numeric outcomes are read from `info` after the
    solve (a timing loop runs this way)."""

    def __init__(self, h, check=True):
        self.h = h
        self.check = check

    def _sync(self, name):
        if not self.check:
            return
        st = tsvd_sync_status(self.h)
        if st != TSVD_OK:
            raise TsvdError(name, st)

    def colexp(self, A, m, n, lda):
        E = torch.empty(n, dtype=torch.int32, device=A.device)
        tsvd_gram_colexp(self.h, A, m, n, lda, TSVD_FP32, E)
        self._sync("tsvd_gram_colexp")
        return E

    def partial(self, A, m, n, lda, E):
        limbs = torch.empty(4, n, n, dtype=torch.int64, device=A.device)
        tsvd_gram_partial(self.h, A, m, n, lda, TSVD_FP32, E, limbs)
        self._sync("tsvd_gram_partial")
        return limbs

    def finish(self, limbs, E, n):
        G = torch.empty(n, n, dtype=torch.float64, device=limbs.device)
        tsvd_gram_finish(self.h, limbs, E, n, TSVD_FP64, G, n)
        return G

    def solve(self, G, A, m, n, lda, sigma, V, U=None, ldu=0, info=None):
        tsvd_solve_gram(self.h, G, n, A, m, n, lda, TSVD_FP32, TSVD_FP64, sigma, V, n, U, ldu, info)


def _distributed():
    # any initialised process group takes part, a one-rank group included
    return dist.is_available() and dist.is_initialized()


def sharded_gram(A, m, n, lda, ops, group=None):
    """G = A^T A over all ranks' rows (this rank holds A: m x n, leading dimension lda)."""
    E = ops.colexp(A, m, n, lda)
    if _distributed():
        dist.all_reduce(E, op=dist.ReduceOp.MAX, group=group)   # the exponents must bound every rank's rows
    limbs = ops.partial(A, m, n, lda, E)
    if _distributed():
        dist.all_reduce(limbs, op=dist.ReduceOp.SUM, group=group)  # integer sums: exact in any order
    return ops.finish(limbs, E, n)


def sharded_solve(A, m, n, lda, sigma, V, ops, U=None, ldu=0, info=None, group=None):
    """Algorithm 1 on the row-sharded A: sigma and V (the same on every rank) and this rank's
    rows of U.  Returns the Gram matrix."""
    G = sharded_gram(A, m, n, lda, ops, group)
    ops.solve(G, A, m, n, lda, sigma, V, U, ldu, info)
    return G
