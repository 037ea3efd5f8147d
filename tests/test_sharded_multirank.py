"""The row-sharded Gram's exchange (paper_2603_11953_gb300/sharded.py; Sec. 4.2.1's
single global reduction of A^T A) on gloo ranks on the CPU.

The per-rank arithmetic is replaced by an exact integer model with the library's
interface (column exponents E_j with max |a_rj| < 2^E_j; each rank's part of A^T A
as an integer in units 2^(E_i + E_j - 60) split into four 32-bit limbs; one
rounding at the end), so what is tested here is the plumbing that the GPU ranks
use unchanged: the all-reduce MAX of the exponents (a rank whose rows are small
must take the other ranks' exponents), the all-reduce SUM of the limbs (signed
values, carries between limbs), and that two or three ranks give bitwise the
result of one rank holding every row.  No GPU is involved; on GPUs the same
driver runs with NCCL and the library's kernels (GPU tests cover those).
"""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

EMPTY = -(1 << 20)


class IntegerModelOps:
    """CPU stand-in for LibraryOps: exact integer arithmetic with the same data layout."""

    def colexp(self, A, m, n, lda):
        E = torch.full((n,), EMPTY, dtype=torch.int32)
        for j in range(n):
            mx = float(A[:m, j].abs().max()) if m > 0 else 0.0
            if mx > 0.0:
                E[j] = int(np.frexp(np.float32(mx))[1])  # least e with mx < 2^e (mx = f 2^e, f in [0.5, 1))
        return E

    def partial(self, A, m, n, lda, E):
        # integer digits q = trunc(a 2^(30 - E)), the part sum_r q_ri q_rj, as four 32-bit limbs
        limbs = torch.zeros(4, n, n, dtype=torch.int64)
        q = [[int(np.trunc(np.ldexp(float(A[r, j]), 30 - int(E[j])))) if int(E[j]) != EMPTY else 0
              for j in range(n)] for r in range(m)]
        for i in range(n):
            for j in range(n):
                t = sum(q[r][i] * q[r][j] for r in range(m))
                u = t % (1 << 128)  # two's complement
                for k in range(3):
                    limbs[k, i, j] = (u >> (32 * k)) & 0xFFFFFFFF
                limbs[3, i, j] = t >> 96
        return limbs

    def finish(self, limbs, E, n):
        G = torch.zeros(n, n, dtype=torch.float64)
        for i in range(n):
            for j in range(n):
                if int(E[i]) == EMPTY or int(E[j]) == EMPTY:
                    continue
                t = sum(int(limbs[k, i, j]) << (32 * k) for k in range(4))
                G[i, j] = float(Fraction(t) * Fraction(2) ** (int(E[i]) + int(E[j]) - 60))
        return G


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix(m, n, seed):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(m, n, generator=g, dtype=torch.float64) * torch.exp2(torch.randint(-8, 8, (n,), generator=g))
    A[: m // 3] *= 1e-3  # rank 0 gets the small rows: its own exponents would be too small
    A[:, 2] = 0.0        # an all-zero column
    return A.float()


def _rank_main(rank, world, port, m, n, bounds, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    from paper_2603_11953_gb300 import sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = _matrix(m, n, 5)
    r0, r1 = bounds[rank], bounds[rank + 1]
    Ar = A[r0:r1].contiguous()
    G = sharded.sharded_gram(Ar, r1 - r0, n, max(r1 - r0, 1), IntegerModelOps())
    out.put((rank, G.numpy()))
    dist.destroy_process_group()


def _run(world, bounds, m=24, n=5):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, m, n, bounds, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.timeout(240)
@pytest.mark.parametrize("world,bounds", [(2, [0, 11, 24]), (3, [0, 8, 9, 24])])
def test_sharded_gram_on_gloo_ranks_matches_one_rank(world, bounds):
    m, n = 24, 5
    res = _run(world, bounds, m, n)
    # every rank holds the same Gram, bitwise
    for r in range(1, world):
        assert np.array_equal(res[r], res[0])
    # and it is the single-rank result of the same model on all rows, bitwise
    from paper_2603_11953_gb300 import sharded
    A = _matrix(m, n, 5)
    G1 = sharded.sharded_gram(A, m, n, m, IntegerModelOps()).numpy()
    assert np.array_equal(res[0], G1)
    # the model itself: A^T A up to its truncation (2^-30 of each column's bound per entry)
    A64 = A.double().numpy()
    exact = A64.T @ A64
    E = IntegerModelOps().colexp(A, m, n, m)
    scale = np.where(E.numpy() != EMPTY, np.exp2(E.numpy().astype(float)), 0.0)
    assert np.all(np.abs(G1 - exact) <= 2 * m * 2.0 ** -30 * np.outer(scale, scale) + 1e-300)
    assert not G1[2].any() and not G1[:, 2].any()


def test_limbs_carry_negative_values():
    """A part whose sum is negative and spans all four limbs survives the limb split and sum."""
    ops = IntegerModelOps()
    A = torch.tensor([[-3.0e3, 1.0], [2.5e3, -1.0]], dtype=torch.float32)
    E = ops.colexp(A, 2, 2, 2)
    total = ops.partial(A[:1], 1, 2, 2, E) + ops.partial(A[1:], 1, 2, 2, E)
    G = ops.finish(total, E, 2).numpy()
    A64 = A.double().numpy()
    np.testing.assert_allclose(G, A64.T @ A64, rtol=1e-8)
    assert G[0, 1] < 0
