"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * Gram (Alg. 1 l.2, eq. (ATA) with eps_M = 2^-50): |G - S| <= 2^-50 (|A|^T|A|)
    componentwise, S the exact sum; plus the deterministic any-size bound
    |G - S|_ij <= m * 2^-50 * 2^(E_i + E_j) with 2^E_j <= 2 max_r |a_rj|.
  * eigenvalues (same M into both Jacobis): relative difference
    <= 32 n u_h kappa(C), C = D^-1 M D^-1.
  * sigma end to end, FP32 working: |sigma - sigma_oracle| <= 2 u_32 sigma_oracle
    (the higher-precision errors are far below one FP32 ulp for kappa(B) <= 1e3).
  * U (eq. (AV-0)): |U - RN_32(A W)| <= (n + 13) u_32 (|A| |W|), W = RN_32(V / sigma):
    the FP32 dot-product bound (n + 1) u_32 plus 12 u_32 for the 3-term TF32 split
    of the tensor-core kernel (each rounded low part and the dropped lo x lo term
    contribute at most 2^-22 |a||w| per product); the CUDA-core kernel (u_variant 1)
    is held to (n + 1) u_32.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2603_11953_gb300 as T
from paper_2603_11953_gb300 import build as B
from paper_2603_11953_gb300 import workloads

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
UH = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    T.load_library()


def handle(**kw):
    opts = T.tsvd_opts(**kw) if kw else None
    h, _ = T.tsvd_create(0, torch.cuda.current_stream().cuda_stream, opts)
    return h


def colmajor(ld, n, dtype, device="cuda"):
    return torch.zeros(n, ld, dtype=dtype, device=device).T  # (ld, n), column j contiguous


def gpu_gram(A, m, n, lda, h=None, higher=T.TSVD_FP64):
    own = h is None
    h = handle() if own else h
    G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, lda, T.TSVD_FP32, higher, G, n)
    st = T.tsvd_sync_status(h)
    if own:
        T.tsvd_destroy(h)
    Gh = G[: n * n].view(n, n).T.cpu().numpy()
    Gl = G[n * n:].view(n, n).T.cpu().numpy()
    return Gh, Gl, st


def gpu_solve(A, m, n, lda, want_u=True, h=None):
    own = h is None
    h = handle() if own else h
    sigma = torch.zeros(n, dtype=torch.float32, device="cuda")
    V = colmajor(n, n, torch.float32)
    U = colmajor(max(m, 1), n, torch.float32) if want_u else None
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_solve(h, A, m, n, lda, T.TSVD_FP32, T.TSVD_FP64, sigma, V, n, U, m if want_u else 0, info)
    torch.cuda.synchronize()
    if own:
        T.tsvd_destroy(h)
    inf = info.cpu().numpy()
    return (sigma.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64),
            None if U is None else U[:m].cpu().numpy().astype(np.float64), int(inf[0]), int(inf[1]))


def exp_bound(A):
    mx = np.abs(A).max(axis=0).astype(np.float64)
    return 2.0 * np.where(mx > 0, mx, 0.0)


def check_gram(A_np, Gh, m, n):
    S_hi, S_lo, Sabs = oracle.gram(A_np)
    err = np.abs((Gh - S_hi) - S_lo)  # |G - S| with S = S_hi + S_lo (exact to 2^-106)
    ratio = np.where(Sabs > 0, err / np.where(Sabs > 0, Sabs, 1.0), 0.0)
    any_size = m * 2.0 ** -50 * np.outer(exp_bound(A_np), exp_bound(A_np))
    assert np.all(err <= any_size), float(np.max(err - any_size))
    return float(ratio.max())


# ------------------------------------------------------------------ Gram (a1-a3)
@pytest.mark.parametrize("m,n,split", [(1000, 1, 0), (1000, 5, 0), (20000, 16, 0), (4133, 33, 3),
                                       (70001, 48, 0), (131077, 64, 0), (131077, 64, 5),
                                       (5004, 65, 0), (9000, 96, 0), (4100, 200, 0), (20480, 256, 0)])
def test_gram_matches_exact_sum(m, n, split):
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=m + n, device="cuda")
    h = handle(split_k=split) if split else None
    Gh, Gl, st = gpu_gram(A, m, n, m, h=h)
    if h is not None:
        T.tsvd_destroy(h)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, m)
    worst = check_gram(A_np, Gh, m, n)
    assert worst <= 2.0 ** -50, worst
    assert np.array_equal(Gh, Gh.T)


def test_gram_deterministic_and_dd_output():
    m, n = 50000, 40
    A, _ = workloads.small_case(m, n, seed=3, device="cuda")
    G1, L1, _ = gpu_gram(A, m, n, m, higher=T.TSVD_DD)
    G2, L2, _ = gpu_gram(A, m, n, m, higher=T.TSVD_DD)
    assert np.array_equal(G1, G2) and np.array_equal(L1, L2)
    # the DD pair is a faithful split of one exact number: |lo| <= ulp(hi)/2
    assert np.all(np.abs(L1) <= np.spacing(np.abs(G1)) / 2)


def test_gram_lda_unaligned_and_ragged():
    m, n, lda = 3001, 24, 3010
    base = torch.zeros(lda * n + 1, dtype=torch.float32, device="cuda")
    A, _ = workloads.small_case(m, n, seed=9, device="cuda", lda=lda)
    flat = A.T.reshape(-1)
    base[1:] = flat  # base pointer offset by 4 bytes: not 16-byte aligned
    Au = base[1:]
    Gh, _, st = gpu_gram(Au, m, n, lda)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, m)
    assert check_gram(A_np, Gh, m, n) <= 2.0 ** -50


def test_gram_powers_of_two_and_stacking_are_exact():
    """Invariants the exact construction guarantees bitwise: [A; A] gives 2G
    when both halves land on the same per-CTA scales (one CTA, and row 0
    holds every column's largest magnitude so the running scale is final
    after the first chunk: a later growth would re-grid, i.e. truncate, the
    earlier chunks), and scaling a column by 2^p scales its row/column of G
    by 2^p."""
    m, n = 2048, 8
    A, _ = workloads.small_case(m, n, seed=4, device="cuda")
    A[0, :] = 1.5 * A[:m].abs().max(dim=0).values
    h = handle(split_k=1)
    G, _, _ = gpu_gram(A, m, n, m, h=h)
    AA = torch.cat([A[:m], A[:m]], 0).contiguous()
    AA = AA.T.contiguous().T  # column-major
    G2, _, _ = gpu_gram(AA, 2 * m, n, 2 * m, h=h)
    assert np.array_equal(G2, 2 * G)
    As = A.clone()
    As[:, 3] *= 2.0 ** 20
    Gs, _, _ = gpu_gram(As, m, n, m, h=h)  # same split, so the same per-CTA row ranges
    T.tsvd_destroy(h)
    sc = np.ones(n)
    sc[3] = 2.0 ** 20
    assert np.array_equal(Gs, G * np.outer(sc, sc))


# ------------------------------------------------------------------ fixed scales and the row-sharded Gram (Sec. 4.2.1)
def test_gram_fixed_scale_bitwise_invariant():
    """fixed_scale = 1: every entry is digited against its column's exponent over the whole A and
    every digit-pair product is summed exactly, so the Gram is bitwise the same for any split of the
    rows over CTAs and any order of the rows; it stays within 2^-50 (|A|^T|A|) of the exact sum."""
    m, n = 70004, 48
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=21, device="cuda")
    A_np = workloads.to_numpy_colmajor(A, m)
    ref = None
    for split in (0, 1, 7, 152, 300):
        h = handle(fixed_scale=1, split_k=split) if split else handle(fixed_scale=1)
        Gh, Gl, st = gpu_gram(A, m, n, m, h=h, higher=T.TSVD_DD)
        T.tsvd_destroy(h)
        assert st == T.TSVD_OK
        if ref is None:
            ref = (Gh, Gl)
            S_hi, S_lo, Sabs = oracle.gram(A_np)
            assert np.all(np.abs((Gh - S_hi) + (Gl - S_lo)) <= 2.0 ** -50 * Sabs)
        assert np.array_equal(Gh, ref[0]) and np.array_equal(Gl, ref[1]), split
    perm = torch.randperm(m, generator=torch.Generator().manual_seed(3)).cuda()
    Ap = A[:m][perm].T.contiguous().T
    h = handle(fixed_scale=1)
    Gh, Gl, st = gpu_gram(Ap, m, n, m, h=h, higher=T.TSVD_DD)
    T.tsvd_destroy(h)
    assert st == T.TSVD_OK and np.array_equal(Gh, ref[0]) and np.array_equal(Gl, ref[1])
    # unaligned input is refused with TSVD_ERR_ALIGN
    h = handle(fixed_scale=1)
    G = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    assert T.tsvd_gram(h, A, m - 1, n, m - 1, T.TSVD_FP32, T.TSVD_FP64, G, n, check=False) == T.TSVD_ERR_ALIGN
    T.tsvd_destroy(h)


@pytest.mark.parametrize("bounds", [[0, 70004], [0, 30000, 70004], [0, 4, 40000, 40000, 70004],
                                    [0, 12000, 24000, 36000, 48000, 70004]])
def test_row_sharded_gram_emulated_ranks(bounds):
    """The row-sharded entry points with the ranks emulated in one process (their all-reduces done
    by hand on the device tensors): for one to five shards, empty shards included, the finished
    Gram is bitwise the fixed-scale Gram of the whole A, and tsvd_solve_gram on it gives bitwise the
    sigma and V of tsvd_solve with fixed scales, and every shard's U rows."""
    m, n = bounds[-1], 40
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=77, device="cuda")
    # two shards on few CTAs: many 1024-row periods per CTA
    h = handle(split_k=3) if len(bounds) == 3 else handle()
    shards = [(bounds[k], bounds[k + 1]) for k in range(len(bounds) - 1)]
    Es = []
    for r0, r1 in shards:
        E = torch.zeros(n, dtype=torch.int32, device="cuda")
        T.tsvd_gram_colexp(h, A[r0:], r1 - r0, n, m, T.TSVD_FP32, E)
        Es.append(E)
    E = torch.stack(Es).max(dim=0).values.contiguous()   # the all-reduce MAX
    limbs = torch.zeros(4, n, n, dtype=torch.int64, device="cuda")
    for r0, r1 in shards:
        part = torch.zeros(4, n, n, dtype=torch.int64, device="cuda")
        T.tsvd_gram_partial(h, A[r0:], r1 - r0, n, m, T.TSVD_FP32, E, part)
        assert T.tsvd_sync_status(h) == T.TSVD_OK
        limbs += part                                       # the all-reduce SUM
    G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram_finish(h, limbs, E, n, T.TSVD_DD, G, n)
    hf = handle(fixed_scale=1)
    Gref, Glref, st = gpu_gram(A, m, n, m, h=hf, higher=T.TSVD_DD)
    assert st == T.TSVD_OK
    g = G.cpu().numpy()
    assert np.array_equal(g[: n * n].reshape(n, n).T, Gref) and np.array_equal(g[n * n:].reshape(n, n).T, Glref)
    # the n x n stage on every "rank" and each shard's rows of U
    sig_ref, V_ref, U_ref, st, _ = gpu_solve(A, m, n, m, h=hf)
    T.tsvd_destroy(hf)
    assert st == T.TSVD_OK
    for r0, r1 in shards:
        sig = torch.zeros(n, device="cuda")
        V = colmajor(n, n, torch.float32)
        U = colmajor(max(r1 - r0, 1), n, torch.float32)
        info = torch.zeros(6, dtype=torch.int32, device="cuda")
        T.tsvd_solve_gram(h, G, n, A[r0:], r1 - r0, n, m, T.TSVD_FP32, T.TSVD_FP64, sig, V, n, U, max(r1 - r0, 1),
                          info)
        torch.cuda.synchronize()
        assert int(info[0].item()) == T.TSVD_OK
        assert np.array_equal(sig.cpu().numpy().astype(np.float64), sig_ref)
        assert np.array_equal(V.cpu().numpy().astype(np.float64), V_ref)
        if r1 > r0:
            assert np.array_equal(U[: r1 - r0].cpu().numpy().astype(np.float64), U_ref[r0:r1])
    # exponents that do not bound a column are reported; misaligned shards are refused
    Ebad = E.clone()
    Ebad[3] -= 1
    part = torch.zeros(4, n, n, dtype=torch.int64, device="cuda")
    T.tsvd_gram_partial(h, A, m, n, m, T.TSVD_FP32, Ebad, part)
    assert T.tsvd_sync_status(h) == T.TSVD_ERR_ARG
    assert T.tsvd_gram_partial(h, A[1:], m - 1, n, m, T.TSVD_FP32, E, part, check=False) == T.TSVD_ERR_ALIGN
    T.tsvd_destroy(h)


# ------------------------------------------------------------------ mixed precision Cholesky QR (Sec. 3.1, Theorem 3)
@pytest.mark.parametrize("m,n,kappa,logd", [(20000, 16, 1e3, 3.0), (65537, 33, 1e2, 2.0), (131076, 64, 1e3, 3.0),
                                            (300, 64, 10.0, 1.0)])
def test_cholqr_matches_oracle(m, n, kappa, logd):
    """tsvd_cholqr: R is the plain FP64 Cholesky factor of the Gram tsvd_gram returns (backward
    error |R^T R - M| <= (n + 1) u_h |R|^T |R| componentwise); sampled rows of Q solve q R_w = a
    for R_w = RN_32(R) with the FP32 forward substitution's backward error
    |q R_w - a| <= n u_32 |q| |R_w| (and agree with the oracle's exactly rounded solution within the
    matching forward bound); Q is orthogonal to O(u) kappa(B) (Theorem 3, constant 2n)."""
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=23 * m + n, device="cuda")
    h = handle()
    Q = colmajor(m, n, torch.float32)
    R = colmajor(n, n, torch.float64)
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_cholqr(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, Q, m, R, n, info)
    torch.cuda.synchronize()
    assert int(info[0].item()) == T.TSVD_OK
    M, _, st = gpu_gram(A, m, n, m, h=h)
    T.tsvd_destroy(h)
    assert st == T.TSVD_OK
    Rn = R.cpu().numpy()
    assert np.array_equal(Rn, np.triu(Rn))
    # Cholesky backward error on the same M
    assert np.all(np.abs(Rn.T @ Rn - M) <= (n + 1) * UH * 4 * (np.abs(Rn).T @ np.abs(Rn)))
    Ro, st_o = oracle.cholesky(M)
    assert st_o == 0
    d = np.sqrt(np.diag(M))
    kC = np.linalg.cond(M / np.outer(d, d))
    assert np.all(np.abs(Rn - Ro) <= 64 * n * UH * kC * d[None, :])  # |r_ij| <= d_j = (M_jj)^(1/2)
    # rows of Q
    A_np = workloads.to_numpy_colmajor(A, m)
    Rw = Rn.astype(np.float32).astype(np.float64)
    rows = np.unique(np.concatenate([[0, m - 1], np.linspace(0, m - 1, 40).astype(np.int64)]))
    Qn = Q[:m].cpu().numpy().astype(np.float64)
    resid = np.abs(Qn[rows] @ Rw - A_np[rows].astype(np.float64))
    assert np.all(resid <= n * U32 * (np.abs(Qn[rows]) @ np.abs(Rw)) + 1e-38)
    Qo = oracle.cholqr_rows(A_np, Rw, rows, 24)
    # q - q_exact = q dR R_w^-1 with |dR| <= n u |R_w|, plus the rounding of q_exact
    fwd = (n + 2) * U32 * ((np.abs(Qn[rows]) @ np.abs(Rw)) @ np.abs(np.linalg.inv(Rw))) + U32 * np.abs(Qo) + 1e-38
    assert np.all(np.abs(Qn[rows] - Qo) <= fwd)
    kB = math.sqrt(kC)
    Qt = Q[:m].double()
    orth = torch.linalg.matrix_norm(Qt.T @ Qt - torch.eye(n, dtype=torch.float64, device="cuda"), ord=2).item()
    assert orth <= 2 * n * U32 * kB, (orth, kB)


def test_cholqr_rank_deficient_and_args():
    m, n = 4096, 12
    A, _ = workloads.small_case(m, n, seed=3, device="cuda")
    A[:, 7] = 0.0
    h = handle()
    Q = colmajor(m, n, torch.float32)
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_cholqr(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, Q, m, None, 0, info)
    torch.cuda.synchronize()
    assert int(info[0].item()) == T.TSVD_ERR_NOT_FULL_RANK
    assert T.tsvd_cholqr(h, A, n - 1, n, m, T.TSVD_FP32, T.TSVD_FP64, Q, m, check=False) == T.TSVD_ERR_ARG
    assert T.tsvd_cholqr(h, A, m, 65, m, T.TSVD_FP32, T.TSVD_FP64, Q, m, check=False) in (T.TSVD_ERR_UNSUPPORTED,
                                                                                            T.TSVD_ERR_ARG)
    T.tsvd_destroy(h)


# ------------------------------------------------------------------ Jacobi (a4-a6)
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("n,kappa,logd", [(1, 1.0, 0.0), (2, 10.0, 1.0), (7, 1e2, 2.0), (16, 1e3, 3.0),
                                          (33, 1e3, 3.0), (64, 1e4, 4.0), (65, 1e3, 3.0), (100, 1e3, 3.0),
                                          (128, 1e3, 3.0), (200, 1e2, 2.0), (256, 1e3, 3.0)])
def test_eig_matches_oracle_jacobi(n, kappa, logd, variant):
    """Both FP64 eigen routes on the oracle's exact Gram against the oracle's two-sided Jacobi: the
    two-sided tournament kernel (variant 1) and the pivoted Cholesky + cluster one-sided Jacobi
    (variant 2; 1, 2 and 4 rows per lane for n <= 64, 128, 256)."""
    m = max(4 * n, 200)
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=11 * n)
    S_hi, _, _ = oracle.gram(workloads.to_numpy_colmajor(A, m))
    lam_o, V_o, sw, st = oracle.jacobi_fp64(S_hi)
    assert st == 0
    lam_o = np.sort(lam_o)[::-1]
    M = torch.from_numpy(np.asfortranarray(S_hi)).cuda().T.contiguous().T
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = colmajor(n, n, torch.float64)
    info_d = torch.zeros(6, dtype=torch.int32, device="cuda")
    h = handle(eig_variant=variant)
    T.tsvd_eig(h, M, n, n, lam, V, n, info_d)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    inf = info_d.cpu().numpy()
    assert inf[0] == T.TSVD_OK
    d = np.sqrt(np.diag(S_hi))
    kC = np.linalg.cond(S_hi / np.outer(d, d))
    lam_g = lam.cpu().numpy()
    np.testing.assert_allclose(lam_g, lam_o, rtol=32 * n * UH * kC)
    Vg = V.cpu().numpy()
    assert np.abs(Vg.T @ Vg - np.eye(n)).max() <= 64 * n * UH
    # eigenvectors: scaled residual of every column against the same M
    R = S_hi @ Vg - Vg * lam_g
    assert np.all(np.linalg.norm(R, axis=0) <= 64 * n * UH * kC * np.abs(lam_g).max() + 1e-300)


# ------------------------------------------------------------------ wide n (64 < n <= 256)
@pytest.mark.parametrize("m,n", [(3000, 100), (4100, 256)])
def test_solve_wide_matches_oracle(m, n):
    A, _ = workloads.small_case(m, n, kappa_sigma=1e2, logd=2.0, seed=11 * m + n, device="cuda")
    sig, V, U, st, sweeps = gpu_solve(A, m, n, m)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, m)
    ref = oracle.svd(A_np, higher=1)
    assert ref["status"] == 0
    rel = np.abs(sig - ref["sigma_h"]) / ref["sigma_h"]
    assert rel.max() <= 2 * U32, rel.max()
    W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
    rows = np.unique(np.linspace(0, m - 1, 64).astype(np.int64))
    Uref = oracle.rows_times(A_np, W, rows, 24)
    bound = (n + 1) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
    assert np.all(np.abs(U[rows] - Uref) <= bound)
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-4


# ------------------------------------------------------------------ solve (a1-a7)
@pytest.mark.parametrize("variant", [0, 1])  # 0: defaults (tensor-core U); 1: two-sided Jacobi, CUDA-core U
@pytest.mark.parametrize("m,n,kappa,logd", [(20000, 16, 1e3, 3.0), (5000, 1, 1.0, 0.0), (16, 16, 1e2, 1.0),
                                            (12345, 33, 1e3, 3.0), (65537, 64, 1e3, 3.0),
                                            (40964, 64, 1e3, 3.0), (300, 64, 1e2, 2.0)])
def test_solve_matches_oracle(m, n, kappa, logd, variant):
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=5 * m + n, device="cuda")
    h = handle(eig_variant=variant, u_variant=1) if variant else None
    sig, V, U, st, sweeps = gpu_solve(A, m, n, m, h=h)
    if h is not None:
        T.tsvd_destroy(h)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, m)
    ref = oracle.svd(A_np, higher=1)
    assert ref["status"] == 0
    rel = np.abs(sig - ref["sigma_h"]) / ref["sigma_h"]
    assert rel.max() <= 2 * U32, rel.max()
    assert rel.max() <= 1e-5
    # V: same sign rule; entrywise against the oracle within the cast + eigenvector error
    gaps = np.abs(np.diff(ref["sigma_h"] ** 2)) / ref["sigma_h"][:-1] ** 2 if n > 1 else np.array([1.0])
    if n > 1 and gaps.min() > 1e-3:
        assert np.abs(V - ref["V_w"]).max() <= 4 * U32 + 1e-9 / gaps.min()
    # U against the exactly rounded product with the GPU's own W (eq. (AV-0))
    W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
    rows = np.unique(np.concatenate([np.arange(min(m, 64)), np.linspace(0, m - 1, 200).astype(np.int64)]))
    Uref = oracle.rows_times(A_np, W, rows, 24)
    slack = 1 if variant else 13
    bound = (n + slack) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
    assert np.all(np.abs(U[rows] - Uref) <= bound)
    # Remark 1: U is orthonormal to O(u) + O(u_h) kappa^2(B)
    orth = np.abs(U.T @ U - np.eye(n)).max()
    assert orth <= 1e-4, orth


def test_autotune_choice_and_results():
    """opts.autotune = 1: the first solve of a shape times the Gram's split-K candidates and both FP32 U
    kernels and keeps the fastest; the choice is reported for the shape and reused (a second solve is
    bitwise the first), the Gram stays within 2^-50 (|A|^T|A|) of the exact sum, sigma within 2 u_32 of
    the oracle and U within the tensor-core U's bound (n + 13) u_32 (|A||W|)."""
    m, n = 300000, 48
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=909, device="cuda")
    A_np = workloads.to_numpy_colmajor(A, m)
    h = handle(autotune=1)
    sig, V, U, st, _ = gpu_solve(A, m, n, m, h=h)
    assert st == T.TSVD_OK
    ch = T.tsvd_autotune_choice(h, m, n, T.TSVD_FP32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ch is not None and ch[0] in (0, sms // 2, 2 * sms, 3 * sms) and ch[1] in (0, 1)
    assert ch[2] > 0.0 and ch[3] > 0.0
    assert T.tsvd_autotune_choice(h, m + 1, n, T.TSVD_FP32) is None
    sig2, V2, U2, st2, _ = gpu_solve(A, m, n, m, h=h)
    assert st2 == T.TSVD_OK and T.tsvd_autotune_choice(h, m, n, T.TSVD_FP32) == ch
    assert np.array_equal(sig, sig2) and np.array_equal(V, V2) and np.array_equal(U, U2)
    Gh, _, stg = gpu_gram(A, m, n, m, h=h)
    assert stg == T.TSVD_OK
    assert check_gram(A_np, Gh, m, n) <= 2.0 ** -50
    T.tsvd_destroy(h)
    ref = oracle.svd(A_np, higher=1)
    assert ref["status"] == 0
    assert (np.abs(sig - ref["sigma_h"]) / ref["sigma_h"]).max() <= 2 * U32
    W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
    rows = np.unique(np.concatenate([np.arange(64), np.linspace(0, m - 1, 200).astype(np.int64)]))
    Uref = oracle.rows_times(A_np, W, rows, 24)
    bound = (n + 13) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
    assert np.all(np.abs(U[rows] - Uref) <= bound)


def test_batch_matches_single_solves_and_exact_u():
    """The batched launches (Gram work items on the tcgen05 kernel for instances whose A is 16-byte
    aligned with lda a multiple of 4, on the mma.sync Ozaki kernel otherwise; one CTA per instance
    for the n x n stage) against single solves (tensor-core Gram, cluster Jacobi): both are the same
    exact Gram and FP64 Jacobi up to rounding, so sigma agrees to 2 FP32 ulps and V to 1e-4 (well
    separated spectra); U against the exact product with the batch's own W, (n + 1) u_32 (|A| |W|)."""
    cases = [(3000, 8), (1024, 16), (7777, 24), (2048, 64), (4096, 1), (40000, 48), (16385, 33), (130, 8), (200, 32),
             (33000, 32)]
    As = [workloads.small_case(m, n, seed=31 + i, device="cuda")[0] for i, (m, n) in enumerate(cases)]
    sig = [torch.zeros(n, device="cuda") for _, n in cases]
    Vs = [colmajor(n, n, torch.float32) for _, n in cases]
    Us = [colmajor(m, n, torch.float32) for m, n in cases]
    info = torch.zeros(6 * len(cases), dtype=torch.int32, device="cuda")
    h = handle()
    T.tsvd_batch_solve(h, len(cases), As, [m for m, _ in cases], [n for _, n in cases], [m for m, _ in cases],
                       T.TSVD_FP32, T.TSVD_FP64, sig, Vs, [n for _, n in cases], Us, [m for m, _ in cases],
                       info)
    torch.cuda.synchronize()
    assert T.tsvd_sync_status(h) == T.TSVD_OK
    T.tsvd_destroy(h)
    inf = info.view(len(cases), 6).cpu().numpy()
    assert np.all(inf[:, 0] == 0) and np.all(inf[:, 1] >= 1)
    rng = np.random.default_rng(4)
    for k, (m, n) in enumerate(cases):
        s1, V1, _, st, _ = gpu_solve(As[k], m, n, m, want_u=False)
        sb = sig[k].cpu().numpy().astype(np.float64)
        Vb = Vs[k].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(sb - s1) <= 2.0 ** -22 * s1), k
        assert np.abs(Vb - V1).max() <= 1e-4, k
        A_np = workloads.to_numpy_colmajor(As[k], m)
        W = (Vs[k].cpu().numpy() / sig[k].cpu().numpy()[None, :]).astype(np.float64)
        rows = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 30)]))
        U_ref = oracle.rows_times(A_np, W, rows, 24)
        Ub = Us[k][:m].cpu().numpy().astype(np.float64)
        bound = (n + 1) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
        assert np.all(np.abs(Ub[rows] - U_ref) <= bound), k


def test_batch_statuses_per_instance():
    """Each instance reports its own status; the handle's status is the most severe."""
    m, n = 2000, 6
    good = workloads.small_case(m, n, seed=41, device="cuda")[0]
    bad = good.clone()
    bad[17, 2] = float("nan")
    flat = good.clone()
    flat[:, 3] = 0.0
    As = [good, bad, flat, good]
    sig = [torch.zeros(n, device="cuda") for _ in As]
    Vs = [colmajor(n, n, torch.float32) for _ in As]
    info = torch.zeros(6 * len(As), dtype=torch.int32, device="cuda")
    h = handle()
    T.tsvd_batch_solve(h, len(As), As, [m] * 4, [n] * 4, [m] * 4, T.TSVD_FP32, T.TSVD_FP64, sig, Vs, [n] * 4,
                       None, None, info)
    torch.cuda.synchronize()
    codes = info.view(len(As), 6)[:, 0].cpu().numpy().tolist()
    assert codes == [T.TSVD_OK, T.TSVD_ERR_NONFINITE, T.TSVD_ERR_NOT_FULL_RANK, T.TSVD_OK]
    assert T.tsvd_sync_status(h) == T.TSVD_ERR_NONFINITE
    T.tsvd_destroy(h)


def test_batch_ragged_workload_matches_oracle():
    """The batched workload's recipe (ragged m log-uniform, n from {8,...,64}, lda = m
    rounded up to 4, 256-byte aligned bases in one buffer) at 40 instances with m <= 8192."""
    buf, metas = workloads.make_batch(count=40, device="cuda", m_hi=8192)
    count = len(metas)
    As = [buf[md["offset"]:] for md in metas]
    sig = [torch.zeros(md["n"], device="cuda") for md in metas]
    Vs = [colmajor(md["n"], md["n"], torch.float32) for md in metas]
    info = torch.zeros(6 * count, dtype=torch.int32, device="cuda")
    h = handle()
    T.tsvd_batch_solve(h, count, As, [md["m"] for md in metas], [md["n"] for md in metas],
                       [md["lda"] for md in metas], T.TSVD_FP32, T.TSVD_FP64, sig, Vs,
                       [md["n"] for md in metas], None, None, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    assert np.all(info.view(count, 6)[:, 0].cpu().numpy() == 0)
    for k, md in enumerate(metas):
        m, n, lda = md["m"], md["n"], md["lda"]
        A_np = buf[md["offset"]:md["offset"] + lda * n].view(n, lda).T[:m].cpu().numpy()
        ref = oracle.svd(np.asfortranarray(A_np), higher=1)
        assert ref["status"] == 0
        # this spectrum reaches sigma_n / sigma_1 = 1e-5 (kappa(B) up to ~1e5), past the
        # kappa(B) <= 1e3 range where one FP32 ulp bounds the error: the target 1e-5 applies
        rel = np.abs(sig[k].cpu().numpy().astype(np.float64) - ref["sigma_h"]) / ref["sigma_h"]
        assert rel.max() <= 1e-5, (k, m, n, rel.max())


# ------------------------------------------------------------------ FP64 working (double-double Gram and n x n stage)
def gpu_gram64(A, m, n, lda, higher=T.TSVD_DD):
    h = handle()
    G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, lda, T.TSVD_FP64, higher, G, n)
    st = T.tsvd_sync_status(h)
    T.tsvd_destroy(h)
    return G[: n * n].view(n, n).T.cpu().numpy(), G[n * n:].view(n, n).T.cpu().numpy(), st


def pow2_above(A):
    """2^e_j with e_j the least integer such that max_r |a_rj| < 2^e_j (1 for a zero column)."""
    mx = np.abs(A).max(axis=0).astype(np.float64)
    return np.where(mx > 0, np.ldexp(1.0, np.frexp(mx)[1]), 1.0)


def check_gram64(A_np, Gh, Gl, m):
    """|G - S| <= 2^-88 m 2^(e_i + e_j): the 23-bit pieces' remainder (< 2^-92 of 2^e per entry) and the
    six piece pairs p + q >= 4 that are left out, each at most 2^-92 m 2^(e_i + e_j), plus the
    double-double roundings.  A missing pair with p + q <= 3 is at least ~2^-69 sqrt(m) 2^(e_i + e_j)."""
    S_hi, S_lo, _ = oracle.gram(A_np)
    err = np.abs((Gh - S_hi) + (Gl - S_lo))
    p2 = pow2_above(A_np)
    bound = 2.0 ** -88 * m * np.outer(p2, p2)
    assert np.all(err <= bound), float(np.max(err / bound))
    diag = np.sqrt(np.outer(np.diag(S_hi), np.diag(S_hi)))
    return float(np.max(np.where(diag > 0, err / np.where(diag > 0, diag, 1.0), 0.0)))


@pytest.mark.parametrize("m,n", [(1000, 1), (5003, 7), (20000, 32), (131077, 33), (70001, 64)])
def test_gram_fp64_is_double_double(m, n):
    A, _ = workloads.small_case(m, n, kappa_sigma=1e6, logd=6.0, seed=3 * m + n, dtype=torch.float64,
                                device="cuda")
    Gh, Gl, st = gpu_gram64(A, m, n, m)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, m)
    worst = check_gram64(A_np, Gh, Gl, m)
    assert worst <= 2.0 ** -80, worst
    assert np.array_equal(Gh, Gh.T) and np.array_equal(Gl, Gl.T)
    # FP64 output: the high part alone
    Gh2, _, st = gpu_gram64(A, m, n, m, higher=T.TSVD_FP64)
    assert st == T.TSVD_OK and np.array_equal(Gh2, Gh)


def test_gram_fp64_graded_columns_zero_column_and_lda():
    """Entries spread over 200 binades inside one column, a late large entry (the tensor-core
    kernel's scales grow during the pass), a zero column, and lda > m."""
    m, n, lda = 9001, 5, 9010
    rng = np.random.default_rng(11)
    A = np.zeros((lda, n))
    A[:m, 0] = rng.standard_normal(m) * np.ldexp(1.0, rng.integers(-100, 100, m))
    A[:m, 1] = rng.standard_normal(m) * 1e-3
    A[m - 7, 1] = 5e4
    A[:m, 3] = rng.standard_normal(m)
    A[:m, 4] = -A[:m, 3] + rng.standard_normal(m) * 2.0 ** -40  # nearly cancelling pair
    At = torch.from_numpy(A.T.copy()).to("cuda").T  # column-major (lda, n)
    Gh, Gl, st = gpu_gram64(At, m, n, lda)
    assert st == T.TSVD_OK
    check_gram64(A[:m], Gh, Gl, m)
    assert Gh[2].tolist() == [0.0] * n and Gl[2].tolist() == [0.0] * n


def test_gram_fp64_partition_and_permutation_invariant():
    """Every needed piece Gram is an exact sum before its one rounding, so the double-double Gram
    is bitwise the same for any split of the rows over CTAs (one to hundreds of partial sums, as
    row partitions over several GPUs would give) and for any order of the rows."""
    m, n = 70001, 20
    A, _ = workloads.small_case(m, n, kappa_sigma=1e5, logd=5.0, seed=21, dtype=torch.float64, device="cuda")
    ref = None
    for split in (0, 1, 7, 300):
        h = handle(split_k=split) if split else handle()
        G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        T.tsvd_gram(h, A, m, n, m, T.TSVD_FP64, T.TSVD_DD, G, n)
        assert T.tsvd_sync_status(h) == T.TSVD_OK
        T.tsvd_destroy(h)
        g = G.cpu().numpy()
        if ref is None:
            ref = g
        assert np.array_equal(g, ref), split
    perm = torch.randperm(m, generator=torch.Generator().manual_seed(5)).cuda()
    Ap = A[:m][perm].T.contiguous().T  # rows permuted, column-major again
    Gh, Gl, st = gpu_gram64(Ap, m, n, m)
    assert st == T.TSVD_OK
    assert np.array_equal(Gh, ref[: n * n].reshape(n, n).T) and np.array_equal(Gl, ref[n * n:].reshape(n, n).T)


def gpu_solve64(A, m, n, lda, higher=T.TSVD_DD, want_u=True):
    h = handle()
    sigma = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = colmajor(n, n, torch.float64)
    U = colmajor(max(m, 1), n, torch.float64) if want_u else None
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_solve(h, A, m, n, lda, T.TSVD_FP64, higher, sigma, V, n, U, m if want_u else 0, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    inf = info.cpu().numpy()
    return (sigma.cpu().numpy(), V.cpu().numpy(), None if U is None else U[:m].cpu().numpy(), int(inf[0]),
            int(inf[1]))


@pytest.mark.parametrize("m,n,kappa,logd", [(4000, 8, 1e6, 6.0), (20000, 32, 1e6, 6.0), (50001, 17, 1e4, 3.0),
                                            (3000, 64, 1e5, 4.0), (64, 1, 1.0, 0.0)])
def test_solve_fp64_matches_double_double_oracle(m, n, kappa, logd):
    """sigma within 1e-12 relative of the oracle's double-double Algorithm 1 (exact Gram, DD Jacobi)
    at kappa(B) up to ~1e6; V within 1e-10 (well separated geometric spectra); U against the
    exact product with the same W = RN_64(V / sigma), componentwise (n + 1) u_64 (|A| |W|)."""
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=5 * m + n, dtype=torch.float64,
                                device="cuda")
    sig, V, U, st, sweeps = gpu_solve64(A, m, n, m)
    assert st == T.TSVD_OK, st
    A_np = workloads.to_numpy_colmajor(A, m)
    ref = oracle.svd(A_np, higher=2)
    assert ref["status"] == 0
    s_ref = ref["sigma_h"] + ref["sigma_h_lo"]
    rel = np.abs(sig - ref["sigma_h"] - ref["sigma_h_lo"]) / s_ref
    assert rel.max() <= 1e-12, rel.max()
    assert np.abs(V - ref["V_h"]).max() <= 1e-10
    W = V / sig[None, :]
    rows = np.unique(np.linspace(0, m - 1, 257).astype(np.int64))
    U_ref = oracle.rows_times(A_np, W, rows, 53)
    bound = (n + 1) * UH * (np.abs(A_np[rows]) @ np.abs(W))
    assert np.all(np.abs(U[rows] - U_ref) <= bound)


def test_solve_fp64_with_fp64_stage_and_statuses():
    """higher = FP64 runs the FP64 n x n stage on the double-double Gram's high part (the literal
    reading of the stress configuration); rank deficiency and the plain Gram's missing double-double
    form are reported."""
    m, n = 6000, 12
    A, _ = workloads.small_case(m, n, kappa_sigma=1e2, logd=1.0, seed=77, dtype=torch.float64, device="cuda")
    sig, V, U, st, _ = gpu_solve64(A, m, n, m, higher=T.TSVD_FP64, want_u=False)
    assert st == T.TSVD_OK
    ref = oracle.svd(workloads.to_numpy_colmajor(A, m), higher=2)
    assert (np.abs(sig - ref["sigma_h"]) / ref["sigma_h"]).max() <= 1e-12
    C = A.clone()
    C[:, 4] = 0.0
    assert gpu_solve64(C, m, n, m, want_u=False)[3] == T.TSVD_ERR_NOT_FULL_RANK
    h = handle(gram_variant=1)
    sigma = torch.zeros(n, dtype=torch.float64, device="cuda")
    Vt = colmajor(n, n, torch.float64)
    assert T.tsvd_solve(h, A, m, n, m, T.TSVD_FP64, T.TSVD_DD, sigma, Vt, n, check=False) == T.TSVD_ERR_UNSUPPORTED
    T.tsvd_destroy(h)


# ------------------------------------------------------------------ Algorithm 2 (eig_variant 3)
def alg2_bound(kB, kC):
    """Remark 2: O(u) kappa(B) + O(u_h) kappa(B)^2 -- the FP32 SVD of the cast factor resolves the
    column-scaled factor to ~u_32 kappa(B) (constant 8 n^(1/2) for the dot products and rotations),
    the exact Gram's 2^-50 componentwise error enters through kappa(C) = kappa(B)^2."""
    return 2 * U32 + 64 * U32 * kB + 16 * 2.0 ** -50 * kC


@pytest.mark.parametrize("m,n,kappa,logd", [(2000, 7, 1e2, 2.0), (20000, 16, 1e3, 3.0), (9000, 33, 1e3, 4.0),
                                            (40000, 64, 1e3, 3.0), (40000, 64, 1e4, 4.0)])
def test_alg2_matches_oracle(m, n, kappa, logd):
    """The n x n stage of Algorithm 2 on the exact Gram: GPU (plain FP64 Cholesky, RN_32 cast, FP32
    one-sided Jacobi on the columns of R) against the oracle's Algorithm 2 (the same cast factor, its
    SVD to FP64 accuracy) and against the double-double Algorithm 1, both within Remark 2's bound;
    V orthogonal to FP32 accuracy."""
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=13 * m + n)
    A_np = workloads.to_numpy_colmajor(A, m)
    S = oracle.gram(A_np)[0]
    ref = oracle.alg2(S, working=0)
    assert ref["status"] == 0
    truth = oracle.svd(A_np, higher=2)
    s_true = truth["sigma_h"] + truth["sigma_h_lo"]
    d = np.sqrt(np.diag(S))
    kC = np.linalg.cond(S / np.outer(d, d))
    kB = math.sqrt(kC)
    M = torch.from_numpy(np.asfortranarray(S)).cuda().T.contiguous().T
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = colmajor(n, n, torch.float64)
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    h = handle(eig_variant=3)
    T.tsvd_eig(h, M, n, n, lam, V, n, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    assert int(info[0].item()) == T.TSVD_OK
    sig = np.sqrt(lam.cpu().numpy())
    e_ref = float(np.max(np.abs(sig - ref["sigma"]) / ref["sigma"]))
    e_true = float(np.max(np.abs(sig - s_true) / s_true))
    print(f"alg2 n={n} kappa(B)={kB:.3g}: rel err vs oracle alg2 {e_ref:.2e}, vs DD alg1 {e_true:.2e}")
    assert e_ref <= alg2_bound(kB, kC), (e_ref, kB)
    assert e_true <= alg2_bound(kB, kC), (e_true, kB)
    Vg = V.cpu().numpy()
    assert np.abs(Vg.T @ Vg - np.eye(n)).max() <= 8 * n * U32


def test_alg2_solve_end_to_end_and_unsupported():
    m, n = 50000, 48
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=88, device="cuda")
    h = handle(eig_variant=3)
    sig, V, U, st, sweeps = gpu_solve(A, m, n, m, h=h)
    assert st == T.TSVD_OK and sweeps >= 1
    A_np = workloads.to_numpy_colmajor(A, m)
    truth = oracle.svd(A_np, higher=2)
    s_true = truth["sigma_h"] + truth["sigma_h_lo"]
    S = oracle.gram(A_np)[0]
    d = np.sqrt(np.diag(S))
    kC = np.linalg.cond(S / np.outer(d, d))
    assert np.max(np.abs(sig - s_true) / s_true) <= alg2_bound(math.sqrt(kC), kC)
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-3
    # FP64 working and n > 64 are not built for Algorithm 2
    A64 = A.double()
    s64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    V64 = colmajor(n, n, torch.float64)
    assert T.tsvd_solve(h, A64, m, n, m, T.TSVD_FP64, T.TSVD_DD, s64, V64, n, check=False) == T.TSVD_ERR_UNSUPPORTED
    T.tsvd_destroy(h)


# ------------------------------------------------------------------ kappa(B) in tsvd_info
@pytest.mark.parametrize("m,n,kappa,logd", [(20000, 16, 1e3, 3.0), (9000, 33, 1e2, 2.0), (40000, 64, 1e4, 4.0),
                                            (5000, 8, 10.0, 1.0)])
def test_info_kappa_b_estimate(m, n, kappa, logd):
    """tsvd_info.kappa_B estimates kappa(B) = kappa(C)^(1/2), C = D^-1 M D^-1 the column-scaled exact
    Gram (A = B D): power and inverse iteration can only under-estimate the extreme eigenvalue
    ratio, and after their fixed iteration count they are within 20 %."""
    A, _ = workloads.small_case(m, n, kappa_sigma=kappa, logd=logd, seed=7 * m + n, device="cuda")
    h = handle()
    sigma = torch.zeros(n, device="cuda")
    V = colmajor(n, n, torch.float32)
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_solve(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, sigma, V, n, None, 0, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    assert int(info[0].item()) == T.TSVD_OK
    k_hat = float(info.view(torch.float64)[2].item())
    S = oracle.gram(workloads.to_numpy_colmajor(A, m))[0]
    d = np.sqrt(np.diag(S))
    k_true = math.sqrt(np.linalg.cond(S / np.outer(d, d)))
    assert 0.8 * k_true <= k_hat <= 1.02 * k_true, (k_hat, k_true)


def test_info_kappa_b_rank_deficient_is_infinite():
    m, n = 3000, 12
    A, _ = workloads.small_case(m, n, seed=8, device="cuda")
    A[:, 5] = 0.0
    h = handle()
    sigma = torch.zeros(n, device="cuda")
    V = colmajor(n, n, torch.float32)
    info = torch.zeros(6, dtype=torch.int32, device="cuda")
    T.tsvd_solve(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, sigma, V, n, None, 0, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    assert int(info[0].item()) == T.TSVD_ERR_NOT_FULL_RANK
    assert math.isinf(float(info.view(torch.float64)[2].item()))


# ------------------------------------------------------------------ bounded waits (tsvd_opts.timeout_cycles)
def test_timeout_option_reports_timeout_and_handle_recovers():
    """A wait limit far below the time a TMA load or a period drain takes makes the tcgen05 Gram's
    steady-state waits run out: the kernel records TSVD_ERR_TIMEOUT, drains what it started (those
    waits keep the default limit), frees its TMEM and returns; the status reaches the host, and the
    context stays usable (a default handle then gives the exact Gram)."""
    m, n = 1 << 21, 64
    A, _ = workloads.small_case(m, n, seed=12, device="cuda")
    h = handle(timeout_cycles=1)
    G = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, G, n)
    assert T.tsvd_sync_status(h) == T.TSVD_ERR_TIMEOUT
    T.tsvd_destroy(h)
    torch.cuda.synchronize()
    Gh, _, st = gpu_gram(A, 1 << 16, n, m)  # the first 65536 rows (lda = m)
    assert st == T.TSVD_OK
    A_np = workloads.to_numpy_colmajor(A, 1 << 16)
    assert check_gram(A_np, Gh, 1 << 16, n) <= 2.0 ** -50
    # a negative limit is an argument error
    opts = T.tsvd_opts(timeout_cycles=-5)
    _, st = T.tsvd_create(0, None, opts, check=False)
    assert st == T.TSVD_ERR_ARG


# ------------------------------------------------------------------ statuses and arguments
def test_status_nonfinite_rank_convergence_and_args():
    m, n = 4096, 8
    A, _ = workloads.small_case(m, n, seed=2, device="cuda")
    B = A.clone()
    B[100, 3] = float("nan")
    assert gpu_solve(B, m, n, m, want_u=False)[3] == T.TSVD_ERR_NONFINITE
    C = A.clone()
    C[:, 5] = 0.0
    assert gpu_solve(C, m, n, m, want_u=False)[3] == T.TSVD_ERR_NOT_FULL_RANK
    h = handle(max_sweeps=1)
    assert gpu_solve(A, m, n, m, want_u=False, h=h)[3] == T.TSVD_ERR_NO_CONVERGENCE
    T.tsvd_destroy(h)
    h = handle()
    sig = torch.zeros(n, device="cuda")
    V = colmajor(n, n, torch.float32)
    assert T.tsvd_solve(h, A, n - 1, n, m, 0, 1, sig, V, n, check=False) == T.TSVD_ERR_ARG  # m < n
    assert T.tsvd_solve(h, A, m, n, m - 1, 0, 1, sig, V, n, check=False) == T.TSVD_ERR_ARG  # lda < m
    assert T.tsvd_solve(h, A, m, n, m, 0, 1, sig, V, n - 1, check=False) == T.TSVD_ERR_ARG  # ldv < n
    assert T.tsvd_solve(h, A, m, n, m, 0, 7, sig, V, n, check=False) == T.TSVD_ERR_ARG  # bad tag
    assert T.tsvd_solve(h, A, m, 300, m, 0, 1, sig, V, 300, check=False) == T.TSVD_ERR_UNSUPPORTED
    T.tsvd_destroy(h)


# ------------------------------------------------------------------ full size, bench configuration
@pytest.mark.parametrize("name", ["ozaki_4194304x64_fp32"])
def test_full_size_sampled(name):
    spec = workloads.CONFIGS[name]
    A, meta = workloads.make_config(spec, device="cuda")
    m, n = spec.m, spec.n
    h = handle()
    G = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, G, n)
    sig, V, U, st, _ = gpu_solve(A, m, n, m, h=h)
    T.tsvd_destroy(h)
    assert st == T.TSVD_OK
    Gg = G.view(n, n).T.cpu().numpy()
    # sampled Gram entries against the exact oracle, column pairs one by one
    rng = np.random.default_rng(0)
    pairs = [(0, 0), (n - 1, n - 1), (0, n - 1)] + [tuple(sorted(rng.integers(0, n, 2))) for _ in range(3)]
    for i, j in pairs:
        cols = sorted({i, j})
        Ac = A[:m, cols].cpu().numpy()
        S_hi, S_lo, Sabs = oracle.gram(np.asfortranarray(Ac))
        a, b = cols.index(i), cols.index(j)
        err = abs((Gg[i, j] - S_hi[a, b]) - S_lo[a, b])
        assert err <= 2.0 ** -50 * Sabs[a, b], (i, j, err / Sabs[a, b])
    # the eigen stage on the GPU's own Gram against the oracle's Jacobi
    lam_o, V_o, _, st_o = oracle.jacobi_fp64(Gg)
    assert st_o == 0
    sig_o = np.sqrt(np.sort(lam_o)[::-1])
    d = np.sqrt(np.diag(Gg))
    kC = np.linalg.cond(Gg / np.outer(d, d))
    assert np.all(np.abs(sig - sig_o) <= (2 * U32 + 32 * n * UH * kC) * sig_o)
    # sampled U rows against the exactly rounded product with the GPU's W
    W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
    rows = np.unique(np.concatenate([[0, 1, m - 1], rng.integers(0, m, 61)]))
    A_rows = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    Uref = oracle.rows_times(np.asfortranarray(A_rows), W, np.arange(len(rows)), 24)
    bound = (n + 13) * U32 * (np.abs(A_rows.astype(np.float64)) @ np.abs(W)) + 1e-38
    assert np.all(np.abs(U[rows] - Uref) <= bound)
    Ut = torch.from_numpy(U).cuda()
    orth = (Ut.T @ Ut - torch.eye(n, dtype=torch.float64, device="cuda")).abs().max().item()
    assert orth <= 1e-3, orth


def test_full_size_sampled_wide():
    """The 1,048,576 x 256 FP32 workload (sigma log-uniform in [1e-5, 1], D = 10^U(-3, 3)) at full
    size in the launch configuration the benchmark would time (28 tensor-core passes over pairs of
    32-column blocks, the pivoted Cholesky in global scratch and the cluster one-sided Jacobi with 4
    rows per lane, U in a second pass): sampled Gram entries
    against the exact oracle (column pairs one by one), the eigen stage on the GPU's own Gram
    against the oracle's FP64 Jacobi, sampled U rows against the exactly rounded product."""
    spec = workloads.CONFIGS["wide_1048576x256_fp32"]
    A, _ = workloads.make_config(spec, device="cuda")
    m, n = spec.m, spec.n
    h = handle()
    G = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, G, n)
    assert T.tsvd_sync_status(h) == T.TSVD_OK
    sig, V, U, st, _ = gpu_solve(A, m, n, m, h=h)
    T.tsvd_destroy(h)
    assert st == T.TSVD_OK
    Gg = G.view(n, n).T.cpu().numpy()
    rng = np.random.default_rng(2)
    pairs = [(0, 0), (n - 1, n - 1), (0, n - 1), (31, 32), (100, 200)] + \
            [tuple(sorted(rng.integers(0, n, 2))) for _ in range(3)]
    for i, j in pairs:
        cols = sorted({i, j})
        Ac = np.asfortranarray(A[:m, cols].cpu().numpy())
        S_hi, S_lo, Sabs = oracle.gram(Ac)
        a, b = cols.index(i), cols.index(j)
        err = abs((Gg[i, j] - S_hi[a, b]) - S_lo[a, b])
        assert err <= 2.0 ** -50 * Sabs[a, b], (i, j, err / Sabs[a, b])
    lam_o, _, _, st_o = oracle.jacobi_fp64(Gg)
    assert st_o == 0
    sig_o = np.sqrt(np.sort(lam_o)[::-1])
    d = np.sqrt(np.diag(Gg))
    kC = np.linalg.cond(Gg / np.outer(d, d))
    assert np.all(np.abs(sig - sig_o) <= (2 * U32 + 32 * n * UH * kC) * sig_o)
    W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
    rows = np.unique(np.concatenate([[0, 1, m - 1], rng.integers(0, m, 29)]))
    A_rows = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    Uref = oracle.rows_times(np.asfortranarray(A_rows), W, np.arange(len(rows)), 24)
    bound = (n + 1) * U32 * (np.abs(A_rows.astype(np.float64)) @ np.abs(W)) + 1e-38
    assert np.all(np.abs(U[rows] - Uref) <= bound)


def test_plain_fp64_form_matches_oracle():
    """The all-FP64 plain form (gram_variant 1: FP64 FMA Gram with a fixed-order split-K combine, the
    same n x n stage and U), the comparison form of the benchmark: its Gram within the FP64
    summation bound m 2^-53 (|A|^T |A|) of the exact sum, and sigma, V, U against the oracle at the
    tolerances of the mixed form."""
    for m, n in [(20000, 16), (65537, 64), (3001, 33)]:
        A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=17 * m + n, device="cuda")
        A_np = workloads.to_numpy_colmajor(A, m)
        h = handle(gram_variant=1)
        Gh, _, st = gpu_gram(A, m, n, m, h=h)
        assert st == T.TSVD_OK
        S_hi, S_lo, Sabs = oracle.gram(A_np)
        assert np.all(np.abs((Gh - S_hi) - S_lo) <= m * UH * Sabs)
        sig, V, U, st, _ = gpu_solve(A, m, n, m, h=h)
        T.tsvd_destroy(h)
        assert st == T.TSVD_OK
        ref = oracle.svd(A_np, higher=1)
        assert np.max(np.abs(sig - ref["sigma_h"]) / ref["sigma_h"]) <= 2 * U32
        W = (V.astype(np.float32) / sig.astype(np.float32)).astype(np.float64)
        rows = np.unique(np.linspace(0, m - 1, 100).astype(np.int64))
        Uref = oracle.rows_times(A_np, W, rows, 24)
        bound = (n + 13) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
        assert np.all(np.abs(U[rows] - Uref) <= bound)


def test_batch_full_count_sampled():
    """The 4096-instance ragged batch of the benchmark (m log-uniform in [1024, 65536], n from
    {8, ..., 64}, lda = m rounded up to 4, 256-byte aligned bases), solved in one call with U:
    every instance reports TSVD_OK, and 24 sampled instances (the largest m, the largest n, and
    random ones) match the oracle's double-double Algorithm 1 within 1e-5 (sigma) and the exactly
    rounded product with the batch's own W (U rows)."""
    buf, metas = workloads.make_batch(count=4096, device="cuda")
    count = len(metas)
    As = [buf[md["offset"]:] for md in metas]
    Ubuf = torch.zeros_like(buf)
    Us = [Ubuf[md["offset"]:] for md in metas]
    sig = [torch.zeros(md["n"], device="cuda") for md in metas]
    Vs = [colmajor(md["n"], md["n"], torch.float32) for md in metas]
    info = torch.zeros(6 * count, dtype=torch.int32, device="cuda")
    h = handle()
    T.tsvd_batch_solve(h, count, As, [md["m"] for md in metas], [md["n"] for md in metas],
                       [md["lda"] for md in metas], T.TSVD_FP32, T.TSVD_FP64, sig, Vs,
                       [md["n"] for md in metas], Us, [md["lda"] for md in metas], info)
    torch.cuda.synchronize()
    assert T.tsvd_sync_status(h) == T.TSVD_OK
    T.tsvd_destroy(h)
    assert np.all(info.view(count, 6)[:, 0].cpu().numpy() == 0)
    rng = np.random.default_rng(6)
    picks = {int(np.argmax([md["m"] for md in metas])), int(np.argmax([md["m"] * md["n"] for md in metas]))}
    picks |= set(int(k) for k in rng.choice(count, 22, replace=False))
    for k in sorted(picks):
        md = metas[k]
        m, n, lda = md["m"], md["n"], md["lda"]
        A_np = np.asfortranarray(buf[md["offset"]:md["offset"] + lda * n].view(n, lda).T[:m].cpu().numpy())
        ref = oracle.svd(A_np, higher=2)
        assert ref["status"] == 0
        s_ref = ref["sigma_h"] + ref["sigma_h_lo"]
        got = sig[k].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - s_ref) / s_ref) <= 1e-5, (k, m, n)
        W = (Vs[k].cpu().numpy() / sig[k].cpu().numpy()[None, :]).astype(np.float64)
        rows = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 14)]))
        U_ref = oracle.rows_times(A_np, W, rows, 24)
        Ub = Ubuf[md["offset"]:md["offset"] + lda * n].view(n, lda).T[:m].cpu().numpy().astype(np.float64)
        bound = (n + 1) * U32 * (np.abs(A_np[rows].astype(np.float64)) @ np.abs(W)) + 1e-38
        assert np.all(np.abs(Ub[rows] - U_ref) <= bound), (k, m, n)


def test_full_size_sampled_fp64_stress():
    """The 16,777,216 x 32 FP64 workload (geometric 1 -> 1e-6, D = 10^U(-6, 6)) in the launch
    configuration the benchmark times: sampled Gram entries against the exact oracle (column pairs
    one by one), the double-double n x n stage on the GPU's own Gram against the oracle's
    double-double Jacobi, and sampled U rows against the exact product."""
    spec = workloads.CONFIGS["stress_16777216x32_fp64"]
    A, _ = workloads.make_config(spec, device="cuda")
    m, n = spec.m, spec.n
    h = handle()
    G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, m, T.TSVD_FP64, T.TSVD_DD, G, n)
    T.tsvd_destroy(h)
    sig, V, U, st, _ = gpu_solve64(A, m, n, m)
    assert st == T.TSVD_OK
    Gh = G[: n * n].view(n, n).T.cpu().numpy()
    Gl = G[n * n:].view(n, n).T.cpu().numpy()
    rng = np.random.default_rng(1)
    pairs = [(0, 0), (n - 1, n - 1), (0, n - 1)] + [tuple(sorted(rng.integers(0, n, 2))) for _ in range(3)]
    for i, j in pairs:
        cols = sorted({i, j})
        Ac = np.asfortranarray(A[:m, cols].cpu().numpy())
        S_hi, S_lo, _ = oracle.gram(Ac)
        a, b = cols.index(i), cols.index(j)
        p2 = pow2_above(Ac)
        err = abs((Gh[i, j] - S_hi[a, b]) + (Gl[i, j] - S_lo[a, b]))
        assert err <= 2.0 ** -88 * m * p2[a] * p2[b], (i, j, err)
    lh, ll, _, _, _, st_o = oracle.jacobi_dd(Gh, Gl)
    assert st_o == 0
    lam_o = np.sort(lh + ll)[::-1]
    sig_o = np.sqrt(lam_o)
    assert np.all(np.abs(sig - sig_o) <= 1e-12 * sig_o), float(np.max(np.abs(sig - sig_o) / sig_o))
    W = V / sig[None, :]
    rows = np.unique(np.concatenate([[0, 1, m - 1], rng.integers(0, m, 61)]))
    A_rows = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    U_ref = oracle.rows_times(np.asfortranarray(A_rows), W, np.arange(len(rows)), 53)
    bound = (n + 1) * UH * (np.abs(A_rows) @ np.abs(W))
    assert np.all(np.abs(U[rows] - U_ref) <= bound)


# ------------------------------------------------------------------ accuracy experiment grid (Sec. 4, Fig. 1)
# (MODE of D, MODE of Sigma) of the 16 test-matrix types; the modes are the five diagonal
# distributions (clustered at 1/kappa, clustered at 1, geometric, arithmetic, log-random).
FIG1_TYPES = [(1, 2), (1, 3), (1, 4), (1, 5), (2, 3), (2, 4), (2, 5), (3, 2), (3, 4), (3, 5), (4, 2), (4, 3), (4, 5),
              (5, 2), (5, 3), (5, 4)]


def test_accuracy_sweep_fig1_grid():
    """The accuracy experiment's grid: n = 64, m = 16 n, kappa(B) in {1e1, ..., 1e5}, kappa(D) in
    {1, 1e2, 1e4, 1e6, 1e8}, the 16 matrix types: 400 matrices A = Q diag(sigma) W^T D (FP32), solved
    in one batched call.  Reference: the oracle's double-double Algorithm 1 on the same FP32
    matrices.  Bound per matrix: 2 u_32 (the cast of sigma) + 16 * 2^-50 kappa(C), C the
    column-scaled exact Gram: the Gram's 2^-50 componentwise error carried through the scaled
    eigenvalue perturbation bound (the u_h kappa(B)^2 term of the analysis)."""
    from concurrent.futures import ThreadPoolExecutor
    m, n = 1024, 64
    gen = torch.Generator().manual_seed(20260311)
    grid = []
    for kB in (1e1, 1e2, 1e3, 1e4, 1e5):
        for kD in (1.0, 1e2, 1e4, 1e6, 1e8):
            for mD, mS in FIG1_TYPES:
                sig = workloads.latm1_mode(mS, n, kB, gen)
                d = workloads.latm1_mode(mD, n, kD, gen)
                grid.append((kB, kD, mD, mS, workloads.make_matrix(m, n, sig, d, 1000 + len(grid), torch.float32)))
    count = len(grid)
    buf = torch.stack([A.T.contiguous() for *_, A in grid]).cuda()  # [count][n][m]: column-major blocks
    As = [buf[k] for k in range(count)]
    sig = [torch.zeros(n, device="cuda") for _ in range(count)]
    Vs = [colmajor(n, n, torch.float32) for _ in range(count)]
    info = torch.zeros(6 * count, dtype=torch.int32, device="cuda")
    h = handle()
    T.tsvd_batch_solve(h, count, As, [m] * count, [n] * count, [m] * count, T.TSVD_FP32, T.TSVD_FP64, sig, Vs,
                       [n] * count, None, None, info)
    torch.cuda.synchronize()
    T.tsvd_destroy(h)
    assert np.all(info.view(count, 6)[:, 0].cpu().numpy() == 0)

    def ref(k):
        A_np = np.asfortranarray(grid[k][4].cpu().numpy()[:m])
        r = oracle.svd(A_np, higher=2)
        G = oracle.gram(A_np)[0]
        dd = np.sqrt(np.diag(G))
        return r["status"], r["sigma_h"] + r["sigma_h_lo"], np.linalg.cond(G / np.outer(dd, dd))

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(ref, range(count)))
    worst = {}
    for k, (st, s_ref, kC) in enumerate(refs):
        assert st == 0
        got = sig[k].cpu().numpy().astype(np.float64)
        rel = float(np.max(np.abs(got - s_ref) / s_ref))
        assert rel <= 2.0 ** -23 + 16 * 2.0 ** -50 * kC, (grid[k][:4], rel, kC)
        kB = grid[k][0]
        if kB <= 1e3:
            assert rel <= 1e-5, (grid[k][:4], rel)  # the stated target for kappa(B) <= 1e3
        worst[kB] = max(worst.get(kB, 0.0), rel)
    print("fig1 grid, Algorithm 1 (FP64 n x n stage): max relative sigma error per kappa(B):",
          ", ".join(f"{kB:.0e}: {worst[kB]:.2e}" for kB in sorted(worst)))
    # the same 400 matrices through Algorithm 2 (eig_variant 3), one solve each, held to Remark 2
    h2 = handle(eig_variant=3)
    worst2 = {}
    for k, (st, s_ref, kC) in enumerate(refs):
        s2 = torch.zeros(n, device="cuda")
        V2 = colmajor(n, n, torch.float32)
        inf2 = torch.zeros(6, dtype=torch.int32, device="cuda")
        T.tsvd_solve(h2, As[k], m, n, m, T.TSVD_FP32, T.TSVD_FP64, s2, V2, n, None, 0, inf2)
        torch.cuda.synchronize()
        assert int(inf2[0].item()) == T.TSVD_OK, grid[k][:4]
        got = s2.cpu().numpy().astype(np.float64)
        rel = float(np.max(np.abs(got - s_ref) / s_ref))
        assert rel <= alg2_bound(math.sqrt(kC), kC), (grid[k][:4], rel, kC)
        worst2[grid[k][0]] = max(worst2.get(grid[k][0], 0.0), rel)
    T.tsvd_destroy(h2)
    print("fig1 grid, Algorithm 2 (FP32 SVD of the cast factor): max relative sigma error per kappa(B):",
          ", ".join(f"{kB:.0e}: {worst2[kB]:.2e}" for kB in sorted(worst2)))


@pytest.mark.parametrize("mode_s,kD", [(1, 1.0), (2, 1.0), (2, 1e6), (1, 1e8)])
def test_solve_clustered_spectra(mode_s, kD):
    """Single solves (tensor-core Gram, cluster Jacobi) on spectra clustered at 1/kappa or at 1
    (63 equal singular values): the Jacobi converges and sigma meets the grid test's bound."""
    m, n, kB = 4096, 64, 1e3
    gen = torch.Generator().manual_seed(77 + mode_s)
    sig_t = workloads.latm1_mode(mode_s, n, kB, gen)
    d = workloads.latm1_mode(3, n, kD, gen)
    A = workloads.make_matrix(m, n, sig_t, d, 4242 + mode_s, torch.float32, device="cuda")
    s, V, U, st, sweeps = gpu_solve(A, m, n, m, want_u=False)
    assert st == T.TSVD_OK, (st, sweeps)
    A_np = workloads.to_numpy_colmajor(A, m)
    r = oracle.svd(A_np, higher=2)
    G = oracle.gram(A_np)[0]
    dd = np.sqrt(np.diag(G))
    kC = np.linalg.cond(G / np.outer(dd, dd))
    s_ref = r["sigma_h"] + r["sigma_h_lo"]
    assert np.max(np.abs(s - s_ref) / s_ref) <= 2.0 ** -23 + 16 * 2.0 ** -50 * kC
