"""Seeded synthetic inputs shaped like the paper's test matrices.

This module holds no arithmetic of the SVD method itself: it only builds
inputs.  The CUDA path (through the C-ABI) and the CPU oracle both consume
what it produces, so it is the one module the two sides share.

Recipe (the paper's A = B D construction, Section 4.1, with B = Q diag(sigma) W^T):
  Q     = Q factor of a Householder QR of an m x n N(0,1) matrix (FP64),
  W     = Haar-random orthogonal n x n (QR of N(0,1), signs fixed by diag(R)),
  sigma = the requested spectrum (geometric / log-uniform / Table 3 modes),
  D     = diag(10^u_j), u_j ~ U(-a, a) independently per column,
  A     = RN_working(Q diag(sigma) W^T D).
With D = I the singular values of the FP64 matrix are exactly sigma (up to the
FP64 rounding of the product); with D != I they are not, and the oracle is the
reference.  The paper measures only on random matrices of this form; no
public dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

SEED_BASE = 20260311


@dataclasses.dataclass
class Spec:
    name: str
    m: int
    n: int
    dtype: torch.dtype
    spectrum: str          # "geometric" | "loguniform"
    sigma_min: float       # smallest sigma (largest is 1)
    logd: float            # D = 10^U(-logd, logd)
    seed: int


# The five workloads.  Index i uses seed SEED_BASE + i.
CONFIGS = {
    "plain_20000x16_fp32": Spec("plain_20000x16_fp32", 20000, 16, torch.float32, "geometric", 1e-3, 3.0, SEED_BASE + 0),
    "ozaki_4194304x64_fp32": Spec("ozaki_4194304x64_fp32", 4194304, 64, torch.float32, "geometric", 1e-4, 4.0, SEED_BASE + 1),
    "wide_1048576x256_fp32": Spec("wide_1048576x256_fp32", 1048576, 256, torch.float32, "loguniform", 1e-5, 3.0, SEED_BASE + 2),
    "stress_16777216x32_fp64": Spec("stress_16777216x32_fp64", 16777216, 32, torch.float64, "geometric", 1e-6, 6.0, SEED_BASE + 4),
}
BATCH_SEED = SEED_BASE + 3


def spectrum(kind: str, n: int, sigma_min: float, gen: torch.Generator) -> torch.Tensor:
    """sigma_1 = 1 >= ... >= sigma_n = sigma_min (geometric) or log-uniform draws."""
    if n == 1:
        return torch.ones(1, dtype=torch.float64)
    if kind == "geometric":
        k = torch.arange(n, dtype=torch.float64)
        return sigma_min ** (k / (n - 1))
    if kind == "loguniform":
        u = torch.rand(n, generator=gen, dtype=torch.float64)
        s = 10.0 ** (math.log10(sigma_min) * u)
        s[0], s[-1] = 1.0, sigma_min  # pin the range so kappa(Sigma) is as stated
        return torch.sort(s, descending=True).values
    raise ValueError(kind)


def latm1_mode(mode: int, n: int, kappa: float, gen: torch.Generator) -> torch.Tensor:
    """The five diagonal distributions of Table 3 (d(1) = 1, d(n) ~ 1/kappa)."""
    i = torch.arange(1, n + 1, dtype=torch.float64)
    if mode == 1:
        d = torch.full((n,), 1.0 / kappa, dtype=torch.float64); d[0] = 1.0
    elif mode == 2:
        d = torch.ones(n, dtype=torch.float64); d[-1] = 1.0 / kappa
    elif mode == 3:
        d = kappa ** (-(i - 1) / max(n - 1, 1))
    elif mode == 4:
        d = 1.0 - (i - 1) / max(n - 1, 1) * (1.0 - 1.0 / kappa)
    elif mode == 5:
        u = torch.rand(n, generator=gen, dtype=torch.float64)
        d = torch.exp(-math.log(kappa) * u)
    else:
        raise ValueError(mode)
    return d


def haar_orthogonal(n: int, gen: torch.Generator) -> torch.Tensor:
    X = torch.randn(n, n, generator=gen, dtype=torch.float64)
    Qw, Rw = torch.linalg.qr(X)
    return Qw * torch.sign(torch.diagonal(Rw)).where(torch.diagonal(Rw) != 0, torch.ones(()).double())


def make_matrix(m: int, n: int, sigma: torch.Tensor, d: torch.Tensor, seed: int,
                dtype=torch.float32, device="cpu", lda: int | None = None) -> torch.Tensor:
    """A = RN(Q diag(sigma) W^T diag(d)), column-major with leading dimension lda.

    Returned as a (n, lda) row-major tensor view transposed to (lda, n) so that
    column j is contiguous: the caller passes A.data_ptr(), m, n, lda.
    """
    lda = m if lda is None else lda
    gen = torch.Generator(device="cpu").manual_seed(seed)
    W = haar_orthogonal(n, gen)
    # Built on the CPU (LAPACK QR) whatever the target device, so the same
    # seed gives the same matrix everywhere; only the result is moved.
    G = torch.randn(m, n, generator=gen, dtype=torch.float64)
    Q, _ = torch.linalg.qr(G)
    del G
    A64 = (Q * sigma) @ W.T
    del Q
    A64 *= d
    store = torch.zeros(n, lda, dtype=dtype)
    store[:, :m] = A64.T.to(dtype)
    del A64
    return store.to(device).T  # shape (lda, n), column-major storage


def make_config(spec: Spec, device="cpu", m: int | None = None, seed_offset: int = 0):
    """Build the workload of `spec` (optionally with fewer rows, same recipe)."""
    m = spec.m if m is None else m
    gen = torch.Generator(device="cpu").manual_seed(spec.seed + 104729 * seed_offset)
    sig = spectrum(spec.spectrum, spec.n, spec.sigma_min, gen)
    u = (torch.rand(spec.n, generator=gen, dtype=torch.float64) * 2.0 - 1.0) * spec.logd
    d = 10.0 ** u
    A = make_matrix(m, spec.n, sig, d, spec.seed + 104729 * seed_offset, spec.dtype, device)
    return A, dict(sigma=sig, d=d, m=m, n=spec.n, lda=m)


def make_batch(count: int = 4096, device="cpu", m_lo: int = 1024, m_hi: int = 65536,
               n_choices=(8, 16, 24, 32, 48, 64), seed: int = BATCH_SEED,
               dtype=torch.float32, max_total_rows: int | None = None):
    """Ragged batch: m log-uniform in [m_lo, m_hi], n uniform over n_choices,
    sigma geometric with sigma_n/sigma_1 log-uniform in [1e-5, 1e-2],
    D = 10^U(-3, 3), lda = m rounded up to a multiple of 4.

    All instances live in one device buffer; each base is 256-byte aligned.
    Returns (buffer, list of dict(offset_elems, m, n, lda, sigma, d)).
    """
    gen = torch.Generator(device="cpu").manual_seed(seed)
    metas = []
    esize = torch.empty((), dtype=dtype).element_size()
    align = 256 // esize
    off = 0
    for k in range(count):
        lm = math.log(m_lo) + (math.log(m_hi) - math.log(m_lo)) * torch.rand(1, generator=gen, dtype=torch.float64).item()
        m = int(round(math.exp(lm)))
        n = int(n_choices[int(torch.randint(len(n_choices), (1,), generator=gen).item())])
        m = max(m, n)
        if max_total_rows is not None:
            m = min(m, max_total_rows)
        ratio = 10.0 ** (-2.0 - 3.0 * torch.rand(1, generator=gen, dtype=torch.float64).item())
        sig = ratio ** (torch.arange(n, dtype=torch.float64) / max(n - 1, 1))
        u = (torch.rand(n, generator=gen, dtype=torch.float64) * 2.0 - 1.0) * 3.0
        lda = (m + 3) // 4 * 4
        metas.append(dict(offset=off, m=m, n=n, lda=lda, sigma=sig, d=10.0 ** u, seed=seed * 7 + k))
        off += (lda * n + align - 1) // align * align
    buf = torch.zeros(off, dtype=dtype, device=device)
    for mt in metas:
        A = make_matrix(mt["m"], mt["n"], mt["sigma"], mt["d"], mt["seed"], dtype, device, lda=mt["lda"])
        buf[mt["offset"]:mt["offset"] + mt["lda"] * mt["n"]] = A.T.reshape(-1)
    return buf, metas


def small_case(m: int, n: int, kappa_sigma: float = 1e3, logd: float = 3.0, seed: int = 1,
               dtype=torch.float32, spectrum_kind: str = "geometric", lda: int | None = None,
               device="cpu"):
    """Small instance of the same recipe for parity tests."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    sig = spectrum(spectrum_kind, n, 1.0 / kappa_sigma, gen)
    u = (torch.rand(n, generator=gen, dtype=torch.float64) * 2.0 - 1.0) * logd
    d = 10.0 ** u
    A = make_matrix(m, n, sig, d, seed, dtype, device, lda=lda)
    return A, dict(sigma=sig, d=d)


def to_numpy_colmajor(A: torch.Tensor, m: int) -> np.ndarray:
    """(lda, n) column-major tensor -> numpy (m, n) Fortran-ordered copy."""
    return np.asfortranarray(A[:m].detach().cpu().numpy())
