"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties one oracle function to an independent fact: exact rational
arithmetic (Python ``fractions``), closed forms, exact root isolation
(sympy), LAPACK's SVD, Weyl's perturbation bound, and invariants of the Gram
matrix.  A dropped term, wrong sign, wrong index or transposed operand in the
oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def exact_gram(A):
    """sum_r A[r,i] A[r,j] as Fractions (independent of the oracle)."""
    m, n = A.shape
    F = [[Fraction(float(A[r, c])) for c in range(n)] for r in range(m)]
    return [[sum(F[r][i] * F[r][j] for r in range(m)) for j in range(n)] for i in range(n)]


def round_frac(x: Fraction, p: int) -> float:
    """Round a rational to p significant bits, ties to even (exact)."""
    if x == 0:
        return 0.0
    sign = -1.0 if x < 0 else 1.0
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length() - p
    two = Fraction(2)
    while x / two ** e >= 2 ** p:
        e += 1
    while x / two ** e < 2 ** (p - 1):
        e -= 1
    q = x / two ** e
    k = q.numerator // q.denominator
    r = q - k
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and k % 2 == 1):
        k += 1
    return sign * math.ldexp(k, e)


def wide_random(m, n, seed, dtype=np.float32, erange=30):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-erange, erange, size=(m, n)))
    return np.asfortranarray(A.astype(dtype))


# ---------------------------------------------------------------- Gram (Alg. 1 lines 1-2)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gram_equals_exact_rational_sum(dtype):
    A = wide_random(40, 4, 11, dtype)
    A[7] = -A[3]  # exact cancellation pairs
    Gh, Gl, Ga = oracle.gram(A)
    S = exact_gram(A)
    for i in range(4):
        for j in range(4):
            hi = round_frac(S[i][j], 53)
            lo = round_frac(S[i][j] - Fraction(hi), 53)
            assert Gh[i, j] == hi and Gl[i, j] == lo, (i, j)
            assert Ga[i, j] >= abs(Gh[i, j]) * (1 - 1e-15)


def test_gram_golden_integer_fixture():
    rows = open(os.path.join(GOLDEN, "gram_integer_3x2.txt")).read().split("\n")
    rows = [r for r in rows if r and not r.startswith("#")]
    ia, im = rows.index("A"), rows.index("M")
    A = np.array([[float(x) for x in r.split()] for r in rows[ia + 1:im]], dtype=np.float32)
    M = np.array([[float(x) for x in r.split()] for r in rows[im + 1:]])
    Gh, Gl, _ = oracle.gram(A)
    assert np.array_equal(Gh, M) and not Gl.any()
    res = oracle.svd(A, higher=1)
    lam = [(91 + math.sqrt(8185)) / 2, (91 - math.sqrt(8185)) / 2]
    assert res["status"] == 0
    np.testing.assert_allclose(res["sigma_h"], np.sqrt(lam), rtol=1e-14)


def test_gram_invariants():
    A = wide_random(64, 5, 3)
    Gh, Gl, _ = oracle.gram(A)
    perm = np.random.default_rng(0).permutation(64)
    Gp, Glp, _ = oracle.gram(np.asfortranarray(A[perm]))
    assert np.array_equal(Gh, Gp) and np.array_equal(Gl, Glp)
    # power-of-two column scaling is exact: G_ij -> 2^(p_i + p_j) G_ij
    p = np.array([3, -7, 0, 12, -1])
    As = np.asfortranarray((A * np.exp2(p)).astype(np.float32))
    Gs, Gls, _ = oracle.gram(As)
    scale = np.exp2(p[:, None] + p[None, :])
    assert np.array_equal(Gs, Gh * scale) and np.array_equal(Gls, Gl * scale)
    # stacking [A; A] doubles the exact sum (and both parts of the DD)
    G2, Gl2, _ = oracle.gram(np.asfortranarray(np.vstack([A, A])))
    assert np.array_equal(G2, 2 * Gh) and np.array_equal(Gl2, 2 * Gl)
    # flipping the sign of column 2 flips row/column 2 off the diagonal
    Af = A.copy(order="F")
    Af[:, 2] *= -1
    Gf, _, _ = oracle.gram(Af)
    sgn = np.ones(5)
    sgn[2] = -1
    assert np.array_equal(Gf, Gh * np.outer(sgn, sgn))
    # transposed operands would break symmetry of a non-square product: G is symmetric
    assert np.array_equal(Gh, Gh.T)


def test_gram_orthogonal_columns_exact():
    # Sylvester-Hadamard H_8 / sqrt(8)-free: H^T H = 8 I exactly
    H = np.array([[1.0]])
    for _ in range(3):
        H = np.block([[H, H], [H, -H]])
    A = np.asfortranarray((H[:, :5] * 0.125).astype(np.float32))
    Gh, Gl, _ = oracle.gram(A)
    assert np.array_equal(Gh, 0.125 * np.eye(5)) and not Gl.any()
    res = oracle.svd(A, higher=1)
    np.testing.assert_array_equal(res["sigma_h"], np.full(5, math.sqrt(0.125)))


# ---------------------------------------------------------------- rounding to working (line 6)
def test_rows_times_is_exact_dot_rounded_once():
    A = wide_random(30, 6, 5, erange=8)
    W = np.asfortranarray(np.random.default_rng(9).standard_normal((6, 6)).astype(np.float32).astype(np.float64))
    rows = np.array([0, 3, 29, 17])
    for p in (24, 53):
        out = oracle.rows_times(A, W, rows, p)
        for k, r in enumerate(rows):
            for j in range(6):
                s = sum(Fraction(float(A[r, c])) * Fraction(float(W[c, j])) for c in range(6))
                assert out[k, j] == round_frac(s, p), (p, r, j)


def test_explicit_u_orthonormal_columns():
    # A = Q diag(s) with exactly orthogonal Q (Hadamard/8): U must be Q exactly (up to signs)
    H = np.array([[1.0]])
    for _ in range(4):
        H = np.block([[H, H], [H, -H]])
    Q = H[:, :4] * 0.25  # 16 x 4, Q^T Q = I exactly
    s = np.array([8.0, 4.0, 2.0, 0.5])
    A = np.asfortranarray(Q * s)
    res = oracle.svd(A, higher=1)
    np.testing.assert_array_equal(res["sigma_h"], s)
    np.testing.assert_array_equal(np.abs(res["V_h"]), np.eye(4))
    uh, ul = oracle.rows_explicit_u(A, res["V_h"], None, res["sigma_h"], None, np.arange(16))
    np.testing.assert_array_equal(np.abs(uh), np.abs(Q))


def test_explicit_u_is_exact_rational_quotient():
    """Alg. 1 line 6 / eq. (AV-0) with the higher-precision factors: u_rj = (sum_c a_rc v_cj) / sigma_j
    with v = V_hi + V_lo and sigma = sig_hi + sig_lo, against exact rationals.  V is a full,
    non-symmetric matrix (a transposed index changes the answer), V_lo and sig_lo are non-zero (a
    dropped low part changes it by ~2^-60 relative, far above the 2^-98 tolerance) and sigma is not
    a power of two."""
    rng = np.random.default_rng(17)
    m, n = 9, 5
    A = np.asfortranarray(rng.standard_normal((m, n)).astype(np.float32))
    V_hi = np.asfortranarray(rng.standard_normal((n, n)))
    V_lo = np.asfortranarray(V_hi * rng.uniform(0.25, 0.5, (n, n)) * 2.0 ** -58)
    sig_hi = rng.uniform(0.3, 3.0, n)
    sig_lo = sig_hi * rng.uniform(-0.5, 0.5, n) * 2.0 ** -56
    rows = np.array([0, 4, 8, 2])
    oh, ol = oracle.rows_explicit_u(A, V_hi, V_lo, sig_hi, sig_lo, rows)
    for k, r in enumerate(rows):
        for j in range(n):
            dot = sum(Fraction(float(A[r, c])) * (Fraction(V_hi[c, j]) + Fraction(V_lo[c, j])) for c in range(n))
            u = dot / (Fraction(sig_hi[j]) + Fraction(sig_lo[j]))
            got = Fraction(oh[k, j]) + Fraction(ol[k, j])
            assert abs(got - u) <= abs(u) * Fraction(1, 2 ** 98), (r, j)
            assert oh[k, j] == round_frac(u, 53) or abs(Fraction(oh[k, j]) - u) <= abs(u) * Fraction(1, 2 ** 52)
    # the low parts matter at this tolerance: leaving them out moves the result
    oh0, ol0 = oracle.rows_explicit_u(A, V_hi, None, sig_hi, None, rows)
    assert not (np.array_equal(oh0, oh) and np.array_equal(ol0, ol))


def test_round_dd_single_rounding():
    """Alg. 1 lines 4-5 (cast to the working precision): RN-even of the exact hi + lo, one rounding.
    The FP32 midpoints are the cases a double rounding (DD -> FP64 -> FP32) gets wrong."""
    one = 1.0
    mid = one + 2.0 ** -24            # exactly halfway between 1 and 1 + 2^-23 (FP32)
    his = np.array([mid, mid, mid, -mid, 3.0 + 2.0 ** -22, 0.1, 1e-3, 2.0 ** -30 * (1 + 2.0 ** -24)])
    los = np.array([2.0 ** -80, -2.0 ** -80, 0.0, -2.0 ** -80, 2.0 ** -75, 1e-20, -3e-22, 2.0 ** -100])
    out24 = oracle.round_dd(his, los, 24)
    out53 = oracle.round_dd(his, los, 53)
    for h, l, o24, o53 in zip(his, los, out24, out53):
        x = Fraction(h) + Fraction(l)
        assert o24 == round_frac(x, 24), (h, l)
        assert o53 == round_frac(x, 53), (h, l)
    assert out24[0] == 1.0 + 2.0 ** -23 and out24[1] == 1.0 and out24[2] == 1.0  # above, below, tie to even
    assert out24[3] == -(1.0 + 2.0 ** -23)
    assert np.float64(np.float32(mid)) == 1.0  # what a cast through FP64 alone would give for case 0


@pytest.mark.parametrize("dtype,higher", [(np.float32, 1), (np.float32, 2), (np.float64, 2), (np.float64, 1)])
def test_svd_working_precision_casts(dtype, higher):
    """oracle_svd's sigma_w, V_w and W_w are the single RN-even roundings (to A's precision) of the
    exact higher-precision sigma_h = sig_hi + sig_lo, V_h = V_hi + V_lo, and of V_w / sigma_w."""
    A = wide_random(30, 4, 23, dtype, erange=4)
    res = oracle.svd(A, higher=higher)
    assert res["status"] == 0
    p = 24 if dtype == np.float32 else 53
    n = A.shape[1]
    for j in range(n):
        s = Fraction(res["sigma_h"][j]) + Fraction(res["sigma_h_lo"][j])
        assert res["sigma_w"][j] == round_frac(s, p), j
        for i in range(n):
            v = Fraction(res["V_h"][i, j]) + Fraction(res["V_h_lo"][i, j])
            assert res["V_w"][i, j] == round_frac(v, p), (i, j)
            q = Fraction(res["V_w"][i, j]) / Fraction(res["sigma_w"][j])
            assert res["W_w"][i, j] == round_frac(q, p), (i, j)
    # W is V_w / sigma_w column by column, not row by row (a transposed sigma index fails here)
    assert not np.allclose(res["W_w"], res["V_w"] / res["sigma_w"][:, None])


# ---------------------------------------------------------------- Jacobi (Alg. 1 line 3)
def test_jacobi_n1_and_2x2_closed_form():
    lam, V, sw, st = oracle.jacobi_fp64(np.array([[7.25]]))
    assert st == 0 and lam[0] == 7.25 and V[0, 0] == 1.0
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    a, b, c = 3.0, 1.25, 0.75  # SPD: det = 2.25 - 1.5625 > 0
    lam, V, sw, st = oracle.jacobi_fp64(np.array([[a, b], [b, c]]))
    mid = (Decimal(a) + Decimal(c)) / 2
    rad = (((Decimal(a) - Decimal(c)) / 2) ** 2 + Decimal(b) ** 2).sqrt()
    exact = sorted([float(mid + rad), float(mid - rad)], reverse=True)
    rho = b / math.sqrt(a * c)  # scaled matrix [[1, rho], [rho, 1]], kappa = (1+rho)/(1-rho)
    kC = (1 + rho) / (1 - rho)
    np.testing.assert_allclose(sorted(lam, reverse=True), exact, rtol=16 * kC * 2.0 ** -53)
    # eigenvector of the larger eigenvalue, from (M - lam I) v = 0: v ~ (b, lam - a)
    i = int(np.argmax(lam))
    v = V[:, i] * np.sign(V[0, i])
    ref = np.array([b, exact[0] - a])
    np.testing.assert_allclose(v, ref / np.linalg.norm(ref), rtol=1e-15)


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (4, 3), (4, 4)])
def test_brute_force_exact_eigenvalues(n, seed):
    sympy = pytest.importorskip("sympy")
    A = wide_random(6, n, seed, erange=3)
    S = exact_gram(A)
    Ms = sympy.Matrix(n, n, lambda i, j: sympy.Rational(S[i][j].numerator, S[i][j].denominator))
    lam = sympy.Symbol("lam")
    roots = sympy.Poly(Ms.charpoly(lam).as_expr(), lam).real_roots()
    exact_sigma = sorted([float(sympy.sqrt(r).evalf(40)) for r in roots], reverse=True)
    res = oracle.svd(A, higher=1)
    assert res["status"] == 0
    C = np.array(Ms.evalf(30).tolist(), dtype=float)
    d = np.sqrt(np.diag(C))
    kC = np.linalg.cond(C / np.outer(d, d))
    np.testing.assert_allclose(res["sigma_h"], exact_sigma, rtol=64 * 2.0 ** -53 * kC)
    res2 = oracle.svd(A, higher=2)
    exact_hi = sorted([sympy.sqrt(r).evalf(40) for r in roots], reverse=True)
    for k in range(n):
        err = abs(sympy.Float(res2["sigma_h"][k], 40) + sympy.Float(res2["sigma_h_lo"][k], 40) - exact_hi[k])
        assert float(err / exact_hi[k]) < 1e-28 * kC, (k, float(err / exact_hi[k]))


def test_graded_matrix_relative_accuracy():
    """M = D C D with C well conditioned and D spanning 1e+-8: Jacobi with the
    scaled stopping test keeps every eigenvalue to high RELATIVE accuracy
    (the property Sec. 2.1 picks two-sided Jacobi for)."""
    sympy = pytest.importorskip("sympy")
    C = np.array([[1.0, 0.3, -0.2], [0.3, 1.0, 0.25], [-0.2, 0.25, 1.0]])
    D = np.array([1e8, 1.0, 1e-8])
    M = C * np.outer(D, D)
    Ms = sympy.Matrix(3, 3, lambda i, j: sympy.Rational(Fraction(float(M[i, j]))))
    lam = sympy.Symbol("lam")
    roots = sorted(sympy.Poly(Ms.charpoly(lam).as_expr(), lam).real_roots(), key=lambda r: -float(r.evalf(30)))
    exact = np.array([float(r.evalf(40)) for r in roots])
    lam_o, V, sw, st = oracle.jacobi_fp64(M)
    assert st == 0
    got = np.sort(lam_o)[::-1]
    np.testing.assert_allclose(got, exact, rtol=1e-14)  # smallest is ~1e-16 of the largest


def test_jacobi_residual_orthogonality_and_vs_lapack():
    rng = np.random.default_rng(7)
    n = 24
    X = rng.standard_normal((200, n))
    M = X.T @ X
    lam, V, sw, st = oracle.jacobi_fp64(M)
    assert st == 0 and sw < 15
    scale = np.abs(lam).max()
    assert np.abs(M @ V - V * lam).max() <= 8 * n * 2.0 ** -53 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 8 * n * 2.0 ** -53
    ref = np.linalg.eigvalsh(M)[::-1]
    np.testing.assert_allclose(np.sort(lam)[::-1], ref, rtol=1e-12)
    # full pipeline vs LAPACK SVD on the same (well-conditioned) matrix
    A = np.asfortranarray(X)
    res = oracle.svd(A, higher=1)
    np.testing.assert_allclose(res["sigma_h"], np.linalg.svd(A, compute_uv=False), rtol=1e-13)
    # sort and sign rule
    assert np.all(np.diff(res["sigma_h"]) <= 0)
    for j in range(n):
        col = res["V_h"][:, j]
        k = int(np.argmax(np.abs(col)))
        assert col[k] > 0


def test_known_sigma_weyl_bound():
    """D = I: A64 = Q diag(sigma) W^T has singular values sigma (to FP64
    rounding); rounding to FP32 moves each by at most ||A32 - A64||_2 (Weyl)."""
    import torch
    from paper_2603_11953_gb300 import workloads
    A, meta = workloads.small_case(2000, 12, kappa_sigma=1e3, logd=0.0, seed=5, dtype=torch.float64)
    A64 = workloads.to_numpy_colmajor(A, 2000)
    A32 = np.asfortranarray(A64.astype(np.float32))
    res = oracle.svd(A32, higher=1)
    sig = meta["sigma"].numpy()
    weyl = np.linalg.norm(A32.astype(np.float64) - A64, 2)
    assert res["status"] == 0
    assert np.all(np.abs(res["sigma_h"] - sig) <= weyl + 1e-14)
    res64 = oracle.svd(A64, higher=2)
    np.testing.assert_allclose(res64["sigma_h"], sig, rtol=1e-13)


def test_not_full_rank_and_nonfinite_statuses():
    A = np.asfortranarray(np.ones((8, 2), dtype=np.float32))  # rank 1
    res = oracle.svd(A, higher=1)
    assert res["status"] == oracle.NOT_FULL_RANK
    A[3, 1] = np.inf
    with pytest.raises(ValueError):
        oracle.gram(A)


def test_dd_jacobi_reaches_double_double_accuracy():
    """FP64-working path: Gram in DD and Jacobi in DD reproduce sigma of a
    D = I matrix far below FP64 resolution (checked against DD-exact sympy)."""
    sympy = pytest.importorskip("sympy")
    A = wide_random(9, 3, 21, dtype=np.float64, erange=2)
    S = exact_gram(A)
    Ms = sympy.Matrix(3, 3, lambda i, j: sympy.Rational(S[i][j].numerator, S[i][j].denominator))
    lam = sympy.Symbol("lam")
    roots = sympy.Poly(Ms.charpoly(lam).as_expr(), lam).real_roots()
    exact = sorted([sympy.sqrt(r).evalf(45) for r in roots], reverse=True)
    res = oracle.svd(A, higher=2)
    for k in range(3):
        got = sympy.Float(res["sigma_h"][k], 45) + sympy.Float(res["sigma_h_lo"][k], 45)
        assert float(abs(got - exact[k]) / exact[k]) < 1e-29


def test_dd_jacobi_graded_relative_accuracy():
    """The double-double Algorithm 1 on a strongly graded FP64 matrix (columns scaled over 12
    decades, sigma_n / sigma_1 ~ 1e-6 after scaling): every sigma, the smallest included, to a
    relative 1e-18 of the exact value (exact rational Gram, exact root isolation).  This is the
    truth the FP64-working GPU tests compare against at kappa(B) up to 1e6."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(33)
    m, n = 10, 4
    B = rng.standard_normal((m, n))
    B[:, 3] = B[:, 2] + 1e-6 * rng.standard_normal(m)  # nearly dependent pair: kappa(B) ~ 1e6
    A = np.asfortranarray(B * np.array([1e6, 1e2, 1.0, 1e-6]))
    S = exact_gram(A)
    Ms = sympy.Matrix(n, n, lambda i, j: sympy.Rational(S[i][j].numerator, S[i][j].denominator))
    lam = sympy.Symbol("lam")
    roots = sympy.Poly(Ms.charpoly(lam).as_expr(), lam).real_roots()
    exact = sorted([sympy.sqrt(r).evalf(50) for r in roots], reverse=True)
    res = oracle.svd(A, higher=2)
    assert res["status"] == 0
    for k in range(n):
        got = sympy.Float(res["sigma_h"][k], 50) + sympy.Float(res["sigma_h_lo"][k], 50)
        assert float(abs(got - exact[k]) / exact[k]) < 1e-18, (k, float(abs(got - exact[k]) / exact[k]))
    # the FP64 n x n stage on the same exact Gram loses ~u kappa(B)^2 on the smallest sigma
    res1 = oracle.svd(A, higher=1)
    assert float(abs(sympy.Float(res1["sigma_h"][n - 1], 50) - exact[n - 1]) / exact[n - 1]) > 1e-15


# ---------------------------------------------------------------- Algorithm 2 (Cholesky, cast, SVD of R)
def test_alg2_exact_factor_matches_lapack_svd():
    """M = R0^T R0 with a small-integer upper triangular R0: every step of the FP64 Cholesky is
    exact, so R = R0 (FP32-exact, the cast changes nothing) and Algorithm 2's sigma and V are the
    singular values and right singular vectors of R0, checked against LAPACK's SVD."""
    rng = np.random.default_rng(1)
    n = 7
    R0 = np.triu(rng.integers(-5, 6, (n, n)).astype(float))
    np.fill_diagonal(R0, np.arange(3, 3 + n))
    M = R0.T @ R0
    res = oracle.alg2(M, working=0)
    assert res["status"] == 0
    _, s, Vt = np.linalg.svd(R0)
    np.testing.assert_allclose(res["sigma"], s, rtol=1e-14)
    for j in range(n):  # same subspace, sign fixed by the sign rule
        v = Vt[j] * np.sign(Vt[j][np.argmax(np.abs(Vt[j]))])
        np.testing.assert_allclose(res["V"][:, j], v, atol=1e-13)
    # M V = V diag(sigma^2): the eigen-decomposition of M the algorithm promises
    np.testing.assert_allclose(M @ res["V"], res["V"] * res["sigma"] ** 2, atol=1e-11 * s[0] ** 2)


def test_alg2_casts_r_to_working_precision():
    """Line 2 of Algorithm 2 rounds R_h to the working precision: for FP32 working, sigma is the
    SVD of fl32(R_h) (LAPACK on the rounded factor), not of R_h itself; for FP64 working the cast
    is the identity and sigma^2 are the eigenvalues of M."""
    rng = np.random.default_rng(5)
    n = 9
    B = rng.standard_normal((40, n)) * np.exp2(rng.integers(-6, 6, n))
    M = B.T @ B
    Rh = np.linalg.cholesky(M).T
    s32 = np.linalg.svd(Rh.astype(np.float32).astype(np.float64), compute_uv=False)
    s64 = np.linalg.svd(Rh, compute_uv=False)
    res = oracle.alg2(M, working=0)
    assert res["status"] == 0
    np.testing.assert_allclose(res["sigma"], s32, rtol=1e-12)
    assert np.max(np.abs(res["sigma"] - s64) / s64) > 1e-10  # the cast is really applied
    res64 = oracle.alg2(M, working=1)
    lam = np.sort(np.linalg.eigvalsh(M))[::-1]  # LAPACK: absolute accuracy ~ n u lambda_max
    np.testing.assert_allclose(res64["sigma"] ** 2, lam, rtol=1e-12, atol=64 * 2.0 ** -53 * lam[0])


def test_alg2_not_positive_definite():
    M = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 3.0]])  # rank 2 block
    assert oracle.alg2(M)["status"] == oracle.NOT_FULL_RANK


# ---------------------------------------------------------------- mixed precision Cholesky QR (Sec. 3.1)
def test_cholesky_exact_factor_and_lapack():
    rng = np.random.default_rng(2)
    n = 8
    R0 = np.triu(rng.integers(-4, 5, (n, n)).astype(float))
    np.fill_diagonal(R0, np.arange(2, 2 + n))
    R, st = oracle.cholesky(R0.T @ R0)
    assert st == 0 and np.array_equal(R, R0)  # every step exact on small integers
    B = rng.standard_normal((30, n))
    M = B.T @ B
    R, st = oracle.cholesky(M)
    np.testing.assert_allclose(R, np.linalg.cholesky(M).T, rtol=1e-12, atol=1e-12)
    assert oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == oracle.NOT_FULL_RANK


def test_cholqr_rows_exact_rational_solution():
    """q R = a solved exactly (Fractions, forward substitution) and rounded once: the oracle's
    double-double substitution rounded to 24 and to 53 bits gives the same values."""
    rng = np.random.default_rng(8)
    m, n = 7, 5
    A = np.asfortranarray(rng.standard_normal((m, n)).astype(np.float32))
    Rw = np.triu(rng.standard_normal((n, n))) + np.diag(np.full(n, 2.0))
    Rw = Rw.astype(np.float32).astype(np.float64)
    rows = np.array([0, 3, 6])
    for p in (24, 53):
        out = oracle.cholqr_rows(A, Rw, rows, p)
        for k, r in enumerate(rows):
            q = []
            for j in range(n):
                acc = Fraction(float(A[r, j])) - sum(q[i] * Fraction(Rw[i, j]) for i in range(j))
                q.append(acc / Fraction(Rw[j, j]))
                assert out[k, j] == round_frac(q[j], p), (p, r, j)


def test_cholqr_orthogonality_theorem3():
    """Theorem 3: with the Gram and the Cholesky factorization at u_h = 2^-53 <= u^2 and Q from
    Q R = A at u = 2^-24, ||Q^T Q - I|| is O(u) kappa(B), not O(u) kappa(B)^2 as with u_h = u: a
    graded A with kappa(B) ~ 1e3 and kappa(A) ~ 1e7 keeps Q orthogonal to ~1e-4 (c = 2n)."""
    import torch
    from paper_2603_11953_gb300 import workloads
    m, n = 3000, 10
    A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=2.0, seed=19)
    A_np = workloads.to_numpy_colmajor(A, m)
    M = oracle.gram(A_np)[0]
    R, st = oracle.cholesky(M)
    assert st == 0
    Rw = R.astype(np.float32).astype(np.float64)
    Q = oracle.cholqr_rows(A_np, Rw, np.arange(m), 24)
    d = np.sqrt(np.diag(M))
    kB = math.sqrt(np.linalg.cond(M / np.outer(d, d)))
    orth = np.linalg.norm(Q.T @ Q - np.eye(n), 2)
    assert orth <= 2 * n * 2.0 ** -24 * kB, (orth, kB)
