"""tsvd_gram_static, the allocation-free Gram entry point.

It serves callers that cannot call cudaMalloc (a request path that forbids
allocation, a plug-in that may not own device memory, code that may not risk
the implicit synchronisation of cudaMalloc / cudaFree): it takes no handle and
works in one fixed device array inside the library.

The test calls it through the C ABI on two calls in a row, with different
shapes, so the second call must fully replace what the first left in the
shared array:
  * input that TMA can load (16-byte aligned, lda a multiple of 4) runs the
    tcgen05 Gram with tsvd_gram's own split-K plan: the result must be
    bitwise that of the handle-based tsvd_gram, and, as every Gram here, within
    the parity tests' bound 2^-50 (|A|^T |A|) componentwise of the oracle's
    exact sum (FP64 and double-double outputs);
  * unaligned input (lda odd) runs the mma.sync Ozaki Gram: the same bound
    against the oracle and against tsvd_gram;
and an m too large for the array is refused up front.  The file name makes
pytest collect it last; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2603_11953_gb300 as T
from paper_2603_11953_gb300 import build as B
from paper_2603_11953_gb300 import workloads

pytestmark = pytest.mark.gpu


def _gram_with_handle(A, m, n, lda, higher):
    h, _ = T.tsvd_create(0, torch.cuda.current_stream().cuda_stream)
    G = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, lda, T.TSVD_FP32, higher, G, n)
    assert T.tsvd_sync_status(h) == T.TSVD_OK
    T.tsvd_destroy(h)
    return G.cpu().numpy()


def _check_against_oracle(A_np, Gh, Gl):
    S_hi, S_lo, S_abs = oracle.gram(A_np)
    err = np.abs((Gh - S_hi) + (Gl - S_lo))
    assert np.all(err <= 2.0 ** -50 * S_abs), float(np.max(err / np.where(S_abs > 0, S_abs, 1.0)))


def test_gram_static_two_calls_against_gram_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    T.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    # (m, n, lda, higher): aligned FP64 output, then unaligned (lda odd) double-double output
    cases = [(131076, 64, 131076, T.TSVD_FP64), (7001, 17, 7003, T.TSVD_DD)]
    for k, (m, n, lda, higher) in enumerate(cases):
        A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=400 + k, device="cuda", lda=lda)
        G = torch.full((2 * n * n,), float("nan"), dtype=torch.float64, device="cuda")
        info = torch.full((6,), -1, dtype=torch.int32, device="cuda")
        T.tsvd_gram_static(A, m, n, lda, T.TSVD_FP32, higher, G, n, info, stream)
        torch.cuda.synchronize()
        assert int(info[0].item()) == T.TSVD_OK
        g = G.cpu().numpy()
        Gh = g[: n * n].reshape(n, n).T
        Gl = g[n * n:].reshape(n, n).T if higher == T.TSVD_DD else np.zeros((n, n))
        assert np.all(np.isfinite(Gh)) and np.all(np.isfinite(Gl))
        A_np = workloads.to_numpy_colmajor(A, m)
        _check_against_oracle(A_np, Gh, Gl)
        ref = _gram_with_handle(A, m, n, lda, higher)
        if lda % 4 == 0:
            # the same tcgen05 kernel and split-K plan as tsvd_gram: the same bits
            assert np.array_equal(g[: n * n], ref[: n * n])
        else:
            rh = ref[: n * n].reshape(n, n).T
            S_abs = oracle.gram(A_np)[2]
            assert np.all(np.abs(Gh - rh) <= 2.0 ** -49 * S_abs)
    # an m whose partials would not fit the fixed array is refused up front
    A, _ = workloads.small_case(1024, 64, seed=5, device="cuda")
    G = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    too_many_rows = 8_323_072 + 128
    st = T.tsvd_gram_static(A, too_many_rows, 64, too_many_rows, T.TSVD_FP32, T.TSVD_FP64, G, 64,
                            None, stream, check=False)
    assert st == T.TSVD_ERR_UNSUPPORTED
