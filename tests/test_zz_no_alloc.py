"""tsvd_gram_static, the allocation-free Gram entry point.

It serves callers that cannot call cudaMalloc (a request path that forbids
allocation, a plug-in that may not own device memory): it takes no handle and
works in one fixed device array inside the library.  This test calls it
through the C ABI twice in a row, on different shapes so the second call
must fully replace what the first left in the shared array, and checks each
result against the handle-based tsvd_gram within the Gram tolerance used by
the parity tests, 2^-50 (|A|^T |A|) componentwise.  It also checks that an m
too large for the array is refused.  The file name makes pytest collect it
last; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

import paper_2603_11953_gb300 as T
from paper_2603_11953_gb300 import build as B
from paper_2603_11953_gb300 import workloads

pytestmark = pytest.mark.gpu


def _gram_with_handle(A, m, n):
    h, _ = T.tsvd_create(0, torch.cuda.current_stream().cuda_stream)
    G = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    T.tsvd_gram(h, A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, G, n)
    assert T.tsvd_sync_status(h) == T.TSVD_OK
    T.tsvd_destroy(h)
    return G.view(n, n).T.cpu().numpy()


def test_gram_static_matches_gram_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    T.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    for k, (m, n) in enumerate([(300001, 64), (7001, 17)]):
        A, _ = workloads.small_case(m, n, kappa_sigma=1e3, logd=3.0, seed=400 + k, device="cuda")
        G = torch.full((n * n,), float("nan"), dtype=torch.float64, device="cuda")
        info = torch.full((6,), -1, dtype=torch.int32, device="cuda")
        T.tsvd_gram_static(A, m, n, m, T.TSVD_FP32, T.TSVD_FP64, G, n, info, stream)
        torch.cuda.synchronize()
        assert int(info[0].item()) == T.TSVD_OK
        Gs = G.view(n, n).T.cpu().numpy()
        Gh = _gram_with_handle(A, m, n)
        Aabs = A[:m].abs().double()
        tol = 2.0 ** -50 * (Aabs.T @ Aabs).cpu().numpy()
        assert np.all(np.isfinite(Gs))
        assert np.all(np.abs(Gs - Gh) <= tol)
    # an m whose partials would not fit the fixed array is refused up front
    A, _ = workloads.small_case(1024, 64, seed=5, device="cuda")
    G = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    too_many_rows = 8_323_072 + 128
    st = T.tsvd_gram_static(A, too_many_rows, 64, too_many_rows, T.TSVD_FP32, T.TSVD_FP64, G, 64,
                            None, stream, check=False)
    assert st == T.TSVD_ERR_UNSUPPORTED
