"""The allocation-free Gram entry point, for callers that cannot allocate device memory.

ppcg_gram_noalloc has no counterpart in the paper. Callers under a fixed device-memory budget, inside an
application memory pool that forbids cudaMalloc, or without a ppcg handle (creating one allocates a workspace)
use it: its split-K partial sums live in a static device array inside the library. This test checks it against
the handle-based ppcg_gram on two calls in a row (the second reuses the shared array), using the error bound of
the Gram tests, and checks that a size beyond the array is rejected without any launch. It lives in a file of its
own that pytest collects last and runs the same alone in a fresh process or after the other tests.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_helpers import Handle, dev, host, need_gpu, ptr, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _bound(A, B):
    return 2 * A.shape[0] * EPS * (np.abs(A).T @ np.abs(B))


def test_gram_noalloc_matches_handle_gram_on_two_calls():
    need_gpu()
    N = 16
    n = N ** 3
    rng = np.random.default_rng(2027)
    cases = [(rng.standard_normal((n, 200)), rng.standard_normal((n, 130))),   # general, ragged tiles
             None]                                                             # symmetric A^T A, filled below
    X = rng.standard_normal((n, 96))
    cases[1] = (X, X)
    stream = torch.cuda.current_stream().cuda_stream
    with Handle(np.zeros(n), N, kt=200, sbsize=1) as H:
        for A, B in cases:
            ma, mb = A.shape[1], B.shape[1]
            Ad = dev(A)
            Bd = Ad if B is A else dev(B)
            C_ref = torch.empty((mb, ma), dtype=torch.float64, device="cuda")
            C_new = torch.full((mb, ma), np.nan, dtype=torch.float64, device="cuda")
            pk.ppcg_gram(H.h, ptr(Ad), n, ptr(Bd), n, ma, mb, ptr(C_ref))
            pk.ppcg_gram_noalloc(ptr(Ad), n, ptr(Bd), n, n, ma, mb, ptr(C_new), stream)
            ref, got = host(C_ref), host(C_new)
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - ref) <= 2 * _bound(A, B) + 1e-300)
            assert np.all(np.abs(got - A.T @ B) <= _bound(A, B) + 1e-300)
            if B is A:
                np.testing.assert_array_equal(got, got.T)


def test_gram_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    n = 64
    A = torch.zeros((1025, n), dtype=torch.float64, device="cuda")
    C = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pk.lib().ppcg_gram_noalloc(ptr(A), n, ptr(A), n, n, 1025, 1025, ptr(C), None)   # 1025^2 > 2^20
    assert st == pk.PPCG_ERR_ARG
    torch.cuda.synchronize()
    assert float(C.cpu()[0]) == 0.0
