"""Failure handling on the GPU without a GPU fault: a bounded device-side wait that cannot complete gives up, the
call reports PPCG_ERR_TIMEOUT, and the handle stays usable.

The solver's grid barriers (cooperative Cholesky, Jacobi) wait with a bounded number of polls and set a timeout flag
instead of hanging. ppcg_barrier_timeout_check runs the same barrier code in a kernel where one CTA never arrives,
with a short bound, so the timeout path (flag set, every CTA returns, status mapped) runs for real.
"""
import time

import numpy as np
import pytest

from tests.gpu_helpers import Handle, dev, host, need_gpu, ptr, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_returns_status_and_handle_stays_usable():
    need_gpu()
    m = 96
    rng = np.random.default_rng(77)
    B = rng.standard_normal((m, m))
    M = B + B.T
    with Handle(np.zeros(8 ** 3), 8, kt=m, sbsize=1) as H:
        t0 = time.perf_counter()
        st = pk.ppcg_barrier_timeout_check(H.h, 1 << 14)
        el = time.perf_counter() - t0
        assert st == pk.PPCG_ERR_TIMEOUT
        assert el < 10.0
        assert pk.ppcg_barrier_timeout_check(H.h, 8) == pk.PPCG_ERR_ARG
        # the same handle then solves a dense eigenproblem whose Jacobi start waits at grid barriers
        Md = dev(M)
        ld = torch.empty(m, dtype=torch.float64, device="cuda")
        Cd = torch.empty((m, m), dtype=torch.float64, device="cuda")
        pk.ppcg_dense_eigh(H.h, ptr(Md), m, ptr(ld), ptr(Cd))
        got, C = ld.cpu().numpy(), host(Cd)
    np.testing.assert_allclose(got, np.linalg.eigvalsh(M), rtol=0, atol=1e-13 * np.linalg.norm(M))
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-12)
