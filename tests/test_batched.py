"""Batched solves (many independent problems of uneven n and k, concurrent streams) and the sbsize autotuner.

Each problem of a batch must give exactly the result it gives when solved alone (the kernels are deterministic and
problems share no data), and every result is checked against dense eigh (small grids) or by CPU-recomputed
residuals and orthonormality (the 64-problem workload).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests.gpu_helpers import need_gpu, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _problems(ws):
    out = []
    for w in ws:
        V, X0 = wl.make_inputs(w)
        out.append(({"V": V, "grid": w.N, "k": w.k, "sbsize": w.sbsize, "rr_period": w.rr_period}, X0, V))
    return out


def test_batch_equals_individual_solves_and_dense_eigh():
    ws = wl.batch(count=6, seed=2004, n_range=(6, 9), k_range=(4, 20), sbsize=2)
    probs = _problems(ws)
    bs = pk.BatchSolver([p for p, _, _ in probs], maxiter=3000)
    try:
        results, status = bs.solve([x for _, x, _ in probs], tol=1e-8, max_concurrent=4)
    finally:
        bs.close()
    assert status == "ok"
    for (p, X0, V), w, (lam, X, res, st) in zip(probs, ws, results):
        assert st["status"] == "ok" and st["converged"] == 1 and st["time_ms"] > 0
        s = pk.Solver(V, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=3000)
        try:
            lam1, X1, res1, st1 = s.solve(X0, 1e-8)
        finally:
            s.close()
        np.testing.assert_array_equal(lam, lam1)                    # bit-identical to the lone solve
        np.testing.assert_array_equal(X.cpu().numpy(), X1.cpu().numpy())
        assert st["iters"] == st1["iters"]
        ev = np.linalg.eigvalsh(oracle.assemble_H(V, w.N, 1.0))[:w.k]
        assert np.all(np.abs(lam - ev) / np.maximum(np.abs(ev), 1.0) <= 1e-10)
        Xh = X.cpu().numpy().T
        r = np.linalg.norm(oracle.apply_H(V, w.N, 1.0, Xh) - Xh * lam[None, :], axis=0)
        assert np.max(r) <= 1e-8 * (1 + 1e-6)


def test_batch_of_64_problems():
    ws = wl.batch()                                                 # 64 problems, N in 12..28, k in 32..256
    probs = _problems(ws)
    bs = pk.BatchSolver([p for p, _, _ in probs], maxiter=5000)
    try:
        results, status = bs.solve([x for _, x, _ in probs], tol=1e-8)
    finally:
        bs.close()
    assert status == "ok"
    for (p, X0, V), w, (lam, X, res, st) in zip(probs, ws, results):
        assert st["status"] == "ok" and st["converged"] == 1
        Xh = X.cpu().numpy().T
        r = np.linalg.norm(oracle.apply_H(V, w.N, 1.0, Xh) - Xh * lam[None, :], axis=0)
        assert np.max(r) <= 1e-8 * (1 + 1e-6), (w.name, np.max(r))
        np.testing.assert_allclose(Xh.T @ Xh, np.eye(w.k), atol=1e-12)
        assert np.all(np.diff(lam) >= -1e-14)
        if w.N <= 13:                                               # the definition of the result: dense eigh
            ev = np.linalg.eigvalsh(oracle.assemble_H(V, w.N, 1.0))[:w.k]
            assert np.all(np.abs(lam - ev) / np.maximum(np.abs(ev), 1.0) <= 1e-10), w.name


def test_autotune_sbsize_returns_fastest_converged_candidate():
    w = wl.small("tune", N=10, k=24, sbsize=1, seed=5)
    V, X0 = wl.make_inputs(w)
    Vd = torch.tensor(V, device="cuda")
    X0d = torch.from_numpy(np.ascontiguousarray(X0.T)).cuda()
    import ctypes
    op = pk.ppcg_operator(w.N, w.N, w.N, 1.0, Vd.data_ptr(), (ctypes.c_double * 3)(0, 0, 0), 0)
    opt = pk.ppcg_options()
    opt.maxiter = 3000
    cands = [1, 2, 4, 8, 17, 0]                                     # the last two are invalid and skipped
    best, times = pk.ppcg_autotune_sbsize(op, w.n, w.k, 5, opt, X0d.data_ptr(), 1e-8, cands,
                                          torch.cuda.current_stream().cuda_stream)
    assert best in (1, 2, 4, 8)
    assert times[4] < 0 and times[5] < 0
    ok = [t for t in times[:4] if t > 0]
    assert ok and times[cands.index(best)] == min(ok)
