"""Complex Hermitian (Bloch-twisted) problems on the GPU, solved in the real form of order 2n.

Checked against the oracle's complex operator and solver, complex dense eigh, the closed-form Bloch spectrum of
V = 0, CPU-recomputed residuals and orthonormality, and the Hellmann-Feynman gradient sum_i |x_i|^2.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as wl
from tests.gpu_helpers import Handle, need_gpu, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu
THETA = (0.3, 0.7, 1.1)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _solve(V, N, k, q, X0, tol=1e-8, **kw):
    s = pk.Solver(V, N, k, q, rr_period=5, maxiter=4000, dtype="c128", theta=THETA, **kw)
    try:
        lam, X, res, st = s.solve(X0, tol)
        return lam, X.cpu().numpy().T.copy(), res, st
    finally:
        s.close()


def test_bloch_operator_in_real_form_matches_oracle():
    import ctypes
    N, m = 7, 5                                              # ragged: 7 is not a multiple of the 32-wide tile
    rng = np.random.default_rng(1)
    V = rng.random(N ** 3)
    Z = rng.standard_normal((N ** 3, m)) + 1j * rng.standard_normal((N ** 3, m))
    n = N ** 3
    Vd = torch.tensor(V, device="cuda")
    op = pk.ppcg_operator(N, N, N, 1.0, Vd.data_ptr(), (ctypes.c_double * 3)(*THETA), 1)
    opt = pk.ppcg_options()
    nbytes = pk.ppcg_workspace_bytes(op, n, m, 1, opt)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = pk.ppcg_create(op, n, m, 1, 5, opt, torch.cuda.current_stream().cuda_stream, ws.data_ptr(), nbytes)
    try:
        R = np.vstack([Z.real, Z.imag])                      # real form [Re z; Im z], 2n rows
        Xd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda()
        Yd = torch.empty_like(Xd)
        pk.ppcg_apply_operator(h, Xd.data_ptr(), 2 * n, Yd.data_ptr(), 2 * n, m)
        Y = Yd.cpu().numpy().T
    finally:
        pk.ppcg_destroy(h)
    ref = oracle.apply_H(V, N, 1.0, Z, THETA)
    np.testing.assert_allclose(Y[:n] + 1j * Y[n:], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,k,q,extra", [(6, 8, 2, {}), (7, 11, 3, {}), (8, 12, 4, {"fp64_gemm": "ozaki"}),
                                         (6, 8, 2, {"precision": "mixed"}), (6, 8, 2, {"orth": "polar"})])
def test_complex_solve_matches_dense_and_oracle(N, k, q, extra):
    w = wl.small("cg", N=N, k=k, sbsize=q, potential="wells", n_wells=2, seed=10 + N + k, dtype="c128",
                 theta=THETA)
    V, X0 = wl.make_inputs(w)
    lam, X, res, st = _solve(V, N, k, q, X0, **extra)
    assert st["status"] == "ok" and st["converged"] == 1
    A = oracle.assemble_H(V, N, 1.0, THETA)
    ev, U = np.linalg.eigh(A)
    tol_lam = 1e-10 if not extra.get("precision") else 1e-9
    assert np.all(np.abs(lam - ev[:k]) / np.maximum(np.abs(ev[:k]), 1.0) <= tol_lam)
    r = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.max(r) <= 1e-8 * (1 + 1e-6)
    np.testing.assert_allclose(res, r, rtol=1e-3, atol=1e-13)
    np.testing.assert_allclose(X.conj().T @ X, np.eye(k), atol=1e-12)
    for i in range(k):
        p = int(np.argmax(np.abs(X[:, i])))
        assert abs(X[p, i].imag) <= 1e-14 and X[p, i].real > 0
    ref = oracle.ppcg(V, N, 1.0, k, q, 5, X0, tol=1e-8, theta=THETA, maxiter=4000)
    assert ref.converged and np.all(np.abs(lam - ref.lam) / np.maximum(np.abs(ref.lam), 1.0) <= tol_lam)
    gaps = np.array([np.min(np.abs(np.delete(ev[:k + 1], i) - ev[i])) for i in range(k)])
    for i in range(k):                                       # Davis-Kahan against the exact eigenvectors
        c = U[:, i].conj() @ X[:, i]
        sin = np.linalg.norm(X[:, i] - c * U[:, i])
        assert sin <= r[i] / gaps[i] + 1e-10


def test_complex_zero_potential_closed_form():
    N, k = 6, 12
    lam_all = np.sort([sum(4 * np.sin((2 * np.pi * m[d] + THETA[d]) / (2 * N)) ** 2 for d in range(3))
                       for m in itertools.product(range(N), repeat=3)])
    w = wl.small("cz", N=N, k=k, sbsize=2, potential="zero", seed=4, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    lam, X, res, st = _solve(V, N, k, 2, X0, tol=1e-9)
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, lam_all[:k], rtol=0, atol=1e-12)


def test_complex_energy_gradient_and_finite_differences():
    N, k, q = 6, 8, 2
    w = wl.small("cadj", N=N, k=k, sbsize=q, potential="wells", n_wells=2, seed=21, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    ev, U = np.linalg.eigh(oracle.assemble_H(V, N, 1.0, THETA))
    assert ev[k] - ev[k - 1] > 1e-3
    s = pk.Solver(V, N, k, q, rr_period=5, maxiter=4000, dtype="c128", theta=THETA)
    try:
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        E = pk.smallest_eigsum(Vt, s, X0, tol=1e-11)
        E.backward()
        g = Vt.grad.cpu().numpy()
        np.testing.assert_allclose(float(E.detach()), np.sum(ev[:k]), rtol=1e-12)
        np.testing.assert_allclose(np.sum(g), k, rtol=1e-12)
        ref = oracle.energy_gradient(U[:, :k])
        scale = np.maximum(np.abs(ref), k / N ** 3)
        assert np.max(np.abs(g - ref) / scale) <= 1e-8
        lam0, X, _, _ = s.solve(X0, 1e-11)
        Xw = np.asfortranarray(X.cpu().numpy().T)
        hstep = 1e-5
        for p in np.random.default_rng(3).choice(N ** 3, 6, replace=False):
            e = np.zeros(N ** 3)
            e[p] = hstep
            s.set_potential(torch.tensor(V + e, device="cuda"))
            lp, _, _, sp = s.solve(Xw, 1e-11)
            s.set_potential(torch.tensor(V - e, device="cuda"))
            lm, _, _, sm = s.solve(Xw, 1e-11)
            assert sp["converged"] == 1 and sm["converged"] == 1
            fd = np.sum((lp - lm) / (2 * hstep))
            assert abs(fd - g[p]) <= 1e-6 * max(abs(g[p]), k / N ** 3), (p, fd, g[p])
    finally:
        s.close()


@pytest.mark.slow
def test_complex_gradient_central_differences_32_entries_at_16cubed():
    # the Bloch recipe (twist theta, Gaussian wells) at 16^3 with k = 16: the adjoint dE/dV = sum_i |x_i|^2 against
    # dense eigenvectors, and against central differences (step 1e-5) on 32 random potential entries, each from two
    # solves warm-started at the returned vectors with tol 1e-10, differencing the eigenvalues pair by pair
    N, k, q = 16, 16, 4
    w = wl.small("c5fd", N=N, k=k, sbsize=q, potential="wells", n_wells=4, seed=1005, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    n = N ** 3
    ev, U = np.linalg.eigh(oracle.assemble_H(V, N, 1.0, THETA))
    assert ev[k] - ev[k - 1] > 1e-3                     # a gap above lambda_k: E is differentiable
    s = pk.Solver(V, N, k, q, rr_period=5, maxiter=4000, dtype="c128", theta=THETA, fp64_gemm="ozaki")
    try:
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        E = pk.smallest_eigsum(Vt, s, X0, tol=1e-10)
        E.backward()
        g = Vt.grad.cpu().numpy()
        np.testing.assert_allclose(float(E.detach()), np.sum(ev[:k]), rtol=1e-12)
        np.testing.assert_allclose(np.sum(g), k, rtol=1e-12)          # sum_p dE/dV_p = k for unit vectors
        ref = oracle.energy_gradient(U[:, :k])
        scale = np.maximum(np.abs(ref), k / n)
        assert np.max(np.abs(g - ref) / scale) <= 1e-8
        _, X, _, _ = s.solve(X0, 1e-10)
        Xw = np.asfortranarray(X.cpu().numpy().T)
        # At step 1e-5 the difference quotient carries the eigenvalues' own rounding (a few ulps of ||A|| each,
        # divided by the step): even dense LAPACK eigenvalues give errors of several 1e-6 relative on some entries
        # here. So the step-1e-5 quotients are held to 1e-6 relative plus that rounding bound, and quotients at
        # step 1e-4 (truncation error ~1e-7 relative, rounding ten times smaller) to 1e-6 relative alone.
        norm_a = 12.0 + np.max(np.abs(V))
        for p in np.random.default_rng(11).choice(n, 32, replace=False):
            scale = max(abs(g[p]), k / n)
            for hstep, slack in ((1e-5, k * 4 * np.finfo(float).eps / 2 * norm_a / 1e-5), (1e-4, 0.0)):
                e = np.zeros(n)
                e[p] = hstep
                s.set_potential(torch.tensor(V + e, device="cuda"))
                lp, _, _, sp = s.solve(Xw, 1e-10)
                s.set_potential(torch.tensor(V - e, device="cuda"))
                lm, _, _, sm = s.solve(Xw, 1e-10)
                assert sp["converged"] == 1 and sm["converged"] == 1
                fd = np.sum((lp - lm) / (2 * hstep))
                assert abs(fd - g[p]) <= 1e-6 * scale + slack, (p, hstep, fd, g[p])
    finally:
        s.close()


def test_bloch_wells_recipe_at_12cubed():
    # the 64^3 Bloch recipe (64 wells on a Bloch-twisted grid) scaled to 12^3, k = 24, sbsize = 4
    w = wl.small("c5s", N=12, k=24, sbsize=4, potential="wells", n_wells=8, seed=1005, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    lam, X, res, st = _solve(V, w.N, w.k, w.sbsize, X0, fp64_gemm="ozaki")
    assert st["converged"] == 1
    A = oracle.assemble_H(V, w.N, 1.0, THETA)
    ev = np.linalg.eigvalsh(A)[:w.k]
    assert np.all(np.abs(lam - ev) / np.maximum(np.abs(ev), 1.0) <= 1e-10)
    r = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.max(r) <= 1e-8 * (1 + 1e-6)
