"""GPU adjoint of the solve: dE/dV for E = sum of the k smallest eigenvalues (Hellmann-Feynman density).

Checked element by element against the oracle's density on the same vectors, against the oracle's gradient from
dense eigenvectors, and against central finite differences of GPU solves (step 1e-5, warm-started from the
converged vectors, tol 1e-11, per-pair differences summed). The relative error is measured against
max(|g_p|, k/n), since the density is tiny far from the low-lying states.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests.gpu_helpers import Handle, dev, host, need_gpu, ptr, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_energy_gradient_kernel_matches_oracle_density():
    N, k = 11, 37                                         # ragged: n = 1331, k not a multiple of 4
    rng = np.random.default_rng(5)
    X = rng.standard_normal((N ** 3, k))
    with Handle(np.zeros(N ** 3), N, kt=k, sbsize=1) as H:
        Xd = dev(X)
        g = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        pk.ppcg_energy_gradient(H.h, ptr(Xd), N ** 3, k, 2.5, ptr(g))
        got = g.cpu().numpy()
    np.testing.assert_allclose(got, 2.5 * oracle.energy_gradient(X), rtol=1e-14)


def test_autograd_gradient_matches_oracle_and_finite_differences():
    N, k, q = 8, 10, 2
    w = wl.small("adj", N=N, k=k, sbsize=q, seed=77)
    V, X0 = wl.make_inputs(w)
    ev, U = np.linalg.eigh(oracle.assemble_H(V, N, 1.0))
    assert ev[k] - ev[k - 1] > 1e-3
    solver = pk.Solver(V, N, k, q, rr_period=5, maxiter=3000)
    try:
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        E = pk.smallest_eigsum(Vt, solver, X0, tol=1e-11)
        E.backward()
        g = Vt.grad.cpu().numpy()
        np.testing.assert_allclose(float(E.detach()), np.sum(ev[:k]), rtol=1e-12)
        np.testing.assert_allclose(np.sum(g), k, rtol=1e-12)
        ref = oracle.energy_gradient(U[:, :k])
        scale = np.maximum(np.abs(ref), k / N ** 3)
        assert np.max(np.abs(g - ref) / scale) <= 1e-8
        # central differences of the GPU solve, warm-started from the converged vectors
        lam0, X, _, _ = solver.solve(X0, 1e-11)
        Xw = np.asfortranarray(X.cpu().numpy().T)
        hstep = 1e-5
        rng = np.random.default_rng(3)
        for p in rng.choice(N ** 3, 8, replace=False):
            e = np.zeros(N ** 3)
            e[p] = hstep
            solver.set_potential(torch.tensor(V + e, device="cuda"))
            lp, _, _, sp = solver.solve(Xw, 1e-11)
            solver.set_potential(torch.tensor(V - e, device="cuda"))
            lm, _, _, sm = solver.solve(Xw, 1e-11)
            assert sp["converged"] == 1 and sm["converged"] == 1
            fd = np.sum((lp - lm) / (2 * hstep))
            assert abs(fd - g[p]) <= 1e-6 * max(abs(g[p]), k / N ** 3), (p, fd, g[p])
    finally:
        solver.close()
