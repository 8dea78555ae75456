"""Pins for the CPU oracle: each test checks it against something other than itself.

Pins used: the dense operator assembled entry by entry; plane-wave eigenvectors and the closed-form spectrum
of the periodic (and Bloch-twisted) 7-point Laplacian; separable potentials whose spectrum is a sum of three
1-D spectra; dense LAPACK eigh; textbook Householder QR; LAPACK's generalised eigh; the LOBPCG special case
of Section 5.1; Theorem 2; Courant-Fischer bounds on Ritz values.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
import oracle



def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- operator (row a0)
@pytest.mark.parametrize("N,h", [(3, 1.0), (4, 0.5), (5, 1.0)])
def test_apply_H_matches_assembled(N, h):
    rng = _rng(N)
    V = rng.random(N ** 3)
    X = rng.standard_normal((N ** 3, 3))
    A = oracle.assemble_H(V, N, h)
    assert np.allclose(A, A.T, atol=0)
    np.testing.assert_allclose(oracle.apply_H(V, N, h, X), A @ X, rtol=0, atol=1e-12)


def test_apply_H_bloch_matches_assembled_and_is_hermitian():
    N, theta = 4, (0.3, 0.7, 1.1)
    rng = _rng(3)
    V = rng.random(N ** 3)
    X = rng.standard_normal((N ** 3, 2)) + 1j * rng.standard_normal((N ** 3, 2))
    A = oracle.assemble_H(V, N, 1.0, theta)
    np.testing.assert_allclose(A, A.conj().T, atol=0)
    np.testing.assert_allclose(oracle.apply_H(V, N, 1.0, X, theta), A @ X, atol=1e-12)


def _plane_wave(N, m, theta=(0.0, 0.0, 0.0)):
    i, j, l = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    phase = sum((2 * np.pi * m[d] + theta[d]) / N * c for d, c in enumerate((i, j, l)))
    return np.exp(1j * phase).reshape(-1, order="F")


@pytest.mark.parametrize("m", [(0, 0, 0), (1, 0, 0), (2, 3, 1), (5, 5, 4)])
def test_plane_waves_are_eigenvectors(m):
    # V = 0: eigenvalue sum_d 4 sin^2(pi m_d / N) / h^2
    N, h = 6, 0.7
    x = _plane_wave(N, m)
    lam = sum(4 * np.sin(np.pi * md / N) ** 2 for md in m) / h ** 2
    np.testing.assert_allclose(oracle.apply_H(np.zeros(N ** 3), N, h, x), lam * x, atol=1e-12)


@pytest.mark.parametrize("m", [(0, 0, 0), (1, 2, 3)])
def test_bloch_plane_waves_are_eigenvectors(m):
    # psi = exp(i q.r), q_d = (2 pi m_d + theta_d) / N satisfies the twist; eigenvalue sum 4 sin^2(q_d / 2)
    N, theta = 5, (0.3, 0.7, 1.1)
    x = _plane_wave(N, m, theta)
    lam = sum(4 * np.sin((2 * np.pi * m[d] + theta[d]) / (2 * N)) ** 2 for d in range(3))
    np.testing.assert_allclose(oracle.apply_H(np.zeros(N ** 3), N, 1.0, x, theta), lam * x, atol=1e-12)


# ---------------------------------------------------------------- small dense pieces
def test_cholqr2_equals_textbook_qr():
    rng = _rng(1)
    n, k = 400, 12
    X = rng.standard_normal((n, k)) @ np.diag(np.logspace(0, 5, k)) @ sla.qr(rng.standard_normal((k, k)))[0]
    Q, R = oracle.cholqr2(X)
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(Q @ R, X, rtol=0, atol=1e-10 * np.linalg.norm(X))
    Qh, Rh = np.linalg.qr(X)                 # Householder QR; make diag(R) positive (unique QR)
    s = np.sign(np.diag(Rh))
    np.testing.assert_allclose(Q, Qh * s[None, :], atol=1e-10)


def test_shifted_cholqr3_handles_breakdown():
    rng = _rng(2)
    n, k = 300, 10
    X = rng.standard_normal((n, k))
    X[:, -1] = X[:, 0] + 1e-12 * rng.standard_normal(n)     # kappa ~ 1e12: CholQR breaks down
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholqr2(X)
    Q, R = oracle.shifted_cholqr3(X)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(Q @ R, X, atol=1e-8)


def test_project_removes_span_and_is_idempotent():
    rng = _rng(4)
    X = oracle.cholqr2(rng.standard_normal((200, 7)))[0]
    Y = rng.standard_normal((200, 5))
    Z = oracle.project(Y, X)
    assert np.max(np.abs(X.T @ Z)) < 1e-13 * np.linalg.norm(Y)
    np.testing.assert_allclose(oracle.project(Z, X), Z, atol=1e-13)
    # the part removed lies in span(X)
    D = Y - Z
    np.testing.assert_allclose(X @ (X.T @ D), D, atol=1e-12)


def test_theorem2_identity_and_hpd_preconditioner():
    # x_j* A w_j = r_j* T r_j > 0 with W = (I - XX*) T R, R = (I - XX*) A X (proof of Theorem 2)
    N = 6
    rng = _rng(5)
    V = rng.random(N ** 3)
    X = oracle.cholqr2(rng.standard_normal((N ** 3, 4)))[0]
    HX = oracle.apply_H(V, N, 1.0, X)
    R = oracle.residual(X, HX, X.T @ HX)
    sigma = 0.3
    TR = oracle.precondition(R, V, N, 1.0, sigma)
    W = oracle.project(TR, X)
    lhs = np.einsum("ij,ij->j", X, oracle.apply_H(V, N, 1.0, W))
    d = np.maximum(6.0 + V - sigma, 0.1)
    rhs = np.einsum("ij,ij->j", R, R / d[:, None])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10)
    assert np.all(rhs > 0)
    # Theorem 2: with P = 0 every alpha_j != 0
    for j in range(4):
        CX, CW, CP = oracle.block_coefficients(X[:, j:j + 1], W[:, j:j + 1], None, HX[:, j:j + 1],
                                               oracle.apply_H(V, N, 1.0, W[:, j:j + 1]), None)
        assert abs(CX[0, 0]) > 1e-3 and CP is None


def test_precondition_floor_keeps_T_positive():
    V = np.array([-10.0, 0.0, 1.0, 5.0])
    W = np.ones((4, 1))
    TW = oracle.precondition(W, V, 1, 1.0, sigma=2.0)      # d = max(6 + V - 2, 0.1)
    np.testing.assert_allclose(TW[:, 0], 1.0 / np.array([0.1, 4.0, 5.0, 9.0]))


@pytest.mark.parametrize("q,with_p", [(1, False), (1, True), (3, True), (4, False)])
def test_block_coefficients_solve_projev(q, with_p):
    # eq. projev on S = [X_j, W_j, P_j]: compare with LAPACK's generalised driver
    N = 5
    rng = _rng(10 + q)
    V = rng.random(N ** 3)
    n = N ** 3
    X = oracle.cholqr2(rng.standard_normal((n, q)))[0]
    W = oracle.project(rng.standard_normal((n, q)), X)
    Pm = oracle.project(rng.standard_normal((n, q)), X) if with_p else None
    H = lambda Y: oracle.apply_H(V, N, 1.0, Y)
    CX, CW, CP = oracle.block_coefficients(X, W, Pm, H(X), H(W), None if Pm is None else H(Pm))
    S = np.hstack([X, W] + ([Pm] if with_p else []))
    GA, GB = S.T @ H(S), S.T @ S
    C = np.vstack([CX, CW] + ([CP] if with_p else []))
    theta_ref = sla.eigh(GA, GB, eigvals_only=True, subset_by_index=[0, q - 1])
    np.testing.assert_allclose(C.T @ GB @ C, np.eye(q), atol=1e-12)
    theta = np.linalg.eigvalsh(C.T @ GA @ C)
    np.testing.assert_allclose(theta, theta_ref, rtol=1e-12, atol=1e-12)
    # C's columns are eigenvectors: GA C = GB C Theta
    Th = C.T @ GA @ C
    np.testing.assert_allclose(GA @ C, GB @ C @ Th, atol=1e-10)


def test_block_rr_q1_by_hand():
    # x _|_ w, both unit norm: the 2x2 problem of eq. (proj2) [[a, b], [b, c]] c = theta c, smallest root
    n = 64
    rng = _rng(7)
    x = rng.standard_normal((n, 1)); x /= np.linalg.norm(x)
    w = rng.standard_normal((n, 1)); w -= x * (x.T @ w); w /= np.linalg.norm(w)
    a, b, c = 2.0, 0.5, 5.0
    # choose "A x", "A w" so that x*Ax = a, x*Aw = b, w*Aw = c
    Ax = a * x + b * w
    Aw = b * x + c * w
    CX, CW, CP = oracle.block_coefficients(x, w, None, Ax, Aw, None)
    theta = 0.5 * (a + c) - np.sqrt(0.25 * (a - c) ** 2 + b * b)
    v = np.array([b, theta - a]); v /= np.linalg.norm(v)
    got = np.array([CX[0, 0], CW[0, 0]])
    np.testing.assert_allclose(np.abs(got), np.abs(v), atol=1e-14)
    assert np.sign(got[0] * got[1]) == np.sign(v[0] * v[1])


def test_lobpcg_special_case_one_step():
    # sbsize = k: one block step picks the k smallest Ritz pairs of span[X, W, P] (Section 5.1)
    N, k = 5, 4
    n = N ** 3
    rng = _rng(8)
    V = rng.random(n)
    H = lambda Y: oracle.apply_H(V, N, 1.0, Y)
    X = oracle.cholqr2(rng.standard_normal((n, k)))[0]
    W = oracle.project(rng.standard_normal((n, k)), X)
    Pm = oracle.project(rng.standard_normal((n, k)), X)
    CX, CW, CP = oracle.block_coefficients(X, W, Pm, H(X), H(W), H(Pm))
    Xn, Pn = oracle.block_update(X, W, Pm, CX, CW, CP)
    Q = sla.orth(np.hstack([X, W, Pm]))          # SVD-based basis, independent of CholQR
    ref = np.linalg.eigvalsh(Q.T @ H(Q))[:k]
    Xo = oracle.cholqr2(Xn)[0]
    got = np.linalg.eigvalsh(Xo.T @ H(Xo))
    np.testing.assert_allclose(got, ref, rtol=1e-12)
    np.testing.assert_allclose(Xn - X @ CX, Pn, atol=1e-13)   # step 15: X_j C_X + P_j


def test_subblocks_split():
    assert oracle.subblocks(10, 4) == [(0, 4), (4, 8), (8, 10)]
    assert oracle.subblocks(8, 4) == [(0, 4), (4, 8)]
    assert oracle.subblocks(3, 5) == [(0, 3)]


def test_normalize_phase():
    X = np.array([[0.1, -3.0], [-0.5, 3.0], [0.2, 1.0]])
    Y = oracle.normalize_phase(X)
    np.testing.assert_allclose(np.linalg.norm(Y, axis=0), 1.0)
    assert Y[1, 0] > 0 and Y[0, 1] > 0                    # tie |-3| = |3|: lowest index wins


# ---------------------------------------------------------------- whole solver (rows a1-a14)
def _k_at_gap(lam_sorted, k_min):
    """Smallest k >= k_min with lambda_k < lambda_{k+1} (does not cut a degenerate shell)."""
    for k in range(k_min, len(lam_sorted)):
        if lam_sorted[k] - lam_sorted[k - 1] > 1e-9:
            return k
    raise ValueError


def test_ppcg_zero_potential_closed_form_spectrum():
    N = 6
    lam_all = np.sort([sum(4 * np.sin(np.pi * m / N) ** 2 for m in ms)
                       for ms in itertools.product(range(N), repeat=3)])
    k = _k_at_gap(lam_all, 7)                        # 1 + 6 = 7
    c = 0.25                                         # constant V shifts every eigenvalue by c
    V = np.full(N ** 3, c)
    X0 = _rng(9).standard_normal((N ** 3, k))
    r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-9)
    assert r.converged
    np.testing.assert_allclose(r.lam, lam_all[:k] + c, rtol=0, atol=1e-12)
    assert np.max(r.res) <= 1e-9


def _periodic_1d(v):
    N = len(v)
    T = np.diag(2.0 + v)
    for i in range(N):
        T[i, (i + 1) % N] -= 1.0
        T[i, (i - 1) % N] -= 1.0
    return T


def test_ppcg_separable_potential_spectrum():
    w = wl.small("sep", N=8, k=9, sbsize=3, potential="separable", seed=12)
    rng = np.random.default_rng(w.seed)
    v1, v2, v3 = rng.random(w.N), rng.random(w.N), rng.random(w.N)
    V = (v1[:, None, None] + v2[None, :, None] + v3[None, None, :]).reshape(-1, order="F")
    V_gen, X0 = wl.make_inputs(w)
    np.testing.assert_array_equal(V, V_gen)
    e = [np.linalg.eigvalsh(_periodic_1d(v)) for v in (v1, v2, v3)]
    lam_all = np.sort((e[0][:, None, None] + e[1][None, :, None] + e[2][None, None, :]).ravel())
    k = _k_at_gap(lam_all, w.k)
    r = oracle.ppcg(V, w.N, 1.0, k, w.sbsize, 5, wl.make_inputs(w, ncols=k)[1], tol=1e-9)
    assert r.converged
    np.testing.assert_allclose(r.lam, lam_all[:k], rtol=0, atol=1e-12)


@pytest.mark.parametrize("q,rr", [(1, 5), (3, 4), (10, 5)])
def test_ppcg_matches_dense_eigh(q, rr):
    N, k = 7, 10
    w = wl.small("dense", N=N, k=k, sbsize=q, seed=20 + q)
    V, X0 = wl.make_inputs(w)
    A = oracle.assemble_H(V, N, 1.0)
    ev, U = np.linalg.eigh(A)
    r = oracle.ppcg(V, N, 1.0, k, q, rr, X0, tol=1e-8)
    assert r.converged and np.max(r.res) <= 1e-8
    np.testing.assert_allclose(r.lam, ev[:k], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.X.T @ r.X, np.eye(k), atol=1e-12)
    # Davis-Kahan: sin angle(x_i, u_i) <= r_i / gap_i
    gaps = np.array([min(abs(ev[i] - ev[j]) for j in range(k + 1) if j != i) for i in range(k)])
    c = np.einsum("ij,ij->j", r.X, U[:, :k])
    sines = np.linalg.norm(r.X - U[:, :k] * c[None, :], axis=0)   # |x - (u*x) u| = sin angle
    assert np.all(sines <= 2 * r.res / gaps + 1e-12)


def test_ppcg_ritz_values_bound_eigenvalues_from_above():
    # Courant-Fischer: each Ritz value from an unconverged run is >= the exact eigenvalue of the same index
    N, k = 7, 10
    w = wl.small("cf", N=N, k=k, sbsize=2, seed=31)
    V, X0 = wl.make_inputs(w)
    ev = np.linalg.eigvalsh(oracle.assemble_H(V, N, 1.0))[:k]
    for maxiter in (0, 3, 12):
        r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-8, maxiter=maxiter)
        assert np.all(r.lam >= ev - 1e-12)


def test_ppcg_buffer_vectors_and_no_locking():
    N, k, nbuf = 7, 8, 3
    w = wl.small("buf", N=N, k=k, sbsize=2, seed=41)
    V, X0 = wl.make_inputs(w, ncols=k + nbuf)
    ev = np.linalg.eigvalsh(oracle.assemble_H(V, N, 1.0))[:k]
    for lock in (True, False):
        r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-8, nbuf=nbuf, lock=lock)
        assert r.converged and r.lam.shape == (k,)
        np.testing.assert_allclose(r.lam, ev, atol=1e-10)


def test_ppcg_projection_ablation_slows_convergence():
    # Section 5.4, figure "proj": dropping the projections of steps 4-5 deteriorates convergence
    N, k = 7, 10
    w = wl.small("abl", N=N, k=k, sbsize=2, seed=51)
    V, X0 = wl.make_inputs(w)
    full = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-4, maxiter=150)
    noproj = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-4, maxiter=150, project_W=False, project_P=False)
    assert full.converged
    assert (not noproj.converged) or noproj.iters > full.iters


def test_ppcg_warm_start_converges_immediately():
    N, k = 6, 7
    V = np.zeros(N ** 3)
    ev, U = np.linalg.eigh(oracle.assemble_H(V, N, 1.0))
    r = oracle.ppcg(V, N, 1.0, k, 2, 5, np.asfortranarray(U[:, :k]), tol=1e-9)
    assert r.converged and r.iters == 0


# ---------------------------------------------------------------- complex Hermitian (Bloch) problems
THETA = (0.3, 0.7, 1.1)


def test_ppcg_complex_bloch_matches_dense_eigh():
    N, k = 6, 8
    w = wl.small("cb", N=N, k=k, sbsize=2, potential="wells", n_wells=2, seed=3, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    A = oracle.assemble_H(V, N, 1.0, THETA)
    ev, U = np.linalg.eigh(A)
    r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-8, theta=THETA, maxiter=3000)
    assert r.converged and r.X.dtype == np.complex128
    np.testing.assert_allclose(r.lam, ev[:k], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.X.conj().T @ r.X, np.eye(k), atol=1e-12)
    res = np.linalg.norm(A @ r.X - r.X * r.lam[None, :], axis=0)
    assert np.max(res) <= 1e-8 * (1 + 1e-6)
    for i in range(k):                                # phase convention: largest-modulus entry real positive
        p = int(np.argmax(np.abs(r.X[:, i])))
        assert abs(r.X[p, i].imag) < 1e-14 and r.X[p, i].real > 0


def test_ppcg_complex_zero_potential_closed_form_spectrum():
    # V = 0: Bloch plane waves, eigenvalues sum_d 4 sin^2((2 pi m_d + theta_d) / (2 N)), all distinct for this twist
    N, k = 5, 10
    lam_all = np.sort([sum(4 * np.sin((2 * np.pi * m[d] + THETA[d]) / (2 * N)) ** 2 for d in range(3))
                       for m in itertools.product(range(N), repeat=3)])
    assert lam_all[k] - lam_all[k - 1] > 1e-3
    w = wl.small("cz", N=N, k=k, sbsize=2, potential="zero", seed=4, dtype="c128", theta=THETA)
    V, X0 = wl.make_inputs(w)
    r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-9, theta=THETA, maxiter=3000)
    assert r.converged
    np.testing.assert_allclose(r.lam, lam_all[:k], rtol=0, atol=1e-12)


# ---------------------------------------------------------------- orthonormalisation variants (Section 5.5, R10)
def test_polar_series_sums_to_inverse_square_root():
    # the binomial series of (1 + y)^{-1/2}, summed far out, equals the closed form at scalar y
    c = oracle.polar_coefficients(60)
    for y in (-0.3, -0.01, 0.02, 0.4):
        assert abs(np.polyval(c[::-1], y) - 1.0 / np.sqrt(1.0 + y)) < 1e-14


def test_polar_terms_rule():
    u = np.finfo(np.float64).eps / 2
    c = oracle.polar_coefficients(oracle.POLAR_MAX_TERMS + 1)
    assert oracle.polar_terms(0.0) == 1 and oracle.polar_terms(1e-12) == 1
    assert oracle.polar_terms(0.2) is None
    for nu in (1e-8, 1e-5, 1e-3, 1e-2):
        t = oracle.polar_terms(nu)
        assert abs(c[t + 1]) * nu ** (t + 1) <= u                 # first omitted term below roundoff
        assert t == 1 or abs(c[t]) * nu ** t > u                  # and t is the fewest such


@pytest.mark.parametrize("nu", [1e-9, 1e-5, 1e-2])
def test_orth_polar_equals_svd_polar_factor(nu):
    # X = Q (I + E) with E symmetric, ||X*X - I|| ~ nu: the series result is the orthonormal polar factor of X,
    # computed independently from the SVD (scipy.linalg.polar), to FP64 accuracy
    n, m = 300, 12
    rng = _rng(int(-np.log10(nu)))
    Q = sla.qr(rng.standard_normal((n, m)), mode="economic")[0]
    E = rng.standard_normal((m, m))
    E = 0.5 * (E + E.T)
    E *= 0.5 * nu / np.linalg.norm(E)
    Z = rng.standard_normal((m, m))
    X = Q @ (np.eye(m) + E) @ sla.expm(1e-1 * (Z - Z.T))
    t = oracle.polar_terms(np.linalg.norm(X.T @ X - np.eye(m)))
    U = oracle.orth_polar(X, t)
    Up, Hp = sla.polar(X)
    np.testing.assert_allclose(U, Up, atol=5e-15)
    np.testing.assert_allclose(U.T @ U, np.eye(m), atol=5e-15)


def test_orth_polar_of_scaled_orthonormal_columns_is_exact():
    # X = Q diag(s): X*X = diag(s^2) and the polar factor is Q
    n, m = 200, 6
    rng = _rng(3)
    Q = sla.qr(rng.standard_normal((n, m)), mode="economic")[0]
    s = 1.0 + 1e-4 * rng.standard_normal(m)
    X = Q * s[None, :]
    U = oracle.orth_polar(X, oracle.polar_terms(np.linalg.norm(s ** 2 - 1.0)))
    np.testing.assert_allclose(U, Q, atol=2e-15)


def test_orthonormalize_skip_and_fallback():
    n, m = 200, 5
    rng = _rng(4)
    Q = sla.qr(rng.standard_normal((n, m)), mode="economic")[0]
    st = {"n_orth_skip": 0, "n_polar": 0, "n_cholqr_fallback": 0}
    assert oracle.orthonormalize(Q, "cholqr2", 1e-10, st) is Q and st["n_orth_skip"] == 1
    X = rng.standard_normal((n, m))                          # far from orthonormal: the series is not used
    U = oracle.orthonormalize(X, "polar", 0.0, st)
    assert st["n_polar"] == 0
    np.testing.assert_allclose(U, oracle.cholqr2(X)[0], atol=1e-14)


@pytest.mark.parametrize("mode,skip", [("polar", 0.0), ("cholqr2", 1e-14), ("polar", 1e-3)])
def test_ppcg_orth_variants_match_dense_eigh(mode, skip):
    N, k = 7, 10
    w = wl.small("orthv", N=N, k=k, sbsize=2, seed=61)
    V, X0 = wl.make_inputs(w)
    ev = np.linalg.eigvalsh(oracle.assemble_H(V, N, 1.0))[:k]
    r = oracle.ppcg(V, N, 1.0, k, 2, 5, X0, tol=1e-8, maxiter=2000, orth_mode=mode, orth_skip_tol=skip)
    assert r.converged and np.max(r.res) <= 1e-8
    np.testing.assert_allclose(r.lam, ev, rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.X.T @ r.X, np.eye(k), atol=1e-12)
    assert r.stats["n_polar"] + r.stats["n_orth_skip"] > 0


def test_planted_polar_sign_error_is_caught():
    real = oracle.ppcg.__globals__["polar_coefficients"]

    def wrong(t):
        c = real(t)
        c[1] = -c[1]
        return c
    n, m = 200, 6
    rng = _rng(8)
    Q = sla.qr(rng.standard_normal((n, m)), mode="economic")[0]
    X = Q @ (np.eye(m) + 1e-3 * np.diag(rng.standard_normal(m)))
    t = oracle.polar_terms(np.linalg.norm(X.T @ X - np.eye(m)))
    oracle.ppcg.__globals__["polar_coefficients"] = wrong
    try:
        U = oracle.orth_polar(X, t)
    finally:
        oracle.ppcg.__globals__["polar_coefficients"] = real
    assert np.max(np.abs(U - sla.polar(X)[0])) > 1e-6


# ---------------------------------------------------------------- planted mistakes are caught
def test_planted_stencil_sign_error_is_caught():
    real = oracle.apply_H

    def bad(V, N, h, X, theta=None):                 # one neighbour enters with the wrong sign
        return real(V, N, h, X, theta) + 2.0 * np.roll(np.asarray(X).reshape((N, N, N, -1), order="F"), 1,
                                                       axis=0).reshape(np.asarray(X).shape, order="F")
    N = 4
    V = _rng().random(N ** 3)
    X = _rng(1).standard_normal((N ** 3, 2))
    assert not np.allclose(bad(V, N, 1.0, X), oracle.assemble_H(V, N, 1.0) @ X)


def test_planted_missing_p_term_is_caught():
    N, k = 5, 4
    n = N ** 3
    rng = _rng(8)
    V = rng.random(n)
    H = lambda Y: oracle.apply_H(V, N, 1.0, Y)
    X = oracle.cholqr2(rng.standard_normal((n, k)))[0]
    W = oracle.project(rng.standard_normal((n, k)), X)
    Pm = oracle.project(rng.standard_normal((n, k)), X)
    CX, CW, CP = oracle.block_coefficients(X, W, Pm, H(X), H(W), H(Pm))
    Xbad = X @ CX + W @ CW                           # step 14 without the P_j C_P term
    Q = sla.orth(np.hstack([X, W, Pm]))
    ref = np.linalg.eigvalsh(Q.T @ H(Q))[:k]
    got = np.linalg.eigvalsh(oracle.cholqr2(Xbad)[0].T @ H(oracle.cholqr2(Xbad)[0]))
    assert not np.allclose(got, ref, rtol=1e-8)


def test_planted_transposed_projection_is_caught():
    rng = _rng(4)
    X = oracle.cholqr2(rng.standard_normal((200, 7)))[0]
    Y = rng.standard_normal((200, 7))
    bad = Y - X @ (Y.T @ X)                            # transposed Gram
    assert np.max(np.abs(X.T @ bad)) > 1e-3


# ---------------------------------------------------------------- adjoint (Hellmann-Feynman gradient)
def test_energy_gradient_matches_central_differences_of_dense_eigenvalues():
    N, k, h = 6, 7, 1e-4
    rng = _rng(61)
    V = rng.random(N ** 3)
    ev, U = np.linalg.eigh(oracle.assemble_H(V, N, 1.0))
    assert ev[k] - ev[k - 1] > 1e-3                     # gap above lambda_k: E is differentiable
    g = oracle.energy_gradient(U[:, :k])
    np.testing.assert_allclose(np.sum(g), k, rtol=1e-13)     # sum_p dE/dV_p = k (unit vectors)
    for p in rng.choice(N ** 3, 6, replace=False):
        e = np.zeros(N ** 3)
        e[p] = h
        Ep = np.sum(np.linalg.eigvalsh(oracle.assemble_H(V + e, N, 1.0))[:k])
        Em = np.sum(np.linalg.eigvalsh(oracle.assemble_H(V - e, N, 1.0))[:k])
        assert abs((Ep - Em) / (2 * h) - g[p]) <= 1e-7 * max(abs(g[p]), k / N ** 3)


def test_constant_potential_shift_moves_energy_by_k_c():
    N, k, c = 6, 7, 0.37
    V = _rng(62).random(N ** 3)
    E0 = np.sum(np.linalg.eigvalsh(oracle.assemble_H(V, N, 1.0))[:k])
    E1 = np.sum(np.linalg.eigvalsh(oracle.assemble_H(V + c, N, 1.0))[:k])
    np.testing.assert_allclose(E1 - E0, k * c, rtol=1e-12)


def _kron_operator(V, N):
    """A = -Laplacian + diag(V) on the periodic N^3 grid as a sum of Kronecker products (scipy.sparse): an
    assembly that shares nothing with the oracle's stencil."""
    import scipy.sparse as sp
    one = np.ones(N)
    L1 = sp.diags([2 * one, -one[:-1], -one[:-1], [-1.0], [-1.0]], [0, 1, -1, N - 1, -(N - 1)], format="csr")
    I = sp.identity(N, format="csr")
    # linear index p = i + N j + N^2 l: the x axis is the fastest, i.e. the last Kronecker factor
    return (sp.kron(sp.kron(I, I), L1) + sp.kron(sp.kron(I, L1), I) + sp.kron(sp.kron(L1, I), I) +
            sp.diags(V)).tocsc()


def _smallest_by_lanczos(V, N, count):
    """The `count` algebraically smallest eigenvalues by ARPACK (scipy eigsh) in shift-invert mode with the shift
    below the spectrum (lambda_min >= min V because -Laplacian >= 0)."""
    import scipy.sparse.linalg as spla
    H = _kron_operator(V, N)
    return np.sort(spla.eigsh(H, k=count, sigma=V.min() - 0.5, which="LM", return_eigenvectors=False, tol=1e-13))


@pytest.mark.slow
def test_oracle_ppcg_returns_the_k_smallest_on_a_wells_problem():
    # The result is defined as the k algebraically smallest eigenpairs (Section 2, eq. tracemin); a residual test
    # cannot detect a missed eigenvalue. Oracle PPCG on a 16^3 grid with 8 Gaussian wells (the recipe of the
    # 32^3 workload), k = 64, sbsize = 4, against the 72 smallest eigenvalues from ARPACK.
    w = wl.small("k_smallest_pin", N=16, k=64, sbsize=4, potential="wells", n_wells=8, seed=2020)
    V, X0 = wl.make_inputs(w)
    r = oracle.ppcg(V, w.N, w.h, w.k, w.sbsize, w.rr_period, X0, tol=1e-8, maxiter=2000)
    assert r.converged
    ref = _smallest_by_lanczos(V, w.N, w.k + 8)
    assert ref[w.k] - ref[w.k - 1] > 1e-3                    # a gap above lambda_k: the k smallest are unique
    assert np.max(np.abs(r.lam - ref[:w.k]) / np.maximum(np.abs(ref[:w.k]), 1)) <= 1e-10


@pytest.mark.slow
def test_stored_grid32_k256_values_match_sparse_lanczos():
    # The stored oracle eigenvalues of the 32^3, 8-well operator (the reference values of the full-size GPU tests
    # and of bench.py) against ARPACK on the Kronecker-assembled operator: a library eigensolver that shares
    # nothing with the oracle, so a missed eigenvalue (which no residual test can see) would be caught. About four
    # minutes of CPU.
    w = wl.GRID32_K256
    V, _ = wl.make_inputs(w)
    ref = _smallest_by_lanczos(V, w.N, w.k + 8)
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "grid32_k256_oracle_eigs.txt"))[:, 0]
    assert np.max(np.abs(gold - ref[:w.k]) / np.maximum(np.abs(ref[:w.k]), 1)) <= 1e-12
