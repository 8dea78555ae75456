"""Plain FP64 CPU oracle of the PPCG eigensolver (Vecharynski, Yang, Pask, arXiv 1407.7506).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg,
never by the product path. It shares no code with the CUDA library.

The oracle follows the detailed algorithm of Appendix A (Algorithm 3) step by step, in the paper's order and
notation, with numpy/scipy primitives (matmul, LAPACK Cholesky, LAPACK eigh, triangular solve) as its only
building blocks and no blocking, fusion or reordering beyond what the algorithm states. Every operator
application A*X, A*W, A*P is done explicitly with `apply_H`; the oracle keeps no recurrences.

Readings of the paper taken where it is silent (each is restated where it is used):
  R1  preconditioner T = diag(1 / max(6/h^2 + V_p - sigma, delta)), sigma = smallest Ritz value of the latest
      Rayleigh-Ritz step, delta = 0.1/h^2; a Rayleigh-Ritz step on orth(X0) precedes iteration 1 so that sigma
      exists (Theorem 2 needs an HPD T).
  R2  first iteration: P = [] so the sub-block problems are 2q x 2q (Alg. 2 step 9, Alg. 3 step 12).
  R3  P is kept per column position across a Rayleigh-Ritz step: the new active column at sorted position i
      takes the conjugate direction that belonged to position i (Alg. 3 step 28, "P <- P(J_act)"); a position
      that was locked carries a zero direction.
  R4  the Rayleigh-Ritz step on S = [X, X_lock] (Alg. 3 steps 22-24) solves the generalised eq. (projev) on S
      as written (Cholesky reduction of S* S); only if that Cholesky breaks down is S orthonormalised first.
  R5  Cholesky factor R of X*X is upper triangular with a positive diagonal (the text's "unit upper" cannot
      hold for a Cholesky factor); CholQR is applied twice (CholeskyQR2); on breakdown (a relative pivot
      R_ii / sqrt(G_ii) < CHOL_PIVOT_TOL) the shifted CholeskyQR3 of Fukaya, Kannan, Nakatsukasa, Yamamoto,
      Yamamoto (2020) is used.
  R6  sub-block problems: the columns of S_j = [X_j, W_j, P_j] are scaled to unit norm before S_j*S_j is
      factored; if that Cholesky factorisation fails, a pivot falls below PIVOT_TOL, or C_X is numerically
      singular (sigma_min < ALPHA_TOL; |alpha_j| for q = 1, Theorem 1), the block is redone without P
      (the back-track of Section 3, justified by Theorem 2).
  R7  stop test: r_i = ||A x_i - lambda_i x_i||_2 of the first k (non-buffer) Ritz pairs at a Rayleigh-Ritz
      step, max_i r_i <= tol; a Rayleigh-Ritz step is forced at once when ||W||_F <= tol after step 20.
  R8  locking: at every Rayleigh-Ritz step J_lock = {i < k : r_i <= tol}; locked vectors enter the next
      Rayleigh-Ritz step through S = [X, X_lock] (soft locking, Section 5.7).
  R9  output: Ritz values ascending; each Ritz vector has unit norm and its entry of largest modulus
      (lowest index on ties) real and positive.
  R10 orthonormalisation variants of Section 5.5 (optional; the default is CholeskyQR2 every plain step):
      "polar" replaces step 18 by X <- X (X* X)^{-1/2}, the (X* X)^{-1/2} = (I + Y)^{-1/2} series in
      Y = X* X - I truncated after t terms, t the fewest (at most POLAR_MAX_TERMS) whose first omitted term
      |c_{t+1}| nu^{t+1} is below the FP64 unit roundoff, nu = ||Y||_F; when no such t exists (nu too large
      for the series) CholeskyQR2 is used. "skip" (orth_skip_tol > 0) leaves X as it is when nu <= orth_skip_tol,
      the loss-of-orthogonality heuristic of the same section.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import scipy.linalg as sla

PIVOT_TOL = 1e-7       # R6: smallest Cholesky diagonal of the unit-diagonal S_j* S_j (squared pivot 1e-14)
ALPHA_TOL = 1e-12      # R6: smallest singular value of C_X (|alpha_j| for q = 1), Theorem 1
CHOL_PIVOT_TOL = 1e-7  # R5: smallest relative Cholesky pivot R_ii / sqrt(G_ii) accepted by CholQR
POLAR_MAX_TERMS = 8    # R10: most series terms the polar variant may use


# --------------------------------------------------------------------------------------------------------
# The operator A = H = -Laplacian_h + diag(V) on an N^3 periodic grid (the stencil that stands in for the
# paper's planewave Hamiltonian of Section 6); p = i + N j + N^2 l, x fastest.
# --------------------------------------------------------------------------------------------------------
def _as_block(X):
    return X.reshape(X.shape[0], 1) if X.ndim == 1 else X


def apply_H(V, N, h, X, theta=None):
    """A X with A = (1/h^2)(6 I - sum of the six periodic neighbours) + diag(V).

    theta (radians, total twist across the cell per axis) gives Bloch boundaries x(r + N e_d) = e^{i theta_d} x(r):
    the neighbour across the upper face carries e^{+i theta_d}, the one across the lower face e^{-i theta_d}.
    """
    Xb = _as_block(np.asarray(X))
    m = Xb.shape[1]
    G = Xb.reshape((N, N, N, m), order="F")
    out = 6.0 * G
    for axis in range(3):
        up = np.roll(G, -1, axis=axis)     # value at r + e_axis
        dn = np.roll(G, +1, axis=axis)     # value at r - e_axis
        if theta is not None and theta[axis] != 0.0:
            up = up.astype(np.complex128)
            dn = dn.astype(np.complex128)
            last = [slice(None)] * 4
            last[axis] = N - 1
            first = [slice(None)] * 4
            first[axis] = 0
            up[tuple(last)] *= np.exp(1j * theta[axis])
            dn[tuple(first)] *= np.exp(-1j * theta[axis])
        out = out - up - dn
    out = out.reshape((N ** 3, m), order="F") / (h * h) + V[:, None] * Xb
    return out.reshape(X.shape) if np.ndim(X) == 1 else np.asfortranarray(out)


def diag_H(V, N, h):
    """diag(A) = 6/h^2 + V."""
    return 6.0 / (h * h) + np.asarray(V, dtype=np.float64)


def assemble_H(V, N, h, theta=None):
    """Dense A built entry by entry from the stencil definition (brute-force pin for apply_H, tiny N only)."""
    n = N ** 3
    cplx = theta is not None and any(t != 0.0 for t in theta)
    A = np.zeros((n, n), dtype=np.complex128 if cplx else np.float64)
    th = (0.0, 0.0, 0.0) if theta is None else theta
    for l in range(N):
        for j in range(N):
            for i in range(N):
                p = i + N * j + N * N * l
                A[p, p] += 6.0 / (h * h) + V[p]
                for axis in range(3):
                    c = [i, j, l]
                    for step in (+1, -1):
                        d = list(c)
                        d[axis] += step
                        phase = 1.0
                        if d[axis] == N:
                            d[axis] = 0
                            phase = np.exp(1j * th[axis]) if cplx else 1.0
                        elif d[axis] == -1:
                            d[axis] = N - 1
                            phase = np.exp(-1j * th[axis]) if cplx else 1.0
                        q = d[0] + N * d[1] + N * N * d[2]
                        A[p, q] -= phase / (h * h)
    return A


# --------------------------------------------------------------------------------------------------------
# Steps of Algorithm 3
# --------------------------------------------------------------------------------------------------------
def precondition(W, V, N, h, sigma, delta=None):
    """Step 8, W <- T W with T = diag(1/max(6/h^2 + V_p - sigma, delta)) (reading R1; HPD for Theorem 2)."""
    delta = 0.1 / (h * h) if delta is None else delta
    d = np.maximum(diag_H(V, N, h) - sigma, delta)
    return W / d[:, None]


def project(Y, X):
    """Steps 9-10, Y <- (I - X X*) Y."""
    if Y is None or X is None or X.shape[1] == 0:
        return Y
    return Y - X @ (X.conj().T @ Y)


def cholqr(X):
    """Cholesky QR (Section 5.5): X*X = R*R with R upper triangular, positive diagonal; Q = X R^{-1}.

    Raises numpy.linalg.LinAlgError on a non-positive pivot.
    """
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T)
    L = np.linalg.cholesky(G)                        # G = L L*
    R = L.conj().T
    # breakdown (reading R5): a relative pivot R_ii / sqrt(G_ii) below CHOL_PIVOT_TOL means kappa(X) > ~1e7,
    # beyond what a second CholQR pass can repair
    if np.min(np.real(np.diag(R)) / np.sqrt(np.real(np.diag(G)))) < CHOL_PIVOT_TOL:
        raise np.linalg.LinAlgError("CholQR breakdown: relative pivot below tolerance")
    # Q = X R^{-1}  <=>  R* Q* = X*
    Qh = sla.solve_triangular(R, X.conj().T, trans="C", lower=False)
    return np.asfortranarray(Qh.conj().T), R


def cholqr2(X):
    """CholeskyQR2 (reading R5): two passes of cholqr. Returns Q, R with X = Q R."""
    Q1, R1 = cholqr(X)
    Q2, R2 = cholqr(Q1)
    return Q2, R2 @ R1


def shifted_cholqr3(X):
    """Shifted CholeskyQR3 (Fukaya et al. 2020, Algorithm 4.2): breakdown fallback of reading R5.

    Shift s = 11 (m n + n (n+1)) u ||X||^2 with ||X||_F bounding ||X||_2, then CholeskyQR2.
    """
    m, n = X.shape
    u = np.finfo(np.float64).eps / 2
    s = 11.0 * (m * n + n * (n + 1)) * u * np.linalg.norm(X, "fro") ** 2
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T) + s * np.eye(n)
    R0 = np.linalg.cholesky(G).conj().T
    Qh = sla.solve_triangular(R0, X.conj().T, trans="C", lower=False)
    Q2, R2 = cholqr2(np.asfortranarray(Qh.conj().T))
    return Q2, R2 @ R0


def orth(X, stats=None):
    """X <- orth(X) by CholeskyQR2, falling back to shifted CholeskyQR3 on breakdown (reading R5)."""
    try:
        return cholqr2(X)[0]
    except np.linalg.LinAlgError:
        if stats is not None:
            stats["n_cholqr_fallback"] += 1
        return shifted_cholqr3(X)[0]


def polar_coefficients(t):
    """c_0..c_t of the binomial series (1 + y)^{-1/2} = sum_j c_j y^j, c_j = binom(-1/2, j) (Section 5.5)."""
    c = [1.0]
    for j in range(1, t + 1):
        c.append(c[-1] * (-(2 * j - 1) / (2 * j)))
    return np.array(c)


def polar_terms(nu, tmax=POLAR_MAX_TERMS):
    """Reading R10: the fewest terms t >= 1 whose first omitted series term |c_{t+1}| nu^{t+1} is below the FP64
    unit roundoff, or None when even tmax terms leave a larger one."""
    c = polar_coefficients(tmax + 1)
    u = np.finfo(np.float64).eps / 2
    for t in range(1, tmax + 1):
        if abs(c[t + 1]) * nu ** (t + 1) <= u:
            return t
    return None


def orth_polar(X, t):
    """X <- X (I + Y)^{-1/2} with the series truncated after t terms, Y = X* X - I (Section 5.5)."""
    m = X.shape[1]
    Y = X.conj().T @ X - np.eye(m)
    c = polar_coefficients(t)
    C = np.zeros((m, m), dtype=X.dtype)
    Yj = np.eye(m, dtype=X.dtype)
    for j in range(t + 1):                       # sum_j c_j Y^j with explicit powers
        C = C + c[j] * Yj
        Yj = Yj @ Y
    return np.asfortranarray(X @ C)


def orthonormalize(X, mode="cholqr2", skip_tol=0.0, stats=None):
    """Step 18 with the variants of reading R10. mode "cholqr2" with skip_tol = 0 is plain orth(X)."""
    if mode == "cholqr2" and not skip_tol > 0.0:
        return orth(X, stats)
    m = X.shape[1]
    nu = np.linalg.norm(X.conj().T @ X - np.eye(m))
    if nu <= skip_tol:
        if stats is not None:
            stats["n_orth_skip"] = stats.get("n_orth_skip", 0) + 1
        return X
    if mode == "polar":
        t = polar_terms(nu)
        if t is not None:
            if stats is not None:
                stats["n_polar"] = stats.get("n_polar", 0) + 1
            return orth_polar(X, t)
    return orth(X, stats)


def subblocks(k_act, q):
    """Sub-block column ranges: s = ceil(k_act / q) blocks of q columns, the last one the remainder
    (Section 5.1; Alg. 3 step 5 footnote)."""
    return [(j, min(j + q, k_act)) for j in range(0, k_act, q)]


def _small_rr(S, HS, q):
    """The q smallest eigenpairs of (S* A S) c = theta (S* S) c with c* S* S c = 1 (eq. projev) for one
    sub-block, with the safeguards of reading R6. Returns C (3q x q or 2q x q) or None on breakdown."""
    GA = S.conj().T @ HS
    GB = S.conj().T @ S
    GA = 0.5 * (GA + GA.conj().T)
    GB = 0.5 * (GB + GB.conj().T)
    nrm = np.sqrt(np.real(np.diag(GB)))
    if np.any(nrm <= 0.0) or not np.all(np.isfinite(nrm)):
        return None
    D = 1.0 / nrm
    GAs = GA * D[:, None] * D[None, :]
    GBs = GB * D[:, None] * D[None, :]
    try:
        L = np.linalg.cholesky(GBs)
    except np.linalg.LinAlgError:
        return None
    if np.min(np.real(np.diag(L))) < PIVOT_TOL:
        return None
    # standard form K = L^{-1} GAs L^{-*}
    Y = sla.solve_triangular(L, GAs, lower=True)
    K = sla.solve_triangular(L, Y.conj().T, lower=True).conj().T
    K = 0.5 * (K + K.conj().T)
    theta, Z = np.linalg.eigh(K)
    C = sla.solve_triangular(L, Z[:, :q], trans="C", lower=True)     # L^{-*} Z
    C = C * D[:, None]
    CX = C[:q, :]
    smin = np.linalg.svd(CX, compute_uv=False).min()
    if not (smin >= ALPHA_TOL):
        return None
    return C


def block_coefficients(Xj, Wj, Pj, HXj, HWj, HPj, stats=None):
    """Steps 12-13 for one sub-block: C = [C_X; C_W; C_P] from eq. projev on S = [X_j, W_j, P_j].

    With P_j None (first iteration, R2) the problem is 2q x 2q and C_P is None. On breakdown the block is
    redone without P (reading R6, Theorem 2); if even that fails the block keeps X_j (C_X = I, C_W = 0).
    """
    q = Xj.shape[1]
    if Pj is not None:
        C = _small_rr(np.hstack([Xj, Wj, Pj]), np.hstack([HXj, HWj, HPj]), q)
        if C is not None:
            return C[:q], C[q:2 * q], C[2 * q:]
        if stats is not None:
            stats["n_drop_p"] += 1
    C = _small_rr(np.hstack([Xj, Wj]), np.hstack([HXj, HWj]), q)
    if C is None:
        if stats is not None:
            stats["n_stall"] += 1
        return np.eye(q, dtype=Xj.dtype), np.zeros((q, q), dtype=Xj.dtype), None
    return C[:q], C[q:], None


def block_update(Xj, Wj, Pj, CX, CW, CP):
    """Steps 14-15: P_j <- W_j C_W + P_j C_P ; X_j <- X_j C_X + P_j."""
    Pn = Wj @ CW
    if Pj is not None and CP is not None:
        Pn = Pn + Pj @ CP
    return Xj @ CX + Pn, Pn


def rayleigh_ritz(S, Hop, stats=None):
    """Steps 22-24 (reading R4): eq. projev on S = [X, X_lock] as written, (S* A S) C = (S* S) C Omega with
    C* (S* S) C = I, Omega ascending; X = S C. Solved by LAPACK's generalised driver (Cholesky reduction of
    S* S to standard form). If that Cholesky breaks down (relative pivot below CHOL_PIVOT_TOL, as in CholQR),
    S is orthonormalised first and the standard problem Q* A Q is solved instead (same Ritz pairs)."""
    HS = Hop(S)
    GA = S.conj().T @ HS
    GB = S.conj().T @ S
    GA = 0.5 * (GA + GA.conj().T)
    GB = 0.5 * (GB + GB.conj().T)
    try:
        L = np.linalg.cholesky(GB)
        if np.min(np.real(np.diag(L)) / np.sqrt(np.real(np.diag(GB)))) < CHOL_PIVOT_TOL:
            raise np.linalg.LinAlgError("Rayleigh-Ritz Gram breakdown")
        Omega, C = sla.eigh(GA, GB)
        return np.asfortranarray(S @ C), Omega
    except np.linalg.LinAlgError:
        if stats is not None:
            stats["n_cholqr_fallback"] += 1
        Q = orth(S, stats)
        M = Q.conj().T @ Hop(Q)
        M = 0.5 * (M + M.conj().T)
        Omega, C = np.linalg.eigh(M)
        return np.asfortranarray(Q @ C), Omega


def residual(X, HX, M):
    """Steps 4/20/25: W <- A X - X M, with M = X* A X (k x k) or the Ritz values Lambda (vector)."""
    if np.ndim(M) == 1:
        return HX - X * M[None, :]
    return HX - X @ M


def normalize_phase(X):
    """Reading R9: unit columns whose largest-modulus entry (lowest index on ties) is real positive."""
    X = np.array(X, copy=True, order="F")
    for i in range(X.shape[1]):
        x = X[:, i]
        x /= np.linalg.norm(x)
        p = int(np.argmax(np.abs(x)))          # argmax returns the first maximal index
        X[:, i] = x * (np.conj(x[p]) / abs(x[p]))
    return X


def energy_gradient(X):
    """dE/dV for E = sum of the k smallest eigenvalues of -Laplacian_h + diag(V): by the Hellmann-Feynman theorem
    (d lambda_i / dV_p = |x_i(p)|^2 for a unit eigenvector x_i of a simple eigenvalue; for the sum over a set of
    eigenvalues separated from the rest, the projector's diagonal), the density sum_{i<k} |x_i(p)|^2."""
    return np.sum(np.abs(X) ** 2, axis=1)


# --------------------------------------------------------------------------------------------------------
# Algorithm 3
# --------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class PPCGResult:
    lam: np.ndarray           # k Ritz values, ascending
    X: np.ndarray             # n x k Ritz vectors (reading R9)
    res: np.ndarray           # k residual norms ||A x_i - lambda_i x_i||
    converged: bool
    iters: int
    n_rr: int
    stats: dict
    history: list
    phase_s: dict


def ppcg(V, N, h, k, sbsize, rr_period, X0, tol=1e-8, maxiter=500, nbuf=0, lock=True, theta=None,
         sigma_floor=None, project_W=True, project_P=True, verbose=False, orth_mode="cholqr2", orth_skip_tol=0.0):
    """PPCG (Algorithm 3) for the k algebraically smallest eigenpairs of A = -Laplacian_h + diag(V).

    X0 is n x (k + nbuf). Returns a PPCGResult; `project_W` / `project_P` switch off the projections of
    steps 9 / 10 for the ablation of Section 5.4 (figure "proj"); `orth_mode` ("cholqr2" or "polar") and
    `orth_skip_tol` select the step-18 variants of reading R10.
    """
    V = np.asarray(V, dtype=np.float64)
    n = N ** 3
    kt = k + nbuf                                   # step 2: k <- k + nbuf
    assert X0.shape == (n, kt)
    q = sbsize
    delta = 0.1 / (h * h) if sigma_floor is None else sigma_floor
    stats = {"n_drop_p": 0, "n_stall": 0, "n_cholqr_fallback": 0, "n_locked": 0, "n_early_rr": 0,
             "n_orth_skip": 0, "n_polar": 0}
    phase = {"AX": 0.0, "GEMM": 0.0, "BlockRR": 0.0, "CholQR": 0.0, "RR": 0.0, "Precond": 0.0, "Lock": 0.0}
    history = []

    def Hop(Y):
        t = time.perf_counter()
        out = apply_H(V, N, h, Y, theta)
        phase["AX"] += time.perf_counter() - t
        return out

    # Step 1 (Alg. 2 step 1): X <- orth(X0); X_lock <- [], P <- [].
    t = time.perf_counter()
    X = orth(np.asfortranarray(X0), stats)
    phase["CholQR"] += time.perf_counter() - t
    Xlock = X[:, :0]
    P = None
    act = list(range(kt))                           # J_act as column positions of the sorted Ritz basis
    lck = []                                        # J_lock

    def rr_and_lock(X, Xlock, P, act):
        """Steps 22-31 with readings R3, R7, R8. Returns the new state and the stop flag."""
        t = time.perf_counter()
        S = np.hstack([X, Xlock])                   # step 22
        Xf, Lam = rayleigh_ritz(S, Hop, stats)      # steps 23-24
        phase["RR"] += time.perf_counter() - t
        HXf = Hop(Xf)
        Wf = residual(Xf, HXf, Lam)                 # step 25
        r = np.linalg.norm(Wf, axis=0)
        t = time.perf_counter()
        done = bool(np.max(r[:k]) <= tol)           # R7
        new_lck = [i for i in range(k) if r[i] <= tol] if lock else []       # step 26 (R8)
        new_act = [i for i in range(kt) if i not in new_lck]
        if P is not None:                            # step 28 with R3
            Pfull = np.zeros((n, kt), dtype=P.dtype)
            Pfull[:, act] = P
            P = np.asfortranarray(Pfull[:, new_act])
        phase["Lock"] += time.perf_counter() - t
        return Xf, Lam, Wf, r, done, new_lck, new_act, P

    # Reading R1: a Rayleigh-Ritz step on orth(X0) (iteration 0) provides sigma and the Ritz residual W.
    Xf, Lam, W, r, done, lck, act, P = rr_and_lock(X, Xlock, P, act)
    n_rr = 1
    sigma = Lam[0]
    history.append({"iter": 0, "rr": True, "trace": float(np.sum(Lam[:k])), "max_res": float(np.max(r[:k])),
                    "n_lock": len(lck)})
    it = 0
    last_was_rr = True
    while not done and it < maxiter:
        it += 1
        Xlock = Xf[:, lck]
        X = np.asfortranarray(Xf[:, act]) if last_was_rr else X
        if last_was_rr:
            W = np.asfortranarray(W[:, act])
        stats["n_locked"] = len(lck)
        k_act = X.shape[1]
        # Step 8: W <- T W
        t = time.perf_counter()
        W = precondition(W, V, N, h, sigma, delta)
        phase["Precond"] += time.perf_counter() - t
        # Steps 9-10: projections against X and X_lock
        t = time.perf_counter()
        if project_W:
            W = project(project(W, X), Xlock)
        if P is not None and project_P:
            P = project(project(P, X), Xlock)
        phase["GEMM"] += time.perf_counter() - t
        # Steps 11-16: sub-block updates
        Xn = np.empty_like(X)
        Pn = np.empty_like(W)
        for (a, b) in subblocks(k_act, q):
            Xj, Wj = X[:, a:b], W[:, a:b]
            Pj = None if P is None else P[:, a:b]
            if Pj is not None and np.any(np.linalg.norm(Pj, axis=0) == 0.0):
                Pj = None                            # R3: a zero direction (formerly locked position)
            HXj, HWj = Hop(Xj), Hop(Wj)
            HPj = None if Pj is None else Hop(Pj)
            t = time.perf_counter()
            CX, CW, CP = block_coefficients(Xj, Wj, Pj, HXj, HWj, HPj, stats)
            phase["BlockRR"] += time.perf_counter() - t
            t = time.perf_counter()
            Xn[:, a:b], Pn[:, a:b] = block_update(Xj, Wj, Pj, CX, CW, CP)
            phase["GEMM"] += time.perf_counter() - t
        X, P = Xn, Pn
        if it % rr_period != 0:
            # Steps 18-20: X <- orth(X); W <- A X - X (X* A X)
            t = time.perf_counter()
            X = orthonormalize(X, orth_mode, orth_skip_tol, stats)
            phase["CholQR"] += time.perf_counter() - t
            HX = Hop(X)
            t = time.perf_counter()
            M = X.conj().T @ HX
            W = residual(X, HX, M)
            phase["GEMM"] += time.perf_counter() - t
            wanted = [c for c, pos in enumerate(act) if pos < k]
            wf = float(np.linalg.norm(W[:, wanted]))
            history.append({"iter": it, "rr": False, "trace": float(np.real(np.trace(M))), "w_fro": wf})
            last_was_rr = False
            if wf > tol:
                continue
            stats["n_early_rr"] += 1                 # R7: forced Rayleigh-Ritz step
        # Steps 22-31
        Xf, Lam, W, r, done, lck, act, P = rr_and_lock(X, Xlock, P, act)
        n_rr += 1
        sigma = Lam[0]
        last_was_rr = True
        history.append({"iter": it, "rr": True, "trace": float(np.sum(Lam[:k])), "max_res": float(np.max(r[:k])),
                        "n_lock": len(lck)})
        if verbose:
            print(f"iter {it}: max res {np.max(r[:k]):.3e}, locked {len(lck)}")
    if not last_was_rr:
        # Step 32: a final Rayleigh-Ritz step
        Xf, Lam, W, r, done, lck, act, P = rr_and_lock(X, Xf[:, lck], P, act)
        n_rr += 1
    Xout = normalize_phase(Xf[:, :k])
    lam = np.array(Lam[:k])
    res = np.linalg.norm(apply_H(V, N, h, Xout, theta) - Xout * lam[None, :], axis=0)
    return PPCGResult(lam=lam, X=Xout, res=res, converged=bool(done),
                      iters=it, n_rr=n_rr, stats=stats, history=history, phase_s=phase)
