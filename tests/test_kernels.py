"""GPU parity of each step of Algorithm 3, called through the C ABI, against the CPU oracle element by element.

Sizes span several tiles and a ragged tail (64-row/64-column GEMM tiles, 16-row K slices, 32-row sub-block
chunks, 32 x 32 Cholesky tiles, 32-wide stencil rows). Floating-point bars follow from the arithmetic:
a length-n dot product in FP64 differs between two summation orders by at most ~n eps sum|a_i b_i|.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import Handle, dev, host, need_gpu, ptr, torch  # noqa: F401
import paper_1407_7506_gb300 as pk

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _rng(s):
    return np.random.default_rng(s)


# ------------------------------------------------------------------------------------- operator (a0 / a6)
@pytest.mark.parametrize("N,m,h", [(3, 1, 1.0), (5, 3, 1.0), (12, 7, 0.5), (16, 2, 1.0), (33, 3, 1.0)])
def test_apply_operator(N, m, h):
    rng = _rng(N)
    V = rng.uniform(-5, 1, N ** 3)
    X = rng.standard_normal((N ** 3, m))
    with Handle(V, N, kt=min(8, N ** 3 // 2), sbsize=1, h=h) as H:
        Xd, Yd = dev(X), torch.empty((m, N ** 3), dtype=torch.float64, device="cuda")
        pk.ppcg_apply_operator(H.h, ptr(Xd), N ** 3, ptr(Yd), N ** 3, m)
        Y = host(Yd)
    ref = oracle.apply_H(V, N, h, X)
    scale = (12 / h ** 2 + np.max(np.abs(V))) * np.max(np.abs(X))
    np.testing.assert_allclose(Y, ref, rtol=0, atol=8 * EPS * scale)


# ------------------------------------------------------------------------------------- Gram (a4, a5, a10, a11)
@pytest.mark.parametrize("N,ma,mb,sym", [(4, 1, 1, False), (5, 37, 61, False), (10, 70, 130, False),
                                         (10, 64, 64, True), (16, 130, 130, True), (16, 200, 33, False)])
def test_gram(N, ma, mb, sym):
    n = N ** 3
    rng = _rng(ma * 1000 + mb)
    A = rng.standard_normal((n, ma))
    B = A if sym else rng.standard_normal((n, mb))
    with Handle(np.zeros(n), N, kt=max(ma, mb), sbsize=1) as H:
        Ad = dev(A)
        Bd = Ad if sym else dev(B)
        Cd = torch.empty((mb, ma), dtype=torch.float64, device="cuda")
        pk.ppcg_gram(H.h, ptr(Ad), n, ptr(Bd), n, ma, mb, ptr(Cd))
        C = host(Cd)
    ref = A.T @ B
    bound = 2 * n * EPS * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound + 1e-300)
    if sym:
        np.testing.assert_array_equal(C, C.T)


def test_project():
    N, mx, my = 11, 40, 25
    n = N ** 3
    rng = _rng(3)
    X = oracle.cholqr2(rng.standard_normal((n, mx)))[0]
    Y = rng.standard_normal((n, my))
    with Handle(np.zeros(n), N, kt=mx, sbsize=1) as H:
        Xd, Yd = dev(X), dev(Y)
        pk.ppcg_project(H.h, ptr(Xd), n, mx, ptr(Yd), n, my)
        Z = host(Yd)
    ref = oracle.project(Y, X)
    np.testing.assert_allclose(Z, ref, rtol=0, atol=1e-12 * np.max(np.abs(Y)))
    assert np.max(np.abs(X.T @ Z)) < 1e-12


# ------------------------------------------------------------------------------------- CholQR2 (a1, a10)
@pytest.mark.parametrize("N,m,cond", [(8, 1, 1.0), (10, 33, 1e3), (13, 50, 1e5), (16, 129, 1e2)])
def test_cholqr2(N, m, cond):
    n = N ** 3
    rng = _rng(m)
    U = oracle.cholqr2(rng.standard_normal((n, m)))[0]
    Vm = oracle.cholqr2(rng.standard_normal((m, m)))[0]
    X = U @ np.diag(np.logspace(0, np.log10(cond), m)) @ Vm.T
    with Handle(np.zeros(n), N, kt=m, sbsize=1) as H:
        Xd = dev(X)
        fb = pk.ppcg_cholqr2(H.h, ptr(Xd), n, m)
        Q = host(Xd)
    assert fb == 0
    Qref, _ = oracle.cholqr2(X)
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(Q, Qref, rtol=0, atol=1e-13 * cond)


def test_cholqr2_breakdown_falls_back_to_shifted_cholqr3():
    N, m = 10, 12
    n = N ** 3
    rng = _rng(5)
    X = rng.standard_normal((n, m))
    X[:, -1] = X[:, 0] + 1e-12 * rng.standard_normal(n)
    with Handle(np.zeros(n), N, kt=m, sbsize=1) as H:
        Xd = dev(X)
        fb = pk.ppcg_cholqr2(H.h, ptr(Xd), n, m)
        Q = host(Xd)
    assert fb == 1
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-12)
    Qref, _ = oracle.shifted_cholqr3(X)
    # the QR factor is unique, but its last column is determined by a 1e-12 component: compare the others
    np.testing.assert_allclose(Q[:, :-1], Qref[:, :-1], atol=1e-10)


# ------------------------------------------------------------------------------------- dense eigh (a12)
@pytest.mark.parametrize("m", [1, 2, 3, 17, 64, 101, 256])
def test_dense_eigh(m):
    rng = _rng(m)
    Q = oracle.cholqr2(rng.standard_normal((max(2 * m, 8), m)))[0][:m, :] if m > 1 else np.ones((1, 1))
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    lam = np.sort(rng.uniform(-4, 8, m))
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    with Handle(np.zeros(8 ** 3 if m <= 256 else 16 ** 3), 8, kt=max(m, 1), sbsize=1) as H:
        Md = dev(M)
        ld = torch.empty(m, dtype=torch.float64, device="cuda")
        Cd = torch.empty((m, m), dtype=torch.float64, device="cuda")
        pk.ppcg_dense_eigh(H.h, ptr(Md), m, ptr(ld), ptr(Cd))
        got_l = ld.cpu().numpy()
        C = host(Cd)
    ref_l, ref_C = np.linalg.eigh(M)
    nrm = np.linalg.norm(M)
    np.testing.assert_allclose(got_l, ref_l, rtol=0, atol=1e-13 * max(nrm, 1))
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(M @ C, C * got_l, atol=1e-12 * max(nrm, 1))
    gaps = np.min(np.abs(np.subtract.outer(ref_l, ref_l)) + np.eye(m) * 1e9, axis=1) if m > 1 else np.array([1.0])
    dots = np.abs(np.einsum("ij,ij->j", C, ref_C))
    assert np.all(1.0 - dots <= 1e-20 / np.minimum(gaps, 1.0) ** 2 + 1e-12)


def test_dense_eigh_degenerate_cluster():
    # a multiple eigenvalue: only the invariant subspace is unique; check the defining properties
    m = 40
    rng = _rng(9)
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    lam = np.concatenate([np.full(5, 1.0), np.linspace(2, 5, m - 5)])
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    with Handle(np.zeros(8 ** 3), 8, kt=m, sbsize=1) as H:
        Md = dev(M)
        ld = torch.empty(m, dtype=torch.float64, device="cuda")
        Cd = torch.empty((m, m), dtype=torch.float64, device="cuda")
        pk.ppcg_dense_eigh(H.h, ptr(Md), m, ptr(ld), ptr(Cd))
        got_l, C = ld.cpu().numpy(), host(Cd)
    np.testing.assert_allclose(got_l, np.sort(lam), atol=1e-13)
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(M @ C, C * got_l, atol=1e-12)
    Pg = C[:, :5] @ C[:, :5].T
    Pr = Q[:, :5] @ Q[:, :5].T
    assert np.linalg.norm(Pg - Pr, 2) < 1e-12


def _eigh_dev(M, m, N=8):
    with Handle(np.zeros(N ** 3), N, kt=max(m, 1), sbsize=1) as H:
        Md = dev(M)
        ld = torch.empty(m, dtype=torch.float64, device="cuda")
        Cd = torch.empty((m, m), dtype=torch.float64, device="cuda")
        pk.ppcg_dense_eigh(H.h, ptr(Md), m, ptr(ld), ptr(Cd))
        return ld.cpu().numpy(), host(Cd)


@pytest.mark.parametrize("m,eps", [(40, 1e-6), (256, 1e-9), (256, 1e-6), (200, 3e-5)])
def test_dense_eigh_nearly_diagonal(m, eps):
    # the Rayleigh-Ritz matrices of a converging solve: off-diagonal entries far below the gaps (refinement route)
    rng = _rng(m + 11)
    lam = rng.permutation(np.linspace(-3.0, 5.0, m))
    B = rng.standard_normal((m, m))
    M = np.diag(lam) + eps * (B + B.T)
    got_l, C = _eigh_dev(M, m)
    ref_l = np.linalg.eigvalsh(M)
    nrm = np.linalg.norm(M)
    np.testing.assert_allclose(got_l, ref_l, rtol=0, atol=1e-13 * nrm)
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(M @ C, C * got_l, atol=1e-12 * nrm)


def test_dense_eigh_diagonal_and_cluster():
    m = 64
    rng = _rng(5)
    lam = rng.permutation(np.linspace(-1.0, 2.0, m))
    # exactly diagonal, unsorted: the eigenvectors are unit vectors in ascending order of the diagonal
    got_l, C = _eigh_dev(np.diag(lam), m)
    np.testing.assert_array_equal(got_l, np.sort(lam))
    np.testing.assert_array_equal(C, np.eye(m)[:, np.argsort(lam, kind="stable")])
    # nearly diagonal with two entries 1e-13 apart coupled by 1e-9: refinement cannot separate the pair
    lam2 = lam.copy()
    lam2[7] = lam2[3] + 1e-13
    M = np.diag(lam2)
    M[3, 7] = M[7, 3] = 1e-9
    M[10, 20] = M[20, 10] = 1e-7
    got_l, C = _eigh_dev(M, m)
    np.testing.assert_allclose(got_l, np.linalg.eigvalsh(M), rtol=0, atol=1e-14)
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-13)
    np.testing.assert_allclose(M @ C, C * got_l, atol=1e-14)


def _eigh_case(kind, m, rng):
    """Symmetric test matrices of the shapes a Rayleigh-Ritz step meets: a random spectrum, clusters of ten values
    10^-12 apart, exact multiplicity 8, and a nearly diagonal matrix (off-diagonal 1e-3)."""
    if kind == "neardiag":
        B = rng.standard_normal((m, m))
        return np.diag(np.sort(rng.standard_normal(m)) * 10) + 1e-3 * (B + B.T)
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    if kind == "random":
        lam = rng.standard_normal(m)
    elif kind == "clustered":
        lam = np.concatenate([rng.standard_normal(m - 60), np.repeat(rng.standard_normal(6), 10) +
                              1e-12 * rng.standard_normal(60)])
    else:                                            # "degenerate"
        lam = np.repeat(rng.standard_normal(m // 8), 8)
    M = (Q * lam) @ Q.T
    return 0.5 * (M + M.T)


@pytest.mark.parametrize("fp64_gemm", [0, 1])
@pytest.mark.parametrize("kind", ["random", "clustered", "degenerate", "neardiag"])
@pytest.mark.parametrize("m", [512, 1024])
def test_dense_eigh_large(m, kind, fp64_gemm):
    # the k x k eigensolve at the sizes of the 48^3, k = 1024 workload: the single-precision Jacobi start and the
    # FP64 refinement with cluster solves (m x m products on the FP64 pipe, or on the tensor cores when the handle
    # emulates its FP64 GEMMs), against LAPACK
    rng = _rng(m + len(kind))
    M = _eigh_case(kind, m, rng)
    with Handle(np.zeros(16 ** 3), 16, kt=m, sbsize=1, fp64_gemm=fp64_gemm) as H:
        Md = dev(M)
        ld = torch.empty(m, dtype=torch.float64, device="cuda")
        Cd = torch.empty((m, m), dtype=torch.float64, device="cuda")
        pk.ppcg_dense_eigh(H.h, ptr(Md), m, ptr(ld), ptr(Cd))
        got_l, C = ld.cpu().numpy(), host(Cd)
    ref_l = np.linalg.eigvalsh(M)
    nrm = np.linalg.norm(M)
    np.testing.assert_allclose(got_l, ref_l, rtol=0, atol=1e-13 * nrm)
    np.testing.assert_allclose(C.T @ C, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(M @ C, C * got_l, atol=1e-12 * nrm)
    if kind == "degenerate":                          # 8-fold eigenspaces against LAPACK's projectors
        _, U = np.linalg.eigh(M)
        vals = ref_l[::8]
        for g in range(0, m // 8, 16):
            gap = np.min(np.abs(np.delete(vals, g) - vals[g]))
            P1, P2 = C[:, 8 * g:8 * g + 8] @ C[:, 8 * g:8 * g + 8].T, U[:, 8 * g:8 * g + 8] @ U[:, 8 * g:8 * g + 8].T
            assert np.linalg.norm(P1 - P2, 2) <= 1e-13 * nrm / gap


def test_dense_eigh_tiny_and_repeated_diagonal():
    # m = 1 and m = 2 (diagonal, nearly diagonal, dense) and a diagonal with repeated values: equal eigenvalues
    # keep their index order, so the eigenvectors are the unit vectors in a stable sort of the diagonal
    got_l, C = _eigh_dev(np.array([[-2.5]]), 1)
    np.testing.assert_array_equal(got_l, [-2.5])
    np.testing.assert_array_equal(C, [[1.0]])
    for M in (np.diag([3.0, -1.0]), np.array([[3.0, 1e-9], [1e-9, -1.0]]), np.array([[1.0, 2.0], [2.0, -3.0]])):
        got_l, C = _eigh_dev(M, 2)
        np.testing.assert_allclose(got_l, np.linalg.eigvalsh(M), rtol=0, atol=1e-14 * np.linalg.norm(M))
        np.testing.assert_allclose(C.T @ C, np.eye(2), atol=1e-15)
        np.testing.assert_allclose(M @ C, C * got_l, atol=1e-14 * np.linalg.norm(M))
    d = np.array([2.0, 0.5, 2.0, -1.0, 0.5, 2.0, 0.0, -1.0])
    got_l, C = _eigh_dev(np.diag(d), len(d))
    np.testing.assert_array_equal(got_l, np.sort(d))
    np.testing.assert_array_equal(C, np.eye(len(d))[:, np.argsort(d, kind="stable")])


# ------------------------------------------------------------------------------------- sub-blocks (a7, a8, a9)
def _block_inputs(N, k, seed, with_p):
    n = N ** 3
    rng = _rng(seed)
    V = rng.random(n)
    X = oracle.cholqr2(rng.standard_normal((n, k)))[0]
    W = oracle.project(rng.standard_normal((n, k)), X)
    P = oracle.project(rng.standard_normal((n, k)), X) if with_p else None
    H = lambda Y: oracle.apply_H(V, N, 1.0, Y)
    return V, X, W, P, H(X), H(W), (H(P) if with_p else None)


def _canon(C):
    """Fix each column's sign by its largest-modulus entry."""
    C = C.copy()
    for j in range(C.shape[1]):
        i = np.argmax(np.abs(C[:, j]))
        C[:, j] *= np.sign(C[i, j])
    return C


def _run_block(H, X, W, P, HX, HW, HP, k, q):
    n = X.shape[0]
    s = -(-k // q)
    coef = torch.zeros(s * 3 * q * q, dtype=torch.float64, device="cuda")
    flags = torch.full((s,), -1, dtype=torch.int32, device="cuda")
    Xd, Wd, HXd, HWd = dev(X), dev(W), dev(HX), dev(HW)
    Pd = dev(P) if P is not None else None
    HPd = dev(HP) if HP is not None else None
    pk.ppcg_block_coefficients(H.h, ptr(Xd), ptr(Wd), ptr(Pd), ptr(HXd), ptr(HWd), ptr(HPd), n, k,
                               1 if P is not None else 0, ptr(coef), ptr(flags))
    torch.cuda.synchronize()
    return coef.cpu().numpy(), flags.cpu().numpy()


@pytest.mark.parametrize("N,k,q,with_p", [(8, 7, 1, False), (8, 7, 1, True), (9, 10, 4, True), (9, 10, 4, False),
                                          (10, 9, 3, True), (10, 16, 8, True), (12, 33, 16, True)])
def test_block_coefficients(N, k, q, with_p):
    V, X, W, P, HX, HW, HP = _block_inputs(N, k, 100 + k + q, with_p)
    with Handle(V, N, kt=k, sbsize=q) as H:
        coef, flags = _run_block(H, X, W, P, HX, HW, HP, k, q)
    assert np.all(flags == 0)
    for j, (a, b) in enumerate(oracle.subblocks(k, q)):
        qj = b - a
        CX, CW, CP = oracle.block_coefficients(X[:, a:b], W[:, a:b], None if P is None else P[:, a:b],
                                               HX[:, a:b], HW[:, a:b], None if P is None else HP[:, a:b])
        ref = np.vstack([CX, CW, CP if CP is not None else np.zeros((qj, qj))])
        slot = coef[j * 3 * q * q:(j + 1) * 3 * q * q].reshape(q, 3 * q).T[:3 * qj, :qj]
        np.testing.assert_allclose(_canon(slot), _canon(ref), rtol=0, atol=1e-9 * np.max(np.abs(ref)))


def test_block_coefficients_drop_p_backtrack():
    # P_j = W_j makes S_j rank deficient: the Cholesky pivot test triggers the back-track without P
    N, k, q = 8, 6, 2
    V, X, W, P, HX, HW, HP = _block_inputs(N, k, 7, True)
    P[:, 2:4] = W[:, 2:4]
    HP[:, 2:4] = HW[:, 2:4]
    with Handle(V, N, kt=k, sbsize=q) as H:
        coef, flags = _run_block(H, X, W, P, HX, HW, HP, k, q)
    assert list(flags) == [0, 1, 0]
    CX, CW, CP = oracle.block_coefficients(X[:, 2:4], W[:, 2:4], P[:, 2:4], HX[:, 2:4], HW[:, 2:4], HP[:, 2:4])
    assert CP is None
    slot = coef[1 * 3 * q * q:2 * 3 * q * q].reshape(q, 3 * q).T
    np.testing.assert_allclose(_canon(slot[:2 * q]), _canon(np.vstack([CX, CW])), atol=1e-9)
    np.testing.assert_array_equal(slot[2 * q:], 0.0)


@pytest.mark.parametrize("k,q,with_p", [(7, 1, True), (10, 4, True), (10, 4, False), (33, 16, True)])
def test_block_update(k, q, with_p):
    N = 9
    n = N ** 3
    rng = _rng(k + q)
    X, W = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    P = rng.standard_normal((n, k)) if with_p else np.zeros((n, k))
    s = -(-k // q)
    coef = np.zeros(s * 3 * q * q)
    refX, refP = np.empty_like(X), np.empty_like(X)
    for j, (a, b) in enumerate(oracle.subblocks(k, q)):
        qj = b - a
        C = rng.standard_normal((3 * qj, qj))
        if not with_p:
            C[2 * qj:] = 0.0
        slot = np.zeros((3 * q, q))
        slot[:3 * qj, :qj] = C
        coef[j * 3 * q * q:(j + 1) * 3 * q * q] = slot.T.ravel()
        refX[:, a:b], refP[:, a:b] = oracle.block_update(X[:, a:b], W[:, a:b], P[:, a:b] if with_p else None,
                                                         C[:qj], C[qj:2 * qj], C[2 * qj:] if with_p else None)
    with Handle(np.zeros(n), N, kt=k, sbsize=q) as H:
        Xd, Wd, Pd = dev(X), dev(W), dev(P)
        cd = torch.from_numpy(coef).cuda()
        pk.ppcg_block_update(H.h, ptr(Xd), ptr(Wd), ptr(Pd), n, k, 1 if with_p else 0, ptr(cd))
        gX, gP = host(Xd), host(Pd)
    np.testing.assert_allclose(gP, refP, atol=1e-13 * np.max(np.abs(refP)))
    np.testing.assert_allclose(gX, refX, atol=1e-13 * np.max(np.abs(refX)))


# ------------------------------------------------------------------------------------- residual + precond (a3, a11)
@pytest.mark.parametrize("use_M", [True, False])
def test_residual_preconditioned(use_M):
    N, m = 10, 21
    n = N ** 3
    rng = _rng(11)
    V = rng.uniform(-3, 1, n)
    X = oracle.cholqr2(rng.standard_normal((n, m)))[0]
    HX = oracle.apply_H(V, N, 1.0, X)
    sigma = -1.5
    if use_M:
        M = X.T @ HX
        R = oracle.residual(X, HX, M)
    else:
        lam = np.linspace(-1, 3, m)
        R = oracle.residual(X, HX, lam)
    ref_W = oracle.precondition(R, V, N, 1.0, sigma)
    with Handle(V, N, kt=m, sbsize=1) as H:
        Xd, HXd = dev(X), dev(HX)
        Wd = torch.empty_like(Xd)
        nd = torch.empty(m, dtype=torch.float64, device="cuda")
        Md = dev(M) if use_M else None
        ld = torch.from_numpy(lam).cuda() if not use_M else None
        pk.ppcg_residual(H.h, ptr(Xd), ptr(HXd), n, m, ptr(Md), ptr(ld), sigma, ptr(Wd), ptr(nd))
        W, nrm = host(Wd), nd.cpu().numpy()
    np.testing.assert_allclose(W, ref_W, rtol=0, atol=1e-12 * np.max(np.abs(ref_W)))
    np.testing.assert_allclose(nrm, np.sum(R * R, axis=0), rtol=1e-10)


# ------------------------------------------------------------------------------------- mixed form: tcgen05 TF32
U_TF32 = 2.0 ** -11          # unit roundoff of TF32 (10 explicit mantissa bits, round to nearest)


@pytest.mark.parametrize("N,ma,mb,sym", [(5, 37, 61, False), (10, 70, 130, False), (16, 256, 256, False),
                                         (16, 130, 130, True), (16, 200, 33, False), (10, 1, 1, False),
                                         (30, 300, 260, False), (32, 256, 256, True)])
def test_gram_tensor_core_tf32(N, ma, mb, sym):
    n = N ** 3
    rng = _rng(ma * 1000 + mb + 7)
    A = rng.standard_normal((n, ma))
    B = A if sym else rng.standard_normal((n, mb))
    with Handle(np.zeros(n), N, kt=max(ma, mb), sbsize=1, precision=1) as H:
        Ad = dev(A)
        Bd = Ad if sym else dev(B)
        Cd = torch.empty((mb, ma), dtype=torch.float64, device="cuda")
        pk.ppcg_gram(H.h, ptr(Ad), n, ptr(Bd), n, ma, mb, ptr(Cd))
        C = host(Cd)
    ref = A.T @ B
    # each product carries two TF32 roundings; FP32 accumulation over a chunk adds far less
    bound = (2.2 * U_TF32 + 1e-5) * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert np.max(np.abs(C - ref)) > 0            # it really ran in reduced precision
    if sym:
        np.testing.assert_array_equal(C, C.T)


# n >= 19456 (N = 30, 32) takes the 256-row update tiles, smaller n the 128-row ones
@pytest.mark.parametrize("N,mx,my", [(11, 40, 25), (16, 256, 256), (16, 130, 70), (32, 256, 256), (30, 130, 300)])
def test_project_tensor_core_tf32(N, mx, my):
    n = N ** 3
    rng = _rng(mx + my)
    X = oracle.cholqr2(rng.standard_normal((n, mx)))[0]
    Y = rng.standard_normal((n, my))
    with Handle(np.zeros(n), N, kt=max(mx, my), sbsize=1, precision=1) as H:
        Xd, Yd = dev(X), dev(Y)
        pk.ppcg_project(H.h, ptr(Xd), n, mx, ptr(Yd), n, my)
        Z = host(Yd)
    ref = oracle.project(Y, X)
    # G = X^T Y has TF32 errors ~ 2u |X|^T |Y|; W - X G adds ~ 2u |X| |G|
    G_abs = np.abs(X).T @ np.abs(Y)
    bound = 2.2 * U_TF32 * (np.abs(X) @ G_abs) * 2 + 1e-12
    assert np.all(np.abs(Z - ref) <= bound)
    # the projection still removes span(X) up to the TF32 level
    assert np.max(np.abs(X.T @ Z)) < 50 * U_TF32 * np.max(np.abs(Y)) * np.sqrt(n)


# ------------------------------------------------------------------------------------- mixed form: tcgen05 BF16
U_BF16 = 2.0 ** -8           # unit roundoff of BF16 (7 explicit mantissa bits, round to nearest)


@pytest.mark.parametrize("N,ma,mb,sym", [(5, 37, 61, False), (10, 70, 130, False), (16, 256, 256, False),
                                         (16, 130, 130, True), (16, 200, 33, False), (10, 1, 1, False),
                                         (30, 300, 260, False), (32, 256, 256, True)])
def test_gram_tensor_core_bf16(N, ma, mb, sym):
    # kind::f16 with BF16 operands (converted from FP64 on load, round to nearest) and FP32 accumulation
    n = N ** 3
    rng = _rng(ma * 1000 + mb + 9)
    A = rng.standard_normal((n, ma))
    B = A if sym else rng.standard_normal((n, mb))
    with Handle(np.zeros(n), N, kt=max(ma, mb), sbsize=1, precision=2) as H:
        Ad = dev(A)
        Bd = Ad if sym else dev(B)
        Cd = torch.empty((mb, ma), dtype=torch.float64, device="cuda")
        pk.ppcg_gram(H.h, ptr(Ad), n, ptr(Bd), n, ma, mb, ptr(Cd))
        C = host(Cd)
    ref = A.T @ B
    # each product carries two BF16 roundings; the FP32 accumulation adds far less
    bound = (2.2 * U_BF16 + 1e-5) * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert np.max(np.abs(C - ref) / bound) > 1e-3      # the BF16 rounding is really there
    if sym:
        np.testing.assert_array_equal(C, C.T)


@pytest.mark.parametrize("N,mx,my", [(10, 17, 5), (16, 64, 64), (30, 300, 260), (32, 256, 1)])
def test_project_tensor_core_bf16(N, mx, my):
    n = N ** 3
    rng = _rng(mx + my + 1)
    X = oracle.cholqr2(rng.standard_normal((n, mx)))[0]
    Y = rng.standard_normal((n, my))
    with Handle(np.zeros(n), N, kt=max(mx, my), sbsize=1, precision=2) as H:
        Xd, Yd = dev(X), dev(Y)
        pk.ppcg_project(H.h, ptr(Xd), n, mx, ptr(Yd), n, my)
        Z = host(Yd)
    ref = oracle.project(Y, X)
    # G = X^T Y has BF16 errors ~ 2u |X|^T |Y|; W - X G adds ~ 2u |X| |G|
    G_abs = np.abs(X).T @ np.abs(Y)
    bound = 2.2 * U_BF16 * (np.abs(X) @ G_abs) * 2 + 1e-12
    assert np.all(np.abs(Z - ref) <= bound)
    # the projection still removes span(X) up to the BF16 level
    assert np.max(np.abs(X.T @ Z)) < 50 * U_BF16 * np.max(np.abs(Y)) * np.sqrt(n)


# ------------------------------------------------------------------------------------- FP64 emulation (Ozaki)
@pytest.mark.parametrize("N,ma,mb,sym,spread", [(5, 37, 61, False, 0), (10, 70, 130, False, 30),
                                                (16, 256, 256, False, 0), (16, 130, 130, True, 20),
                                                (16, 200, 33, False, 5), (10, 1, 1, False, 0)])
def test_gram_fp64_emulation(N, ma, mb, sym, spread):
    # columns scaled by 2^[-spread, spread], one zero column: the per-column exponents must follow
    n = N ** 3
    rng = _rng(ma * 31 + mb)
    A = rng.standard_normal((n, ma)) * np.exp2(rng.integers(-spread, spread + 1, ma))[None, :]
    if ma > 2:
        A[:, 1] = 0.0
    B = A if sym else rng.standard_normal((n, mb)) * np.exp2(rng.integers(-spread, spread + 1, mb))[None, :]
    with Handle(np.zeros(n), N, kt=max(ma, mb), sbsize=1, fp64_gemm=1) as H:
        Ad = dev(A)
        Bd = Ad if sym else dev(B)
        Cd = torch.empty((mb, ma), dtype=torch.float64, device="cuda")
        pk.ppcg_gram(H.h, ptr(Ad), n, ptr(Bd), n, ma, mb, ptr(Cd))
        C = host(Cd)
    ref = A.T @ B
    bound = 2 * n * EPS * (np.abs(A).T @ np.abs(B))          # the FP64 GEMM bar of test_gram
    assert np.all(np.abs(C - ref) <= bound + 1e-300), np.max(np.abs(C - ref) / (bound + 1e-300))
    if sym:
        np.testing.assert_array_equal(C, C.T)


@pytest.mark.parametrize("N,mx,my", [(11, 40, 25), (16, 256, 256), (13, 70, 130)])
def test_project_fp64_emulation(N, mx, my):
    n = N ** 3
    rng = _rng(mx + 3 * my)
    X = oracle.cholqr2(rng.standard_normal((n, mx)))[0]
    Y = rng.standard_normal((n, my))
    with Handle(np.zeros(n), N, kt=max(mx, my), sbsize=1, fp64_gemm=1) as H:
        Xd, Yd = dev(X), dev(Y)
        pk.ppcg_project(H.h, ptr(Xd), n, mx, ptr(Yd), n, my)
        Z = host(Yd)
    np.testing.assert_allclose(Z, oracle.project(Y, X), rtol=0, atol=1e-12 * np.max(np.abs(Y)))
    assert np.max(np.abs(X.T @ Z)) < 1e-12


@pytest.mark.parametrize("N,m,cond", [(10, 33, 1e3), (16, 129, 1e2)])
def test_cholqr2_fp64_emulation(N, m, cond):
    n = N ** 3
    rng = _rng(m + 1)
    U = oracle.cholqr2(rng.standard_normal((n, m)))[0]
    Vm = oracle.cholqr2(rng.standard_normal((m, m)))[0]
    X = U @ np.diag(np.logspace(0, np.log10(cond), m)) @ Vm.T
    with Handle(np.zeros(n), N, kt=m, sbsize=1, fp64_gemm=1) as H:
        Xd = dev(X)
        assert pk.ppcg_cholqr2(H.h, ptr(Xd), n, m) == 0
        Q = host(Xd)
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(Q, oracle.cholqr2(X)[0], rtol=0, atol=1e-13 * cond)


def test_residual_fp64_emulation():
    N, m = 10, 21
    n = N ** 3
    rng = _rng(12)
    V = rng.uniform(-3, 1, n)
    X = oracle.cholqr2(rng.standard_normal((n, m)))[0]
    HX = oracle.apply_H(V, N, 1.0, X)
    M = X.T @ HX
    R = oracle.residual(X, HX, M)
    ref_W = oracle.precondition(R, V, N, 1.0, -1.5)
    with Handle(V, N, kt=m, sbsize=1, fp64_gemm=1) as H:
        Xd, HXd, Md = dev(X), dev(HX), dev(M)
        Wd = torch.empty_like(Xd)
        nd = torch.empty(m, dtype=torch.float64, device="cuda")
        pk.ppcg_residual(H.h, ptr(Xd), ptr(HXd), n, m, ptr(Md), None, -1.5, ptr(Wd), ptr(nd))
        W, nrm = host(Wd), nd.cpu().numpy()
    np.testing.assert_allclose(W, ref_W, rtol=0, atol=1e-12 * np.max(np.abs(ref_W)))
    np.testing.assert_allclose(nrm, np.sum(R * R, axis=0), rtol=1e-10)
