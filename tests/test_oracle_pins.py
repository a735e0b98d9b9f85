"""Pins of the FP64 oracle to the paper and to the mathematics (CPU only).

Nothing here re-types an oracle formula and compares it with itself: each
test checks the oracle against a hand-computed example, a closed form, an
invariant, a textbook/library special case, finite differences or the
independent dense assembled-matrix path of tests/assembled.py.
"""
import os

import numpy as np
import pytest

import assembled as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# small grids: every voxel of the first is a boundary voxel; the others span
# a non-integer voxels-per-cell ratio and a full-resolution deformation grid
TINY = [
    ((5, 4, 3), (1.0, 1.0, 1.0), (3, 3, 2)),
    ((6, 5, 4), (1.0, 0.8, 2.5), (4, 3, 3)),
    ((4, 3, 3), (0.7, 1.3, 1.1), (5, 4, 4)),
]


def _inputs(m, n, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    M = m[0] * m[1] * m[2]
    N = n[0] * n[1] * n[2]
    R = rng.random(M)
    T = rng.random(M)
    u = amp * rng.standard_normal(3 * N)
    p = rng.standard_normal(3 * N)
    return R, T, u, p


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = np.array([float(x) for x in v.split()])
    return vals


# ---------------------------------------------------------------- golden


def test_hand_example_residual_and_D(orc):
    g = _read_golden("ngf_3x1x1.txt")
    L = orc.level((3, 1, 1), (1, 1, 1), (2, 2, 2), alpha=0.0, tau=g["tau"][0], rho=g["rho"][0])
    u = np.zeros(3 * 8)
    Tw, _ = orc.warp(L, g["T"], orc.P(L, u))
    np.testing.assert_array_equal(Tw, g["T"])
    r = orc.residual(L, g["R"], Tw)
    np.testing.assert_allclose(r ** 2, g["r2"], rtol=1e-14)
    D, S = orc.objective(L, g["R"], g["T"], u)
    assert abs(D - g["D"][0]) < 1e-14 and S == 0.0
    rh = orc.rho_hat(L, g["R"], Tw)
    np.testing.assert_allclose(rh[1], g["rho_hat_1"], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- grid conversion


@pytest.mark.parametrize("m,h,n", TINY)
def test_P_matches_hat_functions(orc, m, h, n):
    L = orc.level(m, h, n)
    _, _, u, _ = _inputs(m, n, 1)
    Pd = A.P_dense(m, h, n)
    N = n[0] * n[1] * n[2]
    ref = np.concatenate([Pd @ u[d * N:(d + 1) * N] for d in range(3)])
    np.testing.assert_allclose(orc.P(L, u), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("m,h,n", TINY + [((32, 32, 32), (1, 1, 1), (17, 17, 17)),
                                          ((40, 36, 30), (0.8, 0.8, 1.0), (11, 10, 8))])
def test_P_reproduces_node_coordinates(orc, m, h, n):
    """P(x^y) = cell centres (affine reproduction) and P 1 = 1."""
    L = orc.level(m, h, n)
    _, Xs, _ = A.grid_axes(m, h, n)
    xs, _, _ = A.grid_axes(m, h, n)
    N = n[0] * n[1] * n[2]
    X = np.stack(np.meshgrid(*Xs, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(N, 3)
    x = np.stack(np.meshgrid(*xs, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    y = np.concatenate([X[:, d] for d in range(3)])
    out = orc.P(L, y).reshape(3, -1).T
    np.testing.assert_allclose(out, x, rtol=0, atol=1e-12 * max(m[a] * h[a] for a in range(3)))
    np.testing.assert_allclose(orc.P(L, np.ones(3 * N)), 1.0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("m,h,n", TINY)
def test_PT_is_adjoint(orc, m, h, n):
    L = orc.level(m, h, n)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(3 * n[0] * n[1] * n[2])
    b = rng.standard_normal(3 * m[0] * m[1] * m[2])
    lhs = orc.P(L, a) @ b
    rhs = a @ orc.PT(L, b)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


# ---------------------------------------------------------------- warp


def test_warp_identity_is_exact_and_forward(orc):
    m, h, n = (6, 5, 4), (1.0, 2.0, 0.5), (4, 3, 3)
    L = orc.level(m, h, n)
    rng = np.random.default_rng(4)
    T = rng.random(np.prod(m))
    Tw, dT = orc.warp(L, T, np.zeros(3 * np.prod(m)))
    np.testing.assert_array_equal(Tw, T)
    T3 = T.reshape(m[2], m[1], m[0])
    fx = (np.concatenate([T3[:, :, 1:], np.zeros((m[2], m[1], 1))], 2) - T3) / h[0]
    np.testing.assert_allclose(dT[:np.prod(m)], fx.ravel(), rtol=0, atol=1e-15)


def test_warp_linear_image_gradient(orc):
    """T = a . x reproduces dT = a wherever the sample's cell is interior."""
    m, h, n = (9, 8, 7), (1.0, 1.5, 2.0), (5, 5, 4)
    L = orc.level(m, h, n)
    a = np.array([0.3, -1.2, 0.7])
    xs, _, _ = A.grid_axes(m, h, n)
    x = np.stack(np.meshgrid(*xs, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    T = x @ a
    rng = np.random.default_rng(5)
    uh = 0.4 * rng.standard_normal((x.shape[0], 3)) * np.asarray(h)
    Tw, dT = orc.warp(L, T, uh.T.ravel())
    xi = (x + uh) / np.asarray(h) - 0.5
    interior = np.all((xi >= 0) & (xi < np.asarray(m) - 1), axis=1)
    assert interior.sum() > 100
    np.testing.assert_allclose(Tw[interior], ((x + uh) @ a)[interior], rtol=0, atol=1e-12)
    dTm = dT.reshape(3, -1).T
    np.testing.assert_allclose(dTm[interior], np.broadcast_to(a, dTm[interior].shape), rtol=0, atol=1e-12)


def test_warp_outside_is_zero(orc):
    m, h, n = (5, 5, 5), (1, 1, 1), (3, 3, 3)
    L = orc.level(m, h, n)
    T = np.ones(125)
    uh = np.zeros((125, 3))
    uh[:, 0] = 10.0  # every sample leaves the domain in x
    Tw, dT = orc.warp(L, T, uh.T.ravel())
    assert np.all(Tw == 0) and np.all(dT == 0)
    uh[:, 0] = -1.0 - np.arange(5)[None].repeat(25, 0).ravel()  # lands on padded index -1: zero value
    Tw, dT = orc.warp(L, T, uh.T.ravel())
    assert np.all(Tw == 0.0)
    np.testing.assert_allclose(dT[:125], 1.0)  # forward one-sided derivative at the knot


@pytest.mark.parametrize("m,h,n", TINY)
def test_warp_matches_hat_form(orc, m, h, n):
    L = orc.level(m, h, n)
    R, T, u, _ = _inputs(m, n, 6, amp=0.6)
    Tw, dT = orc.warp(L, T, orc.P(L, u))
    Tw2, dT2 = A.warp_dense(T, m, h, n, u)
    np.testing.assert_allclose(Tw, Tw2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dT.reshape(3, -1).T, dT2, rtol=0, atol=1e-8)


# ---------------------------------------------------------------- residual


@pytest.mark.parametrize("m,h,n", TINY)
def test_identical_images_give_r_one(orc, m, h, n):
    L = orc.level(m, h, n, alpha=0.0, tau=0.3, rho=0.3)
    R, _, _, _ = _inputs(m, n, 7)
    N = n[0] * n[1] * n[2]
    u = np.zeros(3 * N)
    np.testing.assert_allclose(orc.residual(L, R, R), 1.0, rtol=1e-14)
    D, S = orc.objective(L, R, R, u)
    assert abs(D) < 1e-12 and S == 0
    g, _, _ = orc.gradient(L, R, R, u)
    assert np.max(np.abs(g)) < 1e-12


def test_one_minus_r2_lagrange_identity(orc):
    """1 - r^2 equals the Lagrange-identity sum of squares divided by A^2 B^2,
    which is a different formula (no cancellation) for the same quantity."""
    m, h, n = (7, 6, 5), (1.0, 0.9, 2.0), (4, 4, 3)
    L = orc.level(m, h, n, tau=0.2, rho=0.4)
    R, T, u, _ = _inputs(m, n, 8)
    Tw, _ = orc.warp(L, T, orc.P(L, u))
    r = orc.residual(L, R, Tw)
    a = orc.short_grad(L, Tw)
    b = orc.short_grad(L, R)
    cross = np.zeros(a.shape[0])
    for p_ in range(6):
        for q_ in range(p_ + 1, 6):
            cross += (a[:, p_] * b[:, q_] - a[:, q_] * b[:, p_]) ** 2
    num = 0.25 * cross + 0.5 * np.sum((L.rho * a - L.tau * b) ** 2, axis=1)
    A2 = 0.5 * np.sum(a * a, 1) + L.tau ** 2
    B2 = 0.5 * np.sum(b * b, 1) + L.rho ** 2
    np.testing.assert_allclose(1.0 - r ** 2, num / (A2 * B2), rtol=1e-10, atol=1e-15)
    assert np.all(r ** 2 <= 1.0 + 1e-15)


def test_residual_scale_invariance(orc):
    m, h, n = (6, 6, 6), (1, 1, 1), (4, 4, 4)
    R, T, u, _ = _inputs(m, n, 9)
    L1 = orc.level(m, h, n, tau=0.2, rho=0.5)
    L2 = orc.level(m, h, n, tau=0.2 * 3.0, rho=0.5 * 7.0)
    Tw, _ = orc.warp(L1, T, orc.P(L1, u))
    np.testing.assert_allclose(orc.residual(L1, R, Tw), orc.residual(L2, 7.0 * R, 3.0 * Tw), rtol=1e-13)


# ---------------------------------------------------------------- derivatives vs assembled matrices


@pytest.mark.parametrize("m,h,n", TINY)
def test_rho_hat_rows_equal_complex_step_dr(orc, m, h, n):
    """Rows of Eq. (dr) built from rho_hat equal dr/dT by complex step, with
    at most 7 non-zeros per row."""
    L = orc.level(m, h, n, tau=0.15, rho=0.25)
    R, T, u, _ = _inputs(m, n, 10)
    Tw, _ = orc.warp(L, T, orc.P(L, u))
    rh = orc.rho_hat(L, R, Tw)
    M = Tw.size
    dense = np.zeros((M, M))
    for j in range(M):
        e = np.zeros(M)
        e[j] = 1.0
        dense[:, j] = orc.dr(L, rh, e)
    ref = A.dr_complex_step(R, Tw, m, h, 0.15, 0.25)
    np.testing.assert_allclose(dense, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert np.max(np.count_nonzero(np.abs(ref) > 1e-14, axis=1)) <= 7
    # dr^T by scattering rows equals the transpose
    v = np.random.default_rng(11).standard_normal(M)
    np.testing.assert_allclose(orc.drT(L, rh, v), ref.T @ v, rtol=0, atol=1e-12)


def test_drTdr_structure(orc):
    """dr^T dr has at most 25 non-zero diagonals (Sec. 4.1.2, Table 2), and
    the pre-image sizes of the 25 offsets add up to 7 x 7 = 49."""
    m, h, n = (6, 5, 5), (1, 1, 1), (4, 3, 3)
    L = orc.level(m, h, n)
    R, T, u, _ = _inputs(m, n, 12)
    Tw, _ = orc.warp(L, T, orc.P(L, u))
    G = A.dr_complex_step(R, Tw, m, h, 0.1, 0.1)
    G = G.T @ G
    ii, jj = np.nonzero(np.abs(G) > 1e-13)
    assert len(np.unique(jj - ii)) <= 25
    Mset = [-m[0] * m[1], -m[0], -1, 0, 1, m[0], m[0] * m[1]]
    pre = {}
    for a in Mset:
        for b in Mset:
            pre.setdefault(b - a, 0)
            pre[b - a] += 1
    assert len(pre) == 25 and sum(pre.values()) == 49
    assert set(np.unique(jj - ii)) <= set(pre.keys())


@pytest.mark.parametrize("m,h,n", TINY)
def test_gradient_matches_assembled(orc, m, h, n):
    L = orc.level(m, h, n, alpha=0.7, tau=0.15, rho=0.25)
    R, T, u, _ = _inputs(m, n, 13)
    g, D, S = orc.gradient(L, R, T, u)
    As = A.Assembled(m, h, n, 0.7, 0.15, 0.25, R, T, u)
    ref = As.gradient()
    assert abs(D - As.D()) < 1e-12 * abs(As.D())
    assert abs(S - As.S()) < 1e-10 * (abs(As.S()) + 1)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-8 * np.max(np.abs(ref)))


@pytest.mark.parametrize("m,h,n", TINY)
def test_hessvec_matches_assembled(orc, m, h, n):
    L = orc.level(m, h, n, alpha=0.7, tau=0.15, rho=0.25)
    R, T, u, p = _inputs(m, n, 14)
    q = orc.hessvec(L, R, T, u, p)
    H = A.Assembled(m, h, n, 0.7, 0.15, 0.25, R, T, u).hess_matrix()
    ref = H @ p
    np.testing.assert_allclose(q, ref, rtol=0, atol=1e-8 * np.max(np.abs(ref)))


@pytest.mark.parametrize("m,h,n", TINY)
def test_diagonal_matches_assembled(orc, m, h, n):
    L = orc.level(m, h, n, alpha=0.7, tau=0.15, rho=0.25)
    R, T, u, _ = _inputs(m, n, 15)
    d = orc.gn_diagonal(L, R, T, u)
    H = A.Assembled(m, h, n, 0.7, 0.15, 0.25, R, T, u).hess_matrix()
    np.testing.assert_allclose(d, np.diag(H), rtol=1e-7, atol=1e-9 * np.max(np.diag(H)))


def test_gradient_finite_differences(orc):
    """Central differences of J along 20 random directions at a random,
    non-knot displacement."""
    m, h, n = (9, 8, 7), (1.0, 1.2, 1.7), (5, 4, 4)
    L = orc.level(m, h, n, alpha=0.5, tau=0.1, rho=0.2)
    R, T, u, _ = _inputs(m, n, 16)
    g, _, _ = orc.gradient(L, R, T, u)
    rng = np.random.default_rng(17)

    def J(v):
        D, S = orc.objective(L, R, T, v)
        return D + L.alpha * S

    eps = 1e-6
    for _ in range(20):
        dvec = rng.standard_normal(u.size)
        fd = (J(u + eps * dvec) - J(u - eps * dvec)) / (2 * eps)
        assert abs(fd - g @ dvec) <= 1e-6 * (abs(fd) + np.linalg.norm(g))


def test_gn_hessian_equals_residual_jacobian_norm(orc):
    """p^T H_D p = 2 hbar ||J p||^2 with J p from finite differences of the
    residual vector r(T(P(u))): independent of every adjoint (P^T, dr^T)."""
    m, h, n = (8, 7, 6), (1.0, 1.0, 2.0), (5, 4, 4)
    L = orc.level(m, h, n, alpha=0.0, tau=0.1, rho=0.2)
    R, T, u, p = _inputs(m, n, 18)

    def rvec(v):
        Tw, _ = orc.warp(L, T, orc.P(L, v))
        return orc.residual(L, R, Tw)

    eps = 1e-6
    Jp = (rvec(u + eps * p) - rvec(u - eps * p)) / (2 * eps)
    hbar = h[0] * h[1] * h[2]
    lhs = p @ orc.hessvec(L, R, T, u, p)
    rhs = 2 * hbar * Jp @ Jp
    assert abs(lhs - rhs) <= 1e-6 * rhs


def test_hessian_symmetric_psd(orc):
    m, h, n = (10, 9, 8), (1.0, 1.0, 1.5), (6, 5, 5)
    L = orc.level(m, h, n, alpha=0.3, tau=0.1, rho=0.1)
    R, T, u, p = _inputs(m, n, 19)
    q = np.random.default_rng(20).standard_normal(p.size)
    Hp = orc.hessvec(L, R, T, u, p)
    Hq = orc.hessvec(L, R, T, u, q)
    assert abs(q @ Hp - p @ Hq) <= 1e-12 * (abs(q @ Hp) + 1)
    for s in range(5):
        v = np.random.default_rng(30 + s).standard_normal(p.size)
        assert v @ orc.hessvec(L, R, T, u, v) >= 0


# ---------------------------------------------------------------- curvature


def test_curvature_1d_neumann_matrix(orc):
    """A field varying only in x sees the textbook 1-D Neumann Laplacian
    tridiag(1,-2,1)/hy^2 with corner rows (-1, 1) and (1, -1)."""
    n = (9, 3, 2)
    m, h = (16, 4, 4), (1.0, 1.0, 1.0)
    L = orc.level(m, h, n)
    hy = m[0] * h[0] / (n[0] - 1)
    f = np.random.default_rng(21).standard_normal(n[0])
    K = np.diag(-2.0 * np.ones(n[0])) + np.diag(np.ones(n[0] - 1), 1) + np.diag(np.ones(n[0] - 1), -1)
    K[0, 0] = K[-1, -1] = -1.0
    expect = K @ f / hy ** 2
    N = n[0] * n[1] * n[2]
    u = np.zeros(3 * N)
    u[:N] = np.tile(f, n[1] * n[2])
    out = orc.lap(L, u)[:N].reshape(n[2], n[1], n[0])
    for z in range(n[2]):
        for y in range(n[1]):
            np.testing.assert_allclose(out[z, y], expect, rtol=1e-13, atol=1e-13)


def test_curvature_quadratic_and_null_space(orc):
    m, h, n = (12, 10, 8), (1.0, 1.0, 2.0), (7, 6, 5)
    L = orc.level(m, h, n)
    N = n[0] * n[1] * n[2]
    rng = np.random.default_rng(22)
    u = rng.standard_normal(3 * N)
    q, S = orc.curvature_apply(L, u)
    # S quadratic: u^T grad^2 S u = 2 S, which needs the clamped Laplacian to be symmetric
    assert abs(u @ q - 2 * S) <= 1e-10 * S
    # finite differences of S
    dvec = rng.standard_normal(3 * N)
    eps = 1e-5
    _, Sp = orc.curvature_apply(L, u + eps * dvec)
    _, Sm = orc.curvature_apply(L, u - eps * dvec)
    assert abs((Sp - Sm) / (2 * eps) - q @ dvec) <= 1e-7 * abs(q @ dvec)
    # translations cost nothing
    c = np.concatenate([np.full(N, 0.3), np.full(N, -1.1), np.full(N, 2.0)])
    qc, Sc = orc.curvature_apply(L, c)
    assert Sc < 1e-20 and np.max(np.abs(qc)) < 1e-12


def test_curvature_affine_interior_and_boundary(orc):
    m, h, n = (16, 16, 16), (1, 1, 1), (9, 9, 9)
    L = orc.level(m, h, n)
    _, Xs, hy = A.grid_axes(m, h, n)
    N = 9 ** 3
    X = np.stack(np.meshgrid(*Xs, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(N, 3)
    a = 0.37
    u = np.zeros(3 * N)
    u[:N] = a * X[:, 0]
    out = orc.lap(L, u)[:N].reshape(9, 9, 9)
    np.testing.assert_allclose(out[:, :, 1:-1], 0.0, atol=1e-12)
    np.testing.assert_allclose(out[:, :, 0], a / hy[0], rtol=1e-12)
    np.testing.assert_allclose(out[:, :, -1], -a / hy[0], rtol=1e-12)


def test_curvature_matches_kronecker_laplacian(orc):
    m, h, n = (10, 8, 6), (1.0, 0.5, 2.0), (6, 5, 4)
    L = orc.level(m, h, n)
    _, _, hy = A.grid_axes(m, h, n)
    Ld = A.lap_dense(n, hy)
    N = n[0] * n[1] * n[2]
    u = np.random.default_rng(23).standard_normal(3 * N)
    out = orc.lap(L, u)
    for d in range(3):
        np.testing.assert_allclose(out[d * N:(d + 1) * N], Ld @ u[d * N:(d + 1) * N], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- PCG


def test_pcg_matches_scipy_and_direct_solve(orc):
    """Jacobi PCG iterates equal scipy's preconditioned CG (a library
    routine for the same Krylov method); run to 3N iterations it reaches the
    dense direct solve."""
    from scipy.sparse.linalg import LinearOperator, cg

    m, h, n = (5, 4, 3), (1, 1, 1), (3, 3, 2)
    L = orc.level(m, h, n, alpha=0.5, tau=0.2, rho=0.2)
    R, T, u, b = _inputs(m, n, 24)
    H = A.Assembled(m, h, n, 0.5, 0.2, 0.2, R, T, u).hess_matrix()
    diag = orc.gn_diagonal(L, R, T, u)
    Minv = LinearOperator(H.shape, matvec=lambda v: v / diag)
    for k in (1, 3, 7):
        x, info = orc.pcg(L, R, T, u, b, diag, k)
        xs, _ = cg(H, b, x0=np.zeros_like(b), rtol=1e-300, atol=0.0, maxiter=k, M=Minv)
        np.testing.assert_allclose(x, xs, rtol=0, atol=1e-9 * np.linalg.norm(xs))
        assert info.iters_done == k
    x, _ = orc.pcg(L, R, T, u, b, diag, 3 * b.size)
    np.testing.assert_allclose(x, np.linalg.solve(H, b), rtol=0, atol=1e-7 * np.linalg.norm(np.linalg.solve(H, b)))


def test_pcg_zero_rhs_stops(orc):
    m, h, n = (5, 4, 3), (1, 1, 1), (3, 3, 2)
    L = orc.level(m, h, n)
    R, T, u, _ = _inputs(m, n, 25)
    diag = orc.gn_diagonal(L, R, T, u)
    x, info = orc.pcg(L, R, T, u, np.zeros(54), diag, 10)
    assert info.status == 1 and info.iters_done == 0 and np.all(x == 0)


# ---------------------------------------------------------------- multilevel


def test_level_sequence():
    import oracle as O
    L = O.level((32, 32, 32), (1, 1, 1), (17, 17, 17))
    c = O.level_at(L, 1)
    assert list(c.m) == [16, 16, 16] and list(c.n) == [9, 9, 9] and list(c.h) == [2, 2, 2]
    L = O.level((256, 256, 120), (1, 1, 2.5), (129, 129, 61))
    seq = [O.level_at(L, k) for k in range(4)]
    assert [list(s.m) for s in seq] == [[256, 256, 120], [128, 128, 60], [64, 64, 30], [32, 32, 15]]
    assert [list(s.n) for s in seq] == [[129, 129, 61], [65, 65, 31], [33, 33, 16], [17, 17, 9]]
    L = O.level((512, 512, 900), (0.8, 0.8, 1.0), (129, 129, 225))
    seq = [O.level_at(L, k) for k in range(5)]
    assert [list(s.m) for s in seq][-1] == [32, 32, 57]
    assert [list(s.n) for s in seq][-1] == [9, 9, 15]
    # the physical extent is kept on every level
    for s in seq:
        np.testing.assert_allclose([s.m[a] * s.h[a] for a in range(3)], [409.6, 409.6, 900.0])


def test_restrict_mean_and_odd_sizes(orc):
    img = np.random.default_rng(26).random(6 * 4 * 2)
    out = orc.restrict((6, 4, 2), img)
    assert abs(out.mean() - img.mean()) < 1e-14
    # odd: the last coarse cell averages only the children that exist
    img = np.arange(5.0)
    out = orc.restrict((5, 1, 1), img)
    np.testing.assert_allclose(out, [0.5, 2.5, 4.0])


def test_prolongate_reproduces_affine(orc):
    nc, nf = (5, 4, 3), (9, 7, 5)
    ext = np.array([8.0, 6.0, 4.0])
    Xc = [np.linspace(0, ext[a], nc[a]) for a in range(3)]
    Xf = [np.linspace(0, ext[a], nf[a]) for a in range(3)]
    Gc = np.stack(np.meshgrid(*Xc, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    Gf = np.stack(np.meshgrid(*Xf, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    Amat = np.array([[0.1, 0.2, -0.3], [0.0, 0.5, 0.1], [1.0, -0.2, 0.0]])
    uc = (Gc @ Amat.T + np.array([1.0, 2.0, 3.0])).T.ravel()
    uf = orc.prolongate(nc, uc, nf)
    np.testing.assert_allclose(uf, (Gf @ Amat.T + np.array([1.0, 2.0, 3.0])).T.ravel(), atol=1e-12)
    np.testing.assert_allclose(orc.prolongate(nc, uc, nc), uc, atol=1e-14)


@pytest.mark.slow
def test_gn_level_monotone_and_armijo(orc):
    from paper_1804_10541_b300 import synth
    m, h, n = (16, 16, 16), (1, 1, 1), (9, 9, 9)
    R, T, _ = synth.blob_pair(m, seed=0)
    R, T = R.double().numpy(), T.double().numpy()
    L = orc.level(m, h, n, alpha=1.0, tau=0.1, rho=0.1)
    opts = orc.gn_options(gn_iters=4, pcg_iters=10)
    u0 = np.zeros(3 * 729)
    u, rep, trace = orc.gn_level(L, R, T, u0, opts)
    Js = trace[0:2 * rep.gn_done + 1:2]
    assert rep.status == 0 and rep.gn_done == 4
    assert np.all(np.diff(Js) < 0) and Js[-1] == rep.J
    assert rep.J < 0.9 * trace[0]


def test_gn_level_diagonal_schedule(orc):
    """The Jacobi preconditioner is computed at the level's first iterate and
    kept (diag_every = 0).  Pinned by recomposing the second step from the
    building blocks: gradient at u1, PCG with the diagonal taken at u0,
    Armijo halving from eta = 1.  Refreshing at every step (diag_every = 1)
    takes the diagonal at u1 instead and gives another second step; a
    refresh interval longer than the level is the once-per-level schedule."""
    from paper_1804_10541_b300 import synth
    m, h, n = (12, 10, 8), (1.0, 1.0, 1.0), (7, 6, 5)
    R, T, _ = synth.blob_pair(m, seed=3)
    R, T = R.double().numpy(), T.double().numpy()
    L = orc.level(m, h, n, alpha=1.0, tau=0.1, rho=0.1)
    nn = 3 * orc.nnod(L)
    u0 = np.zeros(nn)
    u1, rep1, _ = orc.gn_level(L, R, T, u0, orc.gn_options(gn_iters=1, pcg_iters=10))
    u2, rep2, _ = orc.gn_level(L, R, T, u0, orc.gn_options(gn_iters=2, pcg_iters=10))
    u2e, _, _ = orc.gn_level(L, R, T, u0, orc.gn_options(gn_iters=2, pcg_iters=10, diag_every=1))
    u2l, _, _ = orc.gn_level(L, R, T, u0, orc.gn_options(gn_iters=2, pcg_iters=10, diag_every=5))
    assert rep1.gn_done == 1 and rep2.gn_done == 2
    g, D, S = orc.gradient(L, R, T, u1)
    J0 = D + 1.0 * S

    def second_step(diag):
        s, _ = orc.pcg(L, R, T, u1, -g, diag, 10)
        gs = float(g @ s)
        assert gs < 0.0
        eta = 1.0
        for _ in range(10):
            ut = u1 + eta * s
            Dt, St = orc.objective(L, R, T, ut)
            if Dt + St <= J0 + 1e-4 * eta * gs:
                return ut
            eta *= 0.5
        raise AssertionError("no Armijo step")

    np.testing.assert_allclose(u2, second_step(orc.gn_diagonal(L, R, T, u0)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(u2e, second_step(orc.gn_diagonal(L, R, T, u1)), rtol=0, atol=1e-12)
    assert np.max(np.abs(u2 - u2e)) > 1e-9
    assert np.array_equal(u2l, u2)


# ---- L-BFGS (Sec. 2.3.2) ---------------------------------------------------

def _dense_curvature_hessian(orc, L):
    """grad^2 S as a dense matrix, column by column from the curvature operator."""
    n = 3 * orc.nnod(L)
    H = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        H[:, j], _ = orc.curvature_apply(L, e)
    return H


@pytest.mark.parametrize("m,h,n,gamma", [((6, 5, 4), (1.0, 1.2, 2.0), (4, 3, 3), 0.37),
                                         ((9, 4, 3), (0.7, 1.0, 1.3), (6, 3, 2), 5.0)])
def test_h0_solve_inverts_the_curvature_hessian(orc, m, h, n, gamma):
    """(alpha grad^2 S + gamma I) r = q, checked with the curvature operator
    (stencil form, independent of the DCT eigenbasis)."""
    L = orc.level(m, h, n, alpha=0.7)
    q = np.random.default_rng(1).standard_normal(3 * orc.nnod(L))
    r = orc.h0_solve(L, gamma, q)
    cq, _ = orc.curvature_apply(L, r)
    np.testing.assert_allclose(0.7 * cq + gamma * r, q, atol=1e-12 * np.abs(q).max())
    # the translations are the null space of grad^2 S: H0 acts as gamma there
    c = np.concatenate([np.full(orc.nnod(L), v) for v in (1.0, -2.0, 0.5)])
    np.testing.assert_allclose(orc.h0_solve(L, gamma, c), c / gamma, rtol=1e-12)


def test_two_loop_recursion_equals_dense_bfgs_update(orc):
    """d = -H_k g from the two-loop recursion equals the explicit inverse-BFGS
    updates H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T applied to the
    dense inverse of H0, oldest pair first (Nocedal and Wright, Eq. 6.17)."""
    L = orc.level((5, 4, 3), (1.0, 1.0, 1.5), (3, 3, 2), alpha=0.6)
    n = 3 * orc.nnod(L)
    gamma = 0.8
    rng = np.random.default_rng(3)
    H = np.linalg.inv(0.6 * _dense_curvature_hessian(orc, L) + gamma * np.eye(n))
    S, Y = [], []
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)   # SPD: s^T y > 0
    for _ in range(4):
        s = rng.standard_normal(n)
        S.append(s)
        Y.append(A @ s)
    Hk = H.copy()
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        Hk = V.T @ Hk @ V + rho * np.outer(s, s)
    g = rng.standard_normal(n)
    d = orc.lbfgs_direction(L, gamma, S, Y, g)
    np.testing.assert_allclose(d, -Hk @ g, rtol=1e-9, atol=1e-12 * np.abs(Hk @ g).max())
    # secant condition of the newest pair
    np.testing.assert_allclose(-orc.lbfgs_direction(L, gamma, S, Y, Y[-1]), S[-1], rtol=1e-9)
    # no pairs: d = -H0^{-1} g
    np.testing.assert_allclose(orc.lbfgs_direction(L, gamma, [], [], g), -H @ g, rtol=1e-9,
                               atol=1e-12 * np.abs(H @ g).max())


@pytest.mark.slow
def test_lbfgs_level_monotone_armijo_and_default_gamma(orc):
    from paper_1804_10541_b300 import synth
    m, h, n = (16, 16, 16), (1, 1, 1), (9, 9, 9)
    R, T, _ = synth.blob_pair(m, seed=0)
    R, T = R.double().numpy(), T.double().numpy()
    L = orc.level(m, h, n, alpha=1.0, tau=0.1, rho=0.1)
    opts = orc.lbfgs_options(iters=8, memory=4)
    u0 = np.zeros(3 * 729)
    u, rep, trace, gamma = orc.lbfgs_level(L, R, T, u0, opts)
    assert np.isclose(gamma, orc.gn_diagonal(L, R, T, u0).mean(), rtol=1e-12)
    Js = trace[0:2 * rep.gn_done + 1:2]
    assert rep.status == 0 and rep.gn_done == 8 and rep.pcg_total == 0
    assert np.all(np.diff(Js) < 0) and Js[-1] == rep.J
    assert rep.J < 0.9 * trace[0]
    # every accepted step satisfied the Armijo condition: J decreased
    etas = trace[1:2 * rep.gn_done:2]
    assert np.all(etas > 0)


# ---- SSD distance (Sec. 7: dr = I) ------------------------------------------

def _ssd_assembled(m, h, n, alpha, R, T, u):
    """SSD objective, gradient and Gauss-Newton matrix from the independent
    dense factors: D = hbar/2 ||Tw - R||^2, grad = hbar (dT P)^T (Tw - R),
    H = hbar (dT P)^T (dT P) (+ alpha grad^2 S)."""
    As = A.Assembled(m, h, n, alpha, 0.1, 0.1, R, T, u)
    r = As.Tw - np.asarray(R, float)
    Jc = As.dT @ As.P
    D = 0.5 * As.hbar * np.sum(r ** 2)
    g = As.hbar * (r @ Jc) + alpha * 2.0 * As.hbary * (As.Lap.T @ (As.Lap @ As.u))
    H = As.hbar * Jc.T @ Jc + alpha * 2.0 * As.hbary * As.Lap.T @ As.Lap
    return D, g, H


@pytest.mark.parametrize("m,h,n", TINY)
def test_ssd_operators_match_assembled(orc, m, h, n):
    L = orc.level(m, h, n, alpha=0.7, distance=orc.DIST_SSD)
    R, T, u, p = _inputs(m, n, 21)
    D_ref, g_ref, H = _ssd_assembled(m, h, n, 0.7, R, T, u)
    g, D, S = orc.gradient(L, R, T, u)
    D2, _ = orc.objective(L, R, T, u)
    assert abs(D - D_ref) < 1e-12 * abs(D_ref) and D2 == D
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-9 * np.max(np.abs(g_ref)))
    q = orc.hessvec(L, R, T, u, p)
    np.testing.assert_allclose(q, H @ p, rtol=0, atol=1e-9 * np.max(np.abs(H @ p)))
    np.testing.assert_allclose(orc.gn_diagonal(L, R, T, u), np.diag(H), rtol=1e-9,
                               atol=1e-12 * np.max(np.diag(H)))


def test_ssd_gradient_finite_differences_and_identity(orc):
    m, h, n = (7, 6, 5), (1.0, 0.9, 1.3), (4, 4, 3)
    L = orc.level(m, h, n, alpha=0.3, distance=orc.DIST_SSD)
    R, T, u, _ = _inputs(m, n, 22)
    g, _, _ = orc.gradient(L, R, T, u)
    rng = np.random.default_rng(23)
    J = lambda v: (lambda DS: DS[0] + 0.3 * DS[1])(orc.objective(L, R, T, v))
    for _ in range(10):
        dvec = rng.standard_normal(u.size)
        eps = 1e-6
        fd = (J(u + eps * dvec) - J(u - eps * dvec)) / (2 * eps)
        assert abs(fd - g @ dvec) < 1e-6 * (abs(fd) + np.abs(g).max())
    # identical images, identity warp: D = 0 and grad D = 0
    L0 = orc.level(m, h, n, alpha=0.0, distance=orc.DIST_SSD)
    z = np.zeros_like(u)
    g0, D0, _ = orc.gradient(L0, R, R, z)
    assert D0 == 0.0 and np.abs(g0).max() == 0.0
