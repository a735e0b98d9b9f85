"""Pins of the oracle's 2-D method (a planar level: m[2] = n[2] = 1) against
an independent dense assembly of the 2-D factors (bilinear hat functions,
four short differences, complex-step residual Jacobian, 2-D Laplacian), finite
differences, and the planar structure (the z block of every field vanishes)."""
import numpy as np
import pytest

import assembled as A

CASES = [
    ((5, 4, 1), (1.0, 1.0, 1.0), (3, 3, 1)),
    ((6, 5, 1), (1.0, 0.8, 1.0), (4, 3, 1)),
    ((4, 3, 1), (0.7, 1.3, 2.0), (5, 4, 1)),  # full-resolution grid; h[2] has no effect
]


def _problem(m, n, seed):
    rng = np.random.default_rng(seed)
    M, N = m[0] * m[1], n[0] * n[1]
    R, T = rng.random(M), rng.random(M)
    u2 = 0.3 * rng.standard_normal(2 * N)
    u3 = np.concatenate([u2, np.zeros(N)])
    p2 = rng.standard_normal(2 * N)
    p3 = np.concatenate([p2, np.zeros(N)])
    return R, T, u2, u3, p2, p3


@pytest.mark.parametrize("m,h,n", CASES)
def test_2d_operators_match_dense_assembly(orc, m, h, n):
    R, T, u2, u3, p2, p3 = _problem(m, n, sum(m) + 1)
    L = orc.level(m, h, n, 0.7, 0.15, 0.25)
    N = n[0] * n[1]
    a = A.Assembled2D(m, h, n, 0.7, 0.15, 0.25, R, T, u2)
    D, S = orc.objective(L, R, T, u3)
    assert abs(D - a.D()) <= 1e-12 * abs(a.D())
    # the assembly's dT comes from central differences (step 1e-6): ~1e-10
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    g, _, _ = orc.gradient(L, R, T, u3)
    assert rel(g[:2 * N], a.gradient()) < 1e-8
    assert not np.any(g[2 * N:])  # no z component in 2-D
    H = a.hess_matrix()
    q = orc.hessvec(L, R, T, u3, p3)
    assert rel(q[:2 * N], H @ p2) < 1e-8
    assert not np.any(q[2 * N:])
    d = orc.gn_diagonal(L, R, T, u3)
    assert rel(d[:2 * N], np.diag(H)) < 1e-8


@pytest.mark.parametrize("m,h,n", CASES)
def test_2d_ssd_operators_match_dense_assembly(orc, m, h, n):
    """SSD on a planar level (Sec. 7: the residual is Tw - R, its Jacobian the
    identity) against the same dense 2-D factors: D = hbar/2 ||Tw - R||^2,
    grad = hbar (dT P)^T (Tw - R), H = hbar (dT P)^T (dT P), each with the
    2-D curvature term; the z block of every field stays zero."""
    R, T, u2, u3, p2, p3 = _problem(m, n, sum(m) + 7)
    L = orc.level(m, h, n, 0.7, distance=orc.DIST_SSD)
    N = n[0] * n[1]
    a = A.Assembled2D(m, h, n, 0.7, 0.15, 0.25, R, T, u2)
    res = a.Tw - R
    Jc = a.dT @ a.P
    D_ref = 0.5 * a.hbar * np.sum(res ** 2)
    g_ref = a.hbar * (res @ Jc) + 0.7 * 2.0 * a.hbary * (a.Lap.T @ (a.Lap @ u2))
    H = a.hbar * Jc.T @ Jc + 0.7 * 2.0 * a.hbary * a.Lap.T @ a.Lap
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    D, _ = orc.objective(L, R, T, u3)
    assert abs(D - D_ref) <= 1e-12 * abs(D_ref)
    g, Dg, _ = orc.gradient(L, R, T, u3)
    assert Dg == D and rel(g[:2 * N], g_ref) < 1e-8 and not np.any(g[2 * N:])
    q = orc.hessvec(L, R, T, u3, p3)
    assert rel(q[:2 * N], H @ p2) < 1e-8 and not np.any(q[2 * N:])
    d = orc.gn_diagonal(L, R, T, u3)
    assert rel(d[:2 * N], np.diag(H)) < 1e-8


def test_2d_gradient_finite_differences(orc):
    m, h, n = (9, 7, 1), (1.0, 1.2, 1.0), (5, 4, 1)
    R, T, u2, u3, _, _ = _problem(m, n, 11)
    L = orc.level(m, h, n, 0.5, 0.2, 0.2)
    N = n[0] * n[1]
    g, _, _ = orc.gradient(L, R, T, u3)
    rng = np.random.default_rng(12)
    J = lambda v: (lambda DS: DS[0] + 0.5 * DS[1])(orc.objective(L, R, T, v))
    for _ in range(10):
        dirn = np.concatenate([rng.standard_normal(2 * N), np.zeros(N)])
        e = 1e-6
        fd = (J(u3 + e * dirn) - J(u3 - e * dirn)) / (2 * e)
        assert abs(fd - g @ dirn) <= 1e-6 * max(abs(fd), 1e-8)


def test_2d_identical_images_and_planar_levels(orc):
    m, h, n = (8, 6, 1), (1.0, 1.0, 1.0), (5, 4, 1)
    R, _, _, _, _, _ = _problem(m, n, 13)
    L = orc.level(m, h, n, 1.0, 0.3, 0.3)
    D, S = orc.objective(L, R, R, np.zeros(3 * 20))
    assert abs(D) < 1e-12 and S == 0.0
    for lvl in range(3):
        Ll = orc.level_at(L, lvl)
        assert Ll.m[2] == 1 and Ll.n[2] == 1
    # prolongation between planar node grids reproduces affine fields
    nc, nf = (3, 3, 1), (5, 5, 1)
    xs = lambda nn: np.meshgrid(np.linspace(0, 1, nn[0]), np.linspace(0, 1, nn[1]), indexing="xy")
    Xc, Yc = xs(nc)
    Xf, Yf = xs(nf)
    uc = np.concatenate([(2 * Xc + Yc).ravel(), (Xc - Yc).ravel(), np.zeros(9)])
    uf = orc.prolongate(nc, uc, nf)
    assert np.allclose(uf[:25], (2 * Xf + Yf).ravel()) and np.allclose(uf[25:50], (Xf - Yf).ravel())
    assert not np.any(uf[50:])


def _blobs_2d(m, shift):
    y, x = np.mgrid[0:m[1], 0:m[0]] + 0.5
    img = np.zeros((m[1], m[0]))
    for cx, cy, s in ((5.0, 4.0, 2.0), (11.0, 7.0, 2.5), (7.5, 9.0, 1.8)):
        img += np.exp(-((x + shift[0] - cx) ** 2 + (y + shift[1] - cy) ** 2) / (2 * s * s))
    return img.ravel()


def test_2d_gauss_newton_level_descends(orc):
    m, h, n = (16, 12, 1), (1.0, 1.0, 1.0), (9, 7, 1)
    R, T = _blobs_2d(m, (0.0, 0.0)), _blobs_2d(m, (0.7, -0.5))
    L = orc.level(m, h, n, 0.5, 0.05, 0.05)
    u, rep, trace = orc.gn_level(L, R, T, np.zeros(3 * 63), orc.gn_options(gn_iters=4, pcg_iters=10))
    Js = trace[: 2 * rep.gn_done + 1: 2]
    assert rep.gn_done >= 1 and np.all(np.diff(Js) <= 0)
    assert not np.any(u[2 * 63:])
