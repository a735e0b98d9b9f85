"""Dense assembled-matrix evaluation of the method on tiny grids (test only).

This is the second, independent path the oracle is pinned against.  Every
factor of the chain rule of Eqs. (NGF_discretized_gradient) and
(NGF_discretized_hessian) is built as an explicit dense matrix by a route that
shares nothing with the oracle's row formulas:

* P from the tensor-product hat functions of the nodal grid (no floor/frac);
* the warped template and dT/dP from the hat-function form of trilinear
  interpolation on the zero-padded template, dT by central differences at
  points that are not knots (the interpolant is linear there);
* dr = dr/dT by complex-step differentiation of the residual vector, so it is
  independent of Eqs. (rho)/(hatRho) and of any boundary masking rule;
* the curvature Laplacian as a Kronecker sum of 1-D Neumann matrices.
"""
import numpy as np


def hat(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def grid_axes(m, h, n):
    """Cell centres (i + 1/2) h and node positions j * hy per axis."""
    xs = [(np.arange(m[a]) + 0.5) * h[a] for a in range(3)]
    hy = [m[a] * h[a] / (n[a] - 1) for a in range(3)]
    Xs = [np.arange(n[a]) * hy[a] for a in range(3)]
    return xs, Xs, hy


def P_dense(m, h, n):
    """Scalar block of P: (M x N), x fastest in both index spaces."""
    xs, Xs, hy = grid_axes(m, h, n)
    Pa = [hat((xs[a][:, None] - Xs[a][None, :]) / hy[a]) for a in range(3)]
    # lexicographic order with x fastest: kron(z, kron(y, x))
    return np.kron(Pa[2], np.kron(Pa[1], Pa[0]))


def interp_padded(T, m, xi):
    """Trilinear interpolant of T (zero outside) at continuous voxel coords
    xi (K x 3), written as a sum of hat functions over the padded cells."""
    T3 = T.reshape(m[2], m[1], m[0])
    out = np.zeros(xi.shape[0], dtype=np.result_type(xi, T))
    for cz in range(-1, m[2] + 1):
        wz = hat(xi[:, 2] - cz)
        if not np.any(wz):
            continue
        for cy in range(-1, m[1] + 1):
            wy = hat(xi[:, 1] - cy)
            if not np.any(wy):
                continue
            for cx in range(-1, m[0] + 1):
                inside = 0 <= cx < m[0] and 0 <= cy < m[1] and 0 <= cz < m[2]
                if not inside:
                    continue  # the zero padding contributes nothing
                out = out + T3[cz, cy, cx] * hat(xi[:, 0] - cx) * wy * wz
    return out


def warped_points(m, h, n, u):
    """Continuous voxel coordinates of the warped cell centres and the
    physical displacement P u on the image grid (M x 3)."""
    Pd = P_dense(m, h, n)
    N = n[0] * n[1] * n[2]
    uh = np.stack([Pd @ u[d * N:(d + 1) * N] for d in range(3)], axis=1)
    idx = np.stack(np.meshgrid(np.arange(m[0]), np.arange(m[1]), np.arange(m[2]), indexing="ij"), -1)
    idx = idx.transpose(2, 1, 0, 3).reshape(-1, 3).astype(float)  # x fastest
    xi = idx + uh / np.asarray(h)[None, :]
    return xi, uh


def warp_dense(T, m, h, n, u, eps=1e-6):
    xi, _ = warped_points(m, h, n, u)
    Tw = interp_padded(T, m, xi)
    dT = np.zeros((xi.shape[0], 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = eps
        dT[:, a] = (interp_padded(T, m, xi + e) - interp_padded(T, m, xi - e)) / (2 * eps * h[a])
    return Tw, dT


def short_grad_np(I, m, h):
    """6-vector of short differences with clamped neighbours (complex-safe)."""
    I3 = I.reshape(m[2], m[1], m[0])
    out = []
    for sgn in (-1, 1):
        for a, ax in ((0, 2), (1, 1), (2, 0)):
            sl = np.arange(I3.shape[ax])
            nb = np.clip(sl + sgn, 0, I3.shape[ax] - 1)
            J = np.take(I3, nb, axis=ax)
            d = (I3 - J) if sgn < 0 else (J - I3)
            out.append((d / h[a]).reshape(-1))
    return np.stack(out, axis=1)  # order -x,-y,-z,+x,+y,+z


def residual_np(R, Tw, m, h, tau, rho):
    gT = short_grad_np(Tw, m, h)
    gR = short_grad_np(R, m, h)
    num = 0.5 * np.sum(gT * gR, axis=1) + tau * rho
    nT = np.sqrt(0.5 * np.sum(gT * gT, axis=1) + tau * tau)
    nR = np.sqrt(0.5 * np.sum(gR * gR, axis=1) + rho * rho)
    return num / (nT * nR)


def dr_complex_step(R, Tw, m, h, tau, rho, step=1e-30):
    M = Tw.size
    J = np.zeros((M, M))
    for j in range(M):
        Tc = Tw.astype(complex)
        Tc[j] += 1j * step
        J[:, j] = residual_np(R.astype(complex), Tc, m, h, tau, rho).imag / step
    return J


def lap1d(n, hy):
    A = np.zeros((n, n))
    for i in range(n):
        for s in (-1, 1):
            j = min(max(i + s, 0), n - 1)
            A[i, j] += 1.0
            A[i, i] -= 1.0
    return A / (hy * hy)


def lap_dense(n, hy):
    Ix, Iy, Iz = (np.eye(n[a]) for a in range(3))
    Lx, Ly, Lz = (lap1d(n[a], hy[a]) for a in range(3))
    return np.kron(Iz, np.kron(Iy, Lx)) + np.kron(Iz, np.kron(Ly, Ix)) + np.kron(Lz, np.kron(Iy, Ix))


class Assembled:
    """All factors at one (R, T, u) on a tiny grid."""

    def __init__(self, m, h, n, alpha, tau, rho, R, T, u):
        self.m, self.h, self.n = list(m), list(h), list(n)
        self.alpha, self.tau, self.rho = alpha, tau, rho
        self.M = m[0] * m[1] * m[2]
        self.N = n[0] * n[1] * n[2]
        self.hbar = h[0] * h[1] * h[2]
        _, _, hy = grid_axes(m, h, n)
        self.hy = hy
        self.hbary = hy[0] * hy[1] * hy[2]
        Ps = P_dense(m, h, n)
        Z = np.zeros_like(Ps)
        self.P = np.block([[Ps, Z, Z], [Z, Ps, Z], [Z, Z, Ps]])
        self.Tw, dT = warp_dense(np.asarray(T, float), m, h, n, np.asarray(u, float))
        self.dT = np.hstack([np.diag(dT[:, 0]), np.diag(dT[:, 1]), np.diag(dT[:, 2])])  # Eq. (dT)
        self.r = residual_np(np.asarray(R, float), self.Tw, m, h, tau, rho)
        self.dr = dr_complex_step(np.asarray(R, float), self.Tw, m, h, tau, rho)
        Ls = lap_dense(n, hy)
        Zl = np.zeros_like(Ls)
        self.Lap = np.block([[Ls, Zl, Zl], [Zl, Ls, Zl], [Zl, Zl, Ls]])
        self.u = np.asarray(u, float)

    def D(self):
        return self.hbar * np.sum(1.0 - self.r ** 2)

    def S(self):
        return self.hbary * np.sum((self.Lap @ self.u) ** 2)

    def J_chain(self):
        return self.dr @ self.dT @ self.P

    def gradient(self):
        dpsi = -2.0 * self.hbar * self.r
        gD = (dpsi @ self.dr @ self.dT @ self.P)
        gS = 2.0 * self.hbary * (self.Lap.T @ (self.Lap @ self.u))
        return gD + self.alpha * gS

    def hess_matrix(self):
        Jc = self.J_chain()
        H = 2.0 * self.hbar * Jc.T @ Jc
        return H + self.alpha * 2.0 * self.hbary * self.Lap.T @ self.Lap


# ---------------------------------------------------------------------------
# The 2-D method, assembled on its own: pixels m0 x m1, nodes n0 x n1, two
# displacement components, bilinear hat functions, four short differences
# per pixel and the 2-D Laplacian.  Vectors are 2N long (x components, then
# y); the oracle's planar level carries a third (z) block that must vanish.

def P_dense_2d(m, h, n):
    xs = [(np.arange(m[a]) + 0.5) * h[a] for a in range(2)]
    hy = [m[a] * h[a] / (n[a] - 1) for a in range(2)]
    Xs = [np.arange(n[a]) * hy[a] for a in range(2)]
    Pa = [hat((xs[a][:, None] - Xs[a][None, :]) / hy[a]) for a in range(2)]
    return np.kron(Pa[1], Pa[0]), hy


def interp_padded_2d(T, m, xi):
    T2 = T.reshape(m[1], m[0])
    out = np.zeros(xi.shape[0], dtype=np.result_type(xi, T))
    for cy in range(m[1]):
        wy = hat(xi[:, 1] - cy)
        for cx in range(m[0]):
            out = out + T2[cy, cx] * hat(xi[:, 0] - cx) * wy
    return out


def short_grad_2d(I, m, h):
    I2 = I.reshape(m[1], m[0])
    out = []
    for sgn in (-1, 1):
        for a, ax in ((0, 1), (1, 0)):
            sl = np.arange(I2.shape[ax])
            nb = np.clip(sl + sgn, 0, I2.shape[ax] - 1)
            J = np.take(I2, nb, axis=ax)
            d = (I2 - J) if sgn < 0 else (J - I2)
            out.append((d / h[a]).reshape(-1))
    return np.stack(out, axis=1)


def residual_2d(R, Tw, m, h, tau, rho):
    gT = short_grad_2d(Tw, m, h)
    gR = short_grad_2d(R, m, h)
    num = 0.5 * np.sum(gT * gR, axis=1) + tau * rho
    return num / (np.sqrt(0.5 * np.sum(gT * gT, axis=1) + tau * tau) * np.sqrt(0.5 * np.sum(gR * gR, axis=1) + rho * rho))


class Assembled2D:
    """All factors of the 2-D method at one (R, T, u), u given as 2N."""

    def __init__(self, m, h, n, alpha, tau, rho, R, T, u, eps=1e-6):
        self.m, self.h, self.n = m, h, n
        self.alpha = alpha
        M, N = m[0] * m[1], n[0] * n[1]
        self.M, self.N = M, N
        self.hbar = h[0] * h[1]
        Ps, hy = P_dense_2d(m, h, n)
        self.hbary = hy[0] * hy[1]
        Z = np.zeros_like(Ps)
        self.P = np.block([[Ps, Z], [Z, Ps]])
        u = np.asarray(u, float)
        self.u = u
        uh = np.stack([Ps @ u[:N], Ps @ u[N:]], axis=1)
        idx = np.stack(np.meshgrid(np.arange(m[0]), np.arange(m[1]), indexing="ij"), -1)
        idx = idx.transpose(1, 0, 2).reshape(-1, 2).astype(float)
        xi = idx + uh / np.asarray(h[:2])[None, :]
        T = np.asarray(T, float)
        self.Tw = interp_padded_2d(T, m, xi)
        dT = np.zeros((M, 2))
        for a in range(2):
            e = np.zeros(2)
            e[a] = eps
            dT[:, a] = (interp_padded_2d(T, m, xi + e) - interp_padded_2d(T, m, xi - e)) / (2 * eps * h[a])
        self.dT = np.hstack([np.diag(dT[:, 0]), np.diag(dT[:, 1])])
        R = np.asarray(R, float)
        self.r = residual_2d(R, self.Tw, m, h, tau, rho)
        J = np.zeros((M, M))
        for j in range(M):
            Tc = self.Tw.astype(complex)
            Tc[j] += 1e-30j
            J[:, j] = residual_2d(R.astype(complex), Tc, m, h, tau, rho).imag / 1e-30
        self.dr = J
        Lx, Ly = lap1d(n[0], hy[0]), lap1d(n[1], hy[1])
        Ls = np.kron(np.eye(n[1]), Lx) + np.kron(Ly, np.eye(n[0]))
        Zl = np.zeros_like(Ls)
        self.Lap = np.block([[Ls, Zl], [Zl, Ls]])

    def D(self):
        return self.hbar * np.sum(1.0 - self.r ** 2)

    def gradient(self):
        gD = (-2.0 * self.hbar * self.r) @ self.dr @ self.dT @ self.P
        return gD + self.alpha * 2.0 * self.hbary * (self.Lap.T @ (self.Lap @ self.u))

    def hess_matrix(self):
        Jc = self.dr @ self.dT @ self.P
        return 2.0 * self.hbar * Jc.T @ Jc + self.alpha * 2.0 * self.hbary * self.Lap.T @ self.Lap
