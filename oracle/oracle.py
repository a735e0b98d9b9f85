"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg use
this module.  All arrays are float64 numpy arrays in the library's layout:
images m_x*m_y*m_z with x fastest; nodal vector fields component-major
(3 * nodes, all x components first).
"""
import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
import build as _build  # noqa: E402


DIST_NGF, DIST_SSD = 0, 1


class Level(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("h", C.c_double * 3), ("n", C.c_int32 * 3),
                ("alpha", C.c_double), ("tau", C.c_double), ("rho", C.c_double), ("distance", C.c_int32)]


class PcgInfo(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("status", C.c_int32),
                ("delta", C.c_double), ("rr", C.c_double)]


class GnOptions(C.Structure):
    _fields_ = [("gn_iters", C.c_int32), ("pcg_iters", C.c_int32), ("ls_max", C.c_int32),
                ("armijo_c1", C.c_double), ("pcg_rtol", C.c_double), ("diag_every", C.c_int32)]


class GnReport(C.Structure):
    _fields_ = [("J", C.c_double), ("D", C.c_double), ("S", C.c_double),
                ("gn_done", C.c_int32), ("pcg_total", C.c_int32), ("status", C.c_int32),
                ("ls_trials", C.c_int32)]


class LbfgsOptions(C.Structure):
    _fields_ = [("iters", C.c_int32), ("memory", C.c_int32), ("ls_max", C.c_int32),
                ("armijo_c1", C.c_double), ("gamma", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
    return _lib


def level(m, h, n, alpha=1.0, tau=0.1, rho=0.1, distance=DIST_NGF):
    L = Level()
    L.distance = int(distance)
    for a in range(3):
        L.m[a] = int(m[a])
        L.h[a] = float(h[a])
        L.n[a] = int(n[a])
    L.alpha, L.tau, L.rho = float(alpha), float(tau), float(rho)
    return L


def nvox(L):
    return L.m[0] * L.m[1] * L.m[2]


def nnod(L):
    return L.n[0] * L.n[1] * L.n[2]


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def P(L, u):
    out = np.empty(3 * nvox(L))
    lib().orc_P(C.byref(L), _p(_f64(u)), _p(out))
    return out


def PT(L, v):
    out = np.empty(3 * nnod(L))
    lib().orc_PT(C.byref(L), _p(_f64(v)), _p(out))
    return out


def warp(L, T, uh):
    Tw = np.empty(nvox(L))
    dT = np.empty(3 * nvox(L))
    lib().orc_warp(C.byref(L), _p(_f64(T)), _p(_f64(uh)), _p(Tw), _p(dT))
    return Tw, dT


def short_grad(L, I):
    g = np.empty(6 * nvox(L))
    lib().orc_short_grad(C.byref(L), _p(_f64(I)), _p(g))
    return g.reshape(-1, 6)


def residual(L, R, Tw):
    r = np.empty(nvox(L))
    lib().orc_residual(C.byref(L), _p(_f64(R)), _p(_f64(Tw)), _p(r))
    return r


def rho_hat(L, R, Tw):
    rh = np.empty(7 * nvox(L))
    lib().orc_rho_hat(C.byref(L), _p(_f64(R)), _p(_f64(Tw)), _p(rh))
    return rh.reshape(-1, 7)


def dr(L, rh, s):
    v = np.empty(nvox(L))
    lib().orc_dr(C.byref(L), _p(_f64(rh)), _p(_f64(s)), _p(v))
    return v


def drT(L, rh, v):
    t = np.empty(nvox(L))
    lib().orc_drT(C.byref(L), _p(_f64(rh)), _p(_f64(v)), _p(t))
    return t


def lap(L, u):
    out = np.empty(3 * nnod(L))
    lib().orc_lap(C.byref(L), _p(_f64(u)), _p(out))
    return out


def objective(L, R, T, u):
    D, S = C.c_double(), C.c_double()
    lib().orc_objective(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(_f64(u)), C.byref(D), C.byref(S))
    return D.value, S.value


def gradient(L, R, T, u):
    g = np.empty(3 * nnod(L))
    D, S = C.c_double(), C.c_double()
    lib().orc_gradient(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(_f64(u)), _p(g), C.byref(D), C.byref(S))
    return g, D.value, S.value


def hessvec(L, R, T, u, p):
    q = np.empty(3 * nnod(L))
    lib().orc_hessvec(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(_f64(u)), _p(_f64(p)), _p(q))
    return q


def curvature_apply(L, p):
    q = np.empty(3 * nnod(L))
    Sp = C.c_double()
    lib().orc_curvature_apply(C.byref(L), _p(_f64(p)), _p(q), C.byref(Sp))
    return q, Sp.value


def gn_diagonal(L, R, T, u):
    d = np.empty(3 * nnod(L))
    lib().orc_gn_diagonal(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(_f64(u)), _p(d))
    return d


def pcg(L, R, T, u, rhs, diag, iters, rtol=0.0):
    x = np.empty(3 * nnod(L))
    info = PcgInfo()
    lib().orc_pcg(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(_f64(u)), _p(_f64(rhs)), _p(_f64(diag)),
                  C.c_int32(iters), C.c_double(rtol), _p(x), C.byref(info))
    return x, info


def gn_options(gn_iters=10, pcg_iters=20, ls_max=10, armijo_c1=1e-4, pcg_rtol=0.0, diag_every=0):
    o = GnOptions()
    o.gn_iters, o.pcg_iters, o.ls_max = gn_iters, pcg_iters, ls_max
    o.armijo_c1, o.pcg_rtol, o.diag_every = armijo_c1, pcg_rtol, diag_every
    return o


def gn_level(L, R, T, u, opts):
    u = _f64(u).copy()
    rep = GnReport()
    trace = np.empty(2 * opts.gn_iters + 1)
    lib().orc_gn_level(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(u), C.byref(opts), C.byref(rep), _p(trace))
    return u, rep, trace


def h0_solve(L, gamma, q):
    """r = (alpha grad^2 S + gamma I)^{-1} q (Sec. 2.3.2, DCT-II eigenbasis)."""
    r = np.empty(3 * nnod(L))
    lib().orc_h0_solve(C.byref(L), C.c_double(gamma), _p(_f64(q)), _p(r))
    return r


def lbfgs_direction(L, gamma, S, Y, g):
    """d = -H_k g by the two-loop recursion; S, Y: lists of stored pairs, oldest first."""
    n = 3 * nnod(L)
    Sa = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1)) if len(S) else np.zeros(1)
    Ya = np.ascontiguousarray(np.asarray(Y, dtype=np.float64).reshape(-1)) if len(Y) else np.zeros(1)
    d = np.empty(n)
    lib().orc_lbfgs_direction(C.byref(L), C.c_double(gamma), C.c_int32(len(S)), _p(Sa), _p(Ya), _p(_f64(g)),
                              _p(d))
    return d


def lbfgs_options(iters=20, memory=5, ls_max=10, armijo_c1=1e-4, gamma=0.0):
    o = LbfgsOptions()
    o.iters, o.memory, o.ls_max, o.armijo_c1, o.gamma = iters, memory, ls_max, armijo_c1, gamma
    return o


def lbfgs_level(L, R, T, u, opts):
    """(u, report, trace, gamma) after `opts.iters` L-BFGS steps on one level."""
    u = _f64(u).copy()
    rep = GnReport()
    trace = np.empty(2 * opts.iters + 1)
    f = lib().orc_lbfgs_level
    f.restype = C.c_double
    gamma = f(C.byref(L), _p(_f64(R)), _p(_f64(T)), _p(u), C.byref(opts), C.byref(rep), _p(trace))
    return u, rep, trace, gamma


def level_at(L, lvl):
    out = Level()
    lib().orc_level_at(C.byref(L), C.c_int32(lvl), C.byref(out))
    return out


def restrict(m, img):
    mc = [(int(a) + 1) // 2 for a in m]
    out = np.empty(mc[0] * mc[1] * mc[2])
    mm = (C.c_int32 * 3)(*[int(a) for a in m])
    lib().orc_restrict(mm, _p(_f64(img)), _p(out))
    return out


def prolongate(nc, uc, nf):
    out = np.empty(3 * nf[0] * nf[1] * nf[2])
    a = (C.c_int32 * 3)(*[int(v) for v in nc])
    b = (C.c_int32 * 3)(*[int(v) for v in nf])
    lib().orc_prolongate(a, _p(_f64(uc)), b, _p(out))
    return out


def register_multilevel(L, levels, opts, R, T, u_init=None, start_level=0):
    out = np.empty(3 * nnod(L))
    rep = GnReport()
    ui = None if u_init is None else _f64(u_init)
    lib().orc_register_multilevel(C.byref(L), C.c_int32(levels), C.byref(opts), _p(_f64(R)), _p(_f64(T)),
                                  None if ui is None else _p(ui), C.c_int32(start_level), _p(out), C.byref(rep))
    return out, rep
