"""Parity of the 2-D method (a planar level: one image plane, one node
plane) on the GPU with the FP64 oracle, through the C ABI: every operator on
small and multi-tile grids at the stated bars, the z block of every field
exactly zero, Gauss-Newton and L-BFGS registrations with the oracle's
decisions, and a batched planar pair equal to its own plan."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import gpu_util as G  # noqa: E402

CASES = [
    ((5, 4, 1), (1.0, 1.0, 1.0), (3, 3, 1)),
    ((70, 35, 1), (1.0, 0.8, 1.0), (36, 18, 1)),     # 3 x 3 tiles, ragged
    ((97, 66, 1), (0.5, 0.5, 1.0), (25, 17, 1)),     # four pixels per cell
    ((40, 20, 1), (1.0, 1.0, 1.0), (41, 21, 1)),     # one pixel per cell
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _case(m, h, n, seed):
    from paper_1804_10541_b300 import synth
    R, T = synth.tissue_pair_2d(m[:2], h[:2], seed=seed, blobs=max(8, m[0] * m[1] // 100))
    N = n[0] * n[1]
    g = torch.Generator().manual_seed(seed)
    u = torch.cat([0.4 * min(h[:2]) * torch.randn(2 * N, generator=g), torch.zeros(N)])
    p = torch.cat([torch.randn(2 * N, generator=g), torch.zeros(N)])
    return G.Case(m, h, n, 0.7, 0.05, 0.08, R, T, u, p)


@pytest.mark.parametrize("m,h,n", CASES)
def test_2d_ssd_operators_match_oracle(ngf, m, h, n):
    """SSD on a planar level: the halo-free pass with one node plane against
    the oracle's planar SSD operators (pinned by the dense 2-D assembly)."""
    import oracle as O
    c = _case(m, h, n, sum(m) + 3)
    c.desc = ngf.level_desc(m, h, n, 0.7, 0.1, 0.1, distance=ngf.NGF_DIST_SSD)
    c.L = O.level(m, h, n, 0.7, distance=O.DIST_SSD)
    N = c.N
    with ngf.Plan(c.desc) as pl:
        D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
        g, q, dg = c.empty(), c.empty(), c.empty()
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g, want_scalars=False)
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, dg)
        torch.cuda.synchronize()
    Do, So = O.objective(c.L, c.Rh, c.Th, c.uh)
    assert abs(D - Do) / abs(Do) < G.TOL_OBJ and abs(S - So) / So < G.TOL_OBJ
    assert G.rel(G.f64(g), O.gradient(c.L, c.Rh, c.Th, c.uh)[0]) < G.TOL_GRAD
    assert G.rel(G.f64(q), O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)) < G.TOL_HESS
    assert G.rel(G.f64(dg), O.gn_diagonal(c.L, c.Rh, c.Th, c.uh)) < G.TOL_DIAG
    for v in (g, q):  # no z component in 2-D (the diagonal's z block holds the curvature part)
        assert not torch.any(v[2 * N:])


@pytest.mark.parametrize("m,h,n", CASES)
def test_2d_operators_match_oracle(ngf, m, h, n):
    import oracle as O
    c = _case(m, h, n, sum(m))
    N = c.N
    with ngf.Plan(c.desc) as pl:
        D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
        g = c.empty()
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g, want_scalars=False)
        q = c.empty()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        dg = c.empty()
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, dg)
        torch.cuda.synchronize()
    Do, So = O.objective(c.L, c.Rh, c.Th, c.uh)
    go, _, _ = O.gradient(c.L, c.Rh, c.Th, c.uh)
    qo = O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)
    dgo = O.gn_diagonal(c.L, c.Rh, c.Th, c.uh)
    assert abs(D - Do) / abs(Do) < G.TOL_OBJ and abs(S - So) / So < G.TOL_OBJ
    assert G.rel(G.f64(g), go) < G.TOL_GRAD
    assert G.rel(G.f64(q), qo) < G.TOL_HESS
    assert G.rel(G.f64(dg), dgo) < G.TOL_DIAG
    assert not g[2 * N:].any() and not q[2 * N:].any()  # the planar method has no z component


def _blobs(m, shift):
    y, x = np.mgrid[0:m[1], 0:m[0]] + 0.5
    img = np.zeros((m[1], m[0]))
    for cx, cy, s in ((0.3, 0.3, 0.08), (0.7, 0.45, 0.1), (0.45, 0.75, 0.07), (0.8, 0.8, 0.05)):
        img += np.exp(-((x + shift[0] - cx * m[0]) ** 2 + (y + shift[1] - cy * m[1]) ** 2) / (2 * (s * m[0]) ** 2))
    return torch.tensor(img.ravel(), dtype=torch.float32)


@pytest.mark.parametrize("method", ["gn", "lbfgs"])
def test_2d_registration_matches_oracle(ngf, method):
    import oracle as O
    m, h, n = (64, 48, 1), (1.0, 1.0, 1.0), (33, 25, 1)
    R, T = _blobs(m, (0, 0)), _blobs(m, (1.5, -1.0))
    desc = ngf.level_desc(m, h, n, 1.0, 0.05, 0.05)
    L = O.level(m, h, n, 1.0, 0.05, 0.05)
    N = n[0] * n[1]
    u = torch.zeros(3 * N, device="cuda")
    if method == "gn":
        rep = ngf.register_multilevel(desc, ngf.options(levels=2, gn_iters=3, pcg_iters=20), R.cuda(), T.cuda(), u,
                                      torch.cuda.Stream())
        uo, ro = O.register_multilevel(L, 2, O.gn_options(gn_iters=3, pcg_iters=20), G.f64(R), G.f64(T))
        assert rep.gn_done == ro.gn_done and rep.pcg_total == ro.pcg_total
    else:
        rep = ngf.register_multilevel(desc, ngf.options(levels=1, gn_iters=6, method=ngf.NGF_METHOD_LBFGS,
                                                        lbfgs_memory=5), R.cuda(), T.cuda(), u, torch.cuda.Stream())
        uo, ro, _, _ = O.lbfgs_level(L, G.f64(R), G.f64(T), np.zeros(3 * N), O.lbfgs_options(iters=6, memory=5))
        assert rep.gn_done == ro.gn_done
    du = float(np.max(np.abs(G.f64(u) - uo)))
    assert du < 0.01 and abs(rep.J - ro.J) / ro.J < 1e-5, (du, rep.J, ro.J)
    assert not u[2 * N:].any()


def test_2d_batched_pair_equals_plan(ngf):
    c = _case((70, 35, 1), (1.0, 0.8, 1.0), (36, 18, 1), 5)
    c2 = _case((40, 33, 1), (1.0, 1.0, 1.0), (21, 17, 1), 6)
    q = c.empty()
    with ngf.Plan(c.desc, zc=1) as pl:
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        torch.cuda.synchronize()
    qb = [c.empty(), c2.empty()]
    with ngf.Batch([c.desc, c2.desc], 1) as b:
        ngf.ngf_batch_hessvec(b.handle, [c.R, c2.R], [c.T, c2.T], [c.u, c2.u], [c.p, c2.p], qb)
        torch.cuda.synchronize()
    assert torch.equal(qb[0], q)
