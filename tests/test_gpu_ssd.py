"""SSD distance (Sec. 7: the residual Jacobian is the identity) on the GPU.

Objective, gradient, Gauss-Newton Hessian-vector product and Jacobi diagonal
against the FP64 oracle (whose SSD operators are pinned against the dense
assembled factors), and a Gauss-Newton level against the oracle's.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import gpu_util as G  # noqa: E402

CASES = [
    ((5, 4, 3), (1.0, 1.0, 1.0), (3, 3, 2)),
    ((6, 5, 4), (1.0, 0.8, 2.5), (4, 3, 3)),
    ((4, 3, 3), (0.7, 1.3, 1.1), (5, 4, 4)),
    ((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11)),
    ((65, 33, 40), (0.8, 0.8, 1.0), (17, 9, 11)),
    ((256, 256, 120), (1.0, 1.0, 2.5), (129, 129, 61)),
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _ssd_case(ngf, m, h, n, seed):
    import oracle as O
    c = G.random_case(m, h, n, alpha=0.7, seed=seed)
    c.desc = ngf.level_desc(m, h, n, 0.7, 0.1, 0.1, distance=ngf.NGF_DIST_SSD)
    c.L = O.level(m, h, n, 0.7, distance=O.DIST_SSD)
    return c


@pytest.mark.parametrize("m,h,n", CASES)
def test_ssd_operators_match_oracle(ngf, m, h, n):
    import oracle as O
    c = _ssd_case(ngf, m, h, n, seed=sum(m) + 1)
    with ngf.Plan(c.desc) as pl:
        D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
        g, q, dg = c.empty(), c.empty(), c.empty()
        Dg, Sg = ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g)
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, dg)
        torch.cuda.synchronize()
    Do, So = O.objective(c.L, c.Rh, c.Th, c.uh)
    assert abs(D - Do) <= G.TOL_OBJ * abs(Do) and abs(S - So) <= G.TOL_OBJ * max(abs(So), 1e-300)
    assert abs(Dg - Do) <= G.TOL_OBJ * abs(Do) and Sg == S  # the gradient call returns D and S too
    go, _, _ = O.gradient(c.L, c.Rh, c.Th, c.uh)
    assert G.rel(G.f64(g), go) < G.TOL_GRAD
    assert G.rel(G.f64(q), O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)) < G.TOL_HESS
    if c.M < 1e6:  # the oracle's diagonal enumerates every row
        assert G.rel(G.f64(dg), O.gn_diagonal(c.L, c.Rh, c.Th, c.uh)) < G.TOL_DIAG


def test_ssd_gauss_newton_level_matches_oracle(ngf):
    import oracle as O
    from paper_1804_10541_b300 import synth
    m, h, n = (24, 24, 24), (1.0, 1.0, 1.0), (13, 13, 13)
    R, T, _ = synth.blob_pair(m, seed=0, device="cuda")
    d = ngf.level_desc(m, h, n, 1.0, 0.1, 0.1, distance=ngf.NGF_DIST_SSD)
    nn = 3 * 13 ** 3
    u = torch.zeros(nn, device="cuda")
    rep = ngf.register_multilevel(d, ngf.options(1, gn_iters=3, pcg_iters=10), R, T, u)
    L = O.level(m, h, n, 1.0, distance=O.DIST_SSD)
    uo, ro, _ = O.gn_level(L, G.f64(R), G.f64(T), np.zeros(nn), O.gn_options(3, 10))
    assert rep.gn_done == ro.gn_done == 3 and rep.ls_trials == ro.ls_trials
    assert float(np.abs(G.f64(u) - uo).max()) < 0.01
    assert abs(rep.J - ro.J) <= 1e-5 * abs(ro.J)


def test_ssd_rejected_by_the_allocation_free_objective(ngf):
    c = _ssd_case(ngf, (20, 18, 16), (1.0, 1.0, 1.0), (11, 10, 9), seed=3)
    out = torch.zeros(2, device="cuda", dtype=torch.float64)
    with pytest.raises(ngf.NGFError) as e:
        ngf.ngf_objective_noalloc(c.desc, c.R, c.T, c.u, out)
    assert e.value.status == -1
    bad = ngf.level_desc((20, 18, 16), (1.0, 1.0, 1.0), (11, 10, 9), distance=7)
    with pytest.raises(ngf.NGFError) as e:
        ngf.Plan(bad)
    assert e.value.status == -1


def test_ssd_lbfgs_level_matches_oracle(ngf):
    """SSD with the L-BFGS method: same steps and trials as the oracle's
    L-BFGS on the SSD objective, u within 0.01 voxel."""
    import oracle as O
    from paper_1804_10541_b300 import synth
    m, h, n = (24, 24, 24), (1.0, 1.0, 1.0), (13, 13, 13)
    R, T, _ = synth.blob_pair(m, seed=1, device="cuda")
    d = ngf.level_desc(m, h, n, 1.0, 0.1, 0.1, distance=ngf.NGF_DIST_SSD)
    nn = 3 * 13 ** 3
    u = torch.zeros(nn, device="cuda")
    rep = ngf.register_multilevel(d, ngf.options(1, gn_iters=6, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=4), R, T, u)
    L = O.level(m, h, n, 1.0, distance=O.DIST_SSD)
    uo, ro, _, _ = O.lbfgs_level(L, G.f64(R), G.f64(T), np.zeros(nn), O.lbfgs_options(iters=6, memory=4))
    assert rep.gn_done == ro.gn_done == 6 and rep.ls_trials == ro.ls_trials
    assert float(np.abs(G.f64(u) - uo).max()) < 0.01
    assert abs(rep.J - ro.J) <= 1e-5 * abs(ro.J)
