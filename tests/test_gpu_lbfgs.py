"""L-BFGS (Sec. 2.3.2) on the GPU against the FP64 oracle.

The initial Hessian H0 = alpha grad^2 S + gamma I is inverted in the DCT-II
eigenbasis of the clamped Laplacian by `ngf_h0_solve`; `register_multilevel`
with method NGF_METHOD_LBFGS runs the two-loop recursion with Armijo
backtracking.  Both are compared with the oracle's own (pinned) L-BFGS.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import gpu_util as G  # noqa: E402


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("m,h,n,gamma", [((6, 5, 4), (1.0, 1.2, 2.0), (4, 3, 3), 0.37),
                                         ((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11), 3.0),
                                         ((256, 256, 120), (1.0, 1.0, 2.5), (129, 129, 61), 50.0)])
def test_h0_solve_matches_oracle(ngf, m, h, n, gamma):
    import oracle as O
    c = G.random_case(m, h, n, alpha=0.7, seed=7)
    r = c.empty()
    with ngf.Plan(c.desc) as pl:
        ngf.ngf_h0_solve(pl.handle, gamma, c.p, r)
        torch.cuda.synchronize()
    assert G.rel(G.f64(r), O.h0_solve(c.L, gamma, c.ph)) < G.TOL_HESS


def _blob_level(N):
    from paper_1804_10541_b300 import synth
    R, T, _ = synth.blob_pair((N, N, N), seed=0, device="cuda")
    return R, T, (N, N, N), (1.0, 1.0, 1.0), (N // 2 + 1,) * 3


@pytest.mark.parametrize("N,iters,memory", [(16, 6, 3), (24, 8, 5)])
def test_lbfgs_level_matches_oracle(ngf, N, iters, memory):
    """One level: same accepted steps and line-search trials as the oracle, final
    u within 0.01 voxel and final J within 1e-6."""
    import oracle as O
    R, T, m, h, n = _blob_level(N)
    nn = 3 * n[0] * n[1] * n[2]
    u = torch.zeros(nn, device="cuda")
    opts = ngf.options(1, gn_iters=iters, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=memory)
    rep = ngf.register_multilevel(ngf.level_desc(m, h, n, 1.0, 0.1, 0.1), opts, R, T, u)
    L = O.level(m, h, n, 1.0, 0.1, 0.1)
    uo, ro, trace, gamma = O.lbfgs_level(L, G.f64(R), G.f64(T), np.zeros(nn),
                                         O.lbfgs_options(iters=iters, memory=memory))
    assert rep.gn_done == ro.gn_done == iters and rep.ls_trials == ro.ls_trials
    assert rep.pcg_total == 0 and rep.status == 0
    assert float(np.abs(G.f64(u) - uo).max()) < 0.01 * min(h)
    assert abs(rep.J - ro.J) <= 1e-6 * abs(ro.J)


def test_lbfgs_multilevel_decreases_and_rejects_bad_memory(ngf):
    from paper_1804_10541_b300 import synth
    R, T, _, w = synth.make("blobs_32", device="cuda")
    d = ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    nn = 3 * w["n"][0] * w["n"][1] * w["n"][2]
    u = torch.zeros(nn, device="cuda")
    u0 = torch.zeros(nn, device="cuda")
    with ngf.Plan(d) as pl:
        D0, S0 = ngf.ngf_objective(pl.handle, R, T, u0)
    rep = ngf.register_multilevel(d, ngf.options(2, gn_iters=15, method=ngf.NGF_METHOD_LBFGS), R, T, u)
    assert rep.status == 0 and rep.gn_done == 30 and rep.J < 0.6 * (D0 + w["alpha"] * S0)
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_multilevel(d, ngf.options(2, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=0), R, T, u)
    assert e.value.status == -1
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_batch([d], ngf.options(2, method=ngf.NGF_METHOD_LBFGS), [R], [T], [u])
    assert e.value.status == -1
