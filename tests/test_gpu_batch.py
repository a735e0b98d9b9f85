"""Batched form: many independent pairs of uneven size in one launch per stage.

With the same z-chunk length (ZC) on both sides, each pair's result from the
batched entry points must equal, bit for bit, what its own plan gives (same
kernels, same tile geometry, same reduction order); the batched registration
must take each pair's decisions exactly as register_multilevel does on that
pair alone.  The batched Hessian-vector
product and gradient are also compared with the FP64 oracle directly.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import gpu_util as G  # noqa: E402

ZC = 8  # common tile depth of the bitwise comparisons

# uneven sizes, ragged tiles, several z-chunks; the last pair has one voxel
# per cell in x (four-node span in the diagonal kernel)
PAIRS = [
    ((37, 19, 11), (1.0, 1.0, 1.0), (19, 10, 6)),
    ((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11)),
    ((32, 32, 32), (1.0, 1.0, 1.0), (17, 17, 17)),
    ((65, 33, 40), (0.8, 0.8, 1.0), (17, 9, 11)),
    ((40, 20, 10), (1.0, 1.0, 1.0), (41, 11, 6)),
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _cases():
    return [G.random_case(m, h, n, seed=11 + k) for k, (m, h, n) in enumerate(PAIRS)]


def test_batched_operators_equal_single_plans(ngf):
    cs = _cases()
    R, T, U, P = [c.R for c in cs], [c.T for c in cs], [c.u for c in cs], [c.p for c in cs]
    q, g, dg = [c.empty() for c in cs], [c.empty() for c in cs], [c.empty() for c in cs]
    with ngf.Batch([c.desc for c in cs], ZC) as b:
        ngf.ngf_batch_hessvec(b.handle, R, T, U, P, q)
        ngf.ngf_batch_gradient(b.handle, R, T, U, g)
        ngf.ngf_batch_diagonal(b.handle, R, T, U, dg)
        Db, Sb = ngf.ngf_batch_objective(b.handle, R, T, U)
        torch.cuda.synchronize()
    for k, c in enumerate(cs):
        with ngf.Plan(c.desc, zc=ZC) as pl:
            q1, g1, d1 = c.empty(), c.empty(), c.empty()
            ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q1)
            ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g1, want_scalars=False)
            ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d1)
            D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
            torch.cuda.synchronize()
        assert torch.equal(q[k], q1), k
        assert torch.equal(g[k], g1), k
        assert D == Db[k] and S == Sb[k], k
        assert torch.equal(dg[k], d1), k


def test_batched_operators_match_oracle(ngf):
    import oracle as O
    cs = _cases()[:3]
    q, g = [c.empty() for c in cs], [c.empty() for c in cs]
    with ngf.Batch([c.desc for c in cs]) as b:
        ngf.ngf_batch_hessvec(b.handle, [c.R for c in cs], [c.T for c in cs], [c.u for c in cs],
                              [c.p for c in cs], q)
        ngf.ngf_batch_gradient(b.handle, [c.R for c in cs], [c.T for c in cs], [c.u for c in cs], g)
        torch.cuda.synchronize()
    for k, c in enumerate(cs):
        assert G.rel(G.f64(q[k]), O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)) < G.TOL_HESS
        go, _, _ = O.gradient(c.L, c.Rh, c.Th, c.uh)
        assert G.rel(G.f64(g[k]), go) < G.TOL_GRAD


def test_autotune_picks_a_candidate_and_keeps_parity(ngf):
    import oracle as O
    cs = _cases()[:4]
    q = [c.empty() for c in cs]
    with ngf.Batch([c.desc for c in cs]) as b:
        zc, ms = ngf.ngf_batch_autotune(b.handle, [c.R for c in cs], [c.T for c in cs], [c.u for c in cs],
                                        [c.p for c in cs], q)
        assert ngf.ngf_batch_zc(b.handle) == min(zc, cs[0].m[2]) and ms > 0
        deepest = max(c.m[2] for c in cs)
        assert zc in [min(z, deepest) for z in (8, 16, 24, 32, 48, 64)]
        ngf.ngf_batch_hessvec(b.handle, [c.R for c in cs], [c.T for c in cs], [c.u for c in cs],
                              [c.p for c in cs], q)
        torch.cuda.synchronize()
    for k, c in enumerate(cs):
        assert G.rel(G.f64(q[k]), O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)) < G.TOL_HESS


def _blob_batch(sizes):
    from paper_1804_10541_b300 import ngf as m, synth
    out = []
    for k, N in enumerate(sizes):
        R, T, _ = synth.blob_pair((N, N, N), seed=1000 + 4 * k, device="cuda")
        out.append((R, T, m.level_desc((N, N, N), (1.0, 1.0, 1.0), (N // 2 + 1,) * 3, 1.0, 0.1, 0.1)))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("diag_every", [0, 3])
def test_register_batch_equals_per_pair_registration(ngf, use_graph, diag_every):
    """Each pair of a batched registration takes exactly its own
    registration's decisions, with the Jacobi diagonal once per level and
    refreshed every third Gauss-Newton step."""
    pairs = _blob_batch([24, 33, 40, 29])
    opts = ngf.options(2, gn_iters=4, pcg_iters=8, use_graph=use_graph, zc=ZC, diag_every=diag_every)
    ub = [torch.zeros(3 * d.n[0] * d.n[1] * d.n[2], device="cuda") for _, _, d in pairs]
    # graphs need a stream other than the legacy default stream
    stream = torch.cuda.Stream() if use_graph else None
    torch.cuda.synchronize()
    reps = ngf.register_batch([d for _, _, d in pairs], opts, [R for R, _, _ in pairs], [T for _, T, _ in pairs], ub,
                              stream=stream)
    for k, (R, T, d) in enumerate(pairs):
        u1 = torch.zeros_like(ub[k])
        r1 = ngf.register_multilevel(d, opts, R, T, u1, stream)
        assert torch.equal(u1, ub[k]), k
        assert (r1.J, r1.gn_done, r1.ls_trials, r1.pcg_total, r1.ls_fail) == \
               (reps[k].J, reps[k].gn_done, reps[k].ls_trials, reps[k].pcg_total, reps[k].ls_fail), k
        assert reps[k].hessvec_voxels == r1.hessvec_voxels


def test_register_batch_rejects_bad_arguments(ngf):
    pairs = _blob_batch([20, 24])
    descs = [d for _, _, d in pairs]
    ub = [torch.zeros(3 * d.n[0] * d.n[1] * d.n[2], device="cuda") for d in descs]
    R, T = [p[0] for p in pairs], [p[1] for p in pairs]
    init = torch.zeros(16, device="cuda")
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_batch(descs, ngf.options(2, u_init=init), R, T, ub)
    assert e.value.status == -1
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_batch(descs, ngf.options(2), [R[0], np.zeros(8, np.float32)], T, ub)
    assert e.value.status == -1 and "device" in str(e.value)
    bad = R[1].clone()
    bad[5] = float("nan")
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_batch(descs, ngf.options(2), [R[0], bad], T, ub)
    assert e.value.status == -4 and "pair 1" in str(e.value)


def test_batch_larger_than_one_parameter_table(ngf):
    """More pairs than one launch's parameter table holds (two launches per
    image stage): every pair still equals its own plan."""
    g = torch.Generator().manual_seed(5)
    cs = []
    for k in range(130):
        m, n = (4 + k % 5, 3 + k % 3, 3 + k % 2), (3, 2, 2)
        M, N = m[0] * m[1] * m[2], 12
        c = G.Case(m, (1.0, 1.0, 1.0), n, 0.5, 0.2, 0.2, torch.rand(M, generator=g), torch.rand(M, generator=g),
                   0.2 * torch.randn(3 * N, generator=g), torch.randn(3 * N, generator=g))
        cs.append(c)
    q = [c.empty() for c in cs]
    with ngf.Batch([c.desc for c in cs], ZC) as b:
        ngf.ngf_batch_hessvec(b.handle, [c.R for c in cs], [c.T for c in cs], [c.u for c in cs],
                              [c.p for c in cs], q)
        torch.cuda.synchronize()
    for k in (0, 64, 111, 112, 129):
        c = cs[k]
        with ngf.Plan(c.desc, zc=ZC) as pl:
            q1 = c.empty()
            ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q1)
            torch.cuda.synchronize()
        assert torch.equal(q[k], q1), k


def test_mixed_ngf_ssd_batch_equals_single_plans(ngf):
    """Pairs with the SSD distance share the batch's launches with NGF pairs
    (the SSD diagonal on its halo-free tiles); every pair equals its own plan,
    and the batched registration each pair's own."""
    cs = _cases()[:4]
    for k in (1, 3):
        cs[k].desc = ngf.level_desc(cs[k].m, cs[k].h, cs[k].n, 0.7, 0.15, 0.25, distance=ngf.NGF_DIST_SSD)
    R, T, U, P = [c.R for c in cs], [c.T for c in cs], [c.u for c in cs], [c.p for c in cs]
    q, g, dg = [c.empty() for c in cs], [c.empty() for c in cs], [c.empty() for c in cs]
    with ngf.Batch([c.desc for c in cs], ZC) as b:
        ngf.ngf_batch_hessvec(b.handle, R, T, U, P, q)
        ngf.ngf_batch_gradient(b.handle, R, T, U, g)
        ngf.ngf_batch_diagonal(b.handle, R, T, U, dg)
        Db, Sb = ngf.ngf_batch_objective(b.handle, R, T, U)
        torch.cuda.synchronize()
    for k, c in enumerate(cs):
        with ngf.Plan(c.desc, zc=ZC) as pl:
            q1, g1, d1 = c.empty(), c.empty(), c.empty()
            ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q1)
            ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g1, want_scalars=False)
            ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d1)
            D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
            torch.cuda.synchronize()
        assert torch.equal(q[k], q1) and torch.equal(g[k], g1) and torch.equal(dg[k], d1), k
        assert D == Db[k] and S == Sb[k], k
    pairs = _blob_batch([24, 29])
    descs = [pairs[0][2], ngf.level_desc((29, 29, 29), (1.0, 1.0, 1.0), (15, 15, 15), 1.0, 0.1, 0.1,
                                         distance=ngf.NGF_DIST_SSD)]
    opts = ngf.options(2, gn_iters=3, pcg_iters=6, zc=ZC)
    ub = [torch.zeros(3 * d.n[0] * d.n[1] * d.n[2], device="cuda") for d in descs]
    reps = ngf.register_batch(descs, opts, [p[0] for p in pairs], [p[1] for p in pairs], ub)
    for k, d in enumerate(descs):
        u1 = torch.zeros_like(ub[k])
        r1 = ngf.register_multilevel(d, opts, pairs[k][0], pairs[k][1], u1)
        assert torch.equal(u1, ub[k]) and r1.J == reps[k].J, k
