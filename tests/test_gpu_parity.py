"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-by-element comparisons on seeded inputs: tiny odd grids where every
voxel is a boundary voxel, a full-resolution deformation grid, non-integer
voxels-per-cell ratios, several tiles with ragged tails, the 32^3 blob
workload, and the full-size 256x256x120 lung-CT workload in the launch
configuration the benchmark times.  The 512x512x900 workload is checked by
properties that hold at any size.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import gpu_util as G  # noqa: E402

CASES = [
    ((5, 4, 3), (1.0, 1.0, 1.0), (3, 3, 2)),       # every voxel on the boundary
    ((6, 5, 4), (1.0, 0.8, 2.5), (4, 3, 3)),       # anisotropic, non-integer ratio
    ((4, 3, 3), (0.7, 1.3, 1.1), (5, 4, 4)),       # deformation grid at full resolution
    ((37, 19, 11), (1.0, 1.0, 1.0), (19, 10, 6)),  # 2 x 2 tiles, ragged
    ((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11)), # 3 x 3 tiles, ragged, z-chunks
    ((40, 20, 10), (1.0, 1.0, 1.0), (41, 21, 11)), # ratio 1 on every axis
    ((65, 33, 40), (0.8, 0.8, 1.0), (17, 9, 11)),  # ratio 4, non-integer in z
    ((30, 20, 60), (1.0, 1.0, 1.0), (4, 3, 2)),    # coarse grid: every z-chunk covers both node planes
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def fp32_sensitivity(c, seed=0):
    """Relative change of the oracle's own Hessian-vector product and
    diagonal when u is perturbed by half a float32 unit in the last place
    (relative 2^-24 per component, random signs): the conditioning of these
    operators at the float32 precision of their input.  With HU-valued
    images and displacements of many voxels this alone reaches ~1e-5
    (short differences of warped values near 1000 HU cancel, and warped
    samples cross knots of the trilinear template, where its derivative
    jumps), so no float32 evaluation can be held to less."""
    import oracle as O
    rng = np.random.default_rng(seed)
    up = c.uh * (1.0 + 2.0 ** -24 * rng.choice([-1.0, 1.0], size=c.uh.shape))
    kh = G.rel(O.hessvec(c.L, c.Rh, c.Th, up, c.ph), O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph))
    kd = G.rel(O.gn_diagonal(c.L, c.Rh, c.Th, up), O.gn_diagonal(c.L, c.Rh, c.Th, c.uh))
    return kh, kd


def _all_ops(ngf, c):
    import oracle as O
    out = {}
    with ngf.Plan(c.desc) as pl:
        D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
        g = c.empty()
        Dg, Sg = ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g)
        q = c.empty()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        dg = c.empty()
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, dg)
        cq = c.empty()
        Sp = ngf.curvature_apply(pl.handle, c.p, cq)
        torch.cuda.synchronize()
    Do, So = O.objective(c.L, c.Rh, c.Th, c.uh)
    go, _, _ = O.gradient(c.L, c.Rh, c.Th, c.uh)
    qo = O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)
    dgo = O.gn_diagonal(c.L, c.Rh, c.Th, c.uh)
    cqo, Spo = O.curvature_apply(c.L, c.ph)
    out["D"] = abs(D - Do) / abs(Do)
    out["Dg"] = abs(Dg - Do) / abs(Do)
    out["S"] = abs(S - So) / max(abs(So), 1e-300)
    out["grad"] = G.rel(G.f64(g), go)
    out["hess"] = G.rel(G.f64(q), qo)
    out["diag"] = G.rel(G.f64(dg), dgo)
    out["curv"] = G.rel(G.f64(cq), cqo)
    out["Sp"] = abs(Sp - Spo) / max(abs(Spo), 1e-300)
    return out


def _assert_ok(r, tol_hess=G.TOL_HESS, tol_diag=G.TOL_DIAG):
    assert r["D"] < G.TOL_OBJ and r["Dg"] < G.TOL_OBJ and r["S"] < G.TOL_OBJ, r
    assert r["grad"] < G.TOL_GRAD, r
    assert r["hess"] < tol_hess, r
    assert r["diag"] < tol_diag, r
    assert r["curv"] < G.TOL_CURV and r["Sp"] < G.TOL_OBJ, r


@pytest.mark.parametrize("m,h,n", CASES)
def test_operators_match_oracle_small(ngf, m, h, n):
    c = G.random_case(m, h, n, seed=sum(m))
    _assert_ok(_all_ops(ngf, c))


def test_operators_match_oracle_blobs32(ngf):
    c, _ = G.workload_case("blobs_32")
    _assert_ok(_all_ops(ngf, c))


def test_operators_match_oracle_lung_full_size(ngf):
    """256x256x120 lung-CT workload, the benchmark's configuration."""
    import oracle as O
    c, w = G.workload_case("lung_ct", amp_vox=0.7)
    with ngf.Plan(c.desc) as pl:
        D, S = ngf.ngf_objective(pl.handle, c.R, c.T, c.u)
        g = c.empty()
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g, want_scalars=False)
        q = c.empty()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q)
        torch.cuda.synchronize()
    Do, So = O.objective(c.L, c.Rh, c.Th, c.uh)
    assert abs(D - Do) / abs(Do) < G.TOL_OBJ and abs(S - So) / So < G.TOL_OBJ
    go, _, _ = O.gradient(c.L, c.Rh, c.Th, c.uh)
    assert G.rel(G.f64(g), go) < G.TOL_GRAD
    qo = O.hessvec(c.L, c.Rh, c.Th, c.uh, c.ph)
    assert G.rel(G.f64(q), qo) < G.TOL_HESS


def test_hessvec_is_deterministic(ngf):
    c, _ = G.workload_case("blobs_32")
    with ngf.Plan(c.desc) as pl:
        q1, q2 = c.empty(), c.empty()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q1)
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q2)
        g1, g2 = c.empty(), c.empty()
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g1)
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g2)
        # the diagonal sums its rows in a fixed order too
        d1, d2 = c.empty(), c.empty()
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d1)
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d2)
        torch.cuda.synchronize()
    assert torch.equal(q1, q2) and torch.equal(g1, g2) and torch.equal(d1, d2)
    # one voxel per cell (four-node span of the diagonal kernel)
    c = G.random_case((40, 20, 10), (1.0, 1.0, 1.0), (41, 21, 11), seed=4)
    with ngf.Plan(c.desc) as pl:
        d1, d2 = c.empty(), c.empty()
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d1)
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, d2)
        torch.cuda.synchronize()
    assert torch.equal(d1, d2)


def test_identity_and_identical_images(ngf):
    """T = R, u = 0, tau = rho: D = 0 and grad D = 0 (r = 1 everywhere)."""
    m, h, n = (40, 24, 12), (1.0, 1.0, 1.5), (21, 13, 7)
    c = G.random_case(m, h, n, alpha=0.0, tau=0.2, rho=0.2, seed=3)
    c.T = c.R.clone()
    c.u.zero_()
    with ngf.Plan(c.desc) as pl:
        g = c.empty()
        D, S = ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g)
    assert abs(D) < 1e-9 * c.M and S == 0.0
    assert float(g.abs().max()) < 1e-6


def test_thorax_full_size_properties(ngf):
    """512x512x900 workload: symmetric PSD Hessian and a finite gradient."""
    c, w = G.workload_case("thorax_abd", amp_vox=0.5)
    gq = torch.Generator(device="cpu").manual_seed(77)
    p2 = torch.randn(3 * c.N, generator=gq).to("cuda")
    with ngf.Plan(c.desc) as pl:
        q1, q2 = c.empty(), c.empty()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, q1)
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, p2, q2)
        g = c.empty()
        D, S = ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g)
        torch.cuda.synchronize()
    a = float(torch.dot(p2.double(), q1.double()))
    b = float(torch.dot(c.p.double(), q2.double()))
    assert abs(a - b) <= 1e-4 * (abs(a) + abs(b))
    assert float(torch.dot(c.p.double(), q1.double())) > 0
    assert torch.isfinite(g).all() and np.isfinite(D) and D > 0


def test_pcg_matches_oracle_and_graph(ngf):
    """PCG iterates equal the oracle's.  pcg_solve, with direct launches and
    as a captured graph, reproduces repeated pcg_step calls (five launches
    per iteration: Laplacian, image pass, node combine, update, direction)
    bitwise in every state vector and float64 scalar."""
    import oracle as O
    c, _ = G.workload_case("blobs_32")
    iters = 8
    res = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), ngf.Plan(c.desc, stream) as pl:
        g = c.empty()
        ngf.ngf_gradient(pl.handle, c.R, c.T, c.u, g, want_scalars=False)
        dg = c.empty()
        ngf.ngf_gn_diagonal(pl.handle, c.R, c.T, c.u, dg)
        rhs = (-g).contiguous()
        for arm in ("steps", "direct", "graph"):
            vec = [c.empty() for _ in range(5)]
            sc = torch.zeros(8, device="cuda", dtype=torch.float64)
            st = ngf.pcg_state(*vec, dg, sc)
            ngf.pcg_init(pl.handle, st, rhs)
            if arm == "steps":
                for _ in range(iters):
                    ngf.pcg_step(pl.handle, st, c.R, c.T, c.u)
            else:
                ngf.pcg_solve(pl.handle, st, c.R, c.T, c.u, iters, use_graph=(arm == "graph"))
            info = ngf.pcg_read(pl.handle, st)
            stream.synchronize()
            res[arm] = ([v.clone() for v in vec[:4]], sc.clone(), info)
    for arm in ("direct", "graph"):
        for a, b in zip(res[arm][0], res["steps"][0]):
            assert torch.equal(a, b), arm
        assert torch.equal(res[arm][1], res["steps"][1]), arm
    x, info = res["graph"][0][0], res["graph"][2]
    assert info.iters_done == iters and info.status == 0
    xo, _ = O.pcg(c.L, c.Rh, c.Th, c.uh, G.f64(rhs), G.f64(dg), iters)
    assert G.rel(G.f64(x), xo) < G.TOL_PCG


def _registration_pair(ngf, gn_iters, diag_every=0):
    import oracle as O
    from paper_1804_10541_b300 import synth
    R, T, _, w = synth.make("blobs_32", device="cuda")
    desc = ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    N = int(np.prod(w["n"]))
    u = torch.empty(3 * N, device="cuda")
    opts = ngf.options(levels=w["levels"], gn_iters=gn_iters, pcg_iters=20, diag_every=diag_every)
    rep = ngf.register_multilevel(desc, opts, R, T, u, torch.cuda.Stream())
    L = O.level(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    oo = O.gn_options(gn_iters=gn_iters, pcg_iters=20, diag_every=diag_every)
    uo, ro = O.register_multilevel(L, w["levels"], oo, G.f64(R), G.f64(T))
    du = float(np.max(np.abs(G.f64(u) - uo))) / min(w["h"])
    dJ = abs(rep.J - ro.J) / ro.J
    msg = f"max |u - u_oracle| = {du:.3e} voxel, rel J diff = {dJ:.3e}, J = {rep.J} vs {ro.J}"
    return rep, ro, du, dJ, msg


@pytest.mark.parametrize("diag_every", [0, 1])
def test_register_multilevel_matches_oracle_blobs32(ngf, diag_every):
    """Config 0 (2 levels, 20 PCG iterations per step), with the Jacobi
    diagonal once per level (the default) and at every step.  With 3
    Gauss-Newton steps per level both sides take the same step lengths and
    the final u agrees within 0.01 voxel.  With the full 10 steps per level
    an Armijo decision near its threshold can flip between the float32 and
    float64 PCG solutions (a step of 1/4 instead of 1/8), after which u
    differs by a fraction of a voxel while the final objective agrees
    within 0.1%."""
    rep, ro, du, dJ, msg = _registration_pair(ngf, 3, diag_every)
    assert rep.status == 0 and ro.status == 0, msg
    assert rep.gn_done == ro.gn_done and rep.pcg_total == ro.pcg_total, msg
    assert du < 0.01 and dJ < 1e-5, msg
    rep, ro, du, dJ, msg = _registration_pair(ngf, 10, diag_every)
    assert rep.status == 0 and ro.status == 0, msg
    assert rep.gn_done == ro.gn_done and rep.pcg_total == ro.pcg_total, msg
    assert dJ < 1e-3, msg


def test_register_multilevel_host_pointers_equal_device(ngf):
    from paper_1804_10541_b300 import synth
    R, T, _, w = synth.make("blobs_32", device="cuda")
    desc = ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    N = int(np.prod(w["n"]))
    opts = ngf.options(levels=2, gn_iters=3, pcg_iters=5)
    ud = torch.empty(3 * N, device="cuda")
    ngf.register_multilevel(desc, opts, R, T, ud)
    Rh, Th = R.cpu().numpy(), T.cpu().numpy()
    uh = np.empty(3 * N, dtype=np.float32)
    rep = ngf.register_multilevel(desc, opts, Rh, Th, uh)
    assert rep.gn_done > 0
    # every operator sums in a fixed order (no atomics), so the host-pointer
    # call reproduces the device-pointer call bitwise
    assert np.array_equal(uh, ud.cpu().numpy())


def test_nonfinite_input_is_rejected(ngf):
    from paper_1804_10541_b300 import synth
    R, T, _, w = synth.make("blobs_32", device="cuda")
    R[123] = float("nan")
    desc = ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    u = torch.empty(3 * int(np.prod(w["n"])), device="cuda")
    with pytest.raises(ngf.NGFError) as e:
        ngf.register_multilevel(desc, ngf.options(levels=2, gn_iters=1, pcg_iters=1), R, T, u)
    assert e.value.status == -4


def test_host_pointer_rejected_by_plan_ops(ngf):
    c = G.random_case((8, 8, 8), (1, 1, 1), (5, 5, 5))
    with ngf.Plan(c.desc) as pl:
        with pytest.raises(ngf.NGFError) as e:
            ngf.gn_hessvec(pl.handle, c.R.cpu(), c.T, c.u, c.p, c.empty())
        assert e.value.status == -1 and "device" in str(e.value)


def test_launch_counter_counts_kernels(ngf):
    c = G.random_case((8, 8, 8), (1, 1, 1), (5, 5, 5))
    with ngf.Plan(c.desc) as pl:
        before = ngf.ngf_launch_count()
        ngf.gn_hessvec(pl.handle, c.R, c.T, c.u, c.p, c.empty())
        assert ngf.ngf_launch_count() - before == 3


def _random_shapes(count=12, seed=2024):
    """Seeded random grids: 1..80 cells per axis, every voxels-per-cell ratio
    from 1 (nodes = cells + 1) to about 8, anisotropic spacing."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = tuple(int(v) for v in rng.integers(1, 81, size=3))
        n = tuple(max(2, min(mk + 1, mk // int(rng.integers(1, 9)) + 1)) for mk in m)
        h = tuple(float(v) for v in rng.uniform(0.5, 2.5, size=3))
        out.append((m, h, n))
    return out


@pytest.mark.parametrize("m,h,n", _random_shapes())
def test_operators_match_oracle_random_shapes(ngf, m, h, n):
    c = G.random_case(m, h, n, seed=sum(m) + 7)
    _assert_ok(_all_ops(ngf, c))


# Large smooth displacements at the anisotropy and grid ratio of the two CT
# workloads: crops of the thorax-abdomen phantom (0.8 x 0.8 x 1.0 mm, four
# voxels per cell in x and y and a non-integer ratio in z, like 512 x 512 x 900
# with 129 x 129 x 225 nodes) and of the lung phantom (1 x 1 x 2.5 mm, two
# voxels per cell), warped by several voxels so that many samples leave the
# domain (template and its derivative zero there) and warps cross many cells.
LARGE_U_CASES = [
    ("thorax", (96, 80, 70), (0.8, 0.8, 1.0), (25, 21, 18), 6.0),
    ("thorax", (64, 48, 45), (0.8, 0.8, 1.0), (17, 13, 12), 9.0),
    ("lung", (72, 64, 30), (1.0, 1.0, 2.5), (37, 33, 16), 12.0),
]


@pytest.mark.parametrize("kind,m,h,n,max_mm", LARGE_U_CASES)
def test_operators_match_oracle_large_displacement(ngf, kind, m, h, n, max_mm):
    from paper_1804_10541_b300 import synth
    if kind == "thorax":
        R, T, _ = synth.thorax_pair(m, h, seed=20, device="cuda")
        alpha, tau = 10.0, 5.0
    else:
        R, T, _ = synth.lung_pair(m, h, seed=10, device="cuda")
        alpha, tau = 1.0, 10.0
    hy = [m[a] * h[a] / (n[a] - 1) for a in range(3)]
    u = synth.smooth_nodal_field(n, hy, seed=sum(m), max_disp=max_mm)
    g = torch.Generator().manual_seed(sum(n))
    p = torch.randn(3 * int(np.prod(n)), generator=g)
    c = G.Case(m, h, n, alpha, tau, tau, R, T, u, p)
    # the warp leaves the domain on a good part of the boundary
    assert max_mm / min(h) >= 5.0
    r = _all_ops(ngf, c)
    # objective and gradient at the stated bars; the Hessian-vector product
    # and the diagonal at that bar or twice the oracle's own change under a
    # float32-level perturbation of u, whichever is larger
    kh, kd = fp32_sensitivity(c)
    r["kappa_hess"], r["kappa_diag"] = kh, kd
    _assert_ok(r, tol_hess=max(G.TOL_HESS, 2.0 * kh), tol_diag=max(G.TOL_DIAG, 2.0 * kd))


def test_register_multilevel_stops_at_target_objective(ngf):
    """j_target ends the finest level at the first step whose objective is
    at or below it; gn_iters_finest caps that level's steps."""
    from paper_1804_10541_b300 import synth
    R, T, _, w = synth.make("blobs_32", device="cuda")
    desc = ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])
    u = torch.empty(3 * int(np.prod(w["n"])), device="cuda")
    full = ngf.register_multilevel(desc, ngf.options(levels=2, gn_iters=10, pcg_iters=20), R, T, u)
    target = full.J * 1.01
    part = ngf.register_multilevel(desc, ngf.options(levels=2, gn_iters=10, pcg_iters=20, j_target=target), R, T, u)
    assert part.J <= target and part.gn_done < full.gn_done
    capped = ngf.register_multilevel(desc, ngf.options(levels=2, gn_iters=10, pcg_iters=20, gn_iters_finest=2),
                                     R, T, u)
    assert capped.gn_done == 10 + 2
    with pytest.raises(ngf.NGFError):
        ngf.register_multilevel(desc, ngf.options(levels=2, j_target=-1.0), R, T, u)
