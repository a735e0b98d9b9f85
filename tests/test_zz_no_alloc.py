"""The objective entry point that allocates no device memory.

Callers whose device memory is owned by a framework pool, that run in loops
where an allocation is not allowed, or that must not touch the host process's
allocator use ngf_objective_noalloc instead of a plan.  These tests call it
through the C ABI and check, on two calls in a row, that it returns the same
D and S as the plan-based ngf_objective within the objective tolerance of the
other parity tests, and that oversized problems are refused with a clear
error before anything is launched.  This file is collected last on purpose.
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


def _reference(ngf, c):
    with ngf.Plan(c.desc) as pl:
        return ngf.ngf_objective(pl.handle, c.R, c.T, c.u)


@pytest.mark.parametrize("which", ["blobs_32", "random_ragged", "lung_ct"])
def test_noalloc_objective_matches_plan_twice(ngf, which):
    if which == "random_ragged":
        c = G.random_case((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11), seed=9)
    else:
        c, _ = G.workload_case(which)
    D0, S0 = _reference(ngf, c)
    out = torch.full((2,), float("nan"), device="cuda", dtype=torch.float64)
    for _ in range(2):  # two calls in a row share the static scratch
        out.fill_(float("nan"))
        ngf.ngf_objective_noalloc(c.desc, c.R, c.T, c.u, out)
        torch.cuda.synchronize()
        D, S = out.tolist()
        assert np.isfinite(D) and np.isfinite(S)
        assert abs(D - D0) <= G.TOL_OBJ * abs(D0), (D, D0)
        assert abs(S - S0) <= G.TOL_OBJ * max(abs(S0), 1e-300), (S, S0)


def test_noalloc_objective_tracks_new_inputs(ngf):
    """A call after a call on another problem does not reuse stale tables."""
    a = G.random_case((40, 24, 12), (1.0, 1.0, 1.5), (21, 13, 7), seed=1)
    b = G.random_case((33, 17, 9), (1.0, 1.2, 2.0), (12, 9, 5), seed=2)
    out = torch.empty(2, device="cuda", dtype=torch.float64)
    for c in (a, b, a):
        ngf.ngf_objective_noalloc(c.desc, c.R, c.T, c.u, out)
        torch.cuda.synchronize()
        D0, S0 = _reference(ngf, c)
        assert abs(out[0].item() - D0) <= G.TOL_OBJ * abs(D0)
        assert abs(out[1].item() - S0) <= G.TOL_OBJ * max(abs(S0), 1e-300)


def test_noalloc_objective_rejects_oversized(ngf):
    desc = ngf.level_desc((5000, 4, 4), (1, 1, 1), (3, 3, 3))
    t = torch.zeros(16, device="cuda")
    out = torch.zeros(2, device="cuda", dtype=torch.float64)
    with pytest.raises(ngf.NGFError) as e:
        ngf.ngf_objective_noalloc(desc, t, t, t, out)
    assert e.value.status == -8 and "NGF_NOALLOC_MAX_AXIS" in str(e.value)


def test_noalloc_objective_rejects_wide_slices(ngf):
    """A 4096 x 4096 slice needs 128 x 256 image-pass blocks, above
    NGF_NOALLOC_MAX_BLOCKS; the call is refused before any launch."""
    desc = ngf.level_desc((4096, 4096, 1), (1, 1, 1), (3, 3, 2))
    t = torch.zeros(16, device="cuda")
    out = torch.zeros(2, device="cuda", dtype=torch.float64)
    with pytest.raises(ngf.NGFError) as e:
        ngf.ngf_objective_noalloc(desc, t, t, t, out)
    assert e.value.status == -8 and "NGF_NOALLOC_MAX_BLOCKS" in str(e.value)


def test_noalloc_objective_allocates_nothing(ngf):
    """After a first call on the device (which looks up the scratch array's
    address), a further call leaves the device's free memory unchanged."""
    c = G.random_case((70, 35, 21), (1.0, 1.0, 2.5), (36, 18, 11), seed=10)
    out = torch.zeros(2, device="cuda", dtype=torch.float64)
    ngf.ngf_objective_noalloc(c.desc, c.R, c.T, c.u, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ngf.ngf_objective_noalloc(c.desc, c.R, c.T, c.u, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    D0, _ = _reference(ngf, c)
    assert abs(out[0].item() - D0) <= G.TOL_OBJ * abs(D0)
