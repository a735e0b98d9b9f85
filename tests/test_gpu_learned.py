"""The learned initializer end to end on a small scale (64^3 lung-CT-like
pairs, 3 levels, 192 training pairs): targets from the plain method's own registrations, GPU
training, and what the trained network gains over the plain method at equal
final objective on held-out pairs.

Gains checked: the network's prediction on held-out pairs is closer to the
plain method's solution than the zero start it replaces, and Gauss-Newton
refined from it reaches the plain method's final J within 0.1% on most
held-out pairs with fewer Gauss-Newton steps in total.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1804_10541_b300 import learned, ngf
    assert torch.cuda.is_available()
    return ngf, learned


def test_learned_initializer_gains_at_equal_objective(mods):
    ngf, L = mods
    s = 64
    w = L.workload(s)
    ntr = 192
    Rtr, Ttr = L.make_pairs(s, 0, ntr, "cuda")
    Rte, Tte = L.make_pairs(s, 1000, 8, "cuda")
    U0, _ = L.register_all(torch.cat([Rtr, Rte]), torch.cat([Ttr, Tte]), w)
    U1 = L.level1_targets(U0, w["n"][0])
    U1tr, U1te = U1[:ntr].contiguous(), U1[ntr:].contiguous()
    d = ngf.net_desc(s, 8, L.IN_SHIFT, L.IN_SCALE, L.OUT_SCALE)
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(L.init_params(7)))
        losses = L.train(net, Rtr, Ttr, U1tr, epochs=40, batch=8, lr0=2e-3)
        assert ngf.ngf_conv3d_check() == 0
        pred = L.predict(net, Rte, Tte, 8)
        rows = L.compare(net, Rte, Tte, w, k1=3, finest_cap=30)
    assert losses[-1] < 0.5 * losses[0], losses
    err_net = float(((pred - U1te) ** 2).mean())
    err_zero = float((U1te ** 2).mean())
    assert err_net < 0.75 * err_zero, (err_net, err_zero)
    reached = [r for r in rows if r["learned_reached"]]
    assert len(reached) >= 6, rows
    assert all(r["plain_reached"] for r in rows), rows
    assert np.mean([r["learned_gn"] for r in reached]) < np.mean([r["plain_gn"] for r in reached]), rows
