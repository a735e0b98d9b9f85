"""The learned initializer's network on the GPU (forward, gradients, Adam
step) against the FP64 oracle (oracle/cnn_oracle.py), through the C ABI.

The oracle is run twice: with every stored activation and propagated
gradient rounded to bf16 at the points where the kernels store bf16 (the
kernels' precision), and as the plain float64 definition.  Bars (relative
L2 per tensor): 1e-2 against the first (what remains is FP32 against FP64
accumulation ahead of each rounding, which moves an occasional value by
one bf16 step), 1e-1 against the second (about 15 bf16 roundings of
relative size <= 2^-8 along the longest path, amplified where a weight
gradient sums terms of both signs; measured up to 6e-2).
"""
import os
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))
import cnn_oracle as CO  # noqa: E402

SHIFT, SCALE, OUT = -500.0, 1.0 / 500.0, 4.0


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _flat(p):
    return np.concatenate([np.concatenate([p["W" + k].ravel(), p["b" + k].ravel()]) for k, _, _ in CO.NET_LAYERS])


def _unflat(v):
    out, off = {}, 0
    for k, ci, co in CO.NET_LAYERS:
        nw = 27 * ci * co
        out["W" + k] = v[off:off + nw].reshape(co, 3, 3, 3, ci)
        off += nw
        out["b" + k] = v[off:off + co]
        off += co
    return out


def _problem(s, B, seed):
    rng = np.random.default_rng(seed)
    p = CO.net_init(seed)
    for k, _, co in CO.NET_LAYERS:
        p["b" + k] = 0.05 * rng.standard_normal(co)
    p["b7"][3:] = 0.0
    # weights as the tensor cores read them (bf16 values), biases float32
    for k in p:
        p[k] = CO.to_bf16(p[k]) if k.startswith("W") else p[k].astype(np.float32).astype(np.float64)
    R = (rng.standard_normal((B, s, s, s)) * 300.0 - 500.0).astype(np.float32)
    T = (R + rng.standard_normal((B, s, s, s)) * 100.0).astype(np.float32)
    ut = (rng.standard_normal((B, 3, (s // 4 + 1) ** 3)) * 3.0).astype(np.float32)
    return p, R, T, ut


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("s,B", [(16, 2), (32, 1)])
def test_net_forward_and_gradients_match_oracle(ngf, s, B):
    p, R, T, ut = _problem(s, B, seed=s + B)
    d = ngf.net_desc(s, B, SHIFT, SCALE, OUT)
    Rd, Td, utd = (torch.from_numpy(a).cuda() for a in (R, T, ut))
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(_flat(p).astype(np.float32)))
        u = torch.empty(B * 3 * (s // 4 + 1) ** 3, device="cuda")
        ngf.ngf_net_forward(net.handle, Rd, Td, B, u)
        g = torch.empty(net.nparams, device="cuda")
        loss = ngf.ngf_net_grad(net.handle, Rd, Td, utd, B, g)
        assert ngf.ngf_conv3d_check() == 0
    u = u.double().cpu().numpy()
    gg = _unflat(g.double().cpu().numpy())
    R64, T64 = R.astype(np.float64), T.astype(np.float64)
    for rnd, bar in ((CO.to_bf16, 1e-2), (None, 1e-1)):
        a = CO.net_forward(p, R64, T64, SHIFT, SCALE, OUT, rnd=rnd)
        lo = CO.net_loss(a, ut, OUT)
        go = CO.net_backward(p, a, ut, OUT, rnd=rnd)
        assert _rel(u, a["u"].ravel()) < bar
        assert abs(loss - lo) / lo < bar
        for k in go:
            if k in ("W7", "b7"):
                assert _rel(gg[k][:3], go[k][:3]) < bar, k
                assert not np.any(gg[k][3:]), k  # unused output channels get no gradient
            else:
                assert _rel(gg[k], go[k]) < bar, (k, _rel(gg[k], go[k]))


def test_net_gradient_is_deterministic(ngf):
    p, R, T, ut = _problem(16, 2, seed=3)
    d = ngf.net_desc(16, 2, SHIFT, SCALE, OUT)
    Rd, Td, utd = (torch.from_numpy(a).cuda() for a in (R, T, ut))
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(_flat(p).astype(np.float32)))
        g1 = torch.empty(net.nparams, device="cuda")
        g2 = torch.empty(net.nparams, device="cuda")
        l1 = ngf.ngf_net_grad(net.handle, Rd, Td, utd, 2, g1)
        l2 = ngf.ngf_net_grad(net.handle, Rd, Td, utd, 2, g2)
    assert l1 == l2 and torch.equal(g1, g2)


def test_adam_step_matches_oracle(ngf):
    """One training step equals the oracle's Adam update applied to the
    kernel's own gradient at the same parameters (float32 update
    arithmetic: the step of Adam's first iteration is lr * g / (|g| + eps))."""
    p, R, T, ut = _problem(16, 2, seed=4)
    d = ngf.net_desc(16, 2, SHIFT, SCALE, OUT)
    Rd, Td, utd = (torch.from_numpy(a).cuda() for a in (R, T, ut))
    flat = _flat(p).astype(np.float32)
    lr = 1e-3
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(flat))
        g = torch.empty(net.nparams, device="cuda")
        l0 = ngf.ngf_net_grad(net.handle, Rd, Td, utd, 2, g)
        l1 = ngf.ngf_net_train_step(net.handle, Rd, Td, utd, 2, lr)
        out = torch.empty(net.nparams)
        ngf.ngf_net_get_params(net.handle, out)
    assert l0 == l1  # the step's forward pass is the gradient call's
    po = {"w": flat.astype(np.float64)}
    m = {"w": np.zeros_like(po["w"])}
    v = {"w": np.zeros_like(po["w"])}
    CO.adam_step(po, {"w": g.double().cpu().numpy()}, m, v, 1, lr)
    err = np.abs(out.double().numpy() - po["w"])
    assert np.all(err <= 1e-7 + 1e-6 * np.abs(po["w"])), float(err.max())
    assert np.abs(po["w"] - flat).max() > 0.9 * lr  # parameters with a gradient moved by about lr


def test_training_lowers_the_loss_on_a_fixed_batch(ngf):
    p, R, T, ut = _problem(16, 4, seed=5)
    d = ngf.net_desc(16, 4, SHIFT, SCALE, OUT)
    Rd, Td, utd = (torch.from_numpy(a).cuda() for a in (R, T, ut))
    with ngf.Net(d) as net:
        ngf.ngf_net_set_params(net.handle, torch.from_numpy(_flat(p).astype(np.float32)))
        losses = [ngf.ngf_net_train_step(net.handle, Rd, Td, utd, 4, 2e-3) for _ in range(60)]
    # random targets: the network fits part of them; the loss falls steadily
    assert losses[-1] < 0.75 * losses[0], (losses[0], losses[-1])
    assert np.mean(losses[-10:]) < np.mean(losses[:10])
