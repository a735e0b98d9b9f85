"""Pins of the convolution oracle against things fixed outside it: a library
correlation, brute force on a tiny input, and kernels with known effect."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))
import cnn_oracle as CO  # noqa: E402


def test_centre_tap_identity_is_the_input():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 5, 6, 16))
    w = np.zeros((16, 3, 3, 3, 16))
    w[np.arange(16), 1, 1, 1, np.arange(16)] = 1.0
    assert np.array_equal(CO.conv3d(x, w), x)


def test_single_tap_shifts_with_zero_fill():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 5, 4, 3, 2))
    w = np.zeros((2, 3, 3, 3, 2))
    w[0, 2, 1, 0, 1] = 1.0  # y[..., 0] = x[z+1, y, x-1, channel 1]
    y = CO.conv3d(x, w)
    exp = np.zeros((1, 5, 4, 3))
    exp[:, :-1, :, 1:] = x[:, 1:, :, :-1, 1]
    assert np.array_equal(y[..., 0], exp)
    assert not y[..., 1].any()


def test_matches_scipy_correlate_per_channel_pair():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 6, 7, 5, 3))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    y = CO.conv3d(x, w)
    for o in range(2):
        ref = sum(nd.correlate(x[0, ..., c], w[o, ..., c], mode="constant", cval=0.0) for c in range(3))
        assert np.allclose(y[0, ..., o], ref, rtol=1e-12, atol=1e-12)


def test_brute_force_tiny_with_bias_and_relu():
    rng = np.random.default_rng(3)
    B, D, H, W, Ci, Co = 2, 3, 2, 3, 2, 3
    x = rng.standard_normal((B, D, H, W, Ci))
    w = rng.standard_normal((Co, 3, 3, 3, Ci))
    b = rng.standard_normal(Co)
    y = CO.conv3d(x, w, b, relu=True)
    for n in range(B):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    for o in range(Co):
                        s = b[o]
                        for kz in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                        s += w[o, kz, ky, kx] @ x[n, zz, y2, x2]
                        assert abs(y[n, z, yy, xx, o] - max(s, 0.0)) < 1e-12


def test_abs_scale_bounds_the_result():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 4, 4, 4, 2))
    w = rng.standard_normal((2, 3, 3, 3, 2))
    assert np.all(np.abs(CO.conv3d(x, w)) <= CO.conv3d_abs(x, w) + 1e-12)


# ---------------------------------------------------------------- backward


def _inner(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


def test_dgrad_and_wgrad_are_adjoints_of_the_forward():
    """<conv(x, w), dy> = <x, dgrad(dy, w)> = <w, wgrad(dy, x)>: the
    convolution is bilinear, so its two gradients are the transposes of the
    forward in x and in w."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 4, 5, 3, 3))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    dy = rng.standard_normal((2, 4, 5, 3, 4))
    f = _inner(CO.conv3d(x, w), dy)
    assert abs(_inner(x, CO.conv3d_dgrad(dy, w)) - f) <= 1e-12 * abs(f)
    assert abs(_inner(w, CO.conv3d_wgrad(dy, x)) - f) <= 1e-12 * abs(f)
    assert np.allclose(CO.bias_grad(dy), dy.sum(axis=(0, 1, 2, 3)))


def test_wgrad_brute_force_tiny():
    rng = np.random.default_rng(6)
    B, D, H, W, Ci, Co = 1, 3, 2, 4, 2, 3
    x = rng.standard_normal((B, D, H, W, Ci))
    dy = rng.standard_normal((B, D, H, W, Co))
    dw = CO.conv3d_wgrad(dy, x)
    for o in range(Co):
        for kz in range(3):
            for ky in range(3):
                for kx in range(3):
                    for c in range(Ci):
                        s = 0.0
                        for z in range(D):
                            for yy in range(H):
                                for xx in range(W):
                                    zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                        s += dy[0, z, yy, xx, o] * x[0, zz, y2, x2, c]
                        assert abs(dw[o, kz, ky, kx, c] - s) < 1e-12


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((2, 4, 6, 2, 3))
    b = rng.standard_normal((2, 2, 3, 1, 3))
    assert abs(_inner(CO.pool2(a), b) - _inner(a, CO.pool2_adjoint(b))) < 1e-12
    assert abs(_inner(CO.up2(b), a) - _inner(b, CO.up2_adjoint(a))) < 1e-12
    assert np.allclose(CO.pool2(CO.up2(b)), b)
    # a 2x2x2 block of equal children pools to that value
    assert CO.pool2(np.full((1, 2, 2, 2, 1), 3.5))[0, 0, 0, 0, 0] == 3.5


def test_cell_to_node_reproduces_constants_and_interior_linear_fields():
    s = 4
    c = np.zeros((1, s, s, s, 3))
    c[..., 0], c[..., 1], c[..., 2] = 1.5, -2.0, 0.25
    n = CO.cell_to_node(c).reshape(3, s + 1, s + 1, s + 1)
    assert np.allclose(n[0], 1.5) and np.allclose(n[1], -2.0) and np.allclose(n[2], 0.25)
    # linear in x: cell i holds i + 1/2, node k (interior) its position k
    lin = np.zeros((1, s, s, s, 3))
    lin[..., 0] = (np.arange(s) + 0.5)[None, None, None, :]
    nx = CO.cell_to_node(lin).reshape(3, s + 1, s + 1, s + 1)[0]
    assert np.allclose(nx[:, :, 1:s], np.arange(1, s)[None, None, :])
    assert np.allclose(nx[:, :, 0], 0.5) and np.allclose(nx[:, :, s], s - 0.5)  # clamped ends
    rng = np.random.default_rng(8)
    a = rng.standard_normal((2, s, s, s, 3))
    g = rng.standard_normal((2, 3, (s + 1) ** 3))
    assert abs(_inner(CO.cell_to_node(a), g) - _inner(a, CO.cell_to_node_adjoint(g, s))) < 1e-12


def _tiny_net(seed=9, s=8, B=2):
    rng = np.random.default_rng(seed)
    p = CO.net_init(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.05 * rng.standard_normal(p[k].shape)
            if k == "b7":
                p[k][3:] = 0.0
    R = rng.standard_normal((B, s, s, s)) * 300.0 - 500.0
    T = R + rng.standard_normal((B, s, s, s)) * 100.0
    ut = rng.standard_normal((B, 3, (s // 4 + 1) ** 3)) * 2.0
    return p, R, T, ut


def test_network_gradient_matches_finite_differences():
    """Central differences of the loss in float64 along single parameters
    of every layer (weights and biases) match net_backward."""
    p, R, T, ut = _tiny_net()
    sh, sc, os_ = -500.0, 1.0 / 500.0, 3.0
    a = CO.net_forward(p, R, T, sh, sc, os_)
    g = CO.net_backward(p, a, ut, os_)
    rng = np.random.default_rng(10)
    eps = 1e-6
    for k in p:
        for _ in range(3):
            idx = tuple(int(rng.integers(0, d)) for d in p[k].shape)
            if k in ("W7", "b7") and idx[0] >= 3:
                idx = (int(rng.integers(0, 3)),) + idx[1:]
            old = p[k][idx]
            p[k][idx] = old + eps
            lp = CO.net_loss(CO.net_forward(p, R, T, sh, sc, os_), ut, os_)
            p[k][idx] = old - eps
            lm = CO.net_loss(CO.net_forward(p, R, T, sh, sc, os_), ut, os_)
            p[k][idx] = old
            fd = (lp - lm) / (2 * eps)
            # the difference quotient's own rounding is about 1e-16 / eps
            assert abs(fd - g[k][idx]) <= 1e-5 * abs(fd) + 1e-9, (k, idx, fd, g[k][idx])


def test_network_output_shape_and_loss_at_target():
    p, R, T, ut = _tiny_net(s=16, B=1)
    a = CO.net_forward(p, R, T, -500.0, 1.0 / 500.0, 3.0)
    assert a["u"].shape == (1, 3, 5 ** 3)
    assert CO.net_loss(a, a["u"], 3.0) == 0.0


def test_adam_first_step_moves_each_parameter_by_lr():
    """After one step from zero moments, Adam moves each parameter with a
    non-zero gradient by lr * g / (|g| + eps / sqrt(1 - beta2)) ~ lr."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    CO.adam_step(p, g, m, v, 1, 0.01)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-7)


def test_to_bf16_rounds_to_nearest_even():
    # bfloat16 keeps 8 significant bits: the spacing above 1 is 2^-7
    assert CO.to_bf16(1.0) == 1.0
    assert CO.to_bf16(1.0 + 2.0 ** -9) == 1.0                  # below half a spacing
    assert CO.to_bf16(1.0 + 2.0 ** -8) == 1.0                  # tie: even significand kept
    assert CO.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie: rounds up to even
    assert CO.to_bf16(-(1.0 + 3 * 2.0 ** -9)) == -(1.0 + 2.0 ** -7)
    x = np.random.default_rng(11).standard_normal(1000)
    assert np.all(np.abs(CO.to_bf16(x) - x) <= 2.0 ** -8 * np.abs(x))
