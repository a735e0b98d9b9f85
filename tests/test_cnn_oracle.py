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
