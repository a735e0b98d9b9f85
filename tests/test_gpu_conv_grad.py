"""Tensor-core convolution gradients and the bf16-output forward of the
learned initializer against the FP64 oracle (oracle/cnn_oracle.py), on bf16
inputs both sides read exactly.

Bars: float outputs |y - y_oracle| <= 1e-5 * (the sum of |terms|) per
element (FP32 accumulation of exact bf16 products in any order stays far
inside it); bf16 outputs additionally one bf16 rounding, 2^-8 |y_oracle|.
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

# (B, D, H, W, Cin, Cout): every layer shape of the encoder-decoder at small
# sizes, ragged tiles, one and several input-channel chunks
SHAPES = [
    (1, 8, 8, 8, 16, 16),
    (2, 5, 6, 7, 16, 32),
    (1, 9, 7, 18, 32, 64),
    (2, 4, 4, 4, 64, 128),
    (1, 6, 8, 10, 128, 64),
    (1, 8, 8, 8, 64, 64),
    (1, 7, 5, 9, 64, 16),
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _data(shape, seed):
    B, D, H, W, Ci, Co = shape
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(B, D, H, W, Ci, generator=g).to(torch.bfloat16)
    w = (torch.randn(Co, 3, 3, 3, Ci, generator=g) / np.sqrt(27 * Ci)).to(torch.bfloat16)
    dy = torch.randn(B, D, H, W, Co, generator=g).to(torch.bfloat16)
    return x, w, dy


def _f(t):
    return t.float().cpu().double().numpy()


@pytest.mark.parametrize("shape", SHAPES)
def test_wgrad_matches_oracle(ngf, shape):
    x, w, dy = _data(shape, sum(shape))
    Co, Ci = shape[5], shape[4]
    dw = torch.full((Co, 3, 3, 3, Ci), float("nan"), device="cuda")
    db = torch.full((Co,), float("nan"), device="cuda")
    ngf.ngf_conv3d_wgrad(dy.cuda(), x.cuda(), dw, db)
    assert ngf.ngf_conv3d_check() == 0
    ref = CO.conv3d_wgrad(_f(dy), _f(x))
    bound = 1e-5 * CO.wgrad_abs(_f(dy), _f(x)) + 1e-30
    err = np.abs(_f(dw) - ref)
    assert np.all(err <= bound), float((err / bound).max())
    rb = CO.bias_grad(_f(dy))
    assert np.all(np.abs(_f(db) - rb) <= 1e-5 * CO.bias_grad(np.abs(_f(dy))))


@pytest.mark.parametrize("shape", SHAPES)
def test_dgrad_matches_oracle(ngf, shape):
    x, w, dy = _data(shape, sum(shape) + 1)
    B, D, H, W, Ci, Co = shape
    dx = torch.full((B, D, H, W, Ci), float("nan"), device="cuda")
    ngf.ngf_conv3d_dgrad(dy.cuda(), w.cuda(), dx)
    assert ngf.ngf_conv3d_check() == 0
    ref = CO.conv3d_dgrad(_f(dy), _f(w))
    bound = 1e-5 * CO.dgrad_abs(_f(dy), _f(w)) + 1e-30
    err = np.abs(_f(dx) - ref)
    assert np.all(err <= bound), float((err / bound).max())
    # bf16 output: the float result rounded once more
    dxb = torch.empty((B, D, H, W, Ci), device="cuda", dtype=torch.bfloat16)
    ngf.ngf_conv3d_dgrad(dy.cuda(), w.cuda(), dxb, flags=ngf.NGF_CONV_OUT_BF16)
    err = np.abs(_f(dxb) - ref)
    assert np.all(err <= bound + 2.0 ** -8 * np.abs(ref)), float((err / (bound + 2.0 ** -8 * np.abs(ref))).max())


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_forward_bf16_relu_matches_oracle(ngf, shape):
    x, w, _ = _data(shape, sum(shape) + 2)
    B, D, H, W, Ci, Co = shape
    g = torch.Generator().manual_seed(3)
    b = torch.randn(Co, generator=g) * 0.1
    y = torch.empty((B, D, H, W, Co), device="cuda", dtype=torch.bfloat16)
    ngf.ngf_conv3d_fwd_ex(x.cuda(), w.cuda(), b.cuda(), y, flags=ngf.NGF_CONV_RELU | ngf.NGF_CONV_OUT_BF16)
    assert ngf.ngf_conv3d_check() == 0
    ref = CO.conv3d(_f(x), _f(w), b.double().numpy(), relu=True)
    bound = 1e-5 * CO.conv3d_abs(_f(x), _f(w)) + 2.0 ** -8 * np.abs(ref) + 1e-30
    err = np.abs(_f(y) - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_dgrad_large_volume_matches_oracle(ngf):
    """A data gradient on a volume with more tiles than SMs (no output
    channel slicing in the mirrored convolution), checked element-wise."""
    shape = (1, 32, 48, 64, 32, 16)
    x, w, dy = _data(shape, 99)
    B, D, H, W, Ci, Co = shape
    dx = torch.empty((B, D, H, W, Ci), device="cuda", dtype=torch.bfloat16)
    ngf.ngf_conv3d_dgrad(dy.cuda(), w.cuda(), dx, flags=ngf.NGF_CONV_OUT_BF16)
    assert ngf.ngf_conv3d_check() == 0
    ref = CO.conv3d_dgrad(_f(dy), _f(w))
    bound = 1e-5 * CO.dgrad_abs(_f(dy), _f(w)) + 2.0 ** -8 * np.abs(ref) + 1e-30
    err = np.abs(_f(dx) - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_gradients_are_deterministic(ngf):
    x, w, dy = _data((1, 12, 10, 20, 32, 64), 77)
    x, w, dy = x.cuda(), w.cuda(), dy.cuda()
    out = []
    for _ in range(2):
        dw = torch.empty(64, 3, 3, 3, 32, device="cuda")
        dx = torch.empty(1, 12, 10, 20, 32, device="cuda")
        ngf.ngf_conv3d_wgrad(dy, x, dw)
        ngf.ngf_conv3d_dgrad(dy, w, dx)
        out.append((dw, dx))
    torch.cuda.synchronize()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
