"""Tensor-core 3x3x3 convolution (learned-initializer building block) against
the FP64 convolution oracle, on bf16 inputs both sides read exactly.

Bar: |y - y_oracle| <= 1e-5 * sum |w| |x| per output (FP32 accumulation of
27 * Cin exact bf16 products in any order stays far inside it).
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

# (B, D, H, W, Cin, Cout): ragged voxel counts (not multiples of 128), one
# and several channel stages, the smallest and largest Cout
CASES = [
    (1, 4, 5, 7, 16, 16),
    (2, 6, 5, 9, 32, 48),
    (1, 8, 8, 8, 64, 32),
    (1, 5, 6, 7, 128, 64),
    (1, 3, 4, 5, 16, 256),
    (1, 17, 9, 13, 48, 128),
    (3, 7, 3, 11, 192, 16),
]


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import ngf as m
    assert torch.cuda.is_available()
    return m


def _inputs(shape, seed, bias=False):
    B, D, H, W, Ci, Co = shape
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(B, D, H, W, Ci, generator=g).to(torch.bfloat16)
    w = (torch.randn(Co, 3, 3, 3, Ci, generator=g) / np.sqrt(27 * Ci)).to(torch.bfloat16)
    b = torch.randn(Co, generator=g) if bias else None
    return x, w, b


def _check(x, w, y, b=None, relu=False):
    xo, wo = x.float().numpy(), w.float().numpy()
    yo = CO.conv3d(xo, wo, None if b is None else b.numpy(), relu)
    bound = 1e-5 * CO.conv3d_abs(xo, wo) + 1e-30
    err = np.abs(y.double().cpu().numpy() - yo)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("shape", CASES)
def test_conv3d_matches_oracle(ngf, shape):
    x, w, _ = _inputs(shape, seed=sum(shape))
    y = torch.full(shape[:4] + (shape[5],), float("nan"), device="cuda")
    ngf.ngf_conv3d_fwd(x.cuda(), w.cuda(), None, y)
    assert ngf.ngf_conv3d_check() == 0
    _check(x, w, y)


def test_conv3d_bias_relu(ngf):
    shape = (2, 5, 6, 7, 32, 32)
    x, w, b = _inputs(shape, seed=7, bias=True)
    y = torch.empty(shape[:4] + (shape[5],), device="cuda")
    ngf.ngf_conv3d_fwd(x.cuda(), w.cuda(), b.cuda(), y, relu=True)
    assert ngf.ngf_conv3d_check() == 0
    _check(x, w, y, b, relu=True)
    assert (y >= 0).all() and (y == 0).any()


def test_conv3d_deterministic(ngf):
    shape = (1, 9, 10, 11, 64, 64)
    x, w, _ = _inputs(shape, seed=8)
    x, w = x.cuda(), w.cuda()
    y1 = torch.empty(shape[:4] + (64,), device="cuda")
    y2 = torch.empty_like(y1)
    ngf.ngf_conv3d_fwd(x, w, None, y1)
    ngf.ngf_conv3d_fwd(x, w, None, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_conv3d_empty_and_bad_arguments(ngf):
    x = torch.zeros(1, 0, 4, 4, 16, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(16, 3, 3, 3, 16, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(1, 0, 4, 4, 16, device="cuda")
    ngf.ngf_conv3d_fwd(x, w, None, y)  # empty volume: no-op
    x = torch.zeros(1, 2, 2, 2, 8, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(16, 3, 3, 3, 8, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(1, 2, 2, 2, 16, device="cuda")
    with pytest.raises(ngf.NGFError):
        ngf.ngf_conv3d_fwd(x, w, None, y)  # Cin not a multiple of 16
    x = torch.zeros(1, 2, 2, 2, 16, dtype=torch.bfloat16, device="cuda")
    for co in (8, 24, 272):
        w = torch.zeros(co, 3, 3, 3, 16, dtype=torch.bfloat16, device="cuda")
        y = torch.zeros(1, 2, 2, 2, co, device="cuda")
        with pytest.raises(ngf.NGFError):
            ngf.ngf_conv3d_fwd(x, w, None, y)
    assert ngf.ngf_conv3d_check() == 0


# Volumes with at least as many output tiles (8 x 16 x P voxels) as the GPU
# has SMs, so that no output-channel slicing happens and every CTA computes
# all output channels of its tile (the path the 64^3 and 128^3 layers take),
# with 16 to 128 input channels, a batch of two and ragged tiles; the ones
# with at most 64 output channels take the z-stacked taps.
LARGE_CASES = [
    (1, 32, 48, 64, 32, 64),
    (1, 40, 64, 64, 16, 16),
    (2, 24, 48, 40, 16, 32),
    (1, 32, 64, 64, 64, 64),
    (1, 32, 64, 64, 128, 32),  # z-stacked taps, 4 planes per CTA, two 64-channel chunks
]


@pytest.mark.parametrize("shape", LARGE_CASES)
def test_conv3d_matches_oracle_full_grid(ngf, shape):
    B, D, H, W, Ci, Co = shape
    tiles = ((W + 7) // 8) * ((H + 15) // 16) * ((D + 3) // 4) * B
    assert tiles >= torch.cuda.get_device_properties(0).multi_processor_count
    x, w, b = _inputs(shape, seed=sum(shape), bias=True)
    y = torch.full(shape[:4] + (Co,), float("nan"), device="cuda")
    ngf.ngf_conv3d_fwd(x.cuda(), w.cuda(), b.cuda(), y, relu=True)
    assert ngf.ngf_conv3d_check() == 0
    _check(x, w, y, b, relu=True)
