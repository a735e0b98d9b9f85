"""FP64 CPU oracle of the learned initializer's convolution (test
infrastructure only: tests, smoke and the benchmark's CPU leg use it).

A learned initializer supplies the Gauss-Newton method of Sec. 2.3 with a
starting deformation instead of u = 0; its dense work is 3x3x3 convolution.
This module states that convolution by its definition, one tap at a time:

    y[n, z, y, x, o] = b[o] + sum over (dz, dy, dx) in {-1, 0, 1}^3 and c of
                       w[o, dz+1, dy+1, dx+1, c] * x[n, z+dz, y+dy, x+dx, c]

with x = 0 outside the volume (zero padding of one voxel, stride 1), and
optionally max(y, 0).  Layouts are channels last: x [B][D][H][W][Cin],
w [Cout][3][3][3][Cin], y [B][D][H][W][Cout].
"""
import numpy as np


def conv3d(x, w, bias=None, relu=False):
    """Reference convolution in float64 (see the module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, D, H, W, Cin = x.shape
    Cout = w.shape[0]
    assert w.shape == (Cout, 3, 3, 3, Cin)
    xp = np.zeros((B, D + 2, H + 2, W + 2, Cin))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    y = np.zeros((B, D, H, W, Cout))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                # neighbour (z + kz - 1, ...) of every output voxel
                patch = xp[:, kz:kz + D, ky:ky + H, kx:kx + W, :]
                y += patch @ w[:, kz, ky, kx, :].T
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)
    if relu:
        y = np.maximum(y, 0.0)
    return y


def conv3d_abs(x, w):
    """sum |w| |x| over each output's 27 * Cin terms: the scale of the
    rounding error of any summation order of that output."""
    return conv3d(np.abs(np.asarray(x, dtype=np.float64)), np.abs(np.asarray(w, dtype=np.float64)))
