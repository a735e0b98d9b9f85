"""FP64 CPU oracle of the learned initializer (test infrastructure only:
tests, smoke and the benchmark's CPU leg use it).

A learned initializer supplies the Gauss-Newton method of Sec. 2.3 with a
starting deformation instead of u = 0 (the paper has no network; its
multilevel start from u = 0 is what this replaces).  This module states, by
their definitions and in float64, every operation of that network:

  * the 3x3x3 convolution, one tap at a time:
        y[n, z, y, x, o] = b[o] + sum over (dz, dy, dx) in {-1, 0, 1}^3 and c of
                           w[o, dz+1, dy+1, dx+1, c] * x[n, z+dz, y+dy, x+dx, c]
    with x = 0 outside the volume (zero padding of one voxel, stride 1), and
    optionally max(y, 0); layouts channels last: x [B][D][H][W][Cin],
    w [Cout][3][3][3][Cin], y [B][D][H][W][Cout];
  * its data, weight and bias gradients;
  * 2x mean pooling, nearest upsampling, the cell-to-node average of the
    output and their transposes;
  * the encoder-decoder itself, its loss, its gradients by the chain rule,
    and an Adam step.
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


# ---------------------------------------------------------------- backward
#
# The two other products of a convolution layer, stated from the forward
# definition above (y = conv3d(x, w)), in float64:
#   data gradient    dx[n,z,y,x,c]  = sum_{taps, o} w[o, tap, c] dy[n, (z,y,x) - tap, o]
#   weight gradient  dw[o, tap, c]  = sum_{n,z,y,x} dy[n,z,y,x,o] x[n, (z,y,x) + tap, c]
#   bias gradient    db[o]          = sum_{n,z,y,x} dy[n,z,y,x,o]
# with tap = (kz-1, ky-1, kx-1) and zero outside the volume.


def conv3d_dgrad(dy, w):
    """dx = (d conv3d / dx)^T dy, one tap at a time."""
    dy = np.asarray(dy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, D, H, W, Cout = dy.shape
    Cin = w.shape[4]
    dxp = np.zeros((B, D + 2, H + 2, W + 2, Cin))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                # output voxel (z, y, x) read input voxel (z + kz - 1, ...)
                dxp[:, kz:kz + D, ky:ky + H, kx:kx + W, :] += dy @ w[:, kz, ky, kx, :]
    return dxp[:, 1:-1, 1:-1, 1:-1, :]


def conv3d_wgrad(dy, x):
    """dw[o, kz, ky, kx, c] (the layout of w), one tap at a time."""
    dy = np.asarray(dy, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    B, D, H, W, Cout = dy.shape
    Cin = x.shape[4]
    xp = np.zeros((B, D + 2, H + 2, W + 2, Cin))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    dw = np.zeros((Cout, 3, 3, 3, Cin))
    dyf = dy.reshape(-1, Cout)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                dw[:, kz, ky, kx, :] = dyf.T @ xp[:, kz:kz + D, ky:ky + H, kx:kx + W, :].reshape(-1, Cin)
    return dw


def bias_grad(dy):
    dy = np.asarray(dy, dtype=np.float64)
    return dy.reshape(-1, dy.shape[-1]).sum(0)


def wgrad_abs(dy, x):
    """sum |dy| |x| over the terms of each weight gradient (rounding scale)."""
    return conv3d_wgrad(np.abs(dy), np.abs(x))


def dgrad_abs(dy, w):
    return conv3d_dgrad(np.abs(dy), np.abs(w))


# ------------------------------------------------- resampling between levels


def pool2(x):
    """Mean of the 2 x 2 x 2 children: [B, 2D, 2H, 2W, C] -> [B, D, H, W, C]."""
    x = np.asarray(x, dtype=np.float64)
    B, D, H, W, C = x.shape
    return x.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_adjoint(dy):
    """Transpose of pool2: every child receives its parent's value / 8."""
    return up2(dy) / 8.0


def up2(x):
    """Nearest-neighbour upsampling by 2 per axis (each child copies its parent)."""
    x = np.asarray(x, dtype=np.float64)
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def up2_adjoint(dy):
    """Transpose of up2: each parent sums its 8 children."""
    dy = np.asarray(dy, dtype=np.float64)
    B, D, H, W, C = dy.shape
    return dy.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def cell_to_node(v):
    """Cell-centred field [B, s, s, s, 3] -> node field [B, 3, (s+1)^3]
    (component-major, x fastest).  Node k of an axis sits on the face between
    cells k-1 and k and takes their mean; the first and last nodes take the
    outer cell (indices clamped to 0 .. s-1): per axis a 2-tap average,
    applied along x, y and z."""
    v = np.asarray(v, dtype=np.float64)

    def axis_avg(a, ax):
        s = a.shape[ax]
        lo = np.take(a, np.clip(np.arange(s + 1) - 1, 0, s - 1), axis=ax)
        hi = np.take(a, np.clip(np.arange(s + 1), 0, s - 1), axis=ax)
        return 0.5 * (lo + hi)

    out = axis_avg(axis_avg(axis_avg(v, 1), 2), 3)  # [B, s+1, s+1, s+1, 3]
    return np.moveaxis(out, 4, 1).reshape(v.shape[0], 3, -1)


def cell_to_node_adjoint(g, s):
    """Transpose of cell_to_node: node field [B, 3, (s+1)^3] -> cells [B, s, s, s, 3]."""
    g = np.asarray(g, dtype=np.float64)
    B = g.shape[0]
    a = np.moveaxis(g.reshape(B, 3, s + 1, s + 1, s + 1), 1, 4)

    def axis_avg_T(a, ax):
        n = a.shape[ax]
        out_shape = list(a.shape)
        out_shape[ax] = n - 1
        out = np.zeros(out_shape)
        for k in range(n):
            for j in (k - 1, k):
                i = min(max(j, 0), n - 2)
                sl_out = [slice(None)] * a.ndim
                sl_out[ax] = i
                sl_in = [slice(None)] * a.ndim
                sl_in[ax] = k
                out[tuple(sl_out)] += 0.5 * a[tuple(sl_in)]
        return out

    return axis_avg_T(axis_avg_T(axis_avg_T(a, 3), 2), 1)


# ------------------------------------------------------------ the network
#
# A small 3-D encoder-decoder that maps an image pair at s^3 (s divisible by
# 8) to a displacement on the (s/4 + 1)^3 node grid of the registration level
# with s/2 image cells per axis (two image cells per deformation cell), the
# level at which the Gauss-Newton method then starts.  Four resolution
# levels with 16, 32, 64 and 128 channels:
#
#   x0 = [(R - shift) * scale, (T - shift) * scale, 0 x 14]     s^3 x 16
#   e1 = relu(conv(x0, W1) + b1)   s^3     16     p1 = pool2(e1)
#   e2 = relu(conv(p1, W2) + b2)   s/2     32     p2 = pool2(e2)
#   e3 = relu(conv(p2, W3) + b3)   s/4     64     p3 = pool2(e3)
#   e4 = relu(conv(p3, W4) + b4)   s/8    128
#   d3 = relu(conv(up2(e4), W5) + b5)   s/4  64
#   s3 = d3 + e3                        s/4  64   (skip connection)
#   d2 = relu(conv(s3, W6) + b6)        s/4  64
#   o  = conv(d2, W7) + b7              s/4  16   (channels 0..2 used)
#   u  = out_scale * cell_to_node(o[..., :3])    3 x (s/4 + 1)^3
#   loss = mean over pairs, components and nodes of ((u - u_target) / out_scale)^2
#
# The paper has no network: it starts the multilevel Gauss-Newton method from
# u = 0 on the coarsest level (Sec. 2.3); this network only supplies another
# starting point for it.

NET_LAYERS = [  # (name, Cin, Cout)
    ("1", 16, 16), ("2", 16, 32), ("3", 32, 64), ("4", 64, 128), ("5", 128, 64), ("6", 64, 64), ("7", 64, 16)]


def net_init(seed, head_rows=3):
    """He-normal weights (numpy PCG64), zero biases; rows >= head_rows of
    the last layer are zero (those output channels are unused)."""
    r = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co in NET_LAYERS:
        w = r.normal(size=(co, 3, 3, 3, ci)) * np.sqrt(2.0 / (27 * ci))
        if name == "7":
            w *= 0.1
            w[head_rows:] = 0.0
        p["W" + name] = w
        p["b" + name] = np.zeros(co)
    return p


def net_forward(p, R, T, shift, scale, out_scale, rnd=None):
    """Activations of the network for images R, T of shape [B, s, s, s]
    (float64 definitions; `rnd`, if given, is applied to every stored
    activation to model the precision it is stored in)."""
    q = rnd if rnd is not None else (lambda a: a)
    R = np.asarray(R, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = R.shape[0]
    x0 = np.zeros(R.shape + (16,))
    x0[..., 0] = (R - shift) * scale
    x0[..., 1] = (T - shift) * scale
    a = {"x0": q(x0)}
    a["e1"] = q(conv3d(a["x0"], p["W1"], p["b1"], relu=True))
    a["p1"] = q(pool2(a["e1"]))
    a["e2"] = q(conv3d(a["p1"], p["W2"], p["b2"], relu=True))
    a["p2"] = q(pool2(a["e2"]))
    a["e3"] = q(conv3d(a["p2"], p["W3"], p["b3"], relu=True))
    a["p3"] = q(pool2(a["e3"]))
    a["e4"] = q(conv3d(a["p3"], p["W4"], p["b4"], relu=True))
    a["up"] = q(up2(a["e4"]))
    a["d3"] = q(conv3d(a["up"], p["W5"], p["b5"], relu=True))
    a["s3"] = q(a["d3"] + a["e3"])
    a["d2"] = q(conv3d(a["s3"], p["W6"], p["b6"], relu=True))
    a["o"] = conv3d(a["d2"], p["W7"], p["b7"])
    a["u"] = out_scale * cell_to_node(a["o"][..., :3])
    a["B"] = B
    return a


def net_loss(a, u_target, out_scale):
    ut = np.asarray(u_target, dtype=np.float64).reshape(a["u"].shape)
    d = (a["u"] - ut) / out_scale
    return float(np.mean(d * d))


def net_backward(p, a, u_target, out_scale, rnd=None):
    """Gradients of net_loss with respect to every parameter (same keys as
    p), by the chain rule layer by layer (`rnd` models the precision each
    propagated gradient is stored in)."""
    q = rnd if rnd is not None else (lambda t: t)
    ut = np.asarray(u_target, dtype=np.float64).reshape(a["u"].shape)
    s = a["o"].shape[1]
    g = {}
    du = 2.0 * (a["u"] - ut) / (out_scale * out_scale * a["u"].size)
    do = np.zeros(a["o"].shape)
    do[..., :3] = out_scale * cell_to_node_adjoint(du, s)
    do = q(do)
    g["W7"], g["b7"] = conv3d_wgrad(do, a["d2"]), bias_grad(do)
    dz6 = q(conv3d_dgrad(do, p["W7"]) * (a["d2"] > 0))
    g["W6"], g["b6"] = conv3d_wgrad(dz6, a["s3"]), bias_grad(dz6)
    ds3 = q(conv3d_dgrad(dz6, p["W6"]))
    dz5 = q(ds3 * (a["d3"] > 0))
    g["W5"], g["b5"] = conv3d_wgrad(dz5, a["up"]), bias_grad(dz5)
    dup = q(conv3d_dgrad(dz5, p["W5"]))
    dz4 = q(up2_adjoint(dup) * (a["e4"] > 0))
    g["W4"], g["b4"] = conv3d_wgrad(dz4, a["p3"]), bias_grad(dz4)
    dp3 = q(conv3d_dgrad(dz4, p["W4"]))
    dz3 = q((pool2_adjoint(dp3) + ds3) * (a["e3"] > 0))
    g["W3"], g["b3"] = conv3d_wgrad(dz3, a["p2"]), bias_grad(dz3)
    dp2 = q(conv3d_dgrad(dz3, p["W3"]))
    dz2 = q(pool2_adjoint(dp2) * (a["e2"] > 0))
    g["W2"], g["b2"] = conv3d_wgrad(dz2, a["p1"]), bias_grad(dz2)
    dp1 = q(conv3d_dgrad(dz2, p["W2"]))
    dz1 = q(pool2_adjoint(dp1) * (a["e1"] > 0))
    g["W1"], g["b1"] = conv3d_wgrad(dz1, a["x0"]), bias_grad(dz1)
    return g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of every parameter in place;
    t is the 1-based step count."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def to_bf16(a):
    """Round float64/float32 values to the nearest bfloat16 (ties to even),
    returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)
