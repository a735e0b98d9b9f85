"""The learned-initializer workload: synthetic lung-CT-like pairs, their plain
multilevel Gauss-Newton registrations (the training targets), training of the
encoder-decoder, and the comparison with plain Gauss-Newton from zero at equal
final objective.

Orchestration only: every computation is a call of the C ABI
(register_batch, register_multilevel, ngf_net_forward, ngf_net_train) or of
the seeded input generators in `synth`.  The paper starts its multilevel
Gauss-Newton method from u = 0 on the coarsest level (Sec. 2.3); the network
replaces that start by a prediction on the second level, from which the same
method continues, so it is always refined (and judged) by the plain method.

Pairs: built like the lung-CT workload (same phantom, breathing displacement
up to 15 mm, 256 x 256 x 300 mm field of view) but sampled at s^3 voxels
(s = 128: 2 x 2 x 2.34 mm), nodes s/2 + 1 per axis (two voxels per cell),
alpha = 1, tau = rho = 10.  Pair k uses generator seed 40 + k.
"""
import math
import time

import numpy as np
import torch

from . import ngf, synth

SEED0 = 40
GN_ITERS, PCG_ITERS = 10, 20
IN_SHIFT, IN_SCALE, OUT_SCALE = -500.0, 1.0 / 500.0, 5.0
LAYERS = [(16, 16), (16, 32), (32, 64), (64, 128), (128, 64), (64, 64), (64, 16)]


def workload(s=128):
    """Registration level description of the s^3 pairs."""
    levels = int(round(math.log2(s // 8)))
    return dict(m=(s, s, s), h=(256.0 / s, 256.0 / s, 300.0 / s), n=(s // 2 + 1,) * 3, alpha=1.0, tau=10.0,
                rho=10.0, levels=levels, start_level=1)


def make_pairs(s, first, count, device):
    """R, T [count, s^3] float32 for pair indices first .. first + count - 1."""
    w = workload(s)
    M = s ** 3
    R = torch.empty(count, M, device=device)
    T = torch.empty(count, M, device=device)
    for j in range(count):
        R[j], T[j] = synth.lung_pair_windowed(w["m"], w["h"], SEED0 + first + j, device=device)
    return R, T


def desc_of(w):
    return ngf.level_desc(w["m"], w["h"], w["n"], w["alpha"], w["tau"], w["rho"])


def register_all(R, T, w, chunk=64, stream=None):
    """Plain multilevel Gauss-Newton from u = 0 for every pair (batched, one
    register_batch call per `chunk` pairs).  Returns the finest-level u
    [N, 3 n^3] and the final objectives J [N]."""
    N = R.shape[0]
    n0 = w["n"][0] ** 3
    U = torch.zeros(N, 3 * n0, device=R.device)
    J = np.zeros(N)
    d = desc_of(w)
    opts = ngf.options(levels=w["levels"], gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        reps = ngf.register_batch([d] * (c1 - c0), opts, [R[k] for k in range(c0, c1)],
                                  [T[k] for k in range(c0, c1)], [U[k] for k in range(c0, c1)], stream=stream)
        J[c0:c1] = [r.J for r in reps]
    return U, J


def level1_targets(U0, n0):
    """Finest-level u on n0^3 nodes -> the level-1 grid ((n0 + 1) / 2 nodes
    per axis): level-1 node j sits on level-0 node 2j (same domain, half the
    cells), so the target is the even-indexed subsample."""
    N = U0.shape[0]
    u = U0.view(N, 3, n0, n0, n0)[:, :, ::2, ::2, ::2]
    return u.contiguous().view(N, -1)


def init_params(seed):
    """He-normal weights (numpy PCG64), zero biases; the head's unused output
    channels (3..15) start and stay at zero; the head starts small."""
    r = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for k, (ci, co) in enumerate(LAYERS):
        wgt = r.normal(size=(co, 27, ci)) * math.sqrt(2.0 / (27 * ci))
        if k == len(LAYERS) - 1:
            wgt *= 0.1
            wgt[3:] = 0.0
        parts += [wgt.ravel(), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def train(net, R, T, U1, epochs, batch, lr0, seed=1, log=None):
    """Adam over all pairs for `epochs` epochs (a new random order each
    epoch, numpy PCG64 `seed`), learning rate lr0 with a cosine decay per
    epoch to lr0 / 20.  Returns the mean training loss of each epoch."""
    r = np.random.Generator(np.random.PCG64(seed))
    N = R.shape[0]
    out = []
    for ep in range(epochs):
        lr = lr0 * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs))))
        order = r.permutation(N)
        losses = ngf.ngf_net_train(net.handle, R, T, U1, N, order, batch, lr)
        out.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: lr {lr:.2e} loss {out[-1]:.4f}")
    return out


def predict(net, R, T, batch):
    """Network prediction on the level-1 node grid for every pair."""
    s = round(R.shape[1] ** (1.0 / 3.0))
    n1 = s // 4 + 1
    N = R.shape[0]
    U = torch.empty(N, 3 * n1 ** 3, device=R.device)
    for c0 in range(0, N, batch):
        c1 = min(N, c0 + batch)
        ngf.ngf_net_forward(net.handle, R[c0:c1], T[c0:c1], c1 - c0, U[c0:c1])
    return U


def compare(net, R, T, w, k1=3, finest_cap=30, tol=1e-3, stream=None):
    """Per held-out pair: plain Gauss-Newton from zero with its full
    schedule (levels x 10 steps) gives J_ref; then plain Gauss-Newton from
    zero and the network's start refined by Gauss-Newton (k1 steps on level
    1, then the finest level) both stop on the finest level once
    J <= J_ref (1 + tol).  Times include the network's forward pass; every
    call is synchronised, so wall-clock time is device time plus launch
    overhead."""
    d = desc_of(w)
    n0 = w["n"][0] ** 3
    u = torch.empty(3 * n0, device=R.device)
    s = w["m"][0]
    n1 = s // 4 + 1
    u1 = torch.empty(3 * n1 ** 3, device=R.device)
    o_full = ngf.options(levels=w["levels"], gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True)
    rows = []
    for k in range(R.shape[0]):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rf = ngf.register_multilevel(d, o_full, R[k], T[k], u, stream)
        tf = time.perf_counter() - t0
        target = rf.J * (1.0 + tol)
        o_plain = ngf.options(levels=w["levels"], gn_iters=GN_ITERS, pcg_iters=PCG_ITERS, use_graph=True,
                              gn_iters_finest=GN_ITERS, j_target=target)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp = ngf.register_multilevel(d, o_plain, R[k], T[k], u, stream)
        tp = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ngf.ngf_net_forward(net.handle, R[k:k + 1], T[k:k + 1], 1, u1)
        o_l = ngf.options(levels=w["levels"], gn_iters=k1, pcg_iters=PCG_ITERS, use_graph=True,
                          start_level=w["start_level"], u_init=u1, gn_iters_finest=finest_cap, j_target=target)
        rl = ngf.register_multilevel(d, o_l, R[k], T[k], u, stream)
        tl = time.perf_counter() - t0
        rows.append(dict(J_ref=rf.J, full_gn=rf.gn_done, full_s=tf, plain_J=rp.J, plain_gn=rp.gn_done, plain_s=tp,
                         learned_J=rl.J,
                         learned_gn=rl.gn_done, learned_s=tl, learned_reached=bool(rl.J <= target),
                         plain_reached=bool(rp.J <= target)))
    return rows
