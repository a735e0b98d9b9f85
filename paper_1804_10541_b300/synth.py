"""Seeded synthetic image pairs shaped like the paper's workloads.

Analytic phantoms are evaluated at the cell centres x (reference R) and at the
warped points x + u*(x) (template T), so the template needs no interpolation
and the known displacement u* is exact.  This module holds none of the
registration method's arithmetic; the oracle and the CUDA path both take its
outputs as plain input arrays.

Random parameters are drawn with numpy PCG64 from fixed seeds; phantoms are
evaluated with torch on the requested device (float64 for small volumes,
float32 in z-slabs for the large ones).  Every pair comes with its workload
description: image cells m, spacing h (mm), deformation nodes n, NGF
parameters tau = rho, curvature weight alpha and the number of levels.

Workloads (the paper's datasets are not available; these stand in for them):
  blobs_32     32^3 Gaussian blobs, unit spacing, 17^3 nodes, 2 levels.
  lung_ct      256x256x120 at 1x1x2.5 mm, lung-CT-like (body, two lungs,
               300 vessels), breathing displacement up to 15 mm, 129x129x61
               nodes, 4 levels, alpha = 1, tau = rho = 10 (Sec. 6.2.1).
  thorax_abd   512x512x900 at 0.8x0.8x1.0 mm, thorax-abdomen-like (body,
               organs, lungs, spine), smooth displacement up to 20 mm,
               129x129x225 nodes, 5 levels, alpha = 10, tau = rho = 5
               (Sec. 6.2.2).
  batch_64     64 blob pairs of uneven cubic size N ~ U{64..192} (seed 30),
               unit spacing, (N/2+1)^3 nodes, 2 levels; blob centres and
               widths scale with N (batch_pairs).
"""
import math

import numpy as np
import torch

WORKLOADS = {
    "blobs_32": dict(m=(32, 32, 32), h=(1.0, 1.0, 1.0), n=(17, 17, 17), alpha=1.0, tau=0.1,
                     rho=0.1, levels=2, seed=0),
    "lung_ct": dict(m=(256, 256, 120), h=(1.0, 1.0, 2.5), n=(129, 129, 61), alpha=1.0, tau=10.0,
                    rho=10.0, levels=4, seed=10),
    "thorax_abd": dict(m=(512, 512, 900), h=(0.8, 0.8, 1.0), n=(129, 129, 225), alpha=10.0,
                       tau=5.0, rho=5.0, levels=5, seed=20),
}


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _axes(m, h, z0, z1, device, dtype):
    x = ((torch.arange(m[0], device=device, dtype=dtype) + 0.5) * h[0]).view(1, 1, -1)
    y = ((torch.arange(m[1], device=device, dtype=dtype) + 0.5) * h[1]).view(1, -1, 1)
    z = ((torch.arange(z0, z1, device=device, dtype=dtype) + 0.5) * h[2]).view(-1, 1, 1)
    return x, y, z


def _step(d, width):
    """Smooth inside indicator from a signed inside-distance d (mm)."""
    return torch.sigmoid(d / width)


def _ellipsoid_depth(X, Y, Z, c, a):
    q = torch.sqrt(((X - c[0]) / a[0]) ** 2 + ((Y - c[1]) / a[1]) ** 2 + ((Z - c[2]) / a[2]) ** 2)
    return (1.0 - q) * min(a)


def _slabs(mz, planes):
    z = 0
    while z < mz:
        yield z, min(mz, z + planes)
        z += planes


# ------------------------------------------------------------------ blobs


class _Blobs:
    def __init__(self, m, h, seed, n_blobs=12):
        r = _rng(seed)
        ext = np.asarray(m, float) * np.asarray(h, float)
        s = min(ext) / 32.0
        self.c = r.uniform(0.125, 0.875, size=(n_blobs, 3)) * ext
        self.sig = r.uniform(2.0, 5.0, size=n_blobs) * s
        self.amp = r.uniform(0.3, 1.0, size=n_blobs)

    def __call__(self, X, Y, Z):
        out = torch.zeros(torch.broadcast_shapes(X.shape, Y.shape, Z.shape), dtype=X.dtype, device=X.device)
        for k in range(len(self.amp)):
            d2 = (X - self.c[k, 0]) ** 2 + (Y - self.c[k, 1]) ** 2 + (Z - self.c[k, 2]) ** 2
            out = out + self.amp[k] * torch.exp(-d2 / (2 * self.sig[k] ** 2))
        return out


def _sine_field(m, h, seed, max_disp):
    """u*_d(x) = a_d sin(2 pi x_{d+1}/L_{d+1} + phi_d) sin(pi x_d / L_d), scaled so
    that max |u*| over the cell centres is max_disp."""
    r = _rng(seed)
    phi = r.uniform(0, 2 * math.pi, 3)
    amp = r.uniform(0.5, 1.0, 3)
    ext = [m[a] * h[a] for a in range(3)]

    def raw(X, Y, Z):
        C = (X, Y, Z)
        return [amp[d] * torch.sin(2 * math.pi * C[(d + 1) % 3] / ext[(d + 1) % 3] + phi[d])
                * torch.sin(math.pi * C[d] / ext[d]) for d in range(3)]

    return raw


def blob_pair(m, h=(1.0, 1.0, 1.0), seed=0, max_disp_vox=2.0, noise=0.01, device="cpu"):
    """Reference = 12 Gaussian blobs + noise; template = blobs at x + u*(x) +
    fresh noise.  Seeds: seed (blobs), +1 (R noise), +2 (u*), +3 (T noise)."""
    dtype = torch.float64
    X, Y, Z = _axes(m, h, 0, m[2], device, dtype)
    blobs = _Blobs(m, h, seed)
    field = _sine_field(m, h, seed + 2, 1.0)
    U = [c.expand(m[2], m[1], m[0]) for c in field(X, Y, Z)]
    norm = torch.sqrt(U[0] ** 2 + U[1] ** 2 + U[2] ** 2).max()
    scale = max_disp_vox * min(h) / float(norm)
    U = [c * scale for c in U]
    R = blobs(X, Y, Z)
    T = blobs(X + U[0], Y + U[1], Z + U[2])
    gR = torch.Generator(device="cpu").manual_seed(seed + 1)
    gT = torch.Generator(device="cpu").manual_seed(seed + 3)
    R = R + noise * torch.randn(R.shape, generator=gR, dtype=dtype).to(device)
    T = T + noise * torch.randn(T.shape, generator=gT, dtype=dtype).to(device)
    return (R.reshape(-1).to(torch.float32), T.reshape(-1).to(torch.float32),
            torch.stack([c.reshape(-1) for c in U]).to(torch.float32))


# ------------------------------------------------------------------ lung CT


class _Lung:
    def __init__(self, m, h, seed):
        r = _rng(seed)
        ext = np.asarray(m, float) * np.asarray(h, float)
        self.ext = ext
        cx, cy, cz = ext / 2
        self.body = ((cx, cy, cz), (0.46 * ext[0], 0.35 * ext[1], 0.9 * ext[2]))
        self.lungs = [((cx - 0.2 * ext[0], cy - 0.02 * ext[1], cz + 0.03 * ext[2]),
                       (0.15 * ext[0], 0.21 * ext[1], 0.42 * ext[2])),
                      ((cx + 0.2 * ext[0], cy - 0.02 * ext[1], cz + 0.03 * ext[2]),
                       (0.15 * ext[0], 0.21 * ext[1], 0.42 * ext[2]))]
        segs = []
        for v in range(300):
            lc, la = self.lungs[v % 2]
            # start inside the lung, wander as a smooth random polyline
            while True:
                p = np.asarray(lc) + r.uniform(-0.8, 0.8, 3) * np.asarray(la)
                if np.sum(((p - lc) / la) ** 2) < 0.6:
                    break
            d = r.normal(size=3)
            d /= np.linalg.norm(d)
            rad = r.uniform(0.5, 3.0)
            for s in range(6):
                d = d + 0.5 * r.normal(size=3)
                d /= np.linalg.norm(d)
                q = p + d * r.uniform(10.0, 20.0)
                segs.append((p.copy(), q.copy(), rad))
                p = q
        self.segs = segs

    def __call__(self, X, Y, Z, lo, hi):
        """Evaluate on warped coordinates; lo/hi bound (X, Y, Z) per axis."""
        w = 0.75
        v = -1000.0 + 1040.0 * _step(_ellipsoid_depth(X, Y, Z, *self.body), w)
        lung = 0.0
        for c, a in self.lungs:
            lung = lung + _step(_ellipsoid_depth(X, Y, Z, c, a), w)
        v = v - 890.0 * lung
        ves = torch.zeros_like(v)
        sel = [sg for sg in self.segs
               if not (np.any(np.maximum(sg[0], sg[1]) + sg[2] + 2.0 < lo) or
                       np.any(np.minimum(sg[0], sg[1]) - sg[2] - 2.0 > hi))]
        if sel:
            dev, dt = v.device, v.dtype
            P0 = torch.tensor(np.stack([sg[0] for sg in sel]), device=dev, dtype=dt)
            Dv = torch.tensor(np.stack([sg[1] - sg[0] for sg in sel]), device=dev, dtype=dt)
            rad = torch.tensor([sg[2] for sg in sel], device=dev, dtype=dt)
            L2 = (Dv * Dv).sum(1)
            Xe, Ye, Ze = X.unsqueeze(0), Y.unsqueeze(0), Z.unsqueeze(0)
            for c0 in range(0, len(sel), 32):  # segments in batches: one capsule distance each
                sl = slice(c0, c0 + 32)
                px, py, pz = (P0[sl, a].view(-1, 1, 1, 1) for a in range(3))
                dx, dy, dz = (Dv[sl, a].view(-1, 1, 1, 1) for a in range(3))
                t = (((Xe - px) * dx + (Ye - py) * dy + (Ze - pz) * dz) / L2[sl].view(-1, 1, 1, 1)).clamp(0.0, 1.0)
                dist = torch.sqrt((Xe - px - t * dx) ** 2 + (Ye - py - t * dy) ** 2 + (Ze - pz - t * dz) ** 2)
                ves = torch.maximum(ves, _step(rad[sl].view(-1, 1, 1, 1) - dist, 0.3).amax(0))
        v = v + 890.0 * ves * lung
        return v.clamp(-1000.0, 400.0)


def lung_pair(m=(256, 256, 120), h=(1.0, 1.0, 2.5), seed=10, device="cpu", noise=10.0, max_dz=15.0):
    """Lung-CT-shaped pair.  Seeds: seed (geometry), +1 (R noise), +2 (u*),
    +3 (T noise).  u*_z reaches max_dz mm and decays laterally; u*_x, u*_y
    are a few mm."""
    dtype = torch.float32
    ph = _Lung(m, h, seed)
    ext = ph.ext
    r = _rng(seed + 2)
    sx, sy = r.uniform(50, 80), r.uniform(45, 70)
    ax_, ay_ = r.uniform(1.0, 3.0, 2)
    ph_x, ph_y = r.uniform(0, 2 * math.pi, 2)
    cx, cy = ext[0] / 2, ext[1] / 2

    def field(X, Y, Z):
        lat = torch.exp(-((X - cx) ** 2) / (2 * sx * sx) - ((Y - cy) ** 2) / (2 * sy * sy))
        uz = max_dz * lat * torch.sin(math.pi * Z / ext[2])
        ux = ax_ * torch.sin(2 * math.pi * Y / ext[1] + ph_x) * torch.sin(math.pi * X / ext[0]) * torch.sin(math.pi * Z / ext[2])
        uy = ay_ * torch.sin(2 * math.pi * X / ext[0] + ph_y) * torch.sin(math.pi * Y / ext[1]) * torch.sin(math.pi * Z / ext[2])
        return ux, uy, uz

    M = m[0] * m[1] * m[2]
    R = torch.empty(M, dtype=dtype, device=device)
    T = torch.empty(M, dtype=dtype, device=device)
    U = torch.empty(3, M, dtype=dtype, device=device)
    plane = m[0] * m[1]
    for z0, z1 in _slabs(m[2], 8):
        X, Y, Z = _axes(m, h, z0, z1, device, dtype)
        shp = (z1 - z0, m[1], m[0])
        Xb, Yb, Zb = X.expand(shp), Y.expand(shp), Z.expand(shp)
        lo = np.array([0.0, 0.0, z0 * h[2]])
        hi = np.array([ext[0], ext[1], z1 * h[2]])
        R[z0 * plane:z1 * plane] = ph(Xb, Yb, Zb, lo, hi).reshape(-1)
        ux, uy, uz = (c.expand(shp) for c in field(X, Y, Z))
        marg = np.array([float(ux.abs().max()), float(uy.abs().max()), float(uz.abs().max())])
        T[z0 * plane:z1 * plane] = ph(Xb + ux, Yb + uy, Zb + uz, lo - marg, hi + marg).reshape(-1)
        U[0, z0 * plane:z1 * plane] = ux.reshape(-1)
        U[1, z0 * plane:z1 * plane] = uy.reshape(-1)
        U[2, z0 * plane:z1 * plane] = uz.reshape(-1)
    gR = torch.Generator(device="cpu").manual_seed(seed + 1)
    gT = torch.Generator(device="cpu").manual_seed(seed + 3)
    R += noise * torch.randn(M, generator=gR, dtype=dtype).to(device)
    T += noise * torch.randn(M, generator=gT, dtype=dtype).to(device)
    return R, T, U


def _lung_field(m, h, seed, max_dz):
    """Breathing displacement of lung_pair: (ux, uy, uz)(X, Y, Z) in mm."""
    ext = np.asarray(m, float) * np.asarray(h, float)
    r = _rng(seed + 2)
    sx, sy = r.uniform(50, 80), r.uniform(45, 70)
    ax_, ay_ = r.uniform(1.0, 3.0, 2)
    ph_x, ph_y = r.uniform(0, 2 * math.pi, 2)
    cx, cy = ext[0] / 2, ext[1] / 2

    def field(X, Y, Z):
        lat = torch.exp(-((X - cx) ** 2) / (2 * sx * sx) - ((Y - cy) ** 2) / (2 * sy * sy))
        uz = max_dz * lat * torch.sin(math.pi * Z / ext[2])
        ux = ax_ * torch.sin(2 * math.pi * Y / ext[1] + ph_x) * torch.sin(math.pi * X / ext[0]) * torch.sin(math.pi * Z / ext[2])
        uy = ay_ * torch.sin(2 * math.pi * X / ext[0] + ph_y) * torch.sin(math.pi * Y / ext[1]) * torch.sin(math.pi * Z / ext[2])
        return ux, uy, uz

    return field


def lung_pair_windowed(m, h, seed, device="cpu", noise=10.0, max_dz=15.0, chunk=256):
    """The lung_pair phantom and displacement, evaluated faster for many
    pairs: each vessel segment is evaluated only on the voxels of a box
    around it (R) or around its pre-image under the displacement (T: the
    box moved by -u* at the segment's centre and widened by the change of
    u* across it), and the vessel term takes the maximum over segments by
    a scatter.  Beyond the box a segment's smooth indicator is below 1e-3,
    so the noise-free pair differs from lung_pair's by a few hundredths of a
    HU; the noise comes from a generator on `device`.
    Returns R, T (float32, m_x m_y m_z) on `device`."""
    dtype = torch.float32
    ph = _Lung(m, h, seed)
    field = _lung_field(m, h, seed, max_dz)
    hh = torch.tensor(h, dtype=dtype, device=device)
    mm = torch.tensor(m, device=device)
    X, Y, Z = _axes(m, h, 0, m[2], device, dtype)
    shp = (m[2], m[1], m[0])
    Xb, Yb, Zb = X.expand(shp), Y.expand(shp), Z.expand(shp)
    ux, uy, uz = (c.expand(shp) for c in field(X, Y, Z))
    w = 0.75

    def base(Xq, Yq, Zq):
        v = -1000.0 + 1040.0 * _step(_ellipsoid_depth(Xq, Yq, Zq, *ph.body), w)
        lung = 0.0
        for c, a in ph.lungs:
            lung = lung + _step(_ellipsoid_depth(Xq, Yq, Zq, c, a), w)
        return v - 890.0 * lung, lung

    P0 = torch.tensor(np.stack([sg[0] for sg in ph.segs]), dtype=dtype, device=device)
    P1 = torch.tensor(np.stack([sg[1] for sg in ph.segs]), dtype=dtype, device=device)
    rad = torch.tensor([sg[2] for sg in ph.segs], dtype=dtype, device=device)
    lo_mm = torch.minimum(P0, P1) - rad[:, None] - 2.0
    hi_mm = torch.maximum(P0, P1) + rad[:, None] + 2.0
    ctr = 0.5 * (P0 + P1)
    cu = torch.stack(field(ctr[:, 0], ctr[:, 1], ctr[:, 2]), dim=1)
    # u* changes by at most |grad u*| * half the box across it: widen the T box by that
    span = 0.5 * (hi_mm - lo_mm).max(dim=1).values
    gmax = max_dz * (1.0 / 50.0 + math.pi / (m[2] * h[2])) + 6.0 * math.pi / min(m[0] * h[0], m[1] * h[1])
    marg = (gmax * span)[:, None] + 1.0

    def vessels(lo, hi, warped):
        i0 = torch.floor(lo / hh - 0.5).to(torch.int64)
        i1 = torch.ceil(hi / hh - 0.5).to(torch.int64)
        size = (i1 - i0 + 1).max(dim=0).values.tolist()
        ar = [torch.arange(size[a], device=device) for a in range(3)]
        off = torch.stack(torch.meshgrid(ar[2], ar[1], ar[0], indexing="ij"), dim=-1).reshape(-1, 3).flip(-1)
        ves = torch.zeros(m[0] * m[1] * m[2], dtype=dtype, device=device)
        for c0 in range(0, len(rad), chunk):
            sl = slice(c0, c0 + chunk)
            idx = i0[sl, None, :] + off[None]                        # [S, V, 3] voxel (x, y, z)
            ok = ((idx >= 0) & (idx < mm)).all(-1)
            idx = torch.minimum(torch.maximum(idx, torch.zeros_like(mm)), mm - 1)
            flat = (idx[..., 2] * m[1] + idx[..., 1]) * m[0] + idx[..., 0]
            q = (idx.to(dtype) + 0.5) * hh
            if warped:
                q = q + torch.stack([ux.reshape(-1)[flat], uy.reshape(-1)[flat], uz.reshape(-1)[flat]], dim=-1)
            d = (P1 - P0)[sl, None, :]
            t = (((q - P0[sl, None, :]) * d).sum(-1) / (d * d).sum(-1)).clamp(0.0, 1.0)
            dist = torch.linalg.vector_norm(q - P0[sl, None, :] - t[..., None] * d, dim=-1)
            val = torch.where(ok, _step(rad[sl, None] - dist, 0.3), torch.zeros_like(dist))
            ves.scatter_reduce_(0, flat.reshape(-1), val.reshape(-1), reduce="amax")
        return ves.reshape(shp)

    vR, lR = base(Xb, Yb, Zb)
    R = (vR + 890.0 * vessels(lo_mm, hi_mm, False) * lR).clamp(-1000.0, 400.0).reshape(-1)
    vT, lT = base(Xb + ux, Yb + uy, Zb + uz)
    T = (vT + 890.0 * vessels(lo_mm - cu - marg, hi_mm - cu + marg, True) * lT).clamp(-1000.0, 400.0).reshape(-1)
    M = m[0] * m[1] * m[2]
    # noise drawn by a generator on the device itself (seeded, so each pair
    # is reproducible on a given device type)
    gR = torch.Generator(device=device).manual_seed(seed + 1)
    gT = torch.Generator(device=device).manual_seed(seed + 3)
    R = R + noise * torch.randn(M, generator=gR, dtype=dtype, device=device)
    T = T + noise * torch.randn(M, generator=gT, dtype=dtype, device=device)
    return R, T


# ------------------------------------------------------------------ thorax-abdomen


class _Thorax:
    def __init__(self, m, h):
        ext = np.asarray(m, float) * np.asarray(h, float)
        self.ext = ext
        cx, cy = ext[0] / 2, ext[1] / 2
        Lz = ext[2]
        self.body = (cx, cy, 0.45 * ext[0], 0.33 * ext[1])
        self.objs = [  # (centre, semi-axes, HU relative to soft tissue)
            ((cx - 0.18 * ext[0], cy - 0.02 * ext[1], 0.80 * Lz), (0.15 * ext[0], 0.2 * ext[1], 0.19 * Lz), -890.0),
            ((cx + 0.18 * ext[0], cy - 0.02 * ext[1], 0.80 * Lz), (0.15 * ext[0], 0.2 * ext[1], 0.19 * Lz), -890.0),
            ((cx - 0.13 * ext[0], cy - 0.03 * ext[1], 0.52 * Lz), (0.23 * ext[0], 0.18 * ext[1], 0.10 * Lz), 20.0),
            ((cx - 0.17 * ext[0], cy + 0.14 * ext[1], 0.40 * Lz), (0.07 * ext[0], 0.07 * ext[1], 0.06 * Lz), -10.0),
            ((cx + 0.17 * ext[0], cy + 0.14 * ext[1], 0.40 * Lz), (0.07 * ext[0], 0.07 * ext[1], 0.06 * Lz), -10.0),
            ((cx + 0.21 * ext[0], cy + 0.06 * ext[1], 0.53 * Lz), (0.10 * ext[0], 0.085 * ext[1], 0.07 * Lz), 10.0),
        ]
        self.spine = (cx, cy + 0.22 * ext[1], 0.055 * ext[0])

    def __call__(self, X, Y, Z):
        w = 0.75
        bx, by, ax, ay = self.body
        q = torch.sqrt(((X - bx) / ax) ** 2 + ((Y - by) / ay) ** 2)
        v = -1000.0 + 1040.0 * _step((1.0 - q) * min(ax, ay), w)
        for c, a, dv in self.objs:
            v = v + dv * _step(_ellipsoid_depth(X, Y, Z, c, a), w)
        sx, sy, sr = self.spine
        rr = torch.sqrt((X - sx) ** 2 + (Y - sy) ** 2)
        vert = 0.5 + 0.5 * torch.cos(2 * math.pi * Z / 30.0)  # vertebrae along z
        bone = _step(sr - rr, w)
        cortex = _step(rr - 0.7 * sr, w) * bone
        v = v + bone * (660.0 + 200.0 * vert) + cortex * 600.0
        return v.clamp(-1000.0, 1500.0)


def thorax_pair(m=(512, 512, 900), h=(0.8, 0.8, 1.0), seed=20, device="cpu", noise=20.0, max_disp=20.0,
                zrange=None):
    """Thorax-abdomen-shaped pair.  Seeds: +1 (R noise), +2 (u*: 8 Fourier
    modes, scaled to max |u*| = max_disp mm), +3 (T noise).  zrange = (z0, z1)
    evaluates only those image planes of the same phantom and displacement
    (the noise is drawn for the slab alone)."""
    dtype = torch.float32
    ph = _Thorax(m, h)
    ext = ph.ext
    r = _rng(seed + 2)
    freq = r.integers(0, 3, size=(8, 3))
    freq[np.all(freq == 0, axis=1), 0] = 1
    amp = r.normal(size=(8, 3))
    phase = r.uniform(0, 2 * math.pi, size=(8, 3))

    def field(X, Y, Z):
        out = []
        for d in range(3):
            acc = 0.0
            for k in range(8):
                arg = 2 * math.pi * (freq[k, 0] * X / ext[0] + freq[k, 1] * Y / ext[1] + freq[k, 2] * Z / ext[2])
                acc = acc + amp[k, d] * torch.sin(arg / 2 + phase[k, d])
            out.append(acc)
        return out

    # scale from the maximum norm over a coarse sample of the grid
    Xs, Ys, Zs = _axes(m, h, 0, m[2], "cpu", torch.float64)
    f = field(Xs[:, :, ::8], Ys[:, ::8, :], Zs[::8])
    scale = max_disp / float(torch.sqrt(f[0] ** 2 + f[1] ** 2 + f[2] ** 2).max())
    za, zb = (0, m[2]) if zrange is None else zrange
    M = m[0] * m[1] * (zb - za)
    R = torch.empty(M, dtype=dtype, device=device)
    T = torch.empty(M, dtype=dtype, device=device)
    U = torch.empty(3, M, dtype=dtype, device=device)
    plane = m[0] * m[1]
    for z0, z1 in _slabs(zb - za, 16):
        X, Y, Z = _axes(m, h, za + z0, za + z1, device, dtype)
        shp = (z1 - z0, m[1], m[0])
        u = [(c * scale).expand(shp) for c in field(X, Y, Z)]
        R[z0 * plane:z1 * plane] = ph(X.expand(shp), Y.expand(shp), Z.expand(shp)).reshape(-1)
        T[z0 * plane:z1 * plane] = ph(X + u[0], Y + u[1], Z + u[2]).reshape(-1)
        for d in range(3):
            U[d, z0 * plane:z1 * plane] = u[d].reshape(-1)
    gR = torch.Generator(device="cpu").manual_seed(seed + 1)
    gT = torch.Generator(device="cpu").manual_seed(seed + 3)
    for z0, z1 in _slabs(zb - za, 64):
        sl = slice(z0 * plane, z1 * plane)
        R[sl] += noise * torch.randn(sl.stop - sl.start, generator=gR, dtype=dtype).to(device)
        T[sl] += noise * torch.randn(sl.stop - sl.start, generator=gT, dtype=dtype).to(device)
    return R, T, U


def tissue_pair_2d(m, h=(1.0, 1.0), seed=50, device="cpu", blobs=None, max_disp_px=None, noise=0.02):
    """2-D pair (one image plane) standing in for the paper's histological
    serial sections: a smooth background and many small Gaussian "nuclei"
    (about one per 400 pixels, sigma 1.5-4 pixels, amplitude U[0.3, 1]),
    evaluated at the pixel centres (R) and at x + u*(x) (T) with u* a sum of
    6 low-frequency sines scaled to max_disp_px (default m0 / 64 pixels),
    plus noise sd `noise`.  Each nucleus is evaluated on a window of pixels
    (4 sigma around it for R; around its pre-image under u*, widened by the
    change of u* across the window, for T) and added by a scatter.  Seeds:
    seed (blobs), +1 (R noise), +2 (u*), +3 (T noise).  Returns R, T as
    float32 of length m0 m1."""
    r = _rng(seed)
    ext = np.asarray(m[:2], float) * np.asarray(h[:2], float)
    nb = blobs if blobs is not None else max(8, (m[0] * m[1]) // 400)
    c = r.uniform(0.0, 1.0, size=(nb, 2)) * ext
    sig = r.uniform(1.5, 4.0, size=nb) * min(h[:2])
    amp = r.uniform(0.3, 1.0, size=nb)
    rd = _rng(seed + 2)
    freq = rd.integers(0, 3, size=(6, 2))
    freq[np.all(freq == 0, axis=1), 0] = 1
    famp = rd.normal(size=(6, 2))
    phase = rd.uniform(0, 2 * math.pi, size=(6, 2))
    md = (max_disp_px if max_disp_px is not None else m[0] / 64.0) * min(h[:2])
    dtype = torch.float32

    def field(X, Y):
        out = []
        for d in range(2):
            acc = torch.zeros_like(X)
            for k in range(6):
                acc = acc + famp[k, d] * torch.sin(math.pi * (freq[k, 0] * X / ext[0] + freq[k, 1] * Y / ext[1])
                                                   + phase[k, d])
            out.append(acc)
        return out

    Xs = torch.linspace(0, ext[0], 65, dtype=torch.float64).view(1, -1).expand(65, 65)
    Ys = torch.linspace(0, ext[1], 65, dtype=torch.float64).view(-1, 1).expand(65, 65)
    fs = field(Xs, Ys)
    scale = md / float(torch.sqrt(fs[0] ** 2 + fs[1] ** 2).max())
    M = m[0] * m[1]
    x = ((torch.arange(m[0], device=device, dtype=dtype) + 0.5) * h[0]).view(1, -1).expand(m[1], m[0])
    y = ((torch.arange(m[1], device=device, dtype=dtype) + 0.5) * h[1]).view(-1, 1).expand(m[1], m[0])
    ux, uy = (scale * f for f in field(x, y))
    # bound of |grad u*| (pixels per pixel) from the frequencies
    gmax = scale * float(np.abs(famp).sum(0).max()) * math.pi * 2.0 / float(min(ext)) * 2.0

    def render(warped):
        v = 0.2 + 0.1 * torch.sin(2 * math.pi * ((x + ux) if warped else x) / ext[0]) * \
            torch.cos(2 * math.pi * ((y + uy) if warped else y) / ext[1])
        v = v.reshape(-1).clone()
        cb = torch.tensor(c, dtype=dtype, device=device)
        if warped:  # pre-image of each centre under x -> x + u*(x)
            cu = torch.stack(field(cb[:, 0:1].double().cpu(), cb[:, 1:2].double().cpu()), dim=1).view(-1, 2)
            cb = cb - (scale * cu).to(device=device, dtype=dtype)
        rad = 4.0 * float(sig.max())
        half = int(math.ceil((rad + (gmax * rad + 1.0 if warped else 0.0)) / min(h[:2]))) + 1
        off = torch.arange(-half, half + 1, device=device)
        oy, ox = torch.meshgrid(off, off, indexing="ij")
        ox, oy = ox.reshape(1, -1), oy.reshape(1, -1)
        sb = torch.tensor(sig, dtype=dtype, device=device).view(-1, 1)
        ab = torch.tensor(amp, dtype=dtype, device=device).view(-1, 1)
        c0 = torch.tensor(c, dtype=dtype, device=device)
        for k0 in range(0, nb, 2048):
            sl = slice(k0, k0 + 2048)
            px = torch.floor(cb[sl, 0:1] / h[0]).long() + ox
            py = torch.floor(cb[sl, 1:2] / h[1]).long() + oy
            ok = (px >= 0) & (px < m[0]) & (py >= 0) & (py < m[1])
            pxc, pyc = px.clamp(0, m[0] - 1), py.clamp(0, m[1] - 1)
            flat = pyc * m[0] + pxc
            X = (pxc.to(dtype) + 0.5) * h[0]
            Y = (pyc.to(dtype) + 0.5) * h[1]
            if warped:
                X = X + ux.reshape(-1)[flat]
                Y = Y + uy.reshape(-1)[flat]
            d2 = (X - c0[sl, 0:1]) ** 2 + (Y - c0[sl, 1:2]) ** 2
            g = ab[sl] * torch.exp(-d2 / (2 * sb[sl] ** 2)) * ok
            v.index_add_(0, flat.reshape(-1), g.reshape(-1))
        return v

    R = render(False)
    T = render(True)
    gR = torch.Generator(device="cpu").manual_seed(seed + 1)
    gT = torch.Generator(device="cpu").manual_seed(seed + 3)
    R += noise * torch.randn(M, generator=gR, dtype=dtype).to(device)
    T += noise * torch.randn(M, generator=gT, dtype=dtype).to(device)
    return R, T


def make(workload, device="cpu"):
    """(R, T, u_true, desc) for a named workload; R, T are float32 of length
    m_x m_y m_z on `device`, u_true is 3 x M (image grid, mm)."""
    w = dict(WORKLOADS[workload])
    if workload == "blobs_32":
        R, T, U = blob_pair(w["m"], w["h"], seed=w["seed"], device=device)
    elif workload == "lung_ct":
        R, T, U = lung_pair(w["m"], w["h"], seed=w["seed"], device=device)
    elif workload == "thorax_abd":
        R, T, U = thorax_pair(w["m"], w["h"], seed=w["seed"], device=device)
    else:
        raise KeyError(workload)
    return R, T, U, w


def batch_pairs(count=64, lo=64, hi=192, seed=30, device="cpu"):
    """`count` blob pairs of cubic size N ~ U{lo..hi} (numpy PCG64, `seed`);
    pair k uses blob seeds 1000 + 4k ... 1000 + 4k + 3.  Returns a list of
    (R, T, workload dict) with nodes N//2 + 1 per axis (two voxels per cell)."""
    sizes = _rng(seed).integers(lo, hi + 1, size=count)
    out = []
    for k, N in enumerate(sizes):
        N = int(N)
        m = (N, N, N)
        R, T, _ = blob_pair(m, (1.0, 1.0, 1.0), seed=1000 + 4 * k, device=device)
        out.append((R, T, dict(m=m, h=(1.0, 1.0, 1.0), n=(N // 2 + 1,) * 3, alpha=1.0, tau=0.1, rho=0.1,
                               levels=2)))
    return out


def smooth_nodal_field(n, hy, seed, max_disp, modes=6, device="cpu"):
    """Smooth displacement on the node grid (n nodes per axis at spacing hy,
    node j at j * hy): per component a sum of `modes` low-frequency sines
    (numpy PCG64, `seed`), scaled so that the largest |u| over the nodes is
    max_disp (units of hy).  3 * prod(n) float32, component-major."""
    r = _rng(seed)
    freq = r.integers(0, 3, size=(modes, 3))
    freq[np.all(freq == 0, axis=1), 0] = 1
    amp = r.normal(size=(modes, 3))
    phase = r.uniform(0, 2 * math.pi, size=(modes, 3))
    ext = [(n[a] - 1) * hy[a] for a in range(3)]
    X, Y, Z = (((torch.arange(n[a], dtype=torch.float64) * hy[a]) / ext[a]) for a in range(3))
    X, Y, Z = X.view(1, 1, -1), Y.view(1, -1, 1), Z.view(-1, 1, 1)
    comps = []
    for d in range(3):
        acc = torch.zeros(n[2], n[1], n[0], dtype=torch.float64)
        for k in range(modes):
            acc = acc + amp[k, d] * torch.sin(math.pi * (freq[k, 0] * X + freq[k, 1] * Y + freq[k, 2] * Z)
                                              + phase[k, d])
        comps.append(acc.reshape(-1))
    U = torch.stack(comps)
    U = U * (max_disp / float(torch.sqrt((U ** 2).sum(0)).max()))
    return U.reshape(-1).to(torch.float32).to(device)


def random_fields(n_nodes, seed, amp=0.3, device="cpu"):
    """Seeded nodal displacement u (amplitude amp, same units as h) and
    direction p, both 3 * n_nodes float32, for operator-level tests."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    u = amp * torch.randn(3 * n_nodes, generator=g, dtype=torch.float32)
    p = torch.randn(3 * n_nodes, generator=g, dtype=torch.float32)
    return u.to(device), p.to(device)
