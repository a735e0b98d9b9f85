// Kernel bodies of libngf_b300 (declarations and shared-memory layouts are in
// ngf_kernels.cuh).
#include "ngf_kernels.cuh"

#include <climits>

namespace ngf {

// position of ring element k of the (TX+2h) x (TY+2h) region minus the TX x TY core
__device__ __forceinline__ void ring_coord(int k, int halo, int& lx, int& ly) {
    const int W = TX + 2 * halo;
    const int band = halo * W;
    if (k < band) {
        ly = -halo + k / W;
        lx = -halo + k % W;
    } else if (k < 2 * band) {
        k -= band;
        ly = TY + k / W;
        lx = -halo + k % W;
    } else {
        k -= 2 * band;
        const int per = 2 * halo;
        ly = k / per;
        const int c = k % per;
        lx = (c < halo) ? (-halo + c) : (TX + c - halo);
    }
}

// Block-wide float64 sum in a fixed order (all threads see the result):
// shuffle trees within the warps, then over the warp sums in warp 0; two
// barriers instead of one per tree level.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // red may still be read by a previous call
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = (lane < NT / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = NT / 64; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[NT / 32] = t;
    }
    __syncthreads();
    return red[NT / 32];
}

// Deterministic grid-wide float64 sum: each CTA stores its partial, the last
// CTA to finish adds all partials in CTA order.  `scale` multiplies the result.
__device__ __forceinline__ void grid_sum_finish(double blocksum, double* part, unsigned int* count,
                                                double* out, double scale, double* red, int nblocks,
                                                int bid) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        part[bid] = blocksum;
        __threadfence();
        const unsigned int ticket = atomicAdd(count, 1u);
        is_last = (ticket == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += ((volatile double*)part)[i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            *out = red[0] * scale;
            *count = 0u;
        }
    }
}

// Trilinear sample of T at continuous voxel coordinate (g + d) per axis, zero
// outside; returns the value and dT/dx_l in physical units.  The cell is
// floor(d) relative to g (displacement form), so exact knots take the forward
// cell and an identity warp reproduces T exactly.  Voxel counts are < 2^31
// (checked at plan creation), so offsets are 32-bit.
__device__ __forceinline__ float warp_sample(const ImgParams& P, int gx, int gy, int gz, float d0, float d1,
                                             float d2, float& g0, float& g1, float& g2) {
    g0 = g1 = g2 = 0.f;
    if (!(fabsf(d0) < 1.0e9f) || !(fabsf(d1) < 1.0e9f) || !(fabsf(d2) < 1.0e9f)) return 0.f;
    const float f0 = floorf(d0), f1 = floorf(d1), f2 = floorf(d2);
    const int cx = gx + (int)f0, cy = gy + (int)f1, cz = gz + (int)f2;
    if (cx < -1 || cx > P.m0 - 1 || cy < -1 || cy > P.m1 - 1 || cz < -1 || cz > P.m2 - 1) return 0.f;
    const float tx = d0 - f0, ty = d1 - f1, tz = d2 - f2;
    const int sy = P.m0, sz = P.m0 * P.m1;
    float v000, v100, v010, v110, v001, v101, v011, v111;
    if (cx >= 0 && cx + 1 < P.m0 && cy >= 0 && cy + 1 < P.m1 && cz >= 0 && cz + 1 < P.m2) {
        const float* t = P.T + (cx + sy * cy + sz * cz);  // all eight corners inside
        v000 = __ldg(t);
        v100 = __ldg(t + 1);
        v010 = __ldg(t + sy);
        v110 = __ldg(t + sy + 1);
        v001 = __ldg(t + sz);
        v101 = __ldg(t + sz + 1);
        v011 = __ldg(t + sz + sy);
        v111 = __ldg(t + sz + sy + 1);
    } else {
        const bool x0ok = cx >= 0, x1ok = cx + 1 <= P.m0 - 1;
        const bool y0ok = cy >= 0, y1ok = cy + 1 <= P.m1 - 1;
        const bool z0ok = cz >= 0, z1ok = cz + 1 <= P.m2 - 1;
        const int xa = max(cx, 0), xb = min(cx + 1, P.m0 - 1);
        const int ya = max(cy, 0) * sy, yb = min(cy + 1, P.m1 - 1) * sy;
        const int za = max(cz, 0) * sz, zb = min(cz + 1, P.m2 - 1) * sz;
        const float* T = P.T;
        v000 = (x0ok && y0ok && z0ok) ? __ldg(T + xa + ya + za) : 0.f;
        v100 = (x1ok && y0ok && z0ok) ? __ldg(T + xb + ya + za) : 0.f;
        v010 = (x0ok && y1ok && z0ok) ? __ldg(T + xa + yb + za) : 0.f;
        v110 = (x1ok && y1ok && z0ok) ? __ldg(T + xb + yb + za) : 0.f;
        v001 = (x0ok && y0ok && z1ok) ? __ldg(T + xa + ya + zb) : 0.f;
        v101 = (x1ok && y0ok && z1ok) ? __ldg(T + xb + ya + zb) : 0.f;
        v011 = (x0ok && y1ok && z1ok) ? __ldg(T + xa + yb + zb) : 0.f;
        v111 = (x1ok && y1ok && z1ok) ? __ldg(T + xb + yb + zb) : 0.f;
    }
    // lerp along x on the four (y,z) edges
    const float e00 = fmaf(tx, v100 - v000, v000);
    const float e10 = fmaf(tx, v110 - v010, v010);
    const float e01 = fmaf(tx, v101 - v001, v001);
    const float e11 = fmaf(tx, v111 - v011, v011);
    const float a0 = fmaf(ty, e10 - e00, e00);
    const float a1 = fmaf(ty, e11 - e01, e01);
    // x derivative: bilinear (y,z) blend of the x differences
    const float q0 = fmaf(ty, (v110 - v010) - (v100 - v000), v100 - v000);
    const float q1 = fmaf(ty, (v111 - v011) - (v101 - v001), v101 - v001);
    g0 = fmaf(tz, q1 - q0, q0) * P.ih[0];
    g1 = fmaf(tz, (e11 - e01) - (e10 - e00), e10 - e00) * P.ih[1];
    g2 = (a1 - a0) * P.ih[2];  // a planar level has ih[2] = 0: d2 = 0 and no z derivative
    return fmaf(tz, a1 - a0, a0);
}

// ---------------------------------------------------------------------------
// The fused image pass.
//   MODE_OBJ : D = hbar sum (1 - r_i^2)                       (Eq. NGF_discretized)
//   MODE_GRAD: D and the tile partials of P^T[dT (dr^T(-2 hbar r))]   (Eq. gradNGF)
//   MODE_HESS: tile partials of P^T[2 hbar dT dr^T dr (dT . P p)]       (Eq. hessMult)
// The transposed grid conversion is completed by k_node_combine.
//
// A CTA owns the residual rows i of its TX x TY column tile and z-chunk: it
// forms rho_hat_i and w_i = r_i (gradient) or (dr s)_i (Hessian) for those
// rows only, and scatters each row's products pi_i(k) = rho_hat_i(k) w_i to
// the columns j = i + k of dr^T, which lie in the tile or on the face ring
// just outside it (and on the planes just below and above the chunk).  The
// tile's partial holds q_hat_j = qscale dT_j t_j for all those columns, with
// t_j the sum over the tile's own rows; the neighbouring tiles add the rest
// of t_j through their own partials, since P^T is linear.  So the front end
// (warp, dT, s) runs on the halo-1 region only (own columns and face ring,
// no corners) and no residual Jacobian row is evaluated twice.
//
// One barrier per plane.  Every stage of a plane interval reads only what
// earlier intervals wrote, so the buffer between two stages is a ring one
// plane deeper than their distance (plane indices relative to the march
// variable zf):
//   S0(zf+1): node values of u (and p) interpolated in z to plane zf+1;
//   S1(zf)  : warp T and dT (and s = dT . P p) on the own columns and the
//             face ring, first in the interval;
//   S2(zf-2): residual Jacobian row rho_hat (Eqs. rho, hatRho) of the own
//             rows and the products pi_i(k): in-plane ones to shared memory,
//             pi(0) and pi(+-z) in registers;
//   S3(zf-3): t_j = sum_k pi_{j+k}(-k) over the tile's own rows that are
//             true neighbours of j (column j of dr^T), q_hat = qscale dT_j t_j
//             on the halo-1 region; pi(-z) of plane zf-2 comes from this
//             interval's S2 of the same column;
//   A(zf-4) : x-reduction of q_hat onto node columns (separable P^T);
//   B(zf-5) : y-reduction and accumulation into two live node planes; a
//             completed node plane is stored as this tile's partial.
// Besides its own column a thread may carry optional work: the front end of
// the face ring sits on the last RINGF threads, the ring's S3 on the first
// RINGF, and the A, B and S0 items follow one another from thread RINGF on.
// ---------------------------------------------------------------------------
// position of face-ring column k of the halo-1 region: the row below and
// above the tile, then the column left and right of it
__device__ __forceinline__ void ring_face(int k, int& lx, int& ly) {
    if (k < 2 * TX) {
        lx = k & (TX - 1);
        ly = (k < TX) ? -1 : TY;
    } else {
        k -= 2 * TX;
        ly = k % TY;
        lx = (k < TY) ? -1 : TX;
    }
}

template <int MODE, class SM>
__device__ __forceinline__ void image_pass(const ImgParams& P, int bx, int by, int bz) {
    NGF_DYNAMIC_SMEM(smraw);
    SM& S = *reinterpret_cast<SM*>(smraw);
    constexpr int SNBX = SM::kNBX, SNBY = SM::kNBY;
    constexpr bool OBJ = (MODE == MODE_OBJ), HESS = (MODE == MODE_HESS);
    constexpr int NVEC = HESS ? 6 : 3;
    const int tid = threadIdx.x;
    const int xs = bx * TX, ys = by * TY;
    const int z0 = bz * P.zc, z1 = min(P.m2, z0 + P.zc);
    const int txe = min(TX, P.m0 - xs), tye = min(TY, P.m1 - ys);

    // node box of the halo-1 region: z-interpolated node planes and partials
    const int BX0 = P.fx[max(xs - 1, 0)], BY0 = P.fy[max(ys - 1, 0)], BZ0 = P.fz[max(z0 - 1, 0)];
    const int nbx = P.fx[min(xs + TX, P.m0 - 1)] + 1 - BX0 + 1;
    const int nby = P.fy[min(ys + TY, P.m1 - 1)] + 1 - BY0 + 1;
    const long long tile = ((long long)bz * P.nty + by) * P.ntx + bx;

    for (int i = tid; i < SX1; i += NT) {
        const int gx = min(max(xs - 1 + i, 0), P.m0 - 1);
        S.fx1[i] = P.fx[gx] - BX0;
        S.wx1[i] = P.wx[gx];
    }
    for (int i = tid; i < SY1; i += NT) {
        const int gy = min(max(ys - 1 + i, 0), P.m1 - 1);
        S.fy1[i] = P.fy[gy] - BY0;
        S.wy1[i] = P.wy[gy];
    }
    if (!OBJ) {
        for (int i = tid; i < 2 * 3 * SNBY * SNBX; i += NT) (&S.Acc[0][0][0][0])[i] = 0.f;
        // S3 writes every q_hat entry of the region but its four corners
        if (tid < 2 * 4) {
            const int c = tid & 3;
            const int l = ((c >> 1) ? (SY1 - 1) * SX1 : 0) + ((c & 1) ? SX1 - 1 : 0);
            *reinterpret_cast<float4*>(S.Q4[tid >> 2][l]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();  // node floors of the region in shared memory
        // halo-1 columns (in the image) reduced onto each node column / row
        for (int b = tid; b < nbx; b += NT) {
            int lo = SX1, hi = -1;
            for (int l = max(0, 1 - xs); l < min(SX1, P.m0 - xs + 1); ++l) {
                const int f = S.fx1[l];
                if (f == b || f == b - 1) { lo = min(lo, l); hi = max(hi, l); }
            }
            S.xr_lo[b] = lo;
            S.xr_hi[b] = hi;
        }
        for (int b = tid; b < nby; b += NT) {
            int lo = SY1, hi = -1;
            for (int l = max(0, 1 - ys); l < min(SY1, P.m1 - ys + 1); ++l) {
                const int f = S.fy1[l];
                if (f == b || f == b - 1) { lo = min(lo, l); hi = max(hi, l); }
            }
            S.yr_lo[b] = lo;
            S.yr_hi[b] = hi;
        }
    }

    // ---- per-thread work descriptors, fixed for the whole march
    const int lx0 = tid % TX, ly0 = tid / TX;  // owned column
    const int gx0 = xs + lx0, gy0 = ys + ly0;
    const bool own_ok = (lx0 < txe) && (ly0 < tye);
    const int box = nbx * nby;  // S0 items: node columns of the box
    const int nA = OBJ ? 0 : SY1 * nbx, nB = OBJ ? 0 : nby * nbx;
    // The A, B and S0 items form one sequence dealt out to thread positions:
    // first the threads without ring work, then those with the ring's cheap
    // S3; the threads with a second front-end column (the ring's S1) take
    // items only when the layout's items exceed two per other thread.
    constexpr bool FEW_ITEMS = SY1 * SNBX + 2 * SNBY * SNBX <= 2 * (NT - RINGF);
    constexpr int W = FEW_ITEMS ? NT - RINGF : NT;
    const int pos = !FEW_ITEMS ? tid : (tid >= NT - RINGF ? -1 : (tid >= RINGF ? tid - RINGF : tid + NT - 2 * RINGF));
    const int offA = 0, offB = nA % W, offS = (nA + nB) % W;
    // S0 items (<= 2 per thread) as (global node column, Uz offset); A items
    // (row of the halo-1 region, bx) and B items (by, bx) packed as row*64 + col
    int s0_g[2], s0_s[2], a_it[2], b_it[2];
    for (int k = 0; k < 2; ++k) {
        const int i = pos < 0 ? INT_MAX : (pos + W - offS) % W + k * W;
        if (i < box) {
            const int yy = i / nbx, xx = i - yy * nbx;
            s0_g[k] = (BX0 + xx) + P.n0 * (BY0 + yy);
            s0_s[k] = yy * SNBX + xx;
        } else {
            s0_g[k] = 0;
            s0_s[k] = -1;
        }
        const int ia = pos < 0 ? INT_MAX : (pos + W - offA) % W + k * W;
        const int ib = pos < 0 ? INT_MAX : (pos + W - offB) % W + k * W;
        a_it[k] = (ia < nA) ? ((ia / nbx) << 6) + (ia % nbx) : -1;
        b_it[k] = (ib < nB) ? ((ib / nbx) << 6) + (ib % nbx) : -1;
    }
    const int plane_n = P.n0 * P.n1;
    __syncthreads();

    // register queues of the owned column
    float dq0[3] = {0.f, 0.f, 0.f}, dq1[3] = {0.f, 0.f, 0.f}, dq2[3] = {0.f, 0.f, 0.f},
          dq3[3] = {0.f, 0.f, 0.f};  // dT of the last four front-end planes
    float pm_c = 0.f, p0_c = 0.f, pp_c = 0.f;        // pi(-z), pi(0), pi(+z) of plane zf-2
    float p0_prev = 0.f, pp_prev = 0.f, pp_prev2 = 0.f;
    double dacc = 0.0;
    int cur = BZ0;  // lower live node plane of the P^T accumulators

    const int zbeg = z0 - 1;
    const int fe_last = z1;                   // last front-end plane needed
    const int zend = OBJ ? z1 + 1 : z1 + 5;   // S2 (objective) or B of the plane above the chunk

    // S0: node values of plane zf interpolated in z into Uz[zf & 1]
    auto stage0 = [&](int zf) {
        const int fzz = P.fz[zf];
        const float wzz = P.wz[zf];
        const int pl0 = fzz * plane_n;
        float* uz = &S.Uz[zf & 1][0][0][0];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (s0_s[k] < 0) continue;
            const int o = pl0 + s0_g[k];
#pragma unroll
            for (int c = 0; c < NVEC; ++c) {
                const float* src = (c < 3) ? (P.u + c * P.N) : (P.p + (c - 3) * P.N);
                const float a = __ldg(src + o), b = __ldg(src + o + P.znext);
                uz[c * (SNBY * SNBX) + s0_s[k]] = fmaf(wzz, b - a, a);
            }
        }
    };
    // S1 on one column of plane zf; returns dT
    auto stage1 = [&](int lx, int ly, int zf, float& g0, float& g1, float& g2) {
        const int gx = xs + lx, gy = ys + ly;
        const int li = (ly + 1) * SX1 + (lx + 1);
        const int ax = S.fx1[lx + 1], ay = S.fy1[ly + 1];
        const float wxv = S.wx1[lx + 1], wyv = S.wy1[ly + 1];
        const int uzs = zf & 1;
        float uh[NVEC];
#pragma unroll
        for (int c = 0; c < NVEC; ++c) {
            const float v00 = S.Uz[uzs][c][ay][ax], v10 = S.Uz[uzs][c][ay][ax + 1];
            const float v01 = S.Uz[uzs][c][ay + 1][ax], v11 = S.Uz[uzs][c][ay + 1][ax + 1];
            const float a0 = fmaf(wxv, v10 - v00, v00), a1 = fmaf(wxv, v11 - v01, v01);
            uh[c] = fmaf(wyv, a1 - a0, a0);
        }
        const float tw = warp_sample(P, gx, gy, zf, uh[0] * P.ih[0], uh[1] * P.ih[1], uh[2] * P.ih[2], g0, g1, g2);
        const int slot = zf & 3;
        S.R[slot][li] = __ldg(P.R + (gx + P.m0 * (gy + P.m1 * zf)));
        S.Tw[slot][li] = tw;
        if (HESS) S.S[slot][li] = fmaf(g0, uh[NVEC - 3], fmaf(g1, uh[NVEC - 2], g2 * uh[NVEC - 1]));
    };
    // S1 of plane zf: the own column, then (last threads) a face-ring column
    auto front_end = [&](int zf) {
        if (gx0 < P.m0 && gy0 < P.m1) stage1(lx0, ly0, zf, dq0[0], dq0[1], dq0[2]);
        if (tid >= NT - RINGF) {
            const int k = tid - (NT - RINGF);
            int lx, ly;
            ring_face(k, lx, ly);
            const int gx = xs + lx, gy = ys + ly;
            if (gx >= 0 && gx < P.m0 && gy >= 0 && gy < P.m1) {
                float g0, g1, g2;
                stage1(lx, ly, zf, g0, g1, g2);
                if (!OBJ) {
                    S.DTr[zf & 3][0][k] = g0;
                    S.DTr[zf & 3][1][k] = g1;
                    S.DTr[zf & 3][2][k] = g2;
                }
            }
        }
    };
    // S2 on the own column of plane zq: pi of the own row
    auto stage2 = [&](int zq) {
        const int li = (ly0 + 1) * SX1 + (lx0 + 1);
        const int sc = zq & 3;
        const int szm = (zq > 0 ? zq - 1 : zq) & 3, szp = (zq < P.m2 - 1 ? zq + 1 : zq) & 3;
        // clamped neighbours (Eq. boundary_conditions), K order -z,-y,-x,+x,+y,+z
        const int xm = (gx0 > 0) ? li - 1 : li, xp = (gx0 < P.m0 - 1) ? li + 1 : li;
        const int ym = (gy0 > 0) ? li - SX1 : li, yp = (gy0 < P.m1 - 1) ? li + SX1 : li;
        const float r0 = S.R[sc][li], t0 = S.Tw[sc][li];
        const float dR[6] = {S.R[szm][li] - r0, S.R[sc][ym] - r0, S.R[sc][xm] - r0,
                             S.R[sc][xp] - r0, S.R[sc][yp] - r0, S.R[szp][li] - r0};
        const float dT[6] = {S.Tw[szm][li] - t0, S.Tw[sc][ym] - t0, S.Tw[sc][xm] - t0,
                             S.Tw[sc][xp] - t0, S.Tw[sc][yp] - t0, S.Tw[szp][li] - t0};
        const float ihs[6] = {P.ihs[2], P.ihs[1], P.ihs[0], P.ihs[0], P.ihs[1], P.ihs[2]};
        float nn = 0.f, a2 = 0.f, b2 = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            nn = fmaf(dT[j] * dR[j], ihs[j], nn);
            a2 = fmaf(dT[j] * dT[j], ihs[j], a2);
            b2 = fmaf(dR[j] * dR[j], ihs[j], b2);
        }
        nn = fmaf(0.5f, nn, P.tr);   // N   = 1/2 <grad T, grad R> + tau rho
        a2 = fmaf(0.5f, a2, P.tau2); // A^2 = ||grad T||_tau^2
        b2 = fmaf(0.5f, b2, P.rho2); // B^2 = ||grad R||_rho^2
        const float c1 = rsqrtf(a2 * b2);  // 1/(A B)
        if (!HESS) {
            // 1 - r^2 = (A^2 B^2 - N^2)/(A^2 B^2), numerator by the Lagrange identity
            float a[6], b[6];
            const float ih6[6] = {P.ih[2], P.ih[1], P.ih[0], P.ih[0], P.ih[1], P.ih[2]};
#pragma unroll
            for (int j = 0; j < 6; ++j) { a[j] = dT[j] * ih6[j]; b[j] = dR[j] * ih6[j]; }
            float cross = 0.f, sq = 0.f;
#pragma unroll
            for (int pj = 0; pj < 6; ++pj) {
#pragma unroll
                for (int qj = pj + 1; qj < 6; ++qj) {
                    const float t = fmaf(a[pj], b[qj], -a[qj] * b[pj]);
                    cross = fmaf(t, t, cross);
                }
                const float t = fmaf(P.rho, a[pj], -P.tau * b[pj]);
                sq = fmaf(t, t, sq);
            }
            dacc += (double)(fmaf(0.25f, cross, 0.5f * sq) / (a2 * b2));
        }
        if (OBJ) return;
        const float c2 = nn * c1 / a2;     // N/(A^3 B)
        const float hh[6] = {P.hh[2], P.hh[1], P.hh[0], P.hh[0], P.hh[1], P.hh[2]};
        float rh[6], rs = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {       // Eqs. (rho), (hatRho)
            rh[j] = hh[j] * fmaf(dR[j], c1, -dT[j] * c2);
            rs += rh[j];
        }
        const float rh0 = -rs;
        float w;
        if (!HESS) {
            w = nn * c1;  // r_i
        } else {          // v_i = (dr s)_i
            w = rh0 * S.S[sc][li];
            w = fmaf(rh[0], S.S[szm][li], w);
            w = fmaf(rh[1], S.S[sc][ym], w);
            w = fmaf(rh[2], S.S[sc][xm], w);
            w = fmaf(rh[3], S.S[sc][xp], w);
            w = fmaf(rh[4], S.S[sc][yp], w);
            w = fmaf(rh[5], S.S[szp][li], w);
        }
        const int l0 = ly0 * TX + lx0;
        const int pb = zq & 1;
        S.Pi[pb][0][l0] = rh[2] * w;  // pi(-x)
        S.Pi[pb][1][l0] = rh[3] * w;  // pi(+x)
        S.Pi[pb][2][l0] = rh[1] * w;  // pi(-y)
        S.Pi[pb][3][l0] = rh[4] * w;  // pi(+y)
        pm_c = rh[0] * w;
        p0_c = rh0 * w;
        pp_c = rh[5] * w;
    };
    auto store_plane = [&](int pl) {  // node plane `pl` of this tile -> partials
        if (pl >= P.n2) return;  // the empty second plane of a planar level's box: never read
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (b_it[k] < 0) continue;
            const int yy = b_it[k] >> 6, xx = b_it[k] & 63;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float& a = S.Acc[pl & 1][c][yy][xx];
                P.partial[((tile * 3 + c) * P.pbz + (pl - BZ0)) * (long long)(P.pby * P.pbx) + yy * P.pbx + xx] = a;
                a = 0.f;
            }
        }
    };

    if (zbeg >= 0 && zbeg < P.m2) stage0(zbeg);
    __syncthreads();

    for (int zf = zbeg; zf <= zend; ++zf) {
        if (zf + 1 >= 0 && zf + 1 < P.m2 && zf + 1 <= fe_last) stage0(zf + 1);
        // ---- S1(zf)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dq3[c] = dq2[c];
            dq2[c] = dq1[c];
            dq1[c] = dq0[c];
            dq0[c] = 0.f;
        }
        if (zf >= 0 && zf < P.m2 && zf <= fe_last) front_end(zf);
        // ---- S2(zf-2): the own rows of the chunk
        const int zq = zf - 2;
        pm_c = p0_c = pp_c = 0.f;
        if (zq >= z0 && zq < z1 && own_ok) stage2(zq);
        if (!OBJ) {
            // ---- S3(zf-3): column sums of dr^T over the tile's own rows
            const int zo = zf - 3;
            if (zo >= z0 - 1 && zo <= z1 && zo >= 0 && zo < P.m2) {
                const bool in_chunk = (zo >= z0 && zo < z1);
                const int pb = zo & 1;
                const float dqo0 = dq3[0], dqo1 = dq3[1], dqo2 = dq3[2];  // dT(zo)
                float t = 0.f;
                if (own_ok) {
                    const int l0 = ly0 * TX + lx0;
                    if (in_chunk) {
                        t = p0_prev;
                        if (lx0 > 0) t += S.Pi[pb][1][l0 - 1];
                        if (lx0 + 1 < txe) t += S.Pi[pb][0][l0 + 1];
                        if (ly0 > 0) t += S.Pi[pb][3][l0 - TX];
                        if (ly0 + 1 < tye) t += S.Pi[pb][2][l0 + TX];
                    }
                    if (zo > 0 && zo - 1 >= z0) t += pp_prev2;    // row zo-1 of the chunk, its +z
                    if (zo < P.m2 - 1 && zo + 1 < z1) t += pm_c;  // row zo+1 of the chunk, its -z
                    t *= P.qscale;
                }
                *reinterpret_cast<float4*>(S.Q4[pb][(ly0 + 1) * SX1 + (lx0 + 1)]) =
                    own_ok ? make_float4(dqo0 * t, dqo1 * t, dqo2 * t, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (tid < RINGF) {
                    // face-ring column: the one in-plane own row next to it
                    int lx, ly;
                    ring_face(tid, lx, ly);
                    const int gx = xs + lx, gy = ys + ly;
                    float tr = 0.f;
                    if (in_chunk && gx >= 0 && gx < P.m0 && gy >= 0 && gy < P.m1) {
                        if (ly < 0) {
                            if (lx < txe) tr = S.Pi[pb][2][lx];                      // pi(-y) of row (lx, 0)
                        } else if (ly == TY) {
                            if (lx < txe) tr = S.Pi[pb][3][(TY - 1) * TX + lx];      // pi(+y) of row (lx, TY-1)
                        } else if (lx < 0) {
                            if (ly < tye) tr = S.Pi[pb][0][ly * TX];                 // pi(-x) of row (0, ly)
                        } else {
                            if (ly < tye) tr = S.Pi[pb][1][ly * TX + TX - 1];        // pi(+x) of row (TX-1, ly)
                        }
                        tr *= P.qscale;
                    }
                    const int dslot = zo & 3;
                    *reinterpret_cast<float4*>(S.Q4[pb][(ly + 1) * SX1 + (lx + 1)]) =
                        tr != 0.f ? make_float4(S.DTr[dslot][0][tid] * tr, S.DTr[dslot][1][tid] * tr,
                                                S.DTr[dslot][2][tid] * tr, 0.f)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            pp_prev2 = pp_prev;
            pp_prev = pp_c;
            p0_prev = p0_c;
            // ---- A(zf-4): x-reduction of q_hat
            const int za = zf - 4;
            if (za >= z0 - 1 && za <= z1 && za >= 0 && za < P.m2) {
                const int qs = za & 1;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (a_it[k] < 0) continue;
                    const int ly = a_it[k] >> 6, xx = a_it[k] & 63;  // ly: row of the halo-1 region
                    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int l = S.xr_lo[xx]; l <= S.xr_hi[xx]; ++l) {
                        const float wxl = S.wx1[l];
                        const float wx = (S.fx1[l] == xx) ? 1.f - wxl : wxl;
                        const float4 q = *reinterpret_cast<const float4*>(S.Q4[qs][ly * SX1 + l]);
                        r.x = fmaf(wx, q.x, r.x);
                        r.y = fmaf(wx, q.y, r.y);
                        r.z = fmaf(wx, q.z, r.z);
                    }
                    *reinterpret_cast<float4*>(S.Qx4[qs][ly][xx]) = r;
                }
            }
            // ---- B(zf-5): y-reduction and z accumulation
            const int zb = zf - 5;
            if (zb >= z0 - 1 && zb <= z1 && zb >= 0 && zb < P.m2) {
                const int fzo = P.fz[zb];
                const float wzo = P.wz[zb];
                if (fzo > cur) {  // node plane `cur` is complete
                    store_plane(cur);
                    cur = fzo;
                }
                const int qs = zb & 1;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (b_it[k] < 0) continue;
                    const int yy = b_it[k] >> 6, xx = b_it[k] & 63;
                    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
                    for (int l = S.yr_lo[yy]; l <= S.yr_hi[yy]; ++l) {
                        const float wyl = S.wy1[l];
                        const float wy = (S.fy1[l] == yy) ? 1.f - wyl : wyl;
                        const float4 q = *reinterpret_cast<const float4*>(S.Qx4[qs][l][xx]);
                        q0 = fmaf(wy, q.x, q0);
                        q1 = fmaf(wy, q.y, q1);
                        q2 = fmaf(wy, q.z, q2);
                    }
                    const int lo = cur & 1, hi = (cur + 1) & 1;
                    S.Acc[lo][0][yy][xx] = fmaf(1.f - wzo, q0, S.Acc[lo][0][yy][xx]);
                    S.Acc[lo][1][yy][xx] = fmaf(1.f - wzo, q1, S.Acc[lo][1][yy][xx]);
                    S.Acc[lo][2][yy][xx] = fmaf(1.f - wzo, q2, S.Acc[lo][2][yy][xx]);
                    S.Acc[hi][0][yy][xx] = fmaf(wzo, q0, S.Acc[hi][0][yy][xx]);
                    S.Acc[hi][1][yy][xx] = fmaf(wzo, q1, S.Acc[hi][1][yy][xx]);
                    S.Acc[hi][2][yy][xx] = fmaf(wzo, q2, S.Acc[hi][2][yy][xx]);
                }
            }
        }
        __syncthreads();
    }

    if (!OBJ) {  // store the two live node planes
        store_plane(cur);
        store_plane(cur + 1);
    }
    if (!HESS) {
        const double bs = block_sum(dacc, S.red);
        const int nblocks = P.ntx * P.nty * P.ntz;
        grid_sum_finish(bs, P.dpart, P.dcount, P.dout, P.hbar, S.red, nblocks, (int)tile);
    }
}

__global__ void __launch_bounds__(NT, 2) k_image_obj(const ImgParams P) {
    image_pass<MODE_OBJ, ImgSmemC>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_image_grad(const ImgParams P) {
    image_pass<MODE_GRAD, ImgSmemC>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_image_hess(const ImgParams P) {
    image_pass<MODE_HESS, ImgSmemC>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_image_obj_w(const ImgParams P) {
    image_pass<MODE_OBJ, ImgSmemW>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_image_grad_w(const ImgParams P) {
    image_pass<MODE_GRAD, ImgSmemW>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_image_hess_w(const ImgParams P) {
    image_pass<MODE_HESS, ImgSmemW>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// SSD distance (Sec. 7): r = T(x + P u) - R with the identity as residual
// Jacobian, D = hbar/2 sum r^2, grad D = hbar P^T dT^T r, H = hbar P^T dT^T dT P.
// No neighbour of a voxel is needed, so the march has no halo: per plane,
// interval 1 warps the own columns (q_hat to shared memory) and adds the
// previous plane's x-reduced q_hat into the node planes (B), interval 2
// x-reduces this plane's q_hat (A) and z-interpolates the next node plane.
// MODE_SSD_DIAG forms hbar dT_d^2 and reduces it with squared weights, the
// diagonal of hbar (dT P)^T (dT P).
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void ssd_pass(const ImgParams& P, int bx_, int by_, int bz_) {
    NGF_DYNAMIC_SMEM(smraw);
    SsdSmem& S = *reinterpret_cast<SsdSmem*>(smraw);
    constexpr bool OBJ = (MODE == MODE_OBJ), HESS = (MODE == MODE_HESS), DIAG = (MODE == MODE_SSD_DIAG);
    constexpr bool WANT_D = (MODE == MODE_OBJ || MODE == MODE_GRAD);  // the gradient pass also returns D
    constexpr int NVEC = HESS ? 6 : 3;
    const int tid = threadIdx.x;
    const int xs = bx_ * TX, ys = by_ * TY;
    const int z0 = bz_ * P.zc, z1 = min(P.m2, z0 + P.zc);
    const int txe = min(TX, P.m0 - xs), tye = min(TY, P.m1 - ys);
    // node box of the owned columns: z-interpolated planes and tile partials
    const int BX0 = P.fx[xs], BY0 = P.fy[ys], BZ0 = P.fz[z0];
    const int nbx = P.fx[xs + txe - 1] + 1 - BX0 + 1;
    const int nby = P.fy[ys + tye - 1] + 1 - BY0 + 1;
    const long long tile = ((long long)bz_ * P.nty + by_) * P.ntx + bx_;

    for (int i = tid; i < TX; i += NT) {
        const int gx = min(xs + i, P.m0 - 1);
        S.fxb[i] = P.fx[gx] - BX0;
        S.wx2[i] = P.wx[gx];
    }
    for (int i = tid; i < TY; i += NT) {
        const int gy = min(ys + i, P.m1 - 1);
        S.fyb[i] = P.fy[gy] - BY0;
        S.wy2[i] = P.wy[gy];
    }
    if (!OBJ) {
        for (int b = tid; b < nbx; b += NT) {
            int lo = TX, hi = -1;
            for (int lx = 0; lx < txe; ++lx) {
                const int f = P.fx[xs + lx] - BX0;
                if (f == b || f == b - 1) { lo = min(lo, lx); hi = max(hi, lx); }
            }
            S.xr_lo[b] = lo;
            S.xr_hi[b] = hi;
        }
        for (int b = tid; b < nby; b += NT) {
            int lo = TY, hi = -1;
            for (int ly = 0; ly < tye; ++ly) {
                const int f = P.fy[ys + ly] - BY0;
                if (f == b || f == b - 1) { lo = min(lo, ly); hi = max(hi, ly); }
            }
            S.yr_lo[b] = lo;
            S.yr_hi[b] = hi;
        }
        for (int i = tid; i < 2 * 3 * NBY * NBX; i += NT) (&S.Acc[0][0][0][0])[i] = 0.f;
    }
    const int lx0 = tid % TX, ly0 = tid / TX;
    const int gx0 = xs + lx0, gy0 = ys + ly0;
    const bool own_ok = (lx0 < txe) && (ly0 < tye);
    const int box = nbx * nby;
    int s0_g[2], s0_s[2], a_it[2], b_it[2];
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * NT;
        if (i < box) {
            const int by = i / nbx, bx = i - by * nbx;
            s0_g[k] = (BX0 + bx) + P.n0 * (BY0 + by);
            s0_s[k] = by * UBX + bx;
        } else {
            s0_g[k] = 0;
            s0_s[k] = -1;
        }
        a_it[k] = (!OBJ && i < TY * nbx) ? ((i / nbx) << 6) + (i % nbx) : -1;
        b_it[k] = (!OBJ && i < nby * nbx) ? ((i / nbx) << 6) + (i % nbx) : -1;
    }
    const int plane_n = P.n0 * P.n1;
    const float hb = (float)P.hbar;
    double dacc = 0.0;
    int cur = BZ0;

    auto stage0 = [&](int zf) {
        const int fzz = P.fz[zf];
        const float wzz = P.wz[zf];
        const int pl0 = fzz * plane_n;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (s0_s[k] < 0) continue;
            const int o = pl0 + s0_g[k];
#pragma unroll
            for (int c = 0; c < NVEC; ++c) {
                const float* src = (c < 3) ? (P.u + c * P.N) : (P.p + (c - 3) * P.N);
                const float a = __ldg(src + o), b = __ldg(src + o + P.znext);
                (&S.Uz[c][0][0])[s0_s[k]] = fmaf(wzz, b - a, a);
            }
        }
    };
    auto store_plane = [&](int pl) {
        if (pl >= P.n2) return;  // the empty second plane of a planar level's box: never read
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (b_it[k] < 0) continue;
            const int by = b_it[k] >> 6, bx = b_it[k] & 63;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float& a = S.Acc[pl & 1][c][by][bx];
                P.partial[((tile * 3 + c) * P.pbz + (pl - BZ0)) * (long long)(P.pby * P.pbx) + by * P.pbx + bx] = a;
                a = 0.f;
            }
        }
    };
    auto wsel = [](float w, bool upper) {  // trilinear weight, squared for the diagonal
        const float v = upper ? w : 1.f - w;
        return DIAG ? v * v : v;
    };

    stage0(z0);
    __syncthreads();
    for (int zf = z0; zf <= z1; ++zf) {
        // ============ interval 1: warp the own columns of plane zf; B(zf - 1)
        if (zf < z1) {
            float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (own_ok) {
                const int ax = S.fxb[lx0], ay = S.fyb[ly0];
                const float wxv = S.wx2[lx0], wyv = S.wy2[ly0];
                float uh[NVEC];
#pragma unroll
                for (int c = 0; c < NVEC; ++c) {
                    const float v00 = S.Uz[c][ay][ax], v10 = S.Uz[c][ay][ax + 1];
                    const float v01 = S.Uz[c][ay + 1][ax], v11 = S.Uz[c][ay + 1][ax + 1];
                    const float a0 = fmaf(wxv, v10 - v00, v00), a1 = fmaf(wxv, v11 - v01, v01);
                    uh[c] = fmaf(wyv, a1 - a0, a0);
                }
                float g0, g1, g2;
                const float tw = warp_sample(P, gx0, gy0, zf, uh[0] * P.ih[0], uh[1] * P.ih[1], uh[2] * P.ih[2], g0,
                                             g1, g2);
                const float r = tw - __ldg(P.R + (gx0 + P.m0 * (gy0 + P.m1 * zf)));
                if (WANT_D) dacc += (double)(r * r);
                if (OBJ) {
                } else if (DIAG) {
                    qv = make_float4(hb * g0 * g0, hb * g1 * g1, hb * g2 * g2, 0.f);
                } else {
                    const float w = HESS ? hb * fmaf(g0, uh[3], fmaf(g1, uh[4], g2 * uh[5])) : hb * r;
                    qv = make_float4(g0 * w, g1 * w, g2 * w, 0.f);
                }
            }
            if (!OBJ) *reinterpret_cast<float4*>(S.Q4[tid]) = qv;
        }
        const int za = zf - 1;
        if (!OBJ && za >= z0) {  // B: y-reduction and z accumulation of plane za
            const int fzo = P.fz[za];
            const float wzo = P.wz[za];
            if (fzo > cur) {
                store_plane(cur);
                cur = fzo;
            }
            const float wlo = wsel(wzo, false), whi = wsel(wzo, true);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (b_it[k] < 0) continue;
                const int by = b_it[k] >> 6, bx = b_it[k] & 63;
                float q0 = 0.f, q1 = 0.f, q2 = 0.f;
                for (int ly = S.yr_lo[by]; ly <= S.yr_hi[by]; ++ly) {
                    const float wy = wsel(S.wy2[ly], S.fyb[ly] != by);
                    const float4 q = *reinterpret_cast<const float4*>(S.Qx4[ly][bx]);
                    q0 = fmaf(wy, q.x, q0);
                    q1 = fmaf(wy, q.y, q1);
                    q2 = fmaf(wy, q.z, q2);
                }
                const int lo = cur & 1, hi = (cur + 1) & 1;
                S.Acc[lo][0][by][bx] = fmaf(wlo, q0, S.Acc[lo][0][by][bx]);
                S.Acc[lo][1][by][bx] = fmaf(wlo, q1, S.Acc[lo][1][by][bx]);
                S.Acc[lo][2][by][bx] = fmaf(wlo, q2, S.Acc[lo][2][by][bx]);
                S.Acc[hi][0][by][bx] = fmaf(whi, q0, S.Acc[hi][0][by][bx]);
                S.Acc[hi][1][by][bx] = fmaf(whi, q1, S.Acc[hi][1][by][bx]);
                S.Acc[hi][2][by][bx] = fmaf(whi, q2, S.Acc[hi][2][by][bx]);
            }
        }
        __syncthreads();
        // ============ interval 2: A(zf), next node plane
        if (!OBJ && zf < z1) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (a_it[k] < 0) continue;
                const int ly = a_it[k] >> 6, bx = a_it[k] & 63;
                float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int lx = S.xr_lo[bx]; lx <= S.xr_hi[bx]; ++lx) {
                    const float wx = wsel(S.wx2[lx], S.fxb[lx] != bx);
                    const float4 q = *reinterpret_cast<const float4*>(S.Q4[ly * TX + lx]);
                    r4.x = fmaf(wx, q.x, r4.x);
                    r4.y = fmaf(wx, q.y, r4.y);
                    r4.z = fmaf(wx, q.z, r4.z);
                }
                *reinterpret_cast<float4*>(S.Qx4[ly][bx]) = r4;
            }
        }
        if (zf + 1 < z1) stage0(zf + 1);
        __syncthreads();
    }
    if (!OBJ) {
        store_plane(cur);
        store_plane(cur + 1);
    }
    if (WANT_D) {
        const double bs = block_sum(dacc, S.red);
        grid_sum_finish(bs, P.dpart, P.dcount, P.dout, 0.5 * P.hbar, S.red, P.ntx * P.nty * P.ntz, (int)tile);
    }
}

__global__ void __launch_bounds__(NT, 2) k_ssd_obj(const ImgParams P) {
    ssd_pass<MODE_OBJ>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_ssd_grad(const ImgParams P) {
    ssd_pass<MODE_GRAD>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_ssd_hess(const ImgParams P) {
    ssd_pass<MODE_HESS>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_ssd_diag(const ImgParams P) {
    ssd_pass<MODE_SSD_DIAG>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Exact Jacobi diagonal of the Gauss-Newton matrix (without the curvature
// part): diag_{d,n} = 2 hbar sum_i J_{i,(d,n)}^2, J = dr dT P, row i formed
// from the 7 entries of row i of dr (Eq. dr) and the trilinear weights of each
// entry's voxel, using the separable structure of P:
//   J(a,b,g) = ez ey ax + ez by ex + cz ey ex
// with e* the weights of voxel i itself and ax/by/cz the coefficient-weighted
// weights of its x/y/z stencil entries.  The squared entries of the owned
// rows are summed onto node planes (four live planes), which are stored as
// tile partials of the halo-1 geometry.
//
// Each warp is one row of the tile and owns a private accumulator window
// (4 node planes x 3 components x SPAN y-nodes x diag_pxw(SPAN) x-nodes).
// Lanes whose voxels share an x-node floor form runs; a segmented shuffle sum
// gives each run's total to its first lane, which alone adds it (plain
// read-modify-write, distinct addresses within a step; a warp barrier orders
// the steps that reach the same node from neighbouring runs).  The windows of the rows are merged
// in a fixed order when a node plane is complete, so the diagonal is
// deterministic.  SPAN 3 when every axis has two or more voxels per cell,
// SPAN 4 otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pw_weight(int f, float w1, int node) {
    return (node == f) ? 1.f - w1 : ((node == f + 1) ? w1 : 0.f);
}

// DS > 0: the shuffle steps of the run sums as a compile-time count (the
// largest any tile of the plan needs; extra steps add nothing to a run's
// head, so the sums are the same); DS = 0: per tile from the parameters.
// With two or more voxels per cell the first x tile's clamped lane 0 makes
// a run of at least three, so a three-node span needs two steps or more.
template <int SPAN, int DS = 0>
__device__ __forceinline__ void diag_pass(const ImgParams& P, int bx, int by, int bz) {
    NGF_DYNAMIC_SMEM(smraw);
    DiagSmemT<SPAN>& S = *reinterpret_cast<DiagSmemT<SPAN>*>(smraw);
    constexpr int PXWS = diag_pxw(SPAN);
    constexpr int WPLANE = 3 * SPAN * PXWS;  // one node plane of a row's window
    const int tid = threadIdx.x;
    const int xs = bx * TX, ys = by * TY;
    const int z0 = bz * P.zc, z1 = min(P.m2, z0 + P.zc);
    const int txe = min(TX, P.m0 - xs), tye = min(TY, P.m1 - ys);
    const int UX0 = P.fx[max(xs - 1, 0)], UY0 = P.fy[max(ys - 1, 0)];
    const int UXn = P.fx[min(xs + TX, P.m0 - 1)] + 1 - UX0 + 1;
    const int UYn = P.fy[min(ys + TY, P.m1 - 1)] + 1 - UY0 + 1;
    // the partial box of the halo-1 geometry equals the Uz box in x and y
    const int BZ0 = P.fz[max(z0 - 1, 0)], BZ1 = P.fz[min(z1, P.m2 - 1)] + 1;
    const int nbx = UXn, nby = UYn;
    const long long tile = ((long long)bz * P.nty + by) * P.ntx + bx;

    for (int i = tid; i < SX1; i += NT) {
        const int gx = min(max(xs - 1 + i, 0), P.m0 - 1);
        S.fx1[i] = P.fx[gx] - UX0;
        S.wx1[i] = P.wx[gx];
    }
    for (int i = tid; i < SY1; i += NT) {
        const int gy = min(max(ys - 1 + i, 0), P.m1 - 1);
        S.fy1[i] = P.fy[gy] - UY0;
        S.wy1[i] = P.wy[gy];
    }
    for (int i = tid; i < TY * diag_window(SPAN); i += NT) S.Acc[i] = 0.f;
    // y weights of row ly's stencil lines (ly - 1, ly, ly + 1) on the SPAN node
    // rows from the lowest line's floor: fixed for the whole march, uniform
    // over the row's warp, kept in shared memory rather than registers
    for (int i = tid; i < TY * 3 * SPAN; i += NT) {
        const int ly = i / (3 * SPAN), k = (i / SPAN) % 3, a = i % SPAN;
        const int gl = min(max(ys - 1 + ly, 0), P.m1 - 1), gk = min(max(ys - 1 + ly + k, 0), P.m1 - 1);
        S.WYs[ly][k][a] = pw_weight(P.fy[gk] - UY0, P.wy[gk], P.fy[gl] - UY0 + a);
    }
    __syncthreads();

    // lane layout of the owned columns: warp = row ly, lane = lx
    const int lx = tid % TX, ly = tid / TX;
    const bool act = lx < txe;
    const int lxc = min(lx, txe - 1);  // inactive lanes mirror the last column, contribute zero
    // runs of lanes sharing the x-node floor of the stencil's lowest voxel
    const int dsteps = DS > 0 ? DS : ((xs == 0) ? P.dsteps0 : P.dsteps);
    unsigned int same = 0u;
    const int key = S.fx1[lxc];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int o = __shfl_down_sync(0xffffffffu, key, 1 << k);
        if (k < dsteps && lx + (1 << k) < TX && o == key) same |= 1u << k;
    }
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = (lx == 0) || (prev != key);
    float* const priv = S.Acc + ly * (4 * WPLANE);

    const int items = 3 * nby * nbx;
    int next = BZ0;  // next node plane to store
    const float twoh = (float)(2.0 * P.hbar);

    for (int zf = z0 - 1; zf <= z1; ++zf) {
        const bool fe = (zf >= 0) && (zf < P.m2);
        if (fe) {
            const int fzz = P.fz[zf];
            const float wzz = P.wz[zf];
            const long long plane = (long long)P.n0 * P.n1;
            const long long pl0 = (long long)fzz * plane;
            const int box = UXn * UYn;
            for (int i = tid; i < 3 * box; i += NT) {
                const int c = i / box;
                const int rem = i - c * box;
                const int by = rem / UXn, bx = rem - by * UXn;
                const float* src = P.u + c * P.N;
                const long long o = pl0 + (UX0 + bx) + (long long)P.n0 * (UY0 + by);
                const float a = __ldg(src + o), b = __ldg(src + o + P.znext);
                S.Uz[c][by][bx] = fmaf(wzz, b - a, a);
            }
        }
        __syncthreads();
        {  // z weights of the next scattered plane's stencil planes (uniform per plane)
            const int zq = zf - 1;
            if (tid < 3 * SPAN && zq >= z0 && zq < z1) {
                const int k = tid / SPAN, a = tid % SPAN;
                const int vz = min(max(zq - 1 + k, 0), P.m2 - 1), vl = max(zq - 1, 0);
                S.WZs[k][a] = pw_weight(P.fz[vz] - BZ0, P.wz[vz], P.fz[vl] - BZ0 + a);
            }
        }
        if (fe) {
            const int slot = zf % 3;
            for (int k = tid; k < NT + ring_size(1); k += NT) {
                int cx, cy;
                if (k < NT) { cx = k % TX; cy = k / TX; }
                else ring_coord(k - NT, 1, cx, cy);
                const int gx = xs + cx, gy = ys + cy;
                if (gx < 0 || gx >= P.m0 || gy < 0 || gy >= P.m1) continue;
                const int li = (cy + 1) * SX1 + (cx + 1);
                const int ax = S.fx1[cx + 1], ay = S.fy1[cy + 1];
                const float wxv = S.wx1[cx + 1], wyv = S.wy1[cy + 1];
                float uh[3];
                for (int c = 0; c < 3; ++c) {
                    const float v00 = S.Uz[c][ay][ax], v10 = S.Uz[c][ay][ax + 1];
                    const float v01 = S.Uz[c][ay + 1][ax], v11 = S.Uz[c][ay + 1][ax + 1];
                    const float a0 = fmaf(wxv, v10 - v00, v00), a1 = fmaf(wxv, v11 - v01, v01);
                    uh[c] = fmaf(wyv, a1 - a0, a0);
                }
                float g0, g1, g2;
                const float tw = warp_sample(P, gx, gy, zf, uh[0] * P.ih[0], uh[1] * P.ih[1], uh[2] * P.ih[2],
                                             g0, g1, g2);
                const long long gi = (long long)gx + (long long)P.m0 * (gy + (long long)P.m1 * zf);
                S.R[slot][li] = __ldg(P.R + gi);
                S.Tw[slot][li] = tw;
                S.dT[slot][0][li] = g0;
                S.dT[slot][1][li] = g1;
                S.dT[slot][2][li] = g2;
            }
        }
        __syncthreads();
        const int zq = zf - 1;
        if (zq >= z0 && zq < z1 && ly < tye) {  // whole warps (rows) only
            const int gx = xs + lxc, gy = ys + ly;
            const int sc = zq % 3;
            const int szm = (zq > 0 ? zq - 1 : zq) % 3, szp = (zq < P.m2 - 1 ? zq + 1 : zq) % 3;
            const int li = (ly + 1) * SX1 + (lxc + 1);
            const int xm = (gx > 0) ? li - 1 : li, xp = (gx < P.m0 - 1) ? li + 1 : li;
            const int ym = (gy > 0) ? li - SX1 : li, yp = (gy < P.m1 - 1) ? li + SX1 : li;
            const float r0 = S.R[sc][li], t0 = S.Tw[sc][li];
            const float dR[6] = {S.R[szm][li] - r0, S.R[sc][ym] - r0, S.R[sc][xm] - r0,
                                 S.R[sc][xp] - r0, S.R[sc][yp] - r0, S.R[szp][li] - r0};
            const float dTv[6] = {S.Tw[szm][li] - t0, S.Tw[sc][ym] - t0, S.Tw[sc][xm] - t0,
                                  S.Tw[sc][xp] - t0, S.Tw[sc][yp] - t0, S.Tw[szp][li] - t0};
            const float ihs[6] = {P.ihs[2], P.ihs[1], P.ihs[0], P.ihs[0], P.ihs[1], P.ihs[2]};
            float nn = 0.f, a2 = 0.f, b2 = 0.f;
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                nn = fmaf(dTv[j] * dR[j], ihs[j], nn);
                a2 = fmaf(dTv[j] * dTv[j], ihs[j], a2);
                b2 = fmaf(dR[j] * dR[j], ihs[j], b2);
            }
            nn = fmaf(0.5f, nn, P.tr);
            a2 = fmaf(0.5f, a2, P.tau2);
            b2 = fmaf(0.5f, b2, P.rho2);
            const float c1 = rsqrtf(a2 * b2);
            const float c2 = nn * c1 / a2;
            const float hh[6] = {P.hh[2], P.hh[1], P.hh[0], P.hh[0], P.hh[1], P.hh[2]};
            float rh[6], rs = 0.f;
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                rh[j] = hh[j] * fmaf(dR[j], c1, -dTv[j] * c2);
                rs += rh[j];
            }
            const float rh0 = -rs;
            // node floors and weights of the stencil entries' voxels (clamped)
            const int vzm = max(zq - 1, 0), vzp = min(zq + 1, P.m2 - 1);
            const int fxm = S.fx1[lxc], fxc = S.fx1[lxc + 1], fxp = S.fx1[lxc + 2];
            const float wxm = S.wx1[lxc], wxc = S.wx1[lxc + 1], wxp = S.wx1[lxc + 2];
            const int fym = S.fy1[ly], fyp = S.fy1[ly + 2];
            const int fzm = P.fz[vzm] - BZ0, fzp = P.fz[vzp] - BZ0;
            const int bxm = fxm, bym = fym, bzm = fzm;  // lowest node touched per axis
            // trilinear weights of the stencil voxels (offset -1, 0, +1 per
            // axis) on the SPAN nodes from the lowest floor; independent of
            // the component (y and z: the shared tables, uniform over the warp)
            float WX[3][SPAN];
#pragma unroll
            for (int a = 0; a < SPAN; ++a) {
                WX[0][a] = pw_weight(fxm, wxm, bxm + a);
                WX[1][a] = pw_weight(fxc, wxc, bxm + a);
                WX[2][a] = pw_weight(fxp, wxp, bxm + a);
            }
            const float(&WY)[3][SPAN] = S.WYs[ly];
            const float(&WZ)[3][SPAN] = S.WZs;
            int po[SPAN];
#pragma unroll
            for (int g = 0; g < SPAN; ++g) po[g] = ((bzm + g + BZ0) & 3) * WPLANE + bxm;
            // node planes and rows this voxel row reaches: the stencil's lowest
            // floor up to its highest floor + 1 (two, not three, inside a cell);
            // both are uniform over the warp (one row, one plane), and the
            // entries beyond them are exactly zero, so they are skipped
            const int spanY = min(SPAN, fyp - fym + 2), spanZ = min(SPAN, fzp - fzm + 2);
#pragma unroll 1
            for (int d = 0; d < 3; ++d) {
                const float* dTd[3] = {S.dT[szm][d], S.dT[sc][d], S.dT[szp][d]};
                const float cc = rh0 * dTd[1][li];
                const float cxm = rh[2] * dTd[1][xm], cxp = rh[3] * dTd[1][xp];
                const float cym = rh[1] * dTd[1][ym], cyp = rh[4] * dTd[1][yp];
                const float czm = rh[0] * dTd[0][li], czp = rh[5] * dTd[2][li];
                float ax[SPAN], byv[SPAN], cz[SPAN];
#pragma unroll
                for (int a = 0; a < SPAN; ++a) {
                    ax[a] = fmaf(cc, WX[1][a], fmaf(cxm, WX[0][a], cxp * WX[2][a]));
                    byv[a] = fmaf(cym, WY[0][a], cyp * WY[2][a]);
                    cz[a] = fmaf(czm, WZ[0][a], czp * WZ[2][a]);
                }
                // entries outside the support are exactly zero, so only the box
                // bounds are checked; the 2 hbar factor is applied at the store
#pragma unroll
                for (int b = 0; b < SPAN; ++b) {
                    if (b >= spanY || bym + b >= nby) continue;  // uniform over the warp
#pragma unroll
                    for (int a = 0; a < SPAN; ++a) {
                        const bool inb = bxm + a < nbx;
                        const float xy1 = fmaf(WY[1][b], ax[a], byv[b] * WX[1][a]);
                        const float xy2 = WY[1][b] * WX[1][a];
#pragma unroll
                        for (int g = 0; g < SPAN; ++g) {
                            if (g >= spanZ) break;  // uniform over the warp
                            const float J = fmaf(WZ[1][g], xy1, cz[g] * xy2);
                            float v = act ? J * J : 0.f;
#pragma unroll
                            for (int k = 0; k < 5; ++k) {
                                if (k >= dsteps) break;
                                const float t = __shfl_down_sync(0xffffffffu, v, 1 << k);
                                if (same & (1u << k)) v += t;
                            }
                            if (head && inb) priv[po[g] + (d * SPAN + b) * PXWS + a] += v;
                        }
                        // the next a reaches the x-nodes of this one from the neighbouring run
                        __syncwarp();
                    }
                }
            }
        }
        __syncthreads();
        // node planes below fz[zq] receive nothing more from this chunk
        if (zq >= z0 && zq < z1) {
            const int limit = (zq == z1 - 1) ? BZ1 + 1 : P.fz[zq];
            while (next < limit) {
                const int sl = next & 3;
                for (int i = tid; i < items; i += NT) {
                    const int c = i / (nby * nbx), rem = i % (nby * nbx), byy = rem / nbx, bxx = rem % nbx;
                    float sum = 0.f;
                    for (int w = 0; w < tye; ++w) {  // rows in a fixed order
                        const int b = byy - S.fy1[w];
                        if (b < 0 || b >= SPAN) continue;
                        float& e = S.Acc[w * (4 * WPLANE) + sl * WPLANE + (c * SPAN + b) * PXWS + bxx];
                        sum += e;
                        e = 0.f;
                    }
                    P.partial[((tile * 3 + c) * P.pbz + (next - BZ0)) * (long long)(P.pby * P.pbx) + byy * P.pbx + bxx] =
                        twoh * sum;
                }
                ++next;
            }
        }
    }
}

// Three nodes per axis suffice when every axis has at least two voxels per
// deformation cell (2 (n-1) <= m); four otherwise.  The three-node form fits
// 64 registers and its shared memory twice per SM: two CTAs per SM, 27%
// faster on the thorax grid than one CTA of 111 registers.
__global__ void __launch_bounds__(NT, 2) k_diag(const ImgParams P) { diag_pass<3>(P, blockIdx.x, blockIdx.y, blockIdx.z); }
__global__ void __launch_bounds__(NT, 2) k_diag_s2(const ImgParams P) {
    diag_pass<3, 2>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 2) k_diag_s3(const ImgParams P) {
    diag_pass<3, 3>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}
__global__ void __launch_bounds__(NT, 1) k_diag4(const ImgParams P) {
    diag_pass<4>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// nodal kernels
// ---------------------------------------------------------------------------

// coordinates of element i of a 3 x N nodal field (component-major, x fastest)
__device__ __forceinline__ void node_coords(unsigned int i, const NodeGeom& G, int& c, int& n, int& ix, int& iy,
                                            int& iz) {
    c = (int)fdiv(i, G.fN);
    n = (int)(i - (unsigned int)c * (unsigned int)G.N);
    iz = (int)fdiv((unsigned int)n, G.fplane);
    const int rem = n - iz * G.n0 * G.n1;
    iy = (int)fdiv((unsigned int)rem, G.fn0);
    ix = rem - iy * G.n0;
}

// clamped 7-point Laplacian of component array xc at node (ix, iy, iz)
__device__ __forceinline__ float lap_at(const float* __restrict__ xc, const NodeGeom& G, int n, int ix, int iy, int iz) {
    const int sy = G.n0, sz = G.n0 * G.n1;
    const float v = xc[n];
    const float xm = xc[ix > 0 ? n - 1 : n], xp = xc[ix < G.n0 - 1 ? n + 1 : n];
    const float ym = xc[iy > 0 ? n - sy : n], yp = xc[iy < G.n1 - 1 ? n + sy : n];
    const float zm = xc[iz > 0 ? n - sz : n], zp = xc[iz < G.n2 - 1 ? n + sz : n];
    return (xm - 2.f * v + xp) * G.ihy2[0] + (ym - 2.f * v + yp) * G.ihy2[1] + (zm - 2.f * v + zp) * G.ihy2[2];
}

// L = Lap x per component (Eq. laplace_discretized, clamped Neumann
// neighbours); optional S = scale * sum L^2 (deterministic).  One thread per
// node handles the three components.  `bid`/`nb`: this CTA's index and the
// CTA count of the launch (or of its segment in a batched launch).
__device__ __forceinline__ void lap_body(const NodeGeom& G, const float* __restrict__ x, float* __restrict__ L,
                                         double* part, unsigned int* count, double* out, double scale,
                                         unsigned int bid, unsigned int nb) {
    __shared__ double red[NT];
    DFAcc acc;
    const unsigned int N = (unsigned int)G.N;
    for (unsigned int n = bid * NT + threadIdx.x; n < N; n += nb * NT) {
        const int iz = (int)fdiv(n, G.fplane);
        const int rem = (int)n - iz * G.n0 * G.n1;
        const int iy = (int)fdiv((unsigned int)rem, G.fn0);
        const int ix = rem - iy * G.n0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float l = lap_at(x + (size_t)c * N, G, (int)n, ix, iy, iz);
            L[(size_t)c * N + n] = l;
            acc.add_prod(l, l);
        }
    }
    if (out) {
        const double bs = block_sum(acc.value(), red);
        grid_sum_finish(bs, part, count, out, scale, red, (int)nb, (int)bid);
    }
}

__global__ void __launch_bounds__(NT) k_lap(NodeGeom G, const float* __restrict__ x, float* __restrict__ L,
                                            double* part, unsigned int* count, double* out, double scale) {
    lap_body(G, x, L, part, count, out, scale, blockIdx.x, gridDim.x);
}

// out_{c,n} = sum of the tile partials containing node n (fixed order)
//           + alpha 2 hbar^y (Lap L)_{c,n}   or   + alpha 2 hbar^y diag(Lap^T Lap)_n
// One thread per node handles the three components.
__device__ __forceinline__ void combine_body(const CombineParams& P, unsigned int bid, unsigned int nb) {
    __shared__ double red[NT];
    DFAcc acc;
    const NodeGeom& G = P.G;
    const unsigned int N = (unsigned int)G.N;
    for (unsigned int n = bid * NT + threadIdx.x; n < N; n += nb * NT) {
        const int iz = (int)fdiv(n, G.fplane);
        const int rem = (int)n - iz * G.n0 * G.n1;
        const int iy = (int)fdiv((unsigned int)rem, G.fn0);
        const int ix = rem - iy * G.n0;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        // tile partials in a fixed order: ascending tiles, z outermost
        const int box = P.box;
        const int tz1 = __ldg(P.zhi + iz), ty0 = __ldg(P.ylo + iy), ty1 = __ldg(P.yhi + iy);
        const int tx0 = __ldg(P.xlo + ix), tx1 = __ldg(P.xhi + ix);
        for (int tz = __ldg(P.zlo + iz); tz <= tz1; ++tz) {
            const int oz = __ldg(P.ztb + tz) + iz * P.pbxy;
            for (int ty = ty0; ty <= ty1; ++ty) {
                const int oy = oz + __ldg(P.ytb + ty) + iy * P.pbx;
                for (int tx = tx0; tx <= tx1; ++tx) {
                    const float* pp = P.partial + (oy + __ldg(P.xtb + tx) + ix);
                    s0 += __ldg(pp);
                    s1 += __ldg(pp + box);
                    s2 += __ldg(pp + 2 * box);
                }
            }
        }
        if (P.L) {
            s0 = fmaf(P.cscale, lap_at(P.L, G, (int)n, ix, iy, iz), s0);
            s1 = fmaf(P.cscale, lap_at(P.L + N, G, (int)n, ix, iy, iz), s1);
            s2 = fmaf(P.cscale, lap_at(P.L + 2 * (size_t)N, G, (int)n, ix, iy, iz), s2);
        }
        if (P.ctab) {
            // diag(Lap^T Lap) = sum_a diag(K_a^2) + sum_{a != b} diag(K_a) diag(K_b)
            // with K_a the 1-D clamped Laplacian along axis a
            const int o1 = G.n0, o2 = G.n0 + G.n1, od = G.n0 + G.n1 + G.n2;
            const float gx = P.ctab[od + ix], gy = P.ctab[od + o1 + iy], gz = P.ctab[od + o2 + iz];
            const float cd = P.cscale * (P.ctab[ix] + P.ctab[o1 + iy] + P.ctab[o2 + iz] +
                                         2.f * (gx * gy + gx * gz + gy * gz));
            s0 += cd;
            s1 += cd;
            s2 += cd;
        }
        P.out[n] = s0;
        P.out[N + n] = s1;
        P.out[2 * (size_t)N + n] = s2;
        if (P.dotw) {
            acc.add_prod(s0, P.dotw[n]);
            acc.add_prod(s1, P.dotw[N + n]);
            acc.add_prod(s2, P.dotw[2 * (size_t)N + n]);
        }
    }
    if (P.dout) {
        const double bs = block_sum(acc.value(), red);
        grid_sum_finish(bs, P.dpart, P.dcount, P.dout, 1.0, red, (int)nb, (int)bid);
    }
}

__global__ void __launch_bounds__(NT) k_node_combine(const CombineParams P) { combine_body(P, blockIdx.x, gridDim.x); }

// q = scale * Lap(L) with L = Lap p, no partials (curvature_apply)
__global__ void __launch_bounds__(NT) k_lap2(NodeGeom G, const float* __restrict__ L, float* __restrict__ q,
                                             float scale) {
    const unsigned int total = 3u * (unsigned int)G.N;
    for (unsigned int i = blockIdx.x * NT + threadIdx.x; i < total; i += gridDim.x * NT) {
        int c, n, ix, iy, iz;
        node_coords(i, G, c, n, ix, iy, iz);
        q[i] = scale * lap_at(L + (size_t)c * G.N, G, n, ix, iy, iz);
    }
}

// ---------------------------------------------------------------------------
// PCG (Sec. 2.3.1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float minv(const float* diag, unsigned int i) {
    const float dv = diag[i];
    return dv > 0.f ? 1.f / dv : 0.f;
}

// two deterministic float64 sums (e.g. r.z and r.r) finished by the last CTA;
// returns true in thread 0 of the last CTA, with A and B set there
__device__ __forceinline__ bool grid_sum2(double a, double b, double* part, unsigned int* count, double* red,
                                          double& A, double& B, int nb, int bid) {
    __shared__ int is_last;
    const double sa = block_sum(a, red);
    __syncthreads();
    const double sb = block_sum(b, red);
    if (threadIdx.x == 0) {
        part[bid] = sa;
        part[nb + bid] = sb;
        __threadfence();
        is_last = (atomicAdd(count, 1u) == (unsigned int)(nb - 1));
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        x += ((volatile double*)part)[i];
        y += ((volatile double*)part)[nb + i];
    }
    A = block_sum(x, red);
    __syncthreads();
    B = block_sum(y, red);
    if (threadIdx.x == 0) *count = 0u;
    return threadIdx.x == 0;
}

__device__ __forceinline__ void pcg_init_body(const PcgParams& P, unsigned int bid, unsigned int nb) {
    __shared__ double red[NT];
    DFAcc a, b;
    const unsigned int n = (unsigned int)P.n;
    for (unsigned int i = bid * NT + threadIdx.x; i < n; i += nb * NT) {
        const float rv = P.rhs[i];
        const float zv = rv * minv(P.diag, i);
        P.x[i] = 0.f;
        P.r[i] = rv;
        P.z[i] = zv;
        P.d[i] = zv;
        a.add_prod(rv, zv);
        b.add_prod(rv, rv);
    }
    double A, B;
    if (grid_sum2(a.value(), b.value(), P.part, P.count, red, A, B, (int)nb, (int)bid)) {
        P.sc[PS_DELTA] = A;
        P.sc[PS_RR] = B;
        P.sc[PS_BB] = B;
        P.sc[PS_DQ] = 0.0;
        P.sc[PS_ALPHA] = 0.0;
        P.sc[PS_BETA] = 0.0;
        P.sc[PS_ITERS] = 0.0;
        double st = 0.0;
        if (A == 0.0) st = 1.0;
        else if (P.rtol > 0.0 && sqrt(B) <= P.rtol * sqrt(B)) st = 3.0;
        P.sc[PS_STATUS] = st;
    }
}

// after q = A d and sc[PS_DQ] = d.q: x += a d, r -= a q, z = M^-1 r, new delta.
// With P.vec4 (all vectors 16-byte aligned) the body moves float4 groups;
// the elements past the last full group are handled one by one.
__device__ __forceinline__ float pcg_elem(float a, float dv, float qv, float& xv, float& rv, float diag) {
    xv = fmaf(a, dv, xv);
    rv = fmaf(-a, qv, rv);
    return rv * (diag > 0.f ? 1.f / diag : 0.f);
}

__device__ __forceinline__ void pcg_update_body(const PcgParams& P, unsigned int bid, unsigned int nb) {
    __shared__ double red[NT];
    const double st = P.sc[PS_STATUS];
    const double dq = P.sc[PS_DQ];
    const double delta = P.sc[PS_DELTA];
    const bool active = (st == 0.0) && (dq > 0.0) && isfinite(dq);
    const float a = active ? (float)(delta / dq) : 0.f;
    DFAcc sa, sb;
    if (active) {
        const unsigned int n = (unsigned int)P.n;
        const unsigned int n4 = P.vec4 ? n / 4 : 0;
        const unsigned int stride = nb * NT;
        for (unsigned int i = bid * NT + threadIdx.x; i < n4; i += stride) {
            const float4 dv = reinterpret_cast<const float4*>(P.d)[i];
            const float4 qv = reinterpret_cast<const float4*>(P.q)[i];
            const float4 gv = reinterpret_cast<const float4*>(P.diag)[i];
            float4 xv = reinterpret_cast<const float4*>(P.x)[i];
            float4 rv = reinterpret_cast<const float4*>(P.r)[i];
            float4 zv;
            zv.x = pcg_elem(a, dv.x, qv.x, xv.x, rv.x, gv.x);
            zv.y = pcg_elem(a, dv.y, qv.y, xv.y, rv.y, gv.y);
            zv.z = pcg_elem(a, dv.z, qv.z, xv.z, rv.z, gv.z);
            zv.w = pcg_elem(a, dv.w, qv.w, xv.w, rv.w, gv.w);
            reinterpret_cast<float4*>(P.x)[i] = xv;
            reinterpret_cast<float4*>(P.r)[i] = rv;
            reinterpret_cast<float4*>(P.z)[i] = zv;
            sa.add_prod(rv.x, zv.x);
            sa.add_prod(rv.y, zv.y);
            sa.add_prod(rv.z, zv.z);
            sa.add_prod(rv.w, zv.w);
            sb.add_prod(rv.x, rv.x);
            sb.add_prod(rv.y, rv.y);
            sb.add_prod(rv.z, rv.z);
            sb.add_prod(rv.w, rv.w);
        }
        for (unsigned int i = 4 * n4 + bid * NT + threadIdx.x; i < n; i += stride) {
            float xv = P.x[i], rv = P.r[i];
            const float zv = pcg_elem(a, P.d[i], P.q[i], xv, rv, P.diag[i]);
            P.x[i] = xv;
            P.r[i] = rv;
            P.z[i] = zv;
            sa.add_prod(rv, zv);
            sb.add_prod(rv, rv);
        }
    }
    double A, B;
    if (grid_sum2(sa.value(), sb.value(), P.part, P.count, red, A, B, (int)nb, (int)bid)) {
        if (st != 0.0) return;
        if (!active) {
            P.sc[PS_STATUS] = 2.0;
            return;
        }
        P.sc[PS_ALPHA] = delta / dq;
        P.sc[PS_BETA] = A / delta;
        P.sc[PS_DELTA] = A;
        P.sc[PS_RR] = B;
        P.sc[PS_ITERS] += 1.0;
        if (A == 0.0) P.sc[PS_STATUS] = 1.0;
        else if (P.rtol > 0.0 && sqrt(B) <= P.rtol * sqrt(P.sc[PS_BB])) P.sc[PS_STATUS] = 3.0;
    }
}

__device__ __forceinline__ void pcg_dir_body(const PcgParams& P, unsigned int bid, unsigned int nb) {
    if (P.sc[PS_STATUS] != 0.0) return;
    const float beta = (float)P.sc[PS_BETA];
    const unsigned int n = (unsigned int)P.n;
    const unsigned int n4 = P.vec4 ? n / 4 : 0;
    const unsigned int stride = nb * NT;
    for (unsigned int i = bid * NT + threadIdx.x; i < n4; i += stride) {
        const float4 zv = reinterpret_cast<const float4*>(P.z)[i];
        float4 dv = reinterpret_cast<const float4*>(P.d)[i];
        dv.x = fmaf(beta, dv.x, zv.x);
        dv.y = fmaf(beta, dv.y, zv.y);
        dv.z = fmaf(beta, dv.z, zv.z);
        dv.w = fmaf(beta, dv.w, zv.w);
        reinterpret_cast<float4*>(P.d)[i] = dv;
    }
    for (unsigned int i = 4 * n4 + bid * NT + threadIdx.x; i < n; i += stride) P.d[i] = fmaf(beta, P.d[i], P.z[i]);
}

__global__ void __launch_bounds__(NT) k_pcg_init(PcgParams P) { pcg_init_body(P, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(NT) k_pcg_update(PcgParams P) { pcg_update_body(P, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(NT) k_pcg_dir(PcgParams P) { pcg_dir_body(P, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// small vector kernels and multilevel helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dot_body(const DotArgs& A, unsigned int bid, unsigned int nb) {
    __shared__ double red[NT];
    DFAcc acc;
    for (unsigned int i = bid * NT + threadIdx.x; i < (unsigned int)A.n; i += nb * NT)
        acc.add_prod(A.a[i], A.b ? A.b[i] : 1.f);
    const double bs = block_sum(acc.value(), red);
    grid_sum_finish(bs, A.part, A.count, A.out, 1.0, red, (int)nb, (int)bid);
}

__global__ void __launch_bounds__(NT) k_dot(long long n, const float* __restrict__ a, const float* __restrict__ b,
                                            double* part, unsigned int* count, double* out) {
    dot_body(DotArgs{n, a, b, part, count, out}, blockIdx.x, gridDim.x);
}

// y = x + eta * s (eta as float); y = x when s is null
__device__ __forceinline__ void axpy_body(const AxpyArgs& A, unsigned int bid, unsigned int nb) {
    for (long long i = (long long)bid * NT + threadIdx.x; i < A.n; i += (long long)nb * NT)
        A.y[i] = A.s ? fmaf(A.eta, A.s[i], A.x[i]) : A.x[i];
}

__global__ void __launch_bounds__(NT) k_axpy(long long n, float eta, const float* __restrict__ x,
                                             const float* __restrict__ s, float* __restrict__ y) {
    axpy_body(AxpyArgs{n, eta, x, s, y}, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(NT) k_scale(long long n, float a, const float* __restrict__ x, float* __restrict__ y) {
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) y[i] = a * x[i];
}

// count of non-finite values (float64 so the deterministic sum can be reused)
__global__ void __launch_bounds__(NT) k_nonfinite(long long n, const float* __restrict__ a, double* part,
                                                  unsigned int* count, double* out) {
    __shared__ double red[NT];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        acc += isfinite(a[i]) ? 0.0 : 1.0;
    const double bs = block_sum(acc, red);
    grid_sum_finish(bs, part, count, out, 1.0, red, gridDim.x, blockIdx.x);
}

// image pyramid: coarse cell = mean of its existing children (<= 8)
__global__ void __launch_bounds__(NT) k_restrict(int m0, int m1, int m2, const float* __restrict__ img,
                                                 float* __restrict__ out) {
    const int c0 = (m0 + 1) / 2, c1 = (m1 + 1) / 2, c2 = (m2 + 1) / 2;
    const long long total = (long long)c0 * c1 * c2;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < total; i += (long long)gridDim.x * NT) {
        const int x = (int)(i % c0), y = (int)((i / c0) % c1), z = (int)(i / ((long long)c0 * c1));
        float s = 0.f;
        int cnt = 0;
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int fx = 2 * x + a, fy = 2 * y + b, fz = 2 * z + c;
                    if (fx >= m0 || fy >= m1 || fz >= m2) continue;
                    s += img[fx + (long long)m0 * (fy + (long long)m1 * fz)];
                    ++cnt;
                }
        out[i] = s / (float)cnt;
    }
}

// trilinear prolongation between node grids over the same domain; per-axis
// tables (floor, weight) are built on the host
__global__ void __launch_bounds__(NT) k_prolong(int f0, int f1, int f2, int c0, int c1, long long Nc,
                                                const int* __restrict__ tf, const float* __restrict__ tw,
                                                const float* __restrict__ uc, float* __restrict__ uf) {
    const long long Nf = (long long)f0 * f1 * f2;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < 3 * Nf; i += (long long)gridDim.x * NT) {
        const long long d = i / Nf, n = i - d * Nf;
        const int x = (int)(n % f0), y = (int)((n / f0) % f1), z = (int)(n / ((long long)f0 * f1));
        const int bx = tf[x], by = tf[f0 + y], bz = tf[f0 + f1 + z];
        const float wx = tw[x], wy = tw[f0 + y], wz = tw[f0 + f1 + z];
        const float* u = uc + d * Nc;
        const long long o = bx + (long long)c0 * (by + (long long)c1 * bz);
        const long long sy = c0, sz = (long long)c0 * c1;
        const float e00 = fmaf(wx, u[o + 1] - u[o], u[o]);
        const float e10 = fmaf(wx, u[o + sy + 1] - u[o + sy], u[o + sy]);
        const float a0 = fmaf(wy, e10 - e00, e00);
        if (Nc == sz) {  // one coarse node plane (planar level)
            uf[i] = a0;
            continue;
        }
        const float e01 = fmaf(wx, u[o + sz + 1] - u[o + sz], u[o + sz]);
        const float e11 = fmaf(wx, u[o + sz + sy + 1] - u[o + sz + sy], u[o + sz + sy]);
        const float a1 = fmaf(wy, e11 - e01, e01);
        uf[i] = fmaf(wz, a1 - a0, a0);
    }
}

// ---------------------------------------------------------------------------
// L-BFGS initial Hessian (Sec. 2.3.2).  The clamped second difference of n
// nodes is diagonalised by the orthonormal DCT-II C[k][i] = s_k cos(pi k
// (2i+1) / 2n) (s_0 = sqrt(1/n), s_k = sqrt(2/n)); k (2i+1) is reduced mod 4n
// incrementally, so the cosines come from one table of 4n values.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_dct_axis(NodeGeom G, int axis, int inv, const float* __restrict__ costab,
                                                 const float* __restrict__ in, float* __restrict__ out) {
    const unsigned int total = 3u * (unsigned int)G.N;
    const int n = axis == 0 ? G.n0 : (axis == 1 ? G.n1 : G.n2);
    const int stride = axis == 0 ? 1 : (axis == 1 ? G.n0 : G.n0 * G.n1);
    const int n4 = 4 * n;
    const float s0 = sqrtf(1.f / (float)n), s1 = sqrtf(2.f / (float)n);
    for (unsigned int e = blockIdx.x * NT + threadIdx.x; e < total; e += gridDim.x * NT) {
        int c, nd, ix, iy, iz;
        node_coords(e, G, c, nd, ix, iy, iz);
        const int k = axis == 0 ? ix : (axis == 1 ? iy : iz);
        const float* line = in + (e - (unsigned int)(k * stride));
        float acc = 0.f;
        if (!inv) {  // out[k] = s_k sum_i cos(pi k (2i+1) / 2n) in[i]
            const int step = (2 * k) % n4;
            int m = k % n4;
            for (int i = 0; i < n; ++i) {
                acc = fmaf(__ldg(costab + m), __ldg(line + i * stride), acc);
                m += step;
                if (m >= n4) m -= n4;
            }
            acc *= (k == 0) ? s0 : s1;
        } else {     // out[i] = sum_j s_j cos(pi j (2i+1) / 2n) in[j], i = k
            const int step = 2 * k + 1;
            int m = 0;
            for (int j = 0; j < n; ++j) {
                acc = fmaf(((j == 0) ? s0 : s1) * __ldg(costab + m), __ldg(line + j * stride), acc);
                m += step;
                if (m >= n4) m -= n4;
            }
        }
        out[e] = acc;
    }
}

__global__ void __launch_bounds__(NT) k_h0_scale(NodeGeom G, const float* __restrict__ mu, float c, float gamma,
                                                 float* __restrict__ a) {
    const unsigned int total = 3u * (unsigned int)G.N;
    for (unsigned int e = blockIdx.x * NT + threadIdx.x; e < total; e += gridDim.x * NT) {
        int cc, nd, ix, iy, iz;
        node_coords(e, G, cc, nd, ix, iy, iz);
        const float lam = mu[ix] + mu[G.n0 + iy] + mu[G.n0 + G.n1 + iz];
        a[e] = a[e] / fmaf(c * lam, lam, gamma);
    }
}

__global__ void __launch_bounds__(NT) k_lbfgs_q(long long n, double rho, const double* dot,
                                                const float* __restrict__ y, float* __restrict__ q, double* a_out) {
    const double a = rho * dot[0];
    const float af = (float)a;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        q[i] = fmaf(-af, y[i], q[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a_out = a;
}

__global__ void __launch_bounds__(NT) k_lbfgs_r(long long n, double rho, const double* dot, const double* a,
                                                const float* __restrict__ s, float* __restrict__ r) {
    const float coef = (float)(a[0] - rho * dot[0]);
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        r[i] = fmaf(coef, s[i], r[i]);
}

// ---------------------------------------------------------------------------
// Batched forms.  The per-pair parameter block is copied into shared memory
// and the single-problem body runs on it unchanged, so every pair's results
// equal those of its own plan bit for bit.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void copy_to_shared(T& dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "parameter blocks are whole words");
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x)
        reinterpret_cast<int*>(&dst)[i] = __ldg(reinterpret_cast<const int*>(src) + i);
}

__device__ __forceinline__ void queue_release(const BatchQueue& Q) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(Q.done, 1u) == gridDim.x - 1) {  // every CTA has left the queue
            *Q.next = 0u;
            *Q.done = 0u;
            __threadfence();
        }
    }
}

// KIND 0..2: image pass mode (NGF or SSD per pair), 3/4: NGF diagonal (span 3/4), 5: SSD diagonal,
// 7, 8: NGF diagonal of span 3 with 2 or 3 shuffle steps fixed at compile time;
// SM: shared-memory layout of the NGF image pass
template <int KIND, class SM = ImgSmemC>
__device__ __forceinline__ void batch_image_loop(const BatchQueue& Q, const BatchImgTable& T) {
    __shared__ int4 item;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int k = atomicAdd(Q.next, 1u);
            item = (k < (unsigned int)Q.nitems) ? Q.items[k] : make_int4(-1, 0, 0, 0);
        }
        __syncthreads();
        const int4 it = item;
        if (it.x < 0) break;
        if (!Q.active || Q.active[it.x]) {
            const ImgParams& Ps = T.p[it.x - Q.pair0];
            if (KIND == 3) diag_pass<3>(Ps, it.y, it.z, it.w);
            else if (KIND == 7 || KIND == 8) diag_pass<3, (KIND == 7 || KIND == 8) ? KIND - 5 : 0>(Ps, it.y, it.z, it.w);
            else if (KIND == 4) diag_pass<4>(Ps, it.y, it.z, it.w);
            else if (KIND == 5) ssd_pass<MODE_SSD_DIAG>(Ps, it.y, it.z, it.w);
            else if (T.ssd[it.x - Q.pair0]) ssd_pass<KIND>(Ps, it.y, it.z, it.w);
            else image_pass<KIND, SM>(Ps, it.y, it.z, it.w);
        }
        __syncthreads();
    }
    queue_release(Q);
}

__global__ void __launch_bounds__(NT, 2) k_batch_image_obj(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_OBJ>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_image_grad(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_GRAD>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_image_hess(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_HESS>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_image_obj_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_OBJ, ImgSmemW>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_image_grad_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_GRAD, ImgSmemW>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_image_hess_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<MODE_HESS, ImgSmemW>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_diag(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<3>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_diag_s2(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<7>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_diag_s3(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<8>(Q, T);
}
__global__ void __launch_bounds__(NT, 1) k_batch_diag4(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<4>(Q, T);
}
__global__ void __launch_bounds__(NT, 2) k_batch_ssd_diag(const BatchQueue Q, const __grid_constant__ BatchImgTable T) {
    batch_image_loop<5>(Q, T);
}

template <class ARGS, class BODY>
__device__ __forceinline__ void batch_nodal(const ARGS* table, const BatchSegs& S, BODY body) {
    __shared__ ARGS A;
    const int k = __ldg(S.pair_of + blockIdx.x);
    if (S.active && !S.active[k]) return;
    copy_to_shared(A, table + k);
    __syncthreads();
    body(A, (unsigned int)(blockIdx.x - S.first[k]), (unsigned int)(S.first[k + 1] - S.first[k]));
}

__global__ void __launch_bounds__(NT) k_batch_lap(const LapArgs* table, const BatchSegs S) {
    batch_nodal(table, S, [](const LapArgs& a, unsigned int b, unsigned int n) {
        lap_body(a.G, a.x, a.L, a.part, a.count, a.out, a.scale, b, n);
    });
}
__global__ void __launch_bounds__(NT) k_batch_combine(const CombineParams* table, const BatchSegs S) {
    batch_nodal(table, S, [](const CombineParams& a, unsigned int b, unsigned int n) { combine_body(a, b, n); });
}
__global__ void __launch_bounds__(NT) k_batch_pcg_init(const PcgParams* table, const BatchSegs S) {
    batch_nodal(table, S, [](const PcgParams& a, unsigned int b, unsigned int n) { pcg_init_body(a, b, n); });
}
__global__ void __launch_bounds__(NT) k_batch_pcg_update(const PcgParams* table, const BatchSegs S) {
    batch_nodal(table, S, [](const PcgParams& a, unsigned int b, unsigned int n) { pcg_update_body(a, b, n); });
}
__global__ void __launch_bounds__(NT) k_batch_pcg_dir(const PcgParams* table, const BatchSegs S) {
    batch_nodal(table, S, [](const PcgParams& a, unsigned int b, unsigned int n) { pcg_dir_body(a, b, n); });
}
__global__ void __launch_bounds__(NT) k_batch_dot(const DotArgs* table, const BatchSegs S) {
    batch_nodal(table, S, [](const DotArgs& a, unsigned int b, unsigned int n) { dot_body(a, b, n); });
}
__global__ void __launch_bounds__(NT) k_batch_axpy(const AxpyArgs* table, const BatchSegs S) {
    batch_nodal(table, S, [](const AxpyArgs& a, unsigned int b, unsigned int n) { axpy_body(a, b, n); });
}

}  // namespace ngf
