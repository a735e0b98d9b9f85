/*
 * FP64 CPU oracle for the matrix-free NGF + curvature registration method.
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline use it; the CUDA library never does).  See ngf_oracle.h for the
 * conventions.  Every operator is the plain chain-rule definition evaluated
 * with staged full-size arrays, in the order the paper states it; nothing is
 * fused, blocked or reordered.  OpenMP only splits loops whose iterations
 * write disjoint outputs; all scatters (P^T, dr^T) run serially.
 */
#include "ngf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* grid helpers                                                            */
/* ---------------------------------------------------------------------- */

static long nvox(const orc_level* L) { return (long)L->m[0] * L->m[1] * L->m[2]; }
static long nnod(const orc_level* L) { return (long)L->n[0] * L->n[1] * L->n[2]; }
/* The 2-D method (one image plane, one node plane): the paper states every
 * operator for d = 2 and d = 3 alike (Sec. 2.2); in 2-D the cell volumes are
 * h_x h_y and hy_x hy_y, the template is interpolated bilinearly in the
 * plane, and there are no z differences (the clamped ones below vanish). */
static int planar(const orc_level* L) { return L->m[2] == 1 && L->n[2] == 1; }
static double hbar(const orc_level* L) { return planar(L) ? L->h[0] * L->h[1] : L->h[0] * L->h[1] * L->h[2]; }
/* node spacing: the nodal grid spans the image domain [0, m h] (Sec. 2.2);
 * the single node plane of the 2-D method has no spacing (1 is a placeholder) */
static double hy(const orc_level* L, int l) {
    return L->n[l] > 1 ? (double)L->m[l] * L->h[l] / (double)(L->n[l] - 1) : 1.0;
}
static double hbary(const orc_level* L) { return hy(L, 0) * hy(L, 1) * (planar(L) ? 1.0 : hy(L, 2)); }
/* node planes touched by one image plane: 1 in 2-D, 2 (trilinear) in 3-D */
static int zspan(const orc_level* L) { return planar(L) ? 1 : 2; }

static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Neighbour of voxel (x,y,z) in direction k in K = {-z,-y,-x,0,+x,+y,+z}
 * with the clamped indices of Eq. (boundary_conditions). */
static const int KAX[7] = {2, 1, 0, -1, 0, 1, 2};
static const int KDIR[7] = {-1, -1, -1, 0, 1, 1, 1};

static long nb(const orc_level* L, long x, long y, long z, int k) {
    long c[3] = {x, y, z};
    if (KDIR[k] != 0) {
        int a = KAX[k];
        c[a] = clampl(c[a] + KDIR[k], 0, L->m[a] - 1);
    }
    return c[0] + (long)L->m[0] * (c[1] + (long)L->m[1] * c[2]);
}

/* Trilinear weights of Eq. (grid_conversion): image index v on an axis with
 * m cells and n nodes lies at node coordinate c = (v + 1/2)(n - 1)/m; its two
 * nodes are floor(c) and floor(c)+1 with weights 1 - frac and frac. */
static void pw(int v, int m, int n, long* f, double* w1) {
    double c = ((double)v + 0.5) * (double)(n - 1) / (double)m;
    double fl = floor(c);
    *f = (long)fl;
    *w1 = c - fl;
}

/* ---------------------------------------------------------------------- */
/* P and P^T (Sec. 4.3)                                                    */
/* ---------------------------------------------------------------------- */

void orc_P(const orc_level* L, const double* u, double* uh) {
    const long M = nvox(L), N = nnod(L);
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
    const long n0 = L->n[0], n1 = L->n[1];
#pragma omp parallel for
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long fx, fy, fz;
                double wx, wy, wz;
                pw(x, m0, L->n[0], &fx, &wx);
                pw(y, m1, L->n[1], &fy, &wy);
                pw(z, m2, L->n[2], &fz, &wz);
                long i = x + (long)m0 * (y + (long)m1 * z);
                for (int d = 0; d < 3; ++d) {
                    double acc = 0.0;
                    for (int c = 0; c < zspan(L); ++c)
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) {
                                double w = (a ? wx : 1.0 - wx) * (b ? wy : 1.0 - wy) * (c ? wz : 1.0 - wz);
                                long node = (fx + a) + n0 * ((fy + b) + n1 * (fz + c));
                                acc += w * u[d * N + node];
                            }
                    uh[d * M + i] = acc;
                }
            }
}

void orc_PT(const orc_level* L, const double* uh, double* out) {
    const long M = nvox(L), N = nnod(L);
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
    const long n0 = L->n[0], n1 = L->n[1];
    memset(out, 0, sizeof(double) * 3 * N);
    /* column sums of P: every voxel scatters into its 8 nodes (serial) */
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long fx, fy, fz;
                double wx, wy, wz;
                pw(x, m0, L->n[0], &fx, &wx);
                pw(y, m1, L->n[1], &fy, &wy);
                pw(z, m2, L->n[2], &fz, &wz);
                long i = x + (long)m0 * (y + (long)m1 * z);
                for (int c = 0; c < zspan(L); ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) {
                            double w = (a ? wx : 1.0 - wx) * (b ? wy : 1.0 - wy) * (c ? wz : 1.0 - wz);
                            long node = (fx + a) + n0 * ((fy + b) + n1 * (fz + c));
                            for (int d = 0; d < 3; ++d) out[d * N + node] += w * uh[d * M + i];
                        }
            }
}

/* ---------------------------------------------------------------------- */
/* template warp and dT/dP (Sec. 2.2, Eq. dT)                               */
/* ---------------------------------------------------------------------- */

static double tval(const orc_level* L, const double* T, long x, long y, long z) {
    if (x < 0 || y < 0 || z < 0 || x >= L->m[0] || y >= L->m[1] || z >= L->m[2]) return 0.0;
    return T[x + (long)L->m[0] * (y + (long)L->m[1] * z)];
}

void orc_warp(const orc_level* L, const double* T, const double* uh, double* Tw, double* dT) {
    const long M = nvox(L);
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
#pragma omp parallel for
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                long coord[3] = {x, y, z};
                long c[3];
                double t[3];
                int inside = 1;
                /* continuous voxel coordinate xi = index + (P u)/h (displacement
                 * form); the cell is floor(xi), so knots take the forward cell */
                for (int l = 0; l < 3; ++l) {
                    /* 2-D: the sample stays in the image plane */
                    double d = (l == 2 && planar(L)) ? 0.0 : uh[l * M + i] / L->h[l];
                    if (!(fabs(d) < 1.0e9)) { inside = 0; c[l] = 0; t[l] = 0.0; continue; }
                    double fl = floor(d);
                    c[l] = coord[l] + (long)fl;
                    t[l] = d - fl;
                    if (c[l] < -1 || c[l] > L->m[l] - 1) inside = 0;
                }
                if (!inside) {
                    Tw[i] = 0.0;
                    dT[i] = dT[M + i] = dT[2 * M + i] = 0.0;
                    continue;
                }
                double v[2][2][2];
                for (int g = 0; g < 2; ++g)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) v[g][b][a] = tval(L, T, c[0] + a, c[1] + b, c[2] + g);
                double w[3][2];
                for (int l = 0; l < 3; ++l) { w[l][0] = 1.0 - t[l]; w[l][1] = t[l]; }
                double val = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
                for (int g = 0; g < 2; ++g)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) val += w[0][a] * w[1][b] * w[2][g] * v[g][b][a];
                for (int g = 0; g < 2; ++g)
                    for (int b = 0; b < 2; ++b) gx += w[1][b] * w[2][g] * (v[g][b][1] - v[g][b][0]);
                for (int g = 0; g < 2; ++g)
                    for (int a = 0; a < 2; ++a) gy += w[0][a] * w[2][g] * (v[g][1][a] - v[g][0][a]);
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) gz += w[0][a] * w[1][b] * (v[1][b][a] - v[0][b][a]);
                Tw[i] = val;
                dT[i] = gx / L->h[0];
                dT[M + i] = gy / L->h[1];
                dT[2 * M + i] = planar(L) ? 0.0 : gz / L->h[2];  /* 2-D: bilinear, no z derivative */
            }
}

/* ---------------------------------------------------------------------- */
/* NGF residual and its Jacobian (Sec. 3.2, Sec. 4.1.1)                     */
/* ---------------------------------------------------------------------- */

void orc_short_grad(const orc_level* L, const double* I, double* g) {
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
#pragma omp parallel for
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                /* backward differences (k = -x,-y,-z), then forward ones */
                g[6 * i + 0] = (I[i] - I[nb(L, x, y, z, 2)]) / L->h[0];
                g[6 * i + 1] = (I[i] - I[nb(L, x, y, z, 1)]) / L->h[1];
                g[6 * i + 2] = (I[i] - I[nb(L, x, y, z, 0)]) / L->h[2];
                g[6 * i + 3] = (I[nb(L, x, y, z, 4)] - I[i]) / L->h[0];
                g[6 * i + 4] = (I[nb(L, x, y, z, 5)] - I[i]) / L->h[1];
                g[6 * i + 5] = (I[nb(L, x, y, z, 6)] - I[i]) / L->h[2];
            }
}

static double dot6(const double* a, const double* b) {
    double s = 0.0;
    for (int k = 0; k < 6; ++k) s += a[k] * b[k];
    return s;
}

void orc_residual(const orc_level* L, const double* R, const double* Tw, double* r) {
    const long M = nvox(L);
    double* gT = (double*)malloc(sizeof(double) * 6 * M);
    double* gR = (double*)malloc(sizeof(double) * 6 * M);
    orc_short_grad(L, Tw, gT);
    orc_short_grad(L, R, gR);
    const double tr = L->tau * L->rho;
#pragma omp parallel for
    for (long i = 0; i < M; ++i) {
        double num = 0.5 * dot6(gT + 6 * i, gR + 6 * i) + tr;
        double nT = sqrt(0.5 * dot6(gT + 6 * i, gT + 6 * i) + L->tau * L->tau);
        double nR = sqrt(0.5 * dot6(gR + 6 * i, gR + 6 * i) + L->rho * L->rho);
        r[i] = num / (nT * nR);
    }
    free(gT);
    free(gR);
}

void orc_rho_hat(const orc_level* L, const double* R, const double* Tw, double* rh) {
    const long M = nvox(L);
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
    double* gT = (double*)malloc(sizeof(double) * 6 * M);
    double* gR = (double*)malloc(sizeof(double) * 6 * M);
    orc_short_grad(L, Tw, gT);
    orc_short_grad(L, R, gR);
    const double tr = L->tau * L->rho;
#pragma omp parallel for
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                double N_ = 0.5 * dot6(gT + 6 * i, gR + 6 * i) + tr;                  /* r_{1,i} */
                double A = sqrt(0.5 * dot6(gT + 6 * i, gT + 6 * i) + L->tau * L->tau); /* ||grad T||_tau */
                double B = sqrt(0.5 * dot6(gR + 6 * i, gR + 6 * i) + L->rho * L->rho); /* ||grad R||_rho */
                double sum = 0.0;
                for (int k = 0; k < 7; ++k) {
                    if (k == 3) continue;
                    long j = nb(L, x, y, z, k);
                    /* Eq. (rho) */
                    double rk = (R[j] - R[i]) / (A * B) - N_ * (Tw[j] - Tw[i]) / (A * A * A * B);
                    /* Eq. (hatRho): h_hat_k = 1 / (2 h_|k|^2) */
                    double hh = 1.0 / (2.0 * L->h[KAX[k]] * L->h[KAX[k]]);
                    rh[7 * i + k] = hh * rk;
                    sum += hh * rk;
                }
                rh[7 * i + 3] = -sum;
            }
    free(gT);
    free(gR);
}

void orc_dr(const orc_level* L, const double* rh, const double* s, double* v) {
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
#pragma omp parallel for
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                double acc = 0.0;
                /* row i of dr, Eq. (dr): entries at the (clamped) neighbours */
                for (int k = 0; k < 7; ++k) acc += rh[7 * i + k] * s[nb(L, x, y, z, k)];
                v[i] = acc;
            }
}

void orc_drT(const orc_level* L, const double* rh, const double* v, double* t) {
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
    memset(t, 0, sizeof(double) * nvox(L));
    /* transpose by scattering each row (serial) */
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                for (int k = 0; k < 7; ++k) t[nb(L, x, y, z, k)] += rh[7 * i + k] * v[i];
            }
}

/* ---------------------------------------------------------------------- */
/* curvature (Eqs. CURV_discretized, laplace_discretized, curvatureMF)      */
/* ---------------------------------------------------------------------- */

void orc_lap(const orc_level* L, const double* u, double* out) {
    const long N = nnod(L);
    const long n0 = L->n[0], n1 = L->n[1], n2 = L->n[2];
    const double ih2[3] = {1.0 / (hy(L, 0) * hy(L, 0)), 1.0 / (hy(L, 1) * hy(L, 1)), 1.0 / (hy(L, 2) * hy(L, 2))};
    for (int d = 0; d < 3; ++d) {
        const double* ud = u + d * N;
        double* od = out + d * N;
#pragma omp parallel for
        for (long z = 0; z < n2; ++z)
            for (long y = 0; y < n1; ++y)
                for (long x = 0; x < n0; ++x) {
                    long i = x + n0 * (y + n1 * z);
                    double c = ud[i];
                    double lx = ud[clampl(x - 1, 0, n0 - 1) + n0 * (y + n1 * z)] - 2.0 * c +
                                ud[clampl(x + 1, 0, n0 - 1) + n0 * (y + n1 * z)];
                    double ly = ud[x + n0 * (clampl(y - 1, 0, n1 - 1) + n1 * z)] - 2.0 * c +
                                ud[x + n0 * (clampl(y + 1, 0, n1 - 1) + n1 * z)];
                    double lz = ud[x + n0 * (y + n1 * clampl(z - 1, 0, n2 - 1))] - 2.0 * c +
                                ud[x + n0 * (y + n1 * clampl(z + 1, 0, n2 - 1))];
                    od[i] = lx * ih2[0] + ly * ih2[1] + lz * ih2[2];
                }
    }
}

void orc_curvature_apply(const orc_level* L, const double* p, double* q, double* Sp) {
    const long N = nnod(L);
    double* Lp = (double*)malloc(sizeof(double) * 3 * N);
    orc_lap(L, p, Lp);
    if (Sp) {
        double s = 0.0;
        for (long i = 0; i < 3 * N; ++i) s += Lp[i] * Lp[i];
        *Sp = hbary(L) * s;
    }
    if (q) {
        orc_lap(L, Lp, q);
        const double c = 2.0 * hbary(L);
        for (long i = 0; i < 3 * N; ++i) q[i] *= c;
    }
    free(Lp);
}

/* ---------------------------------------------------------------------- */
/* objective, gradient, Gauss-Newton Hessian-vector product                 */
/* ---------------------------------------------------------------------- */

void orc_objective(const orc_level* L, const double* R, const double* T, const double* u, double* D,
                   double* S) {
    const long M = nvox(L);
    double* uh = (double*)malloc(sizeof(double) * 3 * M);
    double* Tw = (double*)malloc(sizeof(double) * M);
    double* dT = (double*)malloc(sizeof(double) * 3 * M);
    double* r = (double*)malloc(sizeof(double) * M);
    orc_P(L, u, uh);
    orc_warp(L, T, uh, Tw, dT);
    double s = 0.0;
    if (L->distance == ORC_DIST_SSD) { /* D = hbar/2 sum (T(x + Pu) - R)^2 */
        for (long i = 0; i < M; ++i) s += (Tw[i] - R[i]) * (Tw[i] - R[i]);
        *D = 0.5 * hbar(L) * s;
    } else {
        orc_residual(L, R, Tw, r);
        for (long i = 0; i < M; ++i) s += 1.0 - r[i] * r[i];
        *D = hbar(L) * s; /* Eq. (NGF_discretized_ri), midpoint rule */
    }
    orc_curvature_apply(L, u, NULL, S);
    free(uh);
    free(Tw);
    free(dT);
    free(r);
}

void orc_gradient(const orc_level* L, const double* R, const double* T, const double* u, double* grad,
                  double* D, double* S) {
    const long M = nvox(L), N = nnod(L);
    double* uh = (double*)malloc(sizeof(double) * 3 * M);
    double* Tw = (double*)malloc(sizeof(double) * M);
    double* dT = (double*)malloc(sizeof(double) * 3 * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* rh = (double*)malloc(sizeof(double) * 7 * M);
    double* dpsi = (double*)malloc(sizeof(double) * M);
    double* g = (double*)malloc(sizeof(double) * M);
    double* gh = (double*)malloc(sizeof(double) * 3 * M);
    double* cg = (double*)malloc(sizeof(double) * 3 * N);
    orc_P(L, u, uh);
    orc_warp(L, T, uh, Tw, dT);
    double s = 0.0;
    if (L->distance == ORC_DIST_SSD) {
        /* r = T(x + Pu) - R, d psi / d r = hbar r, dr = I */
        for (long i = 0; i < M; ++i) s += (Tw[i] - R[i]) * (Tw[i] - R[i]);
        *D = 0.5 * hbar(L) * s;
        for (long i = 0; i < M; ++i) g[i] = hbar(L) * (Tw[i] - R[i]);
    } else {
        orc_residual(L, R, Tw, r);
        orc_rho_hat(L, R, Tw, rh);
        for (long i = 0; i < M; ++i) s += 1.0 - r[i] * r[i];
        *D = hbar(L) * s;
        /* (d psi / d r)^T = -2 hbar r, Eq. (dPsi) */
        for (long i = 0; i < M; ++i) dpsi[i] = -2.0 * hbar(L) * r[i];
        /* dr^T (d psi / d r)^T */
        orc_drT(L, rh, dpsi, g);
    }
    /* dT^T: the three diagonal blocks of Eq. (dT) */
    for (int d = 0; d < 3; ++d)
        for (long i = 0; i < M; ++i) gh[d * M + i] = dT[d * M + i] * g[i];
    /* P^T */
    orc_PT(L, gh, grad);
    /* + alpha grad S = alpha 2 hbar^y Lap Lap u, Eq. (curvatureMF) */
    orc_curvature_apply(L, u, cg, S);
    for (long i = 0; i < 3 * N; ++i) grad[i] += L->alpha * cg[i];
    free(uh);
    free(Tw);
    free(dT);
    free(r);
    free(rh);
    free(dpsi);
    free(g);
    free(gh);
    free(cg);
}

void orc_hessvec(const orc_level* L, const double* R, const double* T, const double* u, const double* p,
                 double* q) {
    const long M = nvox(L), N = nnod(L);
    double* uh = (double*)malloc(sizeof(double) * 3 * M);
    double* ph = (double*)malloc(sizeof(double) * 3 * M);
    double* Tw = (double*)malloc(sizeof(double) * M);
    double* dT = (double*)malloc(sizeof(double) * 3 * M);
    double* rh = (double*)malloc(sizeof(double) * 7 * M);
    double* sv = (double*)malloc(sizeof(double) * M);
    double* v = (double*)malloc(sizeof(double) * M);
    double* t = (double*)malloc(sizeof(double) * M);
    double* qh = (double*)malloc(sizeof(double) * 3 * M);
    double* cq = (double*)malloc(sizeof(double) * 3 * N);
    orc_P(L, u, uh);
    orc_warp(L, T, uh, Tw, dT);
    /* H p = 2 hbar P^T dT^T dr^T dr dT P p, Eq. (NGF_discretized_hessian);
     * the sign is that of the PSD Gauss-Newton matrix (Sec. 3.2).
     * SSD: H p = hbar P^T dT^T dT P p (dr = I, psi'' = hbar) */
    orc_P(L, p, ph);
    for (long i = 0; i < M; ++i) sv[i] = dT[i] * ph[i] + dT[M + i] * ph[M + i] + dT[2 * M + i] * ph[2 * M + i];
    if (L->distance == ORC_DIST_SSD) {
        for (int d = 0; d < 3; ++d)
            for (long i = 0; i < M; ++i) qh[d * M + i] = hbar(L) * dT[d * M + i] * sv[i];
    } else {
        orc_rho_hat(L, R, Tw, rh);
        orc_dr(L, rh, sv, v);
        orc_drT(L, rh, v, t);
        for (int d = 0; d < 3; ++d)
            for (long i = 0; i < M; ++i) qh[d * M + i] = 2.0 * hbar(L) * dT[d * M + i] * t[i];
    }
    orc_PT(L, qh, q);
    /* + alpha grad^2 S p, Eq. (curv_hessMult) */
    orc_curvature_apply(L, p, cq, NULL);
    for (long i = 0; i < 3 * N; ++i) q[i] += L->alpha * cq[i];
    free(uh);
    free(ph);
    free(Tw);
    free(dT);
    free(rh);
    free(sv);
    free(v);
    free(t);
    free(qh);
    free(cq);
}

/* Diagonal of H + alpha grad^2 S.  With J = dr dT P (rows = voxels), the
 * diagonal of H = 2 hbar J^T J is 2 hbar times the column sums of J squared;
 * each row of J is formed explicitly from the 7 entries of its dr row and the
 * 8 trilinear weights of each entry's voxel.  The curvature part is
 * 2 hbar^y times the column sums of the squared entries of the (symmetric)
 * Laplacian matrix. */
void orc_gn_diagonal(const orc_level* L, const double* R, const double* T, const double* u, double* diag) {
    const long M = nvox(L), N = nnod(L);
    const int m0 = L->m[0], m1 = L->m[1], m2 = L->m[2];
    const long n0 = L->n[0], n1 = L->n[1], n2 = L->n[2];
    double* uh = (double*)malloc(sizeof(double) * 3 * M);
    double* Tw = (double*)malloc(sizeof(double) * M);
    double* dT = (double*)malloc(sizeof(double) * 3 * M);
    double* rh = (double*)malloc(sizeof(double) * 7 * M);
    orc_P(L, u, uh);
    orc_warp(L, T, uh, Tw, dT);
    memset(diag, 0, sizeof(double) * 3 * N);
    long ent_n[56];
    double ent_v[56];
    const int ssd = L->distance == ORC_DIST_SSD;
    if (!ssd) orc_rho_hat(L, R, Tw, rh);
    for (int z = 0; z < m2; ++z)
        for (int y = 0; y < m1; ++y)
            for (int x = 0; x < m0; ++x) {
                long i = x + (long)m0 * (y + (long)m1 * z);
                for (int d = 0; d < 3; ++d) {
                    int cnt = 0;
                    for (int k = 0; k < 7; ++k) {
                        /* SSD: the row of dr is the unit row (only k = 0, coefficient 1) */
                        if (ssd && k != 3) continue;
                        long j = nb(L, x, y, z, k);
                        long jx = j % m0, jy = (j / m0) % m1, jz = j / ((long)m0 * m1);
                        double c = (ssd ? 1.0 : rh[7 * i + k]) * dT[d * M + j];
                        long fx, fy, fz;
                        double wx, wy, wz;
                        pw((int)jx, m0, L->n[0], &fx, &wx);
                        pw((int)jy, m1, L->n[1], &fy, &wy);
                        pw((int)jz, m2, L->n[2], &fz, &wz);
                        for (int cc = 0; cc < zspan(L); ++cc)
                            for (int b = 0; b < 2; ++b)
                                for (int a = 0; a < 2; ++a) {
                                    double w = (a ? wx : 1.0 - wx) * (b ? wy : 1.0 - wy) * (cc ? wz : 1.0 - wz);
                                    long node = (fx + a) + n0 * ((fy + b) + n1 * (fz + cc));
                                    int e = 0;
                                    while (e < cnt && ent_n[e] != node) ++e;
                                    if (e == cnt) { ent_n[cnt] = node; ent_v[cnt] = 0.0; ++cnt; }
                                    ent_v[e] += c * w;
                                }
                    }
                    for (int e = 0; e < cnt; ++e)
                        diag[d * N + ent_n[e]] += (ssd ? 1.0 : 2.0) * hbar(L) * ent_v[e] * ent_v[e];
                }
            }
    /* curvature: squared entries of each Laplacian row, summed by column */
    double* cd = (double*)calloc(N, sizeof(double));
    const double ih2[3] = {1.0 / (hy(L, 0) * hy(L, 0)), 1.0 / (hy(L, 1) * hy(L, 1)), 1.0 / (hy(L, 2) * hy(L, 2))};
    for (long z = 0; z < n2; ++z)
        for (long y = 0; y < n1; ++y)
            for (long x = 0; x < n0; ++x) {
                long col[7];
                double val[7];
                int cnt = 0;
                long cidx[3] = {x, y, z};
                long nn[3] = {n0, n1, n2};
                for (int a = 0; a < 3; ++a)
                    for (int s = -1; s <= 1; ++s) {
                        long c3[3] = {cidx[0], cidx[1], cidx[2]};
                        c3[a] = clampl(c3[a] + s, 0, nn[a] - 1);
                        long node = c3[0] + n0 * (c3[1] + n1 * c3[2]);
                        double w = (s == 0 ? -2.0 : 1.0) * ih2[a];
                        int e = 0;
                        while (e < cnt && col[e] != node) ++e;
                        if (e == cnt) { col[cnt] = node; val[cnt] = 0.0; ++cnt; }
                        val[e] += w;
                    }
                for (int e = 0; e < cnt; ++e) cd[col[e]] += val[e] * val[e];
            }
    for (int d = 0; d < 3; ++d)
        for (long n = 0; n < N; ++n) diag[d * N + n] += L->alpha * 2.0 * hbary(L) * cd[n];
    free(cd);
    free(uh);
    free(Tw);
    free(dT);
    free(rh);
}

/* ---------------------------------------------------------------------- */
/* PCG (Sec. 2.3.1) with the Jacobi preconditioner                          */
/* ---------------------------------------------------------------------- */

static double vdot(long n, const double* a, const double* b) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

void orc_pcg(const orc_level* L, const double* R, const double* T, const double* u, const double* rhs,
             const double* diag, int32_t iters, double rtol, double* x, orc_pcg_info* info) {
    const long n = 3 * nnod(L);
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    /* a zero diagonal entry means a zero row and column: leave it alone */
#define MINV(i) (diag[i] > 0.0 ? 1.0 / diag[i] : 0.0)
    for (long i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = rhs[i];
        z[i] = r[i] * MINV(i);
        d[i] = z[i];
    }
    double delta = vdot(n, r, z);
    double rr = vdot(n, r, r);
    const double bb = rr;
    int status = 0, it = 0;
    for (it = 0; it < iters; ++it) {
        if (delta == 0.0) { status = 1; break; }
        if (rtol > 0.0 && sqrt(rr) <= rtol * sqrt(bb)) { status = 3; break; }
        orc_hessvec(L, R, T, u, d, q);
        double dq = vdot(n, d, q);
        if (!(dq > 0.0) || !isfinite(dq)) { status = 2; break; }
        double a = delta / dq;
        for (long i = 0; i < n; ++i) {
            x[i] += a * d[i];
            r[i] -= a * q[i];
            z[i] = r[i] * MINV(i);
        }
        double dnew = vdot(n, r, z);
        rr = vdot(n, r, r);
        double beta = dnew / delta;
        for (long i = 0; i < n; ++i) d[i] = z[i] + beta * d[i];
        delta = dnew;
    }
#undef MINV
    if (info) {
        info->iters_done = it;
        info->status = status;
        info->delta = delta;
        info->rr = rr;
    }
    free(r);
    free(z);
    free(d);
    free(q);
}

/* ---------------------------------------------------------------------- */
/* Gauss-Newton with Armijo backtracking (Sec. 2.3)                         */
/* ---------------------------------------------------------------------- */

void orc_gn_level(const orc_level* L, const double* R, const double* T, double* u, const orc_gn_options* o,
                  orc_gn_report* rep, double* trace) {
    const long n = 3 * nnod(L);
    double* g = (double*)malloc(sizeof(double) * n);
    double* diag = (double*)malloc(sizeof(double) * n);
    double* rhs = (double*)malloc(sizeof(double) * n);
    double* s = (double*)malloc(sizeof(double) * n);
    double* ut = (double*)malloc(sizeof(double) * n);
    memset(rep, 0, sizeof(*rep));
    double D, S;
    for (int k = 0; k < o->gn_iters; ++k) {
        orc_gradient(L, R, T, u, g, &D, &S);
        double J0 = D + L->alpha * S;
        if (trace) trace[2 * k] = J0;
        double gg = vdot(n, g, g);
        if (gg == 0.0) { rep->status = 8; break; }
        /* the preconditioner is refreshed on the level's schedule and
           otherwise kept from an earlier iterate of the level */
        if (o->diag_every > 0 ? k % o->diag_every == 0 : k == 0) orc_gn_diagonal(L, R, T, u, diag);
        for (long i = 0; i < n; ++i) rhs[i] = -g[i];
        orc_pcg_info info;
        orc_pcg(L, R, T, u, rhs, diag, o->pcg_iters, o->pcg_rtol, s, &info);
        rep->pcg_total += info.iters_done;
        double gs = vdot(n, g, s);
        if (!(gs < 0.0)) { /* not a descent direction: steepest descent */
            for (long i = 0; i < n; ++i) s[i] = -g[i];
            gs = -gg;
        }
        double eta = 1.0;
        int accepted = 0;
        for (int t = 0; t < o->ls_max; ++t) {
            for (long i = 0; i < n; ++i) ut[i] = u[i] + eta * s[i];
            double Dt, St;
            orc_objective(L, R, T, ut, &Dt, &St);
            rep->ls_trials++;
            if (Dt + L->alpha * St <= J0 + o->armijo_c1 * eta * gs) { accepted = 1; break; }
            eta *= 0.5;
        }
        if (trace) trace[2 * k + 1] = accepted ? eta : 0.0;
        if (!accepted) { rep->status = 6; break; }
        memcpy(u, ut, sizeof(double) * n);
        rep->gn_done++;
    }
    orc_objective(L, R, T, u, &D, &S);
    rep->D = D;
    rep->S = S;
    rep->J = D + L->alpha * S;
    if (trace) trace[2 * o->gn_iters] = rep->J;
    free(g);
    free(diag);
    free(rhs);
    free(s);
    free(ut);
}

/* ---------------------------------------------------------------------- */
/* L-BFGS (Sec. 2.3.2)                                                      */
/* ---------------------------------------------------------------------- */

static const double PI_ = 3.14159265358979323846;

/* orthonormal DCT-II of the lines of one component along axis `ax`
 * (inverse = transpose when `inv`) */
static void dct_axis(const orc_level* L, int ax, int inv, double* a) {
    const int n = L->n[ax];
    const long stride = ax == 0 ? 1 : (ax == 1 ? (long)L->n[0] : (long)L->n[0] * L->n[1]);
    const long lines = nnod(L) / n;
    double* in = (double*)malloc(sizeof(double) * n);
    for (long ln = 0; ln < lines; ++ln) {
        /* first element of line ln: the other two indices in lexicographic order */
        long base;
        if (ax == 0) base = ln * n;
        else if (ax == 1) base = (ln % L->n[0]) + (ln / L->n[0]) * (long)L->n[0] * L->n[1];
        else base = ln;
        for (int i = 0; i < n; ++i) in[i] = a[base + i * stride];
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                /* C[row][col] = s_row cos(pi row (2 col + 1) / 2n) */
                const int row = inv ? i : k, col = inv ? k : i;
                const double sr = row == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
                acc += sr * cos(PI_ * row * (2.0 * col + 1.0) / (2.0 * n)) * in[i];
            }
            a[base + k * stride] = acc;
        }
    }
    free(in);
}

void orc_h0_solve(const orc_level* L, double gamma, const double* q, double* r) {
    const long N = nnod(L);
    const double c = L->alpha * 2.0 * hbary(L);
    memcpy(r, q, sizeof(double) * 3 * N);
    for (int comp = 0; comp < 3; ++comp) {
        double* a = r + comp * N;
        for (int ax = 0; ax < 3; ++ax) dct_axis(L, ax, 0, a);
        for (int z = 0; z < L->n[2]; ++z)
            for (int y = 0; y < L->n[1]; ++y)
                for (int x = 0; x < L->n[0]; ++x) {
                    const int kk[3] = {x, y, z};
                    double lam = 0.0;
                    for (int l = 0; l < 3; ++l) {
                        const double sn = sin(PI_ * kk[l] / (2.0 * L->n[l]));
                        lam -= 4.0 * sn * sn / (hy(L, l) * hy(L, l));
                    }
                    a[x + (long)L->n[0] * (y + (long)L->n[1] * z)] /= c * lam * lam + gamma;
                }
        for (int ax = 2; ax >= 0; --ax) dct_axis(L, ax, 1, a);
    }
}

void orc_lbfgs_direction(const orc_level* L, double gamma, int32_t count, const double* S, const double* Y,
                         const double* g, double* d) {
    const long n = 3 * nnod(L);
    double* q = (double*)malloc(sizeof(double) * n);
    double* a = (double*)malloc(sizeof(double) * (count > 0 ? count : 1));
    memcpy(q, g, sizeof(double) * n);
    for (int i = count - 1; i >= 0; --i) { /* newest to oldest */
        const double rho = 1.0 / vdot(n, Y + i * n, S + i * n);
        a[i] = rho * vdot(n, S + i * n, q);
        for (long j = 0; j < n; ++j) q[j] -= a[i] * Y[i * n + j];
    }
    orc_h0_solve(L, gamma, q, d);
    for (int i = 0; i < count; ++i) { /* oldest to newest */
        const double rho = 1.0 / vdot(n, Y + i * n, S + i * n);
        const double b = rho * vdot(n, Y + i * n, d);
        for (long j = 0; j < n; ++j) d[j] += (a[i] - b) * S[i * n + j];
    }
    for (long j = 0; j < n; ++j) d[j] = -d[j];
    free(q);
    free(a);
}

double orc_lbfgs_level(const orc_level* L, const double* R, const double* T, double* u, const orc_lbfgs_options* o,
                       orc_gn_report* rep, double* trace) {
    const long n = 3 * nnod(L);
    const int m = o->memory > 0 ? o->memory : 1;
    double* g = (double*)malloc(sizeof(double) * n);
    double* gp = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    double* ut = (double*)malloc(sizeof(double) * n);
    double* sl = (double*)malloc(sizeof(double) * n); /* last accepted step */
    double* S = (double*)malloc(sizeof(double) * n * m);
    double* Y = (double*)malloc(sizeof(double) * n * m);
    memset(rep, 0, sizeof(*rep));
    double gamma = o->gamma;
    if (!(gamma > 0.0)) { /* mean of the Gauss-Newton diagonal at the start */
        orc_gn_diagonal(L, R, T, u, d);
        double sum = 0.0;
        for (long j = 0; j < n; ++j) sum += d[j];
        gamma = sum / n;
    }
    int count = 0, have_step = 0;
    double D, S_, J0;
    for (int k = 0; k < o->iters; ++k) {
        orc_gradient(L, R, T, u, g, &D, &S_);
        J0 = D + L->alpha * S_;
        if (trace) trace[2 * k] = J0;
        if (have_step) { /* pair from the last accepted step */
            double* yn = (double*)malloc(sizeof(double) * n);
            for (long j = 0; j < n; ++j) yn[j] = g[j] - gp[j];
            if (vdot(n, sl, yn) > 0.0) {
                if (count == m) { /* drop the oldest */
                    memmove(S, S + n, sizeof(double) * n * (m - 1));
                    memmove(Y, Y + n, sizeof(double) * n * (m - 1));
                    --count;
                }
                memcpy(S + count * n, sl, sizeof(double) * n);
                memcpy(Y + count * n, yn, sizeof(double) * n);
                ++count;
            }
            free(yn);
        }
        const double gg = vdot(n, g, g);
        if (gg == 0.0) { rep->status = 8; break; }
        orc_lbfgs_direction(L, gamma, count, S, Y, g, d);
        double gs = vdot(n, g, d);
        if (!(gs < 0.0)) {
            for (long j = 0; j < n; ++j) d[j] = -g[j];
            gs = -gg;
        }
        double eta = 1.0;
        int accepted = 0;
        for (int t = 0; t < o->ls_max; ++t) {
            for (long j = 0; j < n; ++j) ut[j] = u[j] + eta * d[j];
            double Dt, St;
            orc_objective(L, R, T, ut, &Dt, &St);
            rep->ls_trials++;
            if (Dt + L->alpha * St <= J0 + o->armijo_c1 * eta * gs) { accepted = 1; break; }
            eta *= 0.5;
        }
        if (trace) trace[2 * k + 1] = accepted ? eta : 0.0;
        if (!accepted) { rep->status = 6; break; }
        for (long j = 0; j < n; ++j) sl[j] = ut[j] - u[j];
        memcpy(gp, g, sizeof(double) * n);
        memcpy(u, ut, sizeof(double) * n);
        have_step = 1;
        rep->gn_done++;
    }
    orc_objective(L, R, T, u, &D, &S_);
    rep->D = D;
    rep->S = S_;
    rep->J = D + L->alpha * S_;
    if (trace) trace[2 * o->iters] = rep->J;
    free(g);
    free(gp);
    free(d);
    free(ut);
    free(sl);
    free(S);
    free(Y);
    return gamma;
}

/* ---------------------------------------------------------------------- */
/* multilevel (Sec. 2.3, coarse to fine)                                    */
/* ---------------------------------------------------------------------- */

void orc_level_at(const orc_level* finest, int32_t level, orc_level* out) {
    *out = *finest;
    for (int k = 0; k < level; ++k) {
        for (int l = 0; l < (planar(finest) ? 2 : 3); ++l) {  /* 2-D levels stay planar */
            int m = out->m[l];
            int mc = (m + 1) / 2;
            int cells = out->n[l] - 1;
            int cc = (cells + 1) / 2;
            if (cc > mc) cc = mc;
            if (cc < 1) cc = 1;
            out->h[l] = out->h[l] * (double)m / (double)mc;
            out->m[l] = mc;
            out->n[l] = cc + 1;
        }
    }
}

void orc_restrict(const int32_t m[3], const double* img, double* out) {
    const int mc[3] = {(m[0] + 1) / 2, (m[1] + 1) / 2, (m[2] + 1) / 2};
    for (int z = 0; z < mc[2]; ++z)
        for (int y = 0; y < mc[1]; ++y)
            for (int x = 0; x < mc[0]; ++x) {
                double s = 0.0;
                int cnt = 0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) {
                            int fx = 2 * x + a, fy = 2 * y + b, fz = 2 * z + c;
                            if (fx >= m[0] || fy >= m[1] || fz >= m[2]) continue;
                            s += img[fx + (long)m[0] * (fy + (long)m[1] * fz)];
                            ++cnt;
                        }
                out[x + (long)mc[0] * (y + (long)mc[1] * z)] = s / cnt;
            }
}

void orc_prolongate(const int32_t nc[3], const double* uc, const int32_t nf[3], double* uf) {
    const long Nc = (long)nc[0] * nc[1] * nc[2], Nf = (long)nf[0] * nf[1] * nf[2];
    for (int z = 0; z < nf[2]; ++z)
        for (int y = 0; y < nf[1]; ++y)
            for (int x = 0; x < nf[0]; ++x) {
                int idx[3] = {x, y, z};
                long f[3];
                double w[3];
                for (int l = 0; l < 3; ++l) {
                    /* same physical position: fine node i sits at coarse
                     * coordinate i (nc-1)/(nf-1) */
                    double c = nf[l] > 1 ? (double)idx[l] * (double)(nc[l] - 1) / (double)(nf[l] - 1) : 0.0;
                    double fl = floor(c);
                    if (fl > nc[l] - 2) fl = nc[l] - 2;
                    if (fl < 0) fl = 0; /* a single node plane (2-D) */
                    f[l] = (long)fl;
                    w[l] = c - fl;
                }
                long o = x + (long)nf[0] * (y + (long)nf[1] * z);
                for (int d = 0; d < 3; ++d) {
                    double acc = 0.0;
                    for (int c = 0; c < (nc[2] > 1 ? 2 : 1); ++c)
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) {
                                double ww = (a ? w[0] : 1.0 - w[0]) * (b ? w[1] : 1.0 - w[1]) * (c ? w[2] : 1.0 - w[2]);
                                acc += ww * uc[d * Nc + (f[0] + a) + (long)nc[0] * ((f[1] + b) + (long)nc[1] * (f[2] + c))];
                            }
                    uf[d * Nf + o] = acc;
                }
            }
}

void orc_register_multilevel(const orc_level* finest, int32_t levels, const orc_gn_options* o, const double* R,
                             const double* T, const double* u_init, int32_t start_level, double* u_out,
                             orc_gn_report* rep) {
    orc_level* Ls = (orc_level*)malloc(sizeof(orc_level) * levels);
    double** Rs = (double**)malloc(sizeof(double*) * levels);
    double** Ts = (double**)malloc(sizeof(double*) * levels);
    for (int l = 0; l < levels; ++l) orc_level_at(finest, l, &Ls[l]);
    Rs[0] = (double*)R;
    Ts[0] = (double*)T;
    for (int l = 1; l < levels; ++l) {
        long Mc = nvox(&Ls[l]);
        Rs[l] = (double*)malloc(sizeof(double) * Mc);
        Ts[l] = (double*)malloc(sizeof(double) * Mc);
        orc_restrict(Ls[l - 1].m, Rs[l - 1], Rs[l]);
        orc_restrict(Ls[l - 1].m, Ts[l - 1], Ts[l]);
    }
    int start = u_init ? start_level : levels - 1;
    double* u = (double*)calloc(3 * nnod(&Ls[start]), sizeof(double));
    if (u_init) memcpy(u, u_init, sizeof(double) * 3 * nnod(&Ls[start]));
    memset(rep, 0, sizeof(*rep));
    for (int l = start; l >= 0; --l) {
        if (l != start) {
            double* uf = (double*)malloc(sizeof(double) * 3 * nnod(&Ls[l]));
            orc_prolongate(Ls[l + 1].n, u, Ls[l].n, uf);
            free(u);
            u = uf;
        }
        orc_gn_report lr;
        orc_gn_level(&Ls[l], Rs[l], Ts[l], u, o, &lr, NULL);
        rep->gn_done += lr.gn_done;
        rep->pcg_total += lr.pcg_total;
        rep->ls_trials += lr.ls_trials;
        if (lr.status) rep->status = lr.status;
        rep->J = lr.J;
        rep->D = lr.D;
        rep->S = lr.S;
    }
    memcpy(u_out, u, sizeof(double) * 3 * nnod(&Ls[0]));
    free(u);
    for (int l = 1; l < levels; ++l) {
        free(Rs[l]);
        free(Ts[l]);
    }
    free(Rs);
    free(Ts);
    free(Ls);
}
