/*
 * FP64 CPU oracle for the matrix-free NGF + curvature registration method
 * (Koenig, Ruehaak, Derksen, Lellmann, "A matrix-free approach to parallel and
 * memory-efficient deformable image registration").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares no source with the CUDA
 * library: every quantity is evaluated here from its definition in the paper,
 * with staged full-size arrays, in double precision, in the paper's order.
 *
 * Conventions (readings of the paper, all listed in the design notes):
 *  - 0-based indices; image cell centres at (i + 1/2) h (Sec. 2.2);
 *  - lexicographic order, x fastest; vector fields are stored
 *    component-major (all x components, then y, then z) (Sec. 2.2, Table 1);
 *  - n[] are deformation-grid NODES per axis, node spacing
 *    hy_l = m_l h_l / (n_l - 1), so nodes span the image domain (Sec. 2.2);
 *  - the unknown is the displacement u = y - x^y; the warped point of voxel i
 *    is x_i + (P u)_i (P reproduces affine fields, so P y = x + P u).
 */
#ifndef NGF_ORACLE_H
#define NGF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t m[3];   /* image cells per axis                         */
    double  h[3];   /* image spacing per axis                       */
    int32_t n[3];   /* deformation-grid nodes per axis (>= 2)       */
    double  alpha;  /* curvature weight                             */
    double  tau;    /* NGF edge parameter of the template           */
    double  rho;    /* NGF edge parameter of the reference          */
    int32_t distance; /* ORC_DIST_NGF, or ORC_DIST_SSD: the sum of
                         squared differences, whose residual Jacobian
                         is the identity (Sec. 7); tau, rho unused    */
} orc_level;
enum { ORC_DIST_NGF = 0, ORC_DIST_SSD = 1 };

/* ---- building blocks (each cites the passage it evaluates) ------------ */

/* Grid conversion P, Eq. (grid_conversion)/(xi): nodes -> cell centres.
 * u: 3*N, uh: 3*M. */
void orc_P(const orc_level* L, const double* u, double* uh);
/* Transposed grid conversion P^T (Sec. 4.3): uh: 3*M -> out: 3*N. */
void orc_PT(const orc_level* L, const double* uh, double* out);
/* Template warp with trilinear interpolation, zero (Dirichlet) outside
 * (Sec. 2.2), and its spatial derivative dT/dP, Eq. (dT).
 * Tw: M, dT: 3*M. */
void orc_warp(const orc_level* L, const double* T, const double* uh,
              double* Tw, double* dT);
/* Short-difference gradient (Eq. gradient_discretized, clamped neighbours of
 * Eq. boundary_conditions); g: 6 values per voxel, voxel-major. */
void orc_short_grad(const orc_level* L, const double* I, double* g);
/* NGF residual r_i, Eq. (residual). */
void orc_residual(const orc_level* L, const double* R, const double* Tw,
                  double* r);
/* Residual Jacobian coefficients rho_hat_i(k), Eqs. (rho), (hatRho); 7 values
 * per voxel in the order K = {-z,-y,-x,0,+x,+y,+z} (Eq. k). */
void orc_rho_hat(const orc_level* L, const double* R, const double* Tw,
                 double* rh);
/* v = dr s and t = dr^T v with dr from Eq. (dr). */
void orc_dr(const orc_level* L, const double* rh, const double* s, double* v);
void orc_drT(const orc_level* L, const double* rh, const double* v, double* t);
/* Discrete Laplacian on the nodal grid, Eq. (laplace_discretized), one
 * application per component: in/out 3*N. */
void orc_lap(const orc_level* L, const double* u, double* out);

/* ---- the operators of the method -------------------------------------- */

/* D (Eq. NGF_discretized) and S (Eq. CURV_discretized); J = D + alpha S. */
void orc_objective(const orc_level* L, const double* R, const double* T,
                   const double* u, double* D, double* S);
/* grad J = grad D + alpha grad S, Eqs. (NGF_discretized_gradient),
 * (dPsi), (curvatureMF). */
void orc_gradient(const orc_level* L, const double* R, const double* T,
                  const double* u, double* grad, double* D, double* S);
/* q = (H + alpha grad^2 S) p, Eqs. (NGF_discretized_hessian),
 * (curv_hessMult). */
void orc_hessvec(const orc_level* L, const double* R, const double* T,
                 const double* u, const double* p, double* q);
/* q = 2 hbar^y Lap(Lap p) (Eq. curv_hessMult, without alpha);
 * Sp = hbar^y sum (Lap p)^2 (Eq. CURV_discretized). */
void orc_curvature_apply(const orc_level* L, const double* p, double* q,
                         double* Sp);
/* Exact diagonal of H + alpha grad^2 S (the Jacobi preconditioner). */
void orc_gn_diagonal(const orc_level* L, const double* R, const double* T,
                     const double* u, double* diag);

/* ---- iterative parts (algorithms of Sec. 2.3) ------------------------- */

typedef struct {
    int32_t iters_done;  /* PCG iterations actually performed             */
    int32_t status;      /* 0 ok, 1 exact convergence, 2 breakdown, 3 rtol */
    double  delta;       /* final r^T z                                   */
    double  rr;          /* final r^T r                                   */
} orc_pcg_info;

/* Jacobi-preconditioned CG for (H + alpha grad^2 S) x = rhs, x0 = 0,
 * at most `iters` iterations; rtol <= 0 disables the residual test. */
void orc_pcg(const orc_level* L, const double* R, const double* T,
             const double* u, const double* rhs, const double* diag,
             int32_t iters, double rtol, double* x, orc_pcg_info* info);

typedef struct {
    int32_t gn_iters;    /* Gauss-Newton steps per level                  */
    int32_t pcg_iters;   /* PCG iterations per Gauss-Newton step          */
    int32_t ls_max;      /* Armijo halvings allowed                       */
    double  armijo_c1;   /* sufficient-decrease constant                  */
    double  pcg_rtol;    /* <= 0: fixed iteration count                   */
    int32_t diag_every;  /* Jacobi diagonal at steps 0, k, 2k, ... of the
                            level (k = diag_every), kept in between;
                            0: at the first step only                     */
} orc_gn_options;

typedef struct {
    double  J, D, S;     /* objective at the returned u                   */
    int32_t gn_done;     /* accepted Gauss-Newton steps                   */
    int32_t pcg_total;   /* PCG iterations over all steps                 */
    int32_t status;      /* 0 ok, 6 line search failed, 8 zero gradient   */
    int32_t ls_trials;   /* objective evaluations in line searches        */
} orc_gn_report;

/* Gauss-Newton on one level (Sec. 2.3.1) with Armijo backtracking;
 * u is updated in place.  trace (nullable, 2*gn_iters+1 doubles) receives
 * J before each step and the accepted step length after it. */
void orc_gn_level(const orc_level* L, const double* R, const double* T,
                  double* u, const orc_gn_options* o, orc_gn_report* rep,
                  double* trace);

/* ---- L-BFGS (Sec. 2.3.2) ----------------------------------------------- */
/* r = H0^{-1} q with the initial Hessian H0 = alpha grad^2 S + gamma I
 * (Sec. 2.3.2).  grad^2 S = 2 hbar^y Lap^T Lap, Lap the clamped (Neumann)
 * Laplacian of Eq. (laplace_discretized); the 1-D clamped second difference
 * of n nodes is diagonalised by the orthonormal DCT-II (basis
 * cos(pi k (2i+1) / 2n), eigenvalue -4 sin^2(pi k / 2n) / hy^2), so H0 is
 * diagonal in the 3-D DCT-II basis with eigenvalue alpha 2 hbar^y lambda^2
 * + gamma, lambda the sum of the three 1-D eigenvalues.  Evaluated by
 * explicit cosine sums.  q, r: 3*N. */
void orc_h0_solve(const orc_level* L, double gamma, const double* q, double* r);
typedef struct {
    int32_t iters;       /* L-BFGS steps per level                        */
    int32_t memory;      /* stored (s, y) pairs                           */
    int32_t ls_max;      /* Armijo halvings allowed                       */
    double  armijo_c1;   /* sufficient-decrease constant                  */
    double  gamma;       /* H0 = alpha grad^2 S + gamma I; <= 0: the mean
                            of the Gauss-Newton diagonal at the level's start */
} orc_lbfgs_options;
/* L-BFGS on one level with the two-loop recursion (Nocedal and Wright,
 * Alg. 7.4) and H0 as above; the Armijo rule of the Gauss-Newton level; a
 * pair (s, y) = (u_{k+1} - u_k, g_{k+1} - g_k) is kept only when s^T y > 0
 * (oldest dropped beyond `memory`); a non-descent direction falls back to
 * -g.  u is updated in place; report and trace as for orc_gn_level
 * (pcg_total stays 0).  Returns the gamma used. */
double orc_lbfgs_level(const orc_level* L, const double* R, const double* T,
                       double* u, const orc_lbfgs_options* o,
                       orc_gn_report* rep, double* trace);
/* One direction of the two-loop recursion: d = -H_k g from `count` stored
 * pairs (oldest first, each 3*N) and H0 as above. */
void orc_lbfgs_direction(const orc_level* L, double gamma, int32_t count,
                         const double* S, const double* Y, const double* g,
                         double* d);

/* Image pyramid restriction: coarse cell = mean of its (up to 8) children,
 * m' = ceil(m/2), the physical extent is kept (h' = h m / m'). */
void orc_restrict(const int32_t m[3], const double* img, double* out);
/* Trilinear prolongation of a nodal field between two node grids spanning
 * the same domain. */
void orc_prolongate(const int32_t nc[3], const double* uc,
                    const int32_t nf[3], double* uf);
/* The coarse-to-fine level sequence: level 0 = finest. */
void orc_level_at(const orc_level* finest, int32_t level, orc_level* out);

/* Multilevel Gauss-Newton registration (Sec. 2.3, coarse to fine).
 * u_out: 3*N of the finest level.  u_init (nullable) starts the level
 * `start_level` (0 = finest) instead of the coarsest level from zero. */
void orc_register_multilevel(const orc_level* finest, int32_t levels,
                             const orc_gn_options* o, const double* R,
                             const double* T, const double* u_init,
                             int32_t start_level, double* u_out,
                             orc_gn_report* rep);

#ifdef __cplusplus
}
#endif
#endif
