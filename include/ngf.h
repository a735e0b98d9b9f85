/*
 * ngf.h -- C ABI of the B300 (sm_103a) matrix-free NGF + curvature
 * registration library (libngf_b300.so).
 *
 * The method (Koenig, Ruehaak, Derksen, Lellmann, "A matrix-free approach to
 * parallel and memory-efficient deformable image registration"): minimise
 * J(y) = D(y) + alpha S(y) over a nodal deformation grid y, with D the
 * normalized-gradient-fields distance (Eq. NGF_discretized) and S the
 * curvature regulariser (Eq. CURV_discretized), by Gauss-Newton with a
 * (preconditioned) CG inner solve or by L-BFGS, with Armijo line search,
 * coarse to fine (Sec. 2.3).  Every derivative is evaluated matrix-free
 * (Sec. 4): no Jacobian, sparse matrix or other O(voxels) derivative storage
 * is kept.  The sum of squared differences (Sec. 7) can replace NGF per
 * level; many pairs can be processed together by the batched form.
 *
 * Layout (Sec. 2.2, Table 1), 0-based:
 *  - images R, T: m[0]*m[1]*m[2] float32, x fastest, cell centres at
 *    (i + 1/2) h; the template T lives on the same grid as R and is zero
 *    outside it (trilinear interpolation with Dirichlet boundary);
 *  - nodal vector fields (u, p, q, grad, diag): 3*N float32 with
 *    N = n[0]*n[1]*n[2], component-major (all x components, then y, then z),
 *    x fastest; node j sits at j * hy with hy_k = m_k h_k / (n_k - 1), so the
 *    nodes span the image domain [0, m h];
 *  - the unknown is the displacement u = y - x^y (physical units of h); the
 *    warped point of voxel i is x_i + (P u)_i.
 *
 * Precision: bulk arithmetic float32; every global reduction (D, S, PCG
 * inner products), the line-search comparison and the stopping tests in
 * float64 on the device.
 *
 * Ownership and streams: every data pointer is caller-owned and is never
 * freed by the library.  Plan functions take CUDA device pointers (device or
 * managed memory) and enqueue their kernels on the plan's stream; a function
 * that returns host scalars synchronises that stream first, the *_dev
 * variants write float64 results to device memory and never synchronise.
 * Workspace is allocated at plan creation, never in an operator call.  A
 * plan must not be used from two streams or threads at the same time.
 *
 * Errors: no exception crosses the ABI; every call returns an ngf_status.
 * Arguments are validated before any launch (sizes, 2 <= n_k <= m_k + 1,
 * tau, rho > 0, alpha >= 0, pointer kinds via cudaPointerGetAttributes);
 * ngf_last_error() returns a message for the last failure.
 */
#ifndef NGF_B300_H
#define NGF_B300_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NGF_ABI_VERSION 3

typedef enum {
    NGF_OK = 0,
    NGF_EINVAL = -1,       /* bad size, parameter or pointer kind          */
    NGF_ECUDA = -2,        /* a CUDA runtime call or launch failed          */
    NGF_ENOMEM = -3,       /* device allocation failed                      */
    NGF_ENONFINITE = -4,   /* NaN or Inf in an input image or field         */
    NGF_EBREAKDOWN = -5,   /* PCG: d^T A d <= 0 or not finite               */
    NGF_ELINESEARCH = -6,  /* Armijo: no acceptable step in ls_max trials   */
    NGF_EMAXITER = -7,     /* iteration budget exhausted (not an error)     */
    NGF_EBOUNDS = -8       /* a size exceeds a documented limit             */
} ngf_status;

/* One resolution level (Sec. 2.2, Table 1). */
typedef struct {
    int32_t m[3];   /* image cells per axis, >= 1                                 */
    double  h[3];   /* image spacing per axis (e.g. mm), > 0                      */
    int32_t n[3];   /* deformation-grid NODES per axis, 2 <= n_k <= m_k + 1
                       (the image grid is at least as fine, Sec. 2.2)            */
    double  alpha;  /* curvature weight, >= 0 (Eq. discreteenergy)               */
    double  tau;    /* NGF edge parameter of the template, > 0 (Eq. ngf)         */
    double  rho;    /* NGF edge parameter of the reference, > 0 (Eq. ngf)        */
    int32_t distance; /* NGF_DIST_NGF (0, the paper's distance) or NGF_DIST_SSD:
                         D = hbar/2 sum (T(x + Pu) - R)^2, whose residual
                         Jacobian is the identity (Sec. 7); tau, rho unused  */
} ngf_level_desc;
enum { NGF_DIST_NGF = 0, NGF_DIST_SSD = 1 };

typedef struct ngf_plan ngf_plan;

/* Create a plan for one level: validates desc, allocates the workspace (grid
 * conversion tables, the tile partials of the transposed conversion, reduction
 * buffers) on the current device and binds the plan to cuda_stream
 * (cudaStream_t; NULL = legacy default stream). */
ngf_status ngf_plan_create(ngf_plan** plan, const ngf_level_desc* desc, void* cuda_stream);
/* As ngf_plan_create with a given z-chunk length of the image-pass tiles
 * (32 x 16 x zc voxels, capped by m[2]; 0 = the default model).  The tile
 * geometry fixes the summation order of the transposed conversion, so plans
 * (or batches) with the same zc give bitwise equal results. */
ngf_status ngf_plan_create_ex(ngf_plan** plan, const ngf_level_desc* desc, int32_t zc, void* cuda_stream);
ngf_status ngf_plan_destroy(ngf_plan* plan);
ngf_status ngf_plan_set_stream(ngf_plan* plan, void* cuda_stream);
/* Message of the last failure of this plan (plan == NULL: of the last failed
 * call without a plan on this thread).  Never NULL. */
const char* ngf_last_error(const ngf_plan* plan);

/* D and S at u (Eqs. NGF_discretized, CURV_discretized); J = D + alpha S.
 * R, T: device images; u: device 3*N field; D, S: host (synchronises).
 * D is reduced in float64 from a cancellation-free float32 form of 1 - r^2. */
ngf_status ngf_objective(ngf_plan* plan, const float* R, const float* T, const float* u,
                         double* D, double* S);
/* Same, no synchronisation: dev_DS[0] = D, dev_DS[1] = S (device doubles). */
ngf_status ngf_objective_dev(ngf_plan* plan, const float* R, const float* T, const float* u,
                             double* dev_DS);

/* grad = grad D + alpha grad S (Eqs. NGF_discretized_gradient, dPsi,
 * gradNGF, curvatureMF), device 3*N; D, S: host, nullable (if both are NULL
 * the call does not synchronise). */
ngf_status ngf_gradient(ngf_plan* plan, const float* R, const float* T, const float* u,
                        float* grad, double* D, double* S);
/* Same with dev_DS (device, 2 doubles, nullable) instead of host scalars. */
ngf_status ngf_gradient_dev(ngf_plan* plan, const float* R, const float* T, const float* u,
                            float* grad, double* dev_DS);

/* q = (H + alpha grad^2 S) p with H the Gauss-Newton matrix
 * 2 hbar P^T dT^T dr^T dr dT P (Eqs. NGF_discretized_hessian, HNGF, hessMult,
 * curv_hessMult); u, p, q device 3*N; q must not alias p or u.  The
 * transposed grid conversion is a deterministic tile reduction: repeated
 * calls return bitwise identical q. */
ngf_status gn_hessvec(ngf_plan* plan, const float* R, const float* T, const float* u,
                      const float* p, float* q);

/* q = 2 hbar^y Lap(Lap p) (Eq. curv_hessMult without alpha; Eq.
 * curvatureMF for p = u); Sp (host, nullable) = hbar^y sum (Lap p)^2.
 * q may be NULL when only Sp is wanted. */
ngf_status curvature_apply(ngf_plan* plan, const float* p, float* q, double* Sp);

/* Exact diagonal of H + alpha grad^2 S at u (the Jacobi preconditioner of
 * the PCG solve), device 3*N.  Its image-grid part is summed in a fixed
 * order without atomics: repeated calls return bitwise identical results. */
ngf_status ngf_gn_diagonal(ngf_plan* plan, const float* R, const float* T, const float* u,
                           float* diag);

/* ---- PCG on the device (Sec. 2.3.1) ------------------------------------
 * Jacobi-preconditioned CG for (H + alpha grad^2 S) x = rhs from x = 0.
 * All vectors are caller-owned device 3*N floats; dev_scalars is a
 * caller-owned device array of NGF_PCG_NSCALARS doubles holding the state
 * (delta = r^T z, d^T A d, alpha, beta, r^T r, b^T b, status, iterations).
 * A diagonal entry <= 0 preconditions its component by 0 (such a row and
 * column of the PSD matrix are zero).  pcg_step never synchronises and is a
 * no-op once the solve has stopped (exact convergence, breakdown, rtol). */
#define NGF_PCG_NSCALARS 8
typedef struct {
    float* x;
    float* r;
    float* z;
    float* d;
    float* q;
    const float* diag;
    double* dev_scalars;
    double rtol;    /* stop when ||r|| <= rtol ||rhs||; <= 0: fixed iterations */
} ngf_pcg_state;

typedef struct {
    int32_t iters_done;
    int32_t status;     /* 0 running/ok, 1 exact convergence, 2 breakdown, 3 rtol */
    double  delta;      /* r^T z                                                  */
    double  rr;         /* r^T r                                                  */
} ngf_pcg_info;

/* x = 0, r = rhs, z = M^-1 r, d = z and the float64 state; rhs may alias r. */
ngf_status pcg_init(ngf_plan* plan, ngf_pcg_state* st, const float* rhs);
/* One iteration: q = A d (gn_hessvec), then the float64 scalars, x, r, z, d. */
ngf_status pcg_step(ngf_plan* plan, ngf_pcg_state* st, const float* R, const float* T,
                    const float* u);
/* `iters` iterations of pcg_step, replayed as one captured CUDA graph when
 * use_graph != 0 and the plan's stream is not the legacy default stream (the
 * graph is cached in the plan for these pointers and this count). */
ngf_status pcg_solve(ngf_plan* plan, ngf_pcg_state* st, const float* R, const float* T,
                     const float* u, int32_t iters, int32_t use_graph);
/* Read the state (synchronises). */
ngf_status pcg_read(ngf_plan* plan, const ngf_pcg_state* st, ngf_pcg_info* info);

/* ---- L-BFGS initial Hessian (Sec. 2.3.2) ------------------------------
 * r = (alpha grad^2 S + gamma I)^{-1} q, gamma > 0: the clamped Laplacian is
 * diagonal in the 3-D DCT-II basis, so the solve is three forward
 * transforms, one division per coefficient and three inverse transforms
 * (FP32, O(N (n_x + n_y + n_z)) work).  q, r: 3*N device arrays (may
 * alias); enqueued on the plan's stream. */
ngf_status ngf_h0_solve(ngf_plan* plan, double gamma, const float* q, float* r);

/* ---- full registration (Sec. 2.3, coarse to fine) ---------------------- */
typedef struct {
    int32_t levels;       /* >= 1; level 0 is `finest`, each coarser level halves
                             image cells and deformation cells (ceil)           */
    int32_t gn_iters;     /* Gauss-Newton steps per level                       */
    int32_t pcg_iters;    /* PCG iterations per Gauss-Newton step               */
    int32_t ls_max;       /* Armijo trials (step 1, 1/2, 1/4, ...)              */
    double  armijo_c1;    /* sufficient-decrease constant, e.g. 1e-4            */
    double  pcg_rtol;     /* <= 0: fixed PCG iteration count                    */
    int32_t start_level;  /* level at which u_init is given (if u_init)         */
    const float* u_init;  /* nullable: start field on level start_level (3*N of
                             that level; host or device); NULL = zero field on
                             the coarsest level                                 */
    int32_t use_graph;    /* capture each PCG solve as a CUDA graph             */
    int32_t method;       /* NGF_METHOD_GN (Sec. 2.3.1) or NGF_METHOD_LBFGS
                             (Sec. 2.3.2; gn_iters = L-BFGS steps per level,
                             pcg_iters unused)                                 */
    int32_t lbfgs_memory; /* stored (s, y) pairs, >= 1                          */
    double  lbfgs_gamma;  /* H0 = alpha grad^2 S + gamma I; <= 0: the mean of
                             the Gauss-Newton diagonal at each level's start   */
    int32_t zc;           /* z-chunk length of every level's plans; 0 = the
                             default (per plan; per batch in register_batch)  */
    int32_t gn_iters_finest; /* > 0: Gauss-Newton steps on level 0 instead of
                             gn_iters (coarser levels keep gn_iters); GN only  */
    double  j_target;     /* > 0: stop level 0 once J <= j_target (checked at
                             the start of each of its steps, i.e. after every
                             accepted step); 0 = off.  Used to compare starts
                             at equal final objective.  GN only.              */
    int32_t diag_every;   /* the Jacobi diagonal of the PCG solves is recomputed
                             at Gauss-Newton steps 0, k, 2k, ... of each level
                             (k = diag_every) and kept in between; 0 = once per
                             level, at its first step (the default).  GN only. */
} ngf_options;
enum { NGF_METHOD_GN = 0, NGF_METHOD_LBFGS = 1 };

typedef struct {
    double  J, D, S;      /* objective at the returned u (finest level)         */
    int32_t gn_done;      /* accepted Gauss-Newton steps, all levels            */
    int32_t pcg_total;    /* PCG iterations, all levels                         */
    int32_t ls_trials;    /* objective evaluations in line searches             */
    int32_t ls_fail;      /* levels ended by a failed line search               */
    int32_t status;       /* 0, or the ngf_status that ended a level early      */
    double  seconds;      /* wall time of the call                              */
    int64_t hessvec_voxels; /* sum over gn_hessvec calls of the level's voxels  */
} ngf_report;

/* Multilevel Gauss-Newton registration.  R, T: finest-level images, u_out:
 * finest-level 3*N field; each may be a host or a device pointer (host data
 * is copied in once and the result copied out once, inside the call).  The
 * image pyramid (mean of up to 8 children, physical extent kept) and the
 * trilinear prolongation of u run on the device.  Synchronises the stream.
 * R, T and u_init are checked for NaN/Inf (NGF_ENONFINITE). */
ngf_status register_multilevel(const ngf_level_desc* finest, const ngf_options* opts,
                               const float* R, const float* T, float* u_out,
                               ngf_report* report, void* cuda_stream);

/* ---- batched form: many independent pairs of uneven size ----------------
 * A batch holds one plan per pair (own tile geometry, partials and scalars)
 * and runs each stage of the method for all pairs in one launch: the image
 * passes as a persistent grid that takes (pair, tile) work items, largest
 * first, from a device queue; the nodal and PCG kernels with a contiguous
 * range of thread blocks per pair.  Every pair's result is bitwise the one
 * its own plan gives with the same z-chunk length.
 * Pointer arguments R, T, u, p, q, grad, diag are HOST arrays of npairs
 * DEVICE pointers laid out as for the single-pair calls; D and S are host
 * arrays of npairs doubles.  Calls enqueue on the batch's stream; the
 * objective and the autotuner synchronise it.
 * zc: planes per z-chunk of the image-pass tiles (32 x 16 x zc voxels);
 * 0 picks, per pair, the chunk count that minimises rounds of two thread
 * blocks per SM times planes marched. */
typedef struct ngf_batch ngf_batch;
ngf_status ngf_batch_create(ngf_batch** batch, int32_t npairs, const ngf_level_desc* descs, int32_t zc,
                            void* cuda_stream);
ngf_status ngf_batch_destroy(ngf_batch* batch);
ngf_status ngf_batch_objective(ngf_batch* batch, const float* const* R, const float* const* T,
                               const float* const* u, double* D, double* S);
ngf_status ngf_batch_gradient(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, float* const* grad);
ngf_status ngf_batch_hessvec(ngf_batch* batch, const float* const* R, const float* const* T,
                             const float* const* u, const float* const* p, float* const* q);
ngf_status ngf_batch_diagonal(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, float* const* diag);
/* Tile autotuner: times the batched Hessian-vector product (three calls
 * after one warm-up, CUDA events) for each candidate z-chunk length in
 * {8, 16, 24, 32, 48, 64} (capped by the deepest pair), rebuilds the batch
 * with the fastest and returns it in *zc and the time per call in *ms.
 * p and q are work vectors of each pair (contents of q are overwritten). */
ngf_status ngf_batch_autotune(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, const float* const* p, float* const* q,
                              int32_t* zc, double* ms);
int32_t ngf_batch_zc(const ngf_batch* batch);

/* Multilevel Gauss-Newton registration of npairs independent pairs, the same
 * options for all (method NGF_METHOD_GN, u_init NULL; each pair's distance,
 * NGF or SSD, from its descriptor): every Gauss-Newton stage is one
 * batched launch sequence over the pairs still iterating, each PCG solve one
 * captured CUDA graph (when opts->use_graph), each Armijo trial one batched
 * objective over the pairs still searching.  Each pair takes exactly the
 * decisions of register_multilevel on its own.  R, T, u_out: host arrays of
 * npairs DEVICE pointers (finest level); reports: host array of npairs.
 * autotune != 0 runs ngf_batch_autotune once per level.  Synchronises. */
ngf_status register_batch(int32_t npairs, const ngf_level_desc* finest, const ngf_options* opts,
                          const float* const* R, const float* const* T, float* const* u_out,
                          ngf_report* reports, int32_t autotune, void* cuda_stream);

/* ---- objective without any allocation ----------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: code whose device memory is owned
 * by a framework's pool, real-time loops in which an allocation (which can
 * synchronise the device) is not allowed, plugins that must leave the host
 * process's allocator alone.  It computes the same D and S as ngf_objective
 * without a plan and calls no cudaMalloc, cudaFree or allocating routine:
 * its grid-conversion tables and float64 reduction partials live in one
 * fixed file-scope device array of about 225 KB, which every GPU that loads
 * this library holds until the process exits.
 *  - The first call on a device looks up that array's device address and
 *    raises the image kernel's shared-memory limit; make this first call
 *    before any stream capture.
 *  - All calls share the array and it keeps the last call's contents (every
 *    call clears what must start at zero); calls that overlap on the GPU, on
 *    one device, race and give wrong results.
 *  - Limits: at most NGF_NOALLOC_MAX_AXIS image cells per axis, and at
 *    most NGF_NOALLOC_MAX_BLOCKS thread blocks of the image pass, i.e.
 *    ceil(m0/32) * ceil(m1/16) * chunks <= 16384, where chunks (the number
 *    of z-chunks, about 2 * SMs / (ceil(m0/32) * ceil(m1/16)), at least 1)
 *    is 1 or 2 for large slices: only slices wider than about 16384 tiles
 *    of 32 x 16 cells are refused.  Larger problems return NGF_EBOUNDS with
 *    a message before anything is launched.
 * R, T, u: device arrays as for ngf_objective; dev_DS: device, 2 doubles
 * (D, S); enqueued on cuda_stream, no synchronisation. */
#define NGF_NOALLOC_MAX_AXIS 4096
#define NGF_NOALLOC_MAX_BLOCKS 16384
ngf_status ngf_objective_noalloc(const ngf_level_desc* desc, const float* R, const float* T,
                                 const float* u, double* dev_DS, void* cuda_stream);

/* ---- measurement ------------------------------------------------------
 * When enabled, the plan records a CUDA event pair on its stream around every
 * launch of its image-grid kernels issued outside stream capture.
 * ngf_profile_read synchronises, returns the summed milliseconds and the
 * launch count of kernel `which` (NGF_K_OBJECTIVE ... NGF_K_DIAGONAL) since
 * the last read, and clears that record. */
enum { NGF_K_OBJECTIVE = 0, NGF_K_GRADIENT = 1, NGF_K_HESSVEC = 2, NGF_K_DIAGONAL = 3 };
ngf_status ngf_profile_enable(ngf_plan* plan, int32_t enable);
ngf_status ngf_profile_read(ngf_plan* plan, int32_t which, double* ms, int64_t* launches);

/* Kernels launched by this library in this process so far. */
int64_t ngf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
