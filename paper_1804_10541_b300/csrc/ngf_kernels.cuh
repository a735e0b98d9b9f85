// Shared definitions of the device code of libngf_b300: the fused image-grid
// pass (objective, gradient, Gauss-Newton Hessian-vector product), the exact
// Jacobi diagonal, the nodal kernels (curvature, deterministic combination of
// tile partials, PCG vector updates, reductions) and the multilevel helpers.
// Kernel bodies are in ngf_kernels.cu.
//
// Index conventions (Sec. 2.2): 0-based, x fastest; voxel (x,y,z) is cell
// centre (x+1/2)h; node (i,j,k) sits at (i,j,k) hy.  Grid conversion P
// (Eq. grid_conversion) uses per-axis tables f[v] = floor(c_v), w[v] = c_v -
// floor(c_v) with c_v = (v+1/2)(n-1)/m, built in double on the host.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ngf_launch.cuh"

namespace ngf {

// ---------------------------------------------------------------------------
// tiling of the image pass: a CTA owns a TX x TY column tile and a z-chunk and
// marches through its planes; every voxel's warp, residual and stencil is
// evaluated once per plane in shared memory (halo 2 for the front end, halo 1
// for the residual Jacobian), nothing is stored in global memory.
// ---------------------------------------------------------------------------
constexpr int TX = 32, TY = 16, NT = TX * TY;  // 512 threads, one per output column
constexpr int SX2 = TX + 4, SY2 = TY + 4, R2N = SX2 * SY2;  // front-end region (halo 2)
constexpr int SX1 = TX + 2, SY1 = TY + 2, R1N = SX1 * SY1;  // Jacobian region (halo 1)
constexpr int R0N = TX * TY;
constexpr int UBX = TX + 5, UBY = TY + 5;       // node box of the halo-2 region (ratio >= 1)
constexpr int NBX = TX + 1, NBY = TY + 1;       // node box of the owned columns
constexpr int DBX = TX + 3, DBY = TY + 3;       // node box of the halo-1 region (diagonal)
// x-node window of one warp row in the diagonal kernel: 32 voxels plus the
// stencil's neighbours cover at most 20 nodes with two or more voxels per
// cell (three-node span), at most 35 otherwise (four-node span)
__host__ __device__ constexpr int diag_pxw(int span) { return span == 3 ? 20 : 36; }
// four live node planes x 3 components x span y-nodes x window, per row
__host__ __device__ constexpr int diag_window(int span) { return 4 * 3 * span * diag_pxw(span); }

enum Mode { MODE_OBJ = 0, MODE_GRAD = 1, MODE_HESS = 2 };

struct ImgParams {
    int m0, m1, m2, n0, n1, n2;
    int znext;      // offset of the upper node plane of the z interpolation:
                    // n0 n1, or 0 on a planar level (one node plane)
    long long M, N;
    float ih[3];    // 1/h (ih[2] = 0 on a planar level: no z displacement or derivative)
    float ihs[3];   // 1/h^2
    float hh[3];    // 1/(2 h^2)  (h_hat of Eq. hatRho)
    float tau, rho, tr, tau2, rho2;
    float qscale;   // -2 hbar (gradient) or 2 hbar (Hessian)
    double hbar;
    const float* R;
    const float* T;
    const float* u;
    const float* p;
    const int* fx;
    const int* fy;
    const int* fz;
    const float* wx;
    const float* wy;
    const float* wz;
    int zc;                     // planes per z-chunk
    int ntx, nty, ntz;          // tile grid of this geometry
    int dsteps0, dsteps;        // diagonal: shuffle steps that sum a run of voxels sharing an x-node
                                // floor, in the first x tile (clamped lane 0) and in the others
    int pbx, pby, pbz;          // partial box strides of this geometry
    float* partial;             // [tile][3][pbz][pby][pbx]
    double* dpart;              // per-CTA float64 partial sums (D)
    unsigned int* dcount;       // last-CTA ticket
    double* dout;               // D (hbar * sum(1 - r^2))
};

// Shared memory of the SSD pass (no halo, no neighbour stencil)
struct SsdSmem {
    float Uz[6][UBY][UBX];      // u (and p) interpolated to the current plane in z
    alignas(16) float Q4[R0N][4];       // q_hat of the owned columns (3 components + pad)
    alignas(16) float Qx4[TY][NBX][4];  // q_hat reduced onto node columns in x
    float Acc[2][3][NBY][NBX];  // node-plane accumulators of P^T (two live planes)
    float wx2[SX2], wy2[SY2];
    int fx2[SX2], fy2[SY2];     // node floor relative to the Uz box
    int fxb[TX], fyb[TY];       // node floor relative to the partial box
    int xr_lo[NBX], xr_hi[NBX], yr_lo[NBY], yr_hi[NBY];
    double red[NT];
};

// Shared memory of the NGF image pass (one barrier per plane, so every ring
// is one plane deeper than the stages' distance).  The pass works on the
// halo-1 region of its tile: R, Tw, s of the owned columns and the face ring
// in four plane slots, the in-plane products of the owned rows and q_hat of
// the whole region in two.  The tile's node box covers the halo-1 region
// (the z-interpolated node planes and the P^T accumulators use the same
// box); its size is a compile-time bound: the compact layout holds grids
// with two or more voxels per cell in x and y (two CTAs per SM), the wide
// one any ratio.
constexpr int RINGF = 2 * TX + 2 * TY;  // face ring of the halo-1 region (no corners)
template <int NBX_, int NBY_>
struct ImgSmemT {
    static constexpr int kNBX = NBX_, kNBY = NBY_;
    float R[4][R1N];
    float Tw[4][R1N];
    float S[4][R1N];
    union {
        float Pi[2][4][R0N];    // pi(-x), pi(+x), pi(-y), pi(+y) of the owned rows
        double red[NT];         // reductions after the march
    };
    float DTr[4][3][RINGF];     // dT of the face-ring columns
    float Uz[2][6][NBY_][NBX_];           // u (and p) interpolated to a plane in z
    alignas(16) float Q4[2][R1N][4];      // q_hat of the halo-1 region (corners stay zero)
    alignas(16) float Qx4[2][SY1][NBX_][4];  // q_hat reduced onto node columns in x
    float Acc[2][3][NBY_][NBX_];          // node-plane accumulators of P^T (two live planes)
    float wx1[SX1], wy1[SY1];
    int fx1[SX1], fy1[SY1];     // node floor relative to the tile's node box
    int xr_lo[NBX_], xr_hi[NBX_], yr_lo[NBY_], yr_hi[NBY_];
};
// >= 2 voxels per cell: the 34 x 18 halo-1 region spans <= 19 x 11 nodes
// (checked per plan on the host); any ratio: <= 35 x 19
using ImgSmemC = ImgSmemT<19, 11>;
using ImgSmemW = ImgSmemT<DBX, DBY>;
// planes a CTA marches beyond its z-chunk: the halo plane on each side and
// the pipeline's drain from S1 to B
constexpr int IMG_FILL = 7;

// Shared memory of the diagonal pass; the windows are sized for the span, so
// the three-node form (92.7 KB) runs two CTAs per SM
template <int SPAN>
struct DiagSmemT {
    float R[3][R1N];
    float Tw[3][R1N];
    float dT[3][3][R1N];        // [plane slot][component][column]
    float Uz[3][UBY][UBX];
    float Acc[TY * diag_window(SPAN)];  // one private node window per warp row (see diag_pass)
    float WYs[TY][3][SPAN];     // y weights of each row's stencil lines on its SPAN node rows
    float WZs[3][SPAN];         // z weights of the current plane's stencil planes
    float wx1[SX1], wy1[SY1];
    int fx1[SX1], fy1[SY1];     // node floor relative to the Uz (= partial) box
};

// Division by an invariant 32-bit divisor d >= 1 by multiply and shift
// (Granlund-Montgomery): n / d = (t + ((n - t) >> 1)) >> s, t = umulhi(n, m).
struct FastDiv {
    unsigned int d, m, s;
};

inline FastDiv make_fastdiv(unsigned int d) {
    FastDiv f{d, 0u, 0u};
    if (d <= 1) return f;
    unsigned int l = 0;
    while ((1ull << l) < d) ++l;  // smallest l with 2^l >= d
    f.m = (unsigned int)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s = l - 1;
    return f;
}

__device__ __forceinline__ unsigned int fdiv(unsigned int n, const FastDiv& f) {
    if (f.d <= 1) return n;
    const unsigned int t = __umulhi(n, f.m);
    return (t + ((n - t) >> 1)) >> f.s;
}

struct NodeGeom {
    int n0, n1, n2;
    long long N;
    float ihy2[3];         // 1/hy^2
    FastDiv fN, fplane, fn0;  // division by N, n0*n1, n0
};

// Per-thread accumulator of a sum of float products: each product is split
// exactly into p + e (p = a*b rounded, e = fma(a, b, -p)) and p is added with
// an error-free two-sum, so the pair (hi, lo) carries about twice float
// precision; thread results are then combined in float64.
struct DFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

struct CombineParams {
    NodeGeom G;
    const float* partial;
    int box;             // floats per component of one tile partial
    int pbx, pbxy;       // in-box strides in y and z
    const int* xlo;      // tiles [lo, hi] covering each node, per axis
    const int* xhi;
    const int* ylo;
    const int* yhi;
    const int* zlo;
    const int* zhi;
    const int* xtb;      // per-tile base offsets, summed over the axes
    const int* ytb;
    const int* ztb;
    const float* L;      // Lap(input) for the curvature term (nullable)
    const float* ctab;   // curvature diagonal per axis, d1 | dg (nullable)
    float cscale;        // alpha 2 hbar^y
    float* out;
    const float* dotw;   // optional: out . dotw into dout
    double* dpart;
    unsigned int* dcount;
    double* dout;
};

// PCG scalars: 0 delta, 1 dAd, 2 alpha, 3 beta, 4 rr, 5 bb, 6 status
// (0 running, 1 converged, 2 breakdown, 3 rtol), 7 iterations.
enum { PS_DELTA = 0, PS_DQ = 1, PS_ALPHA = 2, PS_BETA = 3, PS_RR = 4, PS_BB = 5, PS_STATUS = 6, PS_ITERS = 7 };

struct PcgParams {
    long long n;
    float* x;
    float* r;
    float* z;
    float* d;
    const float* q;
    const float* diag;
    const float* rhs;
    double* sc;
    double* part;       // 2 * nblocks
    unsigned int* count;
    double rtol;
    int vec4;           // every vector 16-byte aligned: float4 body
};

struct DotArgs {
    long long n;
    const float* a;
    const float* b;  // null: sum of a
    double* part;
    unsigned int* count;
    double* out;
};

struct AxpyArgs {
    long long n;
    float eta;
    const float* x;
    const float* s;  // null: copy
    float* y;
};

struct LapArgs {
    NodeGeom G;
    const float* x;
    float* L;
    double* part;
    unsigned int* count;
    double* out;   // optional: scale * sum L^2
    double scale;
};

__host__ __device__ constexpr int ring_size(int halo) { return 2 * halo * (TX + 2 * halo) + 2 * halo * TY; }

// ---- kernels (defined in ngf_kernels.cu) ----------------------------------
__global__ void k_image_obj(const ImgParams P);   // D only
__global__ void k_image_grad(const ImgParams P);  // D and gradient tile partials
__global__ void k_image_hess(const ImgParams P);  // Hessian-vector tile partials
// the same passes with the wide shared-memory layout (< 2 voxels per cell)
__global__ void k_image_obj_w(const ImgParams P);
__global__ void k_image_grad_w(const ImgParams P);
__global__ void k_image_hess_w(const ImgParams P);
__global__ void k_diag(const ImgParams P);        // Jacobi-diagonal tile partials (>= 2 voxels per cell)
// the same with 2 or 3 shuffle steps per run sum fixed at compile time
__global__ void k_diag_s2(const ImgParams P);
__global__ void k_diag_s3(const ImgParams P);
__global__ void k_diag4(const ImgParams P);       // same, any voxels-per-cell ratio
// SSD distance (identity residual Jacobian): D, gradient, Hessian-vector and
// diagonal tile partials on the halo-0 geometry
constexpr int MODE_SSD_DIAG = 3;
__global__ void k_ssd_obj(const ImgParams P);
__global__ void k_ssd_grad(const ImgParams P);
__global__ void k_ssd_hess(const ImgParams P);
__global__ void k_ssd_diag(const ImgParams P);
__global__ void k_lap(NodeGeom G, const float* __restrict__ x, float* __restrict__ L, double* part,
                      unsigned int* count, double* out, double scale);
__global__ void k_node_combine(const CombineParams P);
__global__ void k_lap2(NodeGeom G, const float* __restrict__ L, float* __restrict__ q, float scale);
__global__ void k_pcg_init(PcgParams P);
__global__ void k_pcg_update(PcgParams P);
__global__ void k_pcg_dir(PcgParams P);
__global__ void k_dot(long long n, const float* __restrict__ a, const float* __restrict__ b, double* part,
                      unsigned int* count, double* out);
__global__ void k_axpy(long long n, float eta, const float* __restrict__ x, const float* __restrict__ s,
                       float* __restrict__ y);
__global__ void k_scale(long long n, float a, const float* __restrict__ x, float* __restrict__ y);
__global__ void k_nonfinite(long long n, const float* __restrict__ a, double* part, unsigned int* count,
                            double* out);
__global__ void k_restrict(int m0, int m1, int m2, const float* __restrict__ img, float* __restrict__ out);

// ---- L-BFGS (Sec. 2.3.2): H0 = alpha grad^2 S + gamma I in the DCT-II basis
// One orthonormal DCT-II (inv = 0) or its transpose (inv = 1) along `axis`
// of a 3 x N nodal field; costab: cos(pi m / 2n) for m in [0, 4n), n the
// axis length.
__global__ void k_dct_axis(NodeGeom G, int axis, int inv, const float* __restrict__ costab,
                           const float* __restrict__ in, float* __restrict__ out);
// a /= c lambda^2 + gamma per DCT coefficient; mu: 1-D eigenvalues of the
// clamped second difference, x | y | z
__global__ void k_h0_scale(NodeGeom G, const float* __restrict__ mu, float c, float gamma, float* __restrict__ a);
// two-loop recursion steps with float64 scalars on the device:
// a = rho (s.q), q -= a y   |   r += (a - rho (y.r)) s
__global__ void k_lbfgs_q(long long n, double rho, const double* dot, const float* __restrict__ y,
                          float* __restrict__ q, double* a_out);
__global__ void k_lbfgs_r(long long n, double rho, const double* dot, const double* a,
                          const float* __restrict__ s, float* __restrict__ r);

// ---- batched forms (independent problems of uneven size in one launch)
// Image passes: a persistent grid takes work items (pair, tile x, tile y,
// tile z) from a queue; the last CTA to finish resets the queue.
// The pairs' parameter blocks travel as one kernel parameter (constant
// bank, read-only), so the pass reads them as cheaply as a single launch's.
constexpr int BATCH_TAB = 112;  // pairs per launch: 112 x (264 + 4) B fit the 32 KB parameter limit
struct BatchImgTable {
    ImgParams p[BATCH_TAB];
    int ssd[BATCH_TAB];  // 1: the pair's distance is SSD
};
struct BatchQueue {
    const int4* items;        // (pair, bx, by, bz), largest tiles first
    int nitems;
    int pair0;                // pair of table entry 0
    const int* active;        // per pair: 0 skips its items (nullable)
    unsigned int* next;       // queue head and finished-CTA count, zero between launches
    unsigned int* done;
};
// Nodal kernels: pair k owns CTAs first[k] .. first[k+1]-1 of the launch.
struct BatchSegs {
    const int* first;    // npairs + 1 prefix
    const int* pair_of;  // pair of each CTA of the launch
    int npairs;
    const int* active;   // nullable
};
__global__ void k_batch_image_obj(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_image_grad(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_image_hess(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_image_obj_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_image_grad_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_image_hess_w(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_diag(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_diag_s2(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_diag_s3(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_diag4(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_ssd_diag(const BatchQueue Q, const __grid_constant__ BatchImgTable T);
__global__ void k_batch_lap(const LapArgs* table, const BatchSegs S);
__global__ void k_batch_combine(const CombineParams* table, const BatchSegs S);
__global__ void k_batch_pcg_init(const PcgParams* table, const BatchSegs S);
__global__ void k_batch_pcg_update(const PcgParams* table, const BatchSegs S);
__global__ void k_batch_pcg_dir(const PcgParams* table, const BatchSegs S);
__global__ void k_batch_dot(const DotArgs* table, const BatchSegs S);
__global__ void k_batch_axpy(const AxpyArgs* table, const BatchSegs S);
__global__ void k_prolong(int f0, int f1, int f2, int c0, int c1, long long Nc, const int* __restrict__ tf,
                          const float* __restrict__ tw, const float* __restrict__ uc, float* __restrict__ uf);

}  // namespace ngf
