// Internal plan structure shared by the C-ABI implementation files.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ngf.h"
#include "ngf_kernels.cuh"

namespace ngf {

// Tile-partial geometry of the transposed grid conversion for one halo:
// per tile its node-box origin, per node the first/last tile whose box
// contains it (device arrays, one allocation).
struct Geometry {
    int ntx = 0, nty = 0, ntz = 0;
    int pbx = 0, pby = 0, pbz = 0;
    // per axis: tiles [lo, hi] that cover each node, and per tile the base
    // offset tb (into the partial array, summed over the three axes) such
    // that the node's entry in tile t is at tb[t] + node * (in-box stride)
    int* xlo = nullptr;
    int* xhi = nullptr;
    int* ylo = nullptr;
    int* yhi = nullptr;
    int* zlo = nullptr;
    int* zhi = nullptr;
    int* xtb = nullptr;
    int* ytb = nullptr;
    int* ztb = nullptr;
    int* mem = nullptr;
    long long tiles() const { return (long long)ntx * nty * ntz; }
    long long partial_floats() const { return tiles() * 3 * pbz * pby * pbx; }
};

struct Plan {
    ngf_level_desc desc{};
    cudaStream_t stream = nullptr;
    int m[3]{}, n[3]{};
    long long M = 0, N = 0;
    double hbar = 0, hbary = 0, hy[3]{};
    int zc = 0;
    bool diag_span3 = false;    // diagonal: three-node span (>= 2 voxels per cell on every axis)
    bool img_wide = false;      // image pass: wide shared-memory layout (< 2 voxels per cell in x or y)
    int dsteps[2] = {0, 0};     // diagonal: shuffle steps covering the longest run of equal x
                                // floors in the first x tile and in the others
    int img_blocks = 0, diag_blocks = 0, node_blocks = 0, node1_blocks = 0;
    // device workspace
    int* ftab = nullptr;    // fx | fy | fz
    float* wtab = nullptr;  // wx | wy | wz
    Geometry g0, g1;        // halo 0 (gradient, Hessian), halo 1 (diagonal)
    float* partial = nullptr;
    float* L = nullptr;      // Laplacian scratch, 3N
    float* ctab = nullptr;   // curvature diagonal per axis: d1 | dg (2 x (n0+n1+n2))
    float* dct_cos = nullptr;  // L-BFGS: cos(pi m / 2n) tables, 4 n per axis (x | y | z)
    float* dct_mu = nullptr;   // L-BFGS: 1-D eigenvalues of the clamped second difference
    float* h0_tmp = nullptr;   // L-BFGS: 3N scratch of the DCT passes
    double* dsc = nullptr;   // scalars: 0 D, 1 S, 2 dot, 3 nonfinite count
    double* dpart = nullptr;
    unsigned int* dcount = nullptr;
    size_t dpart_len = 0;
    std::string err;
    // kernel timing (measurement only)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev[4];  // start/stop pairs per image kernel
    // cached PCG graph
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> graph_key;
    int graph_iters = 0;
    long long graph_kernels = 0;
};

// Device memory of plans and registrations comes from a library-private
// stream-ordered pool per device (kept across calls, freed without a device
// synchronisation).
cudaError_t dev_alloc(void** ptr, size_t bytes, cudaStream_t stream);
void dev_free(void* ptr, cudaStream_t stream);

// tile-partial geometry of the image pass: the NGF pass writes q_hat on the
// halo-1 region of its tile (the face ring carries its rows' transposed
// stencil), the SSD pass on the tile alone
inline const Geometry& img_geom(const Plan* p) {
    return p->desc.distance == NGF_DIST_SSD ? p->g0 : p->g1;
}

// helpers implemented in ngf_api.cu
ngf_status set_error(Plan* p, ngf_status s, const std::string& msg);
ngf_status cuda_check(Plan* p, cudaError_t e, const char* what);
ngf_status validate_desc(const ngf_level_desc* d, std::string& why);
bool is_device_ptr(const void* ptr);
ImgParams img_params(const Plan* p, const float* R, const float* T, const float* u, const float* p_,
                     int mode, const Geometry& g, double* dout);
CombineParams combine_params(const Plan* p, const Geometry& g, float* out, const float* L, const float* ctab,
                             const float* dotw, double* dout);
NodeGeom node_geom(const Plan* p);
ngf_status hessvec_impl(Plan* p, const float* R, const float* T, const float* u, const float* pv, float* q,
                        const float* dotw, double* dout);
ngf_status objective_impl(Plan* p, const float* R, const float* T, const float* u, double* dD, double* dS);
ngf_status gradient_impl(Plan* p, const float* R, const float* T, const float* u, float* g, double* dD,
                         double* dS);
ngf_status diagonal_impl(Plan* p, const float* R, const float* T, const float* u, float* diag);
cudaError_t prof_mark(Plan* p, int which);
ngf_status dot_impl(Plan* p, long long n, const float* a, const float* b, double* dout);
ngf_status h0_impl(Plan* p, double gamma, const float* q, float* r);
int grid_for(long long n, int max_blocks);
// plan with a requested z-chunk length (0: about two CTAs per SM)
ngf_status plan_create(ngf_plan** out, const ngf_level_desc* desc, cudaStream_t stream, int zc);
ngf_level_desc level_at(const ngf_level_desc& finest, int level);

// The 2-D method (a planar level): one image plane and one node plane
// (m[2] == 1 and n[2] == 1).  Images are m0 x m1, u has the in-plane
// components x and y (the z component of the 3N layout is carried along and
// stays zero from a zero start), the template is interpolated bilinearly in
// the plane, short differences and the curvature stencil act in x and y
// only, and the cell volumes are hbar = h0 h1, hbar^y = hy0 hy1 (h[2] is not
// used).
inline bool planar(const ngf_level_desc& d) { return d.m[2] == 1 && d.n[2] == 1; }
// node spacing per axis: the nodes span the image domain [0, m h]; the
// single node plane of a planar level has unit spacing (it is never used)
inline double node_spacing(const ngf_level_desc& d, int a) {
    return d.n[a] > 1 ? (double)d.m[a] * d.h[a] / (double)(d.n[a] - 1) : 1.0;
}
inline double cell_volume(const ngf_level_desc& d) {
    return planar(d) ? d.h[0] * d.h[1] : d.h[0] * d.h[1] * d.h[2];
}
inline double node_cell_volume(const ngf_level_desc& d) {
    return node_spacing(d, 0) * node_spacing(d, 1) * (planar(d) ? 1.0 : node_spacing(d, 2));
}

}  // namespace ngf

struct ngf_plan {
    ngf::Plan impl;
};
