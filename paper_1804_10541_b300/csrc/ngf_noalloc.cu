// Objective evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside a framework that
// owns all device memory through its own pool, real-time loops where an
// allocation (which may synchronise the device) is not allowed, or plugins
// loaded into a process whose allocator they must not touch.  For them,
// ngf_objective_noalloc evaluates D and S without a plan: the grid-conversion
// tables and the float64 reduction partials live in one file-scope device
// array of fixed size, held by every GPU that loads this library until the
// process exits.  Nothing here calls cudaMalloc, cudaFree or an allocating
// library routine.
#include <algorithm>
#include <mutex>
#include <string>

#include "ngf_plan.h"

namespace ngf {
namespace {

constexpr int NA_MAX_AXIS = NGF_NOALLOC_MAX_AXIS;
constexpr int NA_MAX_BLOCKS = NGF_NOALLOC_MAX_BLOCKS;

// layout of the scratch array
constexpr size_t NA_OFF_F = 0;                                            // int   f[3 * MAX_AXIS]
constexpr size_t NA_OFF_W = NA_OFF_F + 3 * NA_MAX_AXIS * sizeof(int);     // float w[3 * MAX_AXIS]
constexpr size_t NA_OFF_P = NA_OFF_W + 3 * NA_MAX_AXIS * sizeof(float);   // double part[MAX_BLOCKS]
constexpr size_t NA_OFF_C = NA_OFF_P + NA_MAX_BLOCKS * sizeof(double);    // unsigned count[4]
constexpr size_t NA_BYTES = NA_OFF_C + 4 * sizeof(unsigned int);

// The scratch array.  In host code this name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress (see scratch_on_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Per-axis grid-conversion tables (same arithmetic, in double, as the plan's
// host-built tables, so the results agree bit for bit) and the counters of
// the last-CTA reductions, which must start at zero on every call.
__global__ void k_na_setup(int m0, int m1, int m2, int n0, int n1, int n2, int* f, float* w, unsigned int* count) {
    const int total = m0 + m1 + m2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int v = i, m = m0, n = n0;
        if (i >= m0 + m1) { v = i - m0 - m1; m = m2; n = n2; }
        else if (i >= m0) { v = i - m0; m = m1; n = n1; }
        const double c = ((double)v + 0.5) * (double)(n - 1) / (double)m;
        const double fl = floor(c);
        f[i] = (int)fl;
        w[i] = (float)(c - fl);
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) count[threadIdx.x] = 0u;
}

// S = scale * sum over nodes and components of (Lap u)^2 (Eqs. CURV_discretized,
// laplace_discretized with clamped neighbours), reduced in float64 with the
// deterministic last-CTA pattern; the Laplacian itself is not stored.
__global__ void __launch_bounds__(256) k_na_curv_energy(NodeGeom G, const float* __restrict__ x, double* part,
                                                      unsigned int* count, double* out, double scale) {
    __shared__ double red[256];
    __shared__ int is_last;
    double acc = 0.0;
    const long long total = 3 * G.N;
    const int plane = G.n0 * G.n1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / G.N);
        const int n = (int)(i - (long long)c * G.N);
        const int iz = n / plane, rem = n - iz * plane, iy = rem / G.n0, ix = rem - iy * G.n0;
        const float* xc = x + (long long)c * G.N;
        const float v = xc[n];
        const float xm = xc[ix > 0 ? n - 1 : n], xp = xc[ix < G.n0 - 1 ? n + 1 : n];
        const float ym = xc[iy > 0 ? n - G.n0 : n], yp = xc[iy < G.n1 - 1 ? n + G.n0 : n];
        const float zm = xc[iz > 0 ? n - plane : n], zp = xc[iz < G.n2 - 1 ? n + plane : n];
        const float l = (xm - 2.f * v + xp) * G.ihy2[0] + (ym - 2.f * v + yp) * G.ihy2[1] + (zm - 2.f * v + zp) * G.ihy2[2];
        acc += (double)l * (double)l;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = red[0];
        __threadfence();
        is_last = (atomicAdd(count, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double a = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) a += ((volatile double*)part)[i];
    red[threadIdx.x] = a;
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

// Device address of the scratch array on the current device, looked up (and
// the image kernel's shared-memory limit raised) once per device.
std::mutex g_na_mu;
unsigned char* g_na_addr[256] = {};

ngf_status scratch_on_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) return set_error(nullptr, NGF_EBOUNDS, "device ordinal above 255");
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        unsigned char* ptr = nullptr;
        e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaGetSymbolAddress(no-allocation scratch)");
        e = cudaFuncSetAttribute(k_image_obj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ImgSmemC));
        if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaFuncSetAttribute(k_image_obj)");
        e = cudaFuncSetAttribute(k_image_obj_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ImgSmemW));
        if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaFuncSetAttribute(k_image_obj_w)");
        g_na_addr[dev] = ptr;
    }
    *out = g_na_addr[dev];
    return NGF_OK;
}

}  // namespace
}  // namespace ngf

using namespace ngf;

extern "C" ngf_status ngf_objective_noalloc(const ngf_level_desc* d, const float* R, const float* T, const float* u,
                                            double* dev_DS, void* cuda_stream) {
    std::string why;
    const ngf_status vs = validate_desc(d, why);
    if (vs != NGF_OK) return set_error(nullptr, vs, why);
    for (int a = 0; a < 3; ++a)
        if (d->m[a] > NA_MAX_AXIS)
            return set_error(nullptr, NGF_EBOUNDS,
                             "ngf_objective_noalloc: more than NGF_NOALLOC_MAX_AXIS (4096) image cells on an axis");
    if (!is_device_ptr(R) || !is_device_ptr(T) || !is_device_ptr(u) || !is_device_ptr(dev_DS))
        return set_error(nullptr, NGF_EINVAL, "ngf_objective_noalloc: R, T, u and dev_DS must be device pointers");

    int dev = 0, sms = 0;
    {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaGetDevice");
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaDeviceGetAttribute(multiprocessor count)");
    }
    // same z-chunking as a plan: about two CTAs per SM, at least 8 planes per chunk
    const long long txy = (long long)((d->m[0] + TX - 1) / TX) * ((d->m[1] + TY - 1) / TY);
    long long nchunk = (2LL * sms + txy / 2) / txy;
    nchunk = std::max<long long>(1, std::min<long long>(nchunk, d->m[2]));
    const int zc = (int)std::max<long long>(std::min<long long>(8, d->m[2]), (d->m[2] + nchunk - 1) / nchunk);
    if (d->distance != NGF_DIST_NGF)
        return set_error(nullptr, NGF_EINVAL, "ngf_objective_noalloc evaluates the NGF distance only");
    const dim3 grid((d->m[0] + TX - 1) / TX, (d->m[1] + TY - 1) / TY, (d->m[2] + zc - 1) / zc);
    const long long img_blocks = (long long)grid.x * grid.y * grid.z;
    const long long N = (long long)d->n[0] * d->n[1] * d->n[2];
    const int node_blocks = (int)std::min<long long>((3 * N + 255) / 256, 4LL * sms);
    if (img_blocks > NA_MAX_BLOCKS)
        return set_error(nullptr, NGF_EBOUNDS,
                         "ngf_objective_noalloc: image needs more than NGF_NOALLOC_MAX_BLOCKS (16384) thread blocks");

    unsigned char* base = nullptr;
    {
        const ngf_status s = scratch_on_device(&base);
        if (s != NGF_OK) return s;
    }
    int* f = reinterpret_cast<int*>(base + NA_OFF_F);
    float* w = reinterpret_cast<float*>(base + NA_OFF_W);
    double* part = reinterpret_cast<double*>(base + NA_OFF_P);
    unsigned int* count = reinterpret_cast<unsigned int*>(base + NA_OFF_C);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    cudaError_t e = launch(k_na_setup, dim3(8), dim3(256), 0, stream, d->m[0], d->m[1], d->m[2], d->n[0], d->n[1],
                           d->n[2], f, w, count);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "k_na_setup");

    ImgParams P{};
    P.m0 = d->m[0];
    P.m1 = d->m[1];
    P.m2 = d->m[2];
    P.n0 = d->n[0];
    P.n1 = d->n[1];
    P.n2 = d->n[2];
    P.M = (long long)P.m0 * P.m1 * P.m2;
    P.N = N;
    for (int a = 0; a < 3; ++a) {
        P.ih[a] = (float)(1.0 / d->h[a]);
        P.ihs[a] = (float)(1.0 / (d->h[a] * d->h[a]));
        P.hh[a] = (float)(1.0 / (2.0 * d->h[a] * d->h[a]));
    }
    if (planar(*d)) P.ih[2] = 0.f;
    P.znext = d->n[2] > 1 ? d->n[0] * d->n[1] : 0;
    P.tau = (float)d->tau;
    P.rho = (float)d->rho;
    P.tr = (float)(d->tau * d->rho);
    P.tau2 = (float)(d->tau * d->tau);
    P.rho2 = (float)(d->rho * d->rho);
    P.hbar = cell_volume(*d);
    P.qscale = (float)(2.0 * P.hbar);
    P.R = R;
    P.T = T;
    P.u = u;
    P.p = nullptr;
    P.fx = f;
    P.fy = f + P.m0;
    P.fz = f + P.m0 + P.m1;
    P.wx = w;
    P.wy = w + P.m0;
    P.wz = w + P.m0 + P.m1;
    P.zc = zc;
    P.ntx = (int)grid.x;
    P.nty = (int)grid.y;
    P.ntz = (int)grid.z;
    P.partial = nullptr;
    P.dpart = part;
    P.dcount = count;
    P.dout = dev_DS;
    // two or more voxels per cell in x and y bound the front-end node box by
    // the compact layout's (the objective pass uses no owned node box)
    const bool compact = 2 * (d->n[0] - 1) <= d->m[0] && 2 * (d->n[1] - 1) <= d->m[1];
    e = compact ? launch(k_image_obj, grid, dim3(NT), sizeof(ImgSmemC), stream, P)
                : launch(k_image_obj_w, grid, dim3(NT), sizeof(ImgSmemW), stream, P);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "k_image_obj");

    NodeGeom G;
    G.n0 = d->n[0];
    G.n1 = d->n[1];
    G.n2 = d->n[2];
    G.N = N;
    double hy[3];
    for (int a = 0; a < 3; ++a) {
        hy[a] = node_spacing(*d, a);
        G.ihy2[a] = (float)(1.0 / (hy[a] * hy[a]));
    }
    e = launch(k_na_curv_energy, dim3(node_blocks), dim3(256), 0, stream, G, u, part, count + 1, dev_DS + 1,
               node_cell_volume(*d));
    if (e != cudaSuccess) return cuda_check(nullptr, e, "k_na_curv_energy");
    return NGF_OK;
}
