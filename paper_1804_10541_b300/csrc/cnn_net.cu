// Learned initializer: a small 3-D encoder-decoder that maps an image pair
// to a starting displacement for the multilevel Gauss-Newton method, with
// its forward pass, backward pass and Adam update on the device.
//
// The paper starts the multilevel method from u = 0 on the coarsest level
// (Sec. 2.3); the network only supplies another starting point.  Layers
// (channels last, bf16 activations, FP32 accumulation; every convolution is
// the tensor-core kernel of cnn_conv3d.cu):
//
//   x0 = [(R - shift) scale, (T - shift) scale, 0 x 14]       s^3 x 16
//   e1 = relu(conv W1)  s^3 16      p1 = pool2(e1)
//   e2 = relu(conv W2)  s/2 32      p2 = pool2(e2)
//   e3 = relu(conv W3)  s/4 64      p3 = pool2(e3)
//   e4 = relu(conv W4)  s/8 128
//   d3 = relu(conv W5 of up2(e4))   s/4 64;   s3 = d3 + e3
//   d2 = relu(conv W6 of s3)        s/4 64
//   o  = conv W7 of d2 (float)      s/4 16 (channels 0..2 used)
//   u  = out_scale * cell_to_node(o[..., 0:3])   3 x (s/4 + 1)^3 nodes
//   loss = mean ((u - u_target) / out_scale)^2
//
// The backward pass follows the chain rule layer by layer (gradients stored
// as bf16 where they feed a tensor-core operand); weight gradients are
// deterministic tensor-core reductions, so a training step is reproducible.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ngf.h"
#include "ngf_cnn.h"
#include "ngf_launch.cuh"
#include "ngf_plan.h"

namespace ngf {
namespace {

constexpr int NET_NL = 7;
constexpr int NET_CIN[NET_NL] = {16, 16, 32, 64, 128, 64, 64};
constexpr int NET_COUT[NET_NL] = {16, 32, 64, 128, 64, 64, 16};

// 8 bf16 (one 16-byte chunk) <-> 8 floats
__device__ __forceinline__ void unpack8(const uint4 q, float (&f)[8]) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// x0[v] = ((R - shift) scale, (T - shift) scale, 0, ..., 0), 16 channels
__global__ void k_net_input(const float* __restrict__ R, const float* __restrict__ T, uint4* __restrict__ x0,
                            long long V, float shift, float scale) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float f[8] = {(R[v] - shift) * scale, (T[v] - shift) * scale, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        x0[2 * v] = pack8(f);
        x0[2 * v + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// y = mean of the 2x2x2 children, per 8-channel group (cg groups)
__global__ void k_net_pool2(const uint4* __restrict__ x, uint4* __restrict__ y, int B, int s, int cg) {
    const int h = s / 2;
    const long long total = (long long)B * h * h * h * cg;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % cg);
        long long v = i / cg;
        const int px = (int)(v % h), py = (int)((v / h) % h), pz = (int)((v / h / h) % h);
        const long long b = v / ((long long)h * h * h);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 8; ++c) {
            const long long cv = ((b * s + 2 * pz + (c >> 2)) * s + 2 * py + ((c >> 1) & 1)) * s + 2 * px + (c & 1);
            float f[8];
            unpack8(x[cv * cg + g], f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += f[k];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] *= 0.125f;
        y[i] = pack8(acc);
    }
}

// dz[child] = (dp[parent] / 8 + extra[child]) * (mask[child] > 0)
__global__ void k_net_pool2_bwd(const uint4* __restrict__ dp, const uint4* __restrict__ extra,
                                const uint4* __restrict__ mask, uint4* __restrict__ dz, int B, int s, int cg) {
    const int h = s / 2;
    const long long total = (long long)B * s * s * s * cg;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % cg);
        const long long v = i / cg;
        const int x = (int)(v % s), y = (int)((v / s) % s), z = (int)((v / s / s) % s);
        const long long b = v / ((long long)s * s * s);
        const long long pv = ((b * h + z / 2) * h + y / 2) * h + x / 2;
        float d[8], m[8], e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        unpack8(dp[pv * cg + g], d);
        unpack8(mask[i], m);
        if (extra) unpack8(extra[i], e);
        float r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = m[k] > 0.f ? d[k] * 0.125f + e[k] : 0.f;
        dz[i] = pack8(r);
    }
}

// y[child] = x[parent] (nearest upsampling by 2)
__global__ void k_net_up2(const uint4* __restrict__ x, uint4* __restrict__ y, int B, int s, int cg) {
    const int S = 2 * s;
    const long long total = (long long)B * S * S * S * cg;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % cg);
        const long long v = i / cg;
        const int X = (int)(v % S), Y = (int)((v / S) % S), Z = (int)((v / S / S) % S);
        const long long b = v / ((long long)S * S * S);
        y[i] = x[(((b * s + Z / 2) * s + Y / 2) * s + X / 2) * cg + g];
    }
}

// dz[parent] = (sum of dup over the 8 children) * (mask[parent] > 0)
__global__ void k_net_up2_bwd(const uint4* __restrict__ dup, const uint4* __restrict__ mask, uint4* __restrict__ dz,
                              int B, int s, int cg) {
    const int S = 2 * s;
    const long long total = (long long)B * s * s * s * cg;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % cg);
        const long long v = i / cg;
        const int x = (int)(v % s), y = (int)((v / s) % s), z = (int)((v / s / s) % s);
        const long long b = v / ((long long)s * s * s);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 8; ++c) {
            const long long cv = ((b * S + 2 * z + (c >> 2)) * S + 2 * y + ((c >> 1) & 1)) * S + 2 * x + (c & 1);
            float f[8];
            unpack8(dup[cv * cg + g], f);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += f[k];
        }
        float m[8];
        unpack8(mask[i], m);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = m[k] > 0.f ? acc[k] : 0.f;
        dz[i] = pack8(acc);
    }
}

// c = a + b (bf16, FP32 add)
__global__ void k_net_add(const uint4* __restrict__ a, const uint4* __restrict__ b, uint4* __restrict__ c, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float fa[8], fb[8];
        unpack8(a[i], fa);
        unpack8(b[i], fb);
#pragma unroll
        for (int k = 0; k < 8; ++k) fa[k] += fb[k];
        c[i] = pack8(fa);
    }
}

// out = d * (act > 0) (ReLU backward; out may alias d)
__global__ void k_net_mask(const uint4* d, const uint4* __restrict__ act, uint4* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float fd[8], fm[8];
        unpack8(d[i], fd);
        unpack8(act[i], fm);
#pragma unroll
        for (int k = 0; k < 8; ++k) fd[k] = fm[k] > 0.f ? fd[k] : 0.f;
        out[i] = pack8(fd);
    }
}

// Per-axis cell-to-node weights: node k is the mean of cells clamp(k - 1)
// and clamp(k), so cell i receives weight 1/2 from each node whose pair
// contains it (1 when both entries of the pair are i).
__device__ __forceinline__ float c2n_w(int k, int i, int s) {
    const int a = k - 1 < 0 ? 0 : k - 1, b = k > s - 1 ? s - 1 : k;
    return 0.5f * ((a == i) + (b == i));
}

// u[b][d][node] = out_scale * cell_to_node(o[b][..][d]) for d < 3; with a
// target, du = d loss / d u = 2 (u - ut) / (out_scale^2 count) and the
// block's float64 partial of sum ((u - ut) / out_scale)^2.
__global__ void k_net_c2n(const float* __restrict__ o, const float* __restrict__ ut, float* __restrict__ u,
                          float* __restrict__ du, double* __restrict__ part, int B, int s, float out_scale,
                          double inv_count) {
    const int n = s + 1;
    const long long Nn = (long long)n * n * n, total = (long long)B * 3 * Nn;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long node = i % Nn;
        const int d = (int)((i / Nn) % 3);
        const long long b = i / (3 * Nn);
        const int kx = (int)(node % n), ky = (int)((node / n) % n), kz = (int)(node / ((long long)n * n));
        float v = 0.f;
        for (int c = 0; c < 8; ++c) {
            const int ix = min(max(kx - 1 + (c & 1), 0), s - 1);
            const int iy = min(max(ky - 1 + ((c >> 1) & 1), 0), s - 1);
            const int iz = min(max(kz - 1 + (c >> 2), 0), s - 1);
            v += 0.125f * o[(((b * s + iz) * s + iy) * s + ix) * 16 + d];
        }
        v *= out_scale;
        u[i] = v;
        if (ut) {
            const float e = (v - ut[i]) / out_scale;
            acc += (double)e * (double)e;
            du[i] = (float)(2.0 * inv_count) * e / out_scale;
        }
    }
    if (!part) return;
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_net_sum(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < n; ++i) a += part[i];
        *out = a * scale;
    }
}

// do[b][cell][c] = out_scale * sum over nodes of w * du (c < 3), 0 (c >= 3)
__global__ void k_net_c2n_bwd(const float* __restrict__ du, uint4* __restrict__ dout, int B, int s, float out_scale) {
    const int n = s + 1;
    const long long Nn = (long long)n * n * n, total = (long long)B * s * s * s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % s), iy = (int)((i / s) % s), iz = (int)((i / s / s) % s);
        const long long b = i / ((long long)s * s * s);
        float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 8; ++c) {
            const int kx = ix + (c & 1), ky = iy + ((c >> 1) & 1), kz = iz + (c >> 2);
            const float w = c2n_w(kx, ix, s) * c2n_w(ky, iy, s) * c2n_w(kz, iz, s);
            if (w == 0.f) continue;
            const long long node = ((long long)kz * n + ky) * n + kx;
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] += w * du[(b * 3 + d) * Nn + node];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] *= out_scale;
        dout[2 * i] = pack8(g);
        dout[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Adam (Kingma and Ba): m, v moments, bias-corrected step; the bf16 copy of
// the weights is refreshed from the float master.
__global__ void k_net_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, __nv_bfloat16* __restrict__ pb, long long n, float lr, float b1,
                           float b2, float eps, float bc1, float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_net_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

unsigned grid_of(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148LL * 16) g = 148LL * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

struct NetImpl {
    ngf_net_desc d{};
    cudaStream_t stream = nullptr;
    long long P = 0;                      // parameter floats
    long long woff[NET_NL]{}, boff[NET_NL]{};
    float* params = nullptr;              // float master copy
    float* grads = nullptr;
    float* mom1 = nullptr;
    float* mom2 = nullptr;
    __nv_bfloat16* pbf = nullptr;         // bf16 copy (weights are read from it)
    long long step = 0;
    // activations (bf16, channels last) and gradients
    void *x0 = nullptr, *e1 = nullptr, *p1 = nullptr, *e2 = nullptr, *p2 = nullptr, *e3 = nullptr, *p3 = nullptr,
         *e4 = nullptr, *up = nullptr, *d3 = nullptr, *s3 = nullptr, *d2 = nullptr;
    float* o = nullptr;
    float* u = nullptr;
    float* du = nullptr;
    void *dout = nullptr, *dz6 = nullptr, *ds3 = nullptr, *dz5 = nullptr, *dup = nullptr, *dz4 = nullptr,
         *dp3 = nullptr, *dz3 = nullptr, *dp2 = nullptr, *dz2 = nullptr, *dp1 = nullptr, *dz1 = nullptr;
    double* part = nullptr;
    double* loss = nullptr;
    int nparts = 0;
    float *Rb = nullptr, *Tb = nullptr, *Ub = nullptr;  // staging of one training batch
    std::vector<void*> owned;
};

}  // namespace ngf

using namespace ngf;

struct ngf_net {
    NetImpl impl;
};

namespace {

long long net_params(int /*s*/, long long* woff, long long* boff) {
    long long off = 0;
    for (int l = 0; l < NET_NL; ++l) {
        if (woff) woff[l] = off;
        off += 27LL * NET_COUT[l] * NET_CIN[l];
        if (boff) boff[l] = off;
        off += NET_COUT[l];
    }
    return off;
}

ngf_status net_check_desc(const ngf_net_desc* d) {
    if (!d) return set_error(nullptr, NGF_EINVAL, "ngf_net: desc is NULL");
    if (d->s < 8 || d->s % 8 != 0 || d->s > 512)
        return set_error(nullptr, NGF_EINVAL, "ngf_net: s must be a multiple of 8 in [8, 512]");
    if (d->max_batch < 1) return set_error(nullptr, NGF_EINVAL, "ngf_net: max_batch must be >= 1");
    if (!(d->in_scale != 0.0f) || !(d->out_scale > 0.0f) || !std::isfinite(d->in_shift))
        return set_error(nullptr, NGF_EINVAL, "ngf_net: in_scale must be non-zero, out_scale positive");
    const long long s3 = (long long)d->s * d->s * d->s;
    if ((long long)d->max_batch * s3 * 16 >= (1LL << 31) * 8LL)
        return set_error(nullptr, NGF_EBOUNDS, "ngf_net: max_batch * s^3 too large");
    return NGF_OK;
}

#define NET_CU(expr, what)                                           \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return cuda_check(nullptr, _e, what); \
    } while (0)
#define NET_TRY(expr)                \
    do {                             \
        ngf_status _s = (expr);      \
        if (_s != NGF_OK) return _s; \
    } while (0)

ngf_status net_alloc(NetImpl& n, void** p, size_t bytes) {
    NET_CU(dev_alloc(p, bytes, n.stream), "ngf_net: allocate");
    n.owned.push_back(*p);
    return NGF_OK;
}

// forward of B pairs; with ut also the loss gradient du and the loss partials
ngf_status net_forward(NetImpl& n, const float* R, const float* T, int B, const float* ut) {
    const int s = n.d.s, s2 = s / 2, s4 = s / 4, s8 = s / 8;
    const long long v1 = (long long)B * s * s * s, v4 = (long long)B * s4 * s4 * s4;
    cudaStream_t st = n.stream;
    const int bf = NGF_CONV_RELU | NGF_CONV_OUT_BF16;
    auto W = [&](int l) { return (const void*)(n.pbf + n.woff[l]); };
    auto Bi = [&](int l) { return (const float*)(n.params + n.boff[l]); };
    NET_CU(launch(k_net_input, dim3(grid_of(v1)), dim3(256), 0, st, R, T, (uint4*)n.x0, v1, n.d.in_shift, n.d.in_scale),
           "k_net_input");
    NET_TRY(ngf_conv3d_fwd_ex(n.x0, W(0), Bi(0), n.e1, B, s, s, s, 16, 16, bf, st));
    NET_CU(launch(k_net_pool2, dim3(grid_of(v1 / 8 * 2)), dim3(256), 0, st, (const uint4*)n.e1, (uint4*)n.p1, B, s, 2),
           "k_net_pool2");
    NET_TRY(ngf_conv3d_fwd_ex(n.p1, W(1), Bi(1), n.e2, B, s2, s2, s2, 16, 32, bf, st));
    NET_CU(launch(k_net_pool2, dim3(grid_of(v4 / 8 * 4)), dim3(256), 0, st, (const uint4*)n.e2, (uint4*)n.p2, B, s2,
                  4),
           "k_net_pool2");
    NET_TRY(ngf_conv3d_fwd_ex(n.p2, W(2), Bi(2), n.e3, B, s4, s4, s4, 32, 64, bf, st));
    NET_CU(launch(k_net_pool2, dim3(grid_of(v4 / 8 * 8)), dim3(256), 0, st, (const uint4*)n.e3, (uint4*)n.p3, B, s4,
                  8),
           "k_net_pool2");
    NET_TRY(ngf_conv3d_fwd_ex(n.p3, W(3), Bi(3), n.e4, B, s8, s8, s8, 64, 128, bf, st));
    NET_CU(launch(k_net_up2, dim3(grid_of(v4 * 16)), dim3(256), 0, st, (const uint4*)n.e4, (uint4*)n.up, B, s8, 16),
           "k_net_up2");
    NET_TRY(ngf_conv3d_fwd_ex(n.up, W(4), Bi(4), n.d3, B, s4, s4, s4, 128, 64, bf, st));
    NET_CU(launch(k_net_add, dim3(grid_of(v4 * 8)), dim3(256), 0, st, (const uint4*)n.d3, (const uint4*)n.e3,
                  (uint4*)n.s3, v4 * 8),
           "k_net_add");
    NET_TRY(ngf_conv3d_fwd_ex(n.s3, W(5), Bi(5), n.d2, B, s4, s4, s4, 64, 64, bf, st));
    NET_TRY(ngf_conv3d_fwd_ex(n.d2, W(6), Bi(6), n.o, B, s4, s4, s4, 64, 16, 0, st));
    const long long nn = (long long)B * 3 * (s4 + 1) * (s4 + 1) * (s4 + 1);
    NET_CU(launch(k_net_c2n, dim3((unsigned)n.nparts), dim3(256), 0, st, (const float*)n.o, ut, n.u, n.du,
                  ut ? n.part : (double*)nullptr, B, s4, n.d.out_scale, 1.0 / (double)nn),
           "k_net_c2n");
    if (ut)
        NET_CU(launch(k_net_sum, dim3(1), dim3(32), 0, st, (const double*)n.part, n.nparts, 1.0 / (double)nn, n.loss),
               "k_net_sum");
    return NGF_OK;
}

// backward after net_forward(..., ut): parameter gradients into n.grads
ngf_status net_backward(NetImpl& n, int B) {
    const int s = n.d.s, s2 = s / 2, s4 = s / 4, s8 = s / 8;
    const long long v1 = (long long)B * s * s * s, v2 = (long long)B * s2 * s2 * s2, v4 = (long long)B * s4 * s4 * s4,
                    v8 = (long long)B * s8 * s8 * s8;
    cudaStream_t st = n.stream;
    const int ob = NGF_CONV_OUT_BF16;
    auto W = [&](int l) { return (const void*)(n.pbf + n.woff[l]); };
    auto GW = [&](int l) { return n.grads + n.woff[l]; };
    auto GB = [&](int l) { return n.grads + n.boff[l]; };
    NET_CU(launch(k_net_c2n_bwd, dim3(grid_of(v4)), dim3(256), 0, st, (const float*)n.du, (uint4*)n.dout, B, s4,
                  n.d.out_scale),
           "k_net_c2n_bwd");
    // layer 7 (head): o = conv(d2)
    NET_TRY(ngf_conv3d_wgrad(n.dout, n.d2, GW(6), GB(6), B, s4, s4, s4, 64, 16, st));
    NET_TRY(ngf_conv3d_dgrad(n.dout, W(6), n.dz6, B, s4, s4, s4, 64, 16, ob, st));
    NET_CU(launch(k_net_mask, dim3(grid_of(v4 * 8)), dim3(256), 0, st, (const uint4*)n.dz6, (const uint4*)n.d2,
                  (uint4*)n.dz6, v4 * 8),
           "k_net_mask");
    // layer 6: d2 = relu(conv(s3))
    NET_TRY(ngf_conv3d_wgrad(n.dz6, n.s3, GW(5), GB(5), B, s4, s4, s4, 64, 64, st));
    NET_TRY(ngf_conv3d_dgrad(n.dz6, W(5), n.ds3, B, s4, s4, s4, 64, 64, ob, st));
    // s3 = d3 + e3; layer 5: d3 = relu(conv(up))
    NET_CU(launch(k_net_mask, dim3(grid_of(v4 * 8)), dim3(256), 0, st, (const uint4*)n.ds3, (const uint4*)n.d3,
                  (uint4*)n.dz5, v4 * 8),
           "k_net_mask");
    NET_TRY(ngf_conv3d_wgrad(n.dz5, n.up, GW(4), GB(4), B, s4, s4, s4, 128, 64, st));
    NET_TRY(ngf_conv3d_dgrad(n.dz5, W(4), n.dup, B, s4, s4, s4, 128, 64, ob, st));
    // up = up2(e4); layer 4: e4 = relu(conv(p3))
    NET_CU(launch(k_net_up2_bwd, dim3(grid_of(v8 * 16)), dim3(256), 0, st, (const uint4*)n.dup, (const uint4*)n.e4,
                  (uint4*)n.dz4, B, s8, 16),
           "k_net_up2_bwd");
    NET_TRY(ngf_conv3d_wgrad(n.dz4, n.p3, GW(3), GB(3), B, s8, s8, s8, 64, 128, st));
    NET_TRY(ngf_conv3d_dgrad(n.dz4, W(3), n.dp3, B, s8, s8, s8, 64, 128, ob, st));
    // p3 = pool2(e3), e3 also feeds s3; layer 3: e3 = relu(conv(p2))
    NET_CU(launch(k_net_pool2_bwd, dim3(grid_of(v4 * 8)), dim3(256), 0, st, (const uint4*)n.dp3, (const uint4*)n.ds3,
                  (const uint4*)n.e3, (uint4*)n.dz3, B, s4, 8),
           "k_net_pool2_bwd");
    NET_TRY(ngf_conv3d_wgrad(n.dz3, n.p2, GW(2), GB(2), B, s4, s4, s4, 32, 64, st));
    NET_TRY(ngf_conv3d_dgrad(n.dz3, W(2), n.dp2, B, s4, s4, s4, 32, 64, ob, st));
    // p2 = pool2(e2); layer 2: e2 = relu(conv(p1))
    NET_CU(launch(k_net_pool2_bwd, dim3(grid_of(v2 * 4)), dim3(256), 0, st, (const uint4*)n.dp2,
                  (const uint4*)nullptr, (const uint4*)n.e2, (uint4*)n.dz2, B, s2, 4),
           "k_net_pool2_bwd");
    NET_TRY(ngf_conv3d_wgrad(n.dz2, n.p1, GW(1), GB(1), B, s2, s2, s2, 16, 32, st));
    NET_TRY(ngf_conv3d_dgrad(n.dz2, W(1), n.dp1, B, s2, s2, s2, 16, 32, ob, st));
    // p1 = pool2(e1); layer 1: e1 = relu(conv(x0))
    NET_CU(launch(k_net_pool2_bwd, dim3(grid_of(v1 * 2)), dim3(256), 0, st, (const uint4*)n.dp1,
                  (const uint4*)nullptr, (const uint4*)n.e1, (uint4*)n.dz1, B, s, 2),
           "k_net_pool2_bwd");
    NET_TRY(ngf_conv3d_wgrad(n.dz1, n.x0, GW(0), GB(0), B, s, s, s, 16, 16, st));
    return NGF_OK;
}

ngf_status net_args(ngf_net* net, const float* R, const float* T, int B) {
    if (!net) return set_error(nullptr, NGF_EINVAL, "ngf_net: net is NULL");
    if (B < 1 || B > net->impl.d.max_batch) return set_error(nullptr, NGF_EINVAL, "ngf_net: B outside [1, max_batch]");
    if (!R || !T) return set_error(nullptr, NGF_EINVAL, "ngf_net: R and T must be device pointers");
    return NGF_OK;
}

}  // namespace

extern "C" int64_t ngf_net_param_count(const ngf_net_desc* d) {
    if (net_check_desc(d) != NGF_OK) return -1;
    return net_params(d->s, nullptr, nullptr);
}

extern "C" ngf_status ngf_net_create(ngf_net** out, const ngf_net_desc* d, void* cuda_stream) {
    if (!out) return set_error(nullptr, NGF_EINVAL, "ngf_net_create: out is NULL");
    *out = nullptr;
    NET_TRY(net_check_desc(d));
    ngf_net* net = new ngf_net();
    NetImpl& n = net->impl;
    n.d = *d;
    n.stream = static_cast<cudaStream_t>(cuda_stream);
    n.P = net_params(d->s, n.woff, n.boff);
    const int s = d->s, s2 = s / 2, s4 = s / 4, s8 = s / 8, Bm = d->max_batch;
    const size_t v1 = (size_t)Bm * s * s * s, v2 = (size_t)Bm * s2 * s2 * s2, v4 = (size_t)Bm * s4 * s4 * s4,
                 v8 = (size_t)Bm * s8 * s8 * s8, nn = (size_t)Bm * 3 * (s4 + 1) * (s4 + 1) * (s4 + 1);
    const size_t b2 = 2;  // bytes per bf16
    const size_t pf = (size_t)n.P * 4, pb = (size_t)n.P * b2;
    struct Req {
        void** p;
        size_t bytes;
    };
    const Req reqs[] = {
        {(void**)&n.params, pf}, {(void**)&n.grads, pf}, {(void**)&n.mom1, pf},
        {(void**)&n.mom2, pf}, {(void**)&n.pbf, pb}, {&n.x0, v1 * 16 * b2}, {&n.e1, v1 * 16 * b2},
        {&n.p1, v2 * 16 * b2}, {&n.e2, v2 * 32 * b2}, {&n.p2, v4 * 32 * b2}, {&n.e3, v4 * 64 * b2},
        {&n.p3, v8 * 64 * b2}, {&n.e4, v8 * 128 * b2}, {&n.up, v4 * 128 * b2}, {&n.d3, v4 * 64 * b2},
        {&n.s3, v4 * 64 * b2}, {&n.d2, v4 * 64 * b2}, {(void**)&n.o, v4 * 16 * 4}, {(void**)&n.u, nn * 4},
        {(void**)&n.du, nn * 4}, {&n.dout, v4 * 16 * b2}, {&n.dz6, v4 * 64 * b2}, {&n.ds3, v4 * 64 * b2},
        {&n.dz5, v4 * 64 * b2}, {&n.dup, v4 * 128 * b2}, {&n.dz4, v8 * 128 * b2}, {&n.dp3, v8 * 64 * b2},
        {&n.dz3, v4 * 64 * b2}, {&n.dp2, v4 * 32 * b2}, {&n.dz2, v2 * 32 * b2}, {&n.dp1, v2 * 16 * b2},
        {&n.dz1, v1 * 16 * b2}, {(void**)&n.Rb, v1 * 4}, {(void**)&n.Tb, v1 * 4}, {(void**)&n.Ub, nn * 4},
    };
    for (const Req& r : reqs) {
        const ngf_status stt = net_alloc(n, r.p, r.bytes);
        if (stt != NGF_OK) {
            ngf_net_destroy(net);
            return stt;
        }
    }
    n.nparts = (int)grid_of((long long)nn);
    if (net_alloc(n, (void**)&n.part, (size_t)n.nparts * sizeof(double)) != NGF_OK ||
        net_alloc(n, (void**)&n.loss, sizeof(double)) != NGF_OK) {
        ngf_net_destroy(net);
        return NGF_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(n.params, 0, n.P * 4, n.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n.mom1, 0, n.P * 4, n.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n.mom2, 0, n.P * 4, n.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n.pbf, 0, n.P * b2, n.stream);
    if (e != cudaSuccess) {
        ngf_net_destroy(net);
        return cuda_check(nullptr, e, "ngf_net_create: clear");
    }
    *out = net;
    return NGF_OK;
}

extern "C" ngf_status ngf_net_destroy(ngf_net* net) {
    if (!net) return NGF_OK;
    for (void* p : net->impl.owned) dev_free(p, net->impl.stream);
    cudaStreamSynchronize(net->impl.stream);
    delete net;
    return NGF_OK;
}

extern "C" ngf_status ngf_net_set_params(ngf_net* net, const float* params) {
    if (!net || !params) return set_error(nullptr, NGF_EINVAL, "ngf_net_set_params: NULL argument");
    NetImpl& n = net->impl;
    NET_CU(cudaMemcpyAsync(n.params, params, n.P * 4, cudaMemcpyDefault, n.stream), "ngf_net_set_params: copy");
    NET_CU(cudaMemsetAsync(n.mom1, 0, n.P * 4, n.stream), "ngf_net_set_params: clear");
    NET_CU(cudaMemsetAsync(n.mom2, 0, n.P * 4, n.stream), "ngf_net_set_params: clear");
    NET_CU(launch(k_net_to_bf16, dim3(grid_of(n.P)), dim3(256), 0, n.stream, (const float*)n.params, n.pbf, n.P),
           "k_net_to_bf16");
    n.step = 0;
    NET_CU(cudaStreamSynchronize(n.stream), "ngf_net_set_params: sync");
    return NGF_OK;
}

extern "C" ngf_status ngf_net_get_params(ngf_net* net, float* params) {
    if (!net || !params) return set_error(nullptr, NGF_EINVAL, "ngf_net_get_params: NULL argument");
    NetImpl& n = net->impl;
    NET_CU(cudaMemcpyAsync(params, n.params, n.P * 4, cudaMemcpyDefault, n.stream), "ngf_net_get_params: copy");
    NET_CU(cudaStreamSynchronize(n.stream), "ngf_net_get_params: sync");
    return NGF_OK;
}

extern "C" ngf_status ngf_net_forward(ngf_net* net, const float* R, const float* T, int32_t B, float* u) {
    NET_TRY(net_args(net, R, T, B));
    if (!u) return set_error(nullptr, NGF_EINVAL, "ngf_net_forward: u is NULL");
    NetImpl& n = net->impl;
    NET_TRY(net_forward(n, R, T, B, nullptr));
    const int s4 = n.d.s / 4;
    const size_t nn = (size_t)B * 3 * (s4 + 1) * (s4 + 1) * (s4 + 1);
    NET_CU(cudaMemcpyAsync(u, n.u, nn * 4, cudaMemcpyDefault, n.stream), "ngf_net_forward: copy u");
    return NGF_OK;
}

extern "C" ngf_status ngf_net_grad(ngf_net* net, const float* R, const float* T, const float* u_target, int32_t B,
                                   float* grads, double* loss) {
    NET_TRY(net_args(net, R, T, B));
    if (!u_target) return set_error(nullptr, NGF_EINVAL, "ngf_net_grad: u_target is NULL");
    NetImpl& n = net->impl;
    NET_TRY(net_forward(n, R, T, B, u_target));
    NET_TRY(net_backward(n, B));
    if (grads) NET_CU(cudaMemcpyAsync(grads, n.grads, n.P * 4, cudaMemcpyDefault, n.stream), "ngf_net_grad: copy");
    if (loss) {
        NET_CU(cudaMemcpyAsync(loss, n.loss, sizeof(double), cudaMemcpyDefault, n.stream), "ngf_net_grad: loss");
        NET_CU(cudaStreamSynchronize(n.stream), "ngf_net_grad: sync");
    }
    return NGF_OK;
}

namespace {

ngf_status net_adam(NetImpl& n, double lr) {
    n.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    NET_CU(launch(k_net_adam, dim3(grid_of(n.P)), dim3(256), 0, n.stream, n.params, (const float*)n.grads, n.mom1,
                  n.mom2, n.pbf, n.P, (float)lr, (float)b1, (float)b2, 1e-8f,
                  (float)(1.0 - std::pow(b1, (double)n.step)), (float)(1.0 - std::pow(b2, (double)n.step))),
           "k_net_adam");
    return NGF_OK;
}

}  // namespace

extern "C" ngf_status ngf_net_train(ngf_net* net, const float* R, const float* T, const float* u_target,
                                    int32_t npairs, const int32_t* order, int32_t count, int32_t batch, double lr,
                                    double* losses) {
    if (!net || !R || !T || !u_target || !order)
        return set_error(nullptr, NGF_EINVAL, "ngf_net_train: NULL argument");
    NetImpl& n = net->impl;
    if (batch < 1 || batch > n.d.max_batch) return set_error(nullptr, NGF_EINVAL, "ngf_net_train: batch outside [1, max_batch]");
    if (count < 0 || npairs < 1) return set_error(nullptr, NGF_EINVAL, "ngf_net_train: count >= 0, npairs >= 1");
    if (!(lr > 0.0)) return set_error(nullptr, NGF_EINVAL, "ngf_net_train: lr must be positive");
    for (int i = 0; i < count; ++i)
        if (order[i] < 0 || order[i] >= npairs) return set_error(nullptr, NGF_EINVAL, "ngf_net_train: order entry out of range");
    const int s = n.d.s, s4 = s / 4;
    const size_t vox = (size_t)s * s * s, nod = (size_t)3 * (s4 + 1) * (s4 + 1) * (s4 + 1);
    const int nb = (count + batch - 1) / batch;
    double* dl = nullptr;
    if (losses && nb > 0) NET_CU(dev_alloc((void**)&dl, nb * sizeof(double), n.stream), "ngf_net_train: allocate");
    ngf_status st = NGF_OK;
    for (int b = 0; b < nb && st == NGF_OK; ++b) {
        const int B = std::min(batch, count - b * batch);
        for (int j = 0; j < B && st == NGF_OK; ++j) {
            const long long k = order[b * batch + j];
            cudaError_t e = cudaMemcpyAsync(n.Rb + j * vox, R + k * vox, vox * 4, cudaMemcpyDeviceToDevice, n.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(n.Tb + j * vox, T + k * vox, vox * 4, cudaMemcpyDeviceToDevice, n.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(n.Ub + j * nod, u_target + k * nod, nod * 4, cudaMemcpyDeviceToDevice, n.stream);
            if (e != cudaSuccess) st = cuda_check(nullptr, e, "ngf_net_train: gather batch");
        }
        if (st == NGF_OK) st = net_forward(n, n.Rb, n.Tb, B, n.Ub);
        if (st == NGF_OK) st = net_backward(n, B);
        if (st == NGF_OK) st = net_adam(n, lr);
        if (st == NGF_OK && dl) {
            const cudaError_t e = cudaMemcpyAsync(dl + b, n.loss, sizeof(double), cudaMemcpyDeviceToDevice, n.stream);
            if (e != cudaSuccess) st = cuda_check(nullptr, e, "ngf_net_train: loss");
        }
    }
    if (st == NGF_OK && dl) {
        const cudaError_t e = cudaMemcpyAsync(losses, dl, nb * sizeof(double), cudaMemcpyDeviceToHost, n.stream);
        if (e != cudaSuccess) st = cuda_check(nullptr, e, "ngf_net_train: read losses");
    }
    if (dl) dev_free(dl, n.stream);
    if (st == NGF_OK) NET_CU(cudaStreamSynchronize(n.stream), "ngf_net_train: sync");
    return st;
}

extern "C" ngf_status ngf_net_train_step(ngf_net* net, const float* R, const float* T, const float* u_target,
                                         int32_t B, double lr, double* loss) {
    NET_TRY(net_args(net, R, T, B));
    if (!u_target) return set_error(nullptr, NGF_EINVAL, "ngf_net_train_step: u_target is NULL");
    if (!(lr > 0.0)) return set_error(nullptr, NGF_EINVAL, "ngf_net_train_step: lr must be positive");
    NetImpl& n = net->impl;
    NET_TRY(net_forward(n, R, T, B, u_target));
    NET_TRY(net_backward(n, B));
    NET_TRY(net_adam(n, lr));
    if (loss) {
        NET_CU(cudaMemcpyAsync(loss, n.loss, sizeof(double), cudaMemcpyDefault, n.stream), "ngf_net_train_step: loss");
        NET_CU(cudaStreamSynchronize(n.stream), "ngf_net_train_step: sync");
    }
    return NGF_OK;
}
