// C-ABI of libngf_b300: plan creation (grid-conversion tables, tile-partial
// geometry, workspace), validation, and the operator entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ngf_plan.h"

namespace ngf {

std::atomic<int64_t>& launch_counter() {
    static std::atomic<int64_t> c{0};
    return c;
}

static thread_local std::string g_last_error = "no error";

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[256] = {};

cudaError_t dev_alloc(void** ptr, size_t bytes, cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pools[dev], &props);
            if (e != cudaSuccess) return e;
            unsigned long long keep = ~0ull;  // keep freed blocks for the next call
            cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes ? bytes : 1, pool, stream);
}

void dev_free(void* ptr, cudaStream_t stream) {
    if (ptr) cudaFreeAsync(ptr, stream);
}

ngf_status set_error(Plan* p, ngf_status s, const std::string& msg) {
    if (p) p->err = msg;
    g_last_error = msg;
    return s;
}

ngf_status cuda_check(Plan* p, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return NGF_OK;
    return set_error(p, e == cudaErrorMemoryAllocation ? NGF_ENOMEM : NGF_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

#define NGF_TRY(expr)                \
    do {                             \
        ngf_status _s = (expr);      \
        if (_s != NGF_OK) return _s; \
    } while (0)
#define NGF_CU(p, expr, what) NGF_TRY(cuda_check((p), (expr), (what)))

ngf_status validate_desc(const ngf_level_desc* d, std::string& why) {
    if (!d) { why = "level descriptor is NULL"; return NGF_EINVAL; }
    for (int a = 0; a < 3; ++a) {
        if (d->m[a] < 1) { why = "image cells m must be >= 1 on every axis"; return NGF_EINVAL; }
        if (!(d->h[a] > 0.0) || !std::isfinite(d->h[a])) { why = "spacing h must be finite and > 0"; return NGF_EINVAL; }
        if (d->n[a] < 2 && !(a == 2 && d->m[2] == 1 && d->n[2] == 1)) {
            why = "deformation nodes n must be >= 2 on every axis (n[2] == 1 only with m[2] == 1: a 2-D level)";
            return NGF_EINVAL;
        }
        if (d->n[a] - 1 > d->m[a]) {
            why = "deformation grid finer than the image grid: need n_k - 1 <= m_k (Sec. 2.2)";
            return NGF_EINVAL;
        }
    }
    if (d->distance != NGF_DIST_NGF && d->distance != NGF_DIST_SSD) {
        why = "distance must be NGF_DIST_NGF or NGF_DIST_SSD";
        return NGF_EINVAL;
    }
    if (d->distance == NGF_DIST_NGF &&
        (!(d->tau > 0.0) || !(d->rho > 0.0) || !std::isfinite(d->tau) || !std::isfinite(d->rho))) {
        why = "NGF parameters tau and rho must be finite and > 0";
        return NGF_EINVAL;
    }
    if (!(d->alpha >= 0.0) || !std::isfinite(d->alpha)) { why = "alpha must be finite and >= 0"; return NGF_EINVAL; }
    const long long M = (long long)d->m[0] * d->m[1] * d->m[2];
    const long long N = (long long)d->n[0] * d->n[1] * d->n[2];
    if (M > (1LL << 31) - 1 || 3 * N > (1LL << 31) - 1) {
        why = "grid too large: image voxels and 3 x nodes must be < 2^31";
        return NGF_EBOUNDS;
    }
    return NGF_OK;
}

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int grid_for(long long n, int max_blocks) {
    long long b = (n + NT - 1) / NT;
    if (b < 1) b = 1;
    return (int)std::min<long long>(b, max_blocks);
}

// per-axis grid-conversion table of Eq. (grid_conversion): image index v on
// an axis with m cells and n nodes sits at node coordinate (v+1/2)(n-1)/m
static void pw_table(int m, int n, std::vector<int>& f, std::vector<float>& w) {
    f.resize(m);
    w.resize(m);
    for (int v = 0; v < m; ++v) {
        const double c = ((double)v + 0.5) * (double)(n - 1) / (double)m;
        const double fl = std::floor(c);
        f[v] = (int)fl;
        w[v] = (float)(c - fl);
    }
}

// node boxes of the tiles along one axis and, per node, the tiles containing it
static void axis_geometry(int m, int n, const std::vector<int>& f, int TL, int halo, std::vector<int>& b0,
                          std::vector<int>& lo, std::vector<int>& hi, int& ntiles, int& maxbox) {
    ntiles = (m + TL - 1) / TL;
    b0.assign(ntiles, 0);
    std::vector<int> b1(ntiles, 0);
    maxbox = 0;
    for (int t = 0; t < ntiles; ++t) {
        const int start = t * TL, end = std::min(m, start + TL);
        if (halo == 0) {
            b0[t] = f[start];
            b1[t] = f[end - 1] + 1;
        } else {
            b0[t] = f[std::max(start - 1, 0)];
            b1[t] = f[std::min(start + TL, m - 1)] + 1;
        }
        maxbox = std::max(maxbox, b1[t] - b0[t] + 1);
    }
    lo.assign(n, INT_MAX);
    hi.assign(n, -1);
    for (int t = 0; t < ntiles; ++t)
        for (int k = b0[t]; k <= std::min(b1[t], n - 1); ++k) {  // a planar level's box has a second, empty plane
            lo[k] = std::min(lo[k], t);
            hi[k] = std::max(hi[k], t);
        }
}

static ngf_status build_geometry(Plan* p, int halo, const std::vector<int>* f, Geometry& g) {
    std::vector<int> b0[3], lo[3], hi[3];
    int nt[3], mb[3];
    const int TL[3] = {TX, TY, p->zc};
    for (int a = 0; a < 3; ++a) {
        axis_geometry(p->m[a], p->n[a], f[a], TL[a], halo, b0[a], lo[a], hi[a], nt[a], mb[a]);
        for (int k = 0; k < p->n[a]; ++k)
            if (lo[a][k] > hi[a][k]) return set_error(p, NGF_EINVAL, "internal: node not covered by a tile");
    }
    g.ntx = nt[0];
    g.nty = nt[1];
    g.ntz = nt[2];
    g.pbx = mb[0];
    g.pby = mb[1];
    g.pbz = mb[2];
    if (g.partial_floats() >= INT_MAX) return set_error(p, NGF_EBOUNDS, "tile partials exceed 2^31 floats");
    const long long box = (long long)g.pbx * g.pby * g.pbz;
    const long long tile_stride[3] = {3 * box, (long long)g.ntx * 3 * box, (long long)g.ntx * g.nty * 3 * box};
    const long long in_stride[3] = {1, g.pbx, (long long)g.pbx * g.pby};
    const size_t total = 2 * (size_t)(p->n[0] + p->n[1] + p->n[2]) + nt[0] + nt[1] + nt[2];
    std::vector<int> h(total);
    size_t o = 0;
    size_t off[9];
    for (int a = 0; a < 3; ++a) {
        off[2 * a] = o;
        std::copy(lo[a].begin(), lo[a].end(), h.begin() + o);
        o += p->n[a];
        off[2 * a + 1] = o;
        std::copy(hi[a].begin(), hi[a].end(), h.begin() + o);
        o += p->n[a];
    }
    for (int a = 0; a < 3; ++a) {
        off[6 + a] = o;
        for (int t = 0; t < nt[a]; ++t) h[o + t] = (int)(t * tile_stride[a] - b0[a][t] * in_stride[a]);
        o += nt[a];
    }
    NGF_CU(p, dev_alloc((void**)&g.mem, total * sizeof(int), p->stream), "allocate geometry");
    NGF_CU(p, cudaMemcpyAsync(g.mem, h.data(), total * sizeof(int), cudaMemcpyHostToDevice, p->stream), "copy geometry");
    NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    g.xlo = g.mem + off[0];
    g.xhi = g.mem + off[1];
    g.ylo = g.mem + off[2];
    g.yhi = g.mem + off[3];
    g.zlo = g.mem + off[4];
    g.zhi = g.mem + off[5];
    g.xtb = g.mem + off[6];
    g.ytb = g.mem + off[7];
    g.ztb = g.mem + off[8];
    return NGF_OK;
}

// Record one event on the plan's stream for kernel `which` (called before and
// after each image-kernel launch) when timing is enabled and the stream is not
// being captured.
cudaError_t prof_mark(Plan* p, int which) {
    if (!p->prof) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    p->prof_ev[which].push_back(e);
    return cudaEventRecord(e, p->stream);
}

static void clear_prof(Plan* p, int which) {
    for (cudaEvent_t e : p->prof_ev[which]) cudaEventDestroy(e);
    p->prof_ev[which].clear();
}

static void free_plan(Plan* p) {
    for (int k = 0; k < 4; ++k) clear_prof(p, k);
    for (void* ptr : {(void*)p->ftab, (void*)p->wtab, (void*)p->g0.mem, (void*)p->g1.mem, (void*)p->partial,
                      (void*)p->L, (void*)p->ctab, (void*)p->dsc, (void*)p->dpart, (void*)p->dcount,
                      (void*)p->dct_cos, (void*)p->dct_mu, (void*)p->h0_tmp})
        dev_free(ptr, p->stream);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
}

// curvature part of the Jacobi diagonal, per axis: for the 1-D clamped
// Laplacian K (symmetric), d1 = diag(K^2) (column sums of squares) and
// dg = diag(K); k_node_combine forms diag(Lap^T Lap) from them per node.
static void curvature_tables(const Plan* p, std::vector<float>& t) {
    const int tot = p->n[0] + p->n[1] + p->n[2];
    t.assign(2 * tot, 0.f);
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        const double ih2 = 1.0 / (p->hy[a] * p->hy[a]);
        const int nn = p->n[a];
        std::vector<double> d1(nn, 0.0);
        for (int i = 0; i < nn; ++i) {
            double row[3] = {0, 0, 0};  // entries at columns i-1, i, i+1 after clamping
            for (int s = -1; s <= 1; s += 2) {
                const int j = std::min(std::max(i + s, 0), nn - 1);
                row[j - i + 1] += 1.0;
                row[1] -= 1.0;
            }
            for (int k = 0; k < 3; ++k) {
                const int j = i + k - 1;
                if (j >= 0 && j < nn) d1[j] += row[k] * row[k] * ih2 * ih2;
            }
            t[tot + off + i] = (float)(row[1] * ih2);
        }
        for (int i = 0; i < nn; ++i) t[off + i] = (float)d1[i];
        off += nn;
    }
}

static ngf_status build_dct_tables(Plan* p);

static ngf_status create_plan(Plan* p, const ngf_level_desc* d, cudaStream_t stream, int zc_req) {
    std::string why;
    const ngf_status vs = validate_desc(d, why);
    if (vs != NGF_OK) return set_error(p, vs, why);
    p->desc = *d;
    p->stream = stream;
    for (int a = 0; a < 3; ++a) {
        p->m[a] = d->m[a];
        p->n[a] = d->n[a];
        p->hy[a] = node_spacing(*d, a);
    }
    p->M = (long long)p->m[0] * p->m[1] * p->m[2];
    p->N = (long long)p->n[0] * p->n[1] * p->n[2];
    p->hbar = cell_volume(*d);
    p->hbary = node_cell_volume(*d);

    // z-chunking: k chunks per column of tiles, chosen to minimise
    // (rounds of 2 CTAs per SM) x (planes marched per chunk, 7 of them fill
    // and drain the image pass's pipeline); small levels get short chunks,
    // since a CTA's march over its planes is sequential
    int dev = 0, sms = 0;
    NGF_CU(p, cudaGetDevice(&dev), "cudaGetDevice");
    NGF_CU(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
           "cudaDeviceGetAttribute(multiprocessor count)");
    const long long txy = (long long)((p->m[0] + TX - 1) / TX) * ((p->m[1] + TY - 1) / TY);
    const long long slots = 2LL * sms;
    long long best_k = 1, best_cost = LLONG_MAX;
    for (long long k = 1; k <= std::min<long long>(p->m[2], 1024); ++k) {
        const long long zc = (p->m[2] + k - 1) / k;
        const long long chunks = (p->m[2] + zc - 1) / zc;
        const long long cost = ((txy * chunks + slots - 1) / slots) * (zc + IMG_FILL);
        if (cost < best_cost) {
            best_cost = cost;
            best_k = k;
        }
    }
    p->zc = (int)((p->m[2] + best_k - 1) / best_k);
    if (zc_req > 0) p->zc = std::min(zc_req, p->m[2]);

    std::vector<int> f[3];
    std::vector<float> w[3];
    for (int a = 0; a < 3; ++a) pw_table(p->m[a], p->n[a], f[a], w[a]);
    // diagonal variant: a three-node span per axis needs two or more voxels per
    // cell, four nodes otherwise; the per-row windows hold diag_pxw(span) x-nodes
    {
        bool span3 = true;
        for (int a = 0; a < 3; ++a) span3 = span3 && 2 * (p->n[a] - 1) <= p->m[a];
        // runs of equal keys as the kernel's lanes see them: lane l of a tile
        // starting at xs holds the floor of voxel xs - 1 + l (clamped)
        int longest[2] = {1, 1}, widest = 0;  // first x tile (clamped lane 0), the others
        for (int xs = 0; xs < p->m[0]; xs += TX) {
            const int txe = std::min(TX, p->m[0] - xs);
            int run = 1;
            for (int l = 1; l < txe; ++l) {
                const int k0 = f[0][std::max(xs - 2 + l, 0)], k1 = f[0][std::max(xs - 1 + l, 0)];
                run = (k1 == k0) ? run + 1 : 1;
                longest[xs > 0] = std::max(longest[xs > 0], run);
            }
            widest = std::max(widest, f[0][std::min(xs + TX, p->m[0] - 1)] + 2 - f[0][std::max(xs - 1, 0)]);
        }
        for (int k = 0; k < 2; ++k) {
            p->dsteps[k] = 0;
            while ((1 << p->dsteps[k]) < std::min(longest[k], TX)) ++p->dsteps[k];
        }
        p->diag_span3 = span3;
        if (widest > diag_pxw(span3 ? 3 : 4))
            return set_error(p, NGF_EINVAL, "internal: x-node window of the diagonal kernel too small");
    }
    const size_t tl = (size_t)p->m[0] + p->m[1] + p->m[2];
    std::vector<int> fh;
    std::vector<float> wh;
    for (int a = 0; a < 3; ++a) {
        fh.insert(fh.end(), f[a].begin(), f[a].end());
        wh.insert(wh.end(), w[a].begin(), w[a].end());
    }
    NGF_CU(p, dev_alloc((void**)&p->ftab, tl * sizeof(int), p->stream), "allocate tables");
    NGF_CU(p, dev_alloc((void**)&p->wtab, tl * sizeof(float), p->stream), "allocate tables");
    NGF_CU(p, cudaMemcpyAsync(p->ftab, fh.data(), tl * sizeof(int), cudaMemcpyHostToDevice, p->stream), "copy tables");
    NGF_CU(p, cudaMemcpyAsync(p->wtab, wh.data(), tl * sizeof(float), cudaMemcpyHostToDevice, p->stream), "copy tables");

    NGF_TRY(build_geometry(p, 0, f, p->g0));
    NGF_TRY(build_geometry(p, 1, f, p->g1));
    if (p->g0.pbx > NBX || p->g0.pby > NBY || p->g1.pbx > DBX || p->g1.pby > DBY)
        return set_error(p, NGF_EBOUNDS, "internal: tile node box exceeds the kernel's shared-memory box");
    // image-pass layout: the compact one when every tile's halo-1 node box
    // fits it (always with two or more voxels per cell in x and y)
    p->img_wide = p->g1.pbx > ImgSmemC::kNBX || p->g1.pby > ImgSmemC::kNBY;
    const long long pf = std::max(p->g0.partial_floats(), p->g1.partial_floats());
    NGF_CU(p, dev_alloc((void**)&p->partial, pf * sizeof(float), p->stream), "allocate partials");
    NGF_CU(p, dev_alloc((void**)&p->L, 3 * p->N * sizeof(float), p->stream), "allocate L");
    {
        std::vector<float> ct;
        curvature_tables(p, ct);
        NGF_CU(p, dev_alloc((void**)&p->ctab, ct.size() * sizeof(float), p->stream), "allocate curvature tables");
        NGF_CU(p, cudaMemcpyAsync(p->ctab, ct.data(), ct.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream),
               "copy curvature tables");
        NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    }

    p->img_blocks = (int)p->g0.tiles();
    p->diag_blocks = (int)p->g1.tiles();
    p->node_blocks = grid_for(3 * p->N, sms);   // element-wise vector kernels (float4 bodies)
    p->node1_blocks = grid_for(p->N, 4 * sms);      // one thread per node
    p->dpart_len = 2 * (size_t)std::max({p->img_blocks, p->diag_blocks, p->node_blocks, p->node1_blocks, 8 * sms});
    NGF_CU(p, dev_alloc((void**)&p->dsc, 16 * sizeof(double), p->stream), "allocate scalars");
    NGF_CU(p, cudaMemsetAsync(p->dsc, 0, 16 * sizeof(double), p->stream), "clear scalars");
    NGF_CU(p, dev_alloc((void**)&p->dpart, p->dpart_len * sizeof(double), p->stream), "allocate partials64");
    NGF_CU(p, dev_alloc((void**)&p->dcount, 4 * sizeof(unsigned int), p->stream), "allocate counter");
    NGF_CU(p, cudaMemsetAsync(p->dcount, 0, 4 * sizeof(unsigned int), p->stream), "clear counter");

    for (auto kern : {k_image_obj, k_image_grad, k_image_hess})
        NGF_CU(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ImgSmemC)),
               "smem attr");
    for (auto kern : {k_image_obj_w, k_image_grad_w, k_image_hess_w})
        NGF_CU(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ImgSmemW)),
               "smem attr");
    for (auto kern : {k_ssd_obj, k_ssd_grad, k_ssd_hess, k_ssd_diag})
        NGF_CU(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsdSmem)),
               "smem attr");
    for (auto kern : {k_diag, k_diag_s2, k_diag_s3})
        NGF_CU(p, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DiagSmemT<3>)),
               "smem attr");
    NGF_CU(p, cudaFuncSetAttribute(k_diag4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DiagSmemT<4>)), "smem attr");
    return build_dct_tables(p);  // L-BFGS initial Hessian (ngf_h0_solve)
}

NodeGeom node_geom(const Plan* p) {
    NodeGeom G;
    G.n0 = p->n[0];
    G.n1 = p->n[1];
    G.n2 = p->n[2];
    G.N = p->N;
    for (int a = 0; a < 3; ++a) G.ihy2[a] = (float)(1.0 / (p->hy[a] * p->hy[a]));
    G.fN = make_fastdiv((unsigned int)p->N);
    G.fplane = make_fastdiv((unsigned int)(p->n[0] * p->n[1]));
    G.fn0 = make_fastdiv((unsigned int)p->n[0]);
    return G;
}

ImgParams img_params(const Plan* p, const float* R, const float* T, const float* u, const float* pv, int mode,
                     const Geometry& g, double* dout) {
    ImgParams P;
    const ngf_level_desc& d = p->desc;
    P.m0 = p->m[0];
    P.m1 = p->m[1];
    P.m2 = p->m[2];
    P.n0 = p->n[0];
    P.n1 = p->n[1];
    P.n2 = p->n[2];
    P.M = p->M;
    P.N = p->N;
    for (int a = 0; a < 3; ++a) {
        P.ih[a] = (float)(1.0 / d.h[a]);
        P.ihs[a] = (float)(1.0 / (d.h[a] * d.h[a]));
        P.hh[a] = (float)(1.0 / (2.0 * d.h[a] * d.h[a]));
    }
    // a planar level (the 2-D method) samples its one image plane: no z
    // displacement and no z derivative of the template, one node plane
    if (planar(d)) P.ih[2] = 0.f;
    P.znext = p->n[2] > 1 ? p->n[0] * p->n[1] : 0;
    P.tau = (float)d.tau;
    P.rho = (float)d.rho;
    P.tr = (float)(d.tau * d.rho);
    P.tau2 = (float)(d.tau * d.tau);
    P.rho2 = (float)(d.rho * d.rho);
    P.qscale = (float)((mode == MODE_GRAD ? -2.0 : 2.0) * p->hbar);
    P.hbar = p->hbar;
    P.R = R;
    P.T = T;
    P.u = u;
    P.p = pv;
    P.fx = p->ftab;
    P.fy = p->ftab + p->m[0];
    P.fz = p->ftab + p->m[0] + p->m[1];
    P.wx = p->wtab;
    P.wy = p->wtab + p->m[0];
    P.wz = p->wtab + p->m[0] + p->m[1];
    P.zc = p->zc;
    P.ntx = g.ntx;
    P.nty = g.nty;
    P.ntz = g.ntz;
    P.dsteps0 = p->dsteps[0];
    P.dsteps = p->dsteps[1];
    P.pbx = g.pbx;
    P.pby = g.pby;
    P.pbz = g.pbz;
    P.partial = p->partial;
    P.dpart = p->dpart;
    P.dcount = p->dcount;
    P.dout = dout;
    return P;
}

CombineParams combine_params(const Plan* p, const Geometry& g, float* out, const float* L, const float* ctab,
                             const float* dotw, double* dout) {
    CombineParams C;
    C.G = node_geom(p);
    C.partial = p->partial;
    C.box = g.pbx * g.pby * g.pbz;
    C.pbx = g.pbx;
    C.pbxy = g.pbx * g.pby;
    C.xlo = g.xlo;
    C.xhi = g.xhi;
    C.ylo = g.ylo;
    C.yhi = g.yhi;
    C.zlo = g.zlo;
    C.zhi = g.zhi;
    C.xtb = g.xtb;
    C.ytb = g.ytb;
    C.ztb = g.ztb;
    C.L = L;
    C.ctab = ctab;
    C.cscale = (float)(p->desc.alpha * 2.0 * p->hbary);
    C.out = out;
    C.dotw = dotw;
    C.dpart = p->dpart;
    C.dcount = p->dcount;
    C.dout = dout;
    return C;
}

static dim3 img_grid(const Geometry& g) { return dim3(g.ntx, g.nty, g.ntz); }

static bool ssd(const Plan* p) { return p->desc.distance == NGF_DIST_SSD; }

// the image-pass kernel of a mode for this plan's distance and layout, and
// its shared memory
using ImgKernel = void (*)(const ImgParams);
static ImgKernel img_kernel(const Plan* p, int mode) {
    static const ImgKernel tab[3][3] = {{k_image_obj, k_image_grad, k_image_hess},
                                        {k_image_obj_w, k_image_grad_w, k_image_hess_w},
                                        {k_ssd_obj, k_ssd_grad, k_ssd_hess}};
    return tab[ssd(p) ? 2 : (p->img_wide ? 1 : 0)][mode];
}
static size_t img_smem(const Plan* p) {
    return ssd(p) ? sizeof(SsdSmem) : (p->img_wide ? sizeof(ImgSmemW) : sizeof(ImgSmemC));
}

ngf_status objective_impl(Plan* p, const float* R, const float* T, const float* u, double* dD, double* dS) {
    ImgParams P = img_params(p, R, T, u, nullptr, MODE_OBJ, p->g0, dD);
    NGF_CU(p, prof_mark(p, NGF_K_OBJECTIVE), "cudaEventRecord");
    NGF_CU(p, launch(img_kernel(p, MODE_OBJ), img_grid(p->g0), dim3(NT), img_smem(p), p->stream, P),
           "k_image_obj");
    NGF_CU(p, prof_mark(p, NGF_K_OBJECTIVE), "cudaEventRecord");
    NGF_CU(p, launch(k_lap, dim3(p->node1_blocks), dim3(NT), 0, p->stream, node_geom(p), u, p->L, p->dpart,
                     p->dcount, dS, p->hbary),
           "k_lap");
    return NGF_OK;
}

ngf_status gradient_impl(Plan* p, const float* R, const float* T, const float* u, float* g, double* dD,
                         double* dS) {
    ImgParams P = img_params(p, R, T, u, nullptr, MODE_GRAD, img_geom(p), dD);
    NGF_CU(p, prof_mark(p, NGF_K_GRADIENT), "cudaEventRecord");
    NGF_CU(p, launch(img_kernel(p, MODE_GRAD), img_grid(p->g0), dim3(NT), img_smem(p), p->stream, P),
           "k_image_grad");
    NGF_CU(p, prof_mark(p, NGF_K_GRADIENT), "cudaEventRecord");
    NGF_CU(p, launch(k_lap, dim3(p->node1_blocks), dim3(NT), 0, p->stream, node_geom(p), u, p->L, p->dpart,
                     p->dcount, dS, p->hbary),
           "k_lap");
    CombineParams C = combine_params(p, img_geom(p), g, p->L, nullptr, nullptr, nullptr);
    NGF_CU(p, launch(k_node_combine, dim3(p->node1_blocks), dim3(NT), 0, p->stream, C), "k_node_combine");
    return NGF_OK;
}

ngf_status hessvec_impl(Plan* p, const float* R, const float* T, const float* u, const float* pv, float* q,
                        const float* dotw, double* dout) {
    NGF_CU(p, launch(k_lap, dim3(p->node1_blocks), dim3(NT), 0, p->stream, node_geom(p), pv, p->L, p->dpart,
                     p->dcount, (double*)nullptr, 0.0),
           "k_lap");
    ImgParams P = img_params(p, R, T, u, pv, MODE_HESS, img_geom(p), nullptr);
    NGF_CU(p, prof_mark(p, NGF_K_HESSVEC), "cudaEventRecord");
    NGF_CU(p, launch(img_kernel(p, MODE_HESS), img_grid(p->g0), dim3(NT), img_smem(p), p->stream, P),
           "k_image_hess");
    NGF_CU(p, prof_mark(p, NGF_K_HESSVEC), "cudaEventRecord");
    CombineParams C = combine_params(p, img_geom(p), q, p->L, nullptr, dotw, dout);
    NGF_CU(p, launch(k_node_combine, dim3(p->node1_blocks), dim3(NT), 0, p->stream, C), "k_node_combine");
    return NGF_OK;
}

ngf_status diagonal_impl(Plan* p, const float* R, const float* T, const float* u, float* diag) {
    if (ssd(p)) {  // no neighbour coupling: the halo-0 geometry
        ImgParams P = img_params(p, R, T, u, nullptr, MODE_HESS, p->g0, nullptr);
        NGF_CU(p, prof_mark(p, NGF_K_DIAGONAL), "cudaEventRecord");
        NGF_CU(p, launch(k_ssd_diag, img_grid(p->g0), dim3(NT), sizeof(SsdSmem), p->stream, P), "k_ssd_diag");
        NGF_CU(p, prof_mark(p, NGF_K_DIAGONAL), "cudaEventRecord");
        CombineParams C = combine_params(p, p->g0, diag, nullptr, p->ctab, nullptr, nullptr);
        NGF_CU(p, launch(k_node_combine, dim3(p->node1_blocks), dim3(NT), 0, p->stream, C), "k_node_combine");
        return NGF_OK;
    }
    ImgParams P = img_params(p, R, T, u, nullptr, MODE_HESS, p->g1, nullptr);
    NGF_CU(p, prof_mark(p, NGF_K_DIAGONAL), "cudaEventRecord");
    // three-node span: the kernel with the plan's largest shuffle-step count
    // fixed at compile time when it is 2 or 3
    using DiagKernel = void (*)(const ImgParams);
    const int ds = std::max(p->dsteps[0], p->dsteps[1]);
    DiagKernel dk = k_diag4;
    if (p->diag_span3) dk = ds == 2 ? k_diag_s2 : ds == 3 ? k_diag_s3 : k_diag;
    NGF_CU(p, launch(dk, img_grid(p->g1), dim3(NT), p->diag_span3 ? sizeof(DiagSmemT<3>) : sizeof(DiagSmemT<4>),
                     p->stream, P),
           "k_diag");
    NGF_CU(p, prof_mark(p, NGF_K_DIAGONAL), "cudaEventRecord");
    CombineParams C = combine_params(p, p->g1, diag, nullptr, p->ctab, nullptr, nullptr);
    NGF_CU(p, launch(k_node_combine, dim3(p->node1_blocks), dim3(NT), 0, p->stream, C), "k_node_combine");
    return NGF_OK;
}

// DCT-II tables of the L-BFGS initial Hessian: cos(pi m / 2n) for m < 4n
// and the 1-D eigenvalues -4 sin^2(pi k / 2n) / hy^2, per axis
static ngf_status build_dct_tables(Plan* p) {
    const int nt = p->n[0] + p->n[1] + p->n[2];
    std::vector<float> cs(4 * (size_t)nt), mu(nt);
    int oc = 0, om = 0;
    for (int a = 0; a < 3; ++a) {
        const int n = p->n[a];
        for (int m = 0; m < 4 * n; ++m) cs[oc + m] = (float)std::cos(M_PI * m / (2.0 * n));
        for (int k = 0; k < n; ++k) {
            const double sn = std::sin(M_PI * k / (2.0 * n));
            mu[om + k] = (float)(-4.0 * sn * sn / (p->hy[a] * p->hy[a]));
        }
        oc += 4 * n;
        om += n;
    }
    NGF_CU(p, dev_alloc((void**)&p->dct_cos, cs.size() * sizeof(float), p->stream), "allocate DCT tables");
    NGF_CU(p, dev_alloc((void**)&p->dct_mu, mu.size() * sizeof(float), p->stream), "allocate DCT tables");
    NGF_CU(p, dev_alloc((void**)&p->h0_tmp, 3 * p->N * sizeof(float), p->stream), "allocate DCT scratch");
    NGF_CU(p, cudaMemcpyAsync(p->dct_cos, cs.data(), cs.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream),
           "copy DCT tables");
    NGF_CU(p, cudaMemcpyAsync(p->dct_mu, mu.data(), mu.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream),
           "copy DCT tables");
    NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    return NGF_OK;
}

// r = (alpha grad^2 S + gamma I)^{-1} q through the DCT-II eigenbasis of the
// clamped Laplacian
ngf_status h0_impl(Plan* p, double gamma, const float* q, float* r) {
    const NodeGeom G = node_geom(p);
    const dim3 grid(grid_for(3 * p->N, 16 * 148)), blk(NT);
    const float* cosx = p->dct_cos;
    const float* cosy = cosx + 4 * p->n[0];
    const float* cosz = cosy + 4 * p->n[1];
    float* t = p->h0_tmp;
    // forward x, y, z (q -> t -> r -> t), scale, inverse z, y, x (t -> r -> t -> r)
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 0, 0, cosx, q, t), "k_dct_axis");
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 1, 0, cosy, (const float*)t, r), "k_dct_axis");
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 2, 0, cosz, (const float*)r, t), "k_dct_axis");
    NGF_CU(p, launch(k_h0_scale, grid, blk, 0, p->stream, G, (const float*)p->dct_mu,
                     (float)(p->desc.alpha * 2.0 * p->hbary), (float)gamma, t),
           "k_h0_scale");
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 2, 1, cosz, (const float*)t, r), "k_dct_axis");
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 1, 1, cosy, (const float*)r, t), "k_dct_axis");
    NGF_CU(p, launch(k_dct_axis, grid, blk, 0, p->stream, G, 0, 1, cosx, (const float*)t, r), "k_dct_axis");
    return NGF_OK;
}

ngf_status dot_impl(Plan* p, long long n, const float* a, const float* b, double* dout) {
    NGF_CU(p, launch(k_dot, dim3(grid_for(n, (int)(p->dpart_len / 2))), dim3(NT), 0, p->stream, n, a, b, p->dpart,
                     p->dcount, dout),
           "k_dot");
    return NGF_OK;
}

static ngf_status need_dev(Plan* p, std::initializer_list<std::pair<const void*, const char*>> ptrs) {
    for (auto& kv : ptrs)
        if (!is_device_ptr(kv.first))
            return set_error(p, NGF_EINVAL, std::string(kv.second) + " must be a CUDA device (or managed) pointer");
    return NGF_OK;
}

static ngf_status sync_read(Plan* p, double* h, int count) {
    NGF_CU(p, cudaMemcpyAsync(h, p->dsc, count * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "read scalars");
    NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    return NGF_OK;
}

ngf_status plan_create(ngf_plan** out, const ngf_level_desc* desc, cudaStream_t stream, int zc) {
    if (!out) return set_error(nullptr, NGF_EINVAL, "plan output pointer is NULL");
    *out = nullptr;
    ngf_plan* pl = new (std::nothrow) ngf_plan();
    if (!pl) return set_error(nullptr, NGF_ENOMEM, "host allocation failed");
    ngf_status s = create_plan(&pl->impl, desc, stream, zc);
    if (s != NGF_OK) {
        g_last_error = pl->impl.err;
        free_plan(&pl->impl);
        delete pl;
        return s;
    }
    *out = pl;
    return NGF_OK;
}

}  // namespace ngf

using namespace ngf;

extern "C" {

ngf_status ngf_plan_create(ngf_plan** out, const ngf_level_desc* desc, void* cuda_stream) {
    return plan_create(out, desc, (cudaStream_t)cuda_stream, 0);
}

ngf_status ngf_plan_create_ex(ngf_plan** out, const ngf_level_desc* desc, int32_t zc, void* cuda_stream) {
    if (zc < 0) return set_error(nullptr, NGF_EINVAL, "zc must be >= 0");
    return plan_create(out, desc, (cudaStream_t)cuda_stream, zc);
}

ngf_status ngf_plan_destroy(ngf_plan* plan) {
    if (!plan) return NGF_OK;
    free_plan(&plan->impl);
    delete plan;
    return NGF_OK;
}

ngf_status ngf_plan_set_stream(ngf_plan* plan, void* cuda_stream) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    plan->impl.stream = (cudaStream_t)cuda_stream;
    if (plan->impl.graph) cudaGraphExecDestroy(plan->impl.graph);
    plan->impl.graph = nullptr;
    plan->impl.graph_key.clear();
    return NGF_OK;
}

const char* ngf_last_error(const ngf_plan* plan) {
    if (plan) return plan->impl.err.empty() ? "no error" : plan->impl.err.c_str();
    return g_last_error.c_str();
}

ngf_status ngf_objective_dev(ngf_plan* plan, const float* R, const float* T, const float* u, double* dev_DS) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}, {dev_DS, "dev_DS"}}));
    return objective_impl(p, R, T, u, dev_DS, dev_DS + 1);
}

ngf_status ngf_objective(ngf_plan* plan, const float* R, const float* T, const float* u, double* D, double* S) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}}));
    NGF_TRY(objective_impl(p, R, T, u, p->dsc, p->dsc + 1));
    double h[2];
    NGF_TRY(sync_read(p, h, 2));
    if (D) *D = h[0];
    if (S) *S = h[1];
    return NGF_OK;
}

ngf_status ngf_gradient_dev(ngf_plan* plan, const float* R, const float* T, const float* u, float* grad,
                            double* dev_DS) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}, {grad, "grad"}}));
    if (dev_DS && !is_device_ptr(dev_DS)) return set_error(p, NGF_EINVAL, "dev_DS must be a device pointer");
    double* dD = dev_DS ? dev_DS : p->dsc;
    return gradient_impl(p, R, T, u, grad, dD, dD + 1);
}

ngf_status ngf_gradient(ngf_plan* plan, const float* R, const float* T, const float* u, float* grad, double* D,
                        double* S) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}, {grad, "grad"}}));
    NGF_TRY(gradient_impl(p, R, T, u, grad, p->dsc, p->dsc + 1));
    if (D || S) {
        double h[2];
        NGF_TRY(sync_read(p, h, 2));
        if (D) *D = h[0];
        if (S) *S = h[1];
    }
    return NGF_OK;
}

ngf_status gn_hessvec(ngf_plan* plan, const float* R, const float* T, const float* u, const float* pv, float* q) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}, {pv, "p"}, {q, "q"}}));
    if ((const void*)q == (const void*)pv || (const void*)q == (const void*)u)
        return set_error(p, NGF_EINVAL, "q must not alias p or u");
    return hessvec_impl(p, R, T, u, pv, q, nullptr, nullptr);
}

ngf_status curvature_apply(ngf_plan* plan, const float* pv, float* q, double* Sp) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{pv, "p"}}));
    if (q && !is_device_ptr(q)) return set_error(p, NGF_EINVAL, "q must be a device pointer");
    if (q && (const void*)q == (const void*)pv) return set_error(p, NGF_EINVAL, "q must not alias p");
    NGF_CU(p, launch(k_lap, dim3(p->node1_blocks), dim3(NT), 0, p->stream, node_geom(p), pv, p->L, p->dpart, p->dcount,
                     Sp ? p->dsc + 1 : (double*)nullptr, p->hbary),
           "k_lap");
    if (q)
        NGF_CU(p, launch(k_lap2, dim3(p->node_blocks), dim3(NT), 0, p->stream, node_geom(p), (const float*)p->L, q,
                         (float)(2.0 * p->hbary)),
               "k_lap2");
    if (Sp) {
        double h[2];
        NGF_TRY(sync_read(p, h, 2));
        *Sp = h[1];
    }
    return NGF_OK;
}

ngf_status ngf_gn_diagonal(ngf_plan* plan, const float* R, const float* T, const float* u, float* diag) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}, {diag, "diag"}}));
    return diagonal_impl(p, R, T, u, diag);
}

static PcgParams pcg_params(Plan* p, ngf_pcg_state* st, const float* rhs) {
    PcgParams P;
    P.n = 3 * p->N;
    P.x = st->x;
    P.r = st->r;
    P.z = st->z;
    P.d = st->d;
    P.q = st->q;
    P.diag = st->diag;
    P.rhs = rhs;
    P.sc = st->dev_scalars;
    P.part = p->dpart;
    P.count = p->dcount;
    P.rtol = st->rtol;
    auto al = [](const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; };
    P.vec4 = al(P.x) && al(P.r) && al(P.z) && al(P.d) && al(P.q) && al(P.diag);
    return P;
}

static ngf_status check_state(Plan* p, const ngf_pcg_state* st) {
    if (!st) return set_error(p, NGF_EINVAL, "PCG state is NULL");
    return need_dev(p, {{st->x, "x"}, {st->r, "r"}, {st->z, "z"}, {st->d, "d"}, {st->q, "q"}, {st->diag, "diag"},
                        {st->dev_scalars, "dev_scalars"}});
}

ngf_status pcg_init(ngf_plan* plan, ngf_pcg_state* st, const float* rhs) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(check_state(p, st));
    NGF_TRY(need_dev(p, {{rhs, "rhs"}}));
    PcgParams P = pcg_params(p, st, rhs);
    NGF_CU(p, launch(k_pcg_init, dim3(p->node_blocks), dim3(NT), 0, p->stream, P), "k_pcg_init");
    return NGF_OK;
}

static ngf_status pcg_step_impl(Plan* p, ngf_pcg_state* st, const float* R, const float* T, const float* u) {
    PcgParams P = pcg_params(p, st, nullptr);
    NGF_TRY(hessvec_impl(p, R, T, u, st->d, st->q, st->d, st->dev_scalars + PS_DQ));
    NGF_CU(p, launch(k_pcg_update, dim3(p->node_blocks), dim3(NT), 0, p->stream, P), "k_pcg_update");
    NGF_CU(p, launch(k_pcg_dir, dim3(p->node_blocks), dim3(NT), 0, p->stream, P), "k_pcg_dir");
    return NGF_OK;
}

ngf_status pcg_step(ngf_plan* plan, ngf_pcg_state* st, const float* R, const float* T, const float* u) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(check_state(p, st));
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}}));
    return pcg_step_impl(p, st, R, T, u);
}

ngf_status pcg_solve(ngf_plan* plan, ngf_pcg_state* st, const float* R, const float* T, const float* u,
                     int32_t iters, int32_t use_graph) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    NGF_TRY(check_state(p, st));
    NGF_TRY(need_dev(p, {{R, "R"}, {T, "T"}, {u, "u"}}));
    if (iters < 0) return set_error(p, NGF_EINVAL, "iters must be >= 0");
    if (iters == 0) return NGF_OK;
    // the legacy default stream cannot be captured: launch directly there
    if (!use_graph || p->stream == nullptr || p->stream == cudaStreamLegacy) {
        for (int i = 0; i < iters; ++i) NGF_TRY(pcg_step_impl(p, st, R, T, u));
        return NGF_OK;
    }
    std::vector<const void*> key = {st->x, st->r, st->z, st->d, st->q, st->diag, st->dev_scalars, R, T, u};
    if (!(p->graph && p->graph_iters == iters && key == p->graph_key)) {
        if (p->graph) cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
        cudaGraph_t g;
        const int64_t before = launch_counter().load();
        NGF_CU(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        ngf_status s = NGF_OK;
        for (int i = 0; i < iters && s == NGF_OK; ++i) s = pcg_step_impl(p, st, R, T, u);
        cudaError_t e = cudaStreamEndCapture(p->stream, &g);
        if (s != NGF_OK) {
            if (e == cudaSuccess && g) cudaGraphDestroy(g);
            return s;
        }
        NGF_CU(p, e, "cudaStreamEndCapture");
        p->graph_kernels = launch_counter().load() - before;
        launch_counter().fetch_sub(p->graph_kernels);  // captured, not launched
        cudaError_t ie = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        NGF_CU(p, ie, "cudaGraphInstantiate");
        p->graph_key = key;
        p->graph_iters = iters;
    }
    NGF_CU(p, cudaGraphLaunch(p->graph, p->stream), "cudaGraphLaunch");
    launch_counter().fetch_add(p->graph_kernels);
    return NGF_OK;
}

ngf_status pcg_read(ngf_plan* plan, const ngf_pcg_state* st, ngf_pcg_info* info) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    if (!st || !info) return set_error(p, NGF_EINVAL, "state or info is NULL");
    double h[NGF_PCG_NSCALARS];
    NGF_CU(p, cudaMemcpyAsync(h, st->dev_scalars, sizeof(h), cudaMemcpyDeviceToHost, p->stream), "read PCG state");
    NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    info->iters_done = (int32_t)h[PS_ITERS];
    info->status = (int32_t)h[PS_STATUS];
    info->delta = h[PS_DELTA];
    info->rr = h[PS_RR];
    return NGF_OK;
}

ngf_status ngf_profile_enable(ngf_plan* plan, int32_t enable) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    plan->impl.prof = enable != 0;
    return NGF_OK;
}

ngf_status ngf_profile_read(ngf_plan* plan, int32_t which, double* ms, int64_t* launches) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    if (which < 0 || which > 3 || !ms || !launches) return set_error(p, NGF_EINVAL, "bad kernel index or output");
    NGF_CU(p, cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    double total = 0.0;
    const auto& ev = p->prof_ev[which];
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        float t = 0.f;
        NGF_CU(p, cudaEventElapsedTime(&t, ev[i], ev[i + 1]), "cudaEventElapsedTime");
        total += t;
    }
    *ms = total;
    *launches = (int64_t)(ev.size() / 2);
    clear_prof(p, which);
    return NGF_OK;
}

int64_t ngf_launch_count(void) { return launch_counter().load(); }

ngf_status ngf_h0_solve(ngf_plan* plan, double gamma, const float* q, float* r) {
    if (!plan) return set_error(nullptr, NGF_EINVAL, "plan is NULL");
    Plan* p = &plan->impl;
    if (!(gamma > 0.0)) return set_error(p, NGF_EINVAL, "gamma must be > 0");
    NGF_TRY(need_dev(p, {{q, "q"}, {r, "r"}}));
    return h0_impl(p, gamma, q, r);
}

}  // extern "C"
