// Batched form: independent registration problems (pairs) of uneven size,
// each stage of the method one launch for all of them.  Image passes run as
// a persistent grid that takes (pair, tile) work items from a device queue,
// largest first; nodal and PCG kernels give each pair a contiguous range of
// thread blocks.  Each pair keeps its own plan (tile geometry, partials,
// float64 reduction scratch), so its results equal its own plan's bit for bit.
#include <algorithm>
#include <chrono>
#include <climits>
#include <memory>
#include <cmath>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "ngf_launch.cuh"
#include "ngf_plan.h"

namespace ngf {

// device array with a host mirror, uploaded on the owner's stream
template <class T>
struct DevArray {
    T* d = nullptr;
    std::vector<T> h;
    cudaStream_t s = nullptr;
    DevArray() = default;
    DevArray(const DevArray&) = delete;
    DevArray& operator=(const DevArray&) = delete;
    ~DevArray() { release(); }
    void release() {
        dev_free(d, s);
        d = nullptr;
    }
    cudaError_t alloc(size_t n, cudaStream_t st) {
        release();
        s = st;
        h.assign(n, T{});
        return dev_alloc((void**)&d, std::max<size_t>(n, 1) * sizeof(T), st);
    }
    cudaError_t upload() {
        return h.empty() ? cudaSuccess : cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
};

// pairs [p0, p1) of one batched image-pass launch (at most BATCH_TAB) and
// their work items
struct PairRange {
    int p0 = 0, p1 = 0;
    DevArray<int4> items0, items3, items4;  // image tiles (halo 0); NGF diagonal tiles (halo 1) by span
    DevArray<int4> itemsS;                  // SSD diagonal tiles (halo 0)
};

struct Batch {
    int np = 0;
    int zc = 0;
    int sms = 148;
    cudaStream_t stream = nullptr;
    std::vector<ngf_level_desc> descs;
    std::vector<ngf_plan*> plans;
    std::vector<std::unique_ptr<PairRange>> ranges;
    DevArray<unsigned int> qctr;             // queue head, finished CTAs
    DevArray<int> first1, firstv, firstd;    // block ranges: per node, per vector element, dot
    DevArray<int> pair1, pairv, paird;       // pair of every block of those launches
    // parameter tables of the operator calls
    std::vector<ImgParams> t_img;  // image-pass blocks travel with the launch
    DevArray<LapArgs> t_lap;
    DevArray<CombineParams> t_comb;
    Batch() = default;
    Batch(const Batch&) = delete;
    Batch& operator=(const Batch&) = delete;
    ~Batch() { clear_plans(); }
    void clear_plans() {
        for (ngf_plan* p : plans) ngf_plan_destroy(p);
        plans.clear();
    }
    Plan* plan(int k) const { return &plans[k]->impl; }
};

#define B_CU(expr, what)                                             \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return cuda_check(nullptr, _e, what); \
    } while (0)
#define B_TRY(expr)                  \
    do {                             \
        ngf_status _s = (expr);      \
        if (_s != NGF_OK) return _s; \
    } while (0)

static ngf_status fill_segments(DevArray<int>& first, DevArray<int>& pair_of, const std::vector<int>& counts,
                                cudaStream_t s) {
    B_CU(first.alloc(counts.size() + 1, s), "allocate batch segments");
    first.h[0] = 0;
    for (size_t k = 0; k < counts.size(); ++k) {
        if ((long long)first.h[k] + counts[k] > INT_MAX) return set_error(nullptr, NGF_EBOUNDS, "batch too large");
        first.h[k + 1] = first.h[k] + counts[k];
    }
    B_CU(first.upload(), "upload batch segments");
    B_CU(pair_of.alloc(first.h.back(), s), "allocate batch segments");
    for (size_t k = 0; k < counts.size(); ++k)
        for (int b = first.h[k]; b < first.h[k + 1]; ++b) pair_of.h[b] = (int)k;
    B_CU(pair_of.upload(), "upload batch segments");
    return NGF_OK;
}

// (pair, tile) items of one geometry, by decreasing voxel count (the queue
// hands them out in this order, so the largest start first)
static bool is_ssd(const Plan* p) { return p->desc.distance == NGF_DIST_SSD; }

// want_span3: -1 every pair; 0/1 NGF pairs whose diagonal has span 4/3;
// 2 SSD pairs
static void tile_items(const Batch& b, int p0, int p1, bool halo1, int want_span3, std::vector<int4>& out) {
    std::vector<std::pair<long long, int4>> it;
    for (int k = p0; k < p1; ++k) {
        const Plan* p = b.plan(k);
        if (want_span3 == 2 && !is_ssd(p)) continue;
        if ((want_span3 == 0 || want_span3 == 1) && (is_ssd(p) || (int)p->diag_span3 != want_span3)) continue;
        const Geometry& g = halo1 ? p->g1 : p->g0;
        for (int z = 0; z < g.ntz; ++z)
            for (int y = 0; y < g.nty; ++y)
                for (int x = 0; x < g.ntx; ++x) {
                    const long long vx = std::min(TX, p->m[0] - x * TX), vy = std::min(TY, p->m[1] - y * TY);
                    const long long vz = std::min(p->zc, p->m[2] - z * p->zc) + IMG_FILL;  // plus the march's fill planes
                    it.push_back({vx * vy * vz, make_int4(k, x, y, z)});
                }
    }
    std::stable_sort(it.begin(), it.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
    out.clear();
    for (auto& e : it) out.push_back(e.second);
}

// One z-chunk length for all pairs (capped by each pair's depth), chosen to
// minimise the persistent queue's time: the larger of (all items' marched
// planes / slots of 2 CTAs per SM) and the longest item (zc + IMG_FILL planes).
static int batch_zc(const ngf_level_desc* descs, int np, int sms) {
    int best = 1;
    double best_cost = 1e300;
    for (int zc : {1, 2, 4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256}) {
        double work = 0.0;
        int longest = 0;
        for (int k = 0; k < np; ++k) {
            const int m2 = descs[k].m[2], z = std::min(zc, m2);
            const long long tiles = (long long)((descs[k].m[0] + TX - 1) / TX) * ((descs[k].m[1] + TY - 1) / TY);
            work += (double)tiles * ((m2 + z - 1) / z) * (z + IMG_FILL);
            longest = std::max(longest, z + IMG_FILL);
        }
        const double cost = std::max(work / (2.0 * sms), (double)longest);
        if (cost < best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

// shared memory of a batched image pass: NGF pairs in the compact or wide
// layout and SSD pairs share one launch
static size_t batch_img_smem(bool wide) {
    return std::max(sizeof(SsdSmem), wide ? sizeof(ImgSmemW) : sizeof(ImgSmemC));
}

static ngf_status build_batch(Batch* b, int np, const ngf_level_desc* descs, int zc, cudaStream_t stream) {
    b->clear_plans();
    b->np = np;
    b->zc = zc;
    b->stream = stream;
    b->descs.assign(descs, descs + np);
    int dev = 0;
    B_CU(cudaGetDevice(&dev), "cudaGetDevice");
    B_CU(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev),
         "cudaDeviceGetAttribute(multiprocessor count)");
    if (zc == 0) zc = batch_zc(descs, np, b->sms);
    for (int k = 0; k < np; ++k) {
        ngf_plan* pl = nullptr;
        const ngf_status s = plan_create(&pl, &descs[k], stream, zc);
        if (s != NGF_OK) return set_error(nullptr, s, "pair " + std::to_string(k) + ": " + ngf_last_error(nullptr));
        b->plans.push_back(pl);
    }
    b->ranges.clear();
    for (int p0 = 0; p0 < np; p0 += BATCH_TAB) {
        std::unique_ptr<PairRange> r(new (std::nothrow) PairRange());
        if (!r) return set_error(nullptr, NGF_ENOMEM, "host allocation failed");
        r->p0 = p0;
        r->p1 = std::min(np, p0 + BATCH_TAB);
        std::vector<int4> v;
        DevArray<int4>* lists[4] = {&r->items0, &r->items3, &r->items4, &r->itemsS};
        const int want[4] = {-1, 1, 0, 2};
        for (int li = 0; li < 4; ++li) {
            tile_items(*b, r->p0, r->p1, li == 1 || li == 2, want[li], v);
            B_CU(lists[li]->alloc(v.size(), stream), "allocate batch items");
            lists[li]->h = v;
            B_CU(lists[li]->upload(), "upload batch items");
        }
        b->ranges.push_back(std::move(r));
    }
    B_CU(b->qctr.alloc(2, stream), "allocate batch queue");
    B_CU(b->qctr.upload(), "clear batch queue");
    std::vector<int> c1(np), cv(np), cd(np);
    for (int k = 0; k < np; ++k) {
        const Plan* p = b->plan(k);
        c1[k] = p->node1_blocks;
        cv[k] = p->node_blocks;
        cd[k] = grid_for(3 * p->N, (int)(p->dpart_len / 2));
    }
    B_TRY(fill_segments(b->first1, b->pair1, c1, stream));
    B_TRY(fill_segments(b->firstv, b->pairv, cv, stream));
    B_TRY(fill_segments(b->firstd, b->paird, cd, stream));
    b->t_img.assign(np, ImgParams{});
    B_CU(b->t_lap.alloc(np, stream), "allocate batch tables");
    B_CU(b->t_comb.alloc(np, stream), "allocate batch tables");
    const int csmem = (int)batch_img_smem(false), wsmem = (int)batch_img_smem(true), dsmem = (int)sizeof(DiagSmemT<4>), dsmem3 = (int)sizeof(DiagSmemT<3>);
    for (auto kern : {k_batch_image_obj, k_batch_image_grad, k_batch_image_hess})
        B_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, csmem), "smem attr");
    for (auto kern : {k_batch_image_obj_w, k_batch_image_grad_w, k_batch_image_hess_w})
        B_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem), "smem attr");
    for (auto kern : {k_batch_diag, k_batch_diag_s2, k_batch_diag_s3})
        B_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem3), "smem attr");
    B_CU(cudaFuncSetAttribute(k_batch_diag4, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem), "smem attr");
    B_CU(cudaFuncSetAttribute(k_batch_ssd_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsdSmem)),
         "smem attr");
    B_CU(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    return NGF_OK;
}

static BatchQueue queue(const Batch& b, const PairRange& r, const DevArray<int4>& items, const int* active) {
    BatchQueue Q;
    Q.items = items.d;
    Q.nitems = (int)items.h.size();
    Q.pair0 = r.p0;
    Q.active = active;
    Q.next = b.qctr.d;
    Q.done = b.qctr.d + 1;
    return Q;
}

static BatchSegs segs(const Batch& b, const DevArray<int>& first, const int* active) {
    const int* pair_of = (&first == &b.first1) ? b.pair1.d : ((&first == &b.firstv) ? b.pairv.d : b.paird.d);
    return BatchSegs{first.d, pair_of, b.np, active};
}

// the parameter blocks of one range, passed by value with the launch
static void fill_table(const Batch& b, const PairRange& r, const std::vector<ImgParams>& tab, BatchImgTable& T) {
    for (int k = r.p0; k < r.p1; ++k) {
        T.p[k - r.p0] = tab[k];
        T.ssd[k - r.p0] = is_ssd(b.plan(k)) ? 1 : 0;
    }
}

// ---- launch sequences shared by the operator calls and the registration
// (nodal tables already uploaded)

static ngf_status launch_image(const Batch& b, int mode, const std::vector<ImgParams>& tab, const int* active) {
    std::unique_ptr<BatchImgTable> T(new BatchImgTable());
    for (const auto& rp : b.ranges) {
        const PairRange& r = *rp;
        if (r.items0.h.empty()) continue;
        fill_table(b, r, tab, *T);
        const BatchQueue Q = queue(b, r, r.items0, active);
        const dim3 grid(std::min((int)r.items0.h.size(), 2 * b.sms));
        bool wide = false;  // the wide layout when any NGF pair of the range needs it
        for (int k = r.p0; k < r.p1; ++k) wide = wide || (!is_ssd(b.plan(k)) && b.plan(k)->img_wide);
        using BK = void (*)(const BatchQueue, const BatchImgTable);
        static const BK tab2[2][3] = {{k_batch_image_obj, k_batch_image_grad, k_batch_image_hess},
                                      {k_batch_image_obj_w, k_batch_image_grad_w, k_batch_image_hess_w}};
        B_CU(launch(tab2[wide ? 1 : 0][mode], grid, dim3(NT), batch_img_smem(wide), b.stream, Q, *T),
             "k_batch_image");
    }
    return NGF_OK;
}

static ngf_status launch_diag(const Batch& b, const std::vector<ImgParams>& tab, const int* active) {
    std::unique_ptr<BatchImgTable> T(new BatchImgTable());
    for (const auto& rp : b.ranges) {
        const PairRange& r = *rp;
        fill_table(b, r, tab, *T);
        if (!r.items3.h.empty()) {
            // shuffle steps fixed at compile time: the largest any span-3 pair
            // of the range needs (extra steps leave every run sum unchanged)
            int ds = 0;
            for (int k = r.p0; k < r.p1; ++k) {
                const Plan* p = b.plan(k);
                if (!is_ssd(p) && p->diag_span3) ds = std::max({ds, p->dsteps[0], p->dsteps[1]});
            }
            using BatchKernel = void (*)(const BatchQueue, const BatchImgTable);
            const BatchKernel dk = ds == 2 ? k_batch_diag_s2 : ds == 3 ? k_batch_diag_s3 : k_batch_diag;
            const BatchQueue Q = queue(b, r, r.items3, active);
            const dim3 grid(std::min((int)r.items3.h.size(), 2 * b.sms));
            B_CU(launch(dk, grid, dim3(NT), sizeof(DiagSmemT<3>), b.stream, Q, *T), "k_batch_diag");
        }
        if (!r.items4.h.empty()) {
            const BatchQueue Q = queue(b, r, r.items4, active);
            const dim3 grid(std::min((int)r.items4.h.size(), b.sms));
            B_CU(launch(k_batch_diag4, grid, dim3(NT), sizeof(DiagSmemT<4>), b.stream, Q, *T), "k_batch_diag4");
        }
        if (!r.itemsS.h.empty()) {
            const BatchQueue Q = queue(b, r, r.itemsS, active);
            const dim3 grid(std::min((int)r.itemsS.h.size(), 2 * b.sms));
            B_CU(launch(k_batch_ssd_diag, grid, dim3(NT), sizeof(SsdSmem), b.stream, Q, *T), "k_batch_ssd_diag");
        }
    }
    return NGF_OK;
}

static ngf_status launch_lap(const Batch& b, const LapArgs* tab, const int* active) {
    B_CU(launch(k_batch_lap, dim3(b.first1.h.back()), dim3(NT), 0, b.stream, tab, segs(b, b.first1, active)),
         "k_batch_lap");
    return NGF_OK;
}

static ngf_status launch_combine(const Batch& b, const CombineParams* tab, const int* active) {
    B_CU(launch(k_batch_combine, dim3(b.first1.h.back()), dim3(NT), 0, b.stream, tab, segs(b, b.first1, active)),
         "k_batch_combine");
    return NGF_OK;
}

static LapArgs lap_args(const Plan* p, const float* x, double* out) {
    return LapArgs{node_geom(p), x, p->L, p->dpart, p->dcount, out, p->hbary};
}

static ngf_status check_ptrs(const Batch& b, std::initializer_list<std::pair<const void* const*, const char*>> arrs) {
    for (const auto& a : arrs) {
        if (!a.first) return set_error(nullptr, NGF_EINVAL, std::string(a.second) + " array is NULL");
        for (int k = 0; k < b.np; ++k)
            if (!is_device_ptr(a.first[k]))
                return set_error(nullptr, NGF_EINVAL,
                                 std::string(a.second) + "[" + std::to_string(k) + "] is not a device pointer");
    }
    return NGF_OK;
}

// ---- operator calls

static ngf_status batch_hessvec(Batch& b, const float* const* R, const float* const* T, const float* const* u,
                                const float* const* pv, float* const* q) {
    for (int k = 0; k < b.np; ++k) {
        const Plan* p = b.plan(k);
        b.t_lap.h[k] = lap_args(p, pv[k], nullptr);
        b.t_img[k] = img_params(p, R[k], T[k], u[k], pv[k], MODE_HESS, img_geom(p), nullptr);
        b.t_comb.h[k] = combine_params(p, img_geom(p), q[k], p->L, nullptr, nullptr, nullptr);
    }
    B_CU(b.t_lap.upload(), "upload tables");
    B_CU(b.t_comb.upload(), "upload tables");
    B_TRY(launch_lap(b, b.t_lap.d, nullptr));
    B_TRY(launch_image(b, MODE_HESS, b.t_img, nullptr));
    return launch_combine(b, b.t_comb.d, nullptr);
}

static ngf_status rebuild(Batch& b, int zc) {
    std::vector<ngf_level_desc> d = b.descs;
    return build_batch(&b, b.np, d.data(), zc, b.stream);
}

static ngf_status batch_autotune(Batch& b, const float* const* R, const float* const* T, const float* const* u,
                                 const float* const* pv, float* const* q, int* zc_out, double* ms_out) {
    int deepest = 1;
    for (const auto& d : b.descs) deepest = std::max(deepest, d.m[2]);
    std::vector<int> cand;
    for (int z : {8, 16, 24, 32, 48, 64})
        if (z <= deepest || cand.empty()) cand.push_back(std::min(z, deepest));
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t e0, e1;
    B_CU(cudaEventCreate(&e0), "cudaEventCreate");
    B_CU(cudaEventCreate(&e1), "cudaEventCreate");
    int best = cand[0];
    double best_ms = 1e300;
    ngf_status st = NGF_OK;
    for (int z : cand) {
        st = rebuild(b, z);
        if (st != NGF_OK) break;
        st = batch_hessvec(b, R, T, u, pv, q);  // warm-up
        if (st != NGF_OK) break;
        cudaEventRecord(e0, b.stream);
        for (int r = 0; r < 3 && st == NGF_OK; ++r) st = batch_hessvec(b, R, T, u, pv, q);
        cudaEventRecord(e1, b.stream);
        if (st != NGF_OK) break;
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = cuda_check(nullptr, cudaGetLastError(), "autotune timing");
            break;
        }
        if (ms / 3.0 < best_ms) {
            best_ms = ms / 3.0;
            best = z;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NGF_OK) return st;
    if (b.zc != best) B_TRY(rebuild(b, best));
    if (zc_out) *zc_out = best;
    if (ms_out) *ms_out = best_ms;
    return NGF_OK;
}

}  // namespace ngf

using namespace ngf;

struct ngf_batch {
    ngf::Batch impl;
};

extern "C" {

ngf_status ngf_batch_create(ngf_batch** out, int32_t npairs, const ngf_level_desc* descs, int32_t zc,
                            void* cuda_stream) {
    if (!out) return set_error(nullptr, NGF_EINVAL, "batch output pointer is NULL");
    *out = nullptr;
    if (npairs < 1 || !descs) return set_error(nullptr, NGF_EINVAL, "npairs >= 1 and descs required");
    if (zc < 0) return set_error(nullptr, NGF_EINVAL, "zc must be >= 0");
    ngf_batch* b = new (std::nothrow) ngf_batch();
    if (!b) return set_error(nullptr, NGF_ENOMEM, "host allocation failed");
    const ngf_status s = build_batch(&b->impl, npairs, descs, zc, (cudaStream_t)cuda_stream);
    if (s != NGF_OK) {
        delete b;
        return s;
    }
    *out = b;
    return NGF_OK;
}

ngf_status ngf_batch_destroy(ngf_batch* batch) {
    if (!batch) return NGF_OK;
    cudaStream_t s = batch->impl.stream;
    delete batch;
    const cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? NGF_OK : cuda_check(nullptr, e, "cudaStreamSynchronize");
}

int32_t ngf_batch_zc(const ngf_batch* batch) {
    if (!batch || batch->impl.np == 0) return 0;
    return batch->impl.plan(0)->zc;
}

ngf_status ngf_batch_objective(ngf_batch* batch, const float* const* R, const float* const* T,
                               const float* const* u, double* D, double* S) {
    if (!batch) return set_error(nullptr, NGF_EINVAL, "batch is NULL");
    Batch& b = batch->impl;
    B_TRY(check_ptrs(b, {{(const void* const*)R, "R"}, {(const void* const*)T, "T"}, {(const void* const*)u, "u"}}));
    if (!D || !S) return set_error(nullptr, NGF_EINVAL, "D and S must be non-NULL");
    for (int k = 0; k < b.np; ++k) {
        const Plan* p = b.plan(k);
        b.t_img[k] = img_params(p, R[k], T[k], u[k], nullptr, MODE_OBJ, p->g0, p->dsc);
        b.t_lap.h[k] = lap_args(p, u[k], p->dsc + 1);
    }
    B_CU(b.t_lap.upload(), "upload tables");
    B_TRY(launch_image(b, MODE_OBJ, b.t_img, nullptr));
    B_TRY(launch_lap(b, b.t_lap.d, nullptr));
    std::vector<double> h(2);
    for (int k = 0; k < b.np; ++k) {
        B_CU(cudaMemcpyAsync(h.data(), b.plan(k)->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, b.stream),
             "read scalars");
        B_CU(cudaStreamSynchronize(b.stream), "cudaStreamSynchronize");
        D[k] = h[0];
        S[k] = h[1];
    }
    return NGF_OK;
}

ngf_status ngf_batch_gradient(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, float* const* grad) {
    if (!batch) return set_error(nullptr, NGF_EINVAL, "batch is NULL");
    Batch& b = batch->impl;
    B_TRY(check_ptrs(b, {{(const void* const*)R, "R"},
                         {(const void* const*)T, "T"},
                         {(const void* const*)u, "u"},
                         {(const void* const*)grad, "grad"}}));
    for (int k = 0; k < b.np; ++k) {
        const Plan* p = b.plan(k);
        b.t_img[k] = img_params(p, R[k], T[k], u[k], nullptr, MODE_GRAD, img_geom(p), p->dsc);
        b.t_lap.h[k] = lap_args(p, u[k], p->dsc + 1);
        b.t_comb.h[k] = combine_params(p, img_geom(p), grad[k], p->L, nullptr, nullptr, nullptr);
    }
    B_CU(b.t_lap.upload(), "upload tables");
    B_CU(b.t_comb.upload(), "upload tables");
    B_TRY(launch_image(b, MODE_GRAD, b.t_img, nullptr));
    B_TRY(launch_lap(b, b.t_lap.d, nullptr));
    return launch_combine(b, b.t_comb.d, nullptr);
}

ngf_status ngf_batch_hessvec(ngf_batch* batch, const float* const* R, const float* const* T,
                             const float* const* u, const float* const* p, float* const* q) {
    if (!batch) return set_error(nullptr, NGF_EINVAL, "batch is NULL");
    Batch& b = batch->impl;
    B_TRY(check_ptrs(b, {{(const void* const*)R, "R"},
                         {(const void* const*)T, "T"},
                         {(const void* const*)u, "u"},
                         {(const void* const*)p, "p"},
                         {(const void* const*)q, "q"}}));
    return batch_hessvec(b, R, T, u, p, q);
}

ngf_status ngf_batch_diagonal(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, float* const* diag) {
    if (!batch) return set_error(nullptr, NGF_EINVAL, "batch is NULL");
    Batch& b = batch->impl;
    B_TRY(check_ptrs(b, {{(const void* const*)R, "R"},
                         {(const void* const*)T, "T"},
                         {(const void* const*)u, "u"},
                         {(const void* const*)diag, "diag"}}));
    for (int k = 0; k < b.np; ++k) {
        const Plan* p = b.plan(k);
        const Geometry& gd = is_ssd(p) ? p->g0 : p->g1;  // the SSD diagonal needs no halo
        b.t_img[k] = img_params(p, R[k], T[k], u[k], nullptr, MODE_HESS, gd, nullptr);
        b.t_comb.h[k] = combine_params(p, gd, diag[k], nullptr, p->ctab, nullptr, nullptr);
    }
    B_CU(b.t_comb.upload(), "upload tables");
    B_TRY(launch_diag(b, b.t_img, nullptr));
    return launch_combine(b, b.t_comb.d, nullptr);
}

ngf_status ngf_batch_autotune(ngf_batch* batch, const float* const* R, const float* const* T,
                              const float* const* u, const float* const* p, float* const* q, int32_t* zc,
                              double* ms) {
    if (!batch) return set_error(nullptr, NGF_EINVAL, "batch is NULL");
    Batch& b = batch->impl;
    B_TRY(check_ptrs(b, {{(const void* const*)R, "R"},
                         {(const void* const*)T, "T"},
                         {(const void* const*)u, "u"},
                         {(const void* const*)p, "p"},
                         {(const void* const*)q, "q"}}));
    int z = 0;
    B_TRY(batch_autotune(b, R, T, u, p, q, &z, ms));
    if (zc) *zc = z;
    return NGF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched multilevel registration
// ---------------------------------------------------------------------------
namespace ngf {

struct DBuf {  // stream-ordered device buffer
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
    ~DBuf() { dev_free(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return dev_alloc(&p, bytes, st);
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// per-level tables of the registration, built once per level (the pointers
// they hold do not change within a level; the PCG graph replays them)
struct LevelTables {
    std::vector<ImgParams> obj_u, obj_ut, grad, diag, hess;  // travel with the launches
    DevArray<LapArgs> lap_u, lap_ut, lap_d;
    DevArray<CombineParams> comb_grad, comb_diag, comb_hess;
    DevArray<PcgParams> pcg;
    DevArray<DotArgs> dot_gg, dot_gs;
    DevArray<AxpyArgs> trial, accept;
    DevArray<int> act, srch, acc;
};

static size_t pad64(long long n) { return (size_t)((n + 63) / 64 * 64); }

static ngf_status register_batch_impl(int np, const ngf_level_desc* finest, const ngf_options* o,
                                      const float* const* R, const float* const* T, float* const* u_out,
                                      ngf_report* reps, int autotune, cudaStream_t stream) {
    const auto t_start = std::chrono::steady_clock::now();
    const int L = o->levels;
    std::vector<std::vector<ngf_level_desc>> lv(L, std::vector<ngf_level_desc>(np));
    for (int k = 0; k < np; ++k) {
        std::string why;
        const ngf_status vs = validate_desc(&finest[k], why);
        if (vs != NGF_OK) return set_error(nullptr, vs, "pair " + std::to_string(k) + ": " + why);
        for (int l = 0; l < L; ++l) {
            lv[l][k] = level_at(finest[k], l);
            for (int a = 0; a < 3; ++a)
                if (lv[l][k].n[a] > 4096) return set_error(nullptr, NGF_EBOUNDS, "more than 4096 nodes on an axis");
        }
    }
    std::vector<ngf_report> rep(np);
    for (auto& r : rep) r = ngf_report{};

    // scratch for the input checks and the per-pair scalars (32 doubles each:
    // 0 D, 1 S, 2 dot; 8.. PCG state)
    DBuf bsc, bpart, bcnt, btab;
    B_CU(bsc.alloc((size_t)np * 32 * sizeof(double), stream), "allocate scalars");
    B_CU(cudaMemsetAsync(bsc.p, 0, (size_t)np * 32 * sizeof(double), stream), "clear scalars");
    B_CU(bpart.alloc(4096 * sizeof(double), stream), "allocate partials");
    B_CU(bcnt.alloc(4 * sizeof(unsigned int), stream), "allocate counter");
    B_CU(cudaMemsetAsync(bcnt.p, 0, 4 * sizeof(unsigned int), stream), "clear counter");
    B_CU(btab.alloc(3 * 4096 * (sizeof(int) + sizeof(float)), stream), "allocate prolongation tables");
    double* sc = bsc.as<double>();
    for (int k = 0; k < np; ++k) {
        for (const float* img : {R[k], T[k]}) {
            const long long M = (long long)finest[k].m[0] * finest[k].m[1] * finest[k].m[2];
            B_CU(launch(k_nonfinite, dim3(grid_for(M, 2048)), dim3(NT), 0, stream, M, img, bpart.as<double>(),
                        bcnt.as<unsigned int>(), sc + 3),
                 "k_nonfinite");
            double bad = 0.0;
            B_CU(cudaMemcpyAsync(&bad, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, stream), "read check");
            B_CU(cudaStreamSynchronize(stream), "sync");
            if (bad != 0.0) return set_error(nullptr, NGF_ENONFINITE, "pair " + std::to_string(k) + ": image has NaN/Inf");
        }
    }

    // image pyramids (level 0: the caller's arrays)
    std::vector<DBuf> imgs;
    std::vector<std::vector<const float*>> Rl(L, std::vector<const float*>(np)), Tl = Rl;
    for (int k = 0; k < np; ++k) {
        Rl[0][k] = R[k];
        Tl[0][k] = T[k];
        for (int l = 1; l < L; ++l) {
            const ngf_level_desc& f = lv[l - 1][k];
            const long long Mc = (long long)lv[l][k].m[0] * lv[l][k].m[1] * lv[l][k].m[2];
            for (int w = 0; w < 2; ++w) {
                imgs.emplace_back();
                B_CU(imgs.back().alloc(Mc * sizeof(float), stream), "allocate level image");
                float* dst = imgs.back().as<float>();
                const float* src = w ? Tl[l - 1][k] : Rl[l - 1][k];
                B_CU(launch(k_restrict, dim3(grid_for(Mc, 4096)), dim3(NT), 0, stream, f.m[0], f.m[1], f.m[2], src, dst),
                     "k_restrict");
                (w ? Tl : Rl)[l][k] = dst;
            }
        }
    }

    // concatenated nodal vectors, one 256-byte aligned segment per pair
    size_t total = 0;
    for (int k = 0; k < np; ++k) total += pad64(3LL * lv[0][k].n[0] * lv[0][k].n[1] * lv[0][k].n[2]);
    DBuf vec[9];
    for (auto& v : vec) B_CU(v.alloc(total * sizeof(float), stream), "allocate nodal vectors");
    float* u = vec[0].as<float>();
    float* ut = vec[1].as<float>();
    float* const g = vec[2].as<float>();
    float* const dg = vec[3].as<float>();
    float* const x = vec[4].as<float>();
    float* const r = vec[5].as<float>();
    float* const z = vec[6].as<float>();
    float* const d = vec[7].as<float>();
    float* const q = vec[8].as<float>();
    const int start = L - 1;
    B_CU(cudaMemsetAsync(u, 0, total * sizeof(float), stream), "zero u");

    std::vector<size_t> off(np + 1), prev_off;
    for (int l = start; l >= 0; --l) {
        const std::vector<ngf_level_desc>& D = lv[l];
        off[0] = 0;
        for (int k = 0; k < np; ++k) off[k + 1] = off[k] + pad64(3LL * D[k].n[0] * D[k].n[1] * D[k].n[2]);
        if (l != start) {  // prolongate every pair's u from level l+1
            for (int k = 0; k < np; ++k) {
                const ngf_level_desc& c = lv[l + 1][k];
                std::vector<int> tf;
                std::vector<float> tw;
                for (int a = 0; a < 3; ++a)
                    for (int i = 0; i < D[k].n[a]; ++i) {
                        const double cc =
                            D[k].n[a] > 1 ? (double)i * (double)(c.n[a] - 1) / (double)(D[k].n[a] - 1) : 0.0;
                        double fl = std::floor(cc);
                        if (fl > c.n[a] - 2) fl = c.n[a] - 2;
                    if (fl < 0) fl = 0;  // a single node plane (planar level): weight 0
                        tf.push_back((int)fl);
                        tw.push_back((float)(cc - fl));
                    }
                int* dtf = btab.as<int>();
                float* dtw = reinterpret_cast<float*>(dtf + 3 * 4096);
                B_CU(cudaMemcpyAsync(dtf, tf.data(), tf.size() * sizeof(int), cudaMemcpyHostToDevice, stream), "tables");
                B_CU(cudaMemcpyAsync(dtw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, stream), "tables");
                const long long Nc = (long long)c.n[0] * c.n[1] * c.n[2];
                const long long Nf = (long long)D[k].n[0] * D[k].n[1] * D[k].n[2];
                B_CU(launch(k_prolong, dim3(grid_for(3 * Nf, 4096)), dim3(NT), 0, stream, D[k].n[0], D[k].n[1],
                            D[k].n[2], c.n[0], c.n[1], Nc, (const int*)dtf, (const float*)dtw,
                            (const float*)(u + prev_off[k]), ut + off[k]),
                     "k_prolong");
                B_CU(cudaStreamSynchronize(stream), "sync");  // host tables outlive the copies
            }
            std::swap(u, ut);
        }
        prev_off = off;

        Batch b;
        B_TRY(build_batch(&b, np, D.data(), o->zc, stream));
        auto seg = [&](float* base, int k) { return base + off[k]; };
        if (autotune) {
            B_CU(cudaMemsetAsync(d, 0, total * sizeof(float), stream), "zero d");
            std::vector<const float*> U(np), DD(np);
            std::vector<float*> QQ(np);
            for (int k = 0; k < np; ++k) {
                U[k] = seg(u, k);
                DD[k] = seg(d, k);
                QQ[k] = seg(q, k);
            }
            B_TRY(batch_autotune(b, Rl[l].data(), Tl[l].data(), U.data(), DD.data(), QQ.data(), nullptr, nullptr));
        }

        LevelTables tb;
        auto A = [&](auto& t) { return t.alloc(np, stream); };
        for (auto* t : {&tb.obj_u, &tb.obj_ut, &tb.grad, &tb.diag, &tb.hess}) t->assign(np, ImgParams{});
        B_CU(A(tb.lap_u), "tables");
        B_CU(A(tb.lap_ut), "tables"); B_CU(A(tb.lap_d), "tables"); B_CU(A(tb.comb_grad), "tables");
        B_CU(A(tb.comb_diag), "tables"); B_CU(A(tb.comb_hess), "tables"); B_CU(A(tb.pcg), "tables");
        B_CU(A(tb.dot_gg), "tables"); B_CU(A(tb.dot_gs), "tables"); B_CU(A(tb.trial), "tables");
        B_CU(A(tb.accept), "tables"); B_CU(A(tb.act), "tables"); B_CU(A(tb.srch), "tables"); B_CU(A(tb.acc), "tables");
        auto aligned = [](const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; };
        for (int k = 0; k < np; ++k) {
            const Plan* p = b.plan(k);
            double* sk = sc + 32 * k;
            const long long n = 3 * p->N;
            const float *Rk = Rl[l][k], *Tk = Tl[l][k];
            tb.obj_u[k] = img_params(p, Rk, Tk, seg(u, k), nullptr, MODE_OBJ, p->g0, sk);
            tb.obj_ut[k] = img_params(p, Rk, Tk, seg(ut, k), nullptr, MODE_OBJ, p->g0, sk);
            tb.grad[k] = img_params(p, Rk, Tk, seg(u, k), nullptr, MODE_GRAD, img_geom(p), sk);
            const Geometry& gd = is_ssd(p) ? p->g0 : p->g1;
            tb.diag[k] = img_params(p, Rk, Tk, seg(u, k), nullptr, MODE_HESS, gd, nullptr);
            tb.hess[k] = img_params(p, Rk, Tk, seg(u, k), seg(d, k), MODE_HESS, img_geom(p), nullptr);
            tb.lap_u.h[k] = lap_args(p, seg(u, k), sk + 1);
            tb.lap_ut.h[k] = lap_args(p, seg(ut, k), sk + 1);
            tb.lap_d.h[k] = lap_args(p, seg(d, k), nullptr);
            tb.comb_grad.h[k] = combine_params(p, img_geom(p), seg(g, k), p->L, nullptr, nullptr, nullptr);
            tb.comb_diag.h[k] = combine_params(p, gd, seg(dg, k), nullptr, p->ctab, nullptr, nullptr);
            tb.comb_hess.h[k] = combine_params(p, img_geom(p), seg(q, k), p->L, nullptr, seg(d, k), sk + 8 + PS_DQ);
            PcgParams& P = tb.pcg.h[k];
            P.n = n;
            P.x = seg(x, k);
            P.r = seg(r, k);
            P.z = seg(z, k);
            P.d = seg(d, k);
            P.q = seg(q, k);
            P.diag = seg(dg, k);
            P.rhs = seg(r, k);
            P.sc = sk + 8;
            P.part = p->dpart;
            P.count = p->dcount;
            P.rtol = o->pcg_rtol;
            P.vec4 = aligned(P.x) && aligned(P.r) && aligned(P.z) && aligned(P.d) && aligned(P.q) && aligned(P.diag);
            tb.dot_gg.h[k] = DotArgs{n, seg(g, k), seg(g, k), p->dpart, p->dcount, sk + 2};
            tb.dot_gs.h[k] = DotArgs{n, seg(g, k), seg(x, k), p->dpart, p->dcount, sk + 2};
            tb.trial.h[k] = AxpyArgs{n, 1.0f, seg(u, k), seg(x, k), seg(ut, k)};
            tb.accept.h[k] = AxpyArgs{n, 0.0f, seg(ut, k), nullptr, seg(u, k)};
        }
        for (auto* t : {&tb.lap_u, &tb.lap_ut, &tb.lap_d}) B_CU(t->upload(), "upload tables");
        for (auto* t : {&tb.comb_grad, &tb.comb_diag, &tb.comb_hess}) B_CU(t->upload(), "upload tables");
        for (auto* t : {&tb.dot_gg, &tb.dot_gs}) B_CU(t->upload(), "upload tables");
        B_CU(tb.pcg.upload(), "upload tables");
        B_CU(tb.accept.upload(), "upload tables");

        const dim3 gv(b.firstv.h.back()), gd(b.firstd.h.back());
        int* act = tb.act.d;
        auto pcg_iteration = [&]() -> ngf_status {
            B_TRY(launch_lap(b, tb.lap_d.d, act));
            B_TRY(launch_image(b, MODE_HESS, tb.hess, act));
            B_TRY(launch_combine(b, tb.comb_hess.d, act));
            B_CU(launch(k_batch_pcg_update, gv, dim3(NT), 0, stream, (const PcgParams*)tb.pcg.d, segs(b, b.firstv, act)),
                 "k_batch_pcg_update");
            B_CU(launch(k_batch_pcg_dir, gv, dim3(NT), 0, stream, (const PcgParams*)tb.pcg.d, segs(b, b.firstv, act)),
                 "k_batch_pcg_dir");
            return NGF_OK;
        };
        cudaGraphExec_t graph = nullptr;
        int64_t graph_kernels = 0;
        struct GraphGuard {
            cudaGraphExec_t* g;
            ~GraphGuard() {
                if (*g) cudaGraphExecDestroy(*g);
            }
        } graph_guard{&graph};
        // the legacy default stream cannot be captured: direct launches there
        if (o->use_graph && o->pcg_iters > 0 && stream != nullptr && stream != cudaStreamLegacy) {
            const int64_t before = launch_counter().load();
            cudaGraph_t gr = nullptr;
            const cudaError_t be = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
            if (be != cudaSuccess) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                    cudaStreamEndCapture(stream, &gr);
                    if (gr) cudaGraphDestroy(gr);
                }
                return cuda_check(nullptr, be, "cudaStreamBeginCapture");
            }
            ngf_status cs = NGF_OK;
            for (int it = 0; it < o->pcg_iters && cs == NGF_OK; ++it) cs = pcg_iteration();
            const cudaError_t ce = cudaStreamEndCapture(stream, &gr);
            if (cs != NGF_OK) {
                if (gr) cudaGraphDestroy(gr);
                return cs;
            }
            B_CU(ce, "cudaStreamEndCapture");
            const cudaError_t ie = cudaGraphInstantiate(&graph, gr, 0);
            cudaGraphDestroy(gr);
            B_CU(ie, "cudaGraphInstantiate");
            graph_kernels = launch_counter().load() - before;
            launch_counter().fetch_sub(graph_kernels);  // captured, counted when replayed
        }

        std::vector<int> active(np, 1);
        std::vector<double> hsc((size_t)np * 32), J0(np), gg(np), gs(np), eta(np);
        auto read_scalars = [&]() -> ngf_status {
            B_CU(cudaMemcpyAsync(hsc.data(), sc, hsc.size() * sizeof(double), cudaMemcpyDeviceToHost, stream),
                 "read scalars");
            B_CU(cudaStreamSynchronize(stream), "sync");
            return NGF_OK;
        };
        auto put = [&](DevArray<int>& t, const std::vector<int>& v) {
            t.h = v;
            return t.upload();
        };
        for (int it = 0; it < o->gn_iters; ++it) {
            if (std::none_of(active.begin(), active.end(), [](int a) { return a != 0; })) break;
            B_CU(put(tb.act, active), "upload mask");
            B_TRY(launch_image(b, MODE_GRAD, tb.grad, act));
            B_TRY(launch_lap(b, tb.lap_u.d, act));
            B_TRY(launch_combine(b, tb.comb_grad.d, act));
            B_CU(launch(k_batch_dot, gd, dim3(NT), 0, stream, (const DotArgs*)tb.dot_gg.d, segs(b, b.firstd, act)),
                 "k_batch_dot");
            B_TRY(read_scalars());
            for (int k = 0; k < np; ++k) {
                if (!active[k]) continue;
                J0[k] = hsc[32 * k] + D[k].alpha * hsc[32 * k + 1];
                gg[k] = hsc[32 * k + 2];
                if (gg[k] == 0.0) active[k] = 0;  // stationary point
            }
            if (std::none_of(active.begin(), active.end(), [](int a) { return a != 0; })) break;
            B_CU(put(tb.act, active), "upload mask");
            // Jacobi diagonal at the level's first step, then every diag_every steps
            if (o->diag_every > 0 ? it % o->diag_every == 0 : it == 0) {
                B_TRY(launch_diag(b, tb.diag, act));
                B_TRY(launch_combine(b, tb.comb_diag.d, act));
            }
            B_CU(launch(k_scale, dim3(grid_for((long long)off[np], 4 * b.sms)), dim3(NT), 0, stream,
                        (long long)off[np], -1.0f, (const float*)g, r),
                 "k_scale");
            B_CU(launch(k_batch_pcg_init, gv, dim3(NT), 0, stream, (const PcgParams*)tb.pcg.d, segs(b, b.firstv, act)),
                 "k_batch_pcg_init");
            if (graph) {
                B_CU(cudaGraphLaunch(graph, stream), "cudaGraphLaunch");
                launch_counter().fetch_add(graph_kernels);
            } else {
                for (int i = 0; i < o->pcg_iters; ++i) B_TRY(pcg_iteration());
            }
            B_CU(launch(k_batch_dot, gd, dim3(NT), 0, stream, (const DotArgs*)tb.dot_gs.d, segs(b, b.firstd, act)),
                 "k_batch_dot");
            B_TRY(read_scalars());
            std::vector<int> srch(np, 0), acc(np, 0);
            for (int k = 0; k < np; ++k) {
                if (!active[k]) continue;
                const Plan* p = b.plan(k);
                rep[k].hessvec_voxels += (int64_t)o->pcg_iters * p->M;
                rep[k].pcg_total += (int32_t)hsc[32 * k + 8 + PS_ITERS];
                gs[k] = hsc[32 * k + 2];
                if (!(gs[k] < 0.0)) {  // not a descent direction: steepest descent
                    B_CU(launch(k_scale, dim3(p->node_blocks), dim3(NT), 0, stream, 3 * p->N, -1.0f,
                                (const float*)seg(g, k), seg(x, k)),
                         "k_scale");
                    gs[k] = -gg[k];
                }
                eta[k] = 1.0;
                srch[k] = 1;
            }
            for (int t = 0; t < o->ls_max; ++t) {
                if (std::none_of(srch.begin(), srch.end(), [](int a) { return a != 0; })) break;
                for (int k = 0; k < np; ++k) tb.trial.h[k].eta = (float)eta[k];
                B_CU(tb.trial.upload(), "upload tables");
                B_CU(put(tb.srch, srch), "upload mask");
                B_CU(launch(k_batch_axpy, gv, dim3(NT), 0, stream, (const AxpyArgs*)tb.trial.d,
                            segs(b, b.firstv, tb.srch.d)),
                     "k_batch_axpy");
                B_TRY(launch_image(b, MODE_OBJ, tb.obj_ut, tb.srch.d));
                B_TRY(launch_lap(b, tb.lap_ut.d, tb.srch.d));
                B_TRY(read_scalars());
                for (int k = 0; k < np; ++k) {
                    if (!srch[k]) continue;
                    rep[k].ls_trials++;
                    const double J = hsc[32 * k] + D[k].alpha * hsc[32 * k + 1];
                    if (J <= J0[k] + o->armijo_c1 * eta[k] * gs[k]) {
                        srch[k] = 0;
                        acc[k] = 1;
                    } else {
                        eta[k] *= 0.5;
                    }
                }
            }
            for (int k = 0; k < np; ++k) {
                if (!active[k]) continue;
                if (acc[k]) {
                    rep[k].gn_done++;
                } else {
                    rep[k].ls_fail++;
                    rep[k].status = NGF_ELINESEARCH;
                    active[k] = 0;
                }
            }
            if (std::any_of(acc.begin(), acc.end(), [](int a) { return a != 0; })) {
                B_CU(put(tb.acc, acc), "upload mask");
                B_CU(launch(k_batch_axpy, gv, dim3(NT), 0, stream, (const AxpyArgs*)tb.accept.d,
                            segs(b, b.firstv, tb.acc.d)),
                     "k_batch_axpy");
            }
        }
        // objective at the level's result, every pair
        B_TRY(launch_image(b, MODE_OBJ, tb.obj_u, nullptr));
        B_TRY(launch_lap(b, tb.lap_u.d, nullptr));
        B_TRY(read_scalars());
        for (int k = 0; k < np; ++k) {
            rep[k].D = hsc[32 * k];
            rep[k].S = hsc[32 * k + 1];
            rep[k].J = rep[k].D + D[k].alpha * rep[k].S;
        }
    }
    for (int k = 0; k < np; ++k) {
        const long long n = 3LL * lv[0][k].n[0] * lv[0][k].n[1] * lv[0][k].n[2];
        B_CU(cudaMemcpyAsync(u_out[k], u + off[k], n * sizeof(float), cudaMemcpyDeviceToDevice, stream), "copy u_out");
    }
    B_CU(cudaStreamSynchronize(stream), "sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    for (int k = 0; k < np; ++k) {
        rep[k].seconds = secs;
        reps[k] = rep[k];
    }
    return NGF_OK;
}

}  // namespace ngf

extern "C" ngf_status register_batch(int32_t npairs, const ngf_level_desc* finest, const ngf_options* o,
                                     const float* const* R, const float* const* T, float* const* u_out,
                                     ngf_report* reports, int32_t autotune, void* cuda_stream) {
    if (npairs < 1 || !finest || !o || !R || !T || !u_out || !reports)
        return set_error(nullptr, NGF_EINVAL, "npairs >= 1 and non-NULL finest, opts, R, T, u_out, reports required");
    if (o->levels < 1 || o->levels > 16) return set_error(nullptr, NGF_EINVAL, "levels must be in [1, 16]");
    if (o->gn_iters < 0 || o->pcg_iters < 0 || o->ls_max < 1)
        return set_error(nullptr, NGF_EINVAL, "gn_iters, pcg_iters >= 0 and ls_max >= 1 required");
    if (o->u_init) return set_error(nullptr, NGF_EINVAL, "u_init is not supported by the batched registration");
    if (o->gn_iters_finest != 0 || o->j_target != 0.0)
        return set_error(nullptr, NGF_EINVAL, "gn_iters_finest and j_target are not supported by the batched registration");
    if (o->method != NGF_METHOD_GN)
        return set_error(nullptr, NGF_EINVAL, "the batched registration runs Gauss-Newton only");
    if (o->zc < 0 || o->diag_every < 0) return set_error(nullptr, NGF_EINVAL, "zc and diag_every must be >= 0");
    for (int k = 0; k < npairs; ++k)
        for (const void* ptr : {(const void*)R[k], (const void*)T[k], (const void*)u_out[k]})
            if (!is_device_ptr(ptr))
                return set_error(nullptr, NGF_EINVAL, "pair " + std::to_string(k) + ": R, T, u_out must be device pointers");
    return register_batch_impl(npairs, finest, o, R, T, u_out, reports, autotune, (cudaStream_t)cuda_stream);
}
