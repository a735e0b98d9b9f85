// Multilevel Gauss-Newton registration (Sec. 2.3): image pyramid and
// prolongation on the device, per-level Gauss-Newton steps with a
// Jacobi-preconditioned CG solve (optionally one captured CUDA graph per
// solve) and Armijo backtracking decided in float64.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "ngf_plan.h"

namespace ngf {

// coarse-to-fine level sequence: each coarser level halves image cells and
// deformation cells (ceil) and keeps the physical extent of the domain
ngf_level_desc level_at(const ngf_level_desc& finest, int level) {
    ngf_level_desc d = finest;
    const bool flat = planar(finest);  // a 2-D level stays planar on every level
    for (int k = 0; k < level; ++k)
        for (int a = 0; a < (flat ? 2 : 3); ++a) {
            const int m = d.m[a], mc = (m + 1) / 2;
            int cc = d.n[a] / 2;  // ceil((n - 1) / 2) deformation cells
            if (cc > mc) cc = mc;
            if (cc < 1) cc = 1;
            d.h[a] = d.h[a] * (double)m / (double)mc;
            d.m[a] = mc;
            d.n[a] = cc + 1;
        }
    return d;
}

struct DevBuf {
    void* ptr = nullptr;
    cudaStream_t stream = nullptr;
    ~DevBuf() { dev_free(ptr, stream); }
    template <class T>
    T* as() const { return static_cast<T*>(ptr); }
};

struct PlanGuard {
    ngf_plan* p = nullptr;
    ~PlanGuard() { ngf_plan_destroy(p); }
};

}  // namespace ngf

using namespace ngf;

#define DRV_CU(expr, what)                                           \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return cuda_check(nullptr, _e, what); \
    } while (0)
#define DRV_TRY(expr)                \
    do {                             \
        ngf_status _s = (expr);      \
        if (_s != NGF_OK) return _s; \
    } while (0)

// Armijo backtracking (Sec. 2.3): the first eta in 1, 1/2, 1/4, ... (at
// most ls_max) with J(u + eta s) <= J0 + c1 eta gs.  On levels of up to 2^21
// voxels a host round trip costs more than an objective pass, so four trial
// points are evaluated per round trip (each into its own float64 slots,
// dsc[16..23]); the decision, the accepted point and the trial count are
// those of evaluating them one by one.  On return ut = u + eta s.
static ngf_status armijo(Plan* p, const ngf_level_desc& d, const ngf_options* o, const float* R, const float* T,
                         const float* u, const float* s, float* ut, double J0, double gs, double* dsc,
                         ngf_report& r, bool& accepted) {
    cudaStream_t stream = p->stream;
    const long long n = 3 * p->N;
    const dim3 gv(p->node_blocks), blk(NT);
    const int K = (p->M <= (1LL << 21)) ? 4 : 1;
    accepted = false;
    double eta = 1.0;
    int t = 0;
    while (t < o->ls_max && !accepted) {
        const int k = std::min(K, o->ls_max - t);
        double e = eta;
        for (int j = 0; j < k; ++j, e *= 0.5) {
            DRV_CU(launch(k_axpy, gv, blk, 0, stream, n, (float)e, u, s, ut), "k_axpy");
            DRV_TRY(objective_impl(p, R, T, ut, dsc + 16 + 2 * j, dsc + 17 + 2 * j));
        }
        double h[8];
        DRV_CU(cudaMemcpyAsync(h, dsc + 16, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, stream), "read J");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        int j = 0;
        for (; j < k; ++j) {
            r.ls_trials++;
            if (h[2 * j] + d.alpha * h[2 * j + 1] <= J0 + o->armijo_c1 * eta * gs) {
                accepted = true;
                break;
            }
            eta *= 0.5;
        }
        t += k;
        if (accepted && j != k - 1)  // ut holds the round's last point
            DRV_CU(launch(k_axpy, gv, blk, 0, stream, n, (float)eta, u, s, ut), "k_axpy");
    }
    return NGF_OK;
}

// L-BFGS on one level (Sec. 2.3.2): two-loop recursion with H0 = alpha
// grad^2 S + gamma I (ngf_h0_solve), the Armijo rule of the Gauss-Newton
// level, pairs (s, y) = (u_{k+1} - u_k, g_{k+1} - g_k) kept when s^T y > 0
// in a ring of `lbfgs_memory`, steepest descent when the direction is not a
// descent direction.  u/ut are swapped on acceptance like the Gauss-Newton
// loop's.  lb: float64 scalars, [0, m) s.q, [m, 2m) a, [2m, 3m) y.r, 3m s.y.
static ngf_status lbfgs_level(Plan* p, const ngf_level_desc& d, const ngf_options* o, const float* R, const float* T,
                              float*& u, float*& ut, float* g, float* dir, float* gp, float* sl, float* yt,
                              float* Sr, float* Yr, double* lb, double* dsc, ngf_report& r) {
    cudaStream_t stream = p->stream;
    const long long n = 3 * p->N;
    const int m = o->lbfgs_memory;
    const dim3 gv(p->node_blocks), blk(NT);
    double gamma = o->lbfgs_gamma;
    if (!(gamma > 0.0)) {  // mean of the Gauss-Newton diagonal at the level's start
        DRV_TRY(diagonal_impl(p, R, T, u, dir));
        DRV_TRY(dot_impl(p, n, dir, nullptr, dsc + 2));
        double sum = 0.0;
        DRV_CU(cudaMemcpyAsync(&sum, dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, stream), "read sum");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        gamma = sum / (double)n;
        if (!(gamma > 0.0)) gamma = 1.0;
    }
    std::vector<double> rho(m);
    int head = 0, count = 0;
    bool have_step = false;
    for (int k = 0; k < o->gn_iters; ++k) {
        DRV_TRY(gradient_impl(p, R, T, u, g, dsc, dsc + 1));
        DRV_TRY(dot_impl(p, n, g, g, dsc + 2));
        if (have_step) {  // y = g - g_prev, s.y
            DRV_CU(launch(k_axpy, gv, blk, 0, stream, n, -1.0f, (const float*)g, (const float*)gp, yt), "k_axpy");
            DRV_TRY(dot_impl(p, n, sl, yt, lb + 3 * m));
        }
        double h[3], sy = 0.0;
        DRV_CU(cudaMemcpyAsync(h, dsc, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream), "read J");
        if (have_step) DRV_CU(cudaMemcpyAsync(&sy, lb + 3 * m, sizeof(double), cudaMemcpyDeviceToHost, stream), "read sy");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        if (have_step && sy > 0.0) {  // keep the pair, dropping the oldest when full
            const int slot = (count == m) ? head : (head + count) % m;
            DRV_CU(cudaMemcpyAsync(Sr + (size_t)slot * n, sl, n * sizeof(float), cudaMemcpyDeviceToDevice, stream),
                   "store s");
            DRV_CU(cudaMemcpyAsync(Yr + (size_t)slot * n, yt, n * sizeof(float), cudaMemcpyDeviceToDevice, stream),
                   "store y");
            rho[slot] = 1.0 / sy;
            if (count == m) head = (head + 1) % m;
            else ++count;
        }
        const double J0 = h[0] + d.alpha * h[1], gg = h[2];
        if (gg == 0.0) break;
        // two-loop recursion: dir = -H_k g
        DRV_CU(cudaMemcpyAsync(dir, g, n * sizeof(float), cudaMemcpyDeviceToDevice, stream), "copy g");
        for (int i = count - 1; i >= 0; --i) {
            const int sl_i = (head + i) % m;
            DRV_TRY(dot_impl(p, n, Sr + (size_t)sl_i * n, dir, lb + i));
            DRV_CU(launch(k_lbfgs_q, gv, blk, 0, stream, n, rho[sl_i], (const double*)(lb + i),
                          (const float*)(Yr + (size_t)sl_i * n), dir, lb + m + i),
                   "k_lbfgs_q");
        }
        DRV_TRY(h0_impl(p, gamma, dir, dir));
        for (int i = 0; i < count; ++i) {
            const int sl_i = (head + i) % m;
            DRV_TRY(dot_impl(p, n, Yr + (size_t)sl_i * n, dir, lb + 2 * m + i));
            DRV_CU(launch(k_lbfgs_r, gv, blk, 0, stream, n, rho[sl_i], (const double*)(lb + 2 * m + i),
                          (const double*)(lb + m + i), (const float*)(Sr + (size_t)sl_i * n), dir),
                   "k_lbfgs_r");
        }
        DRV_CU(launch(k_scale, gv, blk, 0, stream, n, -1.0f, (const float*)dir, dir), "k_scale");
        DRV_TRY(dot_impl(p, n, g, dir, dsc + 2));
        DRV_CU(cudaMemcpyAsync(h + 2, dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, stream), "read gs");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        double gs = h[2];
        if (!(gs < 0.0)) {  // not a descent direction: steepest descent
            DRV_CU(launch(k_scale, gv, blk, 0, stream, n, -1.0f, (const float*)g, dir), "k_scale");
            gs = -gg;
        }
        bool accepted = false;
        DRV_TRY(armijo(p, d, o, R, T, u, dir, ut, J0, gs, dsc, r, accepted));
        if (!accepted) {
            r.ls_fail++;
            r.status = NGF_ELINESEARCH;
            break;
        }
        // last step s = ut - u, previous gradient, accept
        DRV_CU(launch(k_axpy, gv, blk, 0, stream, n, -1.0f, (const float*)ut, (const float*)u, sl), "k_axpy");
        DRV_CU(cudaMemcpyAsync(gp, g, n * sizeof(float), cudaMemcpyDeviceToDevice, stream), "copy g");
        std::swap(u, ut);
        have_step = true;
        r.gn_done++;
    }
    return NGF_OK;
}

extern "C" ngf_status register_multilevel(const ngf_level_desc* finest, const ngf_options* o, const float* R,
                                          const float* T, float* u_out, ngf_report* rep, void* cuda_stream) {
    const auto t_start = std::chrono::steady_clock::now();
    std::string why;
    const ngf_status vs = validate_desc(finest, why);
    if (vs != NGF_OK) return set_error(nullptr, vs, why);
    if (!o || !R || !T || !u_out) return set_error(nullptr, NGF_EINVAL, "options, R, T and u_out must be non-NULL");
    if (o->levels < 1 || o->levels > 16) return set_error(nullptr, NGF_EINVAL, "levels must be in [1, 16]");
    if (o->gn_iters < 0 || o->pcg_iters < 0 || o->ls_max < 1)
        return set_error(nullptr, NGF_EINVAL, "gn_iters, pcg_iters >= 0 and ls_max >= 1 required");
    if (o->zc < 0 || o->diag_every < 0) return set_error(nullptr, NGF_EINVAL, "zc and diag_every must be >= 0");
    if (o->gn_iters_finest < 0 || !(o->j_target >= 0.0))
        return set_error(nullptr, NGF_EINVAL, "gn_iters_finest and j_target must be >= 0");
    if (o->method != NGF_METHOD_GN && o->method != NGF_METHOD_LBFGS)
        return set_error(nullptr, NGF_EINVAL, "method must be NGF_METHOD_GN or NGF_METHOD_LBFGS");
    const bool lbfgs = o->method == NGF_METHOD_LBFGS;
    if (lbfgs && (o->lbfgs_memory < 1 || o->lbfgs_memory > 64))
        return set_error(nullptr, NGF_EINVAL, "lbfgs_memory must be in [1, 64]");
    if (o->u_init && (o->start_level < 0 || o->start_level >= o->levels))
        return set_error(nullptr, NGF_EINVAL, "start_level out of range");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    ngf_report r{};
    auto alloc = [stream](DevBuf& b, size_t bytes) {
        b.stream = stream;
        return dev_alloc(&b.ptr, bytes, stream);
    };

    const int L = o->levels;
    std::vector<ngf_level_desc> lv(L);
    for (int l = 0; l < L; ++l) lv[l] = level_at(*finest, l);
    for (int l = 0; l < L; ++l)
        for (int a = 0; a < 3; ++a)
            if (lv[l].n[a] > 4096) return set_error(nullptr, NGF_EBOUNDS, "more than 4096 nodes on an axis");
    const long long M0 = (long long)lv[0].m[0] * lv[0].m[1] * lv[0].m[2];
    const long long N0 = (long long)lv[0].n[0] * lv[0].n[1] * lv[0].n[2];

    // images of every level (level 0 may be the caller's device arrays)
    std::vector<DevBuf> imgs(2 * L);
    std::vector<const float*> Rl(L), Tl(L);
    const bool R_dev = is_device_ptr(R), T_dev = is_device_ptr(T), U_dev = is_device_ptr(u_out);
    for (int l = 0; l < L; ++l) {
        const long long M = (long long)lv[l].m[0] * lv[l].m[1] * lv[l].m[2];
        if (l == 0 && R_dev) {
            Rl[0] = R;
        } else {
            DRV_CU(alloc(imgs[2 * l], M * sizeof(float)), "allocate R level");
            Rl[l] = imgs[2 * l].as<float>();
        }
        if (l == 0 && T_dev) {
            Tl[0] = T;
        } else {
            DRV_CU(alloc(imgs[2 * l + 1], M * sizeof(float)), "allocate T level");
            Tl[l] = imgs[2 * l + 1].as<float>();
        }
    }
    if (!R_dev) DRV_CU(cudaMemcpyAsync((void*)Rl[0], R, M0 * sizeof(float), cudaMemcpyHostToDevice, stream), "copy R");
    if (!T_dev) DRV_CU(cudaMemcpyAsync((void*)Tl[0], T, M0 * sizeof(float), cudaMemcpyHostToDevice, stream), "copy T");

    // work vectors sized for the finest level
    const long long n3 = 3 * N0;
    DevBuf bu, but, bg, bdiag, bx, br, bz, bd, bq, bsc, bpart, bcnt, btab;
    DRV_CU(alloc(bu, n3 * sizeof(float)), "allocate u");
    DRV_CU(alloc(but, n3 * sizeof(float)), "allocate ut");
    DRV_CU(alloc(bg, n3 * sizeof(float)), "allocate g");
    DRV_CU(alloc(bdiag, n3 * sizeof(float)), "allocate diag");
    DRV_CU(alloc(bx, n3 * sizeof(float)), "allocate x");
    DRV_CU(alloc(br, n3 * sizeof(float)), "allocate r");
    DRV_CU(alloc(bz, n3 * sizeof(float)), "allocate z");
    DRV_CU(alloc(bd, n3 * sizeof(float)), "allocate d");
    DRV_CU(alloc(bq, n3 * sizeof(float)), "allocate q");
    DRV_CU(alloc(bsc, 32 * sizeof(double)), "allocate scalars");
    DRV_CU(cudaMemsetAsync(bsc.ptr, 0, 32 * sizeof(double), stream), "memset(scalars)");
    DRV_CU(alloc(bpart, 4096 * sizeof(double)), "allocate partials");
    DRV_CU(alloc(bcnt, 4 * sizeof(unsigned int)), "allocate counter");
    DRV_CU(cudaMemsetAsync(bcnt.ptr, 0, 4 * sizeof(unsigned int), stream), "memset(counter)");
    DRV_CU(alloc(btab, 3 * 4096 * (sizeof(int) + sizeof(float))), "allocate prolongation tables");
    // L-BFGS: previous gradient, last step, candidate y, the (s, y) ring and
    // float64 scalars of the two-loop recursion
    DevBuf bgp, bsl, byt, bS, bY, blb;
    const int mem = lbfgs ? o->lbfgs_memory : 0;
    if (lbfgs) {
        DRV_CU(alloc(bgp, n3 * sizeof(float)), "allocate g_prev");
        DRV_CU(alloc(bsl, n3 * sizeof(float)), "allocate step");
        DRV_CU(alloc(byt, n3 * sizeof(float)), "allocate y");
        DRV_CU(alloc(bS, (size_t)mem * n3 * sizeof(float)), "allocate s ring");
        DRV_CU(alloc(bY, (size_t)mem * n3 * sizeof(float)), "allocate y ring");
        DRV_CU(alloc(blb, (size_t)(3 * mem + 8) * sizeof(double)), "allocate two-loop scalars");
    }
    double* dsc = bsc.as<double>();  // 0 D, 1 S, 2 dot, 3 non-finite count; 8.. PCG state
    double* pcg_sc = dsc + 8;

    auto count_bad = [&](const float* a, long long n, double& bad) -> ngf_status {
        DRV_CU(launch(k_nonfinite, dim3(grid_for(n, 2048)), dim3(NT), 0, stream, n, a, bpart.as<double>(),
                      bcnt.as<unsigned int>(), dsc + 3),
               "k_nonfinite");
        DRV_CU(cudaMemcpyAsync(&bad, dsc + 3, sizeof(double), cudaMemcpyDeviceToHost, stream), "read check");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        return NGF_OK;
    };
    double bad = 0.0;
    DRV_TRY(count_bad(Rl[0], M0, bad));
    if (bad != 0.0) return set_error(nullptr, NGF_ENONFINITE, "R has NaN/Inf");
    DRV_TRY(count_bad(Tl[0], M0, bad));
    if (bad != 0.0) return set_error(nullptr, NGF_ENONFINITE, "T has NaN/Inf");

    // image pyramid
    for (int l = 1; l < L; ++l) {
        const long long Mc = (long long)lv[l].m[0] * lv[l].m[1] * lv[l].m[2];
        DRV_CU(launch(k_restrict, dim3(grid_for(Mc, 4096)), dim3(NT), 0, stream, lv[l - 1].m[0], lv[l - 1].m[1],
                      lv[l - 1].m[2], Rl[l - 1], (float*)Rl[l]),
               "k_restrict");
        DRV_CU(launch(k_restrict, dim3(grid_for(Mc, 4096)), dim3(NT), 0, stream, lv[l - 1].m[0], lv[l - 1].m[1],
                      lv[l - 1].m[2], Tl[l - 1], (float*)Tl[l]),
               "k_restrict");
    }

    const int start = o->u_init ? o->start_level : L - 1;
    float* u = bu.as<float>();
    float* ut = but.as<float>();
    {
        const long long Ns = (long long)lv[start].n[0] * lv[start].n[1] * lv[start].n[2];
        if (o->u_init) {
            DRV_CU(cudaMemcpyAsync(u, o->u_init, 3 * Ns * sizeof(float), cudaMemcpyDefault, stream), "copy u_init");
            DRV_TRY(count_bad(u, 3 * Ns, bad));
            if (bad != 0.0) return set_error(nullptr, NGF_ENONFINITE, "u_init has NaN/Inf");
        } else {
            DRV_CU(cudaMemsetAsync(u, 0, 3 * Ns * sizeof(float), stream), "zero u");
        }
    }

    for (int l = start; l >= 0; --l) {
        const ngf_level_desc& d = lv[l];
        const long long N = (long long)d.n[0] * d.n[1] * d.n[2];
        const long long M = (long long)d.m[0] * d.m[1] * d.m[2];
        if (l != start) {  // prolongate u from level l+1
            const ngf_level_desc& c = lv[l + 1];
            std::vector<int> tf;
            std::vector<float> tw;
            for (int a = 0; a < 3; ++a)
                for (int i = 0; i < d.n[a]; ++i) {
                    const double cc = d.n[a] > 1 ? (double)i * (double)(c.n[a] - 1) / (double)(d.n[a] - 1) : 0.0;
                    double fl = std::floor(cc);
                    if (fl > c.n[a] - 2) fl = c.n[a] - 2;
                    if (fl < 0) fl = 0;  // a single node plane (planar level): weight 0
                    tf.push_back((int)fl);
                    tw.push_back((float)(cc - fl));
                }
            int* dtf = btab.as<int>();
            float* dtw = reinterpret_cast<float*>(dtf + 3 * 4096);
            DRV_CU(cudaMemcpyAsync(dtf, tf.data(), tf.size() * sizeof(int), cudaMemcpyHostToDevice, stream), "tables");
            DRV_CU(cudaMemcpyAsync(dtw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, stream), "tables");
            const long long Nc = (long long)c.n[0] * c.n[1] * c.n[2];
            DRV_CU(launch(k_prolong, dim3(grid_for(3 * N, 4096)), dim3(NT), 0, stream, d.n[0], d.n[1], d.n[2],
                          c.n[0], c.n[1], Nc, (const int*)dtf, (const float*)dtw, (const float*)u, ut),
                   "k_prolong");
            std::swap(u, ut);
            // the host tables must outlive the asynchronous copies
            DRV_CU(cudaStreamSynchronize(stream), "sync");
        }
        PlanGuard pg;
        DRV_TRY(plan_create(&pg.p, &d, stream, o->zc));
        Plan* p = &pg.p->impl;
        ngf_pcg_state st;
        st.x = bx.as<float>();
        st.r = br.as<float>();
        st.z = bz.as<float>();
        st.d = bd.as<float>();
        st.q = bq.as<float>();
        st.diag = bdiag.as<float>();
        st.dev_scalars = pcg_sc;
        st.rtol = o->pcg_rtol;
        float* g = bg.as<float>();
        const long long n = 3 * N;
        if (lbfgs) {
            DRV_TRY(lbfgs_level(p, d, o, Rl[l], Tl[l], u, ut, g, bdiag.as<float>(), bgp.as<float>(), bsl.as<float>(),
                                byt.as<float>(), bS.as<float>(), bY.as<float>(), blb.as<double>(), dsc, r));
        }
        const int iters = (l == 0 && o->gn_iters_finest > 0) ? o->gn_iters_finest : o->gn_iters;
        for (int k = 0; k < (lbfgs ? 0 : iters); ++k) {
            DRV_TRY(gradient_impl(p, Rl[l], Tl[l], u, g, dsc, dsc + 1));
            DRV_TRY(dot_impl(p, n, g, g, dsc + 2));
            double h[3];
            DRV_CU(cudaMemcpyAsync(h, dsc, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream), "read J");
            DRV_CU(cudaStreamSynchronize(stream), "sync");
            const double J0 = h[0] + d.alpha * h[1], gg = h[2];
            if (gg == 0.0) break;  // stationary point
            if (l == 0 && o->j_target > 0.0 && J0 <= o->j_target) break;  // target objective reached
            // Jacobi diagonal at the level's first step, then every diag_every steps
            if (o->diag_every > 0 ? k % o->diag_every == 0 : k == 0)
                DRV_TRY(diagonal_impl(p, Rl[l], Tl[l], u, bdiag.as<float>()));
            DRV_CU(launch(k_scale, dim3(p->node_blocks), dim3(NT), 0, stream, n, -1.0f, (const float*)g, st.r),
                   "k_scale");
            DRV_TRY(pcg_init(pg.p, &st, st.r));
            DRV_TRY(pcg_solve(pg.p, &st, Rl[l], Tl[l], u, o->pcg_iters, o->use_graph));
            r.hessvec_voxels += (int64_t)o->pcg_iters * M;
            double ps[NGF_PCG_NSCALARS];
            DRV_TRY(dot_impl(p, n, g, st.x, dsc + 2));
            DRV_CU(cudaMemcpyAsync(ps, pcg_sc, sizeof(ps), cudaMemcpyDeviceToHost, stream), "read PCG");
            DRV_CU(cudaMemcpyAsync(h + 2, dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, stream), "read gs");
            DRV_CU(cudaStreamSynchronize(stream), "sync");
            r.pcg_total += (int32_t)ps[PS_ITERS];
            double gs = h[2];
            float* s = st.x;
            if (!(gs < 0.0)) {  // not a descent direction: steepest descent
                DRV_CU(launch(k_scale, dim3(p->node_blocks), dim3(NT), 0, stream, n, -1.0f, (const float*)g, s),
                       "k_scale");
                gs = -gg;
            }
            bool accepted = false;
            DRV_TRY(armijo(p, d, o, Rl[l], Tl[l], u, s, ut, J0, gs, dsc, r, accepted));
            if (!accepted) {
                r.ls_fail++;
                r.status = NGF_ELINESEARCH;
                break;
            }
            std::swap(u, ut);
            r.gn_done++;
        }
        DRV_TRY(objective_impl(p, Rl[l], Tl[l], u, dsc, dsc + 1));
        double h[2];
        DRV_CU(cudaMemcpyAsync(h, dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream), "read J");
        DRV_CU(cudaStreamSynchronize(stream), "sync");
        r.D = h[0];
        r.S = h[1];
        r.J = h[0] + d.alpha * h[1];
    }
    DRV_CU(cudaMemcpyAsync(u_out, u, n3 * sizeof(float), U_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           stream),
           "copy u_out");
    DRV_CU(cudaStreamSynchronize(stream), "sync");
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (rep) *rep = r;
    return NGF_OK;
}
