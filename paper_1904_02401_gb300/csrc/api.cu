// Host side of libnmg: hierarchy set-up, the multigrid V-cycle driver, the
// FP64 flexible GMRES loop and the C ABI declared in include/nmg.h.
//
// Method (Section 4.3): (I) GMRES outer iteration, here flexible GMRES(m) with
// right preconditioning because the preconditioner may run in reduced
// precision; (II) one geometric multigrid V(nu1, nu2)-cycle per iteration on
// nested uniform meshes, each level with its own matrix; (III) the additive
// Vanka smoother of Eq. (vanka) with exactly inverted patch matrices.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "nmg_internal.cuh"

namespace nmg {

thread_local std::string g_last_error = "no error";
thread_local int64_t g_launches = 0;

static nmg_status fail(nmg_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define NMG_CK(call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? NMG_ERR_OOM : NMG_ERR_CUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

static Geom make_geom(int dim, const int* cells) {
    Geom g{};
    g.dim = dim;
    g.nc = dim + 1;
    g.nodes = 1;
    g.patches = 1;
    for (int k = 0; k < 3; ++k) {
        if (k < dim) {
            g.cells[k] = cells[k];
            g.nn[k] = cells[k] + 1;
            g.pc[k] = cells[k] / 2;
        } else {
            g.cells[k] = 0;
            g.nn[k] = 1;
            g.pc[k] = 1;
        }
        g.nodes *= g.nn[k];
        g.patches *= g.pc[k];
    }
    g.ld = (g.nodes + 31) / 32 * 32;
    g.nst = dim == 2 ? 9 : 27;
    g.np = g.nst * g.nc;
    return g;
}

static int64_t pad16(int64_t elems, size_t esize) {
    const int64_t per = 16 / (int64_t)esize;
    return (elems + per - 1) / per * per;
}

static nmg_status dalloc(Hierarchy* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (h->desc.mem_budget_bytes && h->bytes + bytes > h->desc.mem_budget_bytes)
        return fail(NMG_ERR_OOM, "memory budget exceeded");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(NMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    h->bytes += bytes;
    return NMG_OK;
}

#define NMG_TRY(expr)                  \
    do {                               \
        nmg_status st_ = (expr);       \
        if (st_ != NMG_OK) return st_; \
    } while (0)

static size_t prec_size(int prec) { return prec == NMG_PREC_FP64 ? sizeof(double) : sizeof(float); }
static size_t store_size(int prec) {
    return prec == NMG_PREC_FP64 ? sizeof(double) : prec == NMG_PREC_FP32 ? sizeof(float) : sizeof(__nv_bfloat16);
}

// Legacy default stream: the hierarchy works on a private stream and orders
// itself after earlier default-stream work at every call.
static void enter(Hierarchy* h) {
    if (h->desc.stream == nullptr) cudaStreamSynchronize(0);
}

static nmg_status check_flags(Hierarchy* h) {
    int f[FLAG_COUNT];
    NMG_CK(cudaMemcpyAsync(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
    NMG_CK(cudaStreamSynchronize(h->stream));
    NMG_CK(cudaMemsetAsync(h->flags, 0, sizeof(f), h->stream));
    if (f[FLAG_BAD_PATTERN]) return fail(NMG_ERR_INVALID, "matrix block outside the Q1 stencil, duplicate block or bad row_ptr");
    if (f[FLAG_NONFINITE]) return fail(NMG_ERR_NONFINITE, "non-finite matrix value");
    if (f[FLAG_SINGULAR]) return fail(NMG_ERR_SINGULAR_PATCH, "zero pivot in a patch (or coarse) matrix");
    return NMG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------
template <typename T>
static void smooth_level(Hierarchy* h, int l, int prec, const T* b, T* x, int steps, bool x_zero,
                         T omega, bool average) {
    Level& L = h->lev[l];
    PrecData& P = L.p[prec];
    const Geom& g = L.g;
    cudaStream_t s = h->stream;
    if (steps == 0 && x_zero) {
        cudaMemsetAsync(x, 0, g.nodes * g.nc * sizeof(T), s);
        return;
    }
    const bool prof = h->prof && l == h->L - 1;
    if (prof) {
        const double sv = (double)sizeof(T);
        const double si = prec == NMG_PREC_FP64 ? 8.0 : prec == NMG_PREC_FP32 ? 4.0 : 2.0;
        h->prof_bytes = (double)g.patches * g.np * g.np * si + (double)g.nodes * g.nc * sv +
                        (double)g.patches * g.np * sv;
    }
    for (int st = 0; st < steps; ++st) {
        const T* d;
        if (st == 0 && x_zero) {
            d = b;
        } else {
            launch_spmv<T>(g, (const T*)P.A, x, b, (T*)P.r, true, s);
            d = (const T*)P.r;
        }
        const bool rec = prof && h->prof_used < (int)h->prof_ev.size() / 2;
        if (rec) cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
        if (prec == NMG_PREC_FP64)
            launch_vanka_apply<double, double>(g, (const double*)P.inv, P.inv_stride, (const double*)d, (double*)P.corr, s);
        else if (prec == NMG_PREC_FP32)
            launch_vanka_apply<float, float>(g, (const float*)P.inv, P.inv_stride, (const float*)d, (float*)P.corr, s);
        else
            launch_vanka_apply<float, __nv_bfloat16>(g, (const __nv_bfloat16*)P.inv, P.inv_stride, (const float*)d,
                                                    (float*)P.corr, s);
        if (rec) {
            cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
            h->prof_used++;
        }
        launch_vanka_update<T>(g, (const T*)P.corr, x, st == 0 && x_zero, omega, average, s);
    }
}

// z = V-cycle(r) on the finest level; b_fine / x_fine are the finest-level
// right-hand side and result (the level's own buffers when null).
template <typename T>
static void run_vcycle(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting, const T* b_fine,
                       T* x_fine) {
    const int Lc = h->L;
    cudaStream_t s = h->stream;
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    const T om = (T)omega;
    auto bptr = [&](int l) -> T* { return (l == Lc - 1 && b_fine) ? const_cast<T*>(b_fine) : (T*)h->lev[l].p[prec].b; };
    auto xptr = [&](int l) -> T* { return (l == Lc - 1 && x_fine) ? x_fine : (T*)h->lev[l].p[prec].x; };
    for (int l = Lc - 1; l >= 1; --l) {
        Level& L = h->lev[l];
        smooth_level<T>(h, l, prec, bptr(l), xptr(l), nu1, true, om, avg);
        launch_spmv<T>(L.g, (const T*)L.p[prec].A, xptr(l), bptr(l), (T*)L.p[prec].r, true, s);
        launch_restrict<T>(L.g, h->lev[l - 1].g, (const T*)L.p[prec].r, bptr(l - 1), h->lev[l - 1].mask, s);
    }
    launch_coarse_gemv<T>(h->coarse_inv, h->n0, bptr(0), xptr(0), s);
    for (int l = 1; l < Lc; ++l) {
        Level& L = h->lev[l];
        launch_prolong_add<T>(L.g, h->lev[l - 1].g, xptr(l - 1), xptr(l), L.mask, s);
        smooth_level<T>(h, l, prec, bptr(l), xptr(l), nu2, false, om, avg);
    }
}

static void vcycle_dispatch(Hierarchy* h, int prec, const nmg_solve_opts& o, const void* b, void* x) {
    if (prec == NMG_PREC_FP64)
        run_vcycle<double>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, (const double*)b, (double*)x);
    else
        run_vcycle<float>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, (const float*)b, (float*)x);
}

// Replays (capturing first if needed) the V-cycle on the level buffers as a CUDA graph.
static nmg_status vcycle_graph(Hierarchy* h, int prec, const nmg_solve_opts& o) {
    const int key[4] = {o.nu1, o.nu2, o.weighting, 1};
    bool match = h->vgraph[prec] && std::memcmp(key, h->vgraph_key[prec], sizeof(key)) == 0 &&
                 h->vgraph_omega[prec] == o.omega;
    if (!match) {
        if (h->vgraph[prec]) cudaGraphExecDestroy(h->vgraph[prec]);
        h->vgraph[prec] = nullptr;
        cudaGraph_t graph;
        NMG_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const bool prof = h->prof;
        h->prof = false;   // no event nodes inside the graph
        const int64_t before = g_launches;
        vcycle_dispatch(h, prec, o, nullptr, nullptr);
        h->vgraph_nodes[prec] = g_launches - before;
        g_launches = before;
        h->prof = prof;
        NMG_CK(cudaStreamEndCapture(h->stream, &graph));
        cudaError_t e = cudaGraphInstantiate(&h->vgraph[prec], graph, 0);
        cudaGraphDestroy(graph);
        NMG_CK(e);
        std::memcpy(h->vgraph_key[prec], key, sizeof(key));
        h->vgraph_omega[prec] = o.omega;
    }
    NMG_CK(cudaGraphLaunch(h->vgraph[prec], h->stream));
    g_launches += h->vgraph_nodes[prec];
    return NMG_OK;
}

static nmg_status check_ready(Hierarchy* h, int prec) {
    if (prec < 0 || prec > 2 || !(h->prec_mask & (1 << prec)))
        return fail(NMG_ERR_INVALID, "precision not prepared for this hierarchy");
    for (int l = 0; l < h->L; ++l)
        if (!h->lev[l].ready) return fail(NMG_ERR_INVALID, "level matrix " + std::to_string(l) + " not set");
    return NMG_OK;
}

static nmg_status validate_opts(const nmg_solve_opts* o) {
    if (!o) return fail(NMG_ERR_INVALID, "opts is NULL");
    if (!(o->rtol >= 0.0) || o->restart < 1 || o->restart > kMaxRestart || o->maxit < 0 || o->nu1 < 0 ||
        o->nu2 < 0 || o->nu1 > 64 || o->nu2 > 64 || !std::isfinite(o->omega) ||
        (o->weighting != NMG_WEIGHT_AVERAGE && o->weighting != NMG_WEIGHT_SUM))
        return fail(NMG_ERR_INVALID, "invalid solve options");
    return NMG_OK;
}

// z_j = M^{-1} v_j for FP64 vectors v, z on the finest level.
static nmg_status precondition(Hierarchy* h, const nmg_solve_opts& o, const double* v, double* z) {
    Level& F = h->lev[h->L - 1];
    const int64_t n = F.g.nodes * F.g.nc;
    const int prec = o.precision;
    if (prec == NMG_PREC_FP64) {
        if (o.use_graph) {
            NMG_CK(cudaMemcpyAsync(F.p[prec].b, v, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
            NMG_TRY(vcycle_graph(h, prec, o));
            NMG_CK(cudaMemcpyAsync(z, F.p[prec].x, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        } else {
            run_vcycle<double>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, v, z);
        }
    } else {
        launch_convert<double, float>(v, (float*)F.p[prec].b, n, h->stream);
        if (o.use_graph) NMG_TRY(vcycle_graph(h, prec, o));
        else run_vcycle<float>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, nullptr, nullptr);
        launch_convert<float, double>((const float*)F.p[prec].x, z, n, h->stream);
    }
    return NMG_OK;
}

static nmg_status ensure_krylov(Hierarchy* h, int m) {
    if (h->m_alloc >= m) return NMG_OK;
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    if (h->V) { cudaFree(h->V); h->bytes -= (size_t)(h->m_alloc + 1) * n * sizeof(double); }
    if (h->Z) { cudaFree(h->Z); h->bytes -= (size_t)h->m_alloc * n * sizeof(double); }
    for (auto it = h->allocs.begin(); it != h->allocs.end();)
        it = (*it == (void*)h->V || *it == (void*)h->Z) ? h->allocs.erase(it) : it + 1;
    h->V = h->Z = nullptr;
    h->m_alloc = 0;
    NMG_TRY(dalloc(h, (void**)&h->V, (size_t)(m + 1) * n * sizeof(double)));
    NMG_TRY(dalloc(h, (void**)&h->Z, (size_t)m * n * sizeof(double)));
    h->m_alloc = m;
    return NMG_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static nmg_status solve_impl(Hierarchy* h, const double* b_user, double* x_user, const nmg_solve_opts& o,
                             nmg_solve_info* info) {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t launches0 = g_launches;
    NMG_TRY(check_ready(h, o.precision));
    NMG_TRY(ensure_krylov(h, o.restart));
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    const int m = o.restart;
    cudaStream_t s = h->stream;
    double* A64 = h->lev[h->L - 1].A64;
    const bool b_dev = is_device_ptr(b_user), x_dev = is_device_ptr(x_user);
    NMG_CK(cudaMemcpyAsync(h->b64, b_user, n * sizeof(double), b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NMG_CK(cudaMemsetAsync(h->scal, 0, 8 * sizeof(double), s));
    NMG_CK(cudaMemsetAsync(h->x64, 0, n * sizeof(double), s));
    launch_norm2(h->b64, n, h->partial, h->scal + S_BNORM, s);
    NMG_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    NMG_CK(cudaStreamSynchronize(s));
    const double bnorm = h->host_scal[S_BNORM];
    nmg_status st = NMG_OK;
    int its = 0, cycles = 0;
    double relres = 0.0;
    if (!std::isfinite(bnorm)) st = fail(NMG_ERR_NONFINITE, "non-finite right-hand side");
    while (st == NMG_OK && bnorm > 0.0) {
        // true residual r = b - A x and beta = ||r||
        launch_spmv<double>(g, A64, h->x64, h->b64, h->w64, true, s);
        launch_norm2(h->w64, n, h->partial, h->scal + S_BETA, s);
        launch_start_cycle(h->scal, m, s);
        launch_scale(h->w64, h->scal + S_INVH, false, h->V, n, s);
        NMG_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        NMG_CK(cudaStreamSynchronize(s));
        const double beta = h->host_scal[S_BETA];
        relres = beta / bnorm;
        if (!std::isfinite(beta)) { st = fail(NMG_ERR_NONFINITE, "non-finite residual"); break; }
        if (relres <= o.rtol) break;
        if (its >= o.maxit) { st = fail(NMG_ERR_NOT_CONVERGED, "maxit reached"); break; }
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = h->V + (int64_t)j * n;
            double* zj = h->Z + (int64_t)j * n;
            NMG_TRY(precondition(h, o, vj, zj));
            launch_spmv<double>(g, A64, zj, nullptr, h->w64, false, s);
            // classical Gram-Schmidt, two passes
            launch_multidot(h->V, n, j + 1, h->w64, n, h->partial, h->scal + S_HC, false, s);
            launch_gs_update(h->V, n, j + 1, h->scal + S_HC, h->w64, n, h->partial, nullptr, false, s);
            launch_multidot(h->V, n, j + 1, h->w64, n, h->partial, h->scal + S_Y, false, s);
            launch_gs_update(h->V, n, j + 1, h->scal + S_Y, h->w64, n, h->partial, h->scal + S_HC + j + 1, true, s);
            launch_arnoldi_finish(h->scal, j, m, s);
            launch_scale(h->w64, h->scal + S_INVH, false, h->V + (int64_t)(j + 1) * n, n, s);
            NMG_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
            NMG_CK(cudaStreamSynchronize(s));
            ++its;
            k = j + 1;
            if (h->host_scal[S_STATUS] != 0.0) { st = fail(NMG_ERR_NONFINITE, "non-finite value in the Arnoldi process"); break; }
            if (h->host_scal[S_EST] <= o.rtol || its >= o.maxit || h->host_scal[S_INVH] == 0.0) break;
        }
        if (st != NMG_OK) break;
        launch_solve_update(h->scal, k, m, h->Z, n, h->x64, n, s);
        ++cycles;
    }
    NMG_CK(cudaMemcpyAsync(x_user, h->x64, n * sizeof(double), x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    NMG_CK(cudaStreamSynchronize(s));
    NMG_CK(cudaGetLastError());
    if (info) {
        info->iterations = its;
        info->restarts = cycles > 0 ? cycles - 1 : 0;
        info->rel_residual = relres;
        info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->status = st;
        info->launches = g_launches - launches0;
    }
    return st;
}

}  // namespace nmg

using namespace nmg;

struct nmg_hierarchy : public nmg::Hierarchy {};

extern "C" {

const char* nmg_last_error(void) { return g_last_error.c_str(); }

nmg_status nmg_default_opts(nmg_solve_opts* o) {
    if (!o) return fail(NMG_ERR_INVALID, "opts is NULL");
    o->rtol = 1e-8;
    o->restart = 30;
    o->maxit = 1000;
    o->nu1 = 2;
    o->nu2 = 2;
    o->omega = 0.8;
    o->precision = NMG_PREC_FP32;
    o->weighting = NMG_WEIGHT_AVERAGE;
    o->use_graph = 1;
    return NMG_OK;
}

static void free_all(Hierarchy* h) {
    for (int p = 0; p < 3; ++p)
        if (h->vgraph[p]) cudaGraphExecDestroy(h->vgraph[p]);
    for (void* a : h->allocs) cudaFree(a);
    h->allocs.clear();
    if (h->host_scal) cudaFreeHost(h->host_scal);
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    if (h->desc.stream == nullptr && h->stream) cudaStreamDestroy(h->stream);
}

nmg_status nmg_create_hierarchy(const nmg_mesh_desc* d, nmg_hierarchy** out) {
    if (!d || !out) return fail(NMG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return fail(NMG_ERR_INVALID, "dim must be 2 or 3");
    if (d->ncomp != d->dim + 1) return fail(NMG_ERR_INVALID, "ncomp must be dim + 1");
    if (d->patch_cells != 2) return fail(NMG_ERR_INVALID, "only patch_cells = 2 is supported");
    if (d->levels < 1 || d->levels > kMaxLevels) return fail(NMG_ERR_INVALID, "levels out of range");
    if (!d->dirichlet_mask) return fail(NMG_ERR_INVALID, "dirichlet_mask is NULL");
    const int L = d->levels;
    int cells[kMaxLevels][3];
    for (int k = 0; k < d->dim; ++k) {
        const int f = 1 << (L - 1);
        if (d->n[k] < 1 || d->n[k] % f) return fail(NMG_ERR_INVALID, "cells not divisible by 2^(levels-1)");
        for (int l = 0; l < L; ++l) cells[l][k] = d->n[k] >> (L - 1 - l);
    }
    for (int l = 1; l < L; ++l)
        for (int k = 0; k < d->dim; ++k)
            if (cells[l][k] % 2) return fail(NMG_ERR_INVALID, "levels above the coarsest need even cell counts");
    auto* h = new nmg_hierarchy();
    h->desc = *d;
    h->dim = d->dim;
    h->nc = d->ncomp;
    h->L = L;
    h->prec_mask = d->precisions ? (d->precisions & 7) : 7;
    auto cleanup = [&](nmg_status st) { free_all(h); delete h; return st; };
    if (d->stream) h->stream = (cudaStream_t)d->stream;
    else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(NMG_ERR_CUDA, "stream creation failed"));
    for (int l = 0; l < L; ++l) h->lev[l].g = make_geom(d->dim, cells[l]);
    const Geom& c0 = h->lev[0].g;
    h->n0 = c0.nodes * c0.nc;
    if (h->n0 > 2048) return cleanup(fail(NMG_ERR_INVALID, "coarsest level too large for the dense solve (> 2048 unknowns)"));
    nmg_status st;
    // Dirichlet masks: finest from the caller, coarser by injection (node I <- fine node 2I)
    std::vector<std::vector<uint8_t>> masks(L);
    {
        const Geom& gf = h->lev[L - 1].g;
        masks[L - 1].assign(d->dirichlet_mask, d->dirichlet_mask + gf.nodes * gf.nc);
        for (int l = L - 2; l >= 0; --l) {
            const Geom& gc = h->lev[l].g;
            const Geom& gF = h->lev[l + 1].g;
            masks[l].resize(gc.nodes * gc.nc);
            for (int64_t I = 0; I < gc.nodes; ++I) {
                const int64_t X = I % gc.nn[0], Y = (I / gc.nn[0]) % gc.nn[1], Z = I / ((int64_t)gc.nn[0] * gc.nn[1]);
                const int64_t fi = 2 * X + gF.nn[0] * (2 * Y + (int64_t)gF.nn[1] * 2 * Z);
                for (int c = 0; c < gc.nc; ++c) masks[l][I * gc.nc + c] = masks[l + 1][fi * gc.nc + c];
            }
        }
    }
    const bool low = (h->prec_mask & ((1 << NMG_PREC_FP32) | (1 << NMG_PREC_BF16))) != 0;
    for (int l = 0; l < L; ++l) {
        Level& Lv = h->lev[l];
        const Geom& g = Lv.g;
        const int64_t nvec = g.nodes * g.nc;
        const size_t mat = (size_t)g.nst * g.nc * g.nc * g.ld;
        if ((st = dalloc(h, (void**)&Lv.A64, mat * sizeof(double))) != NMG_OK) return cleanup(st);
        if ((st = dalloc(h, (void**)&Lv.mask, nvec)) != NMG_OK) return cleanup(st);
        if (cudaMemcpy(Lv.mask, masks[l].data(), nvec, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(NMG_ERR_CUDA, "mask upload failed"));
        float* A32 = nullptr;
        if (low && (st = dalloc(h, (void**)&A32, mat * sizeof(float))) != NMG_OK) return cleanup(st);
        void* fvec[4] = {nullptr, nullptr, nullptr, nullptr};   // float work vectors shared by FP32 / BF16
        if (low) {
            for (int q = 0; q < 3; ++q)
                if ((st = dalloc(h, &fvec[q], nvec * sizeof(float))) != NMG_OK) return cleanup(st);
            if (l > 0 && (st = dalloc(h, &fvec[3], (size_t)g.patches * g.np * sizeof(float))) != NMG_OK) return cleanup(st);
        }
        for (int p = 0; p < 3; ++p) {
            if (!(h->prec_mask & (1 << p))) continue;
            PrecData& P = Lv.p[p];
            if (p == NMG_PREC_FP64) {
                P.A = Lv.A64;
                for (void** q : {&P.b, &P.x, &P.r})
                    if ((st = dalloc(h, q, nvec * sizeof(double))) != NMG_OK) return cleanup(st);
                if (l > 0 && (st = dalloc(h, &P.corr, (size_t)g.patches * g.np * sizeof(double))) != NMG_OK) return cleanup(st);
            } else {
                P.A = A32;
                P.b = fvec[0]; P.x = fvec[1]; P.r = fvec[2]; P.corr = fvec[3];
            }
            if (l > 0) {
                P.inv_stride = pad16((int64_t)g.np * g.np, store_size(p));
                if ((st = dalloc(h, &P.inv, (size_t)g.patches * P.inv_stride * store_size(p))) != NMG_OK) return cleanup(st);
            }
        }
    }
    const Geom& gf = h->lev[L - 1].g;
    const int64_t n = gf.nodes * gf.nc;
    if ((st = dalloc(h, (void**)&h->coarse_inv, (size_t)h->n0 * h->n0 * sizeof(double))) != NMG_OK) return cleanup(st);
    for (double** q : {&h->b64, &h->x64, &h->w64})
        if ((st = dalloc(h, (void**)q, n * sizeof(double))) != NMG_OK) return cleanup(st);
    if ((st = dalloc(h, (void**)&h->partial, (size_t)(kMaxRestart + 2) * kDotBlocks * sizeof(double))) != NMG_OK) return cleanup(st);
    if ((st = dalloc(h, (void**)&h->scal, S_COUNT * sizeof(double))) != NMG_OK) return cleanup(st);
    if ((st = dalloc(h, (void**)&h->flags, FLAG_COUNT * sizeof(int))) != NMG_OK) return cleanup(st);
    if (cudaMemset(h->flags, 0, FLAG_COUNT * sizeof(int)) != cudaSuccess) return cleanup(fail(NMG_ERR_CUDA, "memset"));
    if (cudaMallocHost((void**)&h->host_scal, 16 * sizeof(double)) != cudaSuccess)
        return cleanup(fail(NMG_ERR_OOM, "pinned host allocation failed"));
    *out = h;
    return NMG_OK;
}

nmg_status nmg_destroy_hierarchy(nmg_hierarchy* h) {
    if (!h) return NMG_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return NMG_OK;
}

nmg_status nmg_hierarchy_bytes(nmg_hierarchy* h, size_t* bytes) {
    if (!h || !bytes) return fail(NMG_ERR_INVALID, "NULL argument");
    *bytes = h->bytes;
    return NMG_OK;
}

nmg_status nmg_set_jacobian(nmg_hierarchy* h, int level, int64_t nrows_blk, int64_t nnzb, const int64_t* row_ptr,
                            const int32_t* col_idx, const double* vals, int ptr_location) {
    if (!h || !row_ptr || (nnzb > 0 && (!col_idx || !vals))) return fail(NMG_ERR_INVALID, "NULL argument");
    if (level < 0 || level >= h->L) return fail(NMG_ERR_INVALID, "level out of range");
    Level& Lv = h->lev[level];
    const Geom& g = Lv.g;
    if (nrows_blk != g.nodes) return fail(NMG_ERR_INVALID, "nrows_blk does not match the level's node count");
    if (nnzb < 0 || nnzb > g.nodes * g.nst) return fail(NMG_ERR_INVALID, "nnzb out of range");
    if (ptr_location != 0 && ptr_location != 1) return fail(NMG_ERR_INVALID, "ptr_location must be 0 or 1");
    enter(h);
    cudaStream_t s = h->stream;
    const int nb = g.nc * g.nc;
    const int64_t* d_rp = row_ptr;
    const int32_t* d_ci = col_idx;
    const double* d_v = vals;
    void* tmp[3] = {nullptr, nullptr, nullptr};
    auto release = [&]() { for (void* t : tmp) if (t) cudaFree(t); };
    if (ptr_location == 0) {
        if (row_ptr[0] != 0 || row_ptr[g.nodes] != nnzb) return fail(NMG_ERR_INVALID, "row_ptr must run from 0 to nnzb");
        if (cudaMalloc(&tmp[0], (g.nodes + 1) * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&tmp[1], std::max<int64_t>(nnzb, 1) * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&tmp[2], std::max<int64_t>(nnzb, 1) * nb * sizeof(double)) != cudaSuccess) {
            release();
            return fail(NMG_ERR_OOM, "staging allocation failed");
        }
        cudaMemcpyAsync(tmp[0], row_ptr, (g.nodes + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (nnzb) {
            cudaMemcpyAsync(tmp[1], col_idx, nnzb * sizeof(int32_t), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(tmp[2], vals, nnzb * nb * sizeof(double), cudaMemcpyHostToDevice, s);
        }
        d_rp = (const int64_t*)tmp[0];
        d_ci = (const int32_t*)tmp[1];
        d_v = (const double*)tmp[2];
    }
    const size_t mat = (size_t)g.nst * nb * g.ld;
    cudaMemsetAsync(Lv.A64, 0, mat * sizeof(double), s);
    launch_bsr_to_stencil(g, d_rp, d_ci, d_v, nnzb, Lv.A64, h->flags, s);
    nmg_status st = check_flags(h);
    release();
    if (st != NMG_OK) return st;
    const bool low = (h->prec_mask & 6) != 0;
    if (low) {
        void* A32 = Lv.p[(h->prec_mask & 2) ? NMG_PREC_FP32 : NMG_PREC_BF16].A;
        launch_convert_f64_f32(Lv.A64, (float*)A32, (int64_t)mat, s);
    }
    if (level > 0) {
        PrecData* P = Lv.p;
        const bool p64 = h->prec_mask & 1, p32 = h->prec_mask & 2, pbf = h->prec_mask & 4;
        NMG_CK(launch_patch_invert(g, Lv.A64, p64 ? (double*)P[0].inv : nullptr, P[0].inv_stride,
                                   p32 ? (float*)P[1].inv : nullptr, P[1].inv_stride,
                                   pbf ? (__nv_bfloat16*)P[2].inv : nullptr, P[2].inv_stride, h->flags, s));
    } else {
        const int64_t n0 = h->n0;
        int* perm = nullptr;
        if (cudaMalloc(&perm, n0 * sizeof(int)) != cudaSuccess) return fail(NMG_ERR_OOM, "perm allocation failed");
        cudaMemsetAsync(h->coarse_inv, 0, n0 * n0 * sizeof(double), s);
        launch_coarse_assemble(g, Lv.A64, h->coarse_inv, s);
        launch_dense_invert(h->coarse_inv, n0, perm, h->flags, s);
        cudaStreamSynchronize(s);
        cudaFree(perm);
    }
    NMG_CK(cudaGetLastError());
    NMG_TRY(check_flags(h));
    Lv.ready = true;
    for (int p = 0; p < 3; ++p)
        if (h->vgraph[p]) { cudaGraphExecDestroy(h->vgraph[p]); h->vgraph[p] = nullptr; }
    return NMG_OK;
}

nmg_status nmg_solve(nmg_hierarchy* h, const double* b, double* x, const nmg_solve_opts* opts, nmg_solve_info* info) {
    if (!h || !b || !x) return fail(NMG_ERR_INVALID, "NULL argument");
    NMG_TRY(validate_opts(opts));
    enter(h);
    nmg_status st = solve_impl(h, b, x, *opts, info);
    if (info) info->status = st;
    return st;
}

static nmg_status op_check(Hierarchy* h, int level, int prec, bool need_smooth) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (level < 0 || level >= h->L) return fail(NMG_ERR_INVALID, "level out of range");
    if (prec < 0 || prec > 2 || !(h->prec_mask & (1 << prec))) return fail(NMG_ERR_INVALID, "precision not prepared");
    if (!h->lev[level].ready) return fail(NMG_ERR_INVALID, "level matrix not set");
    if (need_smooth && level == 0) return fail(NMG_ERR_INVALID, "the coarsest level has no patches");
    return NMG_OK;
}

static nmg_status finish_op(Hierarchy* h) {
    NMG_CK(cudaGetLastError());
    NMG_CK(cudaStreamSynchronize(h->stream));
    return NMG_OK;
}

nmg_status nmg_matvec(nmg_hierarchy* h, int level, int prec, const void* x, void* y) {
    NMG_TRY(op_check(h, level, prec, false));
    enter(h);
    const Geom& g = h->lev[level].g;
    if (prec == NMG_PREC_FP64) launch_spmv<double>(g, h->lev[level].A64, (const double*)x, nullptr, (double*)y, false, h->stream);
    else launch_spmv<float>(g, (const float*)h->lev[level].p[prec].A, (const float*)x, nullptr, (float*)y, false, h->stream);
    return finish_op(h);
}

nmg_status nmg_residual(nmg_hierarchy* h, int level, int prec, const void* b, const void* x, void* r) {
    NMG_TRY(op_check(h, level, prec, false));
    enter(h);
    const Geom& g = h->lev[level].g;
    if (prec == NMG_PREC_FP64) launch_spmv<double>(g, h->lev[level].A64, (const double*)x, (const double*)b, (double*)r, true, h->stream);
    else launch_spmv<float>(g, (const float*)h->lev[level].p[prec].A, (const float*)x, (const float*)b, (float*)r, true, h->stream);
    return finish_op(h);
}

nmg_status nmg_smooth(nmg_hierarchy* h, int level, int prec, const void* b, void* x, int steps, int x_is_zero,
                      double omega, int weighting) {
    NMG_TRY(op_check(h, level, prec, true));
    if (steps < 0 || (weighting != NMG_WEIGHT_AVERAGE && weighting != NMG_WEIGHT_SUM))
        return fail(NMG_ERR_INVALID, "bad smoothing arguments");
    enter(h);
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    if (prec == NMG_PREC_FP64) smooth_level<double>(h, level, prec, (const double*)b, (double*)x, steps, x_is_zero != 0, omega, avg);
    else smooth_level<float>(h, level, prec, (const float*)b, (float*)x, steps, x_is_zero != 0, (float)omega, avg);
    return finish_op(h);
}

nmg_status nmg_restrict(nmg_hierarchy* h, int level, int prec, const void* rf, void* rc) {
    NMG_TRY(op_check(h, level, prec, true));
    enter(h);
    const Geom& f = h->lev[level].g;
    const Geom& c = h->lev[level - 1].g;
    if (prec == NMG_PREC_FP64) launch_restrict<double>(f, c, (const double*)rf, (double*)rc, h->lev[level - 1].mask, h->stream);
    else launch_restrict<float>(f, c, (const float*)rf, (float*)rc, h->lev[level - 1].mask, h->stream);
    return finish_op(h);
}

nmg_status nmg_prolongate_add(nmg_hierarchy* h, int level, int prec, const void* ec, void* xf) {
    NMG_TRY(op_check(h, level, prec, true));
    enter(h);
    const Geom& f = h->lev[level].g;
    const Geom& c = h->lev[level - 1].g;
    if (prec == NMG_PREC_FP64) launch_prolong_add<double>(f, c, (const double*)ec, (double*)xf, h->lev[level].mask, h->stream);
    else launch_prolong_add<float>(f, c, (const float*)ec, (float*)xf, h->lev[level].mask, h->stream);
    return finish_op(h);
}

nmg_status nmg_coarse_solve(nmg_hierarchy* h, int prec, const void* b, void* x) {
    NMG_TRY(op_check(h, 0, prec, false));
    enter(h);
    if (prec == NMG_PREC_FP64) launch_coarse_gemv<double>(h->coarse_inv, h->n0, (const double*)b, (double*)x, h->stream);
    else launch_coarse_gemv<float>(h->coarse_inv, h->n0, (const float*)b, (float*)x, h->stream);
    return finish_op(h);
}

nmg_status nmg_vcycle(nmg_hierarchy* h, const nmg_solve_opts* opts, const void* r, void* z) {
    if (!h || !r || !z) return fail(NMG_ERR_INVALID, "NULL argument");
    NMG_TRY(validate_opts(opts));
    NMG_TRY(check_ready(h, opts->precision));
    enter(h);
    const int prec = opts->precision;
    Level& F = h->lev[h->L - 1];
    const int64_t n = F.g.nodes * F.g.nc;
    const size_t es = prec_size(prec);
    if (opts->use_graph) {
        NMG_CK(cudaMemcpyAsync(F.p[prec].b, r, n * es, cudaMemcpyDeviceToDevice, h->stream));
        NMG_TRY(vcycle_graph(h, prec, *opts));
        NMG_CK(cudaMemcpyAsync(z, F.p[prec].x, n * es, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        vcycle_dispatch(h, prec, *opts, r, z);
    }
    return finish_op(h);
}

nmg_status nmg_get_patch_inverses(nmg_hierarchy* h, int level, int prec, int64_t first, int64_t count, double* out) {
    NMG_TRY(op_check(h, level, prec, true));
    const Geom& g = h->lev[level].g;
    if (first < 0 || count < 0 || first + count > g.patches || (count && !out))
        return fail(NMG_ERR_INVALID, "patch range out of bounds");
    enter(h);
    const PrecData& P = h->lev[level].p[prec];
    const size_t es = store_size(prec);
    std::vector<unsigned char> buf((size_t)count * P.inv_stride * es);
    NMG_CK(cudaMemcpyAsync(buf.data(), (const unsigned char*)P.inv + (size_t)first * P.inv_stride * es, buf.size(),
                           cudaMemcpyDeviceToHost, h->stream));
    NMG_CK(cudaStreamSynchronize(h->stream));
    const int np = g.np;
    for (int64_t p = 0; p < count; ++p)
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
                const size_t idx = (size_t)p * P.inv_stride + (size_t)j * np + i;
                double v;
                if (prec == NMG_PREC_FP64) v = ((const double*)buf.data())[idx];
                else if (prec == NMG_PREC_FP32) v = ((const float*)buf.data())[idx];
                else v = __bfloat162float(((const __nv_bfloat16*)buf.data())[idx]);
                out[(size_t)p * np * np + (size_t)i * np + j] = v;
            }
    return NMG_OK;
}

nmg_status nmg_profile_enable(nmg_hierarchy* h, int enable) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (enable && h->prof_ev.empty()) {
        h->prof_ev.resize(2 * 1024);
        for (auto& e : h->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(NMG_ERR_CUDA, "event creation failed");
    }
    h->prof = enable != 0;
    h->prof_used = 0;
    h->prof_ms = 0.0;
    h->prof_launches = 0;
    h->prof_bytes = 0.0;
    return NMG_OK;
}

nmg_status nmg_profile_read(nmg_hierarchy* h, double* ms_total, int64_t* launches, double* bytes_per_launch) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    NMG_CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < h->prof_used; ++i) {
        float ms = 0.f;
        NMG_CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
        h->prof_ms += ms;
        h->prof_launches++;
    }
    h->prof_used = 0;
    if (ms_total) *ms_total = h->prof_ms;
    if (launches) *launches = h->prof_launches;
    // algorithmic bytes of one finest-level Vanka apply: every patch inverse once,
    // the residual once and the per-patch corrections written once
    if (bytes_per_launch) *bytes_per_launch = h->prof_bytes;
    return NMG_OK;
}

}  // extern "C"
