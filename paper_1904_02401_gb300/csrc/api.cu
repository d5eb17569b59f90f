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
thread_local bool g_no_pdl = false;

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

static Geom make_geom(int dim, int nc, const int* cells) {
    Geom g{};
    g.dim = dim;
    g.nc = nc;
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
    const bool prof = h->prof == 2 && l == h->L - 1;
    if (prof) {
        const double sv = (double)sizeof(T);
        const double si = prec == NMG_PREC_FP64 ? 8.0 : prec == NMG_PREC_FP32 ? 4.0 : 2.0;
        const Mixed& M = L.mixed;
        const double ps = M.on ? (double)M.nsmall : (double)g.patches;
        const double pl = M.on ? (double)M.nlarge : 0.0;
        const double npl = M.on ? (double)M.np_large : 0.0;
        h->prof_bytes = (ps * g.np * g.np + pl * npl * npl) * si + (double)g.nodes * g.nc * sv +
                        (ps * g.np + pl * npl) * sv;
    }
    // mode 3: the residual products of the finest level; algorithmic bytes = the
    // Q1 blocks of the matrix once, x, b and r once
    const bool sprof = h->prof == 3 && l == h->L - 1;
    if (sprof) {
        const double sv = (double)sizeof(T);
        double nnzb = 1.0;
        for (int k = 0; k < g.dim; ++k) nnzb *= 3.0 * g.nn[k] - 2.0;
        h->prof_bytes = nnzb * g.nc * g.nc * sv + 3.0 * (double)g.nodes * g.nc * sv;
    }
    for (int st = 0; st < steps; ++st) {
        const T* d;
        if (st == 0 && x_zero) {
            d = b;
        } else {
            const bool srec = sprof && h->prof_used < (int)h->prof_ev.size() / 2;
            if (srec) cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
            launch_spmv<T>(g, (const T*)P.A, x, b, (T*)P.r, true, s);
            if (srec) {
                cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
                h->prof_used++;
            }
            d = (const T*)P.r;
        }
        const bool rec = prof && h->prof_used < (int)h->prof_ev.size() / 2;
        if (rec) cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
        const Mixed& M = L.mixed;
        const int64_t ns = M.on ? M.nsmall : -1;   // small patches: all of the level, or the listed ones
        const int32_t* ids = M.on ? M.small_id : nullptr;
        if (prec == NMG_PREC_FP64) {
            launch_vanka_apply<double, double>(g, (const double*)P.inv, P.inv_stride, (const double*)d, (double*)P.corr, s,
                                               ns, ids);
            if (M.on)
                launch_vanka_apply_large<double, double>(g, (const double*)M.inv_large[0], M.stride_large[0], M.large_org,
                                                         M.nlarge, (const double*)d, (double*)M.corr_large[0], s);
        } else if (prec == NMG_PREC_FP32) {
            launch_vanka_apply<float, float>(g, (const float*)P.inv, P.inv_stride, (const float*)d, (float*)P.corr, s,
                                             ns, ids);
            if (M.on)
                launch_vanka_apply_large<float, float>(g, (const float*)M.inv_large[1], M.stride_large[1], M.large_org,
                                                       M.nlarge, (const float*)d, (float*)M.corr_large[1], s);
        } else {
            launch_vanka_apply<float, __nv_bfloat16>(g, (const __nv_bfloat16*)P.inv, P.inv_stride, (const float*)d,
                                                    (float*)P.corr, s, ns, ids);
            if (M.on)
                launch_vanka_apply_large<float, __nv_bfloat16>(g, (const __nv_bfloat16*)M.inv_large[2], M.stride_large[2],
                                                               M.large_org, M.nlarge, (const float*)d,
                                                               (float*)M.corr_large[1], s);
        }
        if (rec) {
            cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
            h->prof_used++;
        }
        if (M.on)
            launch_vanka_update_mixed<T>(g, (const T*)P.corr, (const T*)M.corr_large[prec == NMG_PREC_FP64 ? 0 : 1],
                                         M.nsmall * g.np, M.inc, M.inc_n, x, x, st == 0 && x_zero, omega, average, s);
        else
            launch_vanka_update<T>(g, (const T*)P.corr, x, st == 0 && x_zero, omega, average, s);
    }
}

// z = V-cycle(r) on the finest level; b_fine / x_fine are the finest-level
// right-hand side and result (the level's own buffers when null).
// Top level of the cluster tail for the current threshold, at most top: the
// levels 1..c all have at most tail_patches patches and their data fits the
// shared memory of a cluster (-1: no tail).
static int tail_top(const Hierarchy* h, int prec, int top) {
    if (h->tail_patches[prec] <= 0) return -1;
    int c = -1;
    for (int l = 0; l <= top && (l == 0 || h->lev[l].g.patches <= h->tail_patches[prec]); ++l) c = l;
    return c >= 0 ? resident_tail_top(h, prec, c) : -1;
}

// True when level l (above the cluster tail top c) runs tile-fused steps.
static bool tile_level(const Hierarchy* h, int prec, int l, int c) {
    return l >= 1 && l > c && h->tile_patches[prec] > 0 && h->lev[l].g.patches <= h->tile_patches[prec];
}

// One tile-fused launch on level l (tile_kernels.cu) in the level's precision.
template <typename T>
static void tile_launch(Hierarchy* h, int l, int prec, int mode, const T* b, const T* x_in, bool x_zero,
                        const T* corr_in, const T* ec, T* x_out, T* corr_out, T* rc, T omega, bool avg) {
    Level& L = h->lev[l];
    PrecData& P = L.p[prec];
    const Geom& gc = h->lev[l - 1].g;
    const uint8_t* cmask = h->lev[l - 1].mask;
    if constexpr (sizeof(T) == 8) {
        launch_tile_step<double, double>(L.g, gc, mode, (const double*)P.A, (const double*)P.inv, P.inv_stride, b,
                                         x_in, x_zero, corr_in, ec, L.mask, cmask, x_out, corr_out, rc, omega, avg,
                                         h->stream);
    } else if (prec == NMG_PREC_FP32) {
        launch_tile_step<float, float>(L.g, gc, mode, (const float*)P.A, (const float*)P.inv, P.inv_stride, b, x_in,
                                       x_zero, corr_in, ec, L.mask, cmask, x_out, corr_out, rc, omega, avg, h->stream);
    } else {
        launch_tile_step<float, __nv_bfloat16>(L.g, gc, mode, (const float*)P.A, (const __nv_bfloat16*)P.inv,
                                               P.inv_stride, b, x_in, x_zero, corr_in, ec, L.mask, cmask, x_out,
                                               corr_out, rc, omega, avg, h->stream);
    }
}

// Pre-smoothing and restriction of a tile level: nu1 steps of Eq. (vanka)
// from x = 0 and r_{l-1} = P^T (b - A x), in nu1 + 1 launches (the last one
// also restricts).  The iterate alternates between the buffers x and x2 so that
// it ends in x after the whole cycle (tile_up); returns the buffer holding it
// after pre-smoothing.
template <typename T>
static T* tile_down(Hierarchy* h, int l, int prec, const T* b, T* X, int nu1, int nu2, T om, bool avg) {
    PrecData& P = h->lev[l].p[prec];
    const Geom& g = h->lev[l].g;
    T* Y = (T*)P.x2;
    T* C[2] = {(T*)P.corr, (T*)P.corr2};
    T* bc = (T*)h->lev[l - 1].p[prec].b;
    if (nu1 == 0) {
        cudaMemsetAsync(X, 0, g.nodes * g.nc * sizeof(T), h->stream);
        launch_restrict<T>(g, h->lev[l - 1].g, b, bc, h->lev[l - 1].mask, h->stream);
        return X;
    }
    // materialised iterates before the final update: nu1 + nu2; the last must be in Y
    T* out = ((nu1 + nu2) & 1) ? Y : X;
    const T* cur = nullptr;
    tile_launch<T>(h, l, prec, TILE_FIRST, b, nullptr, true, nullptr, nullptr, nullptr, C[0], nullptr, om, avg);
    for (int st = 1; st < nu1; ++st) {
        tile_launch<T>(h, l, prec, TILE_STEP, b, cur, cur == nullptr, C[(st - 1) & 1], nullptr, out, C[st & 1],
                       nullptr, om, avg);
        cur = out;
        out = out == X ? Y : X;
    }
    tile_launch<T>(h, l, prec, TILE_RESTRICT, b, cur, cur == nullptr, C[(nu1 - 1) & 1], nullptr, out, nullptr, bc,
                   om, avg);
    return out;
}

// Coarse-grid correction and post-smoothing of a tile level: x = cur + P e_c,
// nu2 steps of Eq. (vanka), the final update into X (nu2 + 1 launches).
template <typename T>
static void tile_up(Hierarchy* h, int l, int prec, const T* b, T* X, T* cur, int nu2, T om, bool avg) {
    PrecData& P = h->lev[l].p[prec];
    const Geom& g = h->lev[l].g;
    T* Y = (T*)P.x2;
    T* C[2] = {(T*)P.corr, (T*)P.corr2};
    const T* ec = (const T*)h->lev[l - 1].p[prec].x;
    if (nu2 == 0) {
        launch_prolong_add<T>(g, h->lev[l - 1].g, ec, cur, h->lev[l].mask, h->stream);
        if (cur != X) cudaMemcpyAsync(X, cur, g.nodes * g.nc * sizeof(T), cudaMemcpyDeviceToDevice, h->stream);
        return;
    }
    T* out = cur == X ? Y : X;
    tile_launch<T>(h, l, prec, TILE_PROLONG_STEP, b, cur, false, nullptr, ec, out, C[0], nullptr, om, avg);
    cur = out;
    for (int st = 1; st < nu2; ++st) {
        out = cur == X ? Y : X;
        tile_launch<T>(h, l, prec, TILE_STEP, b, cur, false, C[(st - 1) & 1], nullptr, out, C[st & 1], nullptr, om,
                       avg);
        cur = out;
    }
    // cur is Y here (tile_down chose the parity), so the final update never reads what it writes
    tile_launch<T>(h, l, prec, TILE_FINAL, b, cur, false, C[(nu2 - 1) & 1], nullptr, X, nullptr, nullptr, om, avg);
}

// V-cycle on levels 0..top (b_top / x_top override the top level's buffers):
// levels above the cluster tail with one kernel per step (or tile-fused
// steps), the tail (if any) as one cluster launch, else the coarse solve.
template <typename T>
static void vcycle_levels(Hierarchy* h, int prec, int top, int nu1, int nu2, double omega, int weighting,
                          const T* b_top, T* x_top, bool allow_tail) {
    cudaStream_t s = h->stream;
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    const T om = (T)omega;
    auto bptr = [&](int l) -> T* { return (l == top && b_top) ? const_cast<T*>(b_top) : (T*)h->lev[l].p[prec].b; };
    auto xptr = [&](int l) -> T* { return (l == top && x_top) ? x_top : (T*)h->lev[l].p[prec].x; };
    const int c = allow_tail ? tail_top(h, prec, top) : -1;
    T* after_pre[kMaxLevels] = {};
    for (int l = top; l >= 1 && l > c; --l) {
        Level& L = h->lev[l];
        if (tile_level(h, prec, l, c)) {
            after_pre[l] = tile_down<T>(h, l, prec, bptr(l), xptr(l), nu1, nu2, om, avg);
            continue;
        }
        smooth_level<T>(h, l, prec, bptr(l), xptr(l), nu1, true, om, avg);
        launch_spmv<T>(L.g, (const T*)L.p[prec].A, xptr(l), bptr(l), (T*)L.p[prec].r, true, s);
        launch_restrict<T>(L.g, h->lev[l - 1].g, (const T*)L.p[prec].r, bptr(l - 1), h->lev[l - 1].mask, s);
    }
    if (c >= 0) {
        if (!launch_vcycle_tail(h, prec, c, nu1, nu2, omega, weighting, bptr(c), xptr(c)))
            vcycle_levels<T>(h, prec, c, nu1, nu2, omega, weighting, bptr(c), xptr(c), false);
    } else {
        launch_coarse_gemv<T>(h->coarse_inv, h->n0, bptr(0), xptr(0), s);
    }
    for (int l = c >= 1 ? c + 1 : 1; l <= top; ++l) {
        Level& L = h->lev[l];
        if (tile_level(h, prec, l, c)) {
            tile_up<T>(h, l, prec, bptr(l), xptr(l), after_pre[l], nu2, om, avg);
            continue;
        }
        launch_prolong_add<T>(L.g, h->lev[l - 1].g, xptr(l - 1), xptr(l), L.mask, s);
        smooth_level<T>(h, l, prec, bptr(l), xptr(l), nu2, false, om, avg);
    }
}

template <typename T>
static void run_vcycle(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting, const T* b_fine,
                       T* x_fine) {
    vcycle_levels<T>(h, prec, h->L - 1, nu1, nu2, omega, weighting, b_fine, x_fine, true);
}

// The same V-cycle on the level buffers with fewer kernels: each Vanka update
// is fused into the residual that follows it, the prolongation into the first
// post-smoothing residual (the iterate alternates between the buffers x and
// x2 of a level; every level's final iterate ends in x).  The element code and
// its order are those of run_vcycle, so the results are bitwise identical.
template <typename T>
static void run_vcycle_fused(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting) {
    const int Lc = h->L;
    cudaStream_t s = h->stream;
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    const T om = (T)omega;
    const int c = tail_top(h, prec, Lc - 1);
    T* cur_level[kMaxLevels] = {};
    auto apply = [&](int l, const T* d) {
        PrecData& P = h->lev[l].p[prec];
        const Geom& g = h->lev[l].g;
        if (prec == NMG_PREC_FP64)
            launch_vanka_apply<double, double>(g, (const double*)P.inv, P.inv_stride, (const double*)d, (double*)P.corr, s);
        else if (prec == NMG_PREC_FP32)
            launch_vanka_apply<float, float>(g, (const float*)P.inv, P.inv_stride, (const float*)d, (float*)P.corr, s);
        else
            launch_vanka_apply<float, __nv_bfloat16>(g, (const __nv_bfloat16*)P.inv, P.inv_stride, (const float*)d,
                                                    (float*)P.corr, s);
    };
    for (int l = Lc - 1; l >= 1 && l > c; --l) {
        Level& L = h->lev[l];
        PrecData& P = L.p[prec];
        T* X = (T*)P.x;
        T* Y = (T*)P.x2;
        const T* A = (const T*)P.A;
        const T* b = (const T*)P.b;
        T* r = (T*)P.r;
        const T* corr = (const T*)P.corr;
        T* bufs[2] = {X, Y};
        int nb = 0;
        const T* cur = X;
        if (nu1 == 0) {
            cudaMemsetAsync(X, 0, L.g.nodes * L.g.nc * sizeof(T), s);
            launch_restrict<T>(L.g, h->lev[l - 1].g, b, (T*)h->lev[l - 1].p[prec].b, h->lev[l - 1].mask, s);
        } else {
            bool zero = true;
            apply(l, b);
            for (int st = 1; st <= nu1; ++st) {   // the last pass gives the residual for the restriction
                T* out = bufs[nb];
                nb ^= 1;
                launch_update_residual<T>(L.g, A, corr, zero ? nullptr : cur, zero, om, avg, b, out, r, s);
                cur = out;
                zero = false;
                if (st < nu1) apply(l, r);
            }
            launch_restrict<T>(L.g, h->lev[l - 1].g, r, (T*)h->lev[l - 1].p[prec].b, h->lev[l - 1].mask, s);
        }
        cur_level[l] = const_cast<T*>(cur);
    }
    if (c >= 0) {
        if (!launch_vcycle_tail(h, prec, c, nu1, nu2, omega, weighting, nullptr, nullptr))
            vcycle_levels<T>(h, prec, c, nu1, nu2, omega, weighting, nullptr, nullptr, false);
    } else {
        launch_coarse_gemv<T>(h->coarse_inv, h->n0, (const T*)h->lev[0].p[prec].b, (T*)h->lev[0].p[prec].x, s);
    }
    for (int l = c >= 1 ? c + 1 : 1; l < Lc; ++l) {
        Level& L = h->lev[l];
        PrecData& P = L.p[prec];
        T* X = (T*)P.x;
        T* Y = (T*)P.x2;
        const T* A = (const T*)P.A;
        const T* b = (const T*)P.b;
        T* r = (T*)P.r;
        const T* corr = (const T*)P.corr;
        const T* ec = (const T*)h->lev[l - 1].p[prec].x;
        T* cur = cur_level[l];
        if (nu2 == 0) {
            launch_prolong_add<T>(L.g, h->lev[l - 1].g, ec, cur, L.mask, s);
            if (cur != X) cudaMemcpyAsync(X, cur, L.g.nodes * L.g.nc * sizeof(T), cudaMemcpyDeviceToDevice, s);
            continue;
        }
        T* out = cur == X ? Y : X;
        launch_prolong_residual<T>(L.g, h->lev[l - 1].g, A, ec, cur, L.mask, b, out, r, s);
        cur = out;
        apply(l, r);
        for (int st = 1; st < nu2; ++st) {
            out = cur == X ? Y : X;
            launch_update_residual<T>(L.g, A, corr, cur, false, om, avg, b, out, r, s);
            cur = out;
            apply(l, r);
        }
        launch_vanka_update2<T>(L.g, corr, cur, X, false, om, avg, s);
    }
}

static void vcycle_dispatch(Hierarchy* h, int prec, const nmg_solve_opts& o, const void* b, void* x) {
    if (h->fused[prec] && !b && !x) {
        if (prec == NMG_PREC_FP64) run_vcycle_fused<double>(h, prec, o.nu1, o.nu2, o.omega, o.weighting);
        else run_vcycle_fused<float>(h, prec, o.nu1, o.nu2, o.omega, o.weighting);
        return;
    }
    if (prec == NMG_PREC_FP64)
        run_vcycle<double>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, (const double*)b, (double*)x);
    else
        run_vcycle<float>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, (const float*)b, (float*)x);
}

// Replays (capturing first if needed) the V-cycle on the level buffers as a CUDA graph.
static nmg_status vcycle_graph(Hierarchy* h, int prec, const nmg_solve_opts& o) {
    const int key[5] = {o.nu1, o.nu2, o.weighting, 2 * h->tail_patches[prec] + h->fused[prec], h->tile_patches[prec]};
    bool match = h->vgraph[prec] && std::memcmp(key, h->vgraph_key[prec], sizeof(key)) == 0 &&
                 h->vgraph_omega[prec] == o.omega;
    if (!match) {
        if (h->vgraph[prec]) cudaGraphExecDestroy(h->vgraph[prec]);
        h->vgraph[prec] = nullptr;
        cudaGraph_t graph;
        NMG_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int prof = h->prof;
        h->prof = 0;   // no event nodes inside the graph
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
        (o->weighting != NMG_WEIGHT_AVERAGE && o->weighting != NMG_WEIGHT_SUM) || o->use_graph < 0 || o->use_graph > 2 ||
        o->engine < NMG_ENGINE_AUTO || o->engine > NMG_ENGINE_FUSED || o->tail_patches < 0 || o->tile_patches < 0)
        return fail(NMG_ERR_INVALID, "invalid solve options");
    return NMG_OK;
}

// Algorithmic bytes of one V(nu1, nu2) cycle: on every smoothed level each
// smoothing step reads all patch inverses once and writes / reads the
// per-patch corrections, each residual reads the matrix once, and the vector
// traffic of residual (x, b, r), update (x) and transfers is counted once per
// step; the coarse solve reads its dense inverse.  (Unique bytes a perfect
// implementation must move; reuse through the L2 can make a measured rate
// exceed the HBM copy rate on levels that fit in the L2.)
static double vcycle_bytes(const Hierarchy* h, int prec, int nu1, int nu2) {
    const double sv = prec == NMG_PREC_FP64 ? 8.0 : 4.0;
    const double si = prec == NMG_PREC_FP64 ? 8.0 : prec == NMG_PREC_FP32 ? 4.0 : 2.0;
    double bytes = (double)h->n0 * h->n0 * 8.0 + 2.0 * h->n0 * sv;
    for (int l = 1; l < h->L; ++l) {
        const Geom& g = h->lev[l].g;
        const double n = (double)g.nodes * g.nc;
        const double mat = (double)g.nst * g.nc * g.nc * g.nodes * sv;
        const Mixed& M = h->lev[l].mixed;
        const double ps = M.on ? (double)M.nsmall : (double)g.patches, pl = M.on ? (double)M.nlarge : 0.0;
        const double npl = M.on ? (double)M.np_large : 0.0;
        const double inv = (ps * g.np * g.np + pl * npl * npl) * si;
        const double corr = (ps * g.np + pl * npl) * sv;
        const int steps = nu1 + nu2;
        const int residuals = (nu1 > 0 ? nu1 - 1 : 0) + 1 + nu2;
        bytes += steps * (inv + 2.0 * corr + 3.0 * n) + residuals * (mat + 3.0 * n);
        const Geom& c = h->lev[l - 1].g;
        bytes += 2.0 * (n + (double)c.nodes * c.nc);   // restriction and prolongation
    }
    return bytes;
}

// One V-cycle on the finest level's buffers (b -> x) with the given engine.
static nmg_status run_engine(Hierarchy* h, const nmg_solve_opts& o, int engine) {
    const int prec = o.precision;
    if (engine == NMG_ENGINE_PERSISTENT) {
        NMG_CK(launch_vcycle_persistent(h, prec, o.nu1, o.nu2, o.omega, o.weighting, h->pbar, h->flags + FLAG_ABORT,
                                        64));
        return NMG_OK;
    }
    h->fused[prec] = engine == NMG_ENGINE_FUSED;
    if (o.use_graph) return vcycle_graph(h, prec, o);
    vcycle_dispatch(h, prec, o, nullptr, nullptr);
    return NMG_OK;
}

// Autotuner.  For AUTO the V-cycle shape is picked by timing the candidates
// on this hierarchy (finest right-hand side zeroed, so the memory traffic is
// the real one): the per-step-kernel engine, plain or with fused
// update/prolongation + residual, with the cluster tail covering the levels of
// at most {0, 64, 256, 1024, 4096} patches, and the persistent engine.
// The fastest is kept per precision and (nu1, nu2, weighting).
static nmg_status resolve_engine(Hierarchy* h, const nmg_solve_opts& o, int* engine) {
    const int prec = o.precision;
    if (h->nc == h->dim || h->mixed_any) {   // vector problems or patches of two sizes: per-step kernels only
        if (o.engine != NMG_ENGINE_AUTO && o.engine != NMG_ENGINE_KERNELS)
            return fail(NMG_ERR_INVALID,
                        "hierarchies with ncomp = dim or with patches of two sizes run the KERNELS engine only");
        h->tail_patches[prec] = 0;
        h->tile_patches[prec] = 0;
        h->fused[prec] = 0;
        *engine = NMG_ENGINE_KERNELS;
        return NMG_OK;
    }
    if (o.engine != NMG_ENGINE_AUTO) {
        h->tail_patches[prec] = o.engine == NMG_ENGINE_PERSISTENT ? 0 : o.tail_patches;
        h->tile_patches[prec] = o.engine == NMG_ENGINE_KERNELS ? o.tile_patches : 0;
        *engine = o.engine;
        return NMG_OK;
    }
    const int key[3] = {o.nu1, o.nu2, o.weighting};
    if (h->engine_choice[prec] && std::memcmp(key, h->engine_key[prec], sizeof(key)) == 0) {
        h->tail_patches[prec] = h->auto_tail[prec];
        h->tile_patches[prec] = h->auto_tile[prec];
        *engine = h->engine_choice[prec];
        return NMG_OK;
    }
    Level& F = h->lev[h->L - 1];
    const size_t vs = prec == NMG_PREC_FP64 ? sizeof(double) : sizeof(float);
    NMG_CK(cudaMemsetAsync(F.p[prec].b, 0, F.g.nodes * F.g.nc * vs, h->stream));
    cudaEvent_t e0, e1;
    NMG_CK(cudaEventCreate(&e0));
    NMG_CK(cudaEventCreate(&e1));
    struct Cand { int engine, tail, fused, tile; };
    std::vector<Cand> cands;
    int last_level = -2;
    for (int tail : {0, 64, 256, 1024, 4096}) {
        h->tail_patches[prec] = tail;
        const int c = tail_top(h, prec, h->L - 1);
        if (c != last_level) {
            for (int fz : {0, 1}) cands.push_back({fz ? NMG_ENGINE_FUSED : NMG_ENGINE_KERNELS, tail, fz, 0});
            // tile-fused steps on the levels above the tail up to each level size (at most 16384 patches)
            for (int l = c >= 1 ? c + 1 : 1; l < h->L; ++l)
                if (h->lev[l].g.patches <= 16384)
                    cands.push_back({NMG_ENGINE_KERNELS, tail, 0, (int)h->lev[l].g.patches});
        }
        last_level = c;
    }
    cands.push_back({NMG_ENGINE_PERSISTENT, 0, 0, 0});
    double best = 1e300;
    Cand pick = cands[0];
    const int64_t launches0 = g_launches;
    h->tuning[prec].clear();
    for (const Cand& cd : cands) {
        h->tail_patches[prec] = cd.tail;
        h->tile_patches[prec] = cd.tile;
        h->fused[prec] = cd.fused;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) ok = run_engine(h, o, cd.engine) == NMG_OK;
        cudaEventRecord(e0, h->stream);
        for (int rep = 0; rep < 5 && ok; ++rep) ok = run_engine(h, o, cd.engine) == NMG_OK;
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
        float ms = 0.f;
        double us = -1.0;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            us = 1000.0 * ms / 5.0;
            if (us < best) { best = us; pick = cd; }
        }
        h->tuning[prec].push_back({cd.engine, cd.tail, cd.fused, cd.tile, us});
        cudaGetLastError();
    }
    g_launches = launches0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int f[FLAG_COUNT];
    NMG_CK(cudaMemcpy(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (f[FLAG_ABORT]) {   // a persistent trial aborted: never pick it
        NMG_CK(cudaMemset(h->flags + FLAG_ABORT, 0, sizeof(int)));
        if (pick.engine == NMG_ENGINE_PERSISTENT) pick = cands[0];
    }
    h->fused[prec] = pick.fused;
    h->tail_patches[prec] = pick.tail;
    h->auto_tail[prec] = pick.tail;
    h->tile_patches[prec] = pick.tile;
    h->auto_tile[prec] = pick.tile;
    h->engine_choice[prec] = pick.engine;
    std::memcpy(h->engine_key[prec], key, sizeof(key));
    *engine = pick.engine;
    return NMG_OK;
}

// One V-cycle on the finest level's own buffers (b -> x) with the engine the
// options (or the autotuner) select; bracketed by events in profiling mode 1.
static nmg_status vcycle_in_place(Hierarchy* h, const nmg_solve_opts& o) {
    int engine = 0;
    NMG_TRY(resolve_engine(h, o, &engine));
    const bool rec = h->prof == 1 && h->prof_used < (int)h->prof_ev.size() / 2;
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_used], h->stream);
        h->prof_bytes = vcycle_bytes(h, o.precision, o.nu1, o.nu2);
    }
    NMG_TRY(run_engine(h, o, engine));
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], h->stream);
        h->prof_used++;
    }
    return NMG_OK;
}

// v = w * scal[S_INVH] into the Krylov basis (column j + 1 of the current
// step when next, else column 0), also written, converted, as the right-hand
// side of the next V-cycle.
static void scale_into_vcycle_input(Hierarchy* h, const nmg_solve_opts& o, const double* w, bool next) {
    Level& F = h->lev[h->L - 1];
    const int64_t n = F.g.nodes * F.g.nc;
    if (o.precision == NMG_PREC_FP64)
        launch_scale_convert<double>(w, h->scal + S_INVH, h->V, n, h->cyc, next, (double*)F.p[NMG_PREC_FP64].b, n,
                                     h->stream);
    else
        launch_scale_convert<float>(w, h->scal + S_INVH, h->V, n, h->cyc, next, (float*)F.p[o.precision].b, n,
                                    h->stream);
}

// z = V-cycle(v) for vectors of the precision's arithmetic type or FP64 (converted).
static nmg_status vcycle_any(Hierarchy* h, const nmg_solve_opts& o, const void* v, void* z, bool fp64_io) {
    Level& F = h->lev[h->L - 1];
    const int64_t n = F.g.nodes * F.g.nc;
    const int prec = o.precision;
    int engine = 0;
    NMG_TRY(resolve_engine(h, o, &engine));
    if (prec == NMG_PREC_FP64 && engine == NMG_ENGINE_KERNELS && !o.use_graph && h->prof != 1) {
        h->fused[prec] = 0;
        run_vcycle<double>(h, prec, o.nu1, o.nu2, o.omega, o.weighting, (const double*)v, (double*)z);
        return NMG_OK;
    }
    const size_t vs = prec == NMG_PREC_FP64 ? sizeof(double) : sizeof(float);
    if (prec != NMG_PREC_FP64 && fp64_io) launch_convert<double, float>((const double*)v, (float*)F.p[prec].b, n, h->stream);
    else NMG_CK(cudaMemcpyAsync(F.p[prec].b, v, n * vs, cudaMemcpyDeviceToDevice, h->stream));
    const bool rec = h->prof == 1 && h->prof_used < (int)h->prof_ev.size() / 2;
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_used], h->stream);
        h->prof_bytes = vcycle_bytes(h, prec, o.nu1, o.nu2);
    }
    NMG_TRY(run_engine(h, o, engine));
    if (rec) {
        cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], h->stream);
        h->prof_used++;
    }
    if (prec != NMG_PREC_FP64 && fp64_io) launch_convert<float, double>((const float*)F.p[prec].x, (double*)z, n, h->stream);
    else NMG_CK(cudaMemcpyAsync(z, F.p[prec].x, n * vs, cudaMemcpyDeviceToDevice, h->stream));
    return NMG_OK;
}

// ---------------------------------------------------------------------------
// Multi-vector V-cycles: K = 4 or 8 right-hand sides per pass over the level
// matrices and patch inverses (precision FP32 or BF16; FP32 vectors,
// interleaved in the levels' MultiData buffers).  Per column the same
// kernels' arithmetic as the per-step V-cycle, so each column's result equals
// a single V-cycle's bit for bit.
// ---------------------------------------------------------------------------
static size_t many_level_bytes(const Geom& g, int l, int K, int which) {
    if (which == 3) return l > 0 ? (size_t)g.patches * g.np * K * sizeof(float) : 0;
    return (size_t)g.nodes * g.nc * K * sizeof(float);
}

// Level buffers for K columns (kept, and reused by calls with fewer).
static nmg_status ensure_many(Hierarchy* h, int K) {
    if (h->many_k >= K) return NMG_OK;
    NMG_CK(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->L; ++l) {
        MultiData& M = h->lev[l].m;
        float** q[4] = {&M.b, &M.x, &M.r, &M.corr};
        for (int w = 0; w < 4; ++w) {
            if (!*q[w]) continue;
            for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
                if (*it == (void*)*q[w]) { h->allocs.erase(it); break; }
            cudaFree(*q[w]);
            h->bytes -= std::max<size_t>(16, many_level_bytes(h->lev[l].g, l, h->many_k, w));
            *q[w] = nullptr;
        }
    }
    h->many_k = 0;
    h->many_gen++;
    for (int l = 0; l < h->L; ++l) {
        MultiData& M = h->lev[l].m;
        float** q[4] = {&M.b, &M.x, &M.r, &M.corr};
        for (int w = 0; w < 4; ++w) NMG_TRY(dalloc(h, (void**)q[w], many_level_bytes(h->lev[l].g, l, K, w)));
    }
    h->many_k = K;
    return NMG_OK;
}

// False if a level's inverses are not in the layout the streaming apply needs
// (16-byte aligned, unpadded n_p x n_p columns); never the case for
// hierarchies built by nmg_create_hierarchy.
static bool many_layout_ok(const Hierarchy* h, int prec) {
    const size_t es = store_size(prec);
    for (int l = 1; l < h->L; ++l) {
        const PrecData& P = h->lev[l].p[prec];
        const int64_t np = h->lev[l].g.np;
        if ((uintptr_t)P.inv % 16 || (P.inv_stride * (int64_t)es) % 16 || P.inv_stride < np * np ||
            P.inv_stride * (int64_t)es > np * np * (int64_t)es + 16)
            return false;
    }
    return true;
}

template <int K>
static void smooth_level_many(Hierarchy* h, int l, int prec, int steps, bool x_zero, float omega, bool average) {
    Level& L = h->lev[l];
    MultiData& M = L.m;
    const Geom& g = L.g;
    cudaStream_t s = h->stream;
    if (steps == 0 && x_zero) {
        cudaMemsetAsync(M.x, 0, g.nodes * g.nc * K * sizeof(float), s);
        return;
    }
    for (int st = 0; st < steps; ++st) {
        const float* d = M.b;
        if (!(st == 0 && x_zero)) {
            launch_spmv_many<K>(g, (const float*)L.p[prec].A, M.x, M.b, M.r, true, s);
            d = M.r;
        }
        if (prec == NMG_PREC_FP32)
            launch_vanka_apply_many<K, float>(g, (const float*)L.p[prec].inv, L.p[prec].inv_stride, d, M.corr,
                                              h->flags + FLAG_MANY, s);
        else
            launch_vanka_apply_many<K, __nv_bfloat16>(g, (const __nv_bfloat16*)L.p[prec].inv, L.p[prec].inv_stride,
                                                      d, M.corr, h->flags + FLAG_MANY, s);
        launch_vanka_update_many<K>(g, M.corr, M.x, M.x, st == 0 && x_zero, omega, average, s);
    }
}

// One V(nu1, nu2)-cycle on the finest level's multi-vector buffers b -> x,
// the steps of vcycle_levels without cluster tail or tile fusion.
template <int K>
static void vcycle_many_levels(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting) {
    cudaStream_t s = h->stream;
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    const float om = (float)omega;
    const int top = h->L - 1;
    for (int l = top; l >= 1; --l) {
        Level& L = h->lev[l];
        smooth_level_many<K>(h, l, prec, nu1, true, om, avg);
        launch_spmv_many<K>(L.g, (const float*)L.p[prec].A, L.m.x, L.m.b, L.m.r, true, s);
        launch_restrict_many<K>(L.g, h->lev[l - 1].g, L.m.r, h->lev[l - 1].m.b, h->lev[l - 1].mask, s);
    }
    launch_coarse_gemv_many<K>(h->coarse_inv, h->n0, h->lev[0].m.b, h->lev[0].m.x, s);
    for (int l = 1; l <= top; ++l) {
        Level& L = h->lev[l];
        launch_prolong_add_many<K>(L.g, h->lev[l - 1].g, h->lev[l - 1].m.x, L.m.x, L.mask, s);
        smooth_level_many<K>(h, l, prec, nu2, false, om, avg);
    }
}

// The multi-vector V-cycle on the level buffers: replayed from a graph
// (captured on first use per precision, K and options) when use_graph, else
// launched kernel by kernel.
template <int K>
static nmg_status run_vcycle_many(Hierarchy* h, const nmg_solve_opts& o) {
    const int prec = o.precision, ki = K == 4 ? 0 : 1;
    if (!o.use_graph) {
        vcycle_many_levels<K>(h, prec, o.nu1, o.nu2, o.omega, o.weighting);
        return NMG_OK;
    }
    const int key[4] = {o.nu1, o.nu2, o.weighting, h->many_gen};
    cudaGraphExec_t& ex = h->mgraph[prec][ki];
    if (!ex || std::memcmp(key, h->mgraph_key[prec][ki], sizeof(key)) != 0 || h->mgraph_omega[prec][ki] != o.omega) {
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
        cudaGraph_t graph;
        NMG_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = g_launches;
        vcycle_many_levels<K>(h, prec, o.nu1, o.nu2, o.omega, o.weighting);
        h->mgraph_nodes[prec][ki] = g_launches - before;
        g_launches = before;
        NMG_CK(cudaStreamEndCapture(h->stream, &graph));
        cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        NMG_CK(e);
        std::memcpy(h->mgraph_key[prec][ki], key, sizeof(key));
        h->mgraph_omega[prec][ki] = o.omega;
    }
    NMG_CK(cudaGraphLaunch(ex, h->stream));
    g_launches += h->mgraph_nodes[prec][ki];
    return NMG_OK;
}

// z_k = M^{-1} r_k for ncols <= 8 columns given by pointers (FP32 vectors of
// the finest level): interleave, one multi-vector V-cycle, de-interleave.
static nmg_status vcycle_cols(Hierarchy* h, const nmg_solve_opts& o, int ncols, const ColPtrs& in,
                              const ColPtrsOut& out) {
    const Level& F = h->lev[h->L - 1];
    const int64_t n = F.g.nodes * F.g.nc;
    const int K = ncols <= 4 ? 4 : 8;
    NMG_TRY(ensure_many(h, K));
    if (K == 4) {
        launch_pack<4>(in, ncols, n, F.m.b, h->stream);
        NMG_TRY(run_vcycle_many<4>(h, o));
        launch_unpack<4>(F.m.x, out, ncols, n, h->stream);
    } else {
        launch_pack<8>(in, ncols, n, F.m.b, h->stream);
        NMG_TRY(run_vcycle_many<8>(h, o));
        launch_unpack<8>(F.m.x, out, ncols, n, h->stream);
    }
    return NMG_OK;
}

static nmg_status check_many(Hierarchy* h, const nmg_solve_opts& o) {
    if (o.precision != NMG_PREC_FP32 && o.precision != NMG_PREC_BF16)
        return fail(NMG_ERR_INVALID, "multi-vector V-cycles run in precision FP32 or BF16");
    if (!many_layout_ok(h, o.precision)) return fail(NMG_ERR_INVALID, "patch inverse layout");
    if (h->mixed_any) return fail(NMG_ERR_INVALID, "multi-vector V-cycles need patches of one size");
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
    h->krylov_gen++;
    return NMG_OK;
}

// Bytes ensure_krylov(h, m) would add to h->bytes (0 when the bases already hold m).
static size_t krylov_growth(const Hierarchy* h, int m) {
    if (h->m_alloc >= m) return 0;
    const Geom& g = h->lev[h->L - 1].g;
    const size_t vec = (size_t)g.nodes * g.nc * sizeof(double);
    const size_t held = h->V ? (size_t)(2 * h->m_alloc + 1) * vec : 0;
    return (size_t)(2 * m + 1) * vec - held;
}

// Bytes ensure_many(h, K) would add to h->bytes (0 when the buffers already hold K columns).
static size_t many_growth(const Hierarchy* h, int K) {
    if (h->many_k >= K) return 0;
    size_t add = 0, held = 0;
    for (int l = 0; l < h->L; ++l)
        for (int w = 0; w < 4; ++w) {
            add += std::max<size_t>(16, many_level_bytes(h->lev[l].g, l, K, w));
            if (h->many_k) held += std::max<size_t>(16, many_level_bytes(h->lev[l].g, l, h->many_k, w));
        }
    return add - held;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct SolveJob {
    enum Phase { P_NONE, P_NORM, P_CYCLE, P_ITER, P_FINISH, P_DONE, P_WANT };
    bool loop = false;        // the current cycle's steps were enqueued as one graph loop
    bool grouped = false;     // one column of a multi-vector solve: the group enqueues its V-cycles (P_WANT)
    Hierarchy* h = nullptr;
    nmg_solve_opts o{};
    const double* b_user = nullptr;
    double* x_user = nullptr;
    bool b_dev = false, x_dev = false;
    Phase phase = P_NONE;
    int its = 0, cycles = 0, engine = NMG_ENGINE_KERNELS;
    bool used_loop = false;
    bool finish_ready = false;   // the finish copies were enqueued with the last true residual
    double bnorm = 0.0, relres = 0.0;
    nmg_status st = NMG_OK;
    std::string err;
    int64_t launches0 = 0, launches = 0;
    std::chrono::steady_clock::time_point t0;
};

// ---------------------------------------------------------------------------
// One FGMRES solve as a resumable job: job_enqueue() puts the next step on the
// hierarchy's stream, job_advance() runs on the host once that work has
// completed (it reads the few scalars copied back to pinned memory) and picks
// the next step.  nmg_solve drives one job synchronously; the server drives
// many jobs on different streams at once.
// ---------------------------------------------------------------------------
static void job_fail(SolveJob& J, nmg_status st) {
    J.st = st;
    J.err = g_last_error;
}

#define JOB_CK(call)                                                                 \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            fail(NMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
            job_fail(J, NMG_ERR_CUDA);                                               \
            J.phase = SolveJob::P_DONE;                                              \
            return;                                                                  \
        }                                                                            \
    } while (0)

static void job_enqueue_cycle(SolveJob& J) {
    Hierarchy* h = J.h;
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    cudaStream_t s = h->stream;
    // true residual r = b - A x and beta = ||r||, v_0 = r / beta
    launch_spmv<double>(g, h->lev[h->L - 1].A64, h->x64, h->b64, h->w64, true, s);
    launch_norm2(h->w64, n, h->partial, h->scal + S_BETA, s);
    launch_start_cycle(h->scal, J.o.restart, h->cyc, s);
    scale_into_vcycle_input(h, J.o, h->w64, false);
    JOB_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    J.phase = SolveJob::P_CYCLE;
}

// The first cycle from x0 = 0: the residual b - A 0 is b itself (bitwise:
// every product term is a signed zero and b_i - 0 = b_i) and its norm is the
// ||b|| just computed with the same reduction, so the cycle starts from b
// without a product and without another host round trip.
static void job_enqueue_first_cycle(SolveJob& J) {
    Hierarchy* h = J.h;
    cudaStream_t s = h->stream;
    JOB_CK(cudaMemcpyAsync(h->scal + S_BETA, h->scal + S_BNORM, sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_start_cycle(h->scal, J.o.restart, h->cyc, s);
    scale_into_vcycle_input(h, J.o, h->b64, false);
}

// One FGMRES step j (read on the device from cyc[0]): z_j = M^{-1} v_j (v_j is
// already the V-cycle's right-hand side, written by the scaling that produced
// it); w = A z_j in FP64 with z_j stored as basis vector Z_j, fused with the
// first classical Gram-Schmidt pass; the first update fused with the second
// pass, ||w|| and the Givens update; the second update fused with the
// scaling v_{j+1} = w / h_{j+1,j}; and the on-device decision whether the
// cycle goes on.  in_loop: the launches are being captured as the body of a
// graph loop whose condition the decision sets (the V-cycle is captured
// inline then).
static void enqueue_arnoldi(Hierarchy* h, const nmg_solve_opts& o, bool in_loop, cudaGraphConditionalHandle loop);

static nmg_status enqueue_step(Hierarchy* h, const nmg_solve_opts& o, int engine, bool in_loop,
                               cudaGraphConditionalHandle loop) {
    if (in_loop) {
        h->fused[o.precision] = engine == NMG_ENGINE_FUSED;
        vcycle_dispatch(h, o.precision, o, nullptr, nullptr);
    } else {
        NMG_TRY(vcycle_in_place(h, o));
    }
    enqueue_arnoldi(h, o, in_loop, loop);
    return NMG_OK;
}

// The part of an FGMRES step after z_j = M^{-1} v_j (z_j in the finest
// level's V-cycle result buffer of the precision): product, Gram-Schmidt,
// norm, Givens update, scaling into the next V-cycle input and decision.
static void enqueue_arnoldi(Hierarchy* h, const nmg_solve_opts& o, bool in_loop, cudaGraphConditionalHandle loop) {
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    const int m = o.restart;
    cudaStream_t s = h->stream;
    const PrecData& PF = h->lev[h->L - 1].p[o.precision];
    double* A64 = h->lev[h->L - 1].A64;
    if (o.precision == NMG_PREC_FP64)
        launch_spmv_zstore_dots<double>(g, A64, (const double*)PF.x, h->Z, h->w64, h->V, n, h->cyc, h->partial,
                                        h->scal + S_HC, h->counters, s);
    else
        launch_spmv_zstore_dots<float>(g, A64, (const float*)PF.x, h->Z, h->w64, h->V, n, h->cyc, h->partial,
                                       h->scal + S_HC, h->counters, s);
    launch_gs_update_dot_norm(h->V, n, h->cyc, h->w64, n, h->partial, h->scal, m, h->counters, s);
    Level& F = h->lev[h->L - 1];
    if (o.precision == NMG_PREC_FP64)
        launch_gs_update_scale<double>(h->V, n, h->cyc, h->scal, h->w64, (double*)F.p[NMG_PREC_FP64].b, n, m, s);
    else
        launch_gs_update_scale<float>(h->V, n, h->cyc, h->scal, h->w64, (float*)F.p[o.precision].b, n, m, s);
    launch_decide(h->scal, h->cyc, o.rtol, o.maxit, m, loop, in_loop, s);
}

// The steps of one restart cycle as one executable graph: a while-loop node
// whose body is enqueue_step and whose condition the step's decision kernel
// sets, so a cycle needs no host round trip per step.  Built once per
// (precision, options, engine) and replayed; nullptr when the device or the
// driver cannot build it (the host then steps the cycle).
static cudaGraphExec_t cycle_graph(Hierarchy* h, const nmg_solve_opts& o, int engine) {
    if (h->loop_mode < 0 || engine == NMG_ENGINE_PERSISTENT) return nullptr;
    const int prec = o.precision;
    Hierarchy::LoopKey key{};
    key.nu1 = o.nu1; key.nu2 = o.nu2; key.weighting = o.weighting; key.engine = engine;
    key.tail = h->tail_patches[prec]; key.tile = h->tile_patches[prec];
    key.restart = o.restart; key.maxit = o.maxit; key.gen = h->krylov_gen;
    key.omega = o.omega; key.rtol = o.rtol;
    const Hierarchy::LoopKey& k0 = h->cgraph_key[prec];
    if (h->cgraph[prec] && k0.nu1 == key.nu1 && k0.nu2 == key.nu2 && k0.weighting == key.weighting &&
        k0.engine == key.engine && k0.tail == key.tail && k0.tile == key.tile && k0.restart == key.restart &&
        k0.maxit == key.maxit &&
        k0.gen == key.gen && k0.omega == key.omega && k0.rtol == key.rtol)
        return h->cgraph[prec];
    if (h->cgraph[prec]) cudaGraphExecDestroy(h->cgraph[prec]);
    h->cgraph[prec] = nullptr;
    // first with programmatic launch edges inside the body, then without
    for (int mode = h->loop_mode == 2 ? 2 : 1; mode <= 2; ++mode) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
        cudaGraphConditionalHandle cond = 0;
        ok = ok && cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = cond;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) == cudaSuccess;
        if (ok) {
            cudaGraph_t body = p.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                cudaSuccess) {
                const int prof = h->prof;
                h->prof = 0;
                g_no_pdl = mode == 2;
                const int64_t before = g_launches;
                const nmg_status st = enqueue_step(h, o, engine, true, cond);
                h->cgraph_nodes[prec] = g_launches - before;
                g_launches = before;
                g_no_pdl = false;
                h->prof = prof;
                const cudaError_t e = cudaStreamEndCapture(h->stream, &body);
                ok = st == NMG_OK && e == cudaSuccess;
            } else {
                ok = false;
            }
        }
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (ok) {
            h->loop_mode = mode;
            h->cgraph[prec] = exec;
            h->cgraph_key[prec] = key;
            return exec;
        }
        if (exec) cudaGraphExecDestroy(exec);
    }
    h->loop_mode = -1;
    return nullptr;
}

// Enqueues the steps of the current cycle: all of them as one graph loop
// (use_graph 2), or the next single step (the host decides after each).
static void job_enqueue_iter(SolveJob& J) {
    Hierarchy* h = J.h;
    cudaStream_t s = h->stream;
    if (J.grouped) {   // the next step waits for the group's multi-vector V-cycle
        J.phase = SolveJob::P_WANT;
        return;
    }
    cudaGraphExec_t loop = J.o.use_graph == 2 ? cycle_graph(h, J.o, J.engine) : nullptr;
    J.loop = loop != nullptr;
    if (loop) {
        J.used_loop = true;
        JOB_CK(cudaGraphLaunch(loop, s));
    } else {
        const nmg_status st = enqueue_step(h, J.o, J.engine, false, 0);
        if (st != NMG_OK) {
            job_fail(J, st);
            J.phase = SolveJob::P_DONE;
            return;
        }
    }
    JOB_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    JOB_CK(cudaMemcpyAsync(h->host_cyc, h->cyc, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    J.phase = SolveJob::P_ITER;
}

static void job_enqueue_finish(SolveJob& J) {
    Hierarchy* h = J.h;
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    cudaStream_t s = h->stream;
    JOB_CK(cudaMemcpyAsync(J.x_user, h->x64, n * sizeof(double),
                           J.x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    JOB_CK(wait_timeout_enqueue_read(h->host_flags + FLAG_COUNT, s));
    JOB_CK(cudaMemcpyAsync(h->host_flags, h->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    J.phase = SolveJob::P_FINISH;
}

// Starts a job: validates, enqueues the copy of b and the norm of b.
static nmg_status job_start(SolveJob& J, Hierarchy* h, const double* b_user, double* x_user,
                            const nmg_solve_opts& o) {
    J = SolveJob();
    J.h = h;
    J.o = o;
    J.b_user = b_user;
    J.x_user = x_user;
    J.t0 = std::chrono::steady_clock::now();
    J.launches0 = g_launches;
    NMG_TRY(check_ready(h, o.precision));
    NMG_TRY(ensure_krylov(h, o.restart));
    NMG_TRY(resolve_engine(h, o, &J.engine));
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    cudaStream_t s = h->stream;
    J.b_dev = is_device_ptr(b_user);
    J.x_dev = is_device_ptr(x_user);
    NMG_CK(cudaMemcpyAsync(h->b64, b_user, n * sizeof(double), J.b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NMG_CK(cudaMemsetAsync(h->scal, 0, 8 * sizeof(double), s));
    NMG_CK(cudaMemsetAsync(h->x64, 0, n * sizeof(double), s));
    NMG_CK(cudaMemsetAsync(h->cyc, 0, 4 * sizeof(int), s));
    launch_norm2(h->b64, n, h->partial, h->scal + S_BNORM, s);
    NMG_CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    J.launches = g_launches - J.launches0;
    J.phase = SolveJob::P_NORM;
    return NMG_OK;
}

// Host step after the enqueued work has completed.
static void job_advance(SolveJob& J) {
    Hierarchy* h = J.h;
    const double* hs = h->host_scal;
    switch (J.phase) {
    case SolveJob::P_NORM:
        J.bnorm = hs[S_BNORM];
        if (!std::isfinite(J.bnorm)) {
            fail(NMG_ERR_NONFINITE, "non-finite right-hand side");
            job_fail(J, NMG_ERR_NONFINITE);
            job_enqueue_finish(J);
        } else if (J.bnorm == 0.0) {
            job_enqueue_finish(J);
        } else {
            J.relres = 1.0;   // ||b - A 0|| / ||b||
            if (J.relres <= J.o.rtol) {
                job_enqueue_finish(J);
            } else if (J.its >= J.o.maxit) {
                fail(NMG_ERR_NOT_CONVERGED, "maxit reached");
                job_fail(J, NMG_ERR_NOT_CONVERGED);
                job_enqueue_finish(J);
            } else {
                job_enqueue_first_cycle(J);
                if (J.phase != SolveJob::P_DONE) job_enqueue_iter(J);
            }
        }
        break;
    case SolveJob::P_CYCLE: {
        const double beta = hs[S_BETA];
        J.relres = beta / J.bnorm;
        if (!std::isfinite(beta)) {
            fail(NMG_ERR_NONFINITE, "non-finite residual");
            job_fail(J, NMG_ERR_NONFINITE);
            job_enqueue_finish(J);
        } else if (J.relres <= J.o.rtol) {
            if (J.finish_ready) {   // its copies completed with the residual: read the flags now
                J.phase = SolveJob::P_FINISH;
                job_advance(J);
            } else {
                job_enqueue_finish(J);
            }
        } else if (J.its >= J.o.maxit) {
            fail(NMG_ERR_NOT_CONVERGED, "maxit reached");
            job_fail(J, NMG_ERR_NOT_CONVERGED);
            job_enqueue_finish(J);
        } else {
            job_enqueue_iter(J);
        }
        break;
    }
    case SolveJob::P_ITER: {
        // the device counted the steps and decided whether the cycle stops
        const int* cy = h->host_cyc;
        const int k = cy[0] + 1;   // steps of this cycle
        if (J.loop) J.launches += h->cgraph_nodes[J.o.precision] * (int64_t)(cy[1] - J.its);
        J.its = cy[1];
        if (hs[S_STATUS] != 0.0) {
            fail(NMG_ERR_NONFINITE, "non-finite value in the Arnoldi process");
            job_fail(J, NMG_ERR_NONFINITE);
            job_enqueue_finish(J);
        } else if (cy[2]) {
            const Geom& g = h->lev[h->L - 1].g;
            const int64_t n = g.nodes * g.nc;
            launch_solve_update(h->scal, k, J.o.restart, h->Z, n, h->x64, n, h->stream);
            ++J.cycles;
            const bool est_converged = hs[S_EST] <= J.o.rtol;
            job_enqueue_cycle(J);
            // the estimate says converged: the true residual almost always agrees, so the
            // result and status copies go with it (one host round trip fewer; repeated
            // by the finish when the residual disagrees)
            J.finish_ready = false;
            if (est_converged && J.phase == SolveJob::P_CYCLE) {
                job_enqueue_finish(J);
                if (J.phase == SolveJob::P_FINISH) {
                    J.phase = SolveJob::P_CYCLE;
                    J.finish_ready = true;
                }
            }
        } else {
            job_enqueue_iter(J);
        }
        break;
    }
    case SolveJob::P_FINISH: {
        const int* f = h->host_flags;
        // a wait that ran out left the preconditioner's result incomplete: that is the cause of
        // whatever the iteration reported afterwards (no convergence, a non-finite norm)
        const bool overridable = J.st == NMG_OK || J.st == NMG_ERR_NOT_CONVERGED || J.st == NMG_ERR_NONFINITE;
        if (f[FLAG_COUNT]) {
            wait_timeout_clear(h->stream);
            if (overridable) {
                fail(NMG_ERR_TIMEOUT, "a bounded device wait ran out (TMA copy)");
                job_fail(J, NMG_ERR_TIMEOUT);
            }
        }
        if (f[FLAG_ABORT]) {
            cudaMemsetAsync(h->flags + FLAG_ABORT, 0, sizeof(int), h->stream);
            if (overridable || J.st == NMG_ERR_TIMEOUT) {
                fail(NMG_ERR_TIMEOUT, "the persistent V-cycle aborted (grid barrier or copy wait ran out)");
                job_fail(J, NMG_ERR_TIMEOUT);
            }
        }
        J.phase = SolveJob::P_DONE;
        break;
    }
    default:
        J.phase = SolveJob::P_DONE;
        break;
    }
}

static void job_info(const SolveJob& J, nmg_solve_info* info) {
    if (!info) return;
    info->iterations = J.its;
    info->restarts = J.cycles > 0 ? J.cycles - 1 : 0;
    info->rel_residual = J.relres;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - J.t0).count();
    info->status = J.st;
    info->launches = J.launches;
    info->engine = J.engine;
    info->device_loop = J.used_loop ? 1 : 0;
}

static nmg_status solve_impl(Hierarchy* h, const double* b_user, double* x_user, const nmg_solve_opts& o,
                             nmg_solve_info* info) {
    SolveJob J;
    NMG_TRY(job_start(J, h, b_user, x_user, o));
    while (J.phase != SolveJob::P_DONE) {
        NMG_CK(cudaStreamSynchronize(h->stream));
        const int64_t l0 = g_launches;
        job_advance(J);
        J.launches += g_launches - l0;
    }
    NMG_CK(cudaGetLastError());
    if (J.st != NMG_OK) g_last_error = J.err;
    job_info(J, info);
    return J.st;
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
    o->use_graph = 2;
    o->engine = NMG_ENGINE_AUTO;
    o->tail_patches = 0;
    o->tile_patches = 0;
    return NMG_OK;
}

static void free_all(Hierarchy* h) {
    for (Hierarchy* c : h->many_ws) {
        cudaStreamSynchronize(c->stream);
        free_all(c);
        delete c;
    }
    h->many_ws.clear();
    for (int p = 0; p < 3; ++p) {
        if (h->vgraph[p]) cudaGraphExecDestroy(h->vgraph[p]);
        if (h->cgraph[p]) cudaGraphExecDestroy(h->cgraph[p]);
        for (int k = 0; k < 2; ++k)
            if (h->mgraph[p][k]) cudaGraphExecDestroy(h->mgraph[p][k]);
    }
    for (void* a : h->allocs) cudaFree(a);
    h->allocs.clear();
    if (h->host_scal) cudaFreeHost(h->host_scal);
    if (h->host_flags) cudaFreeHost(h->host_flags);
    if (h->host_cyc) cudaFreeHost(h->host_cyc);
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    if (h->desc.stream == nullptr && h->stream) cudaStreamDestroy(h->stream);
}

// The work buffers of one solve on h: V-cycle vectors and per-patch
// corrections of every level and precision (FP32 and BF16 share the float
// ones), the FGMRES workspace on the finest level (the Krylov bases come later,
// sized by the restart length), the device scalars and flags, and their pinned
// host mirrors.  The operator (matrices, masks, inverses) is allocated apart.
static nmg_status alloc_workspace(Hierarchy* h) {
    nmg_status st;
    const bool low = (h->prec_mask & ((1 << NMG_PREC_FP32) | (1 << NMG_PREC_BF16))) != 0;
    for (int l = 0; l < h->L; ++l) {
        Level& Lv = h->lev[l];
        const Geom& g = Lv.g;
        const int64_t nvec = g.nodes * g.nc;
        void* fvec[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        if (low) {
            for (int q = 0; q < 3; ++q)
                if ((st = dalloc(h, &fvec[q], nvec * sizeof(float))) != NMG_OK) return st;
            if ((st = dalloc(h, &fvec[4], nvec * sizeof(float))) != NMG_OK) return st;
            for (int q : {3, 5})
                if (l > 0 && (st = dalloc(h, &fvec[q], (size_t)g.patches * g.np * sizeof(float))) != NMG_OK) return st;
        }
        for (int p = 0; p < 3; ++p) {
            if (!(h->prec_mask & (1 << p))) continue;
            PrecData& P = Lv.p[p];
            if (p == NMG_PREC_FP64) {
                for (void** q : {&P.b, &P.x, &P.r, &P.x2})
                    if ((st = dalloc(h, q, nvec * sizeof(double))) != NMG_OK) return st;
                for (void** q : {&P.corr, &P.corr2})
                    if (l > 0 && (st = dalloc(h, q, (size_t)g.patches * g.np * sizeof(double))) != NMG_OK) return st;
            } else {
                P.b = fvec[0]; P.x = fvec[1]; P.r = fvec[2]; P.corr = fvec[3]; P.x2 = fvec[4]; P.corr2 = fvec[5];
            }
        }
    }
    const Geom& gf = h->lev[h->L - 1].g;
    const int64_t n = gf.nodes * gf.nc;
    for (double** q : {&h->b64, &h->x64, &h->w64})
        if ((st = dalloc(h, (void**)q, n * sizeof(double))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->partial, (size_t)(kMaxRestart + 2) * kDotBlocks * sizeof(double))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->scal, S_COUNT * sizeof(double))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->flags, FLAG_COUNT * sizeof(int))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->pbar, 2 * sizeof(unsigned))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->counters, 4 * sizeof(unsigned))) != NMG_OK) return st;
    if ((st = dalloc(h, (void**)&h->cyc, 4 * sizeof(int))) != NMG_OK) return st;
    if (cudaMemset(h->counters, 0, 4 * sizeof(unsigned)) != cudaSuccess) return fail(NMG_ERR_CUDA, "memset");
    if (cudaMemset(h->flags, 0, FLAG_COUNT * sizeof(int)) != cudaSuccess) return fail(NMG_ERR_CUDA, "memset");
    if (cudaMemset(h->pbar, 0, 2 * sizeof(unsigned)) != cudaSuccess) return fail(NMG_ERR_CUDA, "memset");
    if (cudaMallocHost((void**)&h->host_scal, 16 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&h->host_flags, (FLAG_COUNT + 1) * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&h->host_cyc, 4 * sizeof(int)) != cudaSuccess)
        return fail(NMG_ERR_OOM, "pinned host allocation failed");
    return NMG_OK;
}

// A second solve workspace for base: its own work buffers and stream, and
// base's matrices, masks, patch inverses and coarse inverse (read-only during
// solves), so that two requests on one hierarchy run at the same time with the
// same kernels on the same data (bitwise the same results).  budget: bytes the
// workspace may take (0 = unlimited).  The autotuner's choices are copied.
static nmg_status mixed_alloc(Hierarchy* h, Mixed& M, void** p, size_t bytes);

static nmg_status clone_workspace(Hierarchy* base, size_t budget, Hierarchy** out) {
    *out = nullptr;
    auto* h = new nmg_hierarchy();
    h->desc = base->desc;
    h->desc.stream = nullptr;
    h->desc.mem_budget_bytes = budget;
    h->dim = base->dim;
    h->nc = base->nc;
    h->L = base->L;
    h->prec_mask = base->prec_mask;
    h->n0 = base->n0;
    h->coarse_inv = base->coarse_inv;
    for (int l = 0; l < h->L; ++l) {
        Level& Lv = h->lev[l];
        const Level& B = base->lev[l];
        Lv.g = B.g;
        Lv.ready = B.ready;
        Lv.A64 = B.A64;
        Lv.mask = B.mask;
        for (int p = 0; p < 3; ++p) {
            Lv.p[p].A = B.p[p].A;
            Lv.p[p].inv = B.p[p].inv;
            Lv.p[p].inv_stride = B.p[p].inv_stride;
        }
        if (B.mixed.on) {   // the layout and large inverses are shared; the corrections are the clone's own
            Mixed& M = Lv.mixed;
            M.on = true;
            M.nsmall = B.mixed.nsmall;
            M.nlarge = B.mixed.nlarge;
            M.np_large = B.mixed.np_large;
            M.small_id = B.mixed.small_id;
            M.large_org = B.mixed.large_org;
            M.inc = B.mixed.inc;
            M.inc_n = B.mixed.inc_n;
            for (int p = 0; p < 3; ++p) {
                M.inv_large[p] = B.mixed.inv_large[p];
                M.stride_large[p] = B.mixed.stride_large[p];
            }
        }
    }
    h->mixed_any = base->mixed_any;
    for (int p = 0; p < 3; ++p) {
        h->engine_choice[p] = base->engine_choice[p];
        h->auto_tail[p] = base->auto_tail[p];
        h->auto_tile[p] = base->auto_tile[p];
        h->tail_patches[p] = base->tail_patches[p];
        h->tile_patches[p] = base->tile_patches[p];
        h->fused[p] = base->fused[p];
        std::memcpy(h->engine_key[p], base->engine_key[p], sizeof(h->engine_key[p]));
    }
    h->loop_mode = base->loop_mode;
    nmg_status st = NMG_OK;
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
        st = fail(NMG_ERR_CUDA, "stream creation failed");
    if (st == NMG_OK) st = alloc_workspace(h);
    for (int l = 1; l < h->L && st == NMG_OK; ++l) {
        Mixed& M = h->lev[l].mixed;
        if (!M.on) continue;
        const size_t n = (size_t)M.nlarge * M.np_large;
        if (h->prec_mask & 1) st = mixed_alloc(h, M, &M.corr_large[0], n * sizeof(double));
        if (st == NMG_OK && (h->prec_mask & 6)) st = mixed_alloc(h, M, &M.corr_large[1], n * sizeof(float));
    }
    if (st != NMG_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return NMG_OK;
}

// ---------------------------------------------------------------------------
// Multi-vector solves: FGMRES per column, each on its own workspace (column 0
// on h, the others on workspace clones of h that share its operator), all on
// h's stream and stepped in lockstep by the host: after each host round the
// columns that wait for a preconditioner application get one multi-vector
// V-cycle together, then each column's Arnoldi step.  A column's kernels and
// their order are those of a host-stepped nmg_solve with the per-step
// V-cycle engine, so each column's solution and iteration count equal a
// single solve's bit for bit.
// ---------------------------------------------------------------------------
static nmg_status many_workspaces(Hierarchy* h, int cols) {
    while ((int)h->many_ws.size() < cols - 1) {
        Hierarchy* c = nullptr;
        NMG_TRY(clone_workspace(h, h->desc.mem_budget_bytes, &c));
        h->many_ws.push_back(c);
    }
    // the operator may have been set again since the clones were made
    for (Hierarchy* c : h->many_ws) {
        c->coarse_inv = h->coarse_inv;
        c->n0 = h->n0;
        for (int l = 0; l < h->L; ++l) {
            c->lev[l].ready = h->lev[l].ready;
            c->lev[l].A64 = h->lev[l].A64;
            c->lev[l].mask = h->lev[l].mask;
            for (int p = 0; p < 3; ++p) {
                c->lev[l].p[p].A = h->lev[l].p[p].A;
                c->lev[l].p[p].inv = h->lev[l].p[p].inv;
                c->lev[l].p[p].inv_stride = h->lev[l].p[p].inv_stride;
            }
        }
    }
    return NMG_OK;
}

static nmg_status solve_group(Hierarchy* h, int ncols, const double* const* b, double* const* x,
                              const nmg_solve_opts& o, nmg_solve_info* info) {
    NMG_TRY(many_workspaces(h, ncols));
    Hierarchy* ws[kMaxCols];
    cudaStream_t own[kMaxCols];
    SolveJob J[kMaxCols];
    nmg_solve_opts oc = o;
    oc.engine = NMG_ENGINE_KERNELS;   // the columns' own V-cycles are never launched
    oc.tail_patches = 0;
    oc.tile_patches = 0;
    for (int k = 0; k < ncols; ++k) {
        ws[k] = k == 0 ? h : h->many_ws[k - 1];
        own[k] = ws[k]->stream;
        ws[k]->stream = h->stream;
    }
    nmg_status st = NMG_OK;
    int started = 0;
    for (; started < ncols; ++started) {
        st = job_start(J[started], ws[started], b[started], x[started], oc);
        if (st != NMG_OK) break;
        J[started].grouped = true;
    }
    while (st == NMG_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { st = fail(NMG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e)); break; }
        int want[kMaxCols], nw = 0;
        bool live = false;
        for (int k = 0; k < started; ++k) {
            if (J[k].phase == SolveJob::P_DONE) continue;
            job_advance(J[k]);
            if (J[k].phase == SolveJob::P_WANT) want[nw++] = k;
            live = live || J[k].phase != SolveJob::P_DONE;
        }
        if (!live) break;
        if (nw == 0) continue;
        ColPtrs in{};
        ColPtrsOut out{};
        for (int q = 0; q < nw; ++q) {
            const PrecData& P = ws[want[q]]->lev[h->L - 1].p[o.precision];
            in.p[q] = (const float*)P.b;
            out.p[q] = (float*)P.x;
        }
        st = vcycle_cols(h, o, nw, in, out);
        for (int q = 0; q < nw && st == NMG_OK; ++q) {
            SolveJob& Jk = J[want[q]];
            Hierarchy* w = ws[want[q]];
            enqueue_arnoldi(w, Jk.o, false, 0);
            cudaMemcpyAsync(w->host_scal, w->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            cudaMemcpyAsync(w->host_cyc, w->cyc, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
            Jk.phase = SolveJob::P_ITER;
        }
    }
    // a bounded wait of the multi-vector apply that ran out fails every column
    int abort_flag = 0;
    cudaStreamSynchronize(h->stream);
    if (cudaMemcpy(&abort_flag, h->flags + FLAG_MANY, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
        abort_flag) {
        cudaMemset(h->flags + FLAG_MANY, 0, sizeof(int));
        fail(NMG_ERR_TIMEOUT, "a bounded device wait of the multi-vector apply ran out");
        for (int k = 0; k < started; ++k) job_fail(J[k], NMG_ERR_TIMEOUT);
    }
    for (int k = 0; k < ncols; ++k) ws[k]->stream = own[k];
    nmg_status first = st;
    for (int k = 0; k < ncols; ++k) {
        if (k >= started || st != NMG_OK) {
            J[k].st = st != NMG_OK ? st : NMG_ERR_INVALID;
            J[k].phase = SolveJob::P_DONE;
        }
        if (first == NMG_OK && J[k].st != NMG_OK) {
            first = J[k].st;
            g_last_error = J[k].err;
        }
        job_info(J[k], info ? info + k : nullptr);
    }
    return first;
}

nmg_status nmg_create_hierarchy(const nmg_mesh_desc* d, nmg_hierarchy** out) {
    if (!d || !out) return fail(NMG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return fail(NMG_ERR_INVALID, "dim must be 2 or 3");
    if (d->ncomp != d->dim + 1 && d->ncomp != d->dim) return fail(NMG_ERR_INVALID, "ncomp must be dim + 1 or dim");
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
    for (int l = 0; l < L; ++l) h->lev[l].g = make_geom(d->dim, d->ncomp, cells[l]);
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
    for (int l = 0; l < L; ++l) {   // the operator: matrices, masks, patch inverses
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
        for (int p = 0; p < 3; ++p) {
            if (!(h->prec_mask & (1 << p))) continue;
            PrecData& P = Lv.p[p];
            P.A = p == NMG_PREC_FP64 ? (void*)Lv.A64 : (void*)A32;
            if (l > 0) {
                P.inv_stride = pad16((int64_t)g.np * g.np, store_size(p));
                if ((st = dalloc(h, &P.inv, (size_t)g.patches * P.inv_stride * store_size(p))) != NMG_OK) return cleanup(st);
            }
        }
    }
    if ((st = dalloc(h, (void**)&h->coarse_inv, (size_t)h->n0 * h->n0 * sizeof(double))) != NMG_OK) return cleanup(st);
    if ((st = alloc_workspace(h)) != NMG_OK) return cleanup(st);
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
    for (const Hierarchy* c : h->many_ws) *bytes += c->bytes;
    return NMG_OK;
}

}  // extern "C"

// Copies a level's BSR matrix (host or device arrays) into the stencil layout
// dst (FP64, zero where the pattern has no block) and checks its pattern and
// values on the device.
static nmg_status load_stencil(Hierarchy* h, const Geom& g, int64_t nrows_blk, int64_t nnzb, const int64_t* row_ptr,
                               const int32_t* col_idx, const double* vals, int ptr_location, double* dst) {
    if (!row_ptr || (nnzb > 0 && (!col_idx || !vals))) return fail(NMG_ERR_INVALID, "NULL argument");
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
    cudaMemsetAsync(dst, 0, mat * sizeof(double), s);
    launch_bsr_to_stencil(g, d_rp, d_ci, d_v, nnzb, dst, h->flags, s);
    nmg_status st = check_flags(h);
    release();
    return st;
}

// ---- patches of two sizes (Section 5.5.1)

static void dfree(Hierarchy* h, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
        if (*it == p) {
            h->allocs.erase(it);
            break;
        }
    h->bytes -= bytes;
}

static nmg_status mixed_alloc(Hierarchy* h, Mixed& M, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    NMG_TRY(dalloc(h, p, bytes));
    M.owned.emplace_back(*p, bytes);
    return NMG_OK;
}

static void release_mixed(Hierarchy* h, Mixed& M) {
    for (auto& a : M.owned) dfree(h, a.first, a.second);
    M = Mixed();
}

// The patch layout of level l for the flagged cells cmask (x fastest): large
// patches on the 4-aligned blocks of 4^d cells that are all flagged, small
// patches on the other 2-aligned blocks of 2^d cells, and the per-node
// incidence of both.  No large block: the level keeps its single patch size.
static nmg_status build_mixed(Hierarchy* h, int l, const std::vector<uint8_t>& cmask) {
    Level& Lv = h->lev[l];
    const Geom& g = Lv.g;
    Mixed& M = Lv.mixed;
    const int d = g.dim;
    const int64_t c0 = g.cells[0], c1 = g.cells[1];
    std::vector<uint8_t> covered(g.patches, 0);
    std::vector<int32_t> large, small;
    const int zb = d == 3 ? g.cells[2] : 1;
    for (int bz = 0; d == 2 ? bz == 0 : bz + 4 <= zb; bz += 4)
        for (int by = 0; by + 4 <= g.cells[1]; by += 4)
            for (int bx = 0; bx + 4 <= g.cells[0]; bx += 4) {
                bool all = true;
                for (int z = bz; z < (d == 3 ? bz + 4 : 1) && all; ++z)
                    for (int y = by; y < by + 4 && all; ++y)
                        for (int x = bx; x < bx + 4 && all; ++x) all = cmask[x + c0 * (y + c1 * z)] != 0;
                if (!all) continue;
                const int64_t px = bx / 2, py = by / 2, pz = bz / 2;
                large.push_back((int32_t)(px + g.pc[0] * (py + (int64_t)g.pc[1] * pz)));
                for (int k = 0; k < (d == 3 ? 2 : 1); ++k)
                    for (int j = 0; j < 2; ++j)
                        for (int i = 0; i < 2; ++i)
                            covered[(px + i) + g.pc[0] * ((py + j) + (int64_t)g.pc[1] * (pz + k))] = 1;
            }
    if (large.empty()) return NMG_OK;
    for (int64_t q = 0; q < g.patches; ++q)
        if (!covered[q]) small.push_back((int32_t)q);
    const int nc = g.nc, nps = g.np;
    const int npl = (d == 2 ? 25 : 125) * nc;
    if ((double)small.size() * nps + (double)large.size() * npl >= 2147483647.0)
        return fail(NMG_ERR_INVALID, "too many patch unknowns on a level for the incidence table");
    std::vector<int32_t> inc((size_t)g.nodes * kIncMax, -1);
    std::vector<uint8_t> inc_n(g.nodes, 0);
    auto add = [&](int64_t node, int64_t off) -> bool {
        uint8_t& n = inc_n[node];
        if (n >= kIncMax) return false;
        inc[node * kIncMax + n++] = (int32_t)off;
        return true;
    };
    const int64_t n0 = g.nn[0], n1 = g.nn[1];
    bool ok = true;
    for (size_t k = 0; k < small.size() && ok; ++k) {
        const int64_t q = small[k];
        const int64_t px = q % g.pc[0], py = (q / g.pc[0]) % g.pc[1], pz = q / ((int64_t)g.pc[0] * g.pc[1]);
        for (int an = 0; an < (d == 2 ? 9 : 27) && ok; ++an) {
            const int ax = an % 3, ay = (an / 3) % 3, az = an / 9;
            ok = add((2 * px + ax) + n0 * ((2 * py + ay) + n1 * (2 * pz + az)), (int64_t)k * nps + (int64_t)an * nc);
        }
    }
    const int64_t base = (int64_t)small.size() * nps;
    for (size_t m = 0; m < large.size() && ok; ++m) {
        const int64_t q = large[m];
        const int64_t px = q % g.pc[0], py = (q / g.pc[0]) % g.pc[1], pz = q / ((int64_t)g.pc[0] * g.pc[1]);
        for (int an = 0; an < (d == 2 ? 25 : 125) && ok; ++an) {
            const int ax = an % 5, ay = (an / 5) % 5, az = an / 25;
            ok = add((2 * px + ax) + n0 * ((2 * py + ay) + n1 * (2 * pz + az)),
                     base + (int64_t)m * npl + (int64_t)an * nc);
        }
    }
    if (!ok) return fail(NMG_ERR_INVALID, "a node lies in more patches than the incidence table holds");
    M.nsmall = (int64_t)small.size();
    M.nlarge = (int64_t)large.size();
    M.np_large = npl;
    NMG_TRY(mixed_alloc(h, M, (void**)&M.small_id, small.size() * sizeof(int32_t)));
    NMG_TRY(mixed_alloc(h, M, (void**)&M.large_org, large.size() * sizeof(int32_t)));
    NMG_TRY(mixed_alloc(h, M, (void**)&M.inc, inc.size() * sizeof(int32_t)));
    NMG_TRY(mixed_alloc(h, M, (void**)&M.inc_n, inc_n.size()));
    NMG_CK(cudaMemcpy(M.small_id, small.data(), small.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    NMG_CK(cudaMemcpy(M.large_org, large.data(), large.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    NMG_CK(cudaMemcpy(M.inc, inc.data(), inc.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    NMG_CK(cudaMemcpy(M.inc_n, inc_n.data(), inc_n.size(), cudaMemcpyHostToDevice));
    for (int p = 0; p < 3; ++p) {
        if (!(h->prec_mask & (1 << p))) continue;
        M.stride_large[p] = pad16((int64_t)npl * npl, store_size(p));
        NMG_TRY(mixed_alloc(h, M, &M.inv_large[p], (size_t)M.nlarge * M.stride_large[p] * store_size(p)));
    }
    if (h->prec_mask & 1) NMG_TRY(mixed_alloc(h, M, &M.corr_large[0], (size_t)M.nlarge * npl * sizeof(double)));
    if (h->prec_mask & 6) NMG_TRY(mixed_alloc(h, M, &M.corr_large[1], (size_t)M.nlarge * npl * sizeof(float)));
    M.on = true;
    return NMG_OK;
}

// Extracts and inverts every patch matrix of level l >= 1 from its FP64
// stencil matrix, in the level's patch layout (one size, or two sizes with
// the small patches listed), storing the inverses in every prepared precision.
static nmg_status factor_patches(Hierarchy* h, int l) {
    Level& Lv = h->lev[l];
    const Geom& g = Lv.g;
    cudaStream_t s = h->stream;
    PrecData* P = Lv.p;
    const bool p64 = h->prec_mask & 1, p32 = h->prec_mask & 2, pbf = h->prec_mask & 4;
    const Mixed& M = Lv.mixed;
    NMG_CK(launch_patch_invert(g, Lv.A64, p64 ? (double*)P[0].inv : nullptr, P[0].inv_stride,
                               p32 ? (float*)P[1].inv : nullptr, P[1].inv_stride,
                               pbf ? (__nv_bfloat16*)P[2].inv : nullptr, P[2].inv_stride, h->flags, s,
                               M.on ? M.nsmall : -1, M.on ? M.small_id : nullptr));
    if (M.on)
        NMG_CK(launch_patch_invert_large(g, Lv.A64, M.large_org, M.nlarge,
                                         p64 ? (double*)M.inv_large[0] : nullptr, M.stride_large[0],
                                         p32 ? (float*)M.inv_large[1] : nullptr, M.stride_large[1],
                                         pbf ? (__nv_bfloat16*)M.inv_large[2] : nullptr, M.stride_large[2],
                                         h->flags, s));
    return NMG_OK;
}

extern "C" {

nmg_status nmg_set_jacobian(nmg_hierarchy* h, int level, int64_t nrows_blk, int64_t nnzb, const int64_t* row_ptr,
                            const int32_t* col_idx, const double* vals, int ptr_location) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL argument");
    if (level < 0 || level >= h->L) return fail(NMG_ERR_INVALID, "level out of range");
    Level& Lv = h->lev[level];
    const Geom& g = Lv.g;
    NMG_TRY(load_stencil(h, g, nrows_blk, nnzb, row_ptr, col_idx, vals, ptr_location, Lv.A64));
    cudaStream_t s = h->stream;
    const size_t mat = (size_t)g.nst * g.nc * g.nc * g.ld;
    const bool low = (h->prec_mask & 6) != 0;
    if (low) {
        void* A32 = Lv.p[(h->prec_mask & 2) ? NMG_PREC_FP32 : NMG_PREC_BF16].A;
        launch_convert_f64_f32(Lv.A64, (float*)A32, (int64_t)mat, s);
    }
    if (level > 0) {
        NMG_TRY(factor_patches(h, level));
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
    int timed_out = 0;
    NMG_CK(wait_timeout_flag(&timed_out, h->stream));
    if (timed_out) return fail(NMG_ERR_TIMEOUT, "a bounded device wait ran out (TMA copy)");
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
    NMG_TRY(vcycle_any(h, *opts, r, z, false));
    NMG_TRY(finish_op(h));
    int f[FLAG_COUNT];
    NMG_CK(cudaMemcpy(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (f[FLAG_ABORT]) {
        cudaMemset(h->flags + FLAG_ABORT, 0, sizeof(int));
        return fail(NMG_ERR_TIMEOUT, "the persistent V-cycle aborted (grid barrier or copy wait ran out)");
    }
    return NMG_OK;
}

nmg_status nmg_vcycle_many(nmg_hierarchy* h, const nmg_solve_opts* opts, int nrhs, const void* r, void* z) {
    if (!h || !r || !z || nrhs < 1) return fail(NMG_ERR_INVALID, "NULL argument or nrhs < 1");
    NMG_TRY(validate_opts(opts));
    NMG_TRY(check_ready(h, opts->precision));
    NMG_TRY(check_many(h, *opts));
    enter(h);
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    for (int c0 = 0; c0 < nrhs; c0 += kMaxCols) {
        const int nc = std::min(kMaxCols, nrhs - c0);
        ColPtrs in{};
        ColPtrsOut out{};
        for (int k = 0; k < nc; ++k) {
            in.p[k] = (const float*)r + (int64_t)(c0 + k) * n;
            out.p[k] = (float*)z + (int64_t)(c0 + k) * n;
        }
        NMG_TRY(vcycle_cols(h, *opts, nc, in, out));
    }
    NMG_TRY(finish_op(h));
    int f[FLAG_COUNT];
    NMG_CK(cudaMemcpy(f, h->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (f[FLAG_MANY]) {
        cudaMemset(h->flags + FLAG_MANY, 0, sizeof(int));
        return fail(NMG_ERR_TIMEOUT, "a bounded device wait of the multi-vector apply ran out");
    }
    return NMG_OK;
}

nmg_status nmg_solve_many(nmg_hierarchy* h, int nrhs, const double* b, double* x, const nmg_solve_opts* opts,
                          nmg_solve_info* info) {
    if (!h || !b || !x || nrhs < 1) return fail(NMG_ERR_INVALID, "NULL argument or nrhs < 1");
    NMG_TRY(validate_opts(opts));
    NMG_TRY(check_ready(h, opts->precision));
    NMG_TRY(check_many(h, *opts));
    enter(h);
    const Geom& g = h->lev[h->L - 1].g;
    const int64_t n = g.nodes * g.nc;
    nmg_status first = NMG_OK;
    std::string err;
    for (int c0 = 0; c0 < nrhs; c0 += kMaxCols) {
        const int nc = std::min(kMaxCols, nrhs - c0);
        const double* bp[kMaxCols];
        double* xp[kMaxCols];
        for (int k = 0; k < nc; ++k) {
            bp[k] = b + (int64_t)(c0 + k) * n;
            xp[k] = x + (int64_t)(c0 + k) * n;
        }
        const nmg_status st = solve_group(h, nc, bp, xp, *opts, info ? info + c0 : nullptr);
        if (st != NMG_OK && first == NMG_OK) {
            first = st;
            err = g_last_error;
        }
        if (st == NMG_ERR_CUDA || st == NMG_ERR_OOM) break;
    }
    if (first != NMG_OK) g_last_error = err;
    return first;
}

nmg_status nmg_get_patch_inverses(nmg_hierarchy* h, int level, int prec, int64_t first, int64_t count, double* out) {
    NMG_TRY(op_check(h, level, prec, true));
    const Geom& g = h->lev[level].g;
    const Mixed& M = h->lev[level].mixed;
    const int64_t ns = M.on ? M.nsmall : g.patches, total = M.on ? M.nsmall + M.nlarge : g.patches;
    if (first < 0 || count < 0 || first + count > total || (count && !out))
        return fail(NMG_ERR_INVALID, "patch range out of bounds");
    const bool large = M.on && first >= ns;
    if (count && M.on && first < ns && first + count > ns)
        return fail(NMG_ERR_INVALID, "a patch range holds patches of one size only");
    enter(h);
    const PrecData& P = h->lev[level].p[prec];
    const void* base = large ? M.inv_large[prec] : P.inv;
    const int64_t stride = large ? M.stride_large[prec] : P.inv_stride;
    const int64_t k0 = large ? first - ns : first;
    const size_t es = store_size(prec);
    std::vector<unsigned char> buf((size_t)count * stride * es);
    NMG_CK(cudaMemcpyAsync(buf.data(), (const unsigned char*)base + (size_t)k0 * stride * es, buf.size(),
                           cudaMemcpyDeviceToHost, h->stream));
    NMG_CK(cudaStreamSynchronize(h->stream));
    const int np = large ? M.np_large : g.np;
    for (int64_t p = 0; p < count; ++p)
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
                const size_t idx = (size_t)p * stride + (size_t)j * np + i;
                double v;
                if (prec == NMG_PREC_FP64) v = ((const double*)buf.data())[idx];
                else if (prec == NMG_PREC_FP32) v = ((const float*)buf.data())[idx];
                else v = __bfloat162float(((const __nv_bfloat16*)buf.data())[idx]);
                out[(size_t)p * np * np + (size_t)i * np + j] = v;
            }
    return NMG_OK;
}

nmg_status nmg_patch_layout(nmg_hierarchy* h, int level, int64_t* nsmall, int64_t* nlarge, int* np_small,
                            int* np_large) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (level < 1 || level >= h->L) return fail(NMG_ERR_INVALID, "level out of range (the coarsest has no patches)");
    const Geom& g = h->lev[level].g;
    const Mixed& M = h->lev[level].mixed;
    if (nsmall) *nsmall = M.on ? M.nsmall : g.patches;
    if (nlarge) *nlarge = M.on ? M.nlarge : 0;
    if (np_small) *np_small = g.np;
    if (np_large) *np_large = (g.dim == 2 ? 25 : 125) * g.nc;
    return NMG_OK;
}

// ---- problems (2) and (3) of Section 4.2 around the momentum solve

nmg_status nmg_set_large_patches(nmg_hierarchy* h, const uint8_t* cell_mask) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (!h->many_ws.empty()) return fail(NMG_ERR_INVALID, "set the patch layout before multi-vector solves");
    enter(h);
    NMG_CK(cudaStreamSynchronize(h->stream));
    for (int l = 1; l < h->L; ++l) release_mixed(h, h->lev[l].mixed);
    h->mixed_any = false;
    nmg_status st = NMG_OK;
    if (cell_mask) {
        const Geom& gf = h->lev[h->L - 1].g;
        auto cz = [&](const Geom& q) { return (size_t)(h->dim == 3 ? q.cells[2] : 1); };   // cells[2] is 0 in 2d
        std::vector<uint8_t> m(cell_mask, cell_mask + (size_t)gf.cells[0] * gf.cells[1] * cz(gf));
        for (int l = h->L - 1; l >= 1 && st == NMG_OK; --l) {
            st = build_mixed(h, l, m);
            h->mixed_any = h->mixed_any || h->lev[l].mixed.on;
            // the next coarser level: a cell is flagged iff all its children are
            const Geom& g = h->lev[l].g;
            const Geom& c = h->lev[l - 1].g;
            std::vector<uint8_t> cm((size_t)c.cells[0] * c.cells[1] * cz(c));
            for (int z = 0; z < (int)cz(c); ++z)
                for (int y = 0; y < c.cells[1]; ++y)
                    for (int x = 0; x < c.cells[0]; ++x) {
                        bool all = true;
                        for (int k = 0; k < (h->dim == 3 ? 2 : 1); ++k)
                            for (int j = 0; j < 2; ++j)
                                for (int i = 0; i < 2; ++i)
                                    all = all && m[(2 * x + i) + (size_t)g.cells[0] * ((2 * y + j) +
                                                                   (size_t)g.cells[1] * (2 * z + k))];
                        cm[x + (size_t)c.cells[0] * (y + (size_t)c.cells[1] * z)] = all;
                    }
            m.swap(cm);
        }
    }
    if (st != NMG_OK) {
        for (int l = 1; l < h->L; ++l) release_mixed(h, h->lev[l].mixed);
        h->mixed_any = false;
    }
    // graphs and engine choices were made for the old layout
    for (int p = 0; p < 3; ++p) {
        if (h->vgraph[p]) { cudaGraphExecDestroy(h->vgraph[p]); h->vgraph[p] = nullptr; }
        if (h->cgraph[p]) { cudaGraphExecDestroy(h->cgraph[p]); h->cgraph[p] = nullptr; }
        h->engine_choice[p] = 0;
    }
    // refactor the levels already set, in the new layout
    for (int l = 1; l < h->L && st == NMG_OK; ++l)
        if (h->lev[l].ready) {
            st = factor_patches(h, l);
            if (st == NMG_OK) st = check_flags(h);
        }
    return st;
}

nmg_status nmg_set_lifting_operator(nmg_hierarchy* h, int64_t nrows_blk, int64_t nnzb, const int64_t* row_ptr,
                                    const int32_t* col_idx, const double* vals, int ptr_location) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (h->nc != h->dim) return fail(NMG_ERR_INVALID, "the lifting operator belongs to an extension hierarchy (ncomp = dim)");
    const Geom& g = h->lev[h->L - 1].g;
    if (!h->lift64) NMG_TRY(dalloc(h, (void**)&h->lift64, (size_t)g.nst * g.nc * g.nc * g.ld * sizeof(double)));
    h->lift_ready = false;
    NMG_TRY(load_stencil(h, g, nrows_blk, nnzb, row_ptr, col_idx, vals, ptr_location, h->lift64));
    h->lift_ready = true;
    return NMG_OK;
}

// Work vectors of the sub-steps on an extension hierarchy (finest level).
static nmg_status ensure_substep_buffers(Hierarchy* h) {
    const Geom& g = h->lev[h->L - 1].g;
    for (double*& v : h->sub_vec)
        if (!v) NMG_TRY(dalloc(h, (void**)&v, (size_t)g.nodes * g.nc * sizeof(double)));
    if (!h->sub_nodes) NMG_TRY(dalloc(h, (void**)&h->sub_nodes, (size_t)g.nodes));
    return NMG_OK;
}

static nmg_status check_extension(Hierarchy* h) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (h->nc != h->dim) return fail(NMG_ERR_INVALID, "an extension hierarchy (ncomp = dim) is required");
    if (!h->lev[h->L - 1].ready) return fail(NMG_ERR_INVALID, "finest level matrix not set");
    return NMG_OK;
}

nmg_status nmg_deformation_update(nmg_hierarchy* h, const double* r, const double* dv, double k_theta,
                                  const uint8_t* update_nodes, double* du) {
    NMG_TRY(check_extension(h));
    if (!r || !dv || !update_nodes || !du) return fail(NMG_ERR_INVALID, "NULL argument");
    if (!std::isfinite(k_theta)) return fail(NMG_ERR_INVALID, "k_theta must be finite");
    enter(h);
    const Geom& g = h->lev[h->L - 1].g;
    launch_deformation_update(h->dim, g.nodes, r, dv, k_theta, update_nodes, du, h->stream);
    return finish_op(h);
}

nmg_status nmg_extension_rhs(nmg_hierarchy* h, const double* b5, const double* gv, double* rhs) {
    NMG_TRY(check_extension(h));
    if (!b5 || !gv || !rhs) return fail(NMG_ERR_INVALID, "NULL argument");
    if (!h->lift_ready) return fail(NMG_ERR_INVALID, "lifting operator not set (nmg_set_lifting_operator)");
    enter(h);
    const Level& F = h->lev[h->L - 1];
    launch_extension_rhs(F.g, h->lift64, F.mask, b5, gv, rhs, h->stream);
    return finish_op(h);
}

nmg_status nmg_newton_substeps(nmg_hierarchy* h1, nmg_hierarchy* h3, const double* b1, const double* r, double k_theta,
                               const uint8_t* update_nodes, const double* b5, double* dw, double* du,
                               const nmg_solve_opts* opts1, const nmg_solve_opts* opts3, nmg_solve_info* info1,
                               nmg_solve_info* info3) {
    if (!h1 || !b1 || !r || !update_nodes || !b5 || !dw || !du) return fail(NMG_ERR_INVALID, "NULL argument");
    NMG_TRY(check_extension(h3));
    if (h1->nc != h1->dim + 1) return fail(NMG_ERR_INVALID, "h1 must be a condensed-momentum hierarchy (ncomp = dim + 1)");
    const Geom& g1 = h1->lev[h1->L - 1].g;
    const Geom& g3 = h3->lev[h3->L - 1].g;
    if (h1->dim != h3->dim || g1.nodes != g3.nodes || g1.nn[0] != g3.nn[0] || g1.nn[1] != g3.nn[1] ||
        g1.nn[2] != g3.nn[2])
        return fail(NMG_ERR_INVALID, "the two hierarchies must share the finest mesh");
    if (!h3->lift_ready) return fail(NMG_ERR_INVALID, "lifting operator not set (nmg_set_lifting_operator)");
    if (!std::isfinite(k_theta)) return fail(NMG_ERR_INVALID, "k_theta must be finite");
    NMG_TRY(validate_opts(opts1));
    NMG_TRY(validate_opts(opts3));
    NMG_TRY(ensure_substep_buffers(h3));
    // problem (1): the momentum solve; its FP64 solution stays in h1's iterate buffer
    nmg_status st = nmg_solve(h1, b1, dw, opts1, info1);
    if (st != NMG_OK) return st;
    enter(h3);
    cudaStream_t s = h3->stream;
    const int64_t n3 = g3.nodes * g3.nc;
    const bool r_dev = is_device_ptr(r), b5_dev = is_device_ptr(b5), f_dev = is_device_ptr(update_nodes);
    NMG_CK(cudaMemcpyAsync(h3->sub_vec[0], r, n3 * sizeof(double), r_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NMG_CK(cudaMemcpyAsync(h3->sub_vec[1], b5, n3 * sizeof(double), b5_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NMG_CK(cudaMemcpyAsync(h3->sub_nodes, update_nodes, g3.nodes, f_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    // problem (2): the deformation on the solid and interface nodes
    launch_deformation_update(h3->dim, g3.nodes, h3->sub_vec[0], h1->x64, k_theta, h3->sub_nodes, h3->sub_vec[2], s);
    // problem (3): lift it into the extension's right-hand side, then solve
    const Level& F = h3->lev[h3->L - 1];
    launch_extension_rhs(F.g, h3->lift64, F.mask, h3->sub_vec[1], h3->sub_vec[2], h3->sub_vec[3], s);
    NMG_CK(cudaGetLastError());
    return nmg_solve(h3, h3->sub_vec[3], du, opts3, info3);
}

// ---- Jacobian reuse (Section 5.3)

nmg_status nmg_jacobian_reuse_init(nmg_jacobian_reuse* m, double gamma) {
    if (!m || !(gamma >= 0.0) || !std::isfinite(gamma)) return fail(NMG_ERR_INVALID, "NULL monitor or gamma not >= 0");
    std::memset(m, 0, sizeof(*m));
    m->gamma = gamma;
    return NMG_OK;
}

nmg_status nmg_jacobian_reuse_time_step(nmg_jacobian_reuse* m) {
    if (!m) return fail(NMG_ERR_INVALID, "NULL monitor");
    m->have_last = 0;
    return NMG_OK;
}

nmg_status nmg_jacobian_reuse_decide(nmg_jacobian_reuse* m, double residual_inf, int* assemble) {
    if (!m || !assemble) return fail(NMG_ERR_INVALID, "NULL argument");
    if (!(residual_inf >= 0.0) || !std::isfinite(residual_inf)) return fail(NMG_ERR_NONFINITE, "residual norm not finite");
    int a;
    if (!m->have_jacobian) {
        a = 1;                                   // nothing to reuse yet
        m->rate = -1.0;
    } else if (m->have_last) {
        m->rate = m->last > 0.0 ? residual_inf / m->last : (residual_inf > 0.0 ? INFINITY : 0.0);
        a = m->rate > m->gamma;
    } else {
        m->rate = -1.0;                          // first step of a time step: no rate yet
        a = m->gamma == 0.0;
    }
    m->last = residual_inf;
    m->have_last = 1;
    m->steps += 1;
    if (a) {
        m->have_jacobian = 1;
        m->assemblies += 1;
    }
    *assemble = a;
    return NMG_OK;
}

nmg_status nmg_profile_enable(nmg_hierarchy* h, int enable) {
    if (!h) return fail(NMG_ERR_INVALID, "NULL hierarchy");
    if (enable && h->prof_ev.empty()) {
        h->prof_ev.resize(2 * 1024);
        for (auto& e : h->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(NMG_ERR_CUDA, "event creation failed");
    }
    if (enable < 0 || enable > 3) return fail(NMG_ERR_INVALID, "profile mode must be 0, 1, 2 or 3");
    h->prof = enable;
    h->prof_used = 0;
    h->prof_ms = 0.0;
    h->prof_launches = 0;
    h->prof_bytes = 0.0;
    return NMG_OK;
}

nmg_status nmg_autotune_report(nmg_hierarchy* h, char* buf, size_t len) {
    if (!h || !buf || len == 0) return fail(NMG_ERR_INVALID, "NULL argument");
    std::string js = "{\"choice\": [";
    for (int p = 0; p < 3; ++p) {
        js += "{\"precision\": " + std::to_string(p) + ", \"engine\": " + std::to_string(h->engine_choice[p]) +
              ", \"tail_patches\": " + std::to_string(h->auto_tail[p]) +
              ", \"tile_patches\": " + std::to_string(h->auto_tile[p]) +
              ", \"fused\": " + std::to_string(h->fused[p]) + "}";
        if (p < 2) js += ", ";
    }
    js += "], \"trials\": [";
    for (int p = 0; p < 3; ++p) {
        js += "[";
        for (size_t i = 0; i < h->tuning[p].size(); ++i) {
            const Hierarchy::Trial& t = h->tuning[p][i];
            char tmp[160];
            std::snprintf(tmp, sizeof(tmp),
                          "{\"engine\": %d, \"tail_patches\": %d, \"fused\": %d, \"tile_patches\": %d, "
                          "\"us_per_vcycle\": %.3f}",
                          t.engine, t.tail, t.fused, t.tile, t.us);
            js += tmp;
            if (i + 1 < h->tuning[p].size()) js += ", ";
        }
        js += p < 2 ? "], " : "]";
    }
    js += "], \"device_loop\": {\"mode\": " + std::to_string(h->loop_mode) + ", \"kernels_per_step\": [" +
          std::to_string(h->cgraph_nodes[0]) + ", " + std::to_string(h->cgraph_nodes[1]) + ", " +
          std::to_string(h->cgraph_nodes[2]) + "]}}";
    if (js.size() + 1 > len) return fail(NMG_ERR_INVALID, "buffer too small");
    std::memcpy(buf, js.c_str(), js.size() + 1);
    return NMG_OK;
}

nmg_status nmg_set_wait_limit(nmg_hierarchy* h, int spins) {
    if (!h || spins < 0) return fail(NMG_ERR_INVALID, "NULL hierarchy or negative limit");
    h->wait_limit = spins;
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

// ---------------------------------------------------------------------------
// Serving: continuous batching of solves on resident hierarchies.
//
// A worker thread owns all CUDA calls of the server.  Submitted requests wait
// in a FIFO; a request is admitted when a slot is free, its hierarchy is not
// running another request (a hierarchy's workspace serves one solve at a
// time) and the resident bytes of the hierarchies with running requests stay
// within the memory budget.  Running requests advance as resumable jobs on
// their hierarchies' streams: the worker enqueues a step, records an event,
// and moves a job on as soon as its event has completed, so the steps of
// different requests overlap on the device.  Every step performs the same
// kernels in the same order as nmg_solve, so a result does not depend on what
// else runs beside it.
// ---------------------------------------------------------------------------
#include <atomic>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <unordered_set>

namespace nmg {

struct Group;

struct Request {
    uint64_t ticket = 0;
    Hierarchy* h = nullptr;       // the hierarchy the request was submitted on
    Hierarchy* slot = nullptr;    // where it runs: h itself or a workspace clone of h
    Group* group = nullptr;       // the column group it runs in (batching), else null
    int col = -1;                 // its column in the group
    cudaStream_t own_stream = nullptr;   // the column workspace's own stream, restored when it leaves
    const double* b = nullptr;
    double* x = nullptr;
    nmg_solve_opts o{};
    SolveJob job;
    cudaEvent_t ev = nullptr;
    bool done = false;
    nmg_solve_info info{};
    std::string err;
    std::chrono::steady_clock::time_point t_submit;
};

// Requests on one hierarchy batched as the columns of a multi-vector solve
// (nmg_server_set_batching): column k runs on workspace k (the hierarchy, or
// its k-th column workspace), all on the hierarchy's stream; one event covers
// the group's enqueued work, and each time it completes the worker advances
// every column, runs one multi-vector V-cycle for the columns that need one
// and then their Arnoldi steps.  Columns join and leave at any round.
struct Group {
    Hierarchy* h = nullptr;
    Request* col[kMaxCols] = {};
    int n = 0;                    // occupied columns
    nmg_solve_opts vo{};          // the V-cycle options its columns share
    cudaEvent_t ev = nullptr;
    bool inflight = false;        // work enqueued since the last round
};

struct Server {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> by_ticket;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // workspace clones per hierarchy (server thread only), kept until the server stops;
    // at most extra_workspaces per hierarchy (0: one request per hierarchy at a time)
    std::unordered_map<Hierarchy*, std::vector<Hierarchy*>> clones;
    // bytes of the running requests' hierarchies and workspaces: now, and the most since creation
    std::atomic<size_t> resident{0}, peak{0};
    int extra_workspaces = 0;
    int batch_columns = 0;        // > 1: FP32 / BF16 requests on one hierarchy run as a column group
    std::unordered_map<Hierarchy*, Group*> groups;
};

static bool same_vcycle(const nmg_solve_opts& a, const nmg_solve_opts& b) {
    return a.precision == b.precision && a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.omega == b.omega &&
           a.weighting == b.weighting;
}

static Hierarchy* column_workspace(Hierarchy* h, int k) { return k == 0 ? h : h->many_ws[k - 1]; }

// Hierarchies with running requests.  The memory they hold is read from their
// live byte counts (each such hierarchy once: its operator and first
// workspace), so buffers a request allocates while it runs (Krylov bases,
// multi-vector level buffers) are counted as soon as they exist, and nothing
// is subtracted that was not added.
struct Residency {
    std::unordered_map<Hierarchy*, int> running;   // requests per submitted hierarchy
    void add(Hierarchy* h) { running[h]++; }
    void remove(Hierarchy* h) {
        if (--running[h] == 0) running.erase(h);
    }
    bool has(Hierarchy* h) const { return running.count(h) != 0; }
    size_t bytes() const {
        size_t s = 0;
        for (const auto& kv : running) s += kv.first->bytes;
        return s;
    }
};

// Live bytes of the server's workspace clones and of the column workspaces of
// groups with running columns (a group without columns may outlive its hierarchy).
static size_t workspace_bytes(const Server* S) {
    size_t s = 0;
    for (const auto& kv : S->clones)
        for (const Hierarchy* c : kv.second) s += c->bytes;
    for (const auto& kv : S->groups)
        if (kv.second->n > 0)
            for (const Hierarchy* c : kv.first->many_ws) s += c->bytes;
    return s;
}

static void finish_request(Server* S, Request* r, std::vector<Request*>& active, std::unordered_set<Hierarchy*>& busy,
                           Residency& res) {
    job_info(r->job, &r->info);
    r->info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->t_submit).count();
    r->err = r->job.err;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    busy.erase(r->slot);
    res.remove(r->h);
    active.erase(std::find(active.begin(), active.end(), r));
    std::lock_guard<std::mutex> lk(S->mu);
    r->done = true;
    S->cv_done.notify_all();
}

static void finish_grouped(Server* S, Request* r, std::vector<Request*>& active, Residency& res) {
    Group* G = r->group;
    job_info(r->job, &r->info);
    r->info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->t_submit).count();
    r->err = r->job.err;
    if (r->col > 0) r->slot->stream = r->own_stream;
    G->col[r->col] = nullptr;
    G->n--;
    res.remove(r->h);
    active.erase(std::find(active.begin(), active.end(), r));
    std::lock_guard<std::mutex> lk(S->mu);
    r->done = true;
    S->cv_done.notify_all();
}

// One round of a column group whose enqueued work has completed (q: the
// event's status): advance every column, retire the finished ones, then one
// multi-vector V-cycle for the columns that need one and their Arnoldi steps.
static void advance_group(Server* S, Group* G, cudaError_t q, std::vector<Request*>& active, Residency& res) {
    Hierarchy* h = G->h;
    G->inflight = false;
    int want[kMaxCols], nw = 0;
    for (int k = 0; k < kMaxCols; ++k) {
        Request* r = G->col[k];
        if (!r || r->job.phase == SolveJob::P_DONE) continue;
        if (q != cudaSuccess) {
            fail(NMG_ERR_CUDA, std::string("request failed: ") + cudaGetErrorString(q));
            job_fail(r->job, NMG_ERR_CUDA);
            r->job.phase = SolveJob::P_DONE;
            continue;
        }
        const int64_t l0 = g_launches;
        job_advance(r->job);
        r->job.launches += g_launches - l0;
        if (r->job.phase == SolveJob::P_WANT) want[nw++] = k;
    }
    // before a column leaves: a bounded wait of the shared multi-vector apply
    // that ran out fails every column of the group
    bool leaving = false;
    for (int k = 0; k < kMaxCols; ++k) leaving = leaving || (G->col[k] && G->col[k]->job.phase == SolveJob::P_DONE);
    int many_flag = 0;   // read in the hierarchy's stream order (no device-wide synchronisation)
    if (leaving &&
        cudaMemcpyAsync(&many_flag, h->flags + FLAG_MANY, sizeof(int), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
        cudaStreamSynchronize(h->stream) == cudaSuccess && many_flag) {
        cudaMemsetAsync(h->flags + FLAG_MANY, 0, sizeof(int), h->stream);
        fail(NMG_ERR_TIMEOUT, "a bounded device wait of the multi-vector apply ran out");
        // every column fails; the ones still iterating go straight to their finish (no further
        // V-cycle or Arnoldi step of a result that is discarded)
        for (int k = 0; k < kMaxCols; ++k)
            if (Request* r = G->col[k]) {
                job_fail(r->job, NMG_ERR_TIMEOUT);
                if (r->job.phase != SolveJob::P_DONE) job_enqueue_finish(r->job);
            }
        nw = 0;
    }
    for (int k = 0; k < kMaxCols; ++k)
        if (G->col[k] && G->col[k]->job.phase == SolveJob::P_DONE) finish_grouped(S, G->col[k], active, res);
    if (nw > 0) {
        ColPtrs in{};
        ColPtrsOut out{};
        for (int i = 0; i < nw; ++i) {
            const PrecData& P = G->col[want[i]]->slot->lev[h->L - 1].p[G->vo.precision];
            in.p[i] = (const float*)P.b;
            out.p[i] = (float*)P.x;
        }
        const int64_t l0 = g_launches;
        const nmg_status st = vcycle_cols(h, G->vo, nw, in, out);
        for (int i = 0; i < nw; ++i) {
            Request* r = G->col[want[i]];
            if (st != NMG_OK) {
                job_fail(r->job, st);
                job_enqueue_finish(r->job);
                continue;
            }
            Hierarchy* w = r->slot;
            enqueue_arnoldi(w, r->job.o, false, 0);
            cudaMemcpyAsync(w->host_scal, w->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            cudaMemcpyAsync(w->host_cyc, w->cyc, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
            r->job.phase = SolveJob::P_ITER;
            r->job.launches += (g_launches - l0) / nw;
        }
    }
    if (G->n > 0) {
        cudaEventRecord(G->ev, h->stream);
        G->inflight = true;
    }
}

static void server_loop(Server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> active;
    std::unordered_set<Hierarchy*> busy;   // slots (hierarchies or clones) running a request
    Residency res;
    for (;;) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (active.empty() && S->queue.empty()) {
                if (S->stop) break;
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            // in arrival order: a request starts on its hierarchy, or on an idle clone of it, or on a
            // new clone if the budget holds one more workspace; otherwise it waits.  The budget is
            // checked against the live bytes of the running hierarchies and workspaces plus what the
            // request will add: its hierarchy (once), the Krylov bases its slot still has to
            // allocate, and for a column group the multi-vector buffers and column workspaces.
            size_t pending = 0;   // growth of the requests admitted in this pass (allocated when they start)
            for (auto it = S->queue.begin(); it != S->queue.end() && (int)(active.size() + admit.size()) < S->max_slots;) {
                Request* r = *it;
                const size_t used = res.bytes() + workspace_bytes(S) + pending;
                const size_t base = res.has(r->h) ? 0 : r->h->bytes;
                const bool first = active.empty() && admit.empty();   // always admitted (alone it fits or fails)
                auto fits_with = [&](size_t need) { return S->budget == 0 || used + need <= S->budget || first; };
                Hierarchy* slot = nullptr;
                Group* G = S->groups.count(r->h) ? S->groups[r->h] : nullptr;
                const bool batch = S->batch_columns > 1 && r->o.precision != NMG_PREC_FP64 && !r->h->mixed_any;
                if (batch) {
                    // a column of the hierarchy's group (none runs alone on it)
                    int k = -1;
                    if (fits_with(base) && !busy.count(r->h) &&
                        (!G || G->n == 0 || (G->n < S->batch_columns && same_vcycle(G->vo, r->o))))
                        for (int c = 0; c < S->batch_columns && k < 0; ++c)
                            if (!G || !G->col[c]) k = c;
                    size_t ws_before = 0;
                    for (Hierarchy* c : r->h->many_ws) ws_before += c->bytes;
                    if (k >= 0 && many_workspaces(r->h, k + 1) == NMG_OK) {
                        size_t ws_now = 0;
                        for (Hierarchy* c : r->h->many_ws) ws_now += c->bytes;
                        const bool counted = G && G->n > 0;   // the group's workspaces are already in used
                        const size_t grow = many_growth(r->h, S->batch_columns > 4 ? 8 : 4) +
                                            krylov_growth(column_workspace(r->h, k), r->o.restart);
                        const size_t need = base + grow + (counted ? ws_now - ws_before : ws_now);
                        if (fits_with(need)) {
                            if (!G) {
                                G = new Group();
                                G->h = r->h;
                                S->groups[r->h] = G;
                            }
                            if (G->n == 0) G->vo = r->o;
                            G->col[k] = r;
                            G->n++;
                            r->group = G;
                            r->col = k;
                            res.add(r->h);
                            pending += grow;
                            r->slot = column_workspace(r->h, k);
                            admit.push_back(r);
                            it = S->queue.erase(it);
                            continue;
                        }
                    }
                    ++it;
                    continue;
                }
                if (!(G && G->n > 0)) {   // (a hierarchy running a column group takes no lone request)
                    if (!busy.count(r->h)) slot = r->h;
                    for (size_t c = 0; !slot && c < S->clones[r->h].size(); ++c)
                        if (!busy.count(S->clones[r->h][c])) slot = S->clones[r->h][c];
                    if (slot) {
                        const size_t grow = krylov_growth(slot, r->o.restart);
                        if (fits_with(base + grow)) {
                            pending += grow;
                        } else {
                            slot = nullptr;
                        }
                    } else if ((int)S->clones[r->h].size() < S->extra_workspaces && fits_with(base)) {
                        const size_t room = S->budget == 0 ? 0 : (S->budget > used + base ? S->budget - used - base : 1);
                        Hierarchy* c = nullptr;
                        if (clone_workspace(r->h, room, &c) == NMG_OK) {
                            if (ensure_krylov(c, r->o.restart) == NMG_OK) {   // the Krylov bases inside the budget too
                                c->desc.mem_budget_bytes = 0;
                                S->clones[r->h].push_back(c);
                                slot = c;
                            } else {
                                free_all(c);
                                delete c;
                            }
                        }
                    }
                }
                if (slot) {
                    busy.insert(slot);
                    res.add(r->h);
                    r->slot = slot;
                    admit.push_back(r);
                    it = S->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (Request* r : admit) {
            active.push_back(r);
            if (r->group) {
                Hierarchy* h = r->group->h;
                if (r->col > 0) {
                    r->own_stream = r->slot->stream;
                    r->slot->stream = h->stream;
                }
                nmg_solve_opts oc = r->o;
                oc.engine = NMG_ENGINE_KERNELS;
                oc.tail_patches = 0;
                oc.tile_patches = 0;
                const int64_t l0 = g_launches;
                const nmg_status st = job_start(r->job, r->slot, r->b, r->x, oc);
                if (st != NMG_OK) {
                    r->job.st = st;
                    r->job.err = g_last_error;
                    r->job.phase = SolveJob::P_DONE;
                }
                r->job.grouped = true;
                r->job.launches = g_launches - l0;
                // the multi-vector level buffers the group's V-cycles use, sized for the group's
                // largest column count now (admission counted them)
                if (r->job.phase != SolveJob::P_DONE) {
                    const nmg_status sm = ensure_many(h, S->batch_columns > 4 ? 8 : 4);
                    if (sm != NMG_OK) {
                        r->job.st = sm;
                        r->job.err = g_last_error;
                        r->job.phase = SolveJob::P_DONE;
                    }
                }
                Group* G = r->group;
                if (!G->ev && cudaEventCreateWithFlags(&G->ev, cudaEventDisableTiming) != cudaSuccess) G->ev = nullptr;
                if (G->ev) {
                    cudaEventRecord(G->ev, h->stream);
                    G->inflight = true;
                }
                continue;
            }
            const int64_t l0 = g_launches;
            nmg_status st = job_start(r->job, r->slot, r->b, r->x, r->o);
            if (st == NMG_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(r->ev, r->slot->stream);
            } else {
                if (st == NMG_OK) st = fail(NMG_ERR_CUDA, "event creation failed");
                r->job.st = st;
                r->job.err = g_last_error;
                r->job.phase = SolveJob::P_DONE;
            }
            r->job.launches = g_launches - l0;
        }
        bool progressed = !admit.empty();
        for (auto& kv : S->groups) {
            Group* G = kv.second;
            if (G->n == 0 || !G->inflight) continue;
            const cudaError_t q = cudaEventQuery(G->ev);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            advance_group(S, G, q, active, res);
        }
        for (size_t i = 0; i < active.size();) {
            Request* r = active[i];
            if (r->group) { ++i; continue; }
            if (r->job.phase != SolveJob::P_DONE) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) { ++i; continue; }
                progressed = true;
                if (q != cudaSuccess) {
                    fail(NMG_ERR_CUDA, std::string("request failed: ") + cudaGetErrorString(q));
                    r->job.st = NMG_ERR_CUDA;
                    r->job.err = g_last_error;
                    r->job.phase = SolveJob::P_DONE;
                } else {
                    const int64_t l0 = g_launches;
                    job_advance(r->job);
                    r->job.launches += g_launches - l0;
                    if (r->job.phase != SolveJob::P_DONE) cudaEventRecord(r->ev, r->slot->stream);
                }
            }
            if (r->job.phase == SolveJob::P_DONE) {
                cudaStreamSynchronize(r->slot->stream);
                finish_request(S, r, active, busy, res);
                progressed = true;
                continue;
            }
            ++i;
        }
        const size_t live = res.bytes() + workspace_bytes(S);
        S->resident = live;
        if (live > S->peak) S->peak = live;
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace nmg

extern "C" {

nmg_status nmg_server_create(size_t mem_budget_bytes, int max_slots, nmg_server** out) {
    if (!out || max_slots < 1 || max_slots > 1024) return fail(NMG_ERR_INVALID, "bad server arguments");
    auto* S = new nmg::Server();
    S->budget = mem_budget_bytes;
    S->max_slots = max_slots;
    cudaGetDevice(&S->device);
    S->worker = std::thread(nmg::server_loop, S);
    *out = reinterpret_cast<nmg_server*>(S);
    return NMG_OK;
}

nmg_status nmg_server_set_batching(nmg_server* server, int max_columns) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S || max_columns < 0 || max_columns > kMaxCols) return fail(NMG_ERR_INVALID, "bad server or column count");
    std::lock_guard<std::mutex> lk(S->mu);
    S->batch_columns = max_columns;
    return NMG_OK;
}

nmg_status nmg_server_set_workspaces(nmg_server* server, int extra_per_hierarchy) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S || extra_per_hierarchy < 0 || extra_per_hierarchy > 1024)
        return fail(NMG_ERR_INVALID, "bad server or workspace count");
    std::lock_guard<std::mutex> lk(S->mu);
    S->extra_workspaces = extra_per_hierarchy;
    return NMG_OK;
}

nmg_status nmg_submit(nmg_server* server, nmg_hierarchy* h, const double* b, double* x, const nmg_solve_opts* opts,
                      uint64_t* ticket) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S || !h || !b || !x || !ticket) return fail(NMG_ERR_INVALID, "NULL argument");
    NMG_TRY(validate_opts(opts));
    if (S->budget && h->bytes > S->budget)
        return fail(NMG_ERR_OOM, "hierarchy larger than the server's memory budget");
    auto* r = new nmg::Request();
    r->h = h;
    r->b = b;
    r->x = x;
    r->o = *opts;
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return fail(NMG_ERR_INVALID, "server is shutting down");
        }
        r->ticket = S->next_ticket++;
        S->by_ticket[r->ticket] = r;
        S->queue.push_back(r);
    }
    S->cv_work.notify_one();
    *ticket = r->ticket;
    return NMG_OK;
}

nmg_status nmg_poll(nmg_server* server, uint64_t ticket, int timeout_ms, nmg_solve_info* info) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S) return fail(NMG_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return fail(NMG_ERR_INVALID, "unknown ticket");
    nmg::Request* r = it->second;
    if (!r->done) {
        if (timeout_ms <= 0) return NMG_PENDING;
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
        if (!r->done) return fail(NMG_ERR_TIMEOUT, "request still running at the poll deadline");
    }
    if (info) *info = r->info;
    const nmg_status st = r->info.status;
    if (st != NMG_OK) g_last_error = r->err;
    S->by_ticket.erase(it);
    delete r;
    return st;
}

nmg_status nmg_server_memory(nmg_server* server, size_t* resident_bytes, size_t* peak_bytes) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S) return fail(NMG_ERR_INVALID, "NULL server");
    if (resident_bytes) *resident_bytes = S->resident.load();
    if (peak_bytes) *peak_bytes = S->peak.load();
    return NMG_OK;
}

nmg_status nmg_server_destroy(nmg_server* server) {
    auto* S = reinterpret_cast<nmg::Server*>(server);
    if (!S) return NMG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->by_ticket) delete kv.second;
    for (auto& kv : S->groups) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    for (auto& kv : S->clones)
        for (nmg::Hierarchy* c : kv.second) {
            cudaStreamSynchronize(c->stream);
            free_all(c);
            delete c;
        }
    delete S;
    return NMG_OK;
}

}  // extern "C"
