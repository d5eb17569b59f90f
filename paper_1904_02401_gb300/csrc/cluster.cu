// V-cycle tail on one thread-block cluster with the levels resident in
// distributed shared memory: the coarse level and the small levels 1..top of
// a V-cycle (Section 4.3 (II)-(III)) run as one launch of a cluster of up to
// 16 CTAs.  On those levels each kernel of the per-step path moves only
// kilobytes, and its time is the chain of dependent global-memory round trips
// (about a microsecond each) plus the launch; here every vector of the tail
// levels (x, b, r, the per-patch corrections, the Dirichlet masks) is
// replicated in the shared memory of every CTA, and every CTA keeps the
// matrix rows and patch inverses of the nodes and patches it owns.  A step
// then reads only shared memory: each CTA computes its owned outputs, copies
// them into the other CTAs' replicas (st.shared::cluster), and the cluster
// barrier (release / acquire) publishes them for the next step.
//
// The steps are those of the per-step kernels (residual b - A x, the patch
// solves of Eq. (vanka), the update x += w * sum of corrections, restriction,
// coarse solve, prolongation) with the per-element code of elem.cuh, so the
// result equals that of the other engines bit for bit.  Levels are included
// only while the shared memory they need fits.  There is no spin-wait: only
// hardware barriers that every thread of the cluster reaches in the same order.
#include <algorithm>

#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;
constexpr int kMaxCluster = 16;
constexpr size_t kSmemBudget = 220 * 1024;   // dynamic shared memory per CTA we allow

struct RLevel {
    Geom g;              // geometry of the level
    Geom gA;             // same with ld = node_chunk: layout of the owned matrix rows
    const void* A;       // global matrix (stencil layout, ld = g.ld)
    const void* inv;     // global patch inverses
    int64_t stride;      // elements per patch inverse
    const uint8_t* mask; // global Dirichlet mask
    int node_chunk, patch_chunk;
    // byte offsets into dynamic shared memory
    uint32_t o_x, o_b, o_r, o_corr, o_A, o_inv, o_mask;
};

struct RArgs {
    RLevel lev[kMaxLevels];
    int L;               // levels 0..L-1 (L-1 = top)
    int nu1, nu2;
    double omega;
    int average;
    const double* cinv;  // coarse dense inverse (global, FP64)
    int64_t n0;          // coarse unknowns
    int row_chunk;       // coarse rows per CTA
    const void* b_top;   // global right-hand side of the top level
    void* x_top;         // global result of the top level
};

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

template <typename T>
__device__ __forceinline__ void st_remote(uint32_t addr, T v);
template <>
__device__ __forceinline__ void st_remote<float>(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
template <>
__device__ __forceinline__ void st_remote<double>(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ void own_range(int64_t total, int chunk, int rank, int64_t& lo, int64_t& hi) {
    lo = min((int64_t)rank * chunk, total);
    hi = min(lo + chunk, total);
}

template <typename T, typename TS, int DIM>
struct ResidentVCycle {
    static constexpr int NC = DIM + 1;
    static constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;

    const RArgs& a;
    unsigned char* sm;
    T (*sd)[NP];
    const int rank, csize, lane, warp;
    const T om;
    const bool avg;

    __device__ ResidentVCycle(const RArgs& args, unsigned char* smem, T (*sd_)[NP])
        : a(args), sm(smem), sd(sd_), rank((int)blockIdx.x), csize((int)gridDim.x), lane(threadIdx.x & 31),
          warp(threadIdx.x >> 5), om((T)args.omega), avg(args.average != 0) {}

    __device__ T* vec(uint32_t off) const { return reinterpret_cast<T*>(sm + off); }
    __device__ const uint8_t* msk(uint32_t off) const { return reinterpret_cast<const uint8_t*>(sm + off); }

    // Copies elements [lo, hi) of the array at local offset off into the same
    // place in every other CTA of the cluster, then synchronises the cluster.
    __device__ void publish(uint32_t off, int64_t lo, int64_t hi) {
        __syncthreads();
        const int64_t cnt = hi - lo;
        if (cnt > 0) {
            const T* src = vec(off);
            const uint32_t base = smem_addr(src);
            const uint32_t c32 = (uint32_t)cnt;
            for (uint32_t k = threadIdx.x; k < c32 * (uint32_t)csize; k += blockDim.x) {
                const uint32_t q = k / c32;
                if ((int)q == rank) continue;
                const int64_t e = lo + (k - q * c32);
                st_remote<T>(map_rank(base + (uint32_t)(e * sizeof(T)), q), src[e]);
            }
        }
        cluster_sync();
    }

    __device__ void residual(const RLevel& L) {
        int64_t lo, hi;
        own_range(L.g.nodes, L.node_chunk, rank, lo, hi);
        // owned rows, indexed by the global node (the layout's node stride is 1 in 2d, NB in 3d)
        const T* As = vec(L.o_A) - lo * (DIM == 3 ? NC * NC : 1);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
            spmv_node<T, DIM, T, false>(L.gA, As, vec(L.o_x), vec(L.o_b), vec(L.o_r), true, i);
        publish(L.o_r, lo * NC, hi * NC);
    }

    __device__ void apply(const RLevel& L, const T* d) {
        int64_t lo, hi;
        own_range(L.g.patches, L.patch_chunk, rank, lo, hi);
        const TS* inv = reinterpret_cast<const TS*>(sm + L.o_inv);
        for (int64_t p = lo + warp; p < hi; p += kCWarps) {
            gather_patch<T, DIM>(L.g, d, p, sd[warp], lane);
            __syncwarp();
            apply_patch<T, TS, DIM, false>(inv + (p - lo) * L.stride, sd[warp], vec(L.o_corr) + p * NP, lane);
            __syncwarp();
        }
        publish(L.o_corr, lo * NP, hi * NP);
    }

    __device__ void update(const RLevel& L, bool zero) {
        int64_t lo, hi;
        own_range(L.g.nodes, L.node_chunk, rank, lo, hi);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
            vanka_update_node<T, DIM>(L.g, vec(L.o_corr), vec(L.o_x), vec(L.o_x), zero, om, avg, i);
        publish(L.o_x, lo * NC, hi * NC);
    }

    __device__ void smooth(const RLevel& L, int steps, bool x_zero) {
        if (steps == 0 && x_zero) {
            // every CTA zeroes its whole replica: nothing to publish
            for (int64_t i = threadIdx.x; i < L.g.nodes * NC; i += blockDim.x) vec(L.o_x)[i] = T(0);
            __syncthreads();
            return;
        }
        for (int st = 0; st < steps; ++st) {
            const bool first = st == 0 && x_zero;
            if (!first) residual(L);
            apply(L, first ? vec(L.o_b) : vec(L.o_r));
            update(L, first);
        }
    }

    __device__ void run() {
        const int top = a.L - 1;
        for (int l = top; l >= 1; --l) {
            const RLevel& L = a.lev[l];
            const RLevel& C = a.lev[l - 1];
            smooth(L, a.nu1, true);
            residual(L);
            int64_t lo, hi;
            own_range(C.g.nodes, C.node_chunk, rank, lo, hi);
            for (int64_t I = lo + threadIdx.x; I < hi; I += blockDim.x)
                restrict_node<T, DIM>(L.g, C.g, vec(L.o_r), vec(C.o_b), msk(C.o_mask), I);
            publish(C.o_b, lo * NC, hi * NC);
        }
        {
            const RLevel& Z = a.lev[0];
            int64_t lo, hi;
            own_range(a.n0, a.row_chunk, rank, lo, hi);
            for (int64_t row = lo + warp; row < hi; row += kCWarps)
                coarse_row<T>(a.cinv, a.n0, vec(Z.o_b), vec(Z.o_x), row, lane);
            publish(Z.o_x, lo, hi);
        }
        for (int l = 1; l <= top; ++l) {
            const RLevel& L = a.lev[l];
            const RLevel& C = a.lev[l - 1];
            int64_t lo, hi;
            own_range(L.g.nodes, L.node_chunk, rank, lo, hi);
            for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
                prolong_node<T, DIM>(L.g, C.g, vec(C.o_x), vec(L.o_x), msk(L.o_mask), i);
            publish(L.o_x, lo * NC, hi * NC);
            smooth(L, a.nu2, false);
        }
    }

    // Stages the read-only data (owned matrix rows and patch inverses, masks)
    // into shared memory; every thread keeps 8 loads in flight.
    // dst[dix(k)] = src(k) for k < count
    template <typename E, class SRC, class DIX>
    __device__ void stage(E* dst, int64_t count, SRC&& src, DIX&& dix) {
        constexpr int U = 8;
        for (int64_t k0 = threadIdx.x; k0 < count; k0 += (int64_t)U * blockDim.x) {
            E v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + (int64_t)u * blockDim.x;
                if (k < count) v[u] = src(k);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + (int64_t)u * blockDim.x;
                if (k < count) dst[dix(k)] = v[u];
            }
        }
    }
    template <typename E, class SRC>
    __device__ void stage(E* dst, int64_t count, SRC&& src) {
        stage(dst, count, src, [](int64_t k) { return k; });
    }

    __device__ void load_constants() {
        constexpr int NA = ((DIM == 2) ? 9 : 27) * NC * NC;
        for (int l = 0; l < a.L; ++l) {
            const RLevel& L = a.lev[l];
            stage(reinterpret_cast<uint8_t*>(sm + L.o_mask), L.g.nodes * NC, [&](int64_t k) { return L.mask[k]; });
            if (l == 0) continue;
            int64_t lo, hi;
            own_range(L.g.nodes, L.node_chunk, rank, lo, hi);
            const uint32_t cnt = (uint32_t)(hi - lo);
            const T* A = reinterpret_cast<const T*>(L.A);
            if (cnt > 0) {
                // the owned nodes' entries, in the stencil layout with ld = node_chunk:
                // As[stencil_off(nch, s, e, j)] = A[stencil_off(ld, s, e, lo + j)],
                // a = s * NB + e < NA, j < cnt
                constexpr int NB = NC * NC;
                const int nch = L.node_chunk;
                const int64_t ld = L.g.ld;
                stage(vec(L.o_A), (int64_t)NA * cnt,
                      [&](int64_t k) {
                          const uint32_t a = (uint32_t)k / cnt, j = (uint32_t)k - a * cnt;
                          return A[stencil_off<DIM, NB>(ld, (int)(a / NB), (int)(a % NB), lo + j)];
                      },
                      [&](int64_t k) {
                          const uint32_t a = (uint32_t)k / cnt, j = (uint32_t)k - a * cnt;
                          return stencil_off<DIM, NB>(nch, (int)(a / NB), (int)(a % NB), (int64_t)j);
                      });
            }
            int64_t plo, phi;
            own_range(L.g.patches, L.patch_chunk, rank, plo, phi);
            const TS* inv = reinterpret_cast<const TS*>(L.inv) + plo * L.stride;
            stage(reinterpret_cast<TS*>(sm + L.o_inv), (phi - plo) * L.stride, [&](int64_t k) { return inv[k]; });
        }
    }

    // The top level's right-hand side (written by the kernel before this one).
    __device__ void load_rhs() {
        const RLevel& L = a.lev[a.L - 1];
        const T* b = reinterpret_cast<const T*>(a.b_top);
        stage(vec(L.o_b), L.g.nodes * NC, [&](int64_t k) { return b[k]; });
    }

    // The CTA's owned entries of the top level's result, to global memory.
    __device__ void store_result() {
        const RLevel& L = a.lev[a.L - 1];
        int64_t lo, hi;
        if (a.L == 1) {
            own_range(a.n0, a.row_chunk, rank, lo, hi);
        } else {
            own_range(L.g.nodes, L.node_chunk, rank, lo, hi);
            lo *= NC;
            hi *= NC;
        }
        T* x = reinterpret_cast<T*>(a.x_top);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) x[i] = vec(L.o_x)[i];
    }
};

template <typename T, typename TS, int DIM>
__global__ void __launch_bounds__(kCThreads, 1) k_vcycle_cluster(const __grid_constant__ RArgs a) {
    constexpr int NP = ResidentVCycle<T, TS, DIM>::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sd[kCWarps][NP];
    ResidentVCycle<T, TS, DIM> vc(a, smem_raw, sd);
    // the matrices, inverses and masks do not change during a solve: stage
    // them before waiting for the kernel that produces the right-hand side
    vc.load_constants();
    NMG_PDL_ENTRY();
    vc.load_rhs();
    __syncthreads();
    cluster_sync();   // every CTA of the cluster runs before any remote store
    vc.run();
    vc.store_result();
}

// Shared-memory layout of levels 0..top for a cluster of c CTAs; returns the
// bytes needed (0 when a size overflows the 32-bit offsets).
template <typename T, typename TS, int DIM>
size_t plan_layout(const Hierarchy* h, int prec, int top, int c, RArgs& a) {
    constexpr int NC = DIM + 1;
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    constexpr int NA = ((DIM == 2) ? 9 : 27) * NC * NC;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return (uint32_t)o;
    };
    for (int l = 0; l <= top; ++l) {
        const Level& Lv = h->lev[l];
        const PrecData& P = Lv.p[prec];
        RLevel& q = a.lev[l];
        q.g = Lv.g;
        q.gA = Lv.g;
        q.A = P.A;
        q.inv = P.inv;
        q.stride = P.inv_stride;
        q.mask = Lv.mask;
        const int64_t nv = Lv.g.nodes * NC;
        q.node_chunk = (int)((Lv.g.nodes + c - 1) / c);
        q.patch_chunk = (int)((Lv.g.patches + c - 1) / c);
        q.gA.ld = q.node_chunk;
        q.o_x = take(nv * sizeof(T));
        q.o_b = take(nv * sizeof(T));
        q.o_mask = take(nv);
        if (l > 0) {
            q.o_r = take(nv * sizeof(T));
            q.o_corr = take((size_t)Lv.g.patches * NP * sizeof(T));
            q.o_A = take((size_t)NA * q.node_chunk * sizeof(T));
            q.o_inv = take((size_t)q.patch_chunk * P.inv_stride * sizeof(TS));
        } else {
            q.o_r = q.o_corr = q.o_A = q.o_inv = 0;
        }
    }
    a.n0 = h->n0;
    a.row_chunk = (int)((h->n0 + c - 1) / c);
    return off > 0xffffffffu ? 0 : off;
}

// Launches the tail on the largest cluster (16, 8, ... CTAs) whose layout
// fits the shared-memory budget and that the device can schedule.
template <typename T, typename TS, int DIM>
bool launch_resident(Hierarchy* h, int prec, int top, RArgs& a, cudaStream_t s) {
    auto k = k_vcycle_cluster<T, TS, DIM>;
    cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c = kMaxCluster; c >= 1; c /= 2) {
        const size_t smem = plan_layout<T, TS, DIM>(h, prec, top, c, a);
        if (smem == 0 || smem > kSmemBudget) continue;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kCThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            continue;
        }
        cfg.numAttrs = g_no_pdl ? 1 : 2;
        g_launches += 1;
        return cudaLaunchKernelEx(&cfg, k, a) == cudaSuccess;
    }
    return false;
}

template <typename T, typename TS, int DIM>
bool fits_resident(const Hierarchy* h, int prec, int top) {
    RArgs a{};
    for (int c = kMaxCluster; c >= 1; c /= 2) {
        const size_t smem = plan_layout<T, TS, DIM>(h, prec, top, c, a);
        if (smem && smem <= kSmemBudget) return true;
    }
    return false;
}

}  // namespace

// Largest top level (<= want) whose tail fits the shared memory of a cluster
// (-1 if not even the coarse level does).
int resident_tail_top(const Hierarchy* h, int prec, int want) {
    for (int top = want; top >= 0; --top) {
        bool ok;
        if (h->dim == 2) {
            if (prec == NMG_PREC_FP64) ok = fits_resident<double, double, 2>(h, prec, top);
            else if (prec == NMG_PREC_FP32) ok = fits_resident<float, float, 2>(h, prec, top);
            else ok = fits_resident<float, __nv_bfloat16, 2>(h, prec, top);
        } else {
            if (prec == NMG_PREC_FP64) ok = fits_resident<double, double, 3>(h, prec, top);
            else if (prec == NMG_PREC_FP32) ok = fits_resident<float, float, 3>(h, prec, top);
            else ok = fits_resident<float, __nv_bfloat16, 3>(h, prec, top);
        }
        if (ok) return top;
    }
    return -1;
}

// Host entry: levels 0..top of the V-cycle as one cluster launch.  The b of
// level top is its right-hand side and x of level top receives the result
// (b_top / x_top override the level's own buffers when not null).  Returns
// false when no cluster can hold the levels.
bool launch_vcycle_tail(Hierarchy* h, int prec, int top, int nu1, int nu2, double omega, int weighting,
                        const void* b_top, void* x_top) {
    RArgs a{};
    a.L = top + 1;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.omega = omega;
    a.average = weighting == NMG_WEIGHT_AVERAGE;
    a.cinv = h->coarse_inv;
    a.b_top = b_top ? b_top : h->lev[top].p[prec].b;
    a.x_top = x_top ? x_top : h->lev[top].p[prec].x;
    if (h->dim == 2) {
        if (prec == NMG_PREC_FP64) return launch_resident<double, double, 2>(h, prec, top, a, h->stream);
        if (prec == NMG_PREC_FP32) return launch_resident<float, float, 2>(h, prec, top, a, h->stream);
        return launch_resident<float, __nv_bfloat16, 2>(h, prec, top, a, h->stream);
    }
    if (prec == NMG_PREC_FP64) return launch_resident<double, double, 3>(h, prec, top, a, h->stream);
    if (prec == NMG_PREC_FP32) return launch_resident<float, float, 3>(h, prec, top, a, h->stream);
    return launch_resident<float, __nv_bfloat16, 3>(h, prec, top, a, h->stream);
}

}  // namespace nmg
