// V-cycle tail on one thread-block cluster: the levels 0..top of a V-cycle
// (Section 4.3 (II)-(III)), i.e. the small levels below the point where the
// one-kernel-per-step path stops being bound by bytes, run as one launch of a
// cluster of up to 16 CTAs.  On those levels every kernel of the per-step
// path costs a few microseconds of launch, drain and memory latency while it
// moves only kilobytes; here each step is a phase of one kernel and phases are
// separated by the cluster's hardware barrier (barrier.cluster with release /
// acquire semantics, which orders the global-memory writes of one phase before
// the reads of the next across the cluster's CTAs).
//
// A smoothing step is three phases (residual b - A x, the patch solves of
// Eq. (vanka), the update x += w * sum of corrections), the same steps as the
// per-step kernels; each phase is one or two rounds of independent loads per
// thread.  (Fusing the update into the residual halves the phases but makes
// each thread recompute the updated iterate at all its neighbours, a chain of
// dependent loads that costs more than the barrier it saves.)  The
// per-element arithmetic is the shared code of elem.cuh, so the result equals
// that of the per-step kernels bit for bit.  There is no spin-wait: only
// hardware barriers that every thread of the cluster reaches in the same
// order.
#include <algorithm>

#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;
constexpr int kMaxCluster = 16;

struct CLevel {
    Geom g;
    const void* A;
    const void* inv;
    int64_t stride;
    void* b;
    void* x;     // the level's iterate and result
    void* r;
    void* corr;
    const uint8_t* mask;
};

struct CArgs {
    CLevel lev[kMaxLevels];
    int L;              // levels 0..L-1 (L-1 = top)
    int nu1, nu2;
    double omega;
    int average;
    const double* cinv;
    int64_t n0;
};

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename T, typename TS, int DIM>
struct ClusterVCycle {
    static constexpr int NC = DIM + 1;
    static constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;

    const CArgs& a;
    T (*sd)[NP];
    const int64_t t0, tn;   // this thread's index in the cluster, thread count
    const int64_t w0, wn;   // this warp's index in the cluster, warp count
    const int lane;
    const T om;
    const bool avg;

    __device__ ClusterVCycle(const CArgs& args, T (*sd_)[NP])
        : a(args), sd(sd_), t0(blockIdx.x * (int64_t)blockDim.x + threadIdx.x), tn((int64_t)gridDim.x * blockDim.x),
          w0(blockIdx.x * (int64_t)kCWarps + (threadIdx.x >> 5)), wn((int64_t)gridDim.x * kCWarps),
          lane(threadIdx.x & 31), om((T)args.omega), avg(args.average != 0) {}

    __device__ void apply(const CLevel& L, const T* d) {
        const int w = threadIdx.x >> 5;
        for (int64_t p = w0; p < L.g.patches; p += wn) {
            gather_patch<T, DIM>(L.g, d, p, sd[w], lane);
            __syncwarp();
            apply_patch<T, TS, DIM, true>((const TS*)L.inv + p * L.stride, sd[w], (T*)L.corr + p * NP, lane);
            __syncwarp();
        }
        cluster_sync();
    }

    // r = b - A x
    __device__ void residual(const CLevel& L) {
        for (int64_t i = t0; i < L.g.nodes; i += tn)
            spmv_node<T, DIM>(L.g, (const T*)L.A, (const T*)L.x, (const T*)L.b, (T*)L.r, true, i);
        cluster_sync();
    }

    // x = x (0 when zero) + w * sum of the corrections
    __device__ void update(const CLevel& L, bool zero) {
        for (int64_t i = t0; i < L.g.nodes; i += tn)
            vanka_update_node<T, DIM>(L.g, (const T*)L.corr, (const T*)L.x, (T*)L.x, zero, om, avg, i);
        cluster_sync();
    }

    __device__ void smooth(const CLevel& L, int steps, bool x_zero) {
        if (steps == 0 && x_zero) {
            for (int64_t i = t0; i < L.g.nodes * NC; i += tn) ((T*)L.x)[i] = T(0);
            cluster_sync();
            return;
        }
        for (int st = 0; st < steps; ++st) {
            const bool first = st == 0 && x_zero;
            if (!first) residual(L);
            apply(L, first ? (const T*)L.b : (const T*)L.r);
            update(L, first);
        }
    }

    __device__ void run() {
        const int top = a.L - 1;
        for (int l = top; l >= 1; --l) {
            const CLevel& L = a.lev[l];
            const CLevel& C = a.lev[l - 1];
            smooth(L, a.nu1, true);
            residual(L);
            for (int64_t I = t0; I < C.g.nodes; I += tn)
                restrict_node<T, DIM>(L.g, C.g, (const T*)L.r, (T*)C.b, C.mask, I);
            cluster_sync();
        }
        for (int64_t row = w0; row < a.n0; row += wn)
            coarse_row<T>(a.cinv, a.n0, (const T*)a.lev[0].b, (T*)a.lev[0].x, row, lane);
        cluster_sync();
        for (int l = 1; l <= top; ++l) {
            const CLevel& L = a.lev[l];
            const CLevel& C = a.lev[l - 1];
            for (int64_t i = t0; i < L.g.nodes; i += tn)
                prolong_node<T, DIM>(L.g, C.g, (const T*)C.x, (T*)L.x, L.mask, i);
            cluster_sync();
            smooth(L, a.nu2, false);
        }
    }
};

template <typename T, typename TS, int DIM>
__global__ void __launch_bounds__(kCThreads, 1) k_vcycle_cluster(const __grid_constant__ CArgs a) {
    NMG_PDL_ENTRY();
    constexpr int NP = ClusterVCycle<T, TS, DIM>::NP;
    __shared__ T sd[kCWarps][NP];
    ClusterVCycle<T, TS, DIM> vc(a, sd);
    vc.run();
}

// Largest cluster (<= 16 CTAs) the device can co-schedule for this kernel,
// cached per device and kernel instance.
template <typename T, typename TS, int DIM>
int cluster_size() {
    static int cached[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < kMaxDevices && cached[dev] > 0) return cached[dev];
    auto k = k_vcycle_cluster<T, TS, DIM>;
    cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int best = 1;
    for (int c = kMaxCluster; c >= 1; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kCThreads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) {
            best = c;
            break;
        }
        cudaGetLastError();
    }
    if (dev >= 0 && dev < kMaxDevices) cached[dev] = best;
    return best;
}

template <typename T, typename TS, int DIM>
void launch_cluster_impl(const CArgs& a, cudaStream_t s) {
    auto k = k_vcycle_cluster<T, TS, DIM>;
    const int c = cluster_size<T, TS, DIM>();
    cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_no_pdl ? 1 : 2;
    g_launches += 1;
    cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace

// Host entry: levels 0..top of the V-cycle as one cluster launch.  The b of
// level top is its right-hand side and x of level top receives the result
// (b_top / x_top override the level's own buffers when not null).
void launch_vcycle_tail(Hierarchy* h, int prec, int top, int nu1, int nu2, double omega, int weighting,
                        const void* b_top, void* x_top) {
    CArgs a{};
    a.L = top + 1;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.omega = omega;
    a.average = weighting == NMG_WEIGHT_AVERAGE;
    a.cinv = h->coarse_inv;
    a.n0 = h->n0;
    for (int l = 0; l <= top; ++l) {
        const Level& Lv = h->lev[l];
        const PrecData& P = Lv.p[prec];
        CLevel& q = a.lev[l];
        q.g = Lv.g;
        q.A = P.A;
        q.inv = P.inv;
        q.stride = P.inv_stride;
        q.b = (l == top && b_top) ? const_cast<void*>(b_top) : P.b;
        q.x = (l == top && x_top) ? x_top : P.x;
        q.r = P.r;
        q.corr = P.corr;
        q.mask = Lv.mask;
    }
    if (h->dim == 2) {
        if (prec == NMG_PREC_FP64) launch_cluster_impl<double, double, 2>(a, h->stream);
        else if (prec == NMG_PREC_FP32) launch_cluster_impl<float, float, 2>(a, h->stream);
        else launch_cluster_impl<float, __nv_bfloat16, 2>(a, h->stream);
    } else {
        if (prec == NMG_PREC_FP64) launch_cluster_impl<double, double, 3>(a, h->stream);
        else if (prec == NMG_PREC_FP32) launch_cluster_impl<float, float, 3>(a, h->stream);
        else launch_cluster_impl<float, __nv_bfloat16, 3>(a, h->stream);
    }
}

}  // namespace nmg
