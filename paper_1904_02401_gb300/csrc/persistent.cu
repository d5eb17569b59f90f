// Persistent V-cycle: one cooperative launch runs a whole multigrid V-cycle
// (Section 4.3 (II)-(III)) with one CTA per SM.  On the one-kernel-per-step
// path every step of a small level costs a kernel launch and a grid drain of a
// few microseconds, which dominates the V-cycle below ~10^6 unknowns.  Here
// the steps are phases of one kernel:
//  * phases of large levels run on the whole grid and end at a grid barrier
//    (bounded spin; a timeout sets an abort flag that ends every CTA);
//  * phases of small levels (few patches) run on CTA 0 alone and end at a
//    __syncthreads, the other CTAs wait at the next grid barrier;
//  * the 2d Vanka apply of large levels streams the patch inverses through a
//    double-buffered TMA bulk-copy pipeline in shared memory.
// The per-element arithmetic is the shared code of elem.cuh, so the results
// equal those of the one-kernel-per-step path bit for bit.
#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

constexpr int kPThreads = 1024;
constexpr int kPWarps = kPThreads / 32;
constexpr int kBarrierSpins = 1 << 24;
constexpr int kCopySpins = 1 << 22;
constexpr int kStagePPC = 32;          // patches per staged chunk (2d)

struct PLevel {
    Geom g;
    const void* A;
    const void* inv;
    int64_t stride;
    void* b;
    void* x;
    void* r;
    void* corr;
    const uint8_t* mask;
    int small;
    int staged;
};

struct PArgs {
    PLevel lev[kMaxLevels];
    int L;
    int nu1, nu2;
    double omega;
    int average;
    const double* cinv;
    int64_t n0;
    int coarse_small;
    unsigned* bar;     // [0] arrivals, [1] generation
    int* abort;
    int barrier_spins; // iteration limit of a grid-barrier wait
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier of a cooperative launch; false once any CTA has aborted.
__device__ bool grid_sync(const PArgs& a) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = !ld_volatile(a.abort);
        if (ok) {
            const unsigned gen = ld_acquire(&a.bar[1]);
            __threadfence();
            const unsigned arrived = atomicAdd(&a.bar[0], 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(&a.bar[0], 0u);
                __threadfence();
                atomicAdd(&a.bar[1], 1u);
            } else {
                int it = 0;
                while (ld_acquire(&a.bar[1]) == gen) {
                    if (++it > a.barrier_spins || ld_volatile(a.abort)) {
                        atomicExch(a.abort, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct Ctx {
    bool ok = true;
    bool prev_small = false;
};

// Runs body(first, step, is_warp_level) on the participating threads and
// synchronises them afterwards (see the file comment).
template <class F>
__device__ __forceinline__ void phase(const PArgs& a, Ctx& cx, bool small, F&& body) {
    if (!cx.ok) return;
    if (!small && cx.prev_small) {
        cx.ok = grid_sync(a);
        if (!cx.ok) return;
    }
    if (!small || blockIdx.x == 0) body();
    if (small) {
        if (blockIdx.x == 0) __syncthreads();
    } else {
        cx.ok = grid_sync(a);
    }
    cx.prev_small = small;
}

struct Range {
    int64_t first, step;
};
__device__ __forceinline__ Range threads(bool small) {
    return small ? Range{threadIdx.x, blockDim.x}
                 : Range{blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x};
}
__device__ __forceinline__ Range warps(bool small) {
    const int w = threadIdx.x >> 5;
    return small ? Range{w, kPWarps} : Range{blockIdx.x * (int64_t)kPWarps + w, (int64_t)gridDim.x * kPWarps};
}

template <typename T, typename TS, int DIM>
struct VCycle {
    static constexpr int NC = DIM + 1;
    static constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;

    const PArgs& a;
    Ctx cx;
    T (*sd)[NP];                 // per-warp gathered defects
    TS* buf[2];                  // staged inverse chunks (2d)
    uint32_t bar[2];
    uint32_t parity[2] = {0, 0};

    __device__ VCycle(const PArgs& args, T (*sd_)[NP], TS* b0, TS* b1, uint32_t m0, uint32_t m1) : a(args), sd(sd_) {
        buf[0] = b0;
        buf[1] = b1;
        bar[0] = m0;
        bar[1] = m1;
    }

    __device__ void residual(int l) {
        const PLevel& L = a.lev[l];
        phase(a, cx, L.small, [&] {
            const Range r = threads(L.small);
            for (int64_t i = r.first; i < L.g.nodes; i += r.step)
                spmv_node<T, DIM, T, true, 1>(L.g, (const T*)L.A, (const T*)L.x, (const T*)L.b, (T*)L.r, true, i);
        });
    }

    __device__ void apply_plain(const PLevel& L, const T* d) {
        const Range r = warps(L.small);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int64_t p = r.first; p < L.g.patches; p += r.step) {
            gather_patch<T, DIM>(L.g, d, p, sd[w], lane);
            __syncwarp();
            apply_patch<T, TS, DIM, true>((const TS*)L.inv + p * L.stride, sd[w], (T*)L.corr + p * NP, lane);
            __syncwarp();
        }
    }

    // 2d: chunks of kStagePPC patches, double-buffered TMA bulk copies.
    __device__ void apply_staged(const PLevel& L, const T* d) {
        const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
        const int64_t nchunks = (L.g.patches + kStagePPC - 1) / kStagePPC;
        const TS* inv = (const TS*)L.inv;
        auto issue = [&](int64_t c, int b) {
            const int64_t p0 = c * kStagePPC;
            const int cnt = (int)min((int64_t)kStagePPC, L.g.patches - p0);
            bulk_copy(buf[b], inv + p0 * L.stride, (uint32_t)(cnt * L.stride * (int64_t)sizeof(TS)), bar[b]);
        };
        int64_t c = blockIdx.x;
        if (c >= nchunks) return;
        if (tid == 0) issue(c, 0);
        for (int k = 0; c < nchunks; c += gridDim.x, ++k) {
            const int b = k & 1;
            const int64_t nxt = c + gridDim.x;
            if (tid == 0 && nxt < nchunks) issue(nxt, b ^ 1);
            const int64_t p0 = c * kStagePPC;
            const int cnt = (int)min((int64_t)kStagePPC, L.g.patches - p0);
            if (w < cnt) gather_patch<T, DIM>(L.g, d, p0 + w, sd[w], lane);
            uint32_t done = 0;
            for (int it = 0; it < kCopySpins && !done; ++it) done = mbar_try_wait(bar[b], parity[b]);
            parity[b] ^= 1u;
            if (!__syncthreads_and(done)) {
                // a copy did not complete in time: abort the launch after a bounded wait for it
                if (tid == 0) atomicExch(a.abort, 1);
                for (int it = 0; it < kCopySpins && !done; ++it) done = mbar_try_wait(bar[b], parity[b] ^ 1u);
                if (tid == 0 && nxt < nchunks) {
                    uint32_t d2 = 0;
                    for (int it = 0; it < kCopySpins && !d2; ++it) d2 = mbar_try_wait(bar[b ^ 1], parity[b ^ 1]);
                }
                cx.ok = false;
                return;
            }
            if (w < cnt) apply_patch<T, TS, DIM, false>(buf[b] + (int64_t)w * L.stride, sd[w], (T*)L.corr + (p0 + w) * NP, lane);
            __syncthreads();
        }
    }

    __device__ void smooth(int l, int steps, bool x_zero) {
        const PLevel& L = a.lev[l];
        const T om = (T)a.omega;
        if (steps == 0 && x_zero) {
            phase(a, cx, L.small, [&] {
                const Range r = threads(L.small);
                for (int64_t i = r.first; i < L.g.nodes * NC; i += r.step) ((T*)L.x)[i] = T(0);
            });
            return;
        }
        for (int st = 0; st < steps; ++st) {
            const bool first = st == 0 && x_zero;
            const T* d = first ? (const T*)L.b : (const T*)L.r;
            if (!first) residual(l);
            if (L.staged && !L.small) {
                phase(a, cx, false, [&] { apply_staged(L, d); });
            } else {
                phase(a, cx, L.small, [&] { apply_plain(L, d); });
            }
            phase(a, cx, L.small, [&] {
                const Range r = threads(L.small);
                for (int64_t i = r.first; i < L.g.nodes; i += r.step)
                    vanka_update_node<T, DIM>(L.g, (const T*)L.corr, (const T*)L.x, (T*)L.x, first, om, a.average != 0, i);
            });
        }
    }

    __device__ void run() {
        const int top = a.L - 1;
        for (int l = top; l >= 1; --l) {
            const PLevel& L = a.lev[l];
            const PLevel& C = a.lev[l - 1];
            smooth(l, a.nu1, true);
            residual(l);
            phase(a, cx, L.small, [&] {
                const Range r = threads(L.small);
                for (int64_t I = r.first; I < C.g.nodes; I += r.step)
                    restrict_node<T, DIM>(L.g, C.g, (const T*)L.r, (T*)C.b, C.mask, I);
            });
        }
        phase(a, cx, a.coarse_small != 0, [&] {
            const Range r = warps(a.coarse_small != 0);
            for (int64_t row = r.first; row < a.n0; row += r.step)
                coarse_row<T>(a.cinv, a.n0, (const T*)a.lev[0].b, (T*)a.lev[0].x, row, threadIdx.x & 31);
        });
        for (int l = 1; l <= top; ++l) {
            const PLevel& L = a.lev[l];
            const PLevel& C = a.lev[l - 1];
            phase(a, cx, L.small, [&] {
                const Range r = threads(L.small);
                for (int64_t i = r.first; i < L.g.nodes; i += r.step)
                    prolong_node<T, DIM>(L.g, C.g, (const T*)C.x, (T*)L.x, L.mask, i);
            });
            smooth(l, a.nu2, false);
        }
    }
};

template <typename T, typename TS, int DIM>
__global__ void __launch_bounds__(kPThreads, 1) k_vcycle_persistent(const __grid_constant__ PArgs a) {
    constexpr int NP = VCycle<T, TS, DIM>::NP;
    __shared__ T sd[kPWarps][NP];
    __shared__ __align__(8) uint64_t mbar[2];
    extern __shared__ __align__(128) unsigned char dyn[];
    bool staged = false;
    for (int l = 0; l < a.L; ++l) staged |= a.lev[l].staged != 0;
    TS* b0 = reinterpret_cast<TS*>(dyn);
    TS* b1 = b0;
    int64_t max_stride = 0;
    for (int l = 1; l < a.L; ++l)
        if (a.lev[l].staged && a.lev[l].stride > max_stride) max_stride = a.lev[l].stride;
    b1 = b0 + kStagePPC * max_stride;
    const uint32_t m0 = smem_addr(&mbar[0]), m1 = smem_addr(&mbar[1]);
    if (staged && threadIdx.x == 0) {
        mbar_init(m0);
        mbar_init(m1);
    }
    __syncthreads();
    VCycle<T, TS, DIM> vc(a, sd, b0, b1, m0, m1);
    vc.run();
}

int sm_count_persistent() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    }
    return n;
}

template <typename T, typename TS, int DIM>
cudaError_t launch_impl(const PArgs& a, size_t smem, cudaStream_t s) {
    auto k = k_vcycle_persistent<T, TS, DIM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sm_count_persistent());
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    g_launches += 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace

// Host entry: fills the launch arguments from the hierarchy and launches one
// persistent V-cycle on the finest level's b/x buffers of precision prec.
cudaError_t launch_vcycle_persistent(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting,
                                     unsigned* bar, int* abort, int small_patches) {
    PArgs a{};
    a.barrier_spins = h->wait_limit > 0 ? h->wait_limit : kBarrierSpins;
    a.L = h->L;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.omega = omega;
    a.average = weighting == NMG_WEIGHT_AVERAGE;
    a.cinv = h->coarse_inv;
    a.n0 = h->n0;
    a.coarse_small = h->n0 <= 256;
    a.bar = bar;
    a.abort = abort;
    int64_t max_stride = 0;
    const size_t ts = prec == NMG_PREC_FP64 ? 8 : prec == NMG_PREC_FP32 ? 4 : 2;
    for (int l = 0; l < h->L; ++l) {
        const Level& Lv = h->lev[l];
        const PrecData& P = Lv.p[prec];
        PLevel& q = a.lev[l];
        q.g = Lv.g;
        q.A = P.A;
        q.inv = P.inv;
        q.stride = P.inv_stride;
        q.b = P.b;
        q.x = P.x;
        q.r = P.r;
        q.corr = P.corr;
        q.mask = Lv.mask;
        q.small = l > 0 && Lv.g.patches <= small_patches;
        q.staged = l > 0 && h->dim == 2 && ts <= 4 && !q.small && (P.inv_stride * ts) % 16 == 0 &&
                   ((uintptr_t)P.inv % 16) == 0;
        if (q.staged && P.inv_stride > max_stride) max_stride = P.inv_stride;
    }
    const size_t smem = (size_t)2 * kStagePPC * max_stride * ts;
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), h->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(abort, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return e;
    if (h->dim == 2) {
        if (prec == NMG_PREC_FP64) return launch_impl<double, double, 2>(a, smem, h->stream);
        if (prec == NMG_PREC_FP32) return launch_impl<float, float, 2>(a, smem, h->stream);
        return launch_impl<float, __nv_bfloat16, 2>(a, smem, h->stream);
    }
    if (prec == NMG_PREC_FP64) return launch_impl<double, double, 3>(a, smem, h->stream);
    if (prec == NMG_PREC_FP32) return launch_impl<float, float, 3>(a, smem, h->stream);
    return launch_impl<float, __nv_bfloat16, 3>(a, smem, h->stream);
}

}  // namespace nmg
