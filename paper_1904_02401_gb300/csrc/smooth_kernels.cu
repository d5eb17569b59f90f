// Solve-phase kernels of the multigrid V-cycle (Section 4.3 (II)-(III)):
// block-sparse residual products, the additive Vanka patch step of Eq. (vanka),
// Q1 restriction / prolongation and the coarse solve.  Every kernel is
// memory-bound; the data layouts are chosen so that warps read contiguous,
// coalesced segments of the matrix and of the patch inverses.  All kernels are
// launched with programmatic dependent launch (see nmg_internal.cuh).
#include "elem.cuh"

namespace nmg {

__device__ int g_wait_timeout = 0;

namespace {

using namespace elem;

constexpr int kPPC = 16;           // patches per CTA of the staged 2d apply
constexpr int kStagedWarps = 4;
constexpr int kWaitSpins = 1 << 22;

// y = A x  or  y = b - A x, one thread per node.  A in stencil layout.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_spmv(Geom g, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
       T* __restrict__ y, bool residual) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) spmv_node<T, DIM>(g, A, x, b, y, residual, i);
}

// w = A z in FP64 with z read from the V-cycle output xf (stored as TX) and
// written, converted, to z64 (the FGMRES basis vector Z_j): the outer product
// of one FGMRES iteration without a separate conversion pass.
template <typename TX, int DIM>
__global__ void __launch_bounds__(256)
k_spmv_zstore(Geom g, const double* __restrict__ A, const TX* __restrict__ xf, double* __restrict__ z64,
              double* __restrict__ w) {
    NMG_PDL_ENTRY();
    constexpr int NC = DIM + 1;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.nodes) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) z64[i * NC + c] = (double)xf[i * NC + c];
    spmv_node<double, DIM, TX>(g, A, xf, nullptr, w, false, i);
}

// corr_i = A_i^{-1} R_i d for every patch i: one warp per patch.  The patch
// inverse is column-major, so for each column j the 32 lanes read 32
// consecutive entries (one coalesced 128-byte segment in FP32) and multiply
// them by the broadcast d_j from shared memory; no cross-lane reduction.
// Used for 3d patches (n_p = 108), where each warp streams 46.7 KB.
template <typename T, typename TS, int DIM, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_vanka_apply(Geom g, const TS* __restrict__ inv, int64_t stride, const T* __restrict__ d,
              T* __restrict__ corr) {
    NMG_PDL_ENTRY();
    constexpr int NP = ((DIM == 2) ? 9 : 27) * (DIM + 1);
    __shared__ T sd[WARPS][NP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * WARPS + w;
    if (p >= g.patches) return;
    gather_patch<T, DIM>(g, d, p, sd[w], lane);
    __syncwarp();
    apply_patch<T, TS, DIM, true>(inv + p * stride, sd[w], corr + p * NP, lane);
}

// 2d variant: the inverses of kPPC consecutive patches (contiguous in memory)
// are staged into shared memory by one TMA bulk copy completing on an
// mbarrier, so a CTA keeps kPPC * 2.9 KB (FP32) in flight instead of the few
// hundred bytes a warp of per-lane loads keeps.  Each warp then applies its
// patches from shared memory (same summation order as above).
template <typename T, typename TS>
__global__ void __launch_bounds__(kStagedWarps * 32)
k_vanka_apply_staged2d(Geom g, const TS* __restrict__ inv, int64_t stride, const T* __restrict__ d,
                       T* __restrict__ corr) {
    NMG_PDL_ENTRY();
    constexpr int NP = 27;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ T sd[kPPC][NP];
    TS* sinv = reinterpret_cast<TS*>(smem_raw);
    const int tid = threadIdx.x;
    const int w = tid >> 5, lane = tid & 31;
    const int64_t p0 = (int64_t)blockIdx.x * kPPC;
    const int count = (int)min((int64_t)kPPC, g.patches - p0);
    const uint32_t bytes = (uint32_t)(count * stride * (int64_t)sizeof(TS));   // multiple of 16
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) mbar_init(bar);
    __syncthreads();
    if (tid == 0) bulk_copy(sinv, inv + p0 * stride, bytes, bar);
    // gather the defects of the CTA's patches while the copy is in flight
    for (int q = w; q < count; q += kStagedWarps) gather_patch<T, 2>(g, d, p0 + q, sd[q], lane);
    uint32_t done = 0;
    for (int it = 0; it < kWaitSpins && !done; ++it) done = mbar_try_wait(bar, 0);
    // block-uniform outcome (also orders the gathered defects before use)
    if (!__syncthreads_and(done)) {
        // the copy did not complete in time: record it and wait (bounded) for it before leaving
        if (tid == 0) atomicExch(&g_wait_timeout, 1);
        for (int it = 0; it < kWaitSpins && !done; ++it) done = mbar_try_wait(bar, 0);
        return;
    }
    for (int q = w; q < count; q += kStagedWarps)
        apply_patch<T, TS, 2, false>(sinv + (int64_t)q * stride, sd[q], corr + (p0 + q) * NP, lane);
}

// x += w(node) * sum over the patches that contain the node of their
// corrections (fixed order: ascending patch index), w = omega / multiplicity
// ("average") or omega ("sum").  One thread per node, no atomics.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_vanka_update(Geom g, const T* __restrict__ corr, const T* x_in, T* x_out, bool x_zero, T omega,
               bool average) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) vanka_update_node<T, DIM>(g, corr, x_in, x_out, x_zero, omega, average, i);
}

// Fused Vanka update and residual: x_out = x_in + w * corrections, r = b - A x_out
// (x_out at the neighbours recomputed from x_in and the corrections).
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_update_residual(Geom g, const T* __restrict__ A, const T* __restrict__ corr, const T* __restrict__ x_in,
                  bool x_zero, T omega, bool average, const T* __restrict__ b, T* __restrict__ x_out,
                  T* __restrict__ r) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) update_residual_node<T, DIM>(g, A, corr, x_in, x_zero, omega, average, b, x_out, r, i);
}

// Fused prolongation and residual: x_out = x_in + P e_c, r = b - A x_out.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_prolong_residual(Geom f, Geom c, const T* __restrict__ A, const T* __restrict__ ec, const T* __restrict__ x_in,
                   const uint8_t* __restrict__ fmask, const T* __restrict__ b, T* __restrict__ x_out,
                   T* __restrict__ r) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < f.nodes) prolong_residual_node<T, DIM>(f, c, A, ec, x_in, fmask, b, x_out, r, i);
}

// r_c = P^T r_f (Q1 full weighting), coarse Dirichlet entries zero.  One thread per coarse node.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_restrict(Geom f, Geom c, const T* __restrict__ rf, T* __restrict__ rc, const uint8_t* __restrict__ cmask) {
    NMG_PDL_ENTRY();
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I < c.nodes) restrict_node<T, DIM>(f, c, rf, rc, cmask, I);
}

// x_f += P e_c (Q1 interpolation), fine Dirichlet entries untouched.  One thread per fine node.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_prolong_add(Geom f, Geom c, const T* __restrict__ ec, T* __restrict__ xf, const uint8_t* __restrict__ fmask) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < f.nodes) prolong_node<T, DIM>(f, c, ec, xf, fmask, i);
}

// x = inv * b with the FP64 dense coarse inverse, one warp per row, FP64 sums.
template <typename T>
__global__ void __launch_bounds__(256)
k_coarse_gemv(const double* __restrict__ inv, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
    NMG_PDL_ENTRY();
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row < n) coarse_row<T>(inv, n, b, x, row, threadIdx.x & 31);
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, int64_t n) {
    NMG_PDL_ENTRY();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)in[i];
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t wait_timeout_flag(int* value, cudaStream_t s) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(value, g_wait_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*value) e = cudaMemcpyToSymbolAsync(g_wait_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t wait_timeout_enqueue_read(int* dst, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(dst, g_wait_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
}

cudaError_t wait_timeout_clear(cudaStream_t s) {
    static const int zero = 0;
    return cudaMemcpyToSymbolAsync(g_wait_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}

template <typename T>
void launch_spmv(const Geom& g, const T* A, const T* x, const T* b, T* y, bool residual, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256));
    if (g.dim == 2) pdl_launch(k_spmv<T, 2>, grid, dim3(256), 0, s, g, A, x, b, y, residual);
    else pdl_launch(k_spmv<T, 3>, grid, dim3(256), 0, s, g, A, x, b, y, residual);
}

template <typename TX>
void launch_spmv_zstore(const Geom& g, const double* A, const TX* xf, double* z64, double* w, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256));
    if (g.dim == 2) pdl_launch(k_spmv_zstore<TX, 2>, grid, dim3(256), 0, s, g, A, xf, z64, w);
    else pdl_launch(k_spmv_zstore<TX, 3>, grid, dim3(256), 0, s, g, A, xf, z64, w);
}
template void launch_spmv_zstore<float>(const Geom&, const double*, const float*, double*, double*, cudaStream_t);
template void launch_spmv_zstore<double>(const Geom&, const double*, const double*, double*, double*, cudaStream_t);

template <typename T, typename TS>
void launch_vanka_apply(const Geom& g, const TS* inv, int64_t stride, const T* d, T* corr, cudaStream_t s) {
    g_launches += 1;
    // the bulk copy needs 16-byte aligned source chunks; other layouts use the warp kernel
    const bool aligned = ((uintptr_t)inv % 16 == 0) && ((stride * (int64_t)sizeof(TS)) % 16 == 0) &&
                         stride <= 27 * 27 + 16 && sizeof(TS) <= 4;   // FP64 keeps the warp kernel
    if (g.dim == 2 && aligned) {
        // the stride is at most n_p^2 + 16 elements (padding to 16 bytes)
        cudaFuncSetAttribute(k_vanka_apply_staged2d<T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kPPC * (27 * 27 + 16) * sizeof(TS)));
        const size_t smem = (size_t)kPPC * stride * sizeof(TS);
        const dim3 grid((unsigned)((g.patches + kPPC - 1) / kPPC));
        pdl_launch(k_vanka_apply_staged2d<T, TS>, grid, dim3(kStagedWarps * 32), smem, s, g, inv, stride, d, corr);
    } else if (g.dim == 2) {
        constexpr int W = 4;
        const dim3 grid((unsigned)((g.patches + W - 1) / W));
        pdl_launch(k_vanka_apply<T, TS, 2, W>, grid, dim3(W * 32), 0, s, g, inv, stride, d, corr);
    } else {
        constexpr int W = 4;
        const dim3 grid((unsigned)((g.patches + W - 1) / W));
        pdl_launch(k_vanka_apply<T, TS, 3, W>, grid, dim3(W * 32), 0, s, g, inv, stride, d, corr);
    }
}

template <typename T>
void launch_vanka_update(const Geom& g, const T* corr, T* x, bool x_zero, T omega, bool average, cudaStream_t s) {
    launch_vanka_update2<T>(g, corr, x, x, x_zero, omega, average, s);
}

template <typename T>
void launch_vanka_update2(const Geom& g, const T* corr, const T* x_in, T* x_out, bool x_zero, T omega, bool average,
                          cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256));
    if (g.dim == 2) pdl_launch(k_vanka_update<T, 2>, grid, dim3(256), 0, s, g, corr, x_in, x_out, x_zero, omega, average);
    else pdl_launch(k_vanka_update<T, 3>, grid, dim3(256), 0, s, g, corr, x_in, x_out, x_zero, omega, average);
}

template <typename T>
void launch_update_residual(const Geom& g, const T* A, const T* corr, const T* x_in, bool x_zero, T omega,
                            bool average, const T* b, T* x_out, T* r, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256));
    if (g.dim == 2)
        pdl_launch(k_update_residual<T, 2>, grid, dim3(256), 0, s, g, A, corr, x_in, x_zero, omega, average, b, x_out, r);
    else
        pdl_launch(k_update_residual<T, 3>, grid, dim3(256), 0, s, g, A, corr, x_in, x_zero, omega, average, b, x_out, r);
}

template <typename T>
void launch_prolong_residual(const Geom& f, const Geom& c, const T* A, const T* ec, const T* x_in,
                             const uint8_t* fmask, const T* b, T* x_out, T* r, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(f.nodes, 256));
    if (f.dim == 2) pdl_launch(k_prolong_residual<T, 2>, grid, dim3(256), 0, s, f, c, A, ec, x_in, fmask, b, x_out, r);
    else pdl_launch(k_prolong_residual<T, 3>, grid, dim3(256), 0, s, f, c, A, ec, x_in, fmask, b, x_out, r);
}

template void launch_vanka_update2<double>(const Geom&, const double*, const double*, double*, bool, double, bool,
                                           cudaStream_t);
template void launch_vanka_update2<float>(const Geom&, const float*, const float*, float*, bool, float, bool,
                                          cudaStream_t);
template void launch_update_residual<double>(const Geom&, const double*, const double*, const double*, bool, double,
                                             bool, const double*, double*, double*, cudaStream_t);
template void launch_update_residual<float>(const Geom&, const float*, const float*, const float*, bool, float, bool,
                                            const float*, float*, float*, cudaStream_t);
template void launch_prolong_residual<double>(const Geom&, const Geom&, const double*, const double*, const double*,
                                              const uint8_t*, const double*, double*, double*, cudaStream_t);
template void launch_prolong_residual<float>(const Geom&, const Geom&, const float*, const float*, const float*,
                                             const uint8_t*, const float*, float*, float*, cudaStream_t);

template <typename T>
void launch_restrict(const Geom& f, const Geom& c, const T* rf, T* rc, const uint8_t* cmask, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(c.nodes, 256));
    if (f.dim == 2) pdl_launch(k_restrict<T, 2>, grid, dim3(256), 0, s, f, c, rf, rc, cmask);
    else pdl_launch(k_restrict<T, 3>, grid, dim3(256), 0, s, f, c, rf, rc, cmask);
}

template <typename T>
void launch_prolong_add(const Geom& f, const Geom& c, const T* ec, T* xf, const uint8_t* fmask, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(f.nodes, 256));
    if (f.dim == 2) pdl_launch(k_prolong_add<T, 2>, grid, dim3(256), 0, s, f, c, ec, xf, fmask);
    else pdl_launch(k_prolong_add<T, 3>, grid, dim3(256), 0, s, f, c, ec, xf, fmask);
}

template <typename T>
void launch_coarse_gemv(const double* inv, int64_t n, const T* b, T* x, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_coarse_gemv<T>, dim3(blocks_for(n * 32, 256)), dim3(256), 0, s, inv, n, b, x);
}

template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, int64_t n, cudaStream_t s) {
    g_launches += 1;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    pdl_launch(k_convert<TI, TO>, dim3((unsigned)blocks), dim3(256), 0, s, in, out, n);
}

template void launch_spmv<double>(const Geom&, const double*, const double*, const double*, double*, bool, cudaStream_t);
template void launch_spmv<float>(const Geom&, const float*, const float*, const float*, float*, bool, cudaStream_t);
template void launch_vanka_apply<double, double>(const Geom&, const double*, int64_t, const double*, double*, cudaStream_t);
template void launch_vanka_apply<float, float>(const Geom&, const float*, int64_t, const float*, float*, cudaStream_t);
template void launch_vanka_apply<float, __nv_bfloat16>(const Geom&, const __nv_bfloat16*, int64_t, const float*, float*, cudaStream_t);
template void launch_vanka_update<double>(const Geom&, const double*, double*, bool, double, bool, cudaStream_t);
template void launch_vanka_update<float>(const Geom&, const float*, float*, bool, float, bool, cudaStream_t);
template void launch_restrict<double>(const Geom&, const Geom&, const double*, double*, const uint8_t*, cudaStream_t);
template void launch_restrict<float>(const Geom&, const Geom&, const float*, float*, const uint8_t*, cudaStream_t);
template void launch_prolong_add<double>(const Geom&, const Geom&, const double*, double*, const uint8_t*, cudaStream_t);
template void launch_prolong_add<float>(const Geom&, const Geom&, const float*, float*, const uint8_t*, cudaStream_t);
template void launch_coarse_gemv<double>(const double*, int64_t, const double*, double*, cudaStream_t);
template void launch_coarse_gemv<float>(const double*, int64_t, const float*, float*, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace nmg
