// Vanka smoothing with patches of two sizes (Section 5.5.1): blocks of 2^d
// cells (3^d nodes) and, over a flagged region, blocks of 4^d cells (5^d
// nodes, the paper's four or eight adjacent elements; 75 unknowns in 2d, 500
// in 3d).  The small patches run through the regular apply kernels with a
// patch list; here are the apply of the large patches and the update, which
// gathers per node the corrections of the patches containing it from an
// incidence table built at set-up (in the patches' order), since a node may
// now lie in patches of either size.
#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

// corr_p = A_p^{-1} R_p d for the large patches.  Work item w covers rows
// [rb THREADS, (rb + 1) THREADS) of patch p = w / RB (rb = w % RB), one row per
// thread; the CTA gathers the patch's defect into shared memory, then each
// thread walks the columns in batches of 32 whose loads (column-major
// inverse: consecutive rows read consecutive entries) are all issued before
// their products, and sums the columns in ascending order.
template <typename T, typename TS, int DIM, int NC, int THREADS, int RB>
__global__ void __launch_bounds__(THREADS)
k_vanka_apply_large(Geom g, const TS* __restrict__ inv, int64_t stride, const int32_t* __restrict__ org,
                    int64_t npatch, const T* __restrict__ d, T* __restrict__ corr) {
    constexpr int NN = (DIM == 2) ? 25 : 125;
    constexpr int NP = NN * NC;
    constexpr int JB = 32;
    static_assert(THREADS * RB >= NP, "every row needs a thread");
    __shared__ T sd[NP];
    NMG_PDL_ENTRY();
    for (int64_t w = blockIdx.x; w < npatch * RB; w += gridDim.x) {
        const int64_t p = w / RB;
        const int row = (int)(w - p * RB) * THREADS + threadIdx.x;
        int px, py, pz;
        patch_xyz(g, (int64_t)org[p], px, py, pz);
        for (int t = threadIdx.x; t < NP; t += THREADS) {
            const int an = t / NC, c = t - an * NC;
            const int ax = an % 5, ay = (an / 5) % 5, az = an / 25;
            const int64_t node = (int64_t)(2 * px + ax) +
                                 (int64_t)g.nn[0] * ((2 * py + ay) + (int64_t)g.nn[1] * (2 * pz + az));
            sd[t] = d[node * NC + c];
        }
        __syncthreads();
        const TS* Ap = inv + p * stride + (row < NP ? row : 0);
        T acc = T(0);
        for (int j0 = 0; j0 < NP; j0 += JB) {
            TS a[JB];
#pragma unroll
            for (int u = 0; u < JB; ++u) a[u] = (j0 + u < NP) ? ldg(Ap + (int64_t)(j0 + u) * NP) : TS(0);
#pragma unroll
            for (int u = 0; u < JB; ++u)
                if (j0 + u < NP) acc = fma(Cvt<T, TS>::f(a[u]), sd[j0 + u], acc);
        }
        if (row < NP) corr[p * NP + row] = acc;
        __syncthreads();
    }
}

// x_out_i = x_in_i + w_i * (sum of the corrections of the patches containing
// node i, in the order of the incidence table), w_i = omega / (number of
// those patches) or omega.  inc: kIncMax offsets per node into the
// concatenation [small corrections, large corrections] (component 0), of which
// the first inc_n are used (at most KMAX = 2^d).
template <typename T, int NC, int KMAX>
__global__ void __launch_bounds__(256)
k_vanka_update_mixed(int64_t nodes, const T* __restrict__ corr_s, const T* __restrict__ corr_l, int64_t nsm,
                     const int32_t* __restrict__ inc, const uint8_t* __restrict__ inc_n, const T* x_in,
                     T* x_out, bool x_zero, T omega, bool average) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    const int m = inc_n[i];
    T sum[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sum[c] = T(0);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < m) {
            const int64_t off = inc[i * kIncMax + k];   // the table holds kIncMax entries per node
            const T* src = off < nsm ? corr_s + off : corr_l + (off - nsm);
#pragma unroll
            for (int c = 0; c < NC; ++c) sum[c] += src[c];
        }
    }
    const T wgt = average ? omega / T(m > 0 ? m : 1) : omega;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const T old = x_zero ? T(0) : x_in[i * NC + c];
        x_out[i * NC + c] = fma(wgt, sum[c], old);
    }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int multiprocessors() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

template <typename T, typename TS>
void launch_vanka_apply_large(const Geom& g, const TS* inv, int64_t stride, const int32_t* org, int64_t npatch,
                              const T* d, T* corr, cudaStream_t s) {
    if (npatch <= 0) return;
    g_launches += 1;
    const bool lean = g.nc == g.dim;
    // 2d: one CTA per patch (75 or 50 rows); 3d: 4 or 3 CTAs of 128 rows per patch (500 or 375 rows)
    const int rb = g.dim == 2 ? 1 : (lean ? 3 : 4);
    const dim3 grid((unsigned)std::min<int64_t>(npatch * rb, (int64_t)multiprocessors() * 16));
    if (g.dim == 2)
        pdl_launch(lean ? k_vanka_apply_large<T, TS, 2, 2, 64, 1> : k_vanka_apply_large<T, TS, 2, 3, 96, 1>, grid,
                   dim3(lean ? 64 : 96), 0, s, g, inv, stride, org, npatch, d, corr);
    else
        pdl_launch(lean ? k_vanka_apply_large<T, TS, 3, 3, 128, 3> : k_vanka_apply_large<T, TS, 3, 4, 128, 4>, grid,
                   dim3(128), 0, s, g, inv, stride, org, npatch, d, corr);
}

template <typename T>
void launch_vanka_update_mixed(const Geom& g, const T* corr_s, const T* corr_l, int64_t nsm, const int32_t* inc,
                               const uint8_t* inc_n, const T* x_in, T* x_out, bool x_zero, T omega, bool average,
                               cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256)), block(256);
    if (g.dim == 2) {
        if (g.nc == 2)
            pdl_launch(k_vanka_update_mixed<T, 2, 4>, grid, block, 0, s, g.nodes, corr_s, corr_l, nsm, inc, inc_n,
                       x_in, x_out, x_zero, omega, average);
        else
            pdl_launch(k_vanka_update_mixed<T, 3, 4>, grid, block, 0, s, g.nodes, corr_s, corr_l, nsm, inc, inc_n,
                       x_in, x_out, x_zero, omega, average);
    } else {
        if (g.nc == 3)
            pdl_launch(k_vanka_update_mixed<T, 3, 8>, grid, block, 0, s, g.nodes, corr_s, corr_l, nsm, inc, inc_n,
                       x_in, x_out, x_zero, omega, average);
        else
            pdl_launch(k_vanka_update_mixed<T, 4, 8>, grid, block, 0, s, g.nodes, corr_s, corr_l, nsm, inc, inc_n,
                       x_in, x_out, x_zero, omega, average);
    }
}

template void launch_vanka_apply_large<double, double>(const Geom&, const double*, int64_t, const int32_t*, int64_t,
                                                       const double*, double*, cudaStream_t);
template void launch_vanka_apply_large<float, float>(const Geom&, const float*, int64_t, const int32_t*, int64_t,
                                                     const float*, float*, cudaStream_t);
template void launch_vanka_apply_large<float, __nv_bfloat16>(const Geom&, const __nv_bfloat16*, int64_t,
                                                             const int32_t*, int64_t, const float*, float*,
                                                             cudaStream_t);
template void launch_vanka_update_mixed<double>(const Geom&, const double*, const double*, int64_t, const int32_t*,
                                                const uint8_t*, const double*, double*, bool, double, bool,
                                                cudaStream_t);
template void launch_vanka_update_mixed<float>(const Geom&, const float*, const float*, int64_t, const int32_t*,
                                               const uint8_t*, const float*, float*, bool, float, bool, cudaStream_t);

}  // namespace nmg
