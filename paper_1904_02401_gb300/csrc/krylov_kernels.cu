// FP64 kernels of the outer flexible GMRES (Section 4.3 item (I)): classical
// Gram-Schmidt with re-orthogonalisation (two passes of one multi-dot and one
// multi-axpy each), norms, the Givens update of the Hessenberg column and the
// final x += Z y.  All reductions use a fixed grid and a fixed summation tree,
// so results are bitwise reproducible run to run.
#include "nmg_internal.cuh"

namespace nmg {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;     // Krylov vectors per pass of the multi-dot

__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    __syncthreads();
    return r;   // valid in thread 0
}

// partial[k * kDotBlocks + blk] = sum over this block's indices of V_k . w
__global__ void __launch_bounds__(kThreads)
k_multidot_partial(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ w,
                   int64_t n, double* __restrict__ partial) {
    NMG_PDL_ENTRY();
    __shared__ double red[kThreads / 32];
    for (int kc = 0; kc < nvec; kc += kChunk) {
        double acc[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) acc[q] = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kThreads) {
            const double wi = w[i];
#pragma unroll
            for (int q = 0; q < kChunk; ++q)
                if (kc + q < nvec) acc[q] = fma(V[(int64_t)(kc + q) * ldv + i], wi, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (kc + q >= nvec) break;
            const double s = block_sum(acc[q], red);
            if (threadIdx.x == 0) partial[(int64_t)(kc + q) * kDotBlocks + blockIdx.x] = s;
        }
    }
}

// out[k] (+)= sum_blk partial[k][blk], one warp per k, fixed order.
__global__ void k_finish_dots(const double* __restrict__ partial, int nvec, double* out, bool accumulate,
                              bool take_sqrt) {
    NMG_PDL_ENTRY();
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= nvec) return;
    double s = 0.0;
    for (int b = lane; b < kDotBlocks; b += 32) s += partial[(int64_t)k * kDotBlocks + b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
        if (take_sqrt) s = sqrt(s);
        out[k] = accumulate ? out[k] + s : s;
    }
}

// w -= sum_k h_k V_k ; partial[blk] = sum over block of w_new^2
__global__ void __launch_bounds__(kThreads)
k_gs_update(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
            double* __restrict__ w, int64_t n, double* __restrict__ partial, bool want_norm) {
    NMG_PDL_ENTRY();
    __shared__ double red[kThreads / 32];
    __shared__ double hs[kMaxRestart + 1];
    for (int k = threadIdx.x; k < nvec; k += kThreads) hs[k] = h[k];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kThreads) {
        double v = w[i];
        for (int k = 0; k < nvec; ++k) v = fma(-hs[k], V[(int64_t)k * ldv + i], v);
        w[i] = v;
        acc = fma(v, v, acc);
    }
    if (want_norm) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads)
k_sumsq_partial(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
    NMG_PDL_ENTRY();
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kThreads)
        acc = fma(x[i], x[i], acc);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Column j of the Hessenberg matrix from scal[S_HC + 0..j+1] (h_{0..j,j} and
// ||w||): apply the earlier rotations, build rotation j, update g, write the
// residual estimate |g_{j+1}| / ||b|| and 1 / h_{j+1,j}.
__device__ void arnoldi_column(double* scal, int j, int m) {
    double* H = scal + S_H + (int64_t)j * (m + 1);
    const double* hc = scal + S_HC;
    double* cs = scal + S_CS;
    double* sn = scal + S_SN;
    double* g = scal + S_G;
    // two Gram-Schmidt passes: coefficients of pass 1 in hc, of pass 2 in scal[S_Y]
    for (int i = 0; i <= j; ++i) H[i] = hc[i] + scal[S_Y + i];
    H[j + 1] = hc[j + 1];
    const double hnext = hc[j + 1];
    for (int i = 0; i < j; ++i) {
        const double a = H[i], b = H[i + 1];
        H[i] = cs[i] * a + sn[i] * b;
        H[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double a = H[j], b = H[j + 1];
    double c, s;
    if (b == 0.0) { c = a >= 0.0 ? 1.0 : -1.0; s = 0.0; }
    else { const double r = hypot(a, b); c = a / r; s = b / r; }
    cs[j] = c;
    sn[j] = s;
    H[j] = c * a + s * b;
    H[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double est = fabs(g[j + 1]) / scal[S_BNORM];
    scal[S_EST] = est;
    scal[S_INVH] = hnext != 0.0 ? 1.0 / hnext : 0.0;
    if (!isfinite(est) || !isfinite(hnext)) scal[S_STATUS] = (double)NMG_ERR_NONFINITE;
    scal[S_ITER] += 1.0;
}

__global__ void k_arnoldi_finish(double* scal, int j, int m) {
    NMG_PDL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    arnoldi_column(scal, j, m);
}

__global__ void k_start_cycle(double* scal, int m) {
    NMG_PDL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= m; ++i) scal[S_G + i] = 0.0;
    const double beta = scal[S_BETA];
    scal[S_G] = beta;
    scal[S_INVH] = beta != 0.0 ? 1.0 / beta : 0.0;
    if (!isfinite(beta)) scal[S_STATUS] = (double)NMG_ERR_NONFINITE;
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ sp, double* __restrict__ y, int64_t n) {
    NMG_PDL_ENTRY();
    const double a = *sp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// y = H[:k,:k]^{-1} g[:k] by back substitution (single thread).
__global__ void k_backsolve(double* scal, int k, int m) {
    NMG_PDL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double* H = scal + S_H;
    double* y = scal + S_Y;
    const double* g = scal + S_G;
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int c = i + 1; c < k; ++c) v -= H[(int64_t)c * (m + 1) + i] * y[c];
        y[i] = v / H[(int64_t)i * (m + 1) + i];
    }
}

__global__ void __launch_bounds__(kThreads)
k_update_x(const double* __restrict__ scal, int k, const double* __restrict__ Z, int64_t ldz,
           double* __restrict__ x, int64_t n) {
    NMG_PDL_ENTRY();
    __shared__ double ys[kMaxRestart];
    for (int i = threadIdx.x; i < k; i += kThreads) ys[i] = scal[S_Y + i];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double v = x[i];
        for (int c = 0; c < k; ++c) v = fma(ys[c], Z[(int64_t)c * ldz + i], v);
        x[i] = v;
    }
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
    NMG_PDL_ENTRY();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (unsigned)(b < 1 ? 1 : b);
}


// Sum over the kDotBlocks partials of row k in the fixed order of
// k_finish_dots (lane-strided, then a shuffle tree); valid in lane 0.
__device__ __forceinline__ double finish_row(const double* __restrict__ partial, int k, int lane) {
    double s = 0.0;
    for (int b = lane; b < kDotBlocks; b += 32) s += partial[(int64_t)k * kDotBlocks + b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    return s;
}

// Every block publishes its partials; the last block to finish (ticket) sums
// them in the fixed order above.  Returns true in the last block.
__device__ __forceinline__ bool last_block(unsigned* counter) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        s_last = t == gridDim.x - 1;
        if (s_last) atomicExch(counter, 0u);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// out[k] = V_k . w for k < nvec, in one launch.
__global__ void __launch_bounds__(kThreads)
k_multidot_fused(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ w, int64_t n,
                 double* __restrict__ partial, double* __restrict__ out, unsigned* counter) {
    NMG_PDL_ENTRY();
    __shared__ double red[kThreads / 32];
    for (int kc = 0; kc < nvec; kc += kChunk) {
        double acc[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) acc[q] = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kThreads) {
            const double wi = w[i];
#pragma unroll
            for (int q = 0; q < kChunk; ++q)
                if (kc + q < nvec) acc[q] = fma(V[(int64_t)(kc + q) * ldv + i], wi, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (kc + q >= nvec) break;
            const double s = block_sum(acc[q], red);
            if (threadIdx.x == 0) partial[(int64_t)(kc + q) * kDotBlocks + blockIdx.x] = s;
        }
    }
    if (!last_block(counter)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < nvec; k += kThreads / 32) {
        const double s = finish_row(partial, k, lane);
        if (lane == 0) out[k] = s;
    }
}

// Second Gram-Schmidt pass w -= sum h_k V_k, ||w|| into scal[S_HC + j + 1], then
// the Givens update of Hessenberg column j, in one launch.
__global__ void __launch_bounds__(kThreads)
k_gs_norm_arnoldi(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                  double* __restrict__ w, int64_t n, double* __restrict__ partial, double* scal, int j, int m,
                  unsigned* counter) {
    NMG_PDL_ENTRY();
    __shared__ double red[kThreads / 32];
    __shared__ double hs[kMaxRestart + 1];
    for (int k = threadIdx.x; k < nvec; k += kThreads) hs[k] = h[k];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kThreads) {
        double v = w[i];
        for (int k = 0; k < nvec; ++k) v = fma(-hs[k], V[(int64_t)k * ldv + i], v);
        w[i] = v;
        acc = fma(v, v, acc);
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (!last_block(counter)) return;
    if (threadIdx.x < 32) {
        const double t = finish_row(partial, 0, threadIdx.x);
        if (threadIdx.x == 0) {
            scal[S_HC + j + 1] = sqrt(t);
            arnoldi_column(scal, j, m);
        }
    }
}

// y = x * scal[S_INVH] (the next Krylov vector) and, when y32 is given, its
// FP32 copy (the right-hand side of the next reduced-precision V-cycle).
__global__ void k_scale_convert(const double* __restrict__ x, const double* __restrict__ sp, double* __restrict__ y,
                                float* __restrict__ y32, int64_t n) {
    NMG_PDL_ENTRY();
    const double a = *sp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a * x[i];
        y[i] = v;
        if (y32) y32[i] = (float)v;
    }
}

}  // namespace

void launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t s) {
    g_launches += 2;
    pdl_launch(k_sumsq_partial, dim3(kDotBlocks), dim3(kThreads), 0, s, x, n, partial);
    pdl_launch(k_finish_dots, dim3(1), dim3(32), 0, s, partial, 1, out, false, true);
}

void launch_multidot(const double* V, int64_t ldv, int nvec, const double* w, int64_t n, double* partial,
                     double* out, bool accumulate, cudaStream_t s) {
    g_launches += 2;
    pdl_launch(k_multidot_partial, dim3(kDotBlocks), dim3(kThreads), 0, s, V, ldv, nvec, w, n, partial);
    pdl_launch(k_finish_dots, dim3((nvec + 7) / 8), dim3(256), 0, s, partial, nvec, out, accumulate, false);
}

void launch_gs_update(const double* V, int64_t ldv, int nvec, const double* h, double* w, int64_t n,
                      double* partial, double* nrm2, bool want_norm, cudaStream_t s) {
    g_launches += want_norm ? 2 : 1;
    pdl_launch(k_gs_update, dim3(kDotBlocks), dim3(kThreads), 0, s, V, ldv, nvec, h, w, n, partial, want_norm);
    if (want_norm) pdl_launch(k_finish_dots, dim3(1), dim3(32), 0, s, partial, 1, nrm2, false, true);
}

void launch_arnoldi_finish(double* scal, int j, int m, cudaStream_t s) { pdl_launch(k_arnoldi_finish, dim3(1), dim3(32), 0, s, scal, j, m); }

void launch_scale(const double* x, const double* scal_ptr, bool invert, double* y, int64_t n, cudaStream_t s) {
    g_launches += 1;
    (void)invert;
    pdl_launch(k_scale, dim3(grid_for(n)), dim3(256), 0, s, x, scal_ptr, y, n);
}

void launch_start_cycle(double* scal, int m, cudaStream_t s) { pdl_launch(k_start_cycle, dim3(1), dim3(32), 0, s, scal, m); }

void launch_solve_update(double* scal, int k, int m, const double* Z, int64_t ldz, double* x, int64_t n,
                         cudaStream_t s) {
    g_launches += 2;
    pdl_launch(k_backsolve, dim3(1), dim3(32), 0, s, scal, k, m);
    pdl_launch(k_update_x, dim3(grid_for(n)), dim3(kThreads), 0, s, scal, k, Z, ldz, x, n);
}

void launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_axpby, dim3(grid_for(n)), dim3(256), 0, s, a, x, b, y, n);
}

}  // namespace nmg

namespace nmg {

void launch_multidot_fused(const double* V, int64_t ldv, int nvec, const double* w, int64_t n, double* partial,
                           double* out, unsigned* counter, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_multidot_fused, dim3(kDotBlocks), dim3(kThreads), 0, s, V, ldv, nvec, w, n, partial, out, counter);
}

void launch_gs_norm_arnoldi(const double* V, int64_t ldv, int nvec, const double* h, double* w, int64_t n,
                            double* partial, double* scal, int j, int m, unsigned* counter, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_gs_norm_arnoldi, dim3(kDotBlocks), dim3(kThreads), 0, s, V, ldv, nvec, h, w, n, partial, scal, j,
               m, counter);
}

void launch_scale_convert(const double* x, const double* scal_ptr, double* y, float* y32, int64_t n,
                          cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_scale_convert, dim3(grid_for(n)), dim3(256), 0, s, x, scal_ptr, y, y32, n);
}

}  // namespace nmg
