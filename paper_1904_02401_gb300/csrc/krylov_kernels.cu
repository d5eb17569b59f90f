// FP64 kernels of the outer flexible GMRES (Section 4.3 item (I)): the outer
// product w = A z_j fused with the first classical Gram-Schmidt pass, the
// second pass fused with the first update and the norm, the Givens update of
// the Hessenberg column, the second update fused with the scaling into the
// next basis vector, the on-device step decision and the final x += Z y.  All
// reductions use a fixed grid, a fixed split of the vectors between blocks
// and a fixed summation tree, so results are bitwise reproducible run to run.
#include "elem.cuh"

namespace nmg {

namespace {

constexpr int kThreads = 256;

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

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes
// (coefficients scal[S_HC + i] + scal[S_Y + i], i <= j) and h_{j+1,j} = hnext:
// apply the earlier rotations, build rotation j, update g and write the
// residual estimate |g_{j+1}| / ||b||.  Called by a whole block: the inputs
// are first staged in shared memory by all threads (one memory latency
// instead of one per rotation), then thread 0 runs the serial recurrence.
// The other threads return at once.
__device__ void arnoldi_column(double* scal, int j, int m, double hnext) {
    __shared__ double sH[kMaxRestart + 2], scs[kMaxRestart], ssn[kMaxRestart];
    __shared__ double sg, sbn;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) sH[i] = scal[S_HC + i] + scal[S_Y + i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        scs[i] = scal[S_CS + i];
        ssn[i] = scal[S_SN + i];
    }
    if (threadIdx.x == 0) {
        sH[j + 1] = hnext;
        sg = scal[S_G + j];
        sbn = scal[S_BNORM];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double* H = scal + S_H + (int64_t)j * (m + 1);
    for (int i = 0; i < j; ++i) {
        const double a = sH[i], b = sH[i + 1];
        sH[i] = scs[i] * a + ssn[i] * b;
        sH[i + 1] = -ssn[i] * a + scs[i] * b;
    }
    const double a = sH[j], b = sH[j + 1];
    double c, s;
    if (b == 0.0) { c = a >= 0.0 ? 1.0 : -1.0; s = 0.0; }
    else { const double r = hypot(a, b); c = a / r; s = b / r; }
    for (int i = 0; i < j; ++i) H[i] = sH[i];
    H[j] = c * a + s * b;
    H[j + 1] = 0.0;
    scal[S_CS + j] = c;
    scal[S_SN + j] = s;
    scal[S_G + j + 1] = -s * sg;
    scal[S_G + j] = c * sg;
    const double est = fabs(-s * sg) / sbn;
    scal[S_EST] = est;
    if (!isfinite(est) || !isfinite(hnext)) scal[S_STATUS] = (double)NMG_ERR_NONFINITE;
    scal[S_ITER] += 1.0;
}

__global__ void k_start_cycle(double* scal, int m, int* cyc) {
    NMG_PDL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    cyc[0] = 0;
    cyc[2] = 0;
    for (int i = 0; i <= m; ++i) scal[S_G + i] = 0.0;
    const double beta = scal[S_BETA];
    scal[S_G] = beta;
    scal[S_INVH] = beta != 0.0 ? 1.0 / beta : 0.0;
    if (!isfinite(beta)) scal[S_STATUS] = (double)NMG_ERR_NONFINITE;
}

// y = H[:k,:k]^{-1} g[:k] by back substitution: the triangle and g are
// staged in shared memory by the block, then thread 0 substitutes.
__global__ void __launch_bounds__(kThreads) k_backsolve(double* scal, int k, int m) {
    NMG_PDL_ENTRY();
    __shared__ double sH[kMaxRestart * (kMaxRestart + 1)];
    __shared__ double sg[kMaxRestart], ys[kMaxRestart];
    const double* H = scal + S_H;
    for (int i = threadIdx.x; i < k * (m + 1); i += blockDim.x) sH[i] = H[i];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sg[i] = scal[S_G + i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double* y = scal + S_Y;
    for (int i = k - 1; i >= 0; --i) {
        double v = sg[i];
        for (int c = i + 1; c < k; ++c) v -= sH[c * (m + 1) + i] * ys[c];
        ys[i] = v / sH[i * (m + 1) + i];
        y[i] = ys[i];
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

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (unsigned)(b < 1 ? 1 : b);
}


// v[0] + ... + v[N-1] as a fixed pairwise tree (ceil(log2 N) dependent
// additions instead of N - 1: on GB300 a dependent FP64 addition costs tens of
// cycles, and these sums sit on the serial tail of the Arnoldi step).
template <int N>
__device__ __forceinline__ double tree_sum(double (&v)[N]) {
#pragma unroll
    for (int w = 1; w < N; w *= 2)
#pragma unroll
        for (int u = 0; u + w < N; u += 2 * w) v[u] += v[u + w];
    return v[0];
}

// The kDotBlocks partials of row k, lane-strided: lane l loads blocks l,
// l + 32, ... (all its loads issued together); row_sum then adds them.
constexpr int kRowPer = (kDotBlocks + 31) / 32;
__device__ __forceinline__ void load_row(const double* __restrict__ partial, int k, int lane, double (&v)[kRowPer]) {
#pragma unroll
    for (int r = 0; r < kRowPer; ++r) {
        const int b = lane + 32 * r;
        v[r] = b < kDotBlocks ? __ldcg(partial + (int64_t)k * kDotBlocks + b) : 0.0;
    }
}
// Sum of the loaded row: each lane's values as a tree, then a shuffle tree;
// valid in lane 0.
__device__ __forceinline__ double row_sum(double (&v)[kRowPer]) {
    double s = tree_sum<kRowPer>(v);
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

// Multi-dot machinery.  FP64 arithmetic is a scarce resource here (the FP64
// pipe of an SM retires about two operations per clock), so the reductions
// spend few FP64 additions: a thread accumulates up to 32 dot products, a warp
// reduces its 32 values by a transposing butterfly (31 additions per lane
// instead of 5 per value), the block adds its warps, and the last block sums
// the block partials in a fixed order.  Every block owns one contiguous,
// equal share of the vector (block_range), so the SMs finish together.
// Results are bitwise reproducible run to run.
constexpr int kMdThreads = 256;
constexpr int kMdWarps = kMdThreads / 32;
constexpr int kMdChunk = 32;   // vectors per pass over w
// row of the partial-sum buffer (rows of kDotBlocks doubles) holding the
// block sums of ||w||^2, after the two chunks of multi-dot partials
constexpr int kNormRow = 2 * kMdChunk;
static_assert((kMaxRestart + kMdChunk - 1) / kMdChunk <= 2 && kNormRow < kMaxRestart + 2,
              "two chunks of partials, then the norm row, inside the partial buffer");

// [lo, hi) = this block's share of n items (launched on kDotBlocks blocks).
__device__ __forceinline__ void block_range(int64_t n, int64_t& lo, int64_t& hi) {
    lo = n * blockIdx.x / gridDim.x;
    hi = n * (blockIdx.x + 1) / gridDim.x;
}

// Warp reduction of W per-lane values (W a power of two <= 32): a
// transposing butterfly over the offsets W/2 .. 1 (W - 1 additions per lane)
// leaves lane l with the sum of a[l % W] over the 32 / W lanes of its group,
// and the offsets W .. 16 complete it.  Afterwards lane l holds the warp's
// total of a[l % W].
template <int W>
__device__ __forceinline__ double butterfly(double (&a)[W], int lane) {
#pragma unroll
    for (int c = W / 2; c >= 1; c >>= 1) {
        const bool upper = (lane & c) != 0;
#pragma unroll
        for (int q = 0; q < c; ++q) {
            const double keep = upper ? a[c + q] : a[q];
            const double send = upper ? a[q] : a[c + q];
            a[q] = keep + __shfl_xor_sync(0xffffffffu, send, c);
        }
    }
    double v = a[0];
#pragma unroll
    for (int off = W; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Block totals of the W values -> partial[(chunk * grid + block) * 32 + l], l < W.
template <int W>
__device__ __forceinline__ void block_partials(double (&acc)[W], double* __restrict__ partial, int chunk, int lane,
                                               int warp) {
    __shared__ double red[kMdWarps][kMdChunk];
    const double v = butterfly<W>(acc, lane);
    if (lane < W) red[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && lane < W) {
        double f[kMdWarps];
#pragma unroll
        for (int ww = 0; ww < kMdWarps; ++ww) f[ww] = red[ww][lane];
        partial[((int64_t)chunk * gridDim.x + blockIdx.x) * kMdChunk + lane] = tree_sum<kMdWarps>(f);
    }
    __syncthreads();
}

// acc[k] = sum over this thread's elements i = lo + t, lo + t + 256, ... < hi
// of V_{c0+k}[i] w[i] for k < W (columns at or beyond c0 + nv contribute
// zeros: they are not read).  w may have been written earlier in the same
// kernel (by this block), so it is read through the L2 (ld.global.cg).
template <int W>
__device__ __forceinline__ void dots(const double* __restrict__ V, int64_t ldv, int c0, int nv, const double* w,
                                     int64_t lo, int64_t hi, double (&acc)[W]) {
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kMdThreads) {
        const double wi = __ldcg(w + i);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const double v = k < nv ? __ldg(V + (int64_t)(c0 + k) * ldv + i) : 0.0;
            acc[k] = fma(v, wi, acc[k]);
        }
    }
}

// One chunk of at most 32 dot products, with the accumulator width the
// smallest power of two >= nv (FP64 work not spent on absent vectors).
__device__ __forceinline__ void dots_chunk(const double* __restrict__ V, int64_t ldv, int c0, int nv, const double* w,
                                           int64_t lo, int64_t hi, double* __restrict__ partial, int chunk, int lane,
                                           int warp) {
#define NMG_DOTS(W)                                        \
    {                                                      \
        double acc[W];                                     \
        dots<W>(V, ldv, c0, nv, w, lo, hi, acc);           \
        block_partials<W>(acc, partial, chunk, lane, warp); \
    }
    if (nv > 16) NMG_DOTS(32)
    else if (nv > 8) NMG_DOTS(16)
    else if (nv > 4) NMG_DOTS(8)
    else if (nv > 2) NMG_DOTS(4)
    else if (nv > 1) NMG_DOTS(2)
    else NMG_DOTS(1)
#undef NMG_DOTS
}

// The nvec dot products of the current Arnoldi step for this block's share.
__device__ __forceinline__ void dots_all(const double* __restrict__ V, int64_t ldv, int nvec, const double* w,
                                         int64_t lo, int64_t hi, double* __restrict__ partial, int lane, int warp) {
    for (int c0 = 0, chunk = 0; c0 < nvec; c0 += kMdChunk, ++chunk)
        dots_chunk(V, ldv, c0, min(kMdChunk, nvec - c0), w, lo, hi, partial, chunk, lane, warp);
}

// In the last block: out[k] = sum over the blocks of the partials of value k
// (warp w sums the blocks w, w + kMdWarps, ... as a tree, then the warps'
// sums are added as a tree).  Launched on kDotBlocks blocks: a lane's loads
// are all issued before they are summed (one memory round trip for the whole
// tail).  Returns, in lane l of warp 0, the sum of out[k]^2 over k = l,
// l + 32, ... (fma in ascending k), for ||out||^2.
__device__ double finish_chunks(const double* __restrict__ partial, int nvec, double* __restrict__ out, int lane,
                                int warp) {
    __shared__ double fs[kMdWarps][kMdChunk];
    constexpr int G = kDotBlocks;
    constexpr int PER = (G + kMdWarps - 1) / kMdWarps;
    double sq = 0.0;
    for (int c0 = 0, chunk = 0; c0 < nvec; c0 += kMdChunk, ++chunk) {
        const double* p = partial + (int64_t)chunk * G * kMdChunk + lane;
        double v[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int b = warp + u * kMdWarps;
            v[u] = b < G ? __ldcg(p + (int64_t)b * kMdChunk) : 0.0;
        }
        fs[warp][lane] = tree_sum<PER>(v);
        __syncthreads();
        if (warp == 0 && c0 + lane < nvec) {
            double f[kMdWarps];
#pragma unroll
            for (int ww = 0; ww < kMdWarps; ++ww) f[ww] = fs[ww][lane];
            const double t = tree_sum<kMdWarps>(f);
            out[c0 + lane] = t;
            sq = fma(t, t, sq);
        }
        __syncthreads();
    }
    return sq;
}

// Outer product of step j = cyc[0] fused with the first Gram-Schmidt pass:
// Z_j = z (the V-cycle output xf, widened exactly to FP64), w = A z in FP64,
// and out[k] = V_k . w for k <= j.  Each block first computes w on its share
// of the nodes, then the dot products over the same unknowns.
template <typename TX, int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(kMdThreads)
k_spmv_zstore_dots(Geom g, const double* __restrict__ A, const TX* __restrict__ xf, double* __restrict__ Z,
                   double* w, const double* __restrict__ V, int64_t ldv, const int* __restrict__ cyc,
                   double* __restrict__ partial, double* __restrict__ out, unsigned* counter) {
    NMG_PDL_ENTRY();
    const int j = cyc[0], nvec = j + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* z64 = Z + (int64_t)j * ldv;
    int64_t lo, hi;
    block_range(g.nodes, lo, hi);
    for (int64_t i = lo + threadIdx.x; i < hi; i += kMdThreads) {
#pragma unroll
        for (int c = 0; c < NC; ++c) z64[i * NC + c] = elem::widen<double, TX>(xf[i * NC + c]);
        double acc[NC];
        elem::spmv_acc_f<double, DIM>(
            g, A,
            [&](int64_t jn, int, int, int, double* xv) {
#pragma unroll
                for (int c = 0; c < NC; ++c) xv[c] = elem::widen<double, TX>(xf[jn * NC + c]);
            },
            i, acc);
#pragma unroll
        for (int c = 0; c < NC; ++c) w[i * NC + c] = acc[c];
    }
    __syncthreads();   // the block's w is complete
    dots_all(V, ldv, nvec, w, lo * NC, hi * NC, partial, lane, warp);
    if (!last_block(counter)) return;
    finish_chunks(partial, nvec, out, lane, warp);
}

// Second Gram-Schmidt pass fused with the first update and the norm:
// w <- w - sum_k h1_k V_k (h1 = scal[S_HC..], the first pass), ||w||^2 and
// h2_k = V_k . w (into scal[S_Y..]); then, in the last block,
// h_{j+1,j} = ||w - V h2|| = sqrt(||w||^2 - ||h2||^2) (Pythagoras: the V_k
// are orthonormal, as in low-synchronisation CGS2) and its reciprocal, which
// the next kernel scales by.  Each thread reads back only the elements it
// wrote.  The Givens update of column j runs in the next kernel.
__global__ void __launch_bounds__(kMdThreads)
k_gs_update_dot_norm(const double* __restrict__ V, int64_t ldv, const int* __restrict__ cyc, double* w, int64_t n,
                     double* __restrict__ partial, double* scal, int m, unsigned* counter) {
    NMG_PDL_ENTRY();
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double red[kMdWarps];
    __shared__ double s_hnext;
    const int j = cyc[0], nvec = j + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < nvec; k += kMdThreads) hs[k] = scal[S_HC + k];
    __syncthreads();
    int64_t lo, hi;
    block_range(n, lo, hi);
    double ww = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kMdThreads) {
        double v = w[i];
#pragma unroll 8
        for (int k = 0; k < nvec; ++k) v = fma(-hs[k], V[(int64_t)k * ldv + i], v);
        w[i] = v;
        ww = fma(v, v, ww);
    }
    for (int off = 16; off > 0; off >>= 1) ww += __shfl_down_sync(0xffffffffu, ww, off);
    if (lane == 0) red[warp] = ww;
    __syncthreads();
    if (threadIdx.x == 0) {
        double f[kMdWarps];
#pragma unroll
        for (int k = 0; k < kMdWarps; ++k) f[k] = red[k];
        partial[(int64_t)kNormRow * kDotBlocks + blockIdx.x] = tree_sum<kMdWarps>(f);
    }
    dots_all(V, ldv, nvec, w, lo, hi, partial, lane, warp);
    if (!last_block(counter)) return;
    // warp 0's loads of the ||w||^2 partials are in flight while the chunks are summed
    double nrow[kRowPer];
    if (warp == 0) load_row(partial, kNormRow, lane, nrow);
    // h2 into scal[S_Y..]; lane l of warp 0 gets h2_l^2 + h2_{l+32}^2 (ascending k)
    double hh = finish_chunks(partial, nvec, scal + S_Y, lane, warp);   // ends with a block barrier
    if (warp == 0) {
        const double t = row_sum(nrow);
        // ||h2||^2: the lanes' squares added by a fixed shuffle tree
        for (int off = 16; off > 0; off >>= 1) hh += __shfl_down_sync(0xffffffffu, hh, off);
        if (lane == 0) {
            const double d = t - hh;
            s_hnext = d > 0.0 ? sqrt(d) : 0.0;
            scal[S_HC + j + 1] = s_hnext;
            scal[S_INVH] = s_hnext != 0.0 ? 1.0 / s_hnext : 0.0;
        }
    }
    (void)m;
}

// Second update fused with the scaling: v_{j+1} = (w - sum_k h2_k V_k) *
// scal[S_INVH] into basis column j + 1 and, converted, into vin (the
// right-hand side of the next V-cycle).  Block 0 also runs the Givens update
// of column j (arnoldi_column): a serial chain of dependent FP64 operations
// (about 8 us on GB300) that only the decision after this kernel needs, so
// it overlaps the streaming update instead of delaying it.
template <typename TV>
__global__ void __launch_bounds__(kThreads)
k_gs_update_scale(double* V, int64_t ldv, const int* __restrict__ cyc, double* scal,
                  const double* __restrict__ w, TV* __restrict__ vin, int64_t n, int m) {
    NMG_PDL_ENTRY();
    __shared__ double hs[kMaxRestart + 1];
    const int j = cyc[0], nvec = j + 1;
    for (int k = threadIdx.x; k < nvec; k += kThreads) hs[k] = scal[S_Y + k];
    __syncthreads();
    const double a = scal[S_INVH];
    if (blockIdx.x == 0) arnoldi_column(scal, j, m, scal[S_HC + j + 1]);
    double* y = V + (int64_t)(j + 1) * ldv;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double v = w[i];
#pragma unroll 8
        for (int k = 0; k < nvec; ++k) v = fma(-hs[k], V[(int64_t)k * ldv + i], v);
        const double sv = a * v;
        y[i] = sv;
        vin[i] = (TV)sv;
    }
}

// v = x * scal[S_INVH] into the Krylov basis (column cyc[0] + 1 when next,
// else column 0) and its copy in the V-cycle's arithmetic type TV (the
// right-hand side of the next V-cycle).
template <typename TV>
__global__ void k_scale_convert(const double* __restrict__ x, const double* __restrict__ sp, double* __restrict__ V,
                                int64_t ldv, const int* __restrict__ cyc, bool next, TV* __restrict__ vin, int64_t n) {
    NMG_PDL_ENTRY();
    const double a = *sp;
    double* y = V + (next ? (int64_t)(cyc[0] + 1) * ldv : 0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a * x[i];
        y[i] = v;
        vin[i] = (TV)v;
    }
}

// End of one Arnoldi step: counts the iteration and decides on the device
// whether the cycle goes on (estimate above rtol, iterations below maxit, no
// breakdown, no non-finite value, basis not full); cyc[2] = 1 once it stops.
// Inside a graph loop the decision also sets the loop's condition.
__global__ void k_decide(const double* __restrict__ scal, int* cyc, double rtol, int maxit, int m,
                         cudaGraphConditionalHandle loop, bool in_loop) {
    NMG_PDL_ENTRY();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = cyc[0];
    const int its = cyc[1] + 1;
    cyc[1] = its;
    const bool stop = scal[S_STATUS] != 0.0 || scal[S_EST] <= rtol || its >= maxit || scal[S_INVH] == 0.0 ||
                      j + 1 >= m;
    cyc[2] = stop ? 1 : 0;
    if (!stop) cyc[0] = j + 1;
    if (in_loop) cudaGraphSetConditional(loop, stop ? 0u : 1u);
}

}  // namespace

void launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t s) {
    g_launches += 2;
    pdl_launch(k_sumsq_partial, dim3(kDotBlocks), dim3(kThreads), 0, s, x, n, partial);
    pdl_launch(k_finish_dots, dim3(1), dim3(32), 0, s, partial, 1, out, false, true);
}

void launch_start_cycle(double* scal, int m, int* cyc, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_start_cycle, dim3(1), dim3(32), 0, s, scal, m, cyc);
}

void launch_solve_update(double* scal, int k, int m, const double* Z, int64_t ldz, double* x, int64_t n,
                         cudaStream_t s) {
    g_launches += 2;
    pdl_launch(k_backsolve, dim3(1), dim3(kThreads), 0, s, scal, k, m);
    pdl_launch(k_update_x, dim3(grid_for(n)), dim3(kThreads), 0, s, scal, k, Z, ldz, x, n);
}

}  // namespace nmg

namespace nmg {

template <typename TX>
void launch_spmv_zstore_dots(const Geom& g, const double* A, const TX* xf, double* Z, double* w, const double* V,
                             int64_t ldv, const int* cyc, double* partial, double* out, unsigned* counter,
                             cudaStream_t s) {
    g_launches += 1;
    const bool lean = g.nc == g.dim;   // n_c = d: the vector problems (ALE extension)
    if (g.dim == 2)
        pdl_launch(lean ? k_spmv_zstore_dots<TX, 2, 2> : k_spmv_zstore_dots<TX, 2, 3>, dim3(kDotBlocks),
                   dim3(kMdThreads), 0, s, g, A, xf, Z, w, V, ldv, cyc, partial, out, counter);
    else
        pdl_launch(lean ? k_spmv_zstore_dots<TX, 3, 3> : k_spmv_zstore_dots<TX, 3, 4>, dim3(kDotBlocks),
                   dim3(kMdThreads), 0, s, g, A, xf, Z, w, V, ldv, cyc, partial, out, counter);
}
template void launch_spmv_zstore_dots<float>(const Geom&, const double*, const float*, double*, double*,
                                             const double*, int64_t, const int*, double*, double*, unsigned*,
                                             cudaStream_t);
template void launch_spmv_zstore_dots<double>(const Geom&, const double*, const double*, double*, double*,
                                              const double*, int64_t, const int*, double*, double*, unsigned*,
                                              cudaStream_t);

void launch_gs_update_dot_norm(const double* V, int64_t ldv, const int* cyc, double* w, int64_t n, double* partial,
                               double* scal, int m, unsigned* counter, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_gs_update_dot_norm, dim3(kDotBlocks), dim3(kMdThreads), 0, s, V, ldv, cyc, w, n, partial, scal, m,
               counter);
}

template <typename TV>
void launch_gs_update_scale(double* V, int64_t ldv, const int* cyc, double* scal, const double* w, TV* vin,
                            int64_t n, int m, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_gs_update_scale<TV>, dim3(grid_for(n)), dim3(kThreads), 0, s, V, ldv, cyc, scal, w, vin, n, m);
}
template void launch_gs_update_scale<float>(double*, int64_t, const int*, double*, const double*, float*,
                                            int64_t, int, cudaStream_t);
template void launch_gs_update_scale<double>(double*, int64_t, const int*, double*, const double*, double*,
                                             int64_t, int, cudaStream_t);

template <typename TV>
void launch_scale_convert(const double* x, const double* scal_ptr, double* V, int64_t ldv, const int* cyc, bool next,
                          TV* vin, int64_t n, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_scale_convert<TV>, dim3(grid_for(n)), dim3(256), 0, s, x, scal_ptr, V, ldv, cyc, next, vin, n);
}
template void launch_scale_convert<float>(const double*, const double*, double*, int64_t, const int*, bool, float*,
                                          int64_t, cudaStream_t);
template void launch_scale_convert<double>(const double*, const double*, double*, int64_t, const int*, bool, double*,
                                           int64_t, cudaStream_t);

void launch_decide(const double* scal, int* cyc, double rtol, int maxit, int m, cudaGraphConditionalHandle loop,
                   bool in_loop, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_decide, dim3(1), dim3(32), 0, s, scal, cyc, rtol, maxit, m, loop, in_loop);
}

}  // namespace nmg
