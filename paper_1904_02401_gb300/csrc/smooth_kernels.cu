// Solve-phase kernels of the multigrid V-cycle (Section 4.3 (II)-(III)):
// block-sparse residual products, the additive Vanka patch step of Eq. (vanka),
// Q1 restriction / prolongation and the coarse solve.  Every kernel is
// memory-bound; the data layouts are chosen so that warps read contiguous,
// coalesced segments of the matrix and of the patch inverses.
#include "nmg_internal.cuh"

namespace nmg {

namespace {

template <typename TS> __device__ __forceinline__ float to_f(TS v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename TS> struct Load;
template <> struct Load<double, double> {
    static __device__ __forceinline__ double get(const double* p) { return __ldg(p); }
};
template <> struct Load<float, float> {
    static __device__ __forceinline__ float get(const float* p) { return __ldg(p); }
};
template <> struct Load<float, __nv_bfloat16> {
    static __device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(*p); }
};

__device__ __forceinline__ void node_xyz(const Geom& g, int64_t i, int& x, int& y, int& z) {
    x = (int)(i % g.nn[0]);
    int64_t t = i / g.nn[0];
    y = (int)(t % g.nn[1]);
    z = (int)(t / g.nn[1]);
}

// y = A x  or  y = b - A x, one thread per node.  A in stencil layout.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_spmv(Geom g, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
       T* __restrict__ y, bool residual) {
    constexpr int NC = DIM + 1;
    constexpr int NB = NC * NC;
    constexpr int NST = (DIM == 2) ? 9 : 27;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.nodes) return;
    int ix, iy, iz;
    node_xyz(g, i, ix, iy, iz);
    const int64_t sy = g.nn[0], sz = (int64_t)g.nn[0] * g.nn[1];
    T acc[NC];
#pragma unroll
    for (int r = 0; r < NC; ++r) acc[r] = T(0);
#pragma unroll
    for (int s = 0; s < NST; ++s) {
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
        const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                        (iz + dz >= 0) && (iz + dz < g.nn[2]);
        if (ok) {
            const int64_t j = i + dx + dy * sy + dz * sz;
            T xv[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) xv[c] = x[j * NC + c];
            const T* As = A + (int64_t)s * NB * g.ld + i;
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[r] = fma(__ldg(As + (int64_t)(r * NC + c) * g.ld), xv[c], acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) y[i * NC + r] = residual ? b[i * NC + r] - acc[r] : acc[r];
}

// corr_i = A_i^{-1} R_i d for every patch i: one warp per patch.  The patch
// inverse is column-major, so for each column j the 32 lanes read 32
// consecutive entries (one coalesced 128-byte segment in FP32) and multiply
// them by the broadcast d_j from shared memory; no cross-lane reduction.
template <typename T, typename TS, int DIM, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_vanka_apply(Geom g, const TS* __restrict__ inv, int64_t stride, const T* __restrict__ d,
              T* __restrict__ corr) {
    constexpr int NC = DIM + 1;
    constexpr int NN = (DIM == 2) ? 9 : 27;
    constexpr int NP = NN * NC;
    constexpr int NQ = (NP + 31) / 32;
    __shared__ T sd[WARPS][NP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * WARPS + w;
    if (p >= g.patches) return;
    const int px = (int)(p % g.pc[0]);
    const int py = (int)((p / g.pc[0]) % g.pc[1]);
    const int pz = (int)(p / ((int64_t)g.pc[0] * g.pc[1]));
    for (int t = lane; t < NP; t += 32) {
        const int an = t / NC, c = t - an * NC;
        const int ax = an % 3, ay = (an / 3) % 3, az = an / 9;
        const int64_t node = (int64_t)(2 * px + ax) +
                             (int64_t)g.nn[0] * ((2 * py + ay) + (int64_t)g.nn[1] * (2 * pz + az));
        sd[w][t] = d[node * NC + c];
    }
    __syncwarp();
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    const TS* Ap = inv + p * stride;
#pragma unroll 4
    for (int j = 0; j < NP; ++j) {
        const T dj = sd[w][j];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int row = lane + 32 * q;
            if (row < NP) acc[q] = fma((T)Load<T, TS>::get(Ap + (int64_t)j * NP + row), dj, acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int row = lane + 32 * q;
        if (row < NP) corr[p * NP + row] = acc[q];
    }
}

// x += w(node) * sum over the patches that contain the node of their
// corrections (fixed order: ascending patch index), w = omega / multiplicity
// ("average") or omega ("sum").  One thread per node, no atomics.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_vanka_update(Geom g, const T* __restrict__ corr, T* __restrict__ x, bool x_zero, T omega,
               bool average) {
    constexpr int NC = DIM + 1;
    constexpr int NN = (DIM == 2) ? 9 : 27;
    constexpr int NP = NN * NC;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.nodes) return;
    int xyz[3];
    node_xyz(g, i, xyz[0], xyz[1], xyz[2]);
    int cp[3][2], cl[3][2], cnt[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = xyz[k];
        if (k >= DIM) { cp[k][0] = 0; cl[k][0] = 0; cnt[k] = 1; continue; }
        if (c & 1) { cp[k][0] = (c - 1) >> 1; cl[k][0] = 1; cnt[k] = 1; }
        else {
            int n = 0;
            if (c > 0) { cp[k][n] = (c >> 1) - 1; cl[k][n] = 2; ++n; }
            if (c < g.cells[k]) { cp[k][n] = c >> 1; cl[k][n] = 0; ++n; }
            cnt[k] = n;
        }
    }
    T sum[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sum[c] = T(0);
    for (int a = 0; a < cnt[2]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
            for (int e = 0; e < cnt[0]; ++e) {
                const int64_t p = cp[0][e] + (int64_t)g.pc[0] * (cp[1][b] + (int64_t)g.pc[1] * cp[2][a]);
                const int loc = cl[0][e] + 3 * cl[1][b] + 9 * cl[2][a];
                const T* cpn = corr + p * NP + loc * NC;
#pragma unroll
                for (int c = 0; c < NC; ++c) sum[c] += cpn[c];
            }
    const int m = cnt[0] * cnt[1] * cnt[2];
    const T wgt = average ? omega / T(m) : omega;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const T old = x_zero ? T(0) : x[i * NC + c];
        x[i * NC + c] = old + wgt * sum[c];
    }
}

// r_c = P^T r_f (Q1 full weighting), coarse Dirichlet entries zero.  One thread per coarse node.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_restrict(Geom f, Geom c, const T* __restrict__ rf, T* __restrict__ rc, const uint8_t* __restrict__ cmask) {
    constexpr int NC = DIM + 1;
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= c.nodes) return;
    int X, Y, Z;
    node_xyz(c, I, X, Y, Z);
    T sum[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) sum[k] = T(0);
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    for (int oz = zlo; oz <= zhi; ++oz) {
        const int fz = 2 * Z + oz;
        if (fz < 0 || fz >= f.nn[2]) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            const int fy = 2 * Y + oy;
            if (fy < 0 || fy >= f.nn[1]) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int fx = 2 * X + ox;
                if (fx < 0 || fx >= f.nn[0]) continue;
                const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
                const int64_t fi = fx + (int64_t)f.nn[0] * (fy + (int64_t)f.nn[1] * fz);
#pragma unroll
                for (int k = 0; k < NC; ++k) sum[k] = fma(w, rf[fi * NC + k], sum[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) rc[I * NC + k] = cmask[I * NC + k] ? T(0) : sum[k];
}

// x_f += P e_c (Q1 interpolation), fine Dirichlet entries untouched.  One thread per fine node.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
k_prolong_add(Geom f, Geom c, const T* __restrict__ ec, T* __restrict__ xf, const uint8_t* __restrict__ fmask) {
    constexpr int NC = DIM + 1;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.nodes) return;
    int xyz[3];
    node_xyz(f, i, xyz[0], xyz[1], xyz[2]);
    int ci[3][2], cnt[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int v = xyz[k];
        if (k >= DIM || !(v & 1)) { ci[k][0] = v >> 1; cnt[k] = 1; }
        else { ci[k][0] = (v - 1) >> 1; ci[k][1] = (v + 1) >> 1; cnt[k] = 2; }
    }
    T sum[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) sum[k] = T(0);
    for (int a = 0; a < cnt[2]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
            for (int e = 0; e < cnt[0]; ++e) {
                const T w = (cnt[0] == 2 ? T(0.5) : T(1)) * (cnt[1] == 2 ? T(0.5) : T(1)) *
                            (cnt[2] == 2 ? T(0.5) : T(1));
                const int64_t I = ci[0][e] + (int64_t)c.nn[0] * (ci[1][b] + (int64_t)c.nn[1] * ci[2][a]);
#pragma unroll
                for (int k = 0; k < NC; ++k) sum[k] = fma(w, ec[I * NC + k], sum[k]);
            }
#pragma unroll
    for (int k = 0; k < NC; ++k)
        if (!fmask[i * NC + k]) xf[i * NC + k] += sum[k];
}

// x = inv * b with the FP64 dense coarse inverse, one warp per row, FP64 sums.
template <typename T>
__global__ void __launch_bounds__(256)
k_coarse_gemv(const double* __restrict__ inv, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s = fma(inv[row * n + j], (double)b[j], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) x[row] = (T)s;
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)in[i];
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

template <typename T>
void launch_spmv(const Geom& g, const T* A, const T* x, const T* b, T* y, bool residual, cudaStream_t s) {
    g_launches += 1;
    if (g.dim == 2) k_spmv<T, 2><<<blocks_for(g.nodes, 256), 256, 0, s>>>(g, A, x, b, y, residual);
    else k_spmv<T, 3><<<blocks_for(g.nodes, 256), 256, 0, s>>>(g, A, x, b, y, residual);
}

template <typename T, typename TS>
void launch_vanka_apply(const Geom& g, const TS* inv, int64_t stride, const T* d, T* corr, cudaStream_t s) {
    g_launches += 1;
    constexpr int W = 4;
    const unsigned grid = (unsigned)((g.patches + W - 1) / W);
    if (g.dim == 2) k_vanka_apply<T, TS, 2, W><<<grid, W * 32, 0, s>>>(g, inv, stride, d, corr);
    else k_vanka_apply<T, TS, 3, W><<<grid, W * 32, 0, s>>>(g, inv, stride, d, corr);
}

template <typename T>
void launch_vanka_update(const Geom& g, const T* corr, T* x, bool x_zero, T omega, bool average, cudaStream_t s) {
    g_launches += 1;
    if (g.dim == 2) k_vanka_update<T, 2><<<blocks_for(g.nodes, 256), 256, 0, s>>>(g, corr, x, x_zero, omega, average);
    else k_vanka_update<T, 3><<<blocks_for(g.nodes, 256), 256, 0, s>>>(g, corr, x, x_zero, omega, average);
}

template <typename T>
void launch_restrict(const Geom& f, const Geom& c, const T* rf, T* rc, const uint8_t* cmask, cudaStream_t s) {
    g_launches += 1;
    if (f.dim == 2) k_restrict<T, 2><<<blocks_for(c.nodes, 256), 256, 0, s>>>(f, c, rf, rc, cmask);
    else k_restrict<T, 3><<<blocks_for(c.nodes, 256), 256, 0, s>>>(f, c, rf, rc, cmask);
}

template <typename T>
void launch_prolong_add(const Geom& f, const Geom& c, const T* ec, T* xf, const uint8_t* fmask, cudaStream_t s) {
    g_launches += 1;
    if (f.dim == 2) k_prolong_add<T, 2><<<blocks_for(f.nodes, 256), 256, 0, s>>>(f, c, ec, xf, fmask);
    else k_prolong_add<T, 3><<<blocks_for(f.nodes, 256), 256, 0, s>>>(f, c, ec, xf, fmask);
}

template <typename T>
void launch_coarse_gemv(const double* inv, int64_t n, const T* b, T* x, cudaStream_t s) {
    g_launches += 1;
    k_coarse_gemv<T><<<blocks_for(n * 32, 256), 256, 0, s>>>(inv, n, b, x);
}

template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, int64_t n, cudaStream_t s) {
    g_launches += 1;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_convert<TI, TO><<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
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
