// Set-up kernels: matrix layout conversion, Vanka patch extraction and exact
// inversion (Section 4.3: A_i = R_i A R_i^T, "inverted exactly"), coarse
// matrix inversion.  All set-up arithmetic is FP64.
#include <algorithm>

#include "nmg_internal.cuh"

namespace nmg {

namespace {

__device__ __forceinline__ void node_xyz(const Geom& g, int64_t i, int& x, int& y, int& z) {
    x = (int)(i % g.nn[0]);
    int64_t t = i / g.nn[0];
    y = (int)(t % g.nn[1]);
    z = (int)(t / g.nn[1]);
}

// One thread per block row: scatter the BSR blocks of node i into the stencil
// slots (s, e).  Flags columns outside the Q1 stencil, duplicates and NaN/Inf.
__global__ void k_bsr_to_stencil(Geom g, const int64_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, const double* __restrict__ vals,
                                 int64_t nnzb, double* __restrict__ A, int* flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.nodes) return;
    const int nb = g.nc * g.nc;
    int ix, iy, iz;
    node_xyz(g, i, ix, iy, iz);
    int64_t k0 = rp[i], k1 = rp[i + 1];
    if (k0 < 0 || k1 < k0 || k1 > nnzb) {
        atomicOr(&flags[FLAG_BAD_PATTERN], 1);
        return;
    }
    uint32_t seen = 0;
    for (int64_t k = k0; k < k1; ++k) {
        int64_t j = ci[k];
        if (j < 0 || j >= g.nodes) { atomicOr(&flags[FLAG_BAD_PATTERN], 1); continue; }
        int jx, jy, jz;
        node_xyz(g, j, jx, jy, jz);
        int dx = jx - ix, dy = jy - iy, dz = jz - iz;
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) {
            atomicOr(&flags[FLAG_BAD_PATTERN], 1);
            continue;
        }
        int s = (dx + 1) + 3 * (dy + 1) + (g.dim == 3 ? 9 * (dz + 1) : 0);
        if ((seen >> s) & 1u) { atomicOr(&flags[FLAG_BAD_PATTERN], 1); continue; }
        seen |= 1u << s;
        for (int e = 0; e < nb; ++e) {
            double v = vals[k * nb + e];
            if (!isfinite(v)) atomicOr(&flags[FLAG_NONFINITE], 1);
            A[stencil_off(g.dim, nb, g.ld, s, e, i)] = v;
        }
    }
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// Gauss-Jordan inversion with partial pivoting of the NP x NP matrix a (leading
// dimension LDA) held in shared memory, in place.  perm, col: NP scratch.
// Returns through *singular whether a zero or non-finite pivot appeared.
template <int NP, int LDA>
__device__ void gauss_jordan_smem(double* a, double* col, int* perm, int* s_piv, double* s_pval,
                                  bool* singular) {
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    for (int k = 0; k < NP; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < NP; i += 32) {
                double v = fabs(a[i * LDA + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                double ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                *s_piv = bi;
                perm[k] = bi;
                double pv = a[bi * LDA + k];
                if (pv == 0.0 || !isfinite(pv)) {
                    *singular = true;
                    pv = 1.0;   // keep the arithmetic finite; the caller reports the patch
                    a[bi * LDA + k] = 1.0;
                }
                *s_pval = pv;
            }
        }
        __syncthreads();
        const int piv = *s_piv;
        if (piv != k) {
            for (int j = tid; j < NP; j += nthr) {
                double t = a[k * LDA + j];
                a[k * LDA + j] = a[piv * LDA + j];
                a[piv * LDA + j] = t;
            }
        }
        __syncthreads();
        const double inv = 1.0 / *s_pval;
        for (int i = tid; i < NP; i += nthr) col[i] = a[i * LDA + k];
        __syncthreads();
        for (int j = tid; j < NP; j += nthr) a[k * LDA + j] = (j == k ? 1.0 : a[k * LDA + j]) * inv;
        __syncthreads();
        for (int idx = tid; idx < NP * NP; idx += nthr) {
            const int i = idx / NP;
            const int j = idx - i * NP;
            if (i != k) a[i * LDA + j] = (j == k ? 0.0 : a[i * LDA + j]) - col[i] * a[k * LDA + j];
        }
        __syncthreads();
    }
    for (int k = NP - 1; k >= 0; --k) {
        const int pk = perm[k];
        if (pk != k) {
            for (int i = tid; i < NP; i += nthr) {
                double t = a[i * LDA + k];
                a[i * LDA + k] = a[i * LDA + pk];
                a[i * LDA + pk] = t;
            }
        }
        __syncthreads();
    }
}

// Persistent launch over all patches of a level: gather A_i from the stencil
// matrix, invert it, store A_i^{-1} column-major in every requested precision.
template <int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(256)
k_patch_invert(Geom g, const double* __restrict__ A, double* inv64, int64_t s64, float* inv32,
               int64_t s32, __nv_bfloat16* invbf, int64_t sbf, int* flags, int64_t npatch,
               const int32_t* __restrict__ ids) {
    constexpr int NN = (DIM == 2) ? 9 : 27;      // nodes per patch
    constexpr int NP = NN * NC;
    constexpr int LDA = NP + 1;
    extern __shared__ double smem[];
    double* a = smem;
    double* col = a + NP * LDA;
    int* perm = reinterpret_cast<int*>(col + NP);
    __shared__ int s_piv;
    __shared__ double s_pval;
    __shared__ bool s_sing;
    const int tid = threadIdx.x;
    for (int64_t p = blockIdx.x; p < npatch; p += gridDim.x) {
        const int64_t q = ids ? (int64_t)ids[p] : p;     // index on the regular patch grid
        const int px = (int)(q % g.pc[0]);
        const int py = (int)((q / g.pc[0]) % g.pc[1]);
        const int pz = (int)(q / ((int64_t)g.pc[0] * g.pc[1]));
        if (tid == 0) s_sing = false;
        for (int idx = tid; idx < NP * NP; idx += blockDim.x) {
            const int row = idx / NP, cl = idx - row * NP;
            const int an = row / NC, r = row - an * NC;
            const int bn = cl / NC, c = cl - bn * NC;
            const int ax = an % 3, ay = (an / 3) % 3, az = an / 9;
            const int bx = bn % 3, by = (bn / 3) % 3, bz = bn / 9;
            const int dx = bx - ax, dy = by - ay, dz = bz - az;
            double v = 0.0;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) {
                const int s = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
                const int64_t node = (int64_t)(2 * px + ax) +
                                     (int64_t)g.nn[0] * ((2 * py + ay) + (int64_t)g.nn[1] * (2 * pz + az));
                v = A[stencil_off<DIM, NC * NC>(g.ld, s, r * NC + c, node)];
            }
            a[row * LDA + cl] = v;
        }
        __syncthreads();
        gauss_jordan_smem<NP, LDA>(a, col, perm, &s_piv, &s_pval, &s_sing);
        if (tid == 0 && s_sing) atomicOr(&flags[FLAG_SINGULAR], 1);
        for (int idx = tid; idx < NP * NP; idx += blockDim.x) {
            const int j = idx / NP, i = idx - j * NP;          // column-major output
            const double v = a[i * LDA + j];
            if (inv64) inv64[p * s64 + idx] = v;
            if (inv32) inv32[p * s32 + idx] = (float)v;
            if (invbf) invbf[p * sbf + idx] = __double2bfloat16(v);
        }
        __syncthreads();
    }
}

// Large patches (blocks of 4^d cells, 5^d nodes): A_P gathered from the
// stencil matrix (nodes more than one apart in a direction do not couple),
// inverted by the Gauss-Jordan elimination with partial pivoting above and
// stored column-major in every requested precision.  2d (75 or 50 unknowns):
// the matrix in shared memory; 3d (500 or 375 unknowns, 2 MB in FP64): in a
// global work matrix of the CTA (L2-resident), the pivot column and
// permutation in shared memory.  org[p]: the patch's lowest 2^d-cell block on
// the regular patch grid.
template <int DIM, int NC, bool SMEM>
__global__ void __launch_bounds__(SMEM ? 256 : 1024)
k_patch_invert_large(Geom g, const double* __restrict__ A, const int32_t* __restrict__ org, int64_t npatch,
                     double* work, double* inv64, int64_t s64, float* inv32, int64_t s32, __nv_bfloat16* invbf,
                     int64_t sbf, int* flags) {
    constexpr int NN = (DIM == 2) ? 25 : 125;
    constexpr int NP = NN * NC;
    constexpr int LDA = SMEM ? NP + 1 : NP;
    extern __shared__ double smem[];
    double* a = SMEM ? smem : work + (int64_t)blockIdx.x * NP * LDA;
    double* col = SMEM ? smem + NP * LDA : smem;
    int* perm = reinterpret_cast<int*>(col + NP);
    __shared__ int s_piv;
    __shared__ double s_pval;
    __shared__ bool s_sing;
    const int tid = threadIdx.x;
    for (int64_t p = blockIdx.x; p < npatch; p += gridDim.x) {
        const int64_t q = org[p];
        const int px = (int)(q % g.pc[0]);
        const int py = (int)((q / g.pc[0]) % g.pc[1]);
        const int pz = (int)(q / ((int64_t)g.pc[0] * g.pc[1]));
        if (tid == 0) s_sing = false;
        for (int idx = tid; idx < NP * NP; idx += blockDim.x) {
            const int row = idx / NP, cl = idx - row * NP;
            const int an = row / NC, r = row - an * NC;
            const int bn = cl / NC, c = cl - bn * NC;
            const int ax = an % 5, ay = (an / 5) % 5, az = an / 25;
            const int bx = bn % 5, by = (bn / 5) % 5, bz = bn / 25;
            const int dx = bx - ax, dy = by - ay, dz = bz - az;
            double v = 0.0;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) {
                const int s = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
                const int64_t node = (int64_t)(2 * px + ax) +
                                     (int64_t)g.nn[0] * ((2 * py + ay) + (int64_t)g.nn[1] * (2 * pz + az));
                v = A[stencil_off<DIM, NC * NC>(g.ld, s, r * NC + c, node)];
            }
            a[(int64_t)row * LDA + cl] = v;
        }
        __syncthreads();
        gauss_jordan_smem<NP, LDA>(a, col, perm, &s_piv, &s_pval, &s_sing);
        if (tid == 0 && s_sing) atomicOr(&flags[FLAG_SINGULAR], 1);
        for (int idx = tid; idx < NP * NP; idx += blockDim.x) {
            const int j = idx / NP, i = idx - j * NP;          // column-major output
            const double v = a[(int64_t)i * LDA + j];
            if (inv64) inv64[p * s64 + idx] = v;
            if (inv32) inv32[p * s32 + idx] = (float)v;
            if (invbf) invbf[p * sbf + idx] = __double2bfloat16(v);
        }
        __syncthreads();
    }
}

// Dense coarse matrix (row-major n0 x n0) from the stencil matrix.
__global__ void k_coarse_assemble(Geom g, const double* __restrict__ A, double* __restrict__ D) {
    const int nc = g.nc;
    const int64_t n = g.nodes * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.nodes * g.nst * nc * nc;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % g.nodes;
        const int64_t rest = t / g.nodes;
        const int e = (int)(rest % (nc * nc));
        const int s = (int)(rest / (nc * nc));
        const int r = e / nc, c = e % nc;
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = g.dim == 3 ? s / 9 - 1 : 0;
        int ix, iy, iz;
        node_xyz(g, i, ix, iy, iz);
        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        if (jx < 0 || jx >= g.nn[0] || jy < 0 || jy >= g.nn[1] || jz < 0 || jz >= g.nn[2]) continue;
        const int64_t j = jx + (int64_t)g.nn[0] * (jy + (int64_t)g.nn[1] * jz);
        D[(i * nc + r) * n + j * nc + c] = A[stencil_off(g.dim, nc * nc, g.ld, s, e, i)];
    }
}

// Single-CTA Gauss-Jordan inversion in global memory (coarse level, n <= 2048).
__global__ void __launch_bounds__(1024) k_dense_invert(double* a, int64_t n, int* perm, int* flags) {
    __shared__ int s_piv;
    __shared__ double s_pval;
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    extern __shared__ double col[];    // n doubles
    for (int64_t k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = (int)k;
        for (int64_t i = k + tid; i < n; i += nthr) {
            double v = fabs(a[i * n + k]);
            if (v > best) { best = v; bi = (int)i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            double ob = __shfl_down_sync(0xffffffffu, best, off);
            int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nwarp; ++w)
                if (red_v[w] > best || (red_v[w] == best && red_i[w] < bi)) { best = red_v[w]; bi = red_i[w]; }
            s_piv = bi;
            perm[k] = bi;
            double pv = a[(int64_t)bi * n + k];
            if (pv == 0.0 || !isfinite(pv)) {
                atomicOr(&flags[FLAG_SINGULAR], 1);
                pv = 1.0;
                a[(int64_t)bi * n + k] = 1.0;
            }
            s_pval = pv;
        }
        __syncthreads();
        const int64_t piv = s_piv;
        if (piv != k)
            for (int64_t j = tid; j < n; j += nthr) {
                double t = a[k * n + j];
                a[k * n + j] = a[piv * n + j];
                a[piv * n + j] = t;
            }
        __syncthreads();
        const double inv = 1.0 / s_pval;
        for (int64_t i = tid; i < n; i += nthr) col[i] = a[i * n + k];
        __syncthreads();
        for (int64_t j = tid; j < n; j += nthr) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * inv;
        __syncthreads();
        for (int64_t idx = tid; idx < n * n; idx += nthr) {
            const int64_t i = idx / n, j = idx - i * n;
            if (i != k) a[idx] = (j == k ? 0.0 : a[idx]) - col[i] * a[k * n + j];
        }
        __syncthreads();
    }
    for (int64_t k = n - 1; k >= 0; --k) {
        const int64_t pk = perm[k];
        if (pk != k)
            for (int64_t i = tid; i < n; i += nthr) {
                double t = a[i * n + k];
                a[i * n + k] = a[i * n + pk];
                a[i * n + pk] = t;
            }
        __syncthreads();
    }
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

void launch_bsr_to_stencil(const Geom& g, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* vals, int64_t nnzb, double* A64, int* flags, cudaStream_t s) {
    g_launches += 1;
    const int threads = 128;
    const int64_t blocks = (g.nodes + threads - 1) / threads;
    k_bsr_to_stencil<<<(unsigned)blocks, threads, 0, s>>>(g, row_ptr, col_idx, vals, nnzb, A64, flags);
}

void launch_convert_f64_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
    g_launches += 1;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    k_f64_to_f32<<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
}

cudaError_t launch_patch_invert(const Geom& g, const double* A64, double* inv64, int64_t s64,
                                float* inv32, int64_t s32, __nv_bfloat16* invbf, int64_t sbf,
                                int* flags, cudaStream_t s, int64_t npatch, const int32_t* ids) {
    g_launches += 1;
    if (npatch < 0) npatch = g.patches;
    const int NN = g.dim == 2 ? 9 : 27;
    const int NP = NN * g.nc;
    const size_t smem = (size_t)NP * (NP + 1) * sizeof(double) + NP * sizeof(double) + NP * sizeof(int);
    const int per_sm = g.dim == 2 ? 8 : 2;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > npatch) grid = npatch;
    if (grid < 1) return cudaSuccess;
    cudaError_t e;
    const bool lean = g.nc == g.dim;   // n_c = d: the vector problems (ALE extension)
    auto kern = g.dim == 2 ? (lean ? k_patch_invert<2, 2> : k_patch_invert<2, 3>)
                           : (lean ? k_patch_invert<3, 3> : k_patch_invert<3, 4>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, 256, smem, s>>>(g, A64, inv64, s64, inv32, s32, invbf, sbf, flags, npatch, ids);
    return cudaGetLastError();
}

cudaError_t launch_patch_invert_large(const Geom& g, const double* A64, const int32_t* org, int64_t npatch,
                                      double* inv64, int64_t s64, float* inv32, int64_t s32, __nv_bfloat16* invbf,
                                      int64_t sbf, int* flags, cudaStream_t s) {
    if (npatch <= 0) return cudaSuccess;
    g_launches += 1;
    const bool lean = g.nc == g.dim;
    const int NP = (g.dim == 2 ? 25 : 125) * g.nc;
    cudaError_t e;
    if (g.dim == 2) {
        const size_t smem = (size_t)NP * (NP + 1) * sizeof(double) + NP * sizeof(double) + NP * sizeof(int);
        auto kern = lean ? k_patch_invert_large<2, 2, true> : k_patch_invert_large<2, 3, true>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::min<int64_t>(npatch, (int64_t)sm_count() * 4);
        kern<<<(unsigned)grid, 256, smem, s>>>(g, A64, org, npatch, nullptr, inv64, s64, inv32, s32, invbf, sbf, flags);
        return cudaGetLastError();
    }
    // 3d: one work matrix per CTA in global memory (freed once the launch has completed)
    const int64_t grid = std::min<int64_t>(npatch, (int64_t)sm_count());
    double* work = nullptr;
    e = cudaMalloc(&work, (size_t)grid * NP * NP * sizeof(double));
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)NP * sizeof(double) + NP * sizeof(int);
    auto kern = lean ? k_patch_invert_large<3, 3, false> : k_patch_invert_large<3, 4, false>;
    kern<<<(unsigned)grid, 1024, smem, s>>>(g, A64, org, npatch, work, inv64, s64, inv32, s32, invbf, sbf, flags);
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(work);
    return e != cudaSuccess ? e : e2;
}

void launch_coarse_assemble(const Geom& g, const double* A64, double* dense, cudaStream_t s) {
    g_launches += 1;
    const int64_t total = g.nodes * g.nst * g.nc * g.nc;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_coarse_assemble<<<(unsigned)blocks, 256, 0, s>>>(g, A64, dense);
}

void launch_dense_invert(double* a, int64_t n, int* perm, int* flags, cudaStream_t s) {
    g_launches += 1;
    k_dense_invert<<<1, 1024, n * sizeof(double), s>>>(a, n, perm, flags);
}

}  // namespace nmg
