// Solve-phase kernels of the multigrid V-cycle (Section 4.3 (II)-(III)):
// block-sparse residual products, the additive Vanka patch step of Eq. (vanka),
// Q1 restriction / prolongation and the coarse solve.  Every kernel is
// memory-bound; the data layouts are chosen so that warps read contiguous,
// coalesced segments of the matrix and of the patch inverses.  All kernels are
// launched with programmatic dependent launch (see nmg_internal.cuh).
#include <algorithm>

#include "elem.cuh"

namespace nmg {

__device__ int g_wait_timeout = 0;

namespace {

using namespace elem;

constexpr int kWaitSpins = 1 << 22;
constexpr int64_t kLeanRingPatches = 4096;   // see launch_vanka_apply
constexpr int kGatherDepth = 4;     // chunks of defect gathers in flight per CTA

// y = A x  or  y = b - A x, one thread per node.  A in stencil layout.  Two
// CTAs per SM (at most 128 registers a thread): the finest 2d level's 259 CTAs
// then run in one wave with every thread's stencil loads in flight together.
template <typename T, int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(256, 2)
k_spmv(Geom g, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
       T* __restrict__ y, bool residual) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) spmv_node<T, DIM, T, true, 0, NC>(g, A, x, b, y, residual, i);
}

// The same product with one thread per (block row, node).  2d: thread t
// computes row r = t / nodes of node t % nodes, so a warp reads one contiguous
// segment of each stencil array.  3d: thread t computes row t % NC of node
// t / NC, so a warp's loads of one stencil position (the rows of 8
// consecutive nodes) are one contiguous range of the 3d layout.  Faster where
// a node's row work is long (3d: 108 terms per row; FP64), slower for the 2d
// FP32 product, whose extra reads of x cost more than the added parallelism
// gains.  A thread keeps only one stencil position's loads in flight, so the
// 3d FP32 product needs many resident warps: it is held to 32 registers (8
// CTAs, 64 warps per SM; 40 registers gave 6 CTAs and a 96^3 product 15%
// slower).  FP64 keeps the compiler's choice (capping it at 40 registers made
// the 3d 32^3 FP64 solve 3% slower).
template <typename T, int DIM, int NC = DIM + 1, bool VEC = false>
__global__ void __launch_bounds__(256, (DIM == 3 && sizeof(T) == 4) ? 8 : 1)
k_spmv_rows(Geom g, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
            T* __restrict__ y, bool residual) {
    NMG_PDL_ENTRY();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= g.nodes * NC) return;
    if constexpr (DIM == 3) {
        const uint32_t i = (uint32_t)t / NC;
        spmv_row<T, DIM, NC, VEC>(g, A, x, b, y, residual, (int64_t)i, (int)((uint32_t)t - i * NC));
    } else {
        const uint32_t nodes = (uint32_t)g.nodes, r = (uint32_t)t / nodes;
        spmv_row<T, DIM, NC, VEC>(g, A, x, b, y, residual, (int64_t)((uint32_t)t - r * nodes), (int)r);
    }
}

// corr_i = A_i^{-1} R_i d for every patch i: one warp per patch.  The patch
// inverse is column-major, so for each column j the 32 lanes read 32
// consecutive entries (one coalesced 128-byte segment in FP32) and multiply
// them by the broadcast d_j from shared memory; no cross-lane reduction.
// Used for 3d patches (n_p = 108), where each warp streams 46.7 KB.
template <typename T, typename TS, int DIM, int WARPS, int NC = DIM + 1>
__global__ void __launch_bounds__(WARPS * 32, 1)
k_vanka_apply(Geom g, const TS* __restrict__ inv, int64_t stride, const T* __restrict__ d,
              T* __restrict__ corr, int64_t npatch, const int32_t* __restrict__ ids) {
    NMG_PDL_ENTRY();
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    __shared__ T sd[WARPS][NP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * WARPS + w;
    if (p >= npatch) return;
    gather_patch<T, DIM, NC>(g, d, ids ? (int64_t)ids[p] : p, sd[w], lane);
    __syncwarp();
    apply_patch<T, TS, DIM, true, NC>(inv + p * stride, sd[w], corr + p * NP, lane);
}

// Streaming apply for FP32 / BF16 inverses (2d and 3d): a persistent grid of
// a few CTAs per SM walks the chunks c = blockIdx.x + k * gridDim.x; a chunk
// is PW patches per warp in 2d (a lane sums row `lane` of each, the PW sums
// side by side), or in 3d one patch per n_c warps of 27 rows (4 warps for the
// 108-unknown patches, 3 for the 81-unknown patches of n_c = d).  Each CTA
// keeps STAGES chunk copies
// of inverses (TMA bulk copies completing on one mbarrier per stage) and the
// defect gathers of kGatherDepth chunks (cp.async) in flight, so neither the
// DRAM queue nor the gather latency depends on how many warps are resident,
// and there is no tail wave.  Row i of a patch is summed over the columns j in
// ascending order with one fma per term, as in apply_patch, so the
// corrections equal those of the other apply kernels bit for bit.
template <typename T, typename TS, int DIM, int STAGES, int THREADS, int PW = 1, int NC = DIM + 1>
__global__ void __launch_bounds__(THREADS, 1)
k_vanka_apply_ring(Geom g, const TS* __restrict__ inv, int64_t stride, const T* __restrict__ d,
                   T* __restrict__ corr, int64_t npatch, const int32_t* __restrict__ ids) {
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    constexpr int RW = NP / 27;                    // warps per patch
    static_assert(NP % 27 == 0 && (THREADS / 32) % RW == 0, "a patch is whole warps of 27 rows");
    static_assert(PW == 1 || RW == 1, "two patches a warp only for 27-row patches");
    constexpr int CP = (THREADS / 32) / RW * PW;   // patches per chunk (PW patches per warp)
    constexpr int GD = kGatherDepth;
    static_assert(sizeof(T) == 4, "the streaming apply computes in FP32");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[STAGES];
    // a patch's defect row padded to a whole number of 16-byte units: read back as float4
    constexpr int NPD = (NP + 3) / 4 * 4;
    __shared__ __align__(16) T sd[GD + 1][CP][NPD];
    TS* ring = reinterpret_cast<TS*>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int q0 = (w / RW) * PW, row = (w % RW) * 27 + lane;   // the warp's patches q0 .. q0 + PW - 1
    const int64_t G = gridDim.x;
    const int64_t nchunks = (npatch + CP - 1) / CP;
    const int64_t mine = (nchunks - blockIdx.x + G - 1) / G;   // the grid is at most nchunks
    const int64_t stage_elems = (int64_t)CP * stride;
    auto issue = [&](int64_t k) {
        const int64_t c = blockIdx.x + k * G;
        const int cnt = (int)min((int64_t)CP, npatch - c * CP);
        bulk_copy(ring + (k % STAGES) * stage_elems, inv + c * CP * stride,
                  (uint32_t)(cnt * stride * (int64_t)sizeof(TS)), smem_addr(&mbar[k % STAGES]));
    };
    // this thread's defect entry of chunk k -> sd[k % (GD + 1)], one commit group per chunk
    // The gathers are issued for k = 0, 1, 2, ... in turn.  Without a patch
    // list the patch of chunk k advances by G CP patches per chunk, so its
    // coordinates (gx, gy, gz) are stepped with carries instead of divided
    // out of the index, and this thread's entry of a patch is a fixed offset
    // (lane_off) from the patch's first node: the per-chunk address work is a
    // few integer additions on the critical path of every chunk.
    const int an = row / NC, cc = row - an * NC;
    const int64_t lane_off =
        (int64_t)((an % 3) + (int64_t)g.nn[0] * (((an / 3) % 3) + (int64_t)g.nn[1] * (an / 9))) * NC + cc;
    int gx[PW] = {}, gy[PW] = {}, gz[PW] = {}, sx = 0, sy = 0, sz = 0;
    if (!ids) {
#pragma unroll
        for (int t = 0; t < PW; ++t) patch_xyz(g, (int64_t)blockIdx.x * CP + q0 + t, gx[t], gy[t], gz[t]);
        patch_xyz(g, G * CP, sx, sy, sz);   // the step, as coordinates (G CP < patches)
    }
    auto gather = [&](int64_t k) {
#pragma unroll
        for (int t = 0; t < PW; ++t) {
            const int64_t p = (blockIdx.x + k * G) * CP + q0 + t;
            if (k < mine && lane < 27 && p < npatch) {
                int64_t off;
                if (ids) {
                    int px, py, pz;
                    patch_xyz(g, (int64_t)ids[p], px, py, pz);
                    off = patch_node(g, px, py, pz, an) * NC + cc;
                } else {
                    off = (2 * (int64_t)gx[t] + (int64_t)g.nn[0] * (2 * (int64_t)gy[t] + (int64_t)g.nn[1] * 2 * gz[t])) *
                              NC +
                          lane_off;
                }
                cp_async_elem(&sd[k % (GD + 1)][q0 + t][row], d + off);
            }
            if (!ids) {   // on to the patch of chunk k + 1 (sx < pc0, sy < pc1: one carry each)
                gx[t] += sx;
                const int cx = gx[t] >= g.pc[0];
                gx[t] -= cx ? g.pc[0] : 0;
                gy[t] += sy + cx;
                const int cy = gy[t] >= g.pc[1];
                gy[t] -= cy ? g.pc[1] : 0;
                gz[t] += sz + cy;
            }
        }
        cp_async_commit();
    };
    if (tid == 0)
        for (int st = 0; st < STAGES; ++st) mbar_init(smem_addr(&mbar[st]));
    __syncthreads();
    // the inverses do not change during a solve: fill the ring before waiting
    // for the kernel that produces the defect
    if (tid == 0)
        for (int64_t k = 0; k < min((int64_t)STAGES, mine); ++k) issue(k);
    NMG_PDL_ENTRY();
    for (int k = 0; k < GD; ++k) gather(k);
    for (int64_t k = 0; k < mine; ++k) {
        gather(k + GD);            // slot of chunk k - 1, released by the barrier that ended it
        cp_async_wait<GD>();       // this thread's gather of chunk k has landed
        const int st = (int)(k % STAGES);
        uint32_t done = 0;
        for (int it = 0; it < kWaitSpins && !done; ++it)
            done = mbar_try_wait(smem_addr(&mbar[st]), (uint32_t)((k / STAGES) & 1));
        // block-uniform outcome; also publishes the gathered defects of chunk k
        if (!__syncthreads_and(done)) {
            cp_async_wait_all();
            if (tid == 0) {
                // record the timeout, then wait (bounded) for every copy still in flight
                atomicExch(&g_wait_timeout, 1);
                for (int64_t kk = k; kk < min(k + STAGES, mine); ++kk) {
                    uint32_t ok = 0;
                    for (int it = 0; it < kWaitSpins && !ok; ++it)
                        ok = mbar_try_wait(smem_addr(&mbar[kk % STAGES]), (uint32_t)((kk / STAGES) & 1));
                }
            }
            return;
        }
        const int64_t p0 = (blockIdx.x + k * G) * CP + q0;
        if (lane < 27) {
            // the warp's PW patches side by side (independent sums); a patch's
            // defect (a broadcast to every lane) in NPD / 4 vector loads
            T dv[PW][NPD], acc[PW];
#pragma unroll
            for (int t = 0; t < PW; ++t) {
                const float4* d4 = reinterpret_cast<const float4*>(sd[k % (GD + 1)][q0 + t]);
#pragma unroll
                for (int u = 0; u < NPD / 4; ++u) {
                    const float4 v = d4[u];
                    dv[t][4 * u] = v.x; dv[t][4 * u + 1] = v.y; dv[t][4 * u + 2] = v.z; dv[t][4 * u + 3] = v.w;
                }
                acc[t] = T(0);
            }
            const TS* Ap = ring + st * stage_elems + (int64_t)q0 * stride;
#pragma unroll
            for (int j = 0; j < NP; ++j)
#pragma unroll
                for (int t = 0; t < PW; ++t)
                    acc[t] = fma(Cvt<T, TS>::f(Ap[(int64_t)t * stride + j * NP + row]), dv[t][j], acc[t]);
#pragma unroll
            for (int t = 0; t < PW; ++t)
                if (p0 + t < npatch) corr[(p0 + t) * NP + row] = acc[t];
        }
        __syncthreads();   // stage st and the defect slot of chunk k are free again
        if (tid == 0 && k + STAGES < mine) issue(k + STAGES);
    }
    cp_async_wait_all();
}

// x += w(node) * sum over the patches that contain the node of their
// corrections (fixed order: ascending patch index), w = omega / multiplicity
// ("average") or omega ("sum").  One thread per node, no atomics.
template <typename T, int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(256, 1)
k_vanka_update(Geom g, const T* __restrict__ corr, const T* x_in, T* x_out, bool x_zero, T omega,
               bool average) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) vanka_update_node<T, DIM, NC>(g, corr, x_in, x_out, x_zero, omega, average, i);
}

// Fused Vanka update and residual: x_out = x_in + w * corrections, r = b - A x_out
// (x_out at the neighbours recomputed from x_in and the corrections).
template <typename T, int DIM>
__global__ void __launch_bounds__(256, 1)
k_update_residual(Geom g, const T* __restrict__ A, const T* __restrict__ corr, const T* __restrict__ x_in,
                  bool x_zero, T omega, bool average, const T* __restrict__ b, T* __restrict__ x_out,
                  T* __restrict__ r) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < g.nodes) update_residual_node<T, DIM>(g, A, corr, x_in, x_zero, omega, average, b, x_out, r, i);
}

// Fused prolongation and residual: x_out = x_in + P e_c, r = b - A x_out.
template <typename T, int DIM>
__global__ void __launch_bounds__(256, 1)
k_prolong_residual(Geom f, Geom c, const T* __restrict__ A, const T* __restrict__ ec, const T* __restrict__ x_in,
                   const uint8_t* __restrict__ fmask, const T* __restrict__ b, T* __restrict__ x_out,
                   T* __restrict__ r) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < f.nodes) prolong_residual_node<T, DIM>(f, c, A, ec, x_in, fmask, b, x_out, r, i);
}

// Fused Vanka update (MODE 0) or prolongation (MODE 1) and residual on a 2d
// tile: the CTA computes the new iterate on its TX x TY nodes and their
// one-node halo into shared memory (its own nodes also into x_out), then
// r = b - A x_new for its nodes from shared memory.  The node's matrix blocks
// are loaded into registers before the wait for the previous kernel (the
// matrix does not change during a solve).  A value is computed once per tile
// (the halo adds a ring of neighbours), by the element functions of the
// separate kernels, and the residual sums in spmv_node's order, so the results
// equal the separate kernels' bit for bit.  x_out must not alias x_in.
template <typename T, int MODE, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 2)
k_update_residual_tile(Geom g, Geom gc, const T* __restrict__ A, const T* __restrict__ src, const T* __restrict__ x_in,
                       bool x_zero, T omega, bool average, const uint8_t* __restrict__ fmask, const T* __restrict__ b,
                       T* __restrict__ x_out, T* __restrict__ r) {
    constexpr int NC = 3, NB = NC * NC, HX = TX + 2, HY = TY + 2;
    __shared__ T xs[HX * HY * NC];
    const int tiles_x = (g.nn[0] + TX - 1) / TX;
    const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
    const int x0 = bx * TX - 1, y0 = by * TY - 1;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int ix = x0 + 1 + tx, iy = y0 + 1 + ty;
    const bool inside = ix < g.nn[0] && iy < g.nn[1];
    const int64_t i = inside ? ix + (int64_t)g.nn[0] * iy : 0;
    // the node's blocks of the 9 stencil positions (present in the stencil
    // layout for every position, zero outside the mesh)
    T av[9][NB];
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int e = 0; e < NB; ++e) av[q][e] = inside ? __ldg(A + ((int64_t)q * NB + e) * g.ld + i) : T(0);
    NMG_PDL_ENTRY();
    T bv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) bv[c] = inside ? b[i * NC + c] : T(0);
    for (int t = threadIdx.x; t < HX * HY; t += TX * TY) {
        const int hx = t % HX, hy = t / HX;
        const int gx = x0 + hx, gy = y0 + hy;
        if (gx >= 0 && gx < g.nn[0] && gy >= 0 && gy < g.nn[1]) {
            const int64_t j = gx + (int64_t)g.nn[0] * gy;
            T v[NC];
            if constexpr (MODE == 0) vanka_update_value<T, 2>(g, src, x_in, x_zero, omega, average, j, v);
            else prolong_value<T, 2>(g, gc, src, x_in, fmask, j, v);
#pragma unroll
            for (int c = 0; c < NC; ++c) xs[t * NC + c] = v[c];
            if (hx >= 1 && hx <= TX && hy >= 1 && hy <= TY)
#pragma unroll
                for (int c = 0; c < NC; ++c) x_out[j * NC + c] = v[c];
        }
    }
    __syncthreads();
    if (!inside) return;
    T acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int dx = q % 3 - 1, dy = q / 3 - 1;
        if (ix + dx >= 0 && ix + dx < g.nn[0] && iy + dy >= 0 && iy + dy < g.nn[1]) {
            const T* xn = xs + ((tx + 1 + dx) + HX * (ty + 1 + dy)) * NC;
#pragma unroll
            for (int k = 0; k < NC; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[k] = fma(av[q][k * NC + c], xn[c], acc[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) r[i * NC + k] = bv[k] - acc[k];
}

// r_c = P^T r_f (Q1 full weighting), coarse Dirichlet entries zero.  One thread per coarse node.
template <typename T, int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(256, 1)
k_restrict(Geom f, Geom c, const T* __restrict__ rf, T* __restrict__ rc, const uint8_t* __restrict__ cmask) {
    NMG_PDL_ENTRY();
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I < c.nodes) restrict_node<T, DIM, NC>(f, c, rf, rc, cmask, I);
}

// x_f += P e_c (Q1 interpolation), fine Dirichlet entries untouched.  One thread per fine node.
template <typename T, int DIM, int NC = DIM + 1>
__global__ void __launch_bounds__(256, 1)
k_prolong_add(Geom f, Geom c, const T* __restrict__ ec, T* __restrict__ xf, const uint8_t* __restrict__ fmask) {
    NMG_PDL_ENTRY();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < f.nodes) prolong_node<T, DIM, NC>(f, c, ec, xf, fmask, i);
}

// x = inv * b with the FP64 dense coarse inverse, one warp per row, FP64 sums.
template <typename T>
__global__ void __launch_bounds__(256, 1)
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
    const bool lean = g.nc == g.dim;   // n_c = d: the vector problems (ALE extension)
    // 3d FP64 with 4 unknowns a node: a node block of x is 32 aligned bytes (two
    // 16-byte loads).  The FP32 product reads x entry by entry: its 16-byte x
    // loads took the 32-register kernel past its registers (spills to local
    // memory, 5% more DRAM traffic).
    if (g.dim == 3 && !lean && sizeof(T) == 8 && (uintptr_t)x % 16 == 0)
        pdl_launch(k_spmv_rows<T, 3, 4, sizeof(T) == 8>, dim3(blocks_for(g.nodes * g.nc, 256)), dim3(256), 0, s, g, A, x, b, y,
                   residual);
    else if (g.dim == 3)
        pdl_launch(lean ? k_spmv_rows<T, 3, 3> : k_spmv_rows<T, 3, 4>, dim3(blocks_for(g.nodes * g.nc, 256)),
                   dim3(256), 0, s, g, A, x, b, y, residual);
    else if constexpr (sizeof(T) == 8)
        pdl_launch(lean ? k_spmv_rows<T, 2, 2> : k_spmv_rows<T, 2, 3>, dim3(blocks_for(g.nodes * g.nc, 256)),
                   dim3(256), 0, s, g, A, x, b, y, residual);
    else
        pdl_launch(lean ? k_spmv<T, 2, 2> : k_spmv<T, 2, 3>, dim3(blocks_for(g.nodes, 256)), dim3(256), 0, s, g, A,
                   x, b, y, residual);
}

// Launches the streaming apply on min(chunks, resident CTAs) CTAs.  The
// resident count comes from the occupancy calculator for the kernel's shared
// memory (cached per device and kernel instance).
template <typename T, typename TS, int DIM, int STAGES, int THREADS, int PW = 1, int NC = DIM + 1>
static void launch_ring(const Geom& g, const TS* inv, int64_t stride, const T* d, T* corr, cudaStream_t s,
                        int64_t npatch, const int32_t* ids) {
    constexpr int CP = (THREADS / 32) / (((DIM == 2) ? 9 : 27) * NC / 27) * PW;
    const size_t smem = (size_t)STAGES * CP * stride * sizeof(TS);
    auto kern = k_vanka_apply_ring<T, TS, DIM, STAGES, THREADS, PW, NC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static int resident[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int r = (dev >= 0 && dev < kMaxDevices) ? resident[dev] : 0;
    if (r <= 0) {
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        r = std::max(1, per_sm) * std::max(1, sms);
        if (dev >= 0 && dev < kMaxDevices) resident[dev] = r;
    }
    const int64_t chunks = (npatch + CP - 1) / CP;
    const dim3 grid((unsigned)std::min<int64_t>(chunks, r));
    pdl_launch(kern, grid, dim3(THREADS), smem, s, g, inv, stride, d, corr, npatch, ids);
}

template <typename T, typename TS>
void launch_vanka_apply(const Geom& g, const TS* inv, int64_t stride, const T* d, T* corr, cudaStream_t s,
                        int64_t npatch, const int32_t* ids) {
    g_launches += 1;
    if (npatch < 0) npatch = g.patches;
    // the bulk copies need 16-byte aligned chunks and the unpadded column
    // layout (stride at most n_p^2 rounded up to 16 bytes); FP64 and other
    // layouts use the warp kernel
    const int np = (g.dim == 2 ? 9 : 27) * g.nc;
    // n_c = d: 2d patches (18 rows) take the warp kernel, the ring's warps
    // being 27-row slices; 3d patches (81 rows, three warps) take the ring on
    // levels of at most kLeanRingPatches patches (3d 32^3 extension solve
    // 2.12 -> 1.60 ms) and the warp kernel above (with the ring up to the
    // 48^3 level's 13,824 patches the 96^3 solve went from 16.7 to 17.5 ms)
    const bool lean = g.nc == g.dim;
    const bool ring = (!lean || (g.dim == 3 && npatch <= kLeanRingPatches)) && sizeof(TS) <= 4 &&
                      ((uintptr_t)inv % 16 == 0) && ((stride * (int64_t)sizeof(TS)) % 16 == 0) &&
                      stride >= (int64_t)np * np && stride * (int64_t)sizeof(TS) <= (int64_t)np * np * sizeof(TS) + 16;
    if (npatch == 0) return;
    if constexpr (sizeof(TS) <= 4) {
        if (ring && lean) {   // one 81-row patch a chunk (three warps), 4 stages
            launch_ring<T, TS, 3, 4, 96, 1, 3>(g, inv, stride, d, corr, s, npatch, ids);
            return;
        }
        if (ring) {
            // 2d: about 70 KB of inverses in flight per CTA, 3 CTAs per SM.
            // 3d: one 108-unknown patch a chunk (4 warps), 3 stages of FP32
            // (140 KB, one CTA per SM) or 4 of BF16 (93 KB, two CTAs per SM): the
            // shared memory left free lets the next kernel's CTAs start while this
            // one drains (4 stages of FP32, or BF16 chunks of two patches, measured
            // slower in the solve).
            // 2d: on levels of at least 4096 patches two patches a warp (chunks of 8,
            // 3 (FP32) or 6 (BF16) stages): half the chunk rounds a CTA walks, each
            // with its fixed cost of barriers, waits and copy issue; smaller levels
            // keep one patch a warp (twice the CTAs for their latency-bound steps)
            constexpr int S2 = sizeof(TS) == 4 ? 6 : 12;
            if (g.dim == 2 && npatch >= 4096)
                launch_ring<T, TS, 2, S2 / 2, 128, 2>(g, inv, stride, d, corr, s, npatch, ids);
            else if (g.dim == 2) launch_ring<T, TS, 2, S2, 128>(g, inv, stride, d, corr, s, npatch, ids);
            else if (sizeof(TS) == 4) launch_ring<T, TS, 3, 3, 128>(g, inv, stride, d, corr, s, npatch, ids);
            else launch_ring<T, TS, 3, 4, 128>(g, inv, stride, d, corr, s, npatch, ids);
            return;
        }
    }
    constexpr int W = 4;
    const dim3 grid((unsigned)((npatch + W - 1) / W));
    if (g.dim == 2)
        pdl_launch(lean ? k_vanka_apply<T, TS, 2, W, 2> : k_vanka_apply<T, TS, 2, W, 3>, grid, dim3(W * 32), 0, s, g,
                   inv, stride, d, corr, npatch, ids);
    else
        pdl_launch(lean ? k_vanka_apply<T, TS, 3, W, 3> : k_vanka_apply<T, TS, 3, W, 4>, grid, dim3(W * 32), 0, s, g,
                   inv, stride, d, corr, npatch, ids);
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
    const bool lean = g.nc == g.dim;
    if (g.dim == 2)
        pdl_launch(lean ? k_vanka_update<T, 2, 2> : k_vanka_update<T, 2, 3>, grid, dim3(256), 0, s, g, corr, x_in, x_out,
                   x_zero, omega, average);
    else
        pdl_launch(lean ? k_vanka_update<T, 3, 3> : k_vanka_update<T, 3, 4>, grid, dim3(256), 0, s, g, corr, x_in, x_out,
                   x_zero, omega, average);
}

// 2d FP32 tiles of 32 x 8 nodes (one thread a node).
constexpr int kUrTx = 32, kUrTy = 8;
inline unsigned ur_tiles(const Geom& g) {
    return (unsigned)(((g.nn[0] + kUrTx - 1) / kUrTx) * ((g.nn[1] + kUrTy - 1) / kUrTy));
}

template <typename T>
void launch_update_residual(const Geom& g, const T* A, const T* corr, const T* x_in, bool x_zero, T omega,
                            bool average, const T* b, T* x_out, T* r, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(g.nodes, 256));
    if constexpr (sizeof(T) == 4) {
        if (g.dim == 2 && g.nc == 3) {
            pdl_launch(k_update_residual_tile<T, 0, kUrTx, kUrTy>, dim3(ur_tiles(g)), dim3(kUrTx * kUrTy), 0, s, g, g,
                       A, corr, x_in, x_zero, omega, average, (const uint8_t*)nullptr, b, x_out, r);
            return;
        }
    }
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
    if constexpr (sizeof(T) == 4) {
        if (f.dim == 2 && f.nc == 3) {
            pdl_launch(k_update_residual_tile<T, 1, kUrTx, kUrTy>, dim3(ur_tiles(f)), dim3(kUrTx * kUrTy), 0, s, f, c,
                       A, ec, x_in, false, T(0), false, fmask, b, x_out, r);
            return;
        }
    }
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
    const bool lean = f.nc == f.dim;
    if (f.dim == 2) pdl_launch(lean ? k_restrict<T, 2, 2> : k_restrict<T, 2, 3>, grid, dim3(256), 0, s, f, c, rf, rc, cmask);
    else pdl_launch(lean ? k_restrict<T, 3, 3> : k_restrict<T, 3, 4>, grid, dim3(256), 0, s, f, c, rf, rc, cmask);
}

template <typename T>
void launch_prolong_add(const Geom& f, const Geom& c, const T* ec, T* xf, const uint8_t* fmask, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid(blocks_for(f.nodes, 256));
    const bool lean = f.nc == f.dim;
    if (f.dim == 2) pdl_launch(lean ? k_prolong_add<T, 2, 2> : k_prolong_add<T, 2, 3>, grid, dim3(256), 0, s, f, c, ec, xf, fmask);
    else pdl_launch(lean ? k_prolong_add<T, 3, 3> : k_prolong_add<T, 3, 4>, grid, dim3(256), 0, s, f, c, ec, xf, fmask);
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
template void launch_vanka_apply<double, double>(const Geom&, const double*, int64_t, const double*, double*, cudaStream_t,
                                                 int64_t, const int32_t*);
template void launch_vanka_apply<float, float>(const Geom&, const float*, int64_t, const float*, float*, cudaStream_t,
                                               int64_t, const int32_t*);
template void launch_vanka_apply<float, __nv_bfloat16>(const Geom&, const __nv_bfloat16*, int64_t, const float*, float*,
                                                       cudaStream_t, int64_t, const int32_t*);
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
