// Multi-vector V-cycle kernels: the steps of Section 4.3 (II)-(III) for K
// right-hand sides at once against the same level matrices and patch inverses
// (one factorisation serves many defects: the smoother is applied many hundred
// times per Jacobian, Section 5).  The K vectors are stored interleaved,
// value (u, k) at u * K + k for unknown u = node * nc + c, so a node's K
// values are one contiguous 16- or 32-byte segment.  Every matrix entry and
// every patch-inverse entry is read once per launch for all K columns, which
// divides the dominant traffic of the V-cycle by K.
//
// Each column is computed with the terms, order and rounding of the
// single-vector kernels (smooth_kernels.cu, elem.cuh): per column, the
// results equal those of a single-vector V-cycle bit for bit.
#include <algorithm>

#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

constexpr int kWaitSpinsM = 1 << 22;
constexpr int kGatherDepthM = 4;   // chunks of defect gathers in flight per CTA of the apply

// K consecutive floats (K = 4 or 8; 16-byte aligned) to / from registers.
template <int K>
__device__ __forceinline__ void ldk(const float* p, float (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K / 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(p)[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}
template <int K>
__device__ __forceinline__ void stk(float* p, const float (&v)[K]) {
#pragma unroll
    for (int q = 0; q < K / 4; ++q)
        reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float f4(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}

// y = A X or y = B - A X for K columns (stencil layout of A as in k_spmv),
// NC / RS threads per node (each RS of the node's block rows), with X staged
// in shared memory: a CTA owns a TX x TY (x TZ) tile of nodes and first
// copies the K-column values of the tile and its one-node halo (coalesced
// 16-byte loads), so each node's values cross from L2 about once per tile
// instead of once per neighbour.  A node's K interleaved columns are 12-32
// floats, so one thread per node reading them directly from global memory
// touches a different 128-byte line per lane; from the padded shared-memory
// slots the reads are conflict-free.  A is read with a warp covering rows of
// consecutive nodes (in 3d the threads of one node take consecutive lanes and
// their rows are consecutive 32-byte parts of the node's 64-byte block), the
// blocks of three stencil positions (one x-row of neighbours) loaded together
// (every position's block exists in the stencil layout, zero outside the
// mesh).  Per column and row: stencil positions ascending, block columns
// ascending, one fma per term, as spmv_node / spmv_row.
template <int DIM, int NC, int K, int TX, int TY, int TZ, int RS = NC>
__global__ void __launch_bounds__(TX * TY * TZ * (NC / RS))
k_spmv_many_tile(Geom g, const float* __restrict__ A, const float* __restrict__ x, const float* __restrict__ b,
                 float* __restrict__ y, bool residual) {
    constexpr int NB = NC * NC;
    constexpr int NST = DIM == 2 ? 9 : 27;
    constexpr int H = NC / RS;      // threads per node
    constexpr int NT = TX * TY * TZ * H;
    constexpr int NR = RS * NC;     // matrix entries of a thread's rows per position
    constexpr int HX = TX + 2, HY = TY + 2, HZ = DIM == 3 ? TZ + 2 : 1;
    constexpr int NV = NC * K;      // floats per node
    constexpr int NQ = NV / 4;      // float4 per node
    // shared-memory slot of a node: an odd number of 16-byte units, so that the
    // 16-byte reads of 8 consecutive nodes (one phase of a warp's access) fall
    // in 8 different groups of 4 banks (a slot of 128 bytes would put them all
    // in the same 4 banks)
    constexpr int NS = (NQ % 2) ? NV : NV + 4;
    static_assert(DIM == 3 || TZ == 1, "2d tiles are one node deep");
    static_assert(NC % RS == 0 && (RS == NC || DIM == 3), "a node's rows split over threads in 3d only");
    extern __shared__ float4 xs4[];
    const float* xs = reinterpret_cast<const float*>(xs4);
    const int tiles_x = (g.nn[0] + TX - 1) / TX, tiles_y = (g.nn[1] + TY - 1) / TY;
    int blk = blockIdx.x;
    const int bx = blk % tiles_x;
    blk /= tiles_x;
    const int by = blk % tiles_y, bz = blk / tiles_y;
    const int x0 = bx * TX - 1, y0 = by * TY - 1, z0 = DIM == 3 ? bz * TZ - 1 : 0;
    const int nl = threadIdx.x / H, r0 = (threadIdx.x - nl * H) * RS;   // tile node, first row
    const int tx = nl % TX, ty = (nl / TX) % TY, tz = nl / (TX * TY);
    const int ix = x0 + 1 + tx, iy = y0 + 1 + ty, iz = DIM == 3 ? z0 + 1 + tz : 0;
    const bool inside = ix < g.nn[0] && iy < g.nn[1] && iz < g.nn[2];
    const int64_t i = inside ? ix + (int64_t)g.nn[0] * (iy + (int64_t)g.nn[1] * iz) : 0;
    // The matrix rows of three stencil positions at a time.  The first group
    // is loaded before the wait for the kernel that produces X (the matrix does
    // not change during a solve).  In 2d each next group is loaded while the
    // current one is summed (two buffers); in 3d the second buffer's registers
    // would cost a CTA per SM, so a group is loaded when it is reached.
    constexpr bool PIPE = DIM == 2;
    float av[PIPE ? 2 : 1][3][NR];
    auto load_group = [&](float (&dst)[3][NR], int s0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if constexpr (DIM == 3) {   // the thread's rows of the node's block: one contiguous run
                if (inside) elem::load_arun<float, NR>(A + stencil_off<DIM, NB>(g.ld, s0 + q, r0 * NC, i), dst[q]);
                else
#pragma unroll
                    for (int e = 0; e < NR; ++e) dst[q][e] = 0.f;
            } else {
#pragma unroll
                for (int e = 0; e < NR; ++e)
                    dst[q][e] = inside ? __ldg(A + stencil_off<DIM, NB>(g.ld, s0 + q, e, i)) : 0.f;
            }
        }
    };
    load_group(av[0], 0);
    NMG_PDL_ENTRY();
    for (int t = threadIdx.x; t < HX * HY * HZ * NQ; t += NT) {
        const int hn = t / NQ, q = t - hn * NQ;
        const int hx = hn % HX, hy = (hn / HX) % HY, hz = hn / (HX * HY);
        const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
        if (gx >= 0 && gx < g.nn[0] && gy >= 0 && gy < g.nn[1] && gz >= 0 && gz < g.nn[2])
            xs4[hn * (NS / 4) + q] = ld4(x + (gx + (int64_t)g.nn[0] * (gy + (int64_t)g.nn[1] * gz)) * NV + 4 * q);
    }
    __syncthreads();
    const int hz0 = DIM == 3 ? tz + 1 : 0;   // the node's own plane in the halo tile
    if (!inside) return;
    float acc[RS][K];
#pragma unroll
    for (int r = 0; r < RS; ++r)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[r][k] = 0.f;
#pragma unroll
    for (int s0 = 0; s0 < NST; s0 += 3) {
        const int cur = PIPE ? (s0 / 3) & 1 : 0;
        if constexpr (PIPE) {
            if (s0 + 3 < NST) load_group(av[cur ^ 1], s0 + 3);
        } else {
            if (s0 > 0) load_group(av[0], s0);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int s = s0 + q;
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
            const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                            (iz + dz >= 0) && (iz + dz < g.nn[2]);
            if (ok) {
                const float* xn = xs + ((tx + 1 + dx) + HX * ((ty + 1 + dy) + HY * (hz0 + dz))) * NS;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float xv[K];
                    ldk<K>(xn + c * K, xv);
#pragma unroll
                    for (int r = 0; r < RS; ++r)
#pragma unroll
                        for (int k = 0; k < K; ++k) acc[r][k] = fmaf(av[cur][q][r * NC + c], xv[k], acc[r][k]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        float out[K];
        const int64_t row = i * NC + r0 + r;
        if (residual) {
            float bv[K];
            ldk<K>(b + row * K, bv);
#pragma unroll
            for (int k = 0; k < K; ++k) out[k] = bv[k] - acc[r][k];
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) out[k] = acc[r][k];
        }
        stk<K>(y + row * K, out);
    }
}

// corr_p = A_p^{-1} R_p D for K defect columns and every patch p, streamed as
// in k_vanka_apply_ring: a persistent grid walks chunks of CP patches; the
// inverses of STAGES chunks are in flight as TMA bulk copies (one mbarrier per
// stage) and the defect gathers (K values per patch row, 16-byte cp.async) of
// kGatherDepthM chunks.  A patch is served by PW = ceil(n_p / 32) warps, one
// thread per row; row i of column k is summed over the inverse's columns j in
// ascending order with one fma per term (as apply_patch), so each column's
// corrections equal the single-vector apply's bit for bit.
template <typename TS, int DIM, int NC, int K, int STAGES, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
k_vanka_apply_many(Geom g, const TS* __restrict__ inv, int64_t stride, const float* __restrict__ d,
                   float* __restrict__ corr, int* timeout_flag) {
    constexpr int NP = (DIM == 2 ? 9 : 27) * NC;
    constexpr int PW = (NP + 31) / 32;            // warps per patch
    constexpr int CP = (THREADS / 32) / PW;        // patches per chunk
    constexpr int GD = kGatherDepthM;
    static_assert((THREADS / 32) % PW == 0 && CP >= 1, "a chunk holds whole patches");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[STAGES];
    __shared__ __align__(16) float sd[GD + 1][CP][NP][K];
    TS* ring = reinterpret_cast<TS*>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int q = w / PW, row = (w % PW) * 32 + lane;
    const int64_t G = gridDim.x;
    const int64_t nchunks = (g.patches + CP - 1) / CP;
    const int64_t mine = (nchunks - blockIdx.x + G - 1) / G;   // the grid is at most nchunks
    const int64_t stage_elems = (int64_t)CP * stride;
    auto issue = [&](int64_t k) {
        const int64_t c = blockIdx.x + k * G;
        const int cnt = (int)min((int64_t)CP, g.patches - c * CP);
        bulk_copy(ring + (k % STAGES) * stage_elems, inv + c * CP * stride,
                  (uint32_t)(cnt * stride * (int64_t)sizeof(TS)), smem_addr(&mbar[k % STAGES]));
    };
    auto gather = [&](int64_t k) {
        const int64_t p = (blockIdx.x + k * G) * CP + q;
        if (k < mine && row < NP && p < g.patches) {
            int px, py, pz;
            patch_xyz(g, p, px, py, pz);
            const int an = row / NC, c = row - an * NC;
            const float* src = d + (patch_node(g, px, py, pz, an) * NC + c) * K;
#pragma unroll
            for (int h = 0; h < K / 4; ++h) cp_async16(&sd[k % (GD + 1)][q][row][4 * h], src + 4 * h);
        }
        cp_async_commit();
    };
    if (tid == 0)
        for (int st = 0; st < STAGES; ++st) mbar_init(smem_addr(&mbar[st]));
    __syncthreads();
    if (tid == 0)
        for (int64_t k = 0; k < min((int64_t)STAGES, mine); ++k) issue(k);
    NMG_PDL_ENTRY();
    for (int k = 0; k < GD; ++k) gather(k);
    for (int64_t k = 0; k < mine; ++k) {
        gather(k + GD);
        cp_async_wait<GD>();
        const int st = (int)(k % STAGES);
        uint32_t done = 0;
        for (int it = 0; it < kWaitSpinsM && !done; ++it)
            done = mbar_try_wait(smem_addr(&mbar[st]), (uint32_t)((k / STAGES) & 1));
        if (!__syncthreads_and(done)) {
            cp_async_wait_all();
            if (tid == 0) {
                atomicExch(timeout_flag, 1);
                for (int64_t kk = k; kk < min(k + STAGES, mine); ++kk) {
                    uint32_t ok = 0;
                    for (int it = 0; it < kWaitSpinsM && !ok; ++it)
                        ok = mbar_try_wait(smem_addr(&mbar[kk % STAGES]), (uint32_t)((kk / STAGES) & 1));
                }
            }
            return;
        }
        const int64_t p = (blockIdx.x + k * G) * CP + q;
        if (p < g.patches && row < NP) {
            const TS* Ap = ring + st * stage_elems + (int64_t)q * stride;
            const float* dk = &sd[k % (GD + 1)][q][0][0];
            float acc[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) acc[kk] = 0.f;
#pragma unroll 9
            for (int j = 0; j < NP; ++j) {
                const float a = Cvt<float, TS>::f(Ap[j * NP + row]);
#pragma unroll
                for (int h = 0; h < K / 4; ++h) {
                    const float4 dv = ld4(dk + j * K + 4 * h);
                    acc[4 * h] = fmaf(a, dv.x, acc[4 * h]);
                    acc[4 * h + 1] = fmaf(a, dv.y, acc[4 * h + 1]);
                    acc[4 * h + 2] = fmaf(a, dv.z, acc[4 * h + 2]);
                    acc[4 * h + 3] = fmaf(a, dv.w, acc[4 * h + 3]);
                }
            }
            stk<K>(corr + (p * NP + row) * K, acc);
        }
        __syncthreads();
        if (tid == 0 && k + STAGES < mine) issue(k + STAGES);
    }
    cp_async_wait_all();
}

// x_out = x_in + w(node) * (sum of the corrections of the patches containing
// the node, ascending patch order), as vanka_update_value; one thread per
// (node, group of 4 columns).
template <int DIM, int NC, int K>
__global__ void __launch_bounds__(256)
k_vanka_update_many(Geom g, const float* __restrict__ corr, const float* x_in, float* x_out, bool x_zero,
                    float omega, bool average) {
    NMG_PDL_ENTRY();
    constexpr int NP = (DIM == 2 ? 9 : 27) * NC;
    constexpr int KQ = K / 4;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= g.nodes * KQ) return;
    const int64_t i = t / KQ;
    const int kq = (int)(t - i * KQ);
    int xyz[3];
    node_xyz(g, i, xyz[0], xyz[1], xyz[2]);
    int cp[3][2], cl[3][2], cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c = xyz[a];
        if (a >= DIM) { cp[a][0] = cp[a][1] = 0; cl[a][0] = cl[a][1] = 0; cnt[a] = 1; continue; }
        if (c & 1) {
            cp[a][0] = cp[a][1] = (c - 1) >> 1;
            cl[a][0] = cl[a][1] = 1;
            cnt[a] = 1;
        } else {
            const bool lo = c > 0, hi = c < g.cells[a];
            cp[a][0] = lo ? (c >> 1) - 1 : c >> 1;
            cl[a][0] = lo ? 2 : 0;
            cp[a][1] = c >> 1;
            cl[a][1] = 0;
            cnt[a] = (int)lo + (int)hi;
        }
    }
    constexpr int NZ = DIM == 3 ? 2 : 1;
    int64_t off[NZ][2][2];
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const bool pres = a < cnt[2] && b < cnt[1] && e < cnt[0];
                const int ea = pres ? a : 0, eb = pres ? b : 0, ee = pres ? e : 0;
                const int64_t p = cp[0][ee] + (int64_t)g.pc[0] * (cp[1][eb] + (int64_t)g.pc[1] * cp[2][ea]);
                const int loc = cl[0][ee] + 3 * cl[1][eb] + 9 * cl[2][ea];
                off[a][b][e] = (p * NP + loc * NC) * K + 4 * kq;
            }
    const int m = cnt[0] * cnt[1] * cnt[2];
    const float wgt = average ? omega / float(m) : omega;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float4 cv[NZ][2][2];
#pragma unroll
        for (int a = 0; a < NZ; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e) cv[a][b][e] = ld4(corr + off[a][b][e] + c * K);
        float sum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NZ; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (a < cnt[2] && b < cnt[1] && e < cnt[0])
#pragma unroll
                        for (int k = 0; k < 4; ++k) sum[k] += f4(cv[a][b][e], k);
        const int64_t o = (i * NC + c) * K + 4 * kq;
        const float4 old = x_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(x_in + o);
        st4(x_out + o, make_float4(fmaf(wgt, sum[0], old.x), fmaf(wgt, sum[1], old.y), fmaf(wgt, sum[2], old.z),
                                   fmaf(wgt, sum[3], old.w)));
    }
}

// R_c = P^T R_f (Q1 full weighting) per column, coarse Dirichlet entries zero;
// one thread per (coarse node, group of 4 columns); the order of
// restrict_value_f (planes, then rows and columns of fine nodes).
template <int DIM, int NC, int K>
__global__ void __launch_bounds__(256)
k_restrict_many(Geom f, Geom c, const float* __restrict__ rf, float* __restrict__ rc,
                const uint8_t* __restrict__ cmask) {
    NMG_PDL_ENTRY();
    constexpr int KQ = K / 4;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= c.nodes * KQ) return;
    const int64_t I = t / KQ;
    const int kq = (int)(t - I * KQ);
    int X, Y, Z;
    node_xyz(c, I, X, Y, Z);
    float sum[NC][4];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) sum[k][q] = 0.f;
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
#pragma unroll
    for (int oz = zlo; oz <= zhi; ++oz) {
        const int fz = 2 * Z + oz;
        if (fz < 0 || fz >= f.nn[2]) continue;
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int fy = 2 * Y + oy, fx = 2 * X + ox;
                if (fy < 0 || fy >= f.nn[1] || fx < 0 || fx >= f.nn[0]) continue;
                const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f) * (oz ? 0.5f : 1.f);
                const int64_t node = fx + (int64_t)f.nn[0] * (fy + (int64_t)f.nn[1] * fz);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const float4 v = ld4(rf + (node * NC + k) * K + 4 * kq);
                    sum[k][0] = fmaf(w, v.x, sum[k][0]);
                    sum[k][1] = fmaf(w, v.y, sum[k][1]);
                    sum[k][2] = fmaf(w, v.z, sum[k][2]);
                    sum[k][3] = fmaf(w, v.w, sum[k][3]);
                }
            }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const bool dir = cmask[I * NC + k] != 0;
        st4(rc + (I * NC + k) * K + 4 * kq,
            dir ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(sum[k][0], sum[k][1], sum[k][2], sum[k][3]));
    }
}

// X_f += P E_c per column (Q1 interpolation), fine Dirichlet entries
// untouched; one thread per (fine node, group of 4 columns); the order of
// prolong_value.
template <int DIM, int NC, int K>
__global__ void __launch_bounds__(256)
k_prolong_add_many(Geom f, Geom c, const float* __restrict__ ec, float* __restrict__ xf,
                   const uint8_t* __restrict__ fmask) {
    NMG_PDL_ENTRY();
    constexpr int KQ = K / 4;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= f.nodes * KQ) return;
    const int64_t i = t / KQ;
    const int kq = (int)(t - i * KQ);
    int xyz[3];
    node_xyz(f, i, xyz[0], xyz[1], xyz[2]);
    int ci[3][2], cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int v = xyz[a];
        if (a >= DIM || !(v & 1)) { ci[a][0] = ci[a][1] = v >> 1; cnt[a] = 1; }
        else { ci[a][0] = (v - 1) >> 1; ci[a][1] = (v + 1) >> 1; cnt[a] = 2; }
    }
    const float w = (cnt[0] == 2 ? 0.5f : 1.f) * (cnt[1] == 2 ? 0.5f : 1.f) * (cnt[2] == 2 ? 0.5f : 1.f);
    constexpr int NZ = DIM == 3 ? 2 : 1;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        float sum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NZ; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (a < cnt[2] && b < cnt[1] && e < cnt[0]) {
                        const int64_t I = ci[0][e] + (int64_t)c.nn[0] * (ci[1][b] + (int64_t)c.nn[1] * ci[2][a]);
                        const float4 v = ld4(ec + (I * NC + k) * K + 4 * kq);
                        sum[0] = fmaf(w, v.x, sum[0]);
                        sum[1] = fmaf(w, v.y, sum[1]);
                        sum[2] = fmaf(w, v.z, sum[2]);
                        sum[3] = fmaf(w, v.w, sum[3]);
                    }
        const int64_t o = (i * NC + k) * K + 4 * kq;
        if (!fmask[i * NC + k]) {
            const float4 x = ld4(xf + o);
            st4(xf + o, make_float4(x.x + sum[0], x.y + sum[1], x.z + sum[2], x.w + sum[3]));
        }
    }
}

// X = inv B with the FP64 dense coarse inverse, one warp per row, FP64 sums
// per column in the order of coarse_row (lane-strided terms, then a shuffle
// tree).
template <int K>
__global__ void __launch_bounds__(256)
k_coarse_gemv_many(const double* __restrict__ inv, int64_t n, const float* __restrict__ b, float* __restrict__ x) {
    NMG_PDL_ENTRY();
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        const double a = inv[row * n + j];
        float bv[K];
        ldk<K>(b + j * K, bv);
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] = fma(a, (double)bv[k], s[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], off);
    if (lane == 0) {
        float out[K];
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = (float)s[k];
        stk<K>(x + row * K, out);
    }
}

// Interleaves ncols (<= K) vectors of n floats into out (u * K + k); the
// columns ncols..K-1 are zero.
template <int K>
__global__ void __launch_bounds__(256) k_pack(ColPtrs src, int ncols, int64_t n, float* __restrict__ out) {
    NMG_PDL_ENTRY();
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = k < ncols ? src.p[k][u] : 0.f;
    stk<K>(out + u * K, v);
}

// Writes the first ncols interleaved columns of in back to ncols vectors.
template <int K>
__global__ void __launch_bounds__(256) k_unpack(const float* __restrict__ in, ColPtrsOut dst, int ncols, int64_t n) {
    NMG_PDL_ENTRY();
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    float v[K];
    ldk<K>(in + u * K, v);
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < ncols) dst.p[k][u] = v[k];
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Launches the streaming multi-vector apply on min(chunks, resident CTAs) CTAs.
template <typename TS, int DIM, int NC, int K, int STAGES, int THREADS>
void launch_apply_many(const Geom& g, const TS* inv, int64_t stride, const float* d, float* corr, int* flag,
                       cudaStream_t s) {
    constexpr int NP = (DIM == 2 ? 9 : 27) * NC;
    constexpr int CP = (THREADS / 32) / ((NP + 31) / 32);
    const size_t smem = (size_t)STAGES * CP * stride * sizeof(TS);
    auto kern = k_vanka_apply_many<TS, DIM, NC, K, STAGES, THREADS>;
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
    const int64_t chunks = (g.patches + CP - 1) / CP;
    pdl_launch(kern, dim3((unsigned)std::min<int64_t>(chunks, r)), dim3(THREADS), smem, s, g, inv, stride, d, corr, flag);
}

// Chunk shapes: 2d, four patches of one warp each, six (FP32) or twelve (BF16)
// stages of 11.7 / 5.8 KB; 3d (n_p = 108), one patch of four warps and four
// stages of 46.7 KB (FP32) or two patches and four stages of 23.3 KB each
// (BF16); n_c = d: 2d n_p = 18 as 2d, 3d n_p = 81 with three warps per patch.
template <typename TS, int K>
void apply_many_dispatch(const Geom& g, const TS* inv, int64_t stride, const float* d, float* corr, int* flag,
                         cudaStream_t s) {
    constexpr bool F32 = sizeof(TS) == 4;
    const bool lean = g.nc == g.dim;
    if (g.dim == 2) {
        if (lean) launch_apply_many<TS, 2, 2, K, F32 ? 8 : 16, 128>(g, inv, stride, d, corr, flag, s);
        else launch_apply_many<TS, 2, 3, K, F32 ? 6 : 12, 128>(g, inv, stride, d, corr, flag, s);
    } else {
        if (lean) launch_apply_many<TS, 3, 3, K, F32 ? 6 : 12, 96>(g, inv, stride, d, corr, flag, s);
        else if (F32) launch_apply_many<TS, 3, 4, K, 2, 256>(g, inv, stride, d, corr, flag, s);
        else launch_apply_many<TS, 3, 4, K, 4, 256>(g, inv, stride, d, corr, flag, s);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define NMG_MANY_DISPATCH(g, K, KERN, ...)                               \
    do {                                                                 \
        const bool lean_ = (g).nc == (g).dim;                            \
        if ((g).dim == 2) {                                              \
            if (lean_) pdl_launch(KERN<2, 2, K>, __VA_ARGS__);           \
            else pdl_launch(KERN<2, 3, K>, __VA_ARGS__);                 \
        } else {                                                         \
            if (lean_) pdl_launch(KERN<3, 3, K>, __VA_ARGS__);           \
            else pdl_launch(KERN<3, 4, K>, __VA_ARGS__);                 \
        }                                                                \
    } while (0)

template <int DIM, int NC, int K, int TX, int TY, int TZ, int RS = NC>
static void launch_spmv_many_tile(const Geom& g, const float* A, const float* x, const float* b, float* y,
                                  bool residual, cudaStream_t s) {
    constexpr int NV = NC * K, NS = ((NV / 4) % 2) ? NV : NV + 4;
    const size_t smem = (size_t)(TX + 2) * (TY + 2) * (DIM == 3 ? TZ + 2 : 1) * NS * sizeof(float);
    auto kern = k_spmv_many_tile<DIM, NC, K, TX, TY, TZ, RS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned tiles = (unsigned)(((g.nn[0] + TX - 1) / TX) * ((g.nn[1] + TY - 1) / TY) *
                                      (DIM == 3 ? (g.nn[2] + TZ - 1) / TZ : 1));
    pdl_launch(kern, dim3(tiles), dim3(TX * TY * TZ * (NC / RS)), smem, s, g, A, x, b, y, residual);
}

// Tiles of 3d 16 x 4 x 2 nodes and 2d 32 x 4 nodes.  With 4 unknowns a node
// (3d) two threads share a node, two block rows each (256 threads): a thread
// then holds 16 accumulators and 24 prefetched matrix entries instead of 32
// and 48, and twice the warps are resident.
template <int K>
void launch_spmv_many(const Geom& g, const float* A, const float* x, const float* b, float* y, bool residual,
                      cudaStream_t s) {
    g_launches += 1;
    if (g.dim == 3) {
        if (g.nc == 3) launch_spmv_many_tile<3, 3, K, 16, 4, 2>(g, A, x, b, y, residual, s);
        else launch_spmv_many_tile<3, 4, K, 16, 4, 2, 2>(g, A, x, b, y, residual, s);
    } else {
        if (g.nc == 2) launch_spmv_many_tile<2, 2, K, 32, 4, 1>(g, A, x, b, y, residual, s);
        else launch_spmv_many_tile<2, 3, K, 32, 4, 1>(g, A, x, b, y, residual, s);
    }
}

template <int K, typename TS>
bool launch_vanka_apply_many(const Geom& g, const TS* inv, int64_t stride, const float* d, float* corr, int* flag,
                             cudaStream_t s) {
    // the bulk copies need 16-byte aligned, unpadded-column patch inverses
    const int64_t np = g.np;
    if ((uintptr_t)inv % 16 != 0 || (stride * (int64_t)sizeof(TS)) % 16 != 0 || stride < np * np ||
        stride * (int64_t)sizeof(TS) > np * np * (int64_t)sizeof(TS) + 16)
        return false;
    if (g.patches == 0) return true;
    g_launches += 1;
    apply_many_dispatch<TS, K>(g, inv, stride, d, corr, flag, s);
    return true;
}

template <int K>
void launch_vanka_update_many(const Geom& g, const float* corr, const float* x_in, float* x_out, bool x_zero,
                              float omega, bool average, cudaStream_t s) {
    g_launches += 1;
    NMG_MANY_DISPATCH(g, K, k_vanka_update_many, dim3(blocks_for(g.nodes * (K / 4), 256)), dim3(256), 0, s, g, corr,
                      x_in, x_out, x_zero, omega, average);
}

template <int K>
void launch_restrict_many(const Geom& f, const Geom& c, const float* rf, float* rc, const uint8_t* cmask,
                          cudaStream_t s) {
    g_launches += 1;
    NMG_MANY_DISPATCH(f, K, k_restrict_many, dim3(blocks_for(c.nodes * (K / 4), 256)), dim3(256), 0, s, f, c, rf, rc,
                      cmask);
}

template <int K>
void launch_prolong_add_many(const Geom& f, const Geom& c, const float* ec, float* xf, const uint8_t* fmask,
                             cudaStream_t s) {
    g_launches += 1;
    NMG_MANY_DISPATCH(f, K, k_prolong_add_many, dim3(blocks_for(f.nodes * (K / 4), 256)), dim3(256), 0, s, f, c, ec,
                      xf, fmask);
}

template <int K>
void launch_coarse_gemv_many(const double* inv, int64_t n, const float* b, float* x, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_coarse_gemv_many<K>, dim3(blocks_for(n * 32, 256)), dim3(256), 0, s, inv, n, b, x);
}

template <int K>
void launch_pack(const ColPtrs& src, int ncols, int64_t n, float* out, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_pack<K>, dim3(blocks_for(n, 256)), dim3(256), 0, s, src, ncols, n, out);
}

template <int K>
void launch_unpack(const float* in, const ColPtrsOut& dst, int ncols, int64_t n, cudaStream_t s) {
    g_launches += 1;
    pdl_launch(k_unpack<K>, dim3(blocks_for(n, 256)), dim3(256), 0, s, in, dst, ncols, n);
}

#define NMG_MANY_INST(K)                                                                                          \
    template void launch_spmv_many<K>(const Geom&, const float*, const float*, const float*, float*, bool,         \
                                      cudaStream_t);                                                              \
    template bool launch_vanka_apply_many<K, float>(const Geom&, const float*, int64_t, const float*, float*,      \
                                                    int*, cudaStream_t);                                          \
    template bool launch_vanka_apply_many<K, __nv_bfloat16>(const Geom&, const __nv_bfloat16*, int64_t,            \
                                                            const float*, float*, int*, cudaStream_t);            \
    template void launch_vanka_update_many<K>(const Geom&, const float*, const float*, float*, bool, float, bool,  \
                                              cudaStream_t);                                                      \
    template void launch_restrict_many<K>(const Geom&, const Geom&, const float*, float*, const uint8_t*,          \
                                          cudaStream_t);                                                          \
    template void launch_prolong_add_many<K>(const Geom&, const Geom&, const float*, float*, const uint8_t*,       \
                                             cudaStream_t);                                                       \
    template void launch_coarse_gemv_many<K>(const double*, int64_t, const float*, float*, cudaStream_t);          \
    template void launch_pack<K>(const ColPtrs&, int, int64_t, float*, cudaStream_t);                              \
    template void launch_unpack<K>(const float*, const ColPtrsOut&, int, int64_t, cudaStream_t);
NMG_MANY_INST(4)
NMG_MANY_INST(8)

}  // namespace nmg
