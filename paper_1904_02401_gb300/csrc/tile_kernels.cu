// Tile-fused Vanka smoothing steps for the levels of the V-cycle whose
// kernels are too small to fill the GPU (Section 4.3 (II)-(III), Eq. (vanka)).
//
// One smoothing step of Eq. (vanka) is three data-parallel passes: the defect
// d = b - A x (per node), the patch solves A_i^{-1} R_i d (per patch) and the
// update x += w R_i^T (...) (per node, summing the patches that contain it).
// On a small level each pass is one short kernel whose time is the latency of
// a chain of dependent memory accesses, so a V(2,2) cycle spends ~14 kernel
// latencies per level.  Here one CTA owns a tile of TILE^d patches and does
// all three passes for them in one launch:
//   A. the previous step's update is recomputed on the tile's node region
//      (the owned nodes plus two node layers around them) from the previous
//      iterate and the previous step's patch corrections, kept in shared
//      memory, and written out for the owned nodes (the iterate is stored in
//      the other of two buffers, since neighbouring tiles still read the old
//      one);
//   B. the defect (or the residual) on the tile's patch nodes plus one layer,
//      from the region in shared memory;
//   C. the solves of the owned patches (one warp per patch), corrections to
//      global memory for the next step; or, for the last pre-smoothing step,
//      the full-weighting restriction of the residual to the coarse nodes the
//      tile owns.
// No patch is solved twice; only the cheap update and defect are recomputed
// on the halo.  Every value is produced by the element functions of elem.cuh
// with the same terms in the same order as the one-kernel-per-pass path, so
// the results are bitwise identical to it.
#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

template <typename T, typename TS>
struct TileArgs {
    Geom g, gc;               // the level and the next coarser one (restriction / prolongation)
    int mode;                 // TileMode
    const T* A;               // stencil matrix of the level
    const TS* inv;            // patch inverses (column-major, inv_stride apart)
    int64_t inv_stride;
    const T* b;               // right-hand side of the level
    const T* x_in;            // iterate before the previous update (unused when x_zero)
    const T* corr_in;         // corrections of the previous step
    const T* ec;              // coarse correction (TILE_PROLONG_STEP)
    const uint8_t* fmask;     // Dirichlet mask of the level (TILE_PROLONG_STEP)
    const uint8_t* cmask;     // Dirichlet mask of the coarser level (TILE_RESTRICT)
    T* x_out;                 // iterate after the previous update, owned nodes
    T* corr_out;              // corrections of this step
    T* rc;                    // restricted residual (TILE_RESTRICT)
    T omega;
    bool average;
    bool x_zero;
};

template <int DIM, int TILE>
struct TileShape {
    static constexpr int RX = 2 * TILE + 4;   // region nodes per direction (update recomputed)
    static constexpr int RD = 2 * TILE + 2;   // defect / residual nodes per direction
    static constexpr int NX = DIM == 2 ? RX * RX : RX * RX * RX;
    static constexpr int ND = DIM == 2 ? RD * RD : RD * RD * RD;
    static constexpr int TP = DIM == 2 ? TILE * TILE : TILE * TILE * TILE;
};

template <typename T, typename TS, int DIM, int TILE, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_tile_step(const __grid_constant__ TileArgs<T, TS> a) {
    constexpr int NC = DIM + 1;
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    constexpr int NWARP = THREADS / 32;
    using S = TileShape<DIM, TILE>;
    constexpr int RX = S::RX, RD = S::RD;
    // one warp per owned patch in 2d keeps every patch's 27 inverse loads per
    // lane in flight from the start of the kernel
    constexpr bool PREFETCH = DIM == 2 && NWARP >= S::TP;
    __shared__ T sx[S::NX * NC];
    __shared__ T sd[S::ND * NC];
    __shared__ T sp[NWARP][NP];
    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // tile -> patch range [p0, p1), owned nodes [o0, o1), region [x0, x1),
    // defect nodes [d0, d1) per direction
    int p0[3], p1[3], o0[3], o1[3], x0[3], x1[3], d0[3], d1[3];
    {
        const uint32_t nt0 = (uint32_t)(g.pc[0] + TILE - 1) / TILE;
        const uint32_t nt1 = (uint32_t)(g.pc[1] + TILE - 1) / TILE;
        const uint32_t t = blockIdx.x, ty = t / nt0;
        const int tc[3] = {(int)(t - ty * nt0), DIM == 3 ? (int)(ty % nt1) : (int)ty, DIM == 3 ? (int)(ty / nt1) : 0};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k < DIM) {
                p0[k] = tc[k] * TILE;
                p1[k] = min(p0[k] + TILE, g.pc[k]);
                const bool last = p1[k] == g.pc[k];
                o0[k] = 2 * p0[k];
                o1[k] = last ? 2 * p1[k] + 1 : 2 * p1[k];
                x0[k] = max(0, 2 * p0[k] - 2);
                x1[k] = min(g.nn[k], 2 * p1[k] + 2);
                d0[k] = max(0, 2 * p0[k] - 1);
                d1[k] = min(g.nn[k], 2 * p1[k] + 1);
            } else {
                p0[k] = 0; p1[k] = 1; o0[k] = 0; o1[k] = 1; x0[k] = 0; x1[k] = 1; d0[k] = 0; d1[k] = 1;
            }
        }
    }
    const int np0 = p1[0] - p0[0], np1 = p1[1] - p0[1];
    const int npt = np0 * np1 * (p1[2] - p0[2]);
    const int64_t sy = g.nn[0], sz = (int64_t)g.nn[0] * g.nn[1];
    const bool solve = a.mode == TILE_FIRST || a.mode == TILE_STEP || a.mode == TILE_PROLONG_STEP;

    // the inverses are constant during a solve: their loads may start before
    // the previous kernel has finished
    TS pre[PREFETCH ? NP : 1];
    int64_t my_patch = -1;
    if (solve && warp < npt) {
        const int qx = warp % np0, qr = warp / np0;
        const int qy = qr % np1, qz = qr / np1;
        my_patch = (p0[0] + qx) + (int64_t)g.pc[0] * ((p0[1] + qy) + (int64_t)g.pc[1] * (p0[2] + qz));
        if constexpr (PREFETCH) {
            if (lane < NP) {
                const TS* Ap = a.inv + my_patch * a.inv_stride;
#pragma unroll
                for (int j = 0; j < NP; ++j) pre[j] = ldg(Ap + j * NP + lane);
            }
        }
    }
    NMG_PDL_ENTRY();

    if (a.mode == TILE_FINAL) {   // the last update of the level, owned nodes only
        const int e0 = o1[0] - o0[0], e1 = o1[1] - o0[1], ne = e0 * e1 * (o1[2] - o0[2]);
        for (int li = tid; li < ne; li += THREADS) {
            const int lx = li % e0, lr = li / e0, ly = lr % e1, lz = lr / e1;
            const int64_t j = (o0[0] + lx) + sy * (o0[1] + ly) + sz * (o0[2] + lz);
            T v[NC];
            vanka_update_value<T, DIM>(g, a.corr_in, a.x_in, a.x_zero, a.omega, a.average, j, v);
#pragma unroll
            for (int c = 0; c < NC; ++c) a.x_out[j * NC + c] = v[c];
        }
        return;
    }

    // A. iterate on the region
    if (a.mode != TILE_FIRST) {
        const int e0 = x1[0] - x0[0], e1 = x1[1] - x0[1], ne = e0 * e1 * (x1[2] - x0[2]);
        for (int li = tid; li < ne; li += THREADS) {
            const int lx = li % e0, lr = li / e0, ly = lr % e1, lz = lr / e1;
            const int gx = x0[0] + lx, gy = x0[1] + ly, gz = x0[2] + lz;
            const int64_t j = gx + sy * gy + sz * gz;
            T v[NC];
            if (a.mode == TILE_PROLONG_STEP) prolong_value<T, DIM>(g, a.gc, a.ec, a.x_in, a.fmask, j, v);
            else vanka_update_value<T, DIM>(g, a.corr_in, a.x_in, a.x_zero, a.omega, a.average, j, v);
            const int ls = (gx - x0[0]) + RX * ((gy - x0[1]) + RX * (gz - x0[2]));
#pragma unroll
            for (int c = 0; c < NC; ++c) sx[ls * NC + c] = v[c];
            const bool owned = gx >= o0[0] && gx < o1[0] && gy >= o0[1] && gy < o1[1] && gz >= o0[2] && gz < o1[2];
            if (owned)
#pragma unroll
                for (int c = 0; c < NC; ++c) a.x_out[j * NC + c] = v[c];
        }
        __syncthreads();
    }

    // B. defect (residual) on [d0, d1)
    {
        const int e0 = d1[0] - d0[0], e1 = d1[1] - d0[1], ne = e0 * e1 * (d1[2] - d0[2]);
        for (int li = tid; li < ne; li += THREADS) {
            const int lx = li % e0, lr = li / e0, ly = lr % e1, lz = lr / e1;
            const int gx = d0[0] + lx, gy = d0[1] + ly, gz = d0[2] + lz;
            const int64_t i = gx + sy * gy + sz * gz;
            const int ld = lx + RD * (ly + RD * lz);
            if (a.mode == TILE_FIRST) {
#pragma unroll
                for (int c = 0; c < NC; ++c) sd[ld * NC + c] = a.b[i * NC + c];
            } else {
                const int lc = (gx - x0[0]) + RX * ((gy - x0[1]) + RX * (gz - x0[2]));
                auto sxval = [&](int64_t, int dx, int dy, int dz, T* xv) {
                    const int l = lc + dx + RX * (dy + RX * dz);
#pragma unroll
                    for (int c = 0; c < NC; ++c) xv[c] = sx[l * NC + c];
                };
                T acc[NC];
                // x comes from shared memory; in 2d the matrix loads of 3 stencil positions
                // are in flight together (a larger group does not fit the 512-thread register
                // budget)
                spmv_acc_f<T, DIM, decltype(sxval)&, true, DIM == 2 ? 3 : 1>(g, a.A, sxval, i, acc);
#pragma unroll
                for (int c = 0; c < NC; ++c) sd[ld * NC + c] = a.b[i * NC + c] - acc[c];
            }
        }
        __syncthreads();
    }

    if (a.mode == TILE_RESTRICT) {   // C'. r_c = P^T r on the coarse nodes the tile owns
        const Geom& gc = a.gc;
        int c0[3], c1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c0[k] = k < DIM ? p0[k] : 0;
            c1[k] = k < DIM ? (p1[k] == g.pc[k] ? p1[k] + 1 : p1[k]) : 1;
        }
        const int e0 = c1[0] - c0[0], e1 = c1[1] - c0[1], ne = e0 * e1 * (c1[2] - c0[2]);
        const int64_t csy = gc.nn[0], csz = (int64_t)gc.nn[0] * gc.nn[1];
        const int r0 = d0[0], r1 = d0[1], r2 = d0[2];   // scalars: the lambda keeps them in registers
        for (int li = tid; li < ne; li += THREADS) {
            const int lx = li % e0, lr = li / e0, ly = lr % e1, lz = lr / e1;
            const int64_t I = (c0[0] + lx) + csy * (c0[1] + ly) + csz * (c0[2] + lz);
            T sum[NC];
            restrict_value_f<T, DIM>(
                g, gc,
                [&](int fx, int fy, int fz, int k) {
                    return sd[((fx - r0) + RD * ((fy - r1) + RD * (fz - r2))) * NC + k];
                },
                I, sum);
#pragma unroll
            for (int c = 0; c < NC; ++c) a.rc[I * NC + c] = a.cmask[I * NC + c] ? T(0) : sum[c];
        }
        return;
    }

    // C. patch solves, one warp per patch
    for (int q = warp; q < npt; q += NWARP) {
        const int qx = q % np0, qr = q / np0;
        const int qy = qr % np1, qz = qr / np1;
        const int64_t p = (p0[0] + qx) + (int64_t)g.pc[0] * ((p0[1] + qy) + (int64_t)g.pc[1] * (p0[2] + qz));
        for (int t = lane; t < NP; t += 32) {
            const int an = t / NC, c = t - an * NC;
            const int ax = an % 3, ay = (an / 3) % 3, az = an / 9;
            const int l = (2 * (p0[0] + qx) + ax - d0[0]) +
                          RD * ((2 * (p0[1] + qy) + ay - d0[1]) + RD * (DIM == 3 ? 2 * (p0[2] + qz) + az - d0[2] : 0));
            sp[warp][t] = sd[l * NC + c];
        }
        __syncwarp();
        if constexpr (PREFETCH) {
            // row `lane` summed over the columns in ascending order, as apply_patch
            if (lane < NP) {
                T acc = T(0);
#pragma unroll
                for (int j = 0; j < NP; ++j) acc = fma(Cvt<T, TS>::f(pre[j]), sp[warp][j], acc);
                a.corr_out[p * NP + lane] = acc;
            }
        } else {
            apply_patch<T, TS, DIM, true>(a.inv + p * a.inv_stride, sp[warp], a.corr_out + p * NP, lane);
        }
        __syncwarp();
    }
    (void)my_patch;
}

template <int DIM> struct TileCfg;
template <> struct TileCfg<2> { static constexpr int TILE = 4, THREADS = 512; };
template <> struct TileCfg<3> { static constexpr int TILE = 2, THREADS = 256; };

template <typename T, typename TS, int DIM>
void launch_dim(const TileArgs<T, TS>& a, cudaStream_t s) {
    constexpr int TILE = TileCfg<DIM>::TILE, THREADS = TileCfg<DIM>::THREADS;
    int64_t tiles = 1;
    for (int k = 0; k < DIM; ++k) tiles *= (a.g.pc[k] + TILE - 1) / TILE;
    pdl_launch(k_tile_step<T, TS, DIM, TILE, THREADS>, dim3((unsigned)tiles), dim3(THREADS), 0, s, a);
}

}  // namespace

template <typename T, typename TS>
void launch_tile_step(const Geom& g, const Geom& gc, int mode, const T* A, const TS* inv, int64_t inv_stride,
                      const T* b, const T* x_in, bool x_zero, const T* corr_in, const T* ec, const uint8_t* fmask,
                      const uint8_t* cmask, T* x_out, T* corr_out, T* rc, T omega, bool average, cudaStream_t s) {
    g_launches += 1;
    TileArgs<T, TS> a;
    a.g = g;
    a.gc = gc;
    a.mode = mode;
    a.A = A;
    a.inv = inv;
    a.inv_stride = inv_stride;
    a.b = b;
    a.x_in = x_in;
    a.corr_in = corr_in;
    a.ec = ec;
    a.fmask = fmask;
    a.cmask = cmask;
    a.x_out = x_out;
    a.corr_out = corr_out;
    a.rc = rc;
    a.omega = omega;
    a.average = average;
    a.x_zero = x_zero;
    if (g.dim == 2) launch_dim<T, TS, 2>(a, s);
    else launch_dim<T, TS, 3>(a, s);
}

#define NMG_TILE_INST(T, TS)                                                                                     \
    template void launch_tile_step<T, TS>(const Geom&, const Geom&, int, const T*, const TS*, int64_t, const T*, \
                                          const T*, bool, const T*, const T*, const uint8_t*, const uint8_t*, T*, \
                                          T*, T*, T, bool, cudaStream_t);
NMG_TILE_INST(double, double)
NMG_TILE_INST(float, float)
NMG_TILE_INST(float, __nv_bfloat16)
#undef NMG_TILE_INST

}  // namespace nmg
