// Per-element device functions of the V-cycle, shared by the one-kernel-per-
// step path (smooth_kernels.cu) and the persistent V-cycle (persistent.cu), so
// both paths perform the same arithmetic in the same order.
#pragma once

#include "nmg_internal.cuh"

namespace nmg {
namespace elem {

template <typename T, typename TS> struct Cvt;
template <> struct Cvt<double, double> { static __device__ __forceinline__ double f(double v) { return v; } };
template <> struct Cvt<float, float> { static __device__ __forceinline__ float f(float v) { return v; } };
template <> struct Cvt<float, __nv_bfloat16> {
    static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// Exact float -> double widening with integer instructions (GB300 retires
// about two FP64 operations per SM clock, so conversions on the FP64 pipe are
// not free): the same value as a conversion instruction for zeros, normal and
// subnormal numbers and infinities (IEEE 754 binary32 -> binary64 field
// mapping: exponent rebias by 1023 - 127, fraction shifted left by 29).
__device__ __forceinline__ double widen_exact(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu;
    uint32_t m = u & 0x7fffffu;
    uint64_t bits;
    if (e - 1u < 0xfeu) {                                   // normal
        bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
    } else if (e == 0xffu) {                                // infinity, NaN
        bits = sign | (0x7ffull << 52) | ((uint64_t)m << 29);
    } else if (m == 0u) {                                   // zero
        bits = sign;
    } else {                                                // subnormal: normalise
        const int sh = __clz((int)m) - 8;                   // moves the leading one to bit 23
        m = (m << sh) & 0x7fffffu;
        bits = sign | ((uint64_t)(897 - sh) << 52) | ((uint64_t)m << 29);
    }
    return __longlong_as_double((long long)bits);
}
template <typename T, typename TX> __device__ __forceinline__ T widen(TX v) { return (T)v; }
template <> __device__ __forceinline__ double widen<double, float>(float v) { return widen_exact(v); }

// N consecutive matrix entries at Ab (3d stencil layout: a node's block of
// one position, or consecutive rows of it): float4 loads when N is a multiple
// of 4 (FP32), double2 loads when N is even (FP64), else entry by entry.  The
// 3d layout keeps such runs 16-byte aligned (cudaMalloc'd base, blocks of 16
// entries, rows of 4).
template <typename T, int N>
__device__ __forceinline__ void load_arun(const T* __restrict__ Ab, T (&av)[N]) {
    if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(Ab) + q);
            av[4 * q] = v.x; av[4 * q + 1] = v.y; av[4 * q + 2] = v.z; av[4 * q + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            const double2 v = __ldg(reinterpret_cast<const double2*>(Ab) + q);
            av[2 * q] = v.x; av[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) av[e] = __ldg(Ab + e);
    }
}

template <typename TS> __device__ __forceinline__ TS ldg(const TS* p) { return __ldg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldg<__nv_bfloat16>(const __nv_bfloat16* p) { return *p; }

// Index arithmetic in 32 bits (node and patch counts stay below 2^31; 64-bit
// division is a long emulated sequence on the critical path of small levels).
__device__ __forceinline__ void node_xyz(const Geom& g, int64_t i, int& x, int& y, int& z) {
    const uint32_t ii = (uint32_t)i, n0 = (uint32_t)g.nn[0], n1 = (uint32_t)g.nn[1];
    const uint32_t t = ii / n0;
    x = (int)(ii - t * n0);
    const uint32_t u = t / n1;
    y = (int)(t - u * n1);
    z = (int)u;
}

__device__ __forceinline__ void patch_xyz(const Geom& g, int64_t p, int& px, int& py, int& pz) {
    const uint32_t pp = (uint32_t)p, c0 = (uint32_t)g.pc[0], c1 = (uint32_t)g.pc[1];
    const uint32_t t = pp / c0;
    px = (int)(pp - t * c0);
    const uint32_t u = t / c1;
    py = (int)(t - u * c1);
    pz = (int)u;
}

__device__ __forceinline__ int64_t patch_node(const Geom& g, int px, int py, int pz, int an) {
    const int ax = an % 3, ay = (an / 3) % 3, az = an / 9;
    return (int64_t)(2 * px + ax) + (int64_t)g.nn[0] * ((2 * py + ay) + (int64_t)g.nn[1] * (2 * pz + az));
}

// acc = (A x)_i for node i (stencil layout), summed over the stencil positions
// in ascending order and, inside a block, over the columns; the values of x at
// the neighbour j = i + (dx, dy, dz) come from xval(j, dx, dy, dz, xv) (loaded,
// converted, recomputed or read from a shared-memory tile).  The loads of G
// consecutive stencil positions are issued before their products (an absent
// neighbour reads the node itself and a zero of the padded matrix, and its
// terms are skipped), so a thread waits for one memory round trip per group,
// not per position; the products are the same terms in the same order.
// GB = 0 picks G: for a 2d matrix in global memory 9 (FP32) or 3 (FP64: 9
// positions of 9 doubles and 3 neighbour values take over 200 registers), else
// 1 (a matrix in shared memory has no latency to hide; in 3d a position's
// block is one contiguous run of the layout, read with vector loads, and
// grouping positions measured slower on GB300); kernels with few registers
// per thread pass a smaller G.
template <typename T, int DIM, class XF, bool GLOBAL_A = true, int GB = 0, int NC>
__device__ __forceinline__ void spmv_acc_f(const Geom& g, const T* __restrict__ A, XF&& xval, int64_t i,
                                           T (&acc)[NC]) {
    constexpr int NB = NC * NC;
    constexpr int NST = (DIM == 2) ? 9 : 27;
    constexpr int G = GB > 0 ? GB : (GLOBAL_A && DIM == 2) ? (sizeof(T) == 8 ? 3 : 9) : 1;
    static_assert(NST % G == 0, "stencil positions per load group must divide the stencil");
    int ix, iy, iz;
    node_xyz(g, i, ix, iy, iz);
    const int64_t sy = g.nn[0], sz = (int64_t)g.nn[0] * g.nn[1];
#pragma unroll
    for (int r = 0; r < NC; ++r) acc[r] = T(0);
    if constexpr (G == 1) {   // one position at a time, its loads only when the neighbour exists
#pragma unroll
        for (int s = 0; s < NST; ++s) {
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
            const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                            (iz + dz >= 0) && (iz + dz < g.nn[2]);
            if (ok) {
                const int64_t j = i + dx + dy * sy + dz * sz;
                T xv[NC];
                xval(j, dx, dy, dz, xv);
                const T* As = A + stencil_off<DIM, NB>(g.ld, s, 0, i);
                if constexpr (DIM == 3 && GLOBAL_A) {   // the node's block: one contiguous segment
                    T av[NB];
                    load_arun<T, NB>(As, av);
#pragma unroll
                    for (int r = 0; r < NC; ++r)
#pragma unroll
                        for (int c = 0; c < NC; ++c) acc[r] = fma(av[r * NC + c], xv[c], acc[r]);
                } else {
                    const int64_t es = stencil_estride<DIM>(g.ld);
#pragma unroll
                    for (int r = 0; r < NC; ++r)
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const T* a = As + (int64_t)(r * NC + c) * es;
                            T av;
                            if constexpr (GLOBAL_A) av = __ldg(a);
                            else av = *a;
                            acc[r] = fma(av, xv[c], acc[r]);
                        }
                }
            }
        }
        return;
    }
#pragma unroll
    for (int s0 = 0; s0 < NST; s0 += G) {
        T av[G][NB], xv[G][NC];
        bool okv[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int s = s0 + q;
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
            const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                            (iz + dz >= 0) && (iz + dz < g.nn[2]);
            okv[q] = ok;
            const int64_t j = ok ? i + dx + dy * sy + dz * sz : i;
            xval(j, ok ? dx : 0, ok ? dy : 0, ok ? dz : 0, xv[q]);
            const T* As = A + stencil_off<DIM, NB>(g.ld, s, 0, i);
            const int64_t es = stencil_estride<DIM>(g.ld);
#pragma unroll
            for (int e = 0; e < NB; ++e) {
                if constexpr (GLOBAL_A) av[q][e] = __ldg(As + (int64_t)e * es);
                else av[q][e] = As[(int64_t)e * es];
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q)
            if (okv[q])
#pragma unroll
                for (int r = 0; r < NC; ++r)
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[r] = fma(av[q][r * NC + c], xv[q][c], acc[r]);
    }
}

// y_i = (A x)_i or b_i - (A x)_i for node i (stencil layout); the values of x
// at a node j come from xval(j, xv) (loaded, converted or recomputed).
template <typename T, int DIM, class XF, bool GLOBAL_A = true, int GB = 0, int NC = DIM + 1>
__device__ __forceinline__ void spmv_node_f(const Geom& g, const T* __restrict__ A, XF&& xval,
                                            const T* __restrict__ b, T* __restrict__ y, bool residual, int64_t i) {
    T acc[NC];
    auto xv4 = [&](int64_t j, int, int, int, T* xv) { xval(j, xv); };
    spmv_acc_f<T, DIM, decltype(xv4)&, GLOBAL_A, GB>(g, A, xv4, i, acc);
#pragma unroll
    for (int r = 0; r < NC; ++r) y[i * NC + r] = residual ? b[i * NC + r] - acc[r] : acc[r];
}

// y_i = (A x)_i or b_i - (A x)_i with x stored as TX (converted to T on load);
// GLOBAL_A = false when A lives in shared memory.
template <typename T, int DIM, typename TX = T, bool GLOBAL_A = true, int GB = 0, int NC = DIM + 1>
__device__ __forceinline__ void spmv_node(const Geom& g, const T* __restrict__ A, const TX* __restrict__ x,
                                          const T* __restrict__ b, T* __restrict__ y, bool residual, int64_t i) {
    auto xval = [&](int64_t j, T* xv) {
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] = widen<T, TX>(x[j * NC + c]);
    };
    spmv_node_f<T, DIM, decltype(xval)&, GLOBAL_A, GB, NC>(g, A, xval, b, y, residual, i);
}

// The NC values of node block j of x: with VEC (NC = 4, x 16-byte aligned)
// one float4 or two double2 loads instead of NC scalar loads.
template <typename T, int NC, bool VEC>
__device__ __forceinline__ void load_xblock(const T* __restrict__ xj, T (&xv)[NC]) {
    if constexpr (VEC && NC == 4 && sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(xj);
        xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
    } else if constexpr (VEC && NC == 4 && sizeof(T) == 8) {
        const double2 v0 = reinterpret_cast<const double2*>(xj)[0];
        const double2 v1 = reinterpret_cast<const double2*>(xj)[1];
        xv[0] = v0.x; xv[1] = v0.y; xv[2] = v1.x; xv[3] = v1.y;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] = xj[c];
    }
}

// Row r of node i of y = A x or b - A x: the same terms in the same order as
// row r of spmv_node (stencil positions ascending, then block columns), so the
// value is bitwise equal; lets a kernel spread a node's rows over threads.
// In 2d the loads of the 9 stencil positions are issued before their
// products (in 3d one position at a time measured faster).  VEC: x blocks
// are read with vector loads (NC = 4 and x 16-byte aligned; same values).
template <typename T, int DIM, int NC = DIM + 1, bool VEC = false>
__device__ __forceinline__ void spmv_row(const Geom& g, const T* __restrict__ A, const T* __restrict__ x,
                                         const T* __restrict__ b, T* __restrict__ y, bool residual, int64_t i,
                                         int r) {
    constexpr int NB = NC * NC;
    constexpr int NST = (DIM == 2) ? 9 : 27;
    constexpr int G = DIM == 2 ? 9 : 1;
    int ix, iy, iz;
    node_xyz(g, i, ix, iy, iz);
    const int64_t sy = g.nn[0], sz = (int64_t)g.nn[0] * g.nn[1];
    T acc = T(0);
    if constexpr (G == 1) {   // one position at a time, its loads only when the neighbour exists
#pragma unroll
        for (int s = 0; s < NST; ++s) {
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
            const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                            (iz + dz >= 0) && (iz + dz < g.nn[2]);
            if (ok) {
                const int64_t j = i + dx + dy * sy + dz * sz;
                const T* As = A + stencil_off<DIM, NB>(g.ld, s, r * NC, i);
                T xv[NC];
                load_xblock<T, NC, VEC>(x + j * NC, xv);
                if constexpr (DIM == 3) {   // the row's NC entries are contiguous (vector loads for NC = 4)
                    T av[NC];
                    load_arun<T, NC>(As, av);
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc = fma(av[c], xv[c], acc);
                } else {
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc = fma(__ldg(As + (int64_t)c * g.ld), xv[c], acc);
                }
            }
        }
        y[i * NC + r] = residual ? b[i * NC + r] - acc : acc;
        return;
    }
#pragma unroll
    for (int s0 = 0; s0 < NST; s0 += G) {
        T av[G][NC], xv[G][NC];
        bool okv[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int s = s0 + q;
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
            const bool ok = (ix + dx >= 0) && (ix + dx < g.nn[0]) && (iy + dy >= 0) && (iy + dy < g.nn[1]) &&
                            (iz + dz >= 0) && (iz + dz < g.nn[2]);
            okv[q] = ok;
            const int64_t j = ok ? i + dx + dy * sy + dz * sz : i;
            const T* As = A + stencil_off<DIM, NB>(g.ld, s, r * NC, i);
            const int64_t es = stencil_estride<DIM>(g.ld);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                av[q][c] = __ldg(As + (int64_t)c * es);
                xv[q][c] = x[j * NC + c];
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q)
            if (okv[q])
#pragma unroll
                for (int c = 0; c < NC; ++c) acc = fma(av[q][c], xv[q][c], acc);
    }
    y[i * NC + r] = residual ? b[i * NC + r] - acc : acc;
}

// Gathers R_p d into sd[0..NP) (called by one warp; lane-strided).
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void gather_patch(const Geom& g, const T* __restrict__ d, int64_t p, T* sd, int lane) {
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    int px, py, pz;
    patch_xyz(g, p, px, py, pz);
    for (int t = lane; t < NP; t += 32) {
        const int an = t / NC, c = t - an * NC;
        sd[t] = d[patch_node(g, px, py, pz, an) * NC + c];
    }
}

// corr_p = A_p^{-1} sd for one patch by one warp (lane owns rows lane + 32 q);
// Ap: column-major inverse (global or shared memory).
template <typename T, typename TS, int DIM, bool GLOBAL, int NC = DIM + 1>
__device__ __forceinline__ void apply_patch(const TS* Ap, const T* sd, T* __restrict__ corr_p, int lane) {
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    constexpr int NQ = (NP + 31) / 32;
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    if (DIM == 2) {
        // 27 columns: issue all loads first so they are in flight together (one
        // memory latency per patch instead of one per column), then sum in order
        if (lane < NP) {
            TS a[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) a[j] = GLOBAL ? ldg(Ap + j * NP + lane) : Ap[j * NP + lane];
#pragma unroll
            for (int j = 0; j < NP; ++j) acc[0] = fma(Cvt<T, TS>::f(a[j]), sd[j], acc[0]);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < NP; ++j) {
            const T dj = sd[j];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int row = lane + 32 * q;
                if (row < NP) {
                    const TS a = GLOBAL ? ldg(Ap + j * NP + row) : Ap[j * NP + row];
                    acc[q] = fma(Cvt<T, TS>::f(a), dj, acc[q]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int row = lane + 32 * q;
        if (row < NP) corr_p[row] = acc[q];
    }
}

// v = x_i + w_i * (sum of the corrections of the patches containing node i),
// in ascending patch order; w_i = omega / multiplicity ("average") or omega;
// x_i = 0 when x_zero (x is not read).
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void vanka_update_value(const Geom& g, const T* __restrict__ corr,
                                                   const T* __restrict__ x, bool x_zero, T omega, bool average,
                                                   int64_t i, T* v) {
    constexpr int NP = ((DIM == 2) ? 9 : 27) * NC;
    int xyz[3];
    node_xyz(g, i, xyz[0], xyz[1], xyz[2]);
    int cp[3][2], cl[3][2], cnt[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = xyz[k];
        if (k >= DIM) { cp[k][0] = cp[k][1] = 0; cl[k][0] = cl[k][1] = 0; cnt[k] = 1; continue; }
        if (c & 1) {   // inside one patch
            cp[k][0] = cp[k][1] = (c - 1) >> 1;
            cl[k][0] = cl[k][1] = 1;
            cnt[k] = 1;
        } else {       // on a patch boundary: the lower patch (if any) first, then the upper
            const bool lo = c > 0, hi = c < g.cells[k];
            cp[k][0] = lo ? (c >> 1) - 1 : c >> 1;
            cl[k][0] = lo ? 2 : 0;
            cp[k][1] = c >> 1;
            cl[k][1] = 0;
            cnt[k] = (int)lo + (int)hi;
        }
    }
    // the corrections of the (at most 2^d) patches are loaded first (an absent
    // patch reads the first one again), then summed in ascending patch order
    constexpr int NZ = DIM == 3 ? 2 : 1;
    T cv[NZ][2][2][NC];
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
                const T* cpn = corr + p * NP + loc * NC;
#pragma unroll
                for (int c = 0; c < NC; ++c) cv[a][b][e][c] = cpn[c];
            }
    T sum[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sum[c] = T(0);
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (a < cnt[2] && b < cnt[1] && e < cnt[0])
#pragma unroll
                    for (int c = 0; c < NC; ++c) sum[c] += cv[a][b][e][c];
    const int m = cnt[0] * cnt[1] * cnt[2];
    const T wgt = average ? omega / T(m) : omega;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const T old = x_zero ? T(0) : x[i * NC + c];
        v[c] = fma(wgt, sum[c], old);
    }
}

// x_out_i = x_in_i + w_i * sum of the corrections (x_in may equal x_out).
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void vanka_update_node(const Geom& g, const T* __restrict__ corr, const T* x_in,
                                                  T* x_out, bool x_zero, T omega, bool average, int64_t i) {
    T v[NC];
    vanka_update_value<T, DIM, NC>(g, corr, x_in, x_zero, omega, average, i, v);
#pragma unroll
    for (int c = 0; c < NC; ++c) x_out[i * NC + c] = v[c];
}

// Fused: x_out_i = update of x_in at node i (as above) and
// r_i = b_i - (A x_out)_i with x_out at the neighbours recomputed the same way.
// x_out must not alias x_in.
template <typename T, int DIM>
__device__ __forceinline__ void update_residual_node(const Geom& g, const T* __restrict__ A,
                                                     const T* __restrict__ corr, const T* __restrict__ x_in,
                                                     bool x_zero, T omega, bool average, const T* __restrict__ b,
                                                     T* __restrict__ x_out, T* __restrict__ r, int64_t i) {
    vanka_update_node<T, DIM>(g, corr, x_in, x_out, x_zero, omega, average, i);
    spmv_node_f<T, DIM>(
        g, A, [&](int64_t j, T* xv) { vanka_update_value<T, DIM>(g, corr, x_in, x_zero, omega, average, j, xv); },
        b, r, true, i);
}

// sum = (P^T r_f)_I for coarse node I (Q1 full weighting), the fine values
// coming from rval(fx, fy, fz, k) (global memory or a shared-memory tile).
template <typename T, int DIM, class RF, int NC>
__device__ __forceinline__ void restrict_value_f(const Geom& f, const Geom& c, RF&& rval, int64_t I,
                                                 T (&sum)[NC]) {
    int X, Y, Z;
    node_xyz(c, I, X, Y, Z);
#pragma unroll
    for (int k = 0; k < NC; ++k) sum[k] = T(0);
    // per plane of fine nodes: the 3 x 3 values are loaded first (an absent node
    // reads the centre again), then summed in order with their weights
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
#pragma unroll
    for (int oz = zlo; oz <= zhi; ++oz) {
        const int fz = 2 * Z + oz;
        if (fz < 0 || fz >= f.nn[2]) continue;
        T rv[3][3][NC];
        bool in[3][3];
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int fy = 2 * Y + oy, fx = 2 * X + ox;
                const bool ok = fy >= 0 && fy < f.nn[1] && fx >= 0 && fx < f.nn[0];
                in[oy + 1][ox + 1] = ok;
#pragma unroll
                for (int k = 0; k < NC; ++k) rv[oy + 1][ox + 1][k] = rval(ok ? fx : 2 * X, ok ? fy : 2 * Y, fz, k);
            }
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox)
                if (in[oy + 1][ox + 1]) {
                    const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
#pragma unroll
                    for (int k = 0; k < NC; ++k) sum[k] = fma(w, rv[oy + 1][ox + 1][k], sum[k]);
                }
    }
}

// (r_c)_I = (P^T r_f)_I, zero on coarse Dirichlet entries.
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void restrict_node(const Geom& f, const Geom& c, const T* __restrict__ rf,
                                              T* __restrict__ rc, const uint8_t* __restrict__ cmask, int64_t I) {
    T sum[NC];
    restrict_value_f<T, DIM>(
        f, c,
        [&](int fx, int fy, int fz, int k) {
            return rf[(fx + (int64_t)f.nn[0] * (fy + (int64_t)f.nn[1] * fz)) * NC + k];
        },
        I, sum);
#pragma unroll
    for (int k = 0; k < NC; ++k) rc[I * NC + k] = cmask[I * NC + k] ? T(0) : sum[k];
}

// v = x_in_i + (P e_c)_i, x_in_i on fine Dirichlet entries.
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void prolong_value(const Geom& f, const Geom& c, const T* __restrict__ ec,
                                              const T* __restrict__ x_in, const uint8_t* __restrict__ fmask,
                                              int64_t i, T* v) {
    int xyz[3];
    node_xyz(f, i, xyz[0], xyz[1], xyz[2]);
    int ci[3][2], cnt[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int v = xyz[k];
        if (k >= DIM || !(v & 1)) { ci[k][0] = ci[k][1] = v >> 1; cnt[k] = 1; }
        else { ci[k][0] = (v - 1) >> 1; ci[k][1] = (v + 1) >> 1; cnt[k] = 2; }
    }
    // the (at most 2^d) coarse values are loaded first, then summed in order
    constexpr int NZ = DIM == 3 ? 2 : 1;
    T ev[NZ][2][2][NC];
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t I = ci[0][e] + (int64_t)c.nn[0] * (ci[1][b] + (int64_t)c.nn[1] * ci[2][a]);
#pragma unroll
                for (int k = 0; k < NC; ++k) ev[a][b][e][k] = ec[I * NC + k];
            }
    T sum[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) sum[k] = T(0);
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (a < cnt[2] && b < cnt[1] && e < cnt[0]) {
                    const T w = (cnt[0] == 2 ? T(0.5) : T(1)) * (cnt[1] == 2 ? T(0.5) : T(1)) *
                                (cnt[2] == 2 ? T(0.5) : T(1));
#pragma unroll
                    for (int k = 0; k < NC; ++k) sum[k] = fma(w, ev[a][b][e][k], sum[k]);
                }
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = fmask[i * NC + k] ? x_in[i * NC + k] : x_in[i * NC + k] + sum[k];
}

// (x_f)_i += (P e_c)_i, fine Dirichlet entries untouched.
template <typename T, int DIM, int NC = DIM + 1>
__device__ __forceinline__ void prolong_node(const Geom& f, const Geom& c, const T* __restrict__ ec,
                                             T* __restrict__ xf, const uint8_t* __restrict__ fmask, int64_t i) {
    T v[NC];
    prolong_value<T, DIM, NC>(f, c, ec, xf, fmask, i, v);
#pragma unroll
    for (int k = 0; k < NC; ++k) xf[i * NC + k] = v[k];
}

// Fused: x_out_i = x_in_i + (P e_c)_i and r_i = b_i - (A x_out)_i with x_out at
// the neighbours recomputed the same way.  x_out must not alias x_in.
template <typename T, int DIM>
__device__ __forceinline__ void prolong_residual_node(const Geom& f, const Geom& c, const T* __restrict__ A,
                                                      const T* __restrict__ ec, const T* __restrict__ x_in,
                                                      const uint8_t* __restrict__ fmask, const T* __restrict__ b,
                                                      T* __restrict__ x_out, T* __restrict__ r, int64_t i) {
    T v[DIM + 1];
    prolong_value<T, DIM>(f, c, ec, x_in, fmask, i, v);
#pragma unroll
    for (int k = 0; k < DIM + 1; ++k) x_out[i * (DIM + 1) + k] = v[k];
    spmv_node_f<T, DIM>(
        f, A, [&](int64_t j, T* xv) { prolong_value<T, DIM>(f, c, ec, x_in, fmask, j, xv); }, b, r, true, i);
}

// x_row = (inv b)_row with FP64 sums, by one warp.
template <typename T>
__device__ __forceinline__ void coarse_row(const double* __restrict__ inv, int64_t n, const T* __restrict__ b,
                                           T* __restrict__ x, int64_t row, int lane) {
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s = fma(inv[row * n + j], (double)b[j], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) x[row] = (T)s;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done;
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Asynchronous copy of one 4- or 8-byte element global -> shared (cp.async;
// completion tracked per thread by commit / wait groups).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst_smem)), "l"(src), "n"(sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One TMA bulk copy of `bytes` (multiple of 16, 16-byte aligned ends) completing on bar.
__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst_smem)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace elem
}  // namespace nmg
