// Internal declarations of libnmg: device data layout of a hierarchy and the
// host-side launchers of every kernel.  Nothing here crosses the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/nmg.h"

namespace nmg {

constexpr int kMaxLevels = 16;
constexpr int kMaxRestart = 64;
constexpr int kMaxDevices = 64;       // per-device caches of launch shapes
constexpr int kDotBlocks = 304;        // fixed grid of the deterministic reductions (2 per SM of a GB300's 152)

// ---------------------------------------------------------------------------
// Structured level geometry (uniform Q1 mesh, nodes x fastest)
// ---------------------------------------------------------------------------
struct Geom {
    int dim;
    int nc;            // components per node = dim + 1
    int cells[3];      // cells per direction (1 in unused directions)
    int nn[3];         // nodes per direction (1 in unused directions)
    int64_t nodes;     // nn[0] * nn[1] * nn[2]
    int64_t ld;        // leading dimension of the stencil arrays (nodes rounded up to 32)
    int pc[3];         // patches per direction (cells / 2)
    int64_t patches;
    int np;            // unknowns per patch = 3^dim * nc
    int nst;           // stencil positions 3^dim
};

// Matrix of one level in "stencil" layout: for stencil position s (offset
// o(s) in {-1,0,1}^dim, s = sum (o_k + 1) 3^k) and block entry e = r * nc + c,
// value A[stencil_off(dim, nc * nc, ld, s, e, node)].  Out-of-mesh neighbours
// hold zero.
// * 2d: one array per (s, e), A[(s * nc * nc + e) * ld + node]: a warp's load
//   of one entry for consecutive nodes is one contiguous, coalesced segment.
// * 3d: per position, the node's nc * nc entries contiguous,
//   A[(s * ld + node) * nc * nc + e]: the 16-entry FP32 block of a node and
//   position is one 64-byte segment (four 16-byte loads), and consecutive
//   nodes' blocks follow each other, so a warp's loads of one position cover
//   one contiguous range.  With one array per (s, e) the 3d product's warps
//   kept loads to 432 arrays in flight at once and ran 11-17% slower than in
//   this layout at 64^3 and 96^3 (the same loads, the same order of the sums).
__host__ __device__ __forceinline__ int64_t stencil_off(int dim, int nb, int64_t ld, int s, int e, int64_t node) {
    return dim == 3 ? ((int64_t)s * ld + node) * nb + e : ((int64_t)s * nb + e) * ld + node;
}
template <int DIM, int NB>
__host__ __device__ __forceinline__ int64_t stencil_off(int64_t ld, int s, int e, int64_t node) {
    return DIM == 3 ? ((int64_t)s * ld + node) * NB + e : ((int64_t)s * NB + e) * ld + node;
}
// Distance between block entries e and e + 1 of one node and position.
template <int DIM>
__host__ __device__ __forceinline__ int64_t stencil_estride(int64_t ld) {
    return DIM == 3 ? 1 : ld;
}

template <typename T> struct VTypes;   // vector arithmetic type per storage precision

struct PrecData {                 // per-precision data of one level
    void* A = nullptr;            // stencil matrix in the arithmetic type (double / float)
    void* inv = nullptr;          // patch inverses, column-major n_p x n_p, padded stride
    int64_t inv_stride = 0;       // elements between consecutive patch inverses
    void* b = nullptr;            // V-cycle work vectors of the level (arithmetic type)
    void* x = nullptr;
    void* r = nullptr;
    void* corr = nullptr;         // per-patch corrections A_i^{-1} R_i d, patches * n_p
    void* x2 = nullptr;           // second iterate buffer of the fused V-cycle (ping-pong with x)
    void* corr2 = nullptr;        // second correction buffer of the tile-fused steps (ping-pong with corr)
};

// Multi-vector V-cycle buffers of one level (FP32, K columns interleaved:
// value (u, k) at u * K + k), allocated on the first multi-vector call.
struct MultiData {
    float* b = nullptr;
    float* x = nullptr;
    float* r = nullptr;
    float* corr = nullptr;        // patches * n_p * K
};

// Patches of two sizes on a level (Section 5.5.1; nmg_set_large_patches).
// nsmall blocks of 2^d cells, listed by their index on the level's regular
// patch grid (small_id), with their inverses and corrections stored in list
// order in the level's regular buffers; nlarge blocks of 4^d cells (5^d
// nodes, np_large unknowns), listed by the regular index of their lowest
// 2^d-cell block (large_org), with inverses and corrections of their own.
// inc: per node kIncMax offsets of its correction entries (component 0) in
// the concatenation [small corrections, large corrections], in patch order;
// inc_n: how many.
constexpr int kIncMax = 8;
struct Mixed {
    bool on = false;
    int64_t nsmall = 0, nlarge = 0;
    int np_large = 0;
    int32_t* small_id = nullptr;
    int32_t* large_org = nullptr;
    int32_t* inc = nullptr;
    uint8_t* inc_n = nullptr;
    void* inv_large[3] = {nullptr, nullptr, nullptr};
    int64_t stride_large[3] = {0, 0, 0};
    void* corr_large[2] = {nullptr, nullptr};    // FP64 / FP32 (shared by FP32 and BF16)
    std::vector<std::pair<void*, size_t>> owned;  // allocations to release when the layout changes
};

struct Level {
    Geom g;
    bool ready = false;
    Mixed mixed;
    double* A64 = nullptr;        // FP64 stencil matrix (always kept: outer FGMRES + FP64 mode)
    uint8_t* mask = nullptr;      // Dirichlet flag per unknown
    PrecData p[3];                // NMG_PREC_FP64 / FP32 / BF16
    MultiData m;
};

struct Hierarchy {
    nmg_mesh_desc desc;
    int dim = 0, nc = 0, L = 0;
    int prec_mask = 0;
    cudaStream_t stream = nullptr;
    Level lev[kMaxLevels];
    // coarse level dense inverse (FP64), n0 x n0 row-major
    double* coarse_inv = nullptr;
    int64_t n0 = 0;
    // outer FGMRES (FP64) workspace on the finest level
    double* b64 = nullptr;        // right-hand side copy
    double* x64 = nullptr;        // iterate
    double* w64 = nullptr;        // Arnoldi vector
    double* V = nullptr;          // (m + 1) Krylov vectors
    double* Z = nullptr;          // m preconditioned vectors
    double* partial = nullptr;    // block partial sums of the reductions ((kMaxRestart + 2) * kDotBlocks)
    double* scal = nullptr;       // device scalars (see krylov kernels)
    double* host_scal = nullptr;  // pinned mirror of a few scalars
    int* host_flags = nullptr;    // pinned mirror of the flags and the wait-timeout flag
    int* flags = nullptr;         // device error flags
    int* cyc = nullptr;           // device state of the restart cycle: step j, iterations, stopped
    int* host_cyc = nullptr;      // pinned mirror of cyc
    int m_alloc = 0;
    int krylov_gen = 0;           // bumped when V / Z are reallocated
    // restart cycles as one graph with an on-device loop, per precision
    struct LoopKey {
        int nu1, nu2, weighting, engine, tail, tile, restart, maxit, gen;
        double omega, rtol;
    };
    cudaGraphExec_t cgraph[3] = {nullptr, nullptr, nullptr};
    LoopKey cgraph_key[3] = {};
    int64_t cgraph_nodes[3] = {0, 0, 0};   // kernels per loop step
    int loop_mode = 0;                     // 0 untried, 1 with PDL edges, 2 without, -1 unavailable
    size_t bytes = 0;
    // CUDA graphs of the V-cycle, per precision (rebuilt when options change)
    cudaGraphExec_t vgraph[3] = {nullptr, nullptr, nullptr};
    int vgraph_key[3][5] = {};    // nu1, nu2, weighting, tail / fused, tile threshold
    double vgraph_omega[3] = {0, 0, 0};
    // profiling of the finest-level Vanka apply
    int prof = 0;                        // 0 off, 1 events per V-cycle, 2 per finest-level Vanka apply
    std::vector<cudaEvent_t> prof_ev;   // pairs
    int prof_used = 0;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    int64_t launches = 0;               // kernels enqueued (graph nodes counted per replay)
    int64_t vgraph_nodes[3] = {0, 0, 0};
    // persistent V-cycle: grid barrier state and the engine AUTO picked per precision
    unsigned* pbar = nullptr;
    int wait_limit = 0;                  // > 0: iteration limit of the persistent grid-barrier wait
    bool mixed_any = false;              // some level has patches of two sizes
    // extension problems (ncomp = dim): the finest level's operator before the reduction of its
    // fixed rows and columns (stencil layout, FP64), and the work vectors of nmg_newton_substeps
    double* lift64 = nullptr;
    bool lift_ready = false;
    double* sub_vec[4] = {nullptr, nullptr, nullptr, nullptr};   // r, b5, du on the fixed nodes, rhs
    uint8_t* sub_nodes = nullptr;                                 // flags of the deformation update
    unsigned* counters = nullptr;        // last-block tickets of the fused reductions
    int engine_choice[3] = {0, 0, 0};
    int fused[3] = {0, 0, 0};            // per-step engine: fused update/prolongation + residual kernels
    int tail_patches[3] = {0, 0, 0};     // levels with at most this many patches run in the cluster tail
    int auto_tail[3] = {0, 0, 0};        // the autotuner's pick of tail_patches
                                         // (0: none; the autotuner may pick a threshold)
    int tile_patches[3] = {0, 0, 0};     // levels above the tail with at most this many patches run
                                         // tile-fused smoothing steps (tile_kernels.cu)
    int auto_tile[3] = {0, 0, 0};        // the autotuner's pick of tile_patches
    int engine_key[3][3] = {};
    double engine_us[3][2] = {};
    struct Trial { int engine, tail, fused, tile; double us; };
    std::vector<Trial> tuning[3];          // the autotuner's measurements, per precision
    double prof_bytes = 0.0;
    // multi-vector V-cycles: columns the level buffers hold (0: none yet), and a
    // graph per (precision, K = 4 / 8) keyed by nu1, nu2, weighting and omega
    int many_k = 0;
    int many_gen = 0;
    cudaGraphExec_t mgraph[3][2] = {};
    int mgraph_key[3][2][4] = {};
    double mgraph_omega[3][2] = {};
    int64_t mgraph_nodes[3][2] = {};
    std::vector<Hierarchy*> many_ws;     // workspaces of columns 1.. of multi-vector solves (share the operator)
    std::vector<void*> allocs;
};

// Error flags (device int array)
// FLAG_ABORT: the persistent V-cycle gave up a bounded wait; FLAG_MANY: the
// multi-vector apply did.
enum Flag {
    FLAG_BAD_PATTERN = 0, FLAG_NONFINITE = 1, FLAG_SINGULAR = 2, FLAG_ABORT = 3, FLAG_MANY = 4, FLAG_COUNT = 5
};

// Persistent V-cycle (persistent.cu) on the finest level's buffers of precision prec.
struct Hierarchy;
cudaError_t launch_vcycle_persistent(Hierarchy* h, int prec, int nu1, int nu2, double omega, int weighting,
                                     unsigned* bar, int* abort, int small_patches);
// Levels 0..top of a V-cycle as one thread-block-cluster launch with the
// levels resident in shared memory (cluster.cu); false if no cluster can hold
// them.  resident_tail_top: the largest top <= want that fits (-1: none).
bool launch_vcycle_tail(Hierarchy* h, int prec, int top, int nu1, int nu2, double omega, int weighting,
                        const void* b_top, void* x_top);
int resident_tail_top(const Hierarchy* h, int prec, int want);

// ---------------------------------------------------------------------------
// Launchers (setup_kernels.cu)
// ---------------------------------------------------------------------------
void launch_bsr_to_stencil(const Geom& g, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* vals, int64_t nnzb, double* A64, int* flags, cudaStream_t s);
void launch_convert_f64_f32(const double* in, float* out, int64_t n, cudaStream_t s);
cudaError_t launch_patch_invert(const Geom& g, const double* A64, double* inv64, int64_t s64,
                                float* inv32, int64_t s32, __nv_bfloat16* invbf, int64_t sbf,
                                int* flags, cudaStream_t s, int64_t npatch = -1, const int32_t* ids = nullptr);
// Large patches (4^d cells) listed by org (their lowest 2^d-cell block on the regular patch grid).
cudaError_t launch_patch_invert_large(const Geom& g, const double* A64, const int32_t* org, int64_t npatch,
                                      double* inv64, int64_t s64, float* inv32, int64_t s32, __nv_bfloat16* invbf,
                                      int64_t sbf, int* flags, cudaStream_t s);
void launch_coarse_assemble(const Geom& g, const double* A64, double* dense, cudaStream_t s);
void launch_dense_invert(double* a, int64_t n, int* perm, int* flags, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (smooth_kernels.cu); T = double or float
// ---------------------------------------------------------------------------
template <typename T>
void launch_spmv(const Geom& g, const T* A, const T* x, const T* b, T* y, bool residual,
                 cudaStream_t s);
// npatch >= 0 with ids: the listed patches only (ids[k] = the patch's index on
// the level's regular patch grid; inverse k and correction k stored in list order).
template <typename T, typename TS>
void launch_vanka_apply(const Geom& g, const TS* inv, int64_t stride, const T* d, T* corr,
                        cudaStream_t s, int64_t npatch = -1, const int32_t* ids = nullptr);
template <typename T>
void launch_vanka_update(const Geom& g, const T* corr, T* x, bool x_zero, T omega, bool average,
                         cudaStream_t s);
template <typename T>
void launch_vanka_update2(const Geom& g, const T* corr, const T* x_in, T* x_out, bool x_zero, T omega, bool average,
                          cudaStream_t s);
// fused forms of the V-cycle (same element code as the separate kernels)
template <typename T>
void launch_update_residual(const Geom& g, const T* A, const T* corr, const T* x_in, bool x_zero, T omega,
                            bool average, const T* b, T* x_out, T* r, cudaStream_t s);
template <typename T>
void launch_prolong_residual(const Geom& f, const Geom& c, const T* A, const T* ec, const T* x_in,
                             const uint8_t* fmask, const T* b, T* x_out, T* r, cudaStream_t s);
template <typename T>
void launch_restrict(const Geom& fine, const Geom& coarse, const T* rf, T* rc,
                     const uint8_t* cmask, cudaStream_t s);
template <typename T>
void launch_prolong_add(const Geom& fine, const Geom& coarse, const T* ec, T* xf,
                        const uint8_t* fmask, cudaStream_t s);
template <typename T>
void launch_coarse_gemv(const double* inv, int64_t n, const T* b, T* x, cudaStream_t s);
template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Multi-vector V-cycle launchers (multi_kernels.cu): K = 4 or 8 interleaved
// FP32 columns; per column the arithmetic of the single-vector launchers.
// ---------------------------------------------------------------------------
constexpr int kMaxCols = 8;
struct ColPtrs { const float* p[kMaxCols]; };
struct ColPtrsOut { float* p[kMaxCols]; };
template <int K>
void launch_spmv_many(const Geom& g, const float* A, const float* x, const float* b, float* y, bool residual,
                      cudaStream_t s);
// false (nothing launched) if the inverses are not in the unpadded 16-byte
// aligned column layout the bulk copies need
template <int K, typename TS>
bool launch_vanka_apply_many(const Geom& g, const TS* inv, int64_t stride, const float* d, float* corr, int* flag,
                             cudaStream_t s);
template <int K>
void launch_vanka_update_many(const Geom& g, const float* corr, const float* x_in, float* x_out, bool x_zero,
                              float omega, bool average, cudaStream_t s);
template <int K>
void launch_restrict_many(const Geom& f, const Geom& c, const float* rf, float* rc, const uint8_t* cmask,
                          cudaStream_t s);
template <int K>
void launch_prolong_add_many(const Geom& f, const Geom& c, const float* ec, float* xf, const uint8_t* fmask,
                             cudaStream_t s);
template <int K>
void launch_coarse_gemv_many(const double* inv, int64_t n, const float* b, float* x, cudaStream_t s);
template <int K>
void launch_pack(const ColPtrs& src, int ncols, int64_t n, float* out, cudaStream_t s);
template <int K>
void launch_unpack(const float* in, const ColPtrsOut& dst, int ncols, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tile-fused smoothing steps (tile_kernels.cu): one CTA per tile of patches
// recomputes the previous update on its node region, the defect on its patch
// nodes, and then solves its patches (or restricts the residual).
// ---------------------------------------------------------------------------
enum TileMode {
    TILE_FIRST = 0,          // x = 0: d = b; corr_out = patch solves
    TILE_STEP = 1,           // x = x_in + w corr_in (x_out, owned nodes); d = b - A x; corr_out
    TILE_PROLONG_STEP = 2,   // x = x_in + P ec (x_out, owned nodes); d = b - A x; corr_out
    TILE_RESTRICT = 3,       // x = x_in + w corr_in (x_out, owned nodes); rc = P^T (b - A x)
    TILE_FINAL = 4           // x_out = x_in + w corr_in on every node
};
template <typename T, typename TS>
void launch_tile_step(const Geom& g, const Geom& gc, int mode, const T* A, const TS* inv, int64_t inv_stride,
                      const T* b, const T* x_in, bool x_zero, const T* corr_in, const T* ec, const uint8_t* fmask,
                      const uint8_t* cmask, T* x_out, T* corr_out, T* rc, T omega, bool average, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (krylov_kernels.cu): FP64 outer FGMRES
// ---------------------------------------------------------------------------
// scal layout (doubles):
enum Scal {
    S_BNORM = 0, S_BETA = 1, S_EST = 2, S_INVH = 3, S_STATUS = 4, S_ITER = 5,
    S_H = 8,                                   // (m+1) x m Hessenberg, column-major, ld m+1
    S_CS = S_H + (kMaxRestart + 1) * kMaxRestart,
    S_SN = S_CS + kMaxRestart,
    S_G = S_SN + kMaxRestart,
    S_Y = S_G + kMaxRestart + 1,
    S_HC = S_Y + kMaxRestart,                  // current column h_{0..j}
    S_COUNT = S_HC + kMaxRestart + 2
};
void launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t s);
// Kernels of one FGMRES step.  The step index j of the current restart cycle
// lives on the device (cyc[0]; cyc[1] = iterations so far, cyc[2] = 1 once the
// cycle has stopped), so the same launches serve every step and can be
// replayed by a graph loop.
void launch_start_cycle(double* scal, int m, int* cyc, cudaStream_t s);
void launch_solve_update(double* scal, int k, int m, const double* Z, int64_t ldz, double* x,
                         int64_t n, cudaStream_t s);
// Step j = cyc[0]: Z_j = widened xf, w = A Z_j (FP64) and out = V_{0..j}^T w.
template <typename TX>
void launch_spmv_zstore_dots(const Geom& g, const double* A, const TX* xf, double* Z, double* w, const double* V,
                             int64_t ldv, const int* cyc, double* partial, double* out, unsigned* counter,
                             cudaStream_t s);
// w -= V scal[S_HC..]; scal[S_Y..] = V^T w; h_{j+1,j} and its reciprocal.
void launch_gs_update_dot_norm(const double* V, int64_t ldv, const int* cyc, double* w, int64_t n, double* partial,
                               double* scal, int m, unsigned* counter, cudaStream_t s);
// V_{j+1} = (w - V scal[S_Y..]) * scal[S_INVH], also converted into vin; the
// Givens update of column j of the Hessenberg matrix (restart length m).
template <typename TV>
void launch_gs_update_scale(double* V, int64_t ldv, const int* cyc, double* scal, const double* w, TV* vin,
                            int64_t n, int m, cudaStream_t s);
template <typename TV>
void launch_scale_convert(const double* x, const double* scal_ptr, double* V, int64_t ldv, const int* cyc, bool next,
                          TV* vin, int64_t n, cudaStream_t s);
void launch_decide(const double* scal, int* cyc, double rtol, int maxit, int m, cudaGraphConditionalHandle loop,
                   bool in_loop, cudaStream_t s);

}  // namespace nmg

namespace nmg {
// Kernels enqueued by the calling thread (launchers add to it; a graph replay
// adds the number of kernel nodes it holds).
extern thread_local int64_t g_launches;

// ---------------------------------------------------------------------------
// Launchers (coupling.cu): problems (2) and (3) of Section 4.2, FP64
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Launchers (mixed_kernels.cu): patches of two sizes
// ---------------------------------------------------------------------------
template <typename T, typename TS>
void launch_vanka_apply_large(const Geom& g, const TS* inv, int64_t stride, const int32_t* org, int64_t npatch,
                              const T* d, T* corr, cudaStream_t s);
template <typename T>
void launch_vanka_update_mixed(const Geom& g, const T* corr_s, const T* corr_l, int64_t nsm, const int32_t* inc,
                               const uint8_t* inc_n, const T* x_in, T* x_out, bool x_zero, T omega, bool average,
                               cudaStream_t s);

void launch_deformation_update(int dim, int64_t nodes, const double* r, const double* dv, double k_theta,
                               const uint8_t* update_nodes, double* du, cudaStream_t s);
void launch_extension_rhs(const Geom& g, const double* E, const uint8_t* fixed, const double* b5, const double* gv,
                          double* rhs, cudaStream_t s);
// Set while a graph body is captured whose kernels must not carry programmatic
// (PDL) launch edges.
extern thread_local bool g_no_pdl;

// Programmatic dependent launch: every solve-phase kernel is launched with
// programmatic stream serialisation, so its launch overlaps the drain of the
// kernel before it.  A kernel waits for its predecessor's results with
// NMG_PDL_WAIT() before touching memory and then lets its own successor launch.
#define NMG_PDL_ENTRY()                                      \
    do {                                                     \
        asm volatile("griddepcontrol.wait;" ::: "memory");   \
        asm volatile("griddepcontrol.launch_dependents;");   \
    } while (0)

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_no_pdl ? 0 : 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Device flag raised by a bounded wait that ran out (a TMA copy that did not
// complete); read and cleared by the host after a solve.
cudaError_t wait_timeout_flag(int* value, cudaStream_t s);
// Stream-ordered variants: enqueue a copy of the flag to (pinned) dst; clear it.
cudaError_t wait_timeout_enqueue_read(int* dst, cudaStream_t s);
cudaError_t wait_timeout_clear(cudaStream_t s);
}  // namespace nmg
