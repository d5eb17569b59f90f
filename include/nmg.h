/*
 * nmg.h -- C ABI of libnmg, a GB300 (sm_103a) solver for the condensed momentum
 * system of a monolithic Newton-multigrid fluid-structure solver
 * (Failer & Richter, "A parallel Newton multigrid framework for monolithic
 * fluid-structure interactions", arXiv:1904.02401).
 *
 * The linear problem is problem (1) of Section 4.2 (Eq. (problem:1)): velocity
 * and pressure on the joint fluid/solid mesh after the solid deformation has
 * been eliminated through the discrete relation d_t u = v (Eq. (defgrad)) and
 * all ALE derivatives have been dropped (Eq. (REDUCEDMATRIX)).  It is solved as
 * in Section 4.3: (I) an outer GMRES iteration, (II) preconditioned by one
 * geometric multigrid V-cycle on nested meshes, (III) smoothed by the additive
 * Vanka patch iteration of Eq. (vanka) with exactly inverted patch matrices.
 *
 * Conventions used by every call below.
 *  - Meshes are uniform Cartesian Q1 meshes with n[k] cells per direction on
 *    the finest level and half as many on each coarser level.  Nodes are
 *    numbered lexicographically, x fastest.
 *  - Vectors are node-blocked (Section 4.3): unknown (node, c) sits at index
 *    node * ncomp + c, ncomp = dim + 1, component order (v_x, v_y[, v_z], p).
 *  - Matrices are block-sparse rows (BSR) over nodes with ncomp x ncomp blocks
 *    stored row-major (Section 4.3, "local blocks of size n_c x n_c"); every
 *    block column must be a Q1 neighbour of its row (offsets in {-1,0,1}^dim).
 *  - Levels are numbered 0 (coarsest) .. levels-1 (finest).
 *  - All device work is ordered on the stream given in nmg_mesh_desc.  Calls
 *    that return results to the host synchronise that stream before returning.
 *  - Pointers named "device" must be device (or managed) memory; pointers
 *    named "host or device" may be either, the library detects which.  The
 *    caller owns every pointer it passes; the library copies what it keeps.
 *  - Every call returns an nmg_status.  No C++ exception crosses the ABI.  On
 *    error, nmg_last_error() returns a message for the calling thread.
 */
#ifndef NMG_H
#define NMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int nmg_status;

#define NMG_OK                  0
#define NMG_PENDING             1   /* nmg_poll: the request is still running          */
#define NMG_ERR_INVALID        -1   /* bad argument, size, pattern or call order        */
#define NMG_ERR_OOM            -2   /* device allocation failed or memory budget refused */
#define NMG_ERR_SINGULAR_PATCH -3   /* a Vanka patch matrix (or the coarse matrix) had a zero pivot */
#define NMG_ERR_NOT_CONVERGED  -4   /* maxit reached before rtol                        */
#define NMG_ERR_NONFINITE      -5   /* NaN or Inf met in the input or in a reduction    */
#define NMG_ERR_TIMEOUT        -6   /* nmg_poll deadline passed                         */
#define NMG_ERR_CUDA           -7   /* a CUDA runtime call failed                       */

/* Arithmetic of the multigrid preconditioner (the outer FGMRES is always FP64). */
#define NMG_PREC_FP64 0   /* matrices, patch inverses and V-cycle vectors in FP64        */
#define NMG_PREC_FP32 1   /* FP32 matrices, patch inverses and V-cycle vectors           */
#define NMG_PREC_BF16 2   /* BF16 patch inverses, FP32 matrices and vectors, FP32 sums   */

/* How overlapping Vanka patch corrections are combined (Eq. (vanka)). */
#define NMG_WEIGHT_AVERAGE 0  /* each unknown's summed correction divided by its patch count */
#define NMG_WEIGHT_SUM     1  /* the plain sum as printed in Eq. (vanka)                     */

typedef struct nmg_hierarchy nmg_hierarchy;
typedef struct nmg_server nmg_server;

typedef struct {
    int dim;                        /* 2 or 3                                                      */
    int n[3];                       /* finest-level cells per direction; n[2] ignored when dim==2 */
    int levels;                     /* multigrid levels >= 1; n[k] divisible by 2^(levels-1) and,
                                       above the coarsest level, even (patches of 2^dim cells)    */
    int ncomp;                      /* unknowns per node: dim + 1 for the condensed momentum system
                                       (velocity, pressure; problem (1) of Section 4.2), or dim for
                                       a vector problem such as the ALE extension (problem (3)); the
                                       latter runs the KERNELS engine only                        */
    int patch_cells;                /* cells per patch direction; only 2 is supported              */
    const uint8_t* dirichlet_mask;  /* host, one byte per finest-level unknown, 1 = Dirichlet;
                                       coarse-level masks are taken by injection (node I <- 2I)   */
    int precisions;                 /* bit mask (1 << NMG_PREC_*) of V-cycle precisions to prepare;
                                       0 means FP64 | FP32 | BF16                                  */
    size_t mem_budget_bytes;        /* 0 = unlimited; otherwise creation and set_jacobian fail with
                                       NMG_ERR_OOM once the hierarchy would exceed it             */
    void* stream;                   /* cudaStream_t used for all work on this hierarchy (NULL =
                                       the legacy default stream); owned by the caller             */
} nmg_mesh_desc;

typedef struct {
    double rtol;      /* stop when ||b - A x||_2 <= rtol ||b||_2 (true residual, FP64)            */
    int restart;      /* FGMRES restart length m, 1..64                                           */
    int maxit;        /* maximum total FGMRES iterations (preconditioner applications)            */
    int nu1, nu2;     /* Vanka pre- and post-smoothing steps per level                            */
    double omega;     /* Vanka damping omega_V (Section 4.3: about 0.8)                           */
    int precision;    /* NMG_PREC_* of the V-cycle; must be among the prepared precisions          */
    int weighting;    /* NMG_WEIGHT_*                                                             */
    int use_graph;    /* 0: plain launches, the host decides after every FGMRES step;
                         1: the V-cycle replayed as a captured CUDA graph, host-stepped;
                         2: as 1, and the steps of each restart cycle run as one graph with an
                            on-device loop (one host round trip per cycle); falls back to 1 where
                            the driver cannot build it or the engine is PERSISTENT            */
    int engine;       /* NMG_ENGINE_*: how a V-cycle is executed                                  */
    int tail_patches; /* engines KERNELS and FUSED: the coarse level and every level with at most
                         this many patches run as one thread-block-cluster kernel (0 = none);
                         AUTO picks it itself, PERSISTENT ignores it                              */
    int tile_patches; /* engine KERNELS: every level above the cluster tail with at most this many
                         patches runs each Vanka step as one tile-fused kernel (a CTA per tile of
                         patches recomputes the previous update and the defect on its halo, then
                         solves its patches; 0 = none); AUTO picks it itself, the other engines
                         ignore it.  Results are bitwise those of the one-kernel-per-pass path     */
} nmg_solve_opts;

/* V-cycle execution engines (same arithmetic, same results). */
#define NMG_ENGINE_AUTO       0  /* time the engines (and the tail threshold) on this hierarchy at first
                                    use and keep the fastest (nmg_autotune_report shows the trials)   */
#define NMG_ENGINE_KERNELS    1  /* one kernel per step (optionally replayed as a CUDA graph)         */
#define NMG_ENGINE_PERSISTENT 2  /* one cooperative persistent kernel per V-cycle                     */
#define NMG_ENGINE_FUSED      3  /* per-step kernels, each Vanka update and each prolongation fused
                                    into the residual that follows it (fewer, heavier kernels)        */

typedef struct {
    int iterations;       /* total FGMRES iterations                                      */
    int restarts;         /* completed restart cycles beyond the first                    */
    double rel_residual;  /* final true ||b - A x||_2 / ||b||_2, computed in FP64          */
    double ms_total;      /* wall time of the call, milliseconds                           */
    nmg_status status;    /* status of the solve (also the return value)                  */
    int64_t launches;     /* CUDA kernels this solve launched (graph nodes counted each replay) */
    int engine;           /* NMG_ENGINE_KERNELS, _PERSISTENT or _FUSED, the engine used       */
    int device_loop;      /* 1 when restart cycles ran as graph loops on the device          */
} nmg_solve_info;

/* Fills *opts with rtol 1e-8, restart 30, maxit 1000, nu1 = nu2 = 2, omega 0.8,
 * precision FP32, weighting AVERAGE, use_graph 2, engine AUTO, tail_patches 0, tile_patches 0. */
nmg_status nmg_default_opts(nmg_solve_opts* opts);

/* Creates an empty hierarchy for the mesh in *desc (Section 4.3 (II): nested
 * uniform meshes, one matrix per level).  *out receives an opaque handle owned
 * by the library until nmg_destroy_hierarchy.  NMG_ERR_INVALID on a bad
 * description, NMG_ERR_OOM if the vectors do not fit the budget. */
nmg_status nmg_create_hierarchy(const nmg_mesh_desc* desc, nmg_hierarchy** out);

/* Sets the matrix of one level (Section 4.3: block matrix A with n_c x n_c
 * blocks; Section 5.5.2: a matrix is assembled on every level).  row_ptr has
 * nrows_blk + 1 entries (nrows_blk = nodes of that level), col_idx and vals
 * have nnzb blocks, vals row-major ncomp x ncomp per block, FP64.  ptr_location
 * 0 = the three arrays are host memory, 1 = device memory.  The library copies
 * and converts them; the caller keeps ownership.  On a level above the
 * coarsest this also extracts every patch matrix A_i = R_i A R_i^T and inverts
 * it exactly (LU-equivalent Gauss-Jordan with partial pivoting, FP64), all
 * patches of the level in one launch; on level 0 it inverts the coarse matrix.
 * NMG_ERR_INVALID for a wrong size, a column outside the Q1 stencil or a
 * duplicate block; NMG_ERR_NONFINITE for NaN/Inf values;
 * NMG_ERR_SINGULAR_PATCH for a zero pivot. */
nmg_status nmg_set_jacobian(nmg_hierarchy* h, int level, int64_t nrows_blk, int64_t nnzb,
                            const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                            int ptr_location);

/* Solves A x = b on the finest level with FGMRES(restart) right-preconditioned by
 * one V(nu1, nu2)-cycle per iteration (Section 4.3 (I)-(III)).  b and x are
 * FP64 vectors of ncomp * nodes entries, host or device; x need not be
 * initialised (the initial guess is 0) and is overwritten.  Returns after the
 * solve has completed.  info may be NULL.  NMG_ERR_NOT_CONVERGED if maxit was
 * reached (x then holds the last iterate); NMG_ERR_NONFINITE if a norm became
 * NaN/Inf; NMG_ERR_INVALID if a level matrix is missing. */
nmg_status nmg_solve(nmg_hierarchy* h, const double* b, double* x, const nmg_solve_opts* opts,
                     nmg_solve_info* info);

/* Solves A x_k = b_k for k = 0..nrhs-1 against the same hierarchy (many
 * right-hand sides per factorisation: the smoother is applied many hundred
 * times per Jacobian, Section 5).  b and x hold nrhs FP64 vectors of
 * ncomp * nodes entries, column k at offset k * ncomp * nodes, host or device.
 * The columns run FGMRES in lockstep in groups of up to 8: every V-cycle
 * serves all columns of the group that need one, reading each level matrix
 * and each patch inverse once for all of them.  opts->precision must be
 * NMG_PREC_FP32 or NMG_PREC_BF16 (the V-cycle's vectors are FP32); engine,
 * tail and tile settings do not apply; use_graph != 0 replays the
 * multi-vector V-cycle from a CUDA graph.  Each column's solution, iteration
 * count and status equal those of nmg_solve on that column alone, bit for
 * bit.  info: NULL or an array of nrhs records.  The columns after the first
 * run on workspaces the hierarchy allocates on first need and keeps (vectors,
 * Krylov bases and device scalars, sharing the operator), counted by
 * nmg_hierarchy_bytes.  Returns the first failing column's status, else
 * NMG_OK; NMG_ERR_INVALID for nrhs < 1 or precision FP64. */
nmg_status nmg_solve_many(nmg_hierarchy* h, int nrhs, const double* b, double* x, const nmg_solve_opts* opts,
                          nmg_solve_info* info);

/* ---- serving: many solves of problem (1), one per Newton step of different
 * simulations (Section 4.2, Eq. (newton): every Newton step solves one linear
 * problem), batched continuously on resident hierarchies.
 *
 * nmg_server_create starts a server with a memory budget (bytes of resident
 * hierarchies whose requests may run at once; 0 = unlimited) and at most
 * max_slots requests in flight.  nmg_submit queues a solve of A x = b on
 * hierarchy h and returns a ticket at once; b and x (FP64, host or device, b
 * ready when submitted) must stay valid until the request completes.  A
 * request starts when a slot is free, its hierarchy runs no other request (or
 * has an idle extra workspace, see nmg_server_set_workspaces) and the budget
 * allows; running requests advance concurrently on their own streams, so
 * requests that arrive while others run join them.
 * Results equal those of nmg_solve.  nmg_poll returns NMG_PENDING at once
 * (timeout_ms <= 0) or waits up to timeout_ms and then returns NMG_ERR_TIMEOUT;
 * once a request is done it returns the solve's status, fills *info (ms_total
 * = submit-to-completion latency) and releases the ticket.  Do not call
 * nmg_solve on a hierarchy while the server may run a request on it.
 * NMG_ERR_OOM from nmg_submit if h alone exceeds the budget. */
nmg_status nmg_server_create(size_t mem_budget_bytes, int max_slots, nmg_server** out);
/* Lets up to extra_per_hierarchy further requests on the same hierarchy run at
 * once (default 0).  Each one runs on a workspace the server allocates on first
 * need and keeps until it stops: the hierarchy's vectors, Krylov bases, device
 * scalars and stream, sharing its matrices, masks and patch inverses.  Results
 * are the same as on the hierarchy itself.  The budget counts each such
 * workspace; one is made only when the budget holds it.  NMG_ERR_INVALID for a
 * count outside 0..1024. */
nmg_status nmg_server_set_workspaces(nmg_server* s, int extra_per_hierarchy);
/* Serves requests on the same hierarchy as the columns of one multi-vector
 * solve (see nmg_solve_many): with max_columns > 1, a request whose precision
 * is NMG_PREC_FP32 or NMG_PREC_BF16 joins its hierarchy's column group when a
 * column is free and its V-cycle options (precision, nu1, nu2, omega,
 * weighting) equal the group's, at any point of the others' iterations; every
 * V-cycle then serves all columns that need one.  Columns finish
 * independently.  Results equal nmg_solve's bit for bit.  FP64 requests run
 * alone on their hierarchy when no group runs on it.  The column workspaces
 * are the hierarchy's own (nmg_solve_many's) and are counted by the budget
 * while columns run.  Do not call nmg_solve_many on a hierarchy while the
 * server may run requests on it.  0 or 1 turns batching off (the default);
 * NMG_ERR_INVALID outside 0..8. */
nmg_status nmg_server_set_batching(nmg_server* s, int max_columns);
nmg_status nmg_submit(nmg_server* s, nmg_hierarchy* h, const double* b, double* x,
                      const nmg_solve_opts* opts, uint64_t* ticket);
nmg_status nmg_poll(nmg_server* s, uint64_t ticket, int timeout_ms, nmg_solve_info* info);
/* Device memory held for the server's running requests, in bytes: the
 * hierarchies with a running request (each once), the server's workspace
 * clones and the column workspaces of groups with running columns.  This is
 * the quantity the memory budget bounds.  *resident_bytes: the value after the
 * worker's last round; *peak_bytes: the largest value since the server was
 * created.  Either pointer may be NULL.  NMG_ERR_INVALID for a NULL server. */
nmg_status nmg_server_memory(nmg_server* s, size_t* resident_bytes, size_t* peak_bytes);
/* Finishes every queued and running request, then stops the server. */
nmg_status nmg_server_destroy(nmg_server* s);

/* ---- problems (2) and (3) of Section 4.2 around the momentum solve.
 *
 * With the ALE derivatives dropped (Eq. (REDUCEDMATRIX)) a Newton step splits
 * into problem (1), the momentum system this library solves on a hierarchy
 * with ncomp = dim + 1; problem (2), the Newton step of the zero-order relation
 * u_n = u_{n-1} + k (1 - theta) v_{n-1} + k theta v_n on the interface and in
 * the solid, whose both sides carry the same mass matrix, so that it is one
 * vector addition du = r + k theta dv (velocity components; r the relation's
 * residual in nodal form); and problem (3), the extension of the deformation
 * into the fluid, E_ff du_f = b_5 - E_fi du_i (Eq. (problem:3)), solved on a
 * hierarchy with ncomp = dim whose Dirichlet mask marks the fixed unknowns
 * (every node of a solid cell and the outer boundary).  Vectors hold dim
 * components per node (node-blocked) unless stated otherwise. */

/* Sets the operator of problem (3) on the finest level of an extension
 * hierarchy (ncomp = dim) as assembled, before its fixed rows and columns are
 * reduced to the identity: its free rows carry the coupling E_fi that lifts
 * the deformation of the fixed nodes into the right-hand side.  BSR arguments
 * as in nmg_set_jacobian (the finest level's node count, dim x dim blocks,
 * FP64, host or device per ptr_location); the library keeps an FP64 copy.
 * NMG_ERR_INVALID for a hierarchy with ncomp != dim or a bad pattern. */
nmg_status nmg_set_lifting_operator(nmg_hierarchy* h, int64_t nrows_blk, int64_t nnzb, const int64_t* row_ptr,
                                    const int32_t* col_idx, const double* vals, int ptr_location);

/* Problem (2) on the finest mesh of the extension hierarchy h: du_i = r_i +
 * k_theta (dv_i)_{0..dim-1} on every node i with update_nodes[i] != 0 (the
 * nodes of solid cells off the outer boundary: interface and solid interior),
 * du_i = 0 elsewhere.  r, du: device FP64, dim per node; dv: device FP64, the
 * dim + 1 unknowns per node of problem (1) (velocity, then pressure);
 * update_nodes: device, one byte per node.  Returns after completion. */
nmg_status nmg_deformation_update(nmg_hierarchy* h, const double* r, const double* dv, double k_theta,
                                  const uint8_t* update_nodes, double* du);

/* Right-hand side of problem (3) with its fixed rows reduced to the identity:
 * rhs = g on the fixed unknowns (h's Dirichlet mask), rhs = b5 - E g_hat on
 * the free ones, g_hat = g on the fixed unknowns and 0 elsewhere, E the
 * operator of nmg_set_lifting_operator.  Device FP64 vectors of dim per node.
 * Returns after completion; NMG_ERR_INVALID if no lifting operator is set. */
nmg_status nmg_extension_rhs(nmg_hierarchy* h, const double* b5, const double* g, double* rhs);

/* One linearised Newton step of Section 4.2, the three sub-steps in order on
 * the same finest mesh: dw = (dv, dp) from problem (1) on h1 (nmg_solve with
 * opts1, right-hand side b1, dim + 1 per node); du on the flagged nodes from
 * problem (2) (r, k_theta, update_nodes as in nmg_deformation_update); then
 * du on the free nodes from problem (3) on h3 (nmg_solve with opts3 of the
 * system whose right-hand side nmg_extension_rhs builds from b5 and that
 * deformation).  b1, r, b5, update_nodes, dw, du: host or device.  The
 * sub-steps after the momentum solve run on h3's stream once that solve has
 * completed; the call returns when the extension solve has.  info1, info3:
 * NULL or the two solves' records.  Returns the first failing solve's status
 * (problem (3) does not run when problem (1) fails); NMG_ERR_INVALID for
 * hierarchies of other kinds or meshes or a missing lifting operator. */
nmg_status nmg_newton_substeps(nmg_hierarchy* h1, nmg_hierarchy* h3, const double* b1, const double* r, double k_theta,
                               const uint8_t* update_nodes, const double* b5, double* dw, double* du,
                               const nmg_solve_opts* opts1, const nmg_solve_opts* opts3, nmg_solve_info* info1,
                               nmg_solve_info* info3);

/* ---- Jacobian reuse in the Newton loop (Section 5.3): the Jacobian of
 * problem (1) is assembled again (and every level set with nmg_set_jacobian,
 * which refactors the patches) only when the nonlinear convergence rate
 * rho_l = ||B - A(U^(l))||_inf / ||B - A(U^(l-1))||_inf exceeds gamma_nt.
 * Host-only bookkeeping; no device work.  Readings: with no Jacobian yet one
 * is assembled; the first Newton step of a time step has no rate and reuses
 * the Jacobian unless gamma_nt = 0 (gamma_nt = 0 assembles in every Newton
 * step, as the paper states). */
typedef struct {
    double gamma;         /* the threshold gamma_nt >= 0                                  */
    double last;          /* residual norm of the previous Newton step of this time step   */
    double rate;          /* rho of the last decision; -1 when it had none                 */
    int have_last;        /* a previous Newton step of this time step exists               */
    int have_jacobian;    /* a Jacobian has been assembled                                 */
    int64_t steps;        /* decisions taken                                               */
    int64_t assemblies;   /* decisions that asked for a new Jacobian                       */
} nmg_jacobian_reuse;

/* Clears *m and sets gamma_nt; NMG_ERR_INVALID for a negative or non-finite gamma. */
nmg_status nmg_jacobian_reuse_init(nmg_jacobian_reuse* m, double gamma);
/* Starts a new time step (its first Newton step has no rate). */
nmg_status nmg_jacobian_reuse_time_step(nmg_jacobian_reuse* m);
/* Decides for the Newton step whose current nonlinear residual norm (max
 * norm) is residual_inf: *assemble = 1 when the Jacobian must be assembled and
 * set before this step's linear solves, 0 when the last one is reused.
 * NMG_ERR_NONFINITE for a negative or non-finite norm. */
nmg_status nmg_jacobian_reuse_decide(nmg_jacobian_reuse* m, double residual_inf, int* assemble);

/* ---- operator-level calls (one step of the method each; vectors are device
 * arrays of the precision's arithmetic type: double for NMG_PREC_FP64, float
 * for NMG_PREC_FP32 and NMG_PREC_BF16; sizes are ncomp * nodes of the level) */

/* y = A_level x (Section 4.3 block matrix-vector product). */
nmg_status nmg_matvec(nmg_hierarchy* h, int level, int precision, const void* x, void* y);

/* r = b - A_level x. */
nmg_status nmg_residual(nmg_hierarchy* h, int level, int precision, const void* b, const void* x,
                        void* r);

/* steps iterations of Eq. (vanka) on A_level x = b, in place on x (level >= 1).
 * x_is_zero = 1 treats x as zero on entry (its contents are ignored). */
nmg_status nmg_smooth(nmg_hierarchy* h, int level, int precision, const void* b, void* x, int steps,
                      int x_is_zero, double omega, int weighting);

/* r_coarse = P^T r_fine from level to level-1, Dirichlet entries of level-1 set to 0
 * (Q1 full weighting, the transpose of nodal interpolation). */
nmg_status nmg_restrict(nmg_hierarchy* h, int level, int precision, const void* r_fine,
                        void* r_coarse);

/* x_fine += P e_coarse from level-1 to level, Dirichlet entries of level left unchanged. */
nmg_status nmg_prolongate_add(nmg_hierarchy* h, int level, int precision, const void* e_coarse,
                              void* x_fine);

/* x = A_0^{-1} b on the coarsest level (dense inverse computed in FP64 at set-up). */
nmg_status nmg_coarse_solve(nmg_hierarchy* h, int precision, const void* b, void* x);

/* z = one V(nu1, nu2)-cycle applied to r on the finest level, zero initial guess
 * on every level (Section 4.3 (II)). */
nmg_status nmg_vcycle(nmg_hierarchy* h, const nmg_solve_opts* opts, const void* r, void* z);

/* z_k = one V(nu1, nu2)-cycle applied to r_k, k = 0..nrhs-1 (float vectors of
 * ncomp * nodes entries, column k at offset k * ncomp * nodes, device memory),
 * in groups of up to 8 columns that share every read of the level matrices
 * and patch inverses.  Precision NMG_PREC_FP32 or NMG_PREC_BF16; engine, tail
 * and tile settings do not apply (use_graph != 0: graph replay).  Each
 * column equals nmg_vcycle on that column bit for bit.  NMG_ERR_INVALID for
 * nrhs < 1 or precision FP64. */
nmg_status nmg_vcycle_many(nmg_hierarchy* h, const nmg_solve_opts* opts, int nrhs, const void* r, void* z);

/* Vanka patches of two sizes (Section 5.5.1): over the cells flagged in
 * cell_mask (host, one byte per finest-level cell, x fastest; non-zero =
 * flagged) the smoother uses large patches, blocks of 4^dim cells (5^dim
 * nodes: 75 unknowns in 2d, 500 in 3d for ncomp = dim + 1), on every
 * 4-aligned block whose cells are all flagged; every other cell keeps the
 * small patch of its 2-aligned block of 2^dim cells.  A coarser cell is
 * flagged when all its children are.  Each unknown's summed correction is
 * weighted by the number of patches of either size containing it (with
 * NMG_WEIGHT_AVERAGE).  cell_mask NULL restores small patches everywhere.
 * Levels already set are factored again in the new layout (large patches by
 * FP64 Gauss-Jordan with partial pivoting: in shared memory in 2d, in a
 * global-memory work matrix per CTA in 3d); levels set later use it.  With
 * large patches the V-cycle runs the KERNELS engine (other engines are
 * refused) and multi-vector calls are refused; call this before
 * nmg_solve_many and before serving the hierarchy.  NMG_ERR_INVALID for a
 * NULL hierarchy or after multi-vector solves; NMG_ERR_SINGULAR_PATCH if a
 * refactored patch has a zero pivot. */
nmg_status nmg_set_large_patches(nmg_hierarchy* h, const uint8_t* cell_mask);

/* The patch layout of level (1..levels-1): *nsmall patches of *np_small
 * unknowns (blocks of 2^dim cells) and *nlarge patches of *np_large unknowns
 * (blocks of 4^dim cells; 0 without nmg_set_large_patches or where no large
 * block fits).  nmg_get_patch_inverses numbers the small patches first (in
 * origin order, x fastest), then the large ones (same order); a range must
 * hold patches of one size.  Any output pointer may be NULL. */
nmg_status nmg_patch_layout(nmg_hierarchy* h, int level, int64_t* nsmall, int64_t* nlarge, int* np_small,
                            int* np_large);

/* Copies count patch inverses of a level, starting at patch first, to host
 * memory out (count * n_p * n_p doubles, row-major A_i^{-1}, converted from the
 * precision's storage type).  Patches are ordered by origin with x fastest
 * (with large patches: see nmg_patch_layout); patch-local unknowns node-major
 * over the 3^dim (large: 5^dim) nodes (x fastest), then component. */
nmg_status nmg_get_patch_inverses(nmg_hierarchy* h, int level, int precision, int64_t first,
                                  int64_t count, double* out);

/* The V-cycle autotuner's choices (engine and cluster-tail threshold per
 * precision), its last trial timings and the state of the on-device FGMRES
 * loop (mode 0 not built yet, 1 built with programmatic launch edges, 2 built
 * without them, -1 unavailable; kernels per loop step per precision), as a
 * NUL-terminated JSON object in buf (len bytes).  NMG_ERR_INVALID if buf is
 * too small. */
nmg_status nmg_autotune_report(nmg_hierarchy* h, char* buf, size_t len);

/* Bytes of device memory held by the hierarchy. */
nmg_status nmg_hierarchy_bytes(nmg_hierarchy* h, size_t* bytes);

/* Releases every device allocation of the hierarchy; h is invalid afterwards. */
nmg_status nmg_destroy_hierarchy(nmg_hierarchy* h);

/* ---- kernel timing on the hierarchy's stream.  mode 1: every V-cycle of
 * later solves is bracketed by CUDA events; mode 2: every finest-level Vanka
 * apply launch is; mode 3: every finest-level residual product (block SpMV)
 * launch is (modes 2 and 3: plain launches only, use_graph = 0, engine
 * KERNELS); mode 0: off. */
nmg_status nmg_profile_enable(nmg_hierarchy* h, int mode);
/* Total milliseconds and count of the timed V-cycles / launches since enabling,
 * and the algorithmic bytes one of them moves (every patch inverse, matrix and
 * vector it must read or write once). */
nmg_status nmg_profile_read(nmg_hierarchy* h, double* ms_total, int64_t* launches,
                            double* bytes_per_launch);

/* Iteration limit of the grid-barrier wait of the persistent V-cycle engine
 * (NMG_ENGINE_PERSISTENT) on this hierarchy; 0 restores the default (2^24
 * polls, far beyond any barrier of a running V-cycle).  Every device-side wait
 * of the library is bounded: a wait that runs out sets a device flag, the
 * waiting CTAs leave the kernel, and the solve or V-cycle returns
 * NMG_ERR_TIMEOUT with the flag cleared, so the next call runs normally.  A
 * small limit makes that path testable without a fault (a limit of 1 lets
 * every barrier wait run out).  No counterpart in the paper.  NMG_ERR_INVALID
 * for a NULL hierarchy or a negative limit. */
nmg_status nmg_set_wait_limit(nmg_hierarchy* h, int spins);

/* ---- one Vanka correction that allocates no device memory.  The paper has no
 * counterpart: this call exists for callers that cannot let a library call
 * cudaMalloc, such as code that manages all device memory in its own fixed
 * arena, or a hot loop where cudaMalloc (which can synchronise the device and
 * is not stream-ordered) is not allowed.  It needs no hierarchy; the caller
 * passes every input and output:
 *   x <- (x_is_zero ? 0 : x) + omega * W * sum_i R_i^T A_i^{-1} R_i d
 * on a level with cells[0..dim-1] cells (each even), W as in weighting.
 * inv: device patch inverses in the library's layout (patch i at element
 * i * inv_stride, column-major n_p x n_p, n_p = 3^dim (dim+1); storage double,
 * float or bfloat16 for precision FP64, FP32, BF16; inv_stride >= n_p^2).
 * d, x: device vectors of (dim+1) * nodes entries, double for FP64, float
 * otherwise.  Work is enqueued on stream (a cudaStream_t; NULL = the legacy
 * default stream) and the call returns without waiting for it.
 * The per-patch scratch lives in one fixed 16 MiB device array of the library
 * (patches * n_p * sizeof(element) must fit, else NMG_ERR_INVALID), which
 * every GPU that loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race with each other. */
nmg_status nmg_vanka_correct_noalloc(int dim, const int* cells, int precision, const void* inv,
                                     int64_t inv_stride, const void* d, void* x, double omega,
                                     int weighting, int x_is_zero, void* stream);

/* Thread-local description of the last error (never NULL). */
const char* nmg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NMG_H */
