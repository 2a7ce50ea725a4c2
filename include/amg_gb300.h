/*
 * amg_gb300.h -- C ABI of the GB300 (sm_103a) block smoothed-aggregation AMG
 * preconditioned CG solver for 3D elasticity with rigid-body near-nullspace
 * modes.
 *
 * Method: D. E. Demidov, "Efficient solution of 3D elasticity problems with
 * smoothed aggregation algebraic multigrid and block arithmetics" (2022).
 *   - Alg. 1 (Sec. 2): setup.  Per level: prolongation P_i and next
 *     near-nullspace B_{i+1} from (A_i, B_i); R_i = P_i^T; smoother S_i from
 *     A_i; Galerkin operator A_{i+1} = R_i A_i P_i; a direct solver for the
 *     coarsest A_L.
 *   - Alg. 2 (Sec. 2): V-cycle, applied once per preconditioning step.
 *   - Sec. 2/3: every matrix of the hierarchy is held in block CSR (BSR):
 *     3x3 blocks on the finest level, 6x6 below it (six rigid-body modes;
 *     3x3 when B holds only the three translations);
 *     only the tentative prolongation is built from B in scalar terms, and
 *     here it is built per aggregate inside block-structured kernels (the
 *     paper's "NS Block" route, Sec. 3, Listing 2 semantics).
 *   - Sec. 4: conjugate gradients preconditioned by one V-cycle, stopping at
 *     relative residual 1e-8; the block vs scalar comparison (storage of the
 *     solve's operators, and the Galerkin product in either arithmetic) and
 *     the ILU(0) smoother of the paper's experiments.
 *   - Options the paper does not have: reduced or emulated precision in the
 *     V-cycle, aggregation on the device (MIS-2), a learned 3x3 smoother and
 *     a batched solver for many instances and right-hand sides.
 *
 * Conventions for every call:
 *   - Matrix and vector pointers are DEVICE pointers unless a parameter says
 *     "host".  The caller owns them; the library only borrows them for the
 *     duration of the call (it copies what it keeps).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is ordered on that stream.  Calls that return results
 *     through host pointers synchronise the stream before returning.
 *   - DOF layout is node-major: scalar row 3*I + c is component c of node I.
 *   - Every call returns an int status: AMG_OK (0), AMG_NOT_CONVERGED (1,
 *     results written), or a negative error code; nothing aborts or traps.
 *     amg_last_error() gives a message for the calling thread's last error.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMG_OK 0
#define AMG_NOT_CONVERGED 1
#define AMG_ERR_ARG (-1)          /* bad argument (shape, null pointer, block size) */
#define AMG_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define AMG_ERR_BREAKDOWN (-3)    /* CG breakdown: p.Ap <= 0, r.z <= 0 or non-finite */
#define AMG_ERR_COARSE (-4)       /* coarsest matrix not positive definite */
#define AMG_ERR_LIMIT (-5)        /* a size exceeds a fixed internal limit */
#define AMG_ERR_STATE (-6)        /* handle not usable for this call */

#define AMG_PREC_FP64 0           /* V-cycle matrices and vectors in FP64 */
#define AMG_PREC_FP32 1           /* V-cycle in FP32 storage, FP32 accumulation */
#define AMG_PREC_BF16 2           /* V-cycle matrices stored BF16, FP32 accumulation */
#define AMG_PREC_DF64 3           /* V-cycle in FP64 emulated on FP32 pairs: A, P, R stored
                                     as hi + lo floats (the FP64 value truncated to ~48 bits),
                                     products and sums in FP32-pair arithmetic (about 2^-45
                                     relative per product), FP64 vectors; the CG's A p, dots
                                     and true residual stay FP64.  Not in the paper: an
                                     implementation choice for GB300, whose FP64 rate is
                                     1/64 of its FP32 rate */

/* Storage of the solve's operators (amg_params.storage).  Sec. 4 compares
 * the block-valued solver with a scalar one ("NS Scalar"): the same
 * hierarchy, every operator in scalar CSR.  AMG_STORAGE_SCALAR keeps the
 * block setup and stores the V-cycle's A_l, P_l, R_l and the CG's fine A
 * unblocked (one scalar row per DOF, the blocks' explicit zeros kept), so
 * the two storages run the same arithmetic and differ only in layout. */
#define AMG_STORAGE_BLOCK 0       /* b x b blocks (3x3 fine, 6x6 coarse) */
#define AMG_STORAGE_SCALAR 1      /* scalar CSR rows */

/* Arithmetic of the setup (amg_params.setup), the other axis of Sec. 3/4's
 * comparison.  AMG_SETUP_BLOCK is the paper's "NS Block" route: the
 * transfer operators built per aggregate straight into b x 6 blocks, the
 * Galerkin product and the smoother in block arithmetic.  AMG_SETUP_SCALAR
 * is the scalar setup of "NS Scalar" and "NS Hybrid1": the input is
 * unblocked, and strength (on the node graph condensed from the scalar
 * pattern, point-wise with block size 3, then 6), aggregation, tentative
 * prolongation, its smoothing, R = P^T, the Galerkin product and SPAI0 all
 * run on scalar CSR rows; the levels are then converted into blocks
 * (Listing 1's conversion).  With AMG_STORAGE_BLOCK the solve runs on those
 * blocks ("NS Hybrid1"); with AMG_STORAGE_SCALAR on the scalar matrices
 * themselves ("NS Scalar").  Both setups give the same hierarchy (patterns
 * and aggregates bit for bit, values to rounding).  The scalar setup takes
 * the SPAI0 smoother and single-instance handles only. */
#define AMG_SETUP_BLOCK 0
#define AMG_SETUP_SCALAR 1

/* Aggregation (the coarsening step of Alg. 1, point-wise on block rows as in
 * Sec. 4; the paper does not specify the algorithm).  Both run on the strong
 * connections of the level's block matrix and give every aggregated node
 * exactly one aggregate; nodes without strong neighbours stay unaggregated.
 *   AMG_AGG_GREEDY: three sequential passes in ascending node order on the
 *     host (a node whose strong neighbours are all free roots an aggregate;
 *     leftovers join the lowest-index neighbour placed in the first pass;
 *     the rest start new aggregates).
 *   AMG_AGG_MIS2: on the device, aggregates grown around a distance-2
 *     maximal independent set of the strong graph made undirected: the roots
 *     are those of a visit in descending priority fmix32(node index)
 *     (MurmurHash3's 32-bit finaliser), found by synchronous rounds of
 *     two-hop key maxima; a root with its neighbours forms an aggregate
 *     (numbered by ascending root index), every other node joins the
 *     aggregate of its lowest-index neighbour that has one.  The hierarchy
 *     differs from the greedy one (other aggregates), not the method. */
#define AMG_AGG_GREEDY 0
#define AMG_AGG_MIS2 1

/* Level smoother.  AMG_SMOOTH_SPAI0: damped SPAI0 diagonal (the default).
 * AMG_SMOOTH_ILU0: block ILU(0), the relaxation of the paper's experiments
 * (Sec. 4), factored on each level's own block pattern (b x b blocks,
 * explicit zeros kept: L_IK = A_IK U_KK^-1, A_IJ -= L_IK U_KJ for the blocks
 * J > K that row K holds) and applied with `ilu_sweeps` Jacobi sweeps per
 * triangular factor (y <- r - L_s y from y = r; x <- U_D^-1 (y - U_s x)
 * from x = U_D^-1 y), before and after the coarse correction.  FP64 V-cycle
 * and block storage only.  The sweeps make the preconditioner slightly
 * non-symmetric; on matrices where ILU(0) itself is indefinite (stiff
 * inclusions) CG can break down (AMG_ERR_BREAKDOWN).
 * AMG_SMOOTH_BJACOBI: block damped Jacobi, the damped Jacobi relaxation of
 * Sec. 2 over the node blocks of every smoothing level: M_I = (2 smooth_relax
 * / lambda) A_II^-1, lambda the Rayleigh quotient (x, A x) / (x, D_b x) after
 * 20 power iterations of D_b^-1 A (D_b = the block diagonal of A) from a
 * fixed hashed start vector, an estimate from below of lambda_max(D_b^-1 A);
 * with smooth_relax = 0.8 the damped M A peaks near 1.6 on any material
 * (undamped block Jacobi peaks at 2.6-3.9 on Q1 elasticity, nu 0.2-0.45, and
 * a damping above 2 / lambda_max makes the V-cycle indefinite).  A zero row
 * and column of A_II (a near-nullspace column dropped above) stays zero in
 * M_I.  Block storage only; every V-cycle precision. */
#define AMG_SMOOTH_SPAI0 0
#define AMG_SMOOTH_ILU0 1
#define AMG_SMOOTH_BJACOBI 2

/* Block CSR matrix, borrowed for the duration of a call.
 * row_ptr[nbrows+1] and col[nnzb] are int32 with columns strictly ascending
 * within each block row; val holds nnzb blocks of bs_r x bs_c doubles, each
 * block row-major.  All three arrays are device pointers. */
typedef struct {
    int32_t nbrows, nbcols;
    int32_t bs_r, bs_c;
    int64_t nnzb;
    const int32_t *row_ptr;
    const int32_t *col;
    const double *val;
} amg_bsr;

/* Device memory supplier of a hierarchy (amg_params.allocator).  With
 * allocator == NULL the library allocates stream-ordered with
 * cudaMallocAsync / cudaFreeAsync.  Otherwise every device buffer that a
 * handle holds, and every temporary device buffer of a call on that handle,
 * comes from alloc() and goes back through free(), so that the caller's
 * memory manager (for example PyTorch's caching allocator) sees and bounds
 * the hierarchy.
 *   alloc(ctx, bytes, stream): return a device pointer to at least `bytes`
 *     bytes, 256-byte aligned, usable by work ordered on `stream` (the
 *     stream of the call that allocates; NULL = legacy default stream), or
 *     NULL on failure (the call then returns AMG_ERR_CUDA).
 *   free(ctx, ptr, bytes, stream): take back a pointer alloc() returned,
 *     with its size.  Temporaries are given back while work that uses them
 *     may still be queued on `stream`, as with cudaFreeAsync: the supplier
 *     must not hand the memory to work on another stream before that work
 *     completes.  amg_free and amg_batch_free synchronise the device before
 *     giving back a handle's buffers.
 * The library copies the struct at setup; ctx and the two functions must
 * stay valid until the handle is freed.  Both are called on the thread that
 * makes the library call, except in amg_batch_setup: it sets its instances
 * up on up to 8 host threads at once, each allocating for a stream of its
 * own (non-blocking streams that the library creates per device on first
 * use and keeps for the life of the process, so a caching supplier can reuse
 * what it cached for them at the next batch setup), so there the two
 * functions must be safe to call concurrently.  Memory allocated for such a
 * stream may later be given back with the caller's stream once the setup
 * has synchronised that stream. */
typedef struct {
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
    void *ctx;
} amg_allocator;

/* Setup and cycle parameters (the paper names none of them; defaults are the
 * readings of its silent points, see the design notes shipped with the
 * library). */
typedef struct {
    double eps_strong;     /* strength threshold on level 1; halved per level (0.08) */
    double relax;          /* multiplier of omega = (4/3)/rho in P smoothing (2.0: the
                              Gershgorin rho over-estimates lambda_max(D^-1 A) by
                              1.4-2.2x on elasticity matrices) */
    double smooth_relax;   /* damping of the SPAI0 smoother; with AMG_SMOOTH_BJACOBI,
                              half the target top eigenvalue of M A (0.8) */
    int32_t coarse_enough; /* stop coarsening at <= this many scalar rows (3000); a level
                              below the finest with <= 2 coarse_enough rows also stops
                              when its aggregates would give < coarse_enough / 4 rows */
    int32_t max_levels;    /* at most this many levels (15) */
    int32_t npre, npost;   /* smoothing sweeps before / after the correction (1, 1) */
    int32_t precision;     /* AMG_PREC_* of the V-cycle (AMG_PREC_FP64) */
    int32_t loop_mode;     /* 0: CG loop on the device (graph with a conditional while
                              node); 1: the host launches one captured iteration graph
                              per CG step (for profilers that cannot look inside
                              conditional graphs).  Same kernels, same results. */
    int32_t storage;       /* AMG_STORAGE_* of the solve's operators (AMG_STORAGE_BLOCK) */
    int32_t aggregation;   /* AMG_AGG_* (AMG_AGG_GREEDY) */
    int32_t smoother;      /* AMG_SMOOTH_* (AMG_SMOOTH_SPAI0) */
    int32_t ilu_sweeps;    /* Jacobi sweeps per triangle of AMG_SMOOTH_ILU0, 0..64 (2) */
    int32_t setup;         /* AMG_SETUP_* (AMG_SETUP_BLOCK) */
    int32_t reserved;      /* must be zero */
    const amg_allocator *allocator; /* device memory supplier, or NULL for the library's
                              own stream-ordered allocations (NULL) */
} amg_params;

typedef struct amg_handle_s *amg_handle;

/* Per-level description filled by amg_level_info (host struct). */
typedef struct {
    int32_t nbrows;        /* block rows of A on this level */
    int32_t bs;            /* block size of A (3 on level 0, nb_ns below) */
    int64_t nnzb_A;
    int64_t nnzb_P;        /* 0 on the coarsest level */
    int32_t nagg;          /* aggregates = block rows of the next level (0 on the coarsest) */
    int32_t is_coarsest;
    double eps, omega, rho;
    double smoother_lambda; /* AMG_SMOOTH_BJACOBI: the lambda_max(D_b^-1 A) estimate of
                               this level (0 otherwise) */
} amg_level_desc;

/* Whole-hierarchy statistics (host struct). */
typedef struct {
    int32_t nlevels;
    int32_t coarse_n;          /* scalar size of the dense coarsest system */
    double setup_seconds;      /* wall time of amg_setup (host clock, synchronised) */
    int64_t bytes_matrices;    /* A, P, R of all levels + smoother + coarse inverse */
    int64_t bytes_total;       /* everything the handle holds on the device */
    double operator_complexity;/* sum of nnz over levels / nnz of the finest A */
    int32_t learned;           /* 1 while level 0 smooths with learned 3x3 blocks */
    int32_t reserved0;
    double learned_lambda;     /* lambda_max(M A) estimate of the last learned smoother
                                  offered to amg_set_learned_smoother (0 if none) */
    double spai0_lambda;       /* the same estimate for SPAI0 (0 until one was offered) */
    int64_t bytes_solve;       /* the solve's operator copies (sliced A_l, P_l, R_l in the
                                  V-cycle's precision and storage, plus the fine FP64 A):
                                  values, column indices, slice pointers, row maps */
    double setup_phase_seconds[7]; /* wall time of amg_setup by phase, summed over levels:
                                  0 input copy and pattern check, 1 strength and
                                  aggregation, 2 transfer operators (tentative QR, omega,
                                  smoothed P, R), 3 Galerkin products, 4 smoothers (SPAI0,
                                  ILU(0)), 5 coarsest factor, 6 solve copies and vectors */
} amg_stats;

/* Fill *prm with the defaults listed above.  Returns AMG_OK. */
int amg_params_default(amg_params *prm);

/* Alg. 1: build the hierarchy for A (3x3 BSR, square, symmetric positive
 * definite) with near-nullspace B (device, row-major [nbrows*3][nb_ns]:
 * nb_ns = 6, the three translations and three rotations, or nb_ns = 3, the
 * translations only, which is the block solver of Sec. 4 without a
 * near-nullspace; coarse nodes carry nb_ns DOFs).  prm may be NULL for
 * the defaults.  On success *out owns every level on the device (allocated
 * stream-ordered on `stream`).  A and B are only read.  The block pattern is
 * checked on the device before any other kernel reads it: row pointers
 * within [0, nnzb] and non-decreasing, columns ascending and in range, a
 * diagonal block in every row, and a symmetric pattern; a violation returns
 * AMG_ERR_ARG naming the lowest offending block row.  A NaN or infinite
 * value in A or B also returns AMG_ERR_ARG. */
int amg_setup(const amg_bsr *A, const double *B, int32_t nb_ns, const amg_params *prm,
              void *stream, amg_handle *out);

/* Alg. 2 used as a preconditioner: z = V(r), one V-cycle from a zero initial
 * guess on every level.  r and z are device vectors of 3*nbrows doubles and
 * must not overlap. */
int amg_apply_vcycle(amg_handle h, const double *r, double *z, void *stream);

/* Sec. 4: CG preconditioned by one V-cycle per iteration.  u (device) holds
 * the initial guess on entry and the solution on exit; f is the right-hand
 * side.  The loop runs on the device (a CUDA graph with a conditional while
 * node) until the recurrence residual ||r||/||f|| <= tol is confirmed by the
 * true residual, or maxiter iterations.  *iters (host) receives the number
 * of A*p products and *rel_resid (host) the final true relative residual
 * ||f - A u|| / ||f||.  Returns AMG_OK, AMG_NOT_CONVERGED or an error
 * (AMG_ERR_ARG before any iteration when f or u holds a NaN or infinite
 * value); the call synchronises `stream`. */
int amg_solve(amg_handle h, const double *f, double *u, double tol, int32_t maxiter,
              int32_t *iters, double *rel_resid, void *stream);

/* Statistics of the hierarchy (host struct). */
int amg_get_stats(amg_handle h, amg_stats *out);

/* Description of level `level` (0 = finest). */
int amg_level_info(amg_handle h, int32_t level, amg_level_desc *out);

/* Copy one operator of a level to HOST buffers sized from amg_level_info:
 * which = 0: A (nbrows+1, nnzb_A, nnzb_A*bs*bs), 1: P (bs x nb_ns blocks),
 * 2: R (nb_ns x bs blocks, nagg+1 row pointers).  Any pointer may be NULL.
 * which = 3: the aggregate of every node (row_ptr receives nbrows int32,
 * -1 for an isolated node); which = 4: the smoother diagonal (val receives
 * nbrows*bs doubles); which = 5: the near-nullspace of the level (val
 * receives nbrows*bs*nb_ns doubles); which = 6: the strong-connection flags of A
 * (row_ptr receives nnzb_A bytes); which = 7: the smoother blocks of the
 * level -- block damped Jacobi, or the learned blocks of level 0 -- (val
 * receives nbrows*bs*bs doubles); with AMG_SMOOTH_ILU0, which = 8:
 * the block ILU(0) factor on A's block pattern (val receives nnzb_A*bs*bs
 * doubles: L below the diagonal, U on and above it) and which = 9: the
 * inverses of U's diagonal blocks (val receives nbrows*bs*bs doubles).
 * Synchronises the stream it was set up on. */
int amg_level_export(amg_handle h, int32_t level, int32_t which, int32_t *row_ptr,
                     int32_t *col, double *val);

/* y = op x with the hierarchy's own V-cycle kernel for operator `which` of
 * level `level` (0: A, 1: P, 2: R), in the sliced block-ELL layout the solve
 * uses.  which = 3, 4, 5: the same operators in the FP32-pair copies of an
 * AMG_PREC_DF64 hierarchy (AMG_ERR_STATE otherwise).  x has (columns x block
 * columns) and y (rows x block rows) doubles, device, not overlapping, x
 * 8-byte aligned (AMG_ERR_ARG otherwise).  Asynchronous on `stream`. */
int amg_level_spmv(amg_handle h, int32_t level, int32_t which, const double *x, double *y,
                   void *stream);

/* The Galerkin product A_{l+1} = R_l (A_l P_l) of level `level` (Alg. 1,
 * "A_{i+1} = R_i A_i P_i"; the setup's dominant cost, Sec. 3) recomputed in
 * block storage (AMG_STORAGE_BLOCK: the setup's own block SpGEMMs) or in
 * scalar CSR (AMG_STORAGE_SCALAR: A, P, R unblocked, the same SpGEMM kernels
 * with 1x1 blocks), the setup-phase side of the block vs scalar comparison
 * of Sec. 4.  *seconds (host) receives the wall time of the product (symbolic
 * and numeric passes, their allocations, synchronised), *rel_diff (host) the
 * largest difference from the hierarchy's A_{l+1} (unblocked for scalar)
 * over its largest entry, or -1 if the patterns differ.  The result is
 * freed before returning.  Synchronises the stream the handle was set up on;
 * AMG_ERR_ARG if `level` has no coarser level. */
int amg_level_galerkin(amg_handle h, int32_t level, int32_t storage, double *seconds,
                       double *rel_diff);

/* Padding of the sliced layout of A, P, R on `level` (host double[3]): extra
 * stored blocks / structural blocks (0 for an absent operator). */
int amg_level_padding(amg_handle h, int32_t level, double *pad3);

/* Release everything the handle owns.  NULL is ignored. */
void amg_free(amg_handle h);

/* Message of the calling thread's last error ("" if none). */
const char *amg_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (a graph execution counts each kernel node once per loop iteration).
 * Host-only bookkeeping; needs no GPU. */
int64_t amg_kernel_launches(void);

/* ---- primitives (the hot kernels on their own) ------------------------- */

/* y = A x for a BSR matrix with block shape (bs_r, bs_c) in {(3,3), (6,6),
 * (3,6), (6,3)}: the block SpMV of Sec. 2 (memory-bound primitive).  x has
 * nbcols*bs_c and y nbrows*bs_r doubles (device, not overlapping). */
int amg_bsr_spmv(const amg_bsr *A, const double *x, double *y, void *stream);

/* y = A x and *dot_out (host) = x . y for a square 3x3 or 6x6 BSR matrix,
 * with the dot product reduced in a fixed order (deterministic).  The
 * reduction uses a device scratch array that the call allocates and frees
 * stream-ordered.  Synchronises `stream`. */
int amg_bsr_spmv_dot(const amg_bsr *A, const double *x, double *y, double *dot_out,
                     void *stream);

/* ---- batched form ------------------------------------------------------ */

typedef struct amg_batch_s *amg_batch;

/* Description of a batch (host struct). */
typedef struct {
    int32_t ninst;          /* instances */
    int32_t nrhs_total;     /* right-hand sides over all instances */
    int32_t nlevels;        /* deepest hierarchy */
    int32_t reserved0;
    double setup_seconds;
    int64_t dofs_total;     /* fine-level unknowns over all instances */
    int64_t bytes_total;    /* device memory held by the batch */
    int32_t rhs_tile[48];   /* autotuned right-hand-side tile of A, P, R per level */
    int32_t cta_threads[48];/* autotuned block-row tiling of A, P, R per level: threads
                               per CTA (64, 128, 256; each warp one slice of 32 / G
                               block rows), 0 for an absent operator */
    int32_t ctas_per_sm[48];/* ... and the CTAs per SM before the warp-strided loop
                               wraps (16, 32) */
    double setup_phase_seconds[4]; /* wall time of the setup's phases: the instances'
                               hierarchies (set up by several host threads at once),
                               the concatenated level operators and vectors, the
                               coarse inverses and CG state, the autotuner */
} amg_batch_desc;

/* Many independent instances of Eq. 1, each with its own near-nullspace and
 * nrhs[i] (1..16) load cases, solved together.  Builds one hierarchy per
 * instance exactly as amg_setup would (Alg. 1, same parameters, V(1,1) with
 * SPAI0), on up to 8 host threads at once, and the grouped structures of the
 * batched V-cycle: level l of every instance in one concatenated sliced
 * operator, right-hand sides interleaved so the SpMM reads each block once
 * per tile of right-hand sides, and per operator the tile (1, 2, 4) and the
 * launch shape (threads per CTA, CTAs per SM) chosen by timing the
 * candidates.  A[i] (3x3 BSR) and B[i] (n_i x 6) are device arrays, read
 * only, written on `stream` before the call.  Block storage and the block
 * setup only; prm->precision FP64, FP32 or emulated FP64 (the V-cycle's
 * operators and its coarse solves; CG stays FP64); prm->loop_mode 1 launches one captured
 * iteration per host step, for profilers, with the same results.  An error
 * in an instance's setup is reported as "instance <i>: <message>" for the
 * lowest-numbered failing instance.  Synchronises `stream`. */
int amg_batch_setup(int32_t ninst, const amg_bsr *A, const double *const *B, const int32_t *nrhs,
                    const amg_params *prm, void *stream, amg_batch *out);

/* CG preconditioned by one V-cycle (Sec. 4) for every (instance, rhs) pair at
 * once, each pair with its own scalars and stopping test (relative residual
 * tol confirmed by the true residual, or maxiter); the loop is one graph with
 * a conditional while node.  F[i] and U[i] are device arrays of nrhs[i]
 * contiguous vectors of 3 n_i doubles (U[i]: initial guesses in, solutions
 * out).  iters and rel_resid (host, optional) receive one value per rhs in
 * instance order.  Returns AMG_OK when every rhs converged, AMG_NOT_CONVERGED
 * or an error otherwise (AMG_ERR_ARG, naming the pair, when an f or u holds a
 * NaN or infinite value).  Synchronises `stream`.  A pair's iterates do not
 * depend on the other pairs of the batch. */
int amg_batch_solve(amg_batch h, const double *const *F, double *const *U, double tol,
                    int32_t maxiter, int32_t *iters, double *rel_resid, void *stream);

int amg_batch_info(amg_batch h, amg_batch_desc *out);
void amg_batch_free(amg_batch h);

/* ---- learned smoother ---------------------------------------------------- */

/* Parameters of the smoother network, FP32, flat in this order:
 * W1 [64][12], b1 [64], W2 [6][64], b2 [6] (AMG_LEARNED_NPARAM values). */
#define AMG_LEARNED_NPARAM 1222

/* Replace the fine-level SPAI0 smoother of h by learned 3x3 blocks
 * M_I = S_I L_I L_I^T S_I, S_I = diag(sqrt(SPAI0 diagonal of node I)),
 * L_I the lower triangular factor [[1+o0,0,0],[o3,1+o1,0],[o4,o5,1+o2]] with
 * o = W2 relu(W1 x_I + b1) + b2 and x_I the node's unit-free features (the
 * diagonal block over its Frobenius norm, the sum of squared and the largest
 * neighbour-block norms relative to it, the block count / 27).  The network
 * runs on the tensor cores (BF16 operands, FP32 accumulation).  The paper
 * uses a fixed smoother (Sec. 3 names SPAI); this data-driven stand-in keeps
 * SPAI0 as its fallback: if any L_I is singular (M_I only semidefinite) the
 * call keeps SPAI0 and sets *fell_back (host) to 1; if the estimate of
 * lambda_max(M A) on level 0 (20 power iterations) reaches max(1.9, the same
 * estimate for SPAI0) it keeps SPAI0 and sets *fell_back to 2 (the smoothing
 * step contracts the energy norm only while lambda_max(M A) < 2, and beyond
 * that the V-cycle can stop being positive definite).  params is host memory.
 * Later amg_solve / amg_apply_vcycle calls use the blocks, in every V-cycle
 * precision (the FP32 and BF16 V-cycles apply an FP32 copy); block storage
 * only (AMG_ERR_ARG for AMG_STORAGE_SCALAR). */
int amg_set_learned_smoother(amg_handle h, const float *params, int32_t *fell_back, void *stream);

/* Back to the SPAI0 smoother. */
int amg_clear_learned_smoother(amg_handle h);

typedef struct amg_trainer_s *amg_trainer;

/* Trainer of the smoother network: Adam (learning rate lr) on FP32 master
 * weights, loss L = mean over problems and error samples of the energy-norm
 * error reduction of one smoothing step, ||e_s - M A e_s||_A^2 / ||e_s||_A^2,
 * gradients from the project's own forward/backward kernels.  params: host,
 * initial values.  Problems are borrowed hierarchies that must outlive the
 * trainer. */
int amg_trainer_create(const float *params, double lr, void *stream, amg_trainer *out);
/* Add a problem with given error samples R (device, [nsamples][3 nbrows]). */
int amg_trainer_add_samples(amg_trainer t, amg_handle h, const double *R, int32_t nsamples,
                            void *stream);
/* Add a problem with error samples the method produces: for random e0
 * (SplitMix64 of seed and the index), even samples e = e0 - V(A e0), the error
 * one of the hierarchy's SPAI0 V-cycles leaves, odd samples e = e0 (white
 * noise, so that the loss also sees the top of the spectrum). */
int amg_trainer_add_generated(amg_trainer t, amg_handle h, int32_t nsamples, uint64_t seed,
                              void *stream);
/* Loss and gradient (host, AMG_LEARNED_NPARAM floats; may be NULL) at the
 * current parameters, without an update. */
int amg_trainer_eval(amg_trainer t, double *loss, float *grad, void *stream);
/* nsteps Adam steps; *loss (host) = the loss before the last step. */
int amg_trainer_step(amg_trainer t, int32_t nsteps, double *loss, void *stream);
/* Current parameters (host, AMG_LEARNED_NPARAM floats). */
int amg_trainer_params(amg_trainer t, float *out);
void amg_trainer_free(amg_trainer t);

/* Measured FP64 FMA rate of the current device (host outputs), the
 * denominator of the arithmetic roofline of the FP64 SpMV: every SpMV entry
 * is one FMA (2 b_r b_c flops per block, Sec. 2's block arithmetic), and on
 * GB300 the FP64 pipe, not HBM, bounds that kernel.  Threads of 256-thread
 * CTAs run 4, 8 or 16 independent FMA chains at 2, 4 or 8 CTAs per SM, the
 * same total work (about 8 x 4 x 256 x `iters` FMAs per SM) in every
 * configuration, each timed with CUDA events on `stream` after a short
 * warm-up launch; the fastest configuration's rate is reported.  sink
 * (device, sink_len doubles, caller-owned, at least 2048 x the SM count)
 * receives the chains' sums so that the work is observable.  *fma_per_second = FMAs / s; *seconds (may
 * be NULL) = the duration of the fastest configuration; *num_sms (may be
 * NULL) = the device's SM count.  Synchronises `stream`. */
int amg_fp64_fma_rate(double *sink, int64_t sink_len, int32_t iters, double *fma_per_second,
                      double *seconds, int32_t *num_sms, void *stream);

/* Same result as amg_bsr_spmv_dot, without allocating.  (The paper has no
 * counterpart: this serves callers of the library, not the method.)
 * amg_bsr_spmv_dot allocates device scratch for its per-CTA partial sums; a
 * caller that cannot allow a device allocation inside the call -- because
 * one may fail or wait for the whole device at a point where the caller has
 * a fixed memory budget, or because its device memory is owned by another
 * allocator -- calls this variant, which keeps that scratch in a static
 * device array of AMG_NOALLOC_SCRATCH_DOUBLES doubles (32 KiB, held by every
 * GPU that loads the library until the process exits).  It makes no
 * cudaMalloc, cudaFree or allocating library call; x, y and the result are
 * the caller's.  The launch needs one partial sum per CTA plus one for the
 * total; a launch that would need more than the array holds is rejected with
 * AMG_ERR_LIMIT (on GB300 the launch needs at most 8 x 152 + 1).  The
 * arguments are checked as for amg_bsr_spmv_dot.  The first call on a
 * device (and the first after that device's context was re-created) looks
 * up the array's device address, so make that first call before any stream
 * capture.  All calls share the array, which keeps the last call's partial
 * sums: calls whose work overlaps on the GPU (two streams, two host threads)
 * race on it; calls ordered on one stream are safe.  The call reads the
 * total back to the host and synchronises `stream` before it returns. */
#define AMG_NOALLOC_SCRATCH_DOUBLES 4096
int amg_bsr_spmv_dot_noalloc(const amg_bsr *A, const double *x, double *y, double *dot_out,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AMG_GB300_H */
