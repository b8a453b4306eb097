/*
 * spchol: supernodal sparse Cholesky factorization and solves on one GB300 GPU.
 *
 * The operation is the one of arXiv 1608.00044 ("An Asynchronous Task-based
 * Fan-Both Sparse Cholesky Solver"):
 *   - Section II-A, Eq. 1: A = L L^T for a symmetric positive definite A, then
 *     the two triangular solves L y = b, L^T x = y.
 *   - Section V: a fill-reducing symmetric permutation P is applied first; the
 *     library factors P A P^T = L L^T.
 *   - Section II-B: the columns of L are grouped into supernodes (consecutive
 *     columns with a dense diagonal block whose rows below are each entirely
 *     zero or entirely nonzero); Section III-B caps a supernode's width.
 *   - Section III-A and IV: the factorization is the set of tasks F (factor a
 *     supernode), U (update an ancestor) and A (apply the update), run in any
 *     order that respects the dependencies of Section II-C.  Here the tasks run
 *     in one persistent GPU kernel driven by device-side dependency counters.
 *
 * Conventions for every entry point:
 *   - Matrices are given as the LOWER triangle, diagonal included, in CSC form:
 *     colptr (int64, n+1 entries, colptr[0] = 0, non-decreasing), rowind
 *     (int32, colptr[n] entries, strictly increasing inside each column, every
 *     row >= its column and < n).  values holds colptr[n] doubles in the same
 *     order.  Host arrays passed to analyze are copied; the caller keeps
 *     ownership.
 *   - perm is new -> old: row/column i of P A P^T is row/column perm[i] of A.
 *     NULL means the identity.  The library may refine perm by a postorder of
 *     the elimination tree, which leaves the fill unchanged.
 *   - Dense blocks (B, X) are column-major, n rows, leading dimension ldb >= n.
 *   - Pointers to values and right-hand sides may be host or device memory; the
 *     library inspects the pointer.  Device pointers must be on the device that
 *     was current at analyze.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is stream-ordered; the calls below return after the status
 *     word of their launch has been read back, so results are complete on
 *     return.
 *   - A handle owns all device memory it allocates and frees it in
 *     spchol_destroy (through the caller's allocator when spchol_options
 *     gives one, else stream-ordered from the device's memory pool).  A handle is not safe for concurrent use from two host
 *     threads; distinct handles are independent.
 *
 * Return codes: 0 on success; -k when argument k (1-based) is invalid;
 * k > 0 from factorize when P A P^T is not positive definite, k being the
 * smallest (1-based, permuted) column whose pivot was not positive; otherwise
 * one of the SPCHOL_E* codes below.
 */
#ifndef SPCHOL_H
#define SPCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPCHOL_OK 0
#define SPCHOL_ENOMEM (-1001)   /* device or host allocation failed */
#define SPCHOL_ETIMEOUT (-1002) /* a device wait exceeded wait_budget_ns */
#define SPCHOL_ESTATE (-1003)   /* call out of order (e.g. solve before factorize) */
#define SPCHOL_ENOCONV (-1004)  /* refinement did not reach ir_tol; X holds the best iterate */
#define SPCHOL_ECUDA (-1005)    /* a CUDA runtime call failed */
#define SPCHOL_EINTERNAL (-1006)/* a device-side consistency check failed */
#define SPCHOL_ESCRATCH (-1007) /* spchol_solve_noalloc: n * nrhs (and, with deterministic = 2,
                                   the solves' buffers) too large for its fixed scratch */

/* Arithmetic of the factor. */
#define SPCHOL_FP64 0  /* everything in FP64 */
#define SPCHOL_FP32 1  /* FP32 panels and updates, FP64 diagonal POTRF, FP64 residual + refinement */
#define SPCHOL_TF32 2  /* as FP32, update GEMMs on TF32 tensor cores (tcgen05.mma kind::tf32) */
#define SPCHOL_TF32X3 3 /* as TF32, each operand split into a TF32 head and tail, three products per
                           tile: FP32-level accuracy on the tensor cores */
#define SPCHOL_FP64_TC 4 /* FP64 panels and FP64 result; the update GEMMs of panels at least 16 columns
                            wide run on BF16 tensor cores (tcgen05.mma kind::f16) on an exact 7-way
                            8-bit split of each FP64 row (Ozaki-style error-free transformation),
                            recombined exactly in integers; narrower panels keep DFMA tiles.  The
                            solves' panel tiles (panels 16..64 wide) run the same split on the
                            BF16 tensor cores (mma.sync).  The error of a split product is bounded
                            by 2^-56 max|row| max|column| per term, not per product: FP64 backward
                            error, but rows and columns of very different scales lose forward
                            accuracy that SPCHOL_FP64 keeps */

typedef struct spchol_handle_s* spchol_handle_t;

typedef struct spchol_options {
  int precision;          /* SPCHOL_FP64 (default), SPCHOL_FP32, SPCHOL_TF32, SPCHOL_TF32X3, SPCHOL_FP64_TC */
  int max_width;          /* W: supernode panels are at most W columns (Section III-B caps at 150);
                             1..128 (1..64 with the tensor-core precisions), default 64 */
  int relax_zeros;        /* amalgamation: a child supernode is merged into its parent when every
                             merged column gains at most this many explicit zeros; default 4, 0 = off */
  int tile_rows;          /* rows per update tile, 1..64; 0 = default (64).  The tensor-core tiles
                             ignore it: 128 rows for TF32, 64 for SPCHOL_FP64_TC */
  int ctas_per_sm;        /* persistent-kernel CTAs per SM; 0 = as many as fit */
  int deterministic;      /* 1: the static (target, source) order of Section IV-B: the update tiles
                             into each target panel, and the solve tiles into each panel's
                             entries, run one after another in (source, tile) order, so every
                             sum lands in one fixed order and the factor and solution are
                             bitwise reproducible (run to run, alone or in a batch); slower.
                             2: bitwise reproducible by fan-in aggregation (Section II-C's
                             fan-in family): every update tile stores its product in a private
                             buffer, and each panel adds the buffers into its rows in one fixed
                             (tile) order when it is factored, so the update tiles themselves
                             run in any order; a panel's row pieces are gathered by tasks of
                             their own, in parallel.  The solves aggregate the same way (each
                             solve tile's product in a buffer, added by the diagonal tasks in
                             tile order).  Every entry receives its updates in the same order
                             as with 1, so the results are bitwise those of 1, at a fraction of
                             1's time.  The factor's buffers cost (sum over update tiles of
                             rows x columns) values of device memory, in footprint_bytes; the
                             solves' (sum of solve tile rows + widths) x nrhs more.
                             0 (default): dynamic order, results equal up to rounding */
  int64_t wait_budget_ns; /* bound on any single device-side wait; default 2e9 (2 s) */
  int ir_max_iter;        /* mixed precision: refinement steps; default 10 */
  double ir_tol;          /* mixed precision: target backward error; default 1e-12 */
  int fault_inject;       /* failure-detection test hook, 0 = off.  1: analyze adds one phantom
                             dependency to the last panel, so its diagonal task never becomes ready
                             and factorize must return SPCHOL_ETIMEOUT after wait_budget_ns. */
  int profile;            /* 1: the persistent kernels time every task (per-type busy time and the
                             time spent waiting for a ready task, summed over CTAs) into the stats;
                             2: additionally record each task's start and end (spchol_trace_get) */
  int solve_tile_rows;    /* rows per triangular-solve tile of the panels more than 128 levels below
                             the root, 8..256; 0 = default (64).  Panels nearer the root take 32 */
  int sched;              /* which ready task runs first in the dynamic schedules (deterministic 0,
                             and the update tiles of 2) -- the question of Section V-A:
                             0 (default): two ready rings; the diagonal and panel-solve tasks and,
                             near the root, the update tiles into the etree parent (the critical
                             path) go ahead of the other update tiles; in the solve, tasks made ready
                             by other tasks go ahead of the leaves.
                             1: one FIFO ring: every ready task runs in the order it became ready */
  /*
   * Device memory of the handle.  With dev_alloc = dev_free = NULL (the default)
   * the library allocates with stream-ordered cudaMallocAsync / cudaFreeAsync
   * from the device's default memory pool, so that neither spchol_destroy nor
   * a solve that grows its workspace waits for work that other streams are
   * running.  Otherwise every device allocation of the handle goes through the
   * caller's allocator (e.g. PyTorch's caching allocator):
   *   dev_alloc(bytes, stream, ctx): device memory on the handle's device (the
   *     current device during the call), at least 256-byte aligned, or NULL on
   *     failure (the library then returns SPCHOL_ENOMEM).  stream: the stream
   *     of the call that needs the memory, which first uses it in that stream's
   *     order; NULL from spchol_analyze, whose memory is complete when analyze
   *     returns and is then used on any stream.
   *   dev_free(ptr, bytes, stream, ctx): called only when no work of the
   *     library that uses ptr is pending -- every entry point except
   *     spchol_factorize_enqueue has finished its device work when it returns;
   *     destroy a handle only after the stream of its last enqueued
   *     factorization has completed.  stream: as for dev_alloc (NULL from
   *     spchol_destroy).
   * Set both or neither (-5 from analyze otherwise).  Pinned host memory for
   * status words is the library's own, recycled across handles. */
  void* (*dev_alloc)(size_t bytes, void* stream, void* ctx);
  void (*dev_free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* alloc_ctx;        /* passed to dev_alloc / dev_free as ctx */
  int solve_w_depth;      /* the solves' near-root steps (Section II-A's triangular solves, restated):
                             panels within this many levels of the root of the panel elimination
                             tree (up to 64 columns wide, outside subtree tasks) also keep
                             W = L21 L11^{-1}, formed by the factorization after each L21 tile,
                             so that a forward step is y_below -= W b_s and a backward step
                             x_s -= W^T x_below, with no diagonal solve between two steps of the
                             chain.  Costs the W buffer (the footprint counts it) and
                             2 (rows below) w^2 flops per such panel in the factorization.
                             0 = default (32 for spchol_analyze, none for spchol_batch_analyze);
                             -1 = none; not used with deterministic != 0 */
} spchol_options;

typedef struct spchol_stats {
  int64_t n;
  int64_t nnz_a;          /* stored entries of the lower triangle of A */
  int64_t nnz_l;          /* entries of L (exact structure, no amalgamation zeros) */
  int64_t nnz_l_stored;   /* entries held in the supernode panels (lower part incl. zeros) */
  double flops;           /* sum over columns of c_j^2, c_j the exact column count of L */
  int64_t n_supernodes;   /* panels after amalgamation and the width cap */
  int64_t n_tasks;        /* factorization tasks (diagonal factor + panel solve tiles + update tiles) */
  int64_t max_width;
  int64_t max_rows;
  int64_t footprint_bytes;/* device bytes owned by the handle */
  double analyze_ms;      /* host time of analyze */
  double factor_ms;       /* device time of the last factorize (assembly + factorization) */
  double solve_ms;        /* device time of the last solve */
  int ir_iters;           /* refinement steps of the last solve */
  double berr;            /* backward error of the last solve (mixed precision), else -1 */
  int precision;
  /* filled when spchol_options.profile = 1; CTA-milliseconds summed over all CTAs */
  double factor_task_ms[3];   /* diagonal factor, panel-solve tiles, update tiles */
  int64_t factor_task_count[3];
  double factor_wait_ms;      /* waiting for a ready task */
  double solve_task_ms[4];    /* forward diagonal, forward tiles, backward tiles, backward diagonal */
  double solve_wait_ms;
  double factor_tc_update_ms; /* part of factor_task_ms[2] spent in tensor-core update tiles */
  int grid_factor;            /* CTAs of the persistent factorization launch */
  int grid_solve;
  int tma_staging;            /* 1: update-tile operands arrive by TMA (a tensor map per panel); 0: cp.async */
  int n_subtrees;             /* subtree tasks: small subtrees of the panel tree factored by one CTA each */
  double factor_subtree_ms;   /* profile: time in subtree tasks (summed over CTAs) */
  int64_t factor_subtree_count;
  int ir_gmres_iters;         /* mixed precision: GMRES-IR steps of the last solve (0 when classic
                                 refinement reached the target) */
  double factor_gather_ms[3]; /* profile, deterministic = 2: time of the fan-in gathers (summed over
                                 CTAs) cutting batches, staging them and adding them */
  int64_t factor_gather_batches;
  int64_t factor_gather_tiles;
  int64_t n_warp_subtrees;   /* subtree tasks whose factorization and solves run on single warps (panels
                                at most 32 wide, FP64 or FP32 updates, when the subtrees hold a good
                                part of the work: batches of small matrices) */
} spchol_stats;

/* Fill *opt with the defaults listed above. */
void spchol_default_options(spchol_options* opt);

/*
 * Symbolic analysis of P A P^T (Section II-B): elimination tree, postorder,
 * column counts, supernodes, relaxed amalgamation, the width cap, row
 * structures, and the task graph of Sections III-A / IV.  Uploads the
 * structures to the current device.
 *   n       matrix order, >= 0                                  (argument 1)
 *   colptr  host int64[n+1]                                     (argument 2)
 *   rowind  host int32[colptr[n]]                               (argument 3)
 *   perm    host int64[n] new->old, or NULL                     (argument 4)
 *   opt     options, or NULL for the defaults                   (argument 5)
 *   out     receives the handle                                 (argument 6)
 * Returns 0, -k for an invalid argument k, SPCHOL_ENOMEM or SPCHOL_ECUDA.
 */
int spchol_analyze(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm,
                   const spchol_options* opt, spchol_handle_t* out);

/*
 * Fill-reducing ordering for a general sparse symmetric pattern, for inputs
 * that come without one (Section V applies a fill-reducing permutation first;
 * the paper takes it from Scotch).  Nested dissection by breadth-first level
 * structures (George 1973; George and Liu 1978): a connected set is rooted at a
 * pseudo-peripheral vertex and cut at its smallest level that leaves 35-65 % of
 * the set below; the two parts are ordered first, recursively, and the
 * separator last; sets of at most 64 vertices are ordered by minimum degree.
 * Host code; needs no GPU.
 *   n         matrix order, >= 0                                (argument 1)
 *   colptr    host int64[n+1], as in spchol_analyze             (argument 2)
 *   rowind    host int32[colptr[n]], as in spchol_analyze       (argument 3)
 *   perm_out  host int64[n]: receives the ordering, new -> old,
 *             ready to pass to spchol_analyze                   (argument 4)
 * Only the pattern is read.  Returns 0 or -k for an invalid argument k (the
 * same checks as spchol_analyze).
 */
int spchol_order_nd(int64_t n, const int64_t* colptr, const int32_t* rowind, int64_t* perm_out);

/*
 * Numeric factorization P A P^T = L L^T (Eq. 1) with the structure of analyze.
 * values: colptr[n] doubles of A's lower triangle in analyze's order, host or
 * device.  The factor stays resident in the handle for later solves.
 * Returns 0, k > 0 (not positive definite at permuted column k), or an error.
 */
int spchol_factorize(spchol_handle_t h, const double* values, void* stream);

/*
 * spchol_factorize split in two for CUDA-graph capture.  _enqueue queues the
 * whole factorization (assembly, counter reset, the persistent factorization
 * kernel, and a copy of its status words to pinned host memory) on `stream`
 * without synchronising the host and without allocating; values must be
 * DEVICE memory (for a batch handle: all matrices' values concatenated in
 * batch order).  After the stream (or the graph it was captured into) has
 * completed, _status returns what spchol_factorize would have returned and
 * makes the factor available to the solves.  Returns of _enqueue: 0, -1/-2
 * for bad arguments, SPCHOL_ECUDA.
 */
int spchol_factorize_enqueue(spchol_handle_t h, const double* values, void* stream);
int spchol_factorize_status(spchol_handle_t h);

/*
 * Solve A X = B with the resident factor (Section II-A: L y = P b, L^T z = y,
 * x = P^T z).  B (n x nrhs, column-major, leading dimension ldb) is overwritten
 * by X; host or device memory.  In the mixed-precision modes the solve refines
 * with an FP64 residual until berr <= ir_tol (or ir_max_iter steps) and returns
 * SPCHOL_ENOCONV if the target was not reached.
 */
int spchol_solve(spchol_handle_t h, double* B, int64_t ldb, int nrhs, void* stream);

/*
 * The solve of spchol_solve, for callers that cannot allocate device memory at
 * the time they solve: a service that reserves all of its device memory up
 * front, or code running where cudaMalloc is not allowed.  spchol_solve may
 * allocate its workspace on first use or when nrhs grows; this entry point
 * allocates nothing.  Its workspace (the permuted right-hand sides and the
 * task queue of the solve kernel) lives in one fixed 32 MiB array in device
 * memory that every GPU loading the library holds until the process exits.
 * The paper has no counterpart; it is an interface convenience.
 *   h      a handle with a resident FP64 factor (SPCHOL_FP64 or SPCHOL_FP64_TC;
 *          other precisions return -1), factored by spchol_factorize
 *   B      DEVICE memory, n x nrhs column-major, leading dimension ldb, overwritten
 *          by X (a host pointer returns -2)
 * Returns 0, -k for an invalid argument k, SPCHOL_ESTATE without a factor,
 * SPCHOL_ESCRATCH when 8 n nrhs bytes plus the task queue exceed the scratch
 * (about n * nrhs <= 3.5e6 for grid matrices), SPCHOL_ETIMEOUT, SPCHOL_ECUDA.
 * The first call on a device looks up the array's device address (a CUDA
 * runtime query, no allocation); make that first call before any stream
 * capture.  The address is kept for the life of the process (it assumes the
 * device is not reset meanwhile).  Like spchol_solve, the call returns after
 * its stream's work, and the read-back of its status, have completed.  All
 * calls share the one array: calls whose work overlaps on the GPU (different
 * streams, threads or handles at the same time) race on it and must be
 * serialised by the caller.
 */
int spchol_solve_noalloc(spchol_handle_t h, double* B, int64_t ldb, int nrhs, void* stream);

/* Copy the handle's statistics into *st. */
int spchol_stats_get(spchol_handle_t h, spchol_stats* st);

/*
 * Export the factor in CSC form (permuted ordering, diagonal first in each
 * column, amalgamation zeros dropped only if drop_zeros != 0 and they are
 * exactly zero).  Query form: with Lp/Li/Lx NULL, *nnz receives the size.
 * Host arrays: Lp int64[n+1], Li int64[*nnz], Lx double[*nnz].  perm_out
 * (host int64[n], optional) receives the permutation actually used.
 */
int spchol_export_factor(spchol_handle_t h, int64_t* nnz, int64_t* Lp, int64_t* Li, double* Lx,
                         int64_t* perm_out);

/*
 * Per-task trace of the last factorization (which = 0) or solve (which = 1),
 * recorded when spchol_options.profile = 2: out[2*i] and out[2*i+1] are the
 * device-clock start and end (ns, %globaltimer) of task i, in the task
 * numbering of the launch (factorization: diagonal tasks, then panel-solve
 * tiles, then update tiles, then subtree tasks, then the fan-in mode's gather
 * tasks; a task that never runs on its own -- a panel inside a subtree task --
 * reads 0 / 0).  Query form: out = NULL sets *count to the number of tasks.
 * Returns 0, -2 for a bad `which`, SPCHOL_ESTATE if not traced.
 */
int spchol_trace_get(spchol_handle_t h, int which, uint64_t* out, int64_t* count);

/* Release every resource of the handle.  NULL is accepted. */
int spchol_destroy(spchol_handle_t h);

/* Static, human-readable text for a return code. */
const char* spchol_strerror(int code);

/* The CUDA error name and call site of the last SPCHOL_ECUDA / SPCHOL_ENOMEM
 * returned to this host thread ("" if none).  Valid until the thread's next
 * failing call. */
const char* spchol_last_cuda_error(void);

/*
 * Batch of independent matrices factored in ONE persistent launch: the
 * matrices form the diagonal blocks of one block-diagonal system whose
 * elimination forest has one tree (or more) per matrix.
 *   count           number of matrices, >= 1                       (argument 1)
 *   n[i]            orders                                         (argument 2)
 *   colptr[i], rowind[i], perm[i] as in spchol_analyze             (arguments 3-5; perm or perm[i] may be NULL)
 *   opt, out        as in spchol_analyze                           (arguments 6-7)
 * The handle then accepts spchol_batch_factorize / spchol_batch_solve and the
 * plain spchol_stats_get / spchol_destroy.
 */
int spchol_batch_analyze(int count, const int64_t* n, const int64_t* const* colptr,
                         const int32_t* const* rowind, const int64_t* const* perm,
                         const spchol_options* opt, spchol_handle_t* out);

/* values[i]: matrix i's values, host or device, in matrix i's analyze order.  A positive
 * return k is the failing column of the block-diagonal system; spchol_batch_info maps it
 * back to (matrix, column). */
int spchol_batch_factorize(spchol_handle_t h, const double* const* values, void* stream);

/* B[i]: matrix i's right-hand sides (n[i] x nrhs[i], leading dimension ldb[i]), overwritten. */
int spchol_batch_solve(spchol_handle_t h, double* const* B, const int64_t* ldb, const int* nrhs,
                       void* stream);

/* For a positive factorize return k: which matrix failed and at which of its own
 * permuted columns (1-based).  Returns 0, or -2 if k is out of range. */
int spchol_batch_info(spchol_handle_t h, int64_t k, int* matrix, int64_t* column);

#ifdef __cplusplus
}
#endif

#endif /* SPCHOL_H */
