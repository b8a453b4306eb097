/*
 * spchol_host: the host half of spchol without a GPU, for inspection and testing.
 *
 * libspchol_host.so holds the same symbolic analysis as libspchol.so
 * (elimination tree, column counts, supernodes of Section II-B, amalgamation,
 * the width cap of Section III-B, row structures and the task graph of
 * Sections III-A / IV) and a host simulator of the task protocol.  The
 * simulator executes the factorization and solve task graphs one task at a
 * time, picking the next task uniformly at random among the ready ones
 * (Section II-C: any order that respects the dependencies is valid), with the
 * same dependency counters the GPU kernels use.  It exists to test the plan and
 * the protocol on machines without a GPU; libspchol.so never calls it.
 */
#ifndef SPCHOL_HOST_H
#define SPCHOL_HOST_H

#include <stdint.h>

#include "spchol.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spchol_plan_s* spchol_plan_t;

/* Arrays that spchol_plan_get can copy out (all converted to int64). */
enum {
  SPCHOL_PLAN_PERM = 0,      /* n: final new -> old permutation */
  SPCHOL_PLAN_COLCOUNT = 1,  /* n: exact column counts of L (diagonal included) */
  SPCHOL_PLAN_ETREE = 2,     /* n: elimination tree parent, -1 at roots */
  SPCHOL_PLAN_FCOL = 3,      /* ns+1: first column of each panel */
  SPCHOL_PLAN_NROWS = 4,     /* ns: rows of each panel (diagonal block included) */
  SPCHOL_PLAN_ROWOFF = 5,    /* ns+1: offsets into ROWS */
  SPCHOL_PLAN_ROWS = 6,      /* sum(nrows): sorted row lists */
  SPCHOL_PLAN_PARENT = 7,    /* ns: panel elimination tree, -1 at roots */
  SPCHOL_PLAN_DEPF = 8,      /* ns: update tiles targeting each panel */
  SPCHOL_PLAN_NTRSM = 9,     /* ns: panel-solve tiles per panel */
  SPCHOL_PLAN_NU = 10,       /* ns: update tiles issued by each panel */
  SPCHOL_PLAN_UTASKS = 11,   /* 6 * n_u: (s, t, seg0, seglen, row0, rowlen) per update tile */
  SPCHOL_PLAN_NST = 12,      /* ns: solve tiles per panel */
  SPCHOL_PLAN_SCALARS = 13,  /* 12: n, nnz_l, ns, factor tasks (scheduled), solve tasks, max width,
                                max rows, nnz_l_stored, n_trsm, n_u, high-priority factor tasks,
                                subtree tasks */
  SPCHOL_PLAN_ADEST = 14,    /* nnz(A): pool index of each entry of A */
  SPCHOL_PLAN_NUHI = 15,     /* ns: leading update tiles of each panel scheduled with high priority */
  SPCHOL_PLAN_SUBLO = 16,    /* subtree tasks: first panel of each (a subtree is a contiguous range) */
  SPCHOL_PLAN_SUBHI = 17,    /* subtree tasks: last panel (the subtree's root) of each */
  /* fan-in mode (options.deterministic = 2; length 0 otherwise) */
  SPCHOL_PLAN_FANOFF = 18,   /* n_u+1: offset of each update tile's private buffer (values) */
  SPCHOL_PLAN_FANTASK = 19,  /* ns+n_trsm: first row piece of each diagonal task, then of each panel-solve tile */
  SPCHOL_PLAN_FANPTR = 20,   /* pieces+1: offsets into FANENT */
  SPCHOL_PLAN_FANENT = 21    /* 3 * entries: (update tile, first row, end row) per gather-list entry */
};

/* Host-only analysis; same arguments and return codes as spchol_analyze. */
int spchol_plan_build(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm,
                      const spchol_options* opt, spchol_plan_t* out);

/* Length of array `what`, or -1 for an unknown id. */
int64_t spchol_plan_len(spchol_plan_t p, int what);

/* Copy array `what` into dst (spchol_plan_len(p, what) int64s).  Returns 0 or -2. */
int spchol_plan_get(spchol_plan_t p, int what, int64_t* dst);

/* Sum of c_j^2 over the exact column counts. */
double spchol_plan_flops(spchol_plan_t p);

/*
 * Execute the factorization task graph and then the solve task graph on the
 * host in FP64, choosing each next task uniformly at random among the ready
 * tasks with a generator seeded by `seed`.
 *   values  A's lower-CSC values in the analyze order (host)
 *   B       n x nrhs column-major (host), overwritten by X; may be NULL when nrhs = 0
 *   Lx      optional: receives the panel value pool (spchol_plan_len(p, SPCHOL_PLAN_SCALARS)
 *           does not give its size; pass NULL or a buffer of spchol_plan_pool_len(p) doubles)
 * Returns 0, k > 0 (not positive definite at permuted column k), or
 * SPCHOL_EINTERNAL if the protocol broke (a task ran twice, a counter went
 * negative, or tasks were left that never became ready).
 */
int spchol_plan_simulate(spchol_plan_t p, const double* values, double* B, int64_t ldb, int nrhs,
                         uint64_t seed, double* Lx);

/* Number of doubles in the panel value pool. */
int64_t spchol_plan_pool_len(spchol_plan_t p);

void spchol_plan_destroy(spchol_plan_t p);

#ifdef __cplusplus
}
#endif

#endif /* SPCHOL_HOST_H */
