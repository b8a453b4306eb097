// Argument blocks and host launchers of the device kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "plan.hpp"

namespace spchol {

constexpr int kFactorThreads = 256;
constexpr int kSolveThreads = 256;
constexpr int kUpdTileM = 64;   // rows of C per update-tile pass (matches the 16x16 thread grid x 4)
constexpr int kUpdTileN = 64;   // columns of C per pass
constexpr int kUpdKC = 16;      // k-chunk staged in shared memory
// TMA box of an update-tile operand chunk: rows (tile rows + the alignment
// slack of one 16-byte piece) x kUpdKC columns, per element size
constexpr int kUpdBoxRows(int elem_bytes) { return kUpdTileM + 16 / elem_bytes; }
constexpr int kSolveNRC = 8;    // right-hand sides per pass

// Panel structure (device pointers).
struct PanelView {
  int32_t ns;
  const int32_t* fcol;
  const int32_t* nrows;
  const int32_t* ld;
  const int64_t* rowoff;
  const int32_t* rows;
  const int64_t* valoff;
  const int32_t* parent;
};

// Fan-in mode: one gather-list entry as the gather reads it, built on the
// device at analysis from the list entry (FanEnt), its tile and the buffer
// offsets: the buffer offset of its first listed row, the offset of that
// row's relative index, the offset of its segment's row numbers (into the row
// lists), the buffer's rows, and the listed rows and segment columns.
struct FanRec {
  int64_t fo, rp, rs;
  int32_t rowlen;
  int16_t ni, seglen;
};

struct FactorArgs {
  PanelView pv;
  const int32_t* trsm_first;
  const int32_t* ntrsm;
  const int32_t* trsm_sn;
  const int32_t* trsm_rows_of;  // rows per panel-solve tile, per panel
  const int32_t* u_first;
  const int32_t* nu;
  const UTask* ut;
  const int32_t* relpos;  // relative row indices of the update tiles (UTask::rel)
  const unsigned char* tmaps;  // optional: one 128-byte TMA tensor map per panel (2-D view, see kUpdBox*)
  const int32_t* nu_hi;  // leading update tiles of each panel that go to the high-priority ring
  const int32_t* sub_lo;  // subtree tasks: first and last panel of each
  const int32_t* sub_hi;
  // subtree tasks run by single warps before the task loop (Plan::wsub; FP64
  // DFMA mode only, n_wsub = 0 otherwise); they are not seeded in the rings
  const int32_t* wsub;
  int32_t n_wsub;
  int32_t n_trsm, n_u, ntask, trsm_rows;
  int32_t n_hi;          // high-priority ring size: ring[0, n_hi); the other ring is ring[n_hi, ntask)
  int32_t mma_mode;    // FP32 panels: 0 FFMA update tiles, 1 TF32 tensor cores, 2 split-TF32 (3 products);
                       // FP64 panels: 0 DFMA update tiles, 3 BF16 tensor cores on 7-way split operands
  uint16_t* slices;    // mode 3: BF16 slices of the rows below each diagonal block
  const int64_t* sliceoff;
  int32_t* rexp;       // mode 3: row exponent of every panel row (indexed like rows)
  int32_t tc_min_width;  // mode 3: update tiles of panels at least this wide run on the tensor cores
  int32_t* dep_f;      // update tiles still to land in each panel
  int32_t* trsm_left;  // panel-solve tiles still to finish in each panel
  // deterministic order (null otherwise): next update tile into the same
  // target (-1 at the end) and each tile's live counter (its source's
  // panel-solve tiles + its predecessor)
  const int32_t* u_next;
  int32_t* u_dep;
  // fan-in mode (null otherwise, see Plan::fan_ptr): the update tiles' private
  // buffers (panel type), each tile's offset in them, the first piece of each
  // diagonal / panel-solve task, the pieces' gather lists, and how many values
  // one gather batch stages in shared memory
  void* fan_buf;
  const int64_t* fan_off;
  const int32_t* fan_task;
  const int64_t* fan_ptr;
  const FanRec* fan_rec;
  int32_t fan_cap;
  // its gather tasks (Plan::gat_first): ids gat0 + g (INT32_MAX: none), each
  // panel's range, their pieces, the pieces' owners, the diagonal tasks'
  // initial and live gather counts and the panel-solve tiles' live counters
  int32_t gat0;
  const int32_t* gat_first;
  const int32_t* gat_pc;
  const int32_t* pc_owner;
  const int32_t* gdiag0;
  int32_t* gdiag;
  int32_t* tdep;
  int* ring;
  int* ctrl;
  int64_t budget_ns;
  void* pool;          // double* or float*
  double* inv;         // per panel: L11^{-1} (w x w, column-major, lower part)
  const int64_t* invoff;
  void* wbuf;              // W = L21 L11^{-1} of the W panels (Plan::woff), double* or float*
  const int64_t* woff;     // null: no W panels
  unsigned long long* prof;  // optional: [0..2] busy ns per task type, [3] wait ns, [4..6] counts,
                             // [7] tensor-core update ns, [8] subtree-task ns, [9] subtree tasks,
                             // [10..12] fan-in gather ns (batch cuts, staging, adding), [13] its
                             // batches, [14] its tiles
  unsigned long long* trace; // optional: per task id, start and end ns
};

struct SolveArgs {
  PanelView pv;
  const int32_t* kid_ptr;
  const int32_t* kids;
  const int32_t* st_first;
  const int32_t* nst;
  const int32_t* st_sn;
  int32_t n_st, ntask;
  const int32_t* st_rows;  // solve tile rows per panel
  int32_t n_hi;            // tasks made ready by other tasks: ring[0, n_hi); the seeds: ring[n_hi, ntask)
  const int32_t* st_tptr;  // solve tile -> panels its rows fall in (CSR)
  const int32_t* st_tgt;
  const int32_t* rt_ptr;   // panel -> solve tiles whose rows fall in it (CSR)
  const int32_t* rt_tile;
  int32_t* fdep;    // forward tiles still to land in each panel's rows
  int32_t* bdep;    // per tile: target panels not yet back-solved, + 1 until its panel's forward tiles are done
  int32_t* ftiles;  // forward tiles left per panel
  int32_t* btiles;  // backward tiles left per panel
  int* ring;
  int* ctrl;
  int64_t budget_ns;
  const void* pool;
  const double* inv;     // per panel: L11^{-1}
  const int64_t* invoff;
  const void* wbuf;      // W = L21 L11^{-1} of the W panels (Plan::woff)
  const int64_t* woff;   // null: no W panels
  int32_t n_wpan;        // W panels: their backward diagonal tasks never run
  // The subtree tasks the factorization ran on single warps (FactorArgs::wsub),
  // solved by single warps too: their forward solves in a launch before the
  // task loop, their backward solves in one after it (subtree_solve_kernel).
  // ntask_done: the tasks completed when the task loop may end (its own and
  // the forward subtrees).
  const int32_t* sub_lo;
  const int32_t* sub_hi;
  const int32_t* wsub;
  int32_t n_wsub;
  int32_t ntask_done;
  double* Y;        // n x nrhs, permuted order
  int64_t ldy;
  int nrhs;
  int tc_tiles;     // 1: FP64 panel tiles 16..64 wide as split products on the tensor cores (FP64_TC mode)
  // deterministic order (null otherwise): each forward tile's successors in the
  // chains of its target panels (CSR) and the live counters (own diagonal
  // solve + predecessors); the backward tiles of a panel chain in tile order
  // through bdep
  const int32_t* ft_sptr;
  const int32_t* ft_succ;
  int32_t* ftdep;
  // fan-in mode (null otherwise, see Plan::st_zf): the tiles' forward and
  // backward buffers (nrhs columns each), their offsets, and the records of
  // each panel's forward gather list
  double* zf;
  double* zb;
  const int64_t* st_zf;
  const int64_t* st_zb;
  const Plan::SolveFanRec* rt_rec;
  unsigned long long* prof;  // optional: [0..3] busy ns per task type, [4] wait ns
  unsigned long long* trace; // optional: per task id, start and end ns
};

// factor.cu
size_t factor_smem_bytes(int max_w, int mma_mode);
size_t warp_subtree_smem_bytes();  // shared memory of a CTA of the warp-level subtree tasks
cudaError_t warp_subtree_configure(bool fp32, int* blocks_per_sm);
cudaError_t launch_warp_subtrees(bool fp32, const FactorArgs& a, int grid, cudaStream_t st);
// Fan-in mode: shared memory a gather needs for panels up to max_w wide, and
// the values it stages per batch (*cap).
size_t fanin_smem_bytes(int max_w, bool fp32, int* cap);
cudaError_t factor_configure(bool fp32, int mma_mode, bool fanin, size_t smem, int* blocks_per_sm);
cudaError_t launch_assemble(bool fp32, const double* values, const int64_t* dest, int64_t nnz,
                            void* pool, cudaStream_t st);
cudaError_t launch_factor(bool fp32, const FactorArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_fanrec(const FanEnt* ent, int64_t n, const UTask* ut, const int64_t* fan_off,
                          const int64_t* rowoff, FanRec* rec, cudaStream_t st);

// solve.cu
size_t solve_smem_bytes(int max_w, bool tc_tiles, bool fanin);
cudaError_t solve_configure(bool fp32, bool fanin, bool tc_tiles, size_t smem, int* blocks_per_sm);
cudaError_t launch_solve(bool fp32, const SolveArgs& a, int grid, size_t smem, cudaStream_t st);
// the forward (before the task loop) or backward (after it) solves of the
// subtree tasks run by single warps (SolveArgs::wsub)
cudaError_t launch_subtree_solve(bool fp32, bool forward, const SolveArgs& a, int grid, cudaStream_t st);
cudaError_t launch_permute_in(const double* B, int64_t ldb, double* Y, int64_t ldy, const int32_t* perm,
                              int64_t n, int nrhs, cudaStream_t st);
cudaError_t launch_permute_out(const double* Y, int64_t ldy, double* B, int64_t ldb, const int32_t* perm,
                               int64_t n, int nrhs, cudaStream_t st);

// Fixed device scratch of spchol_solve_noalloc (solve.cu): 32 MiB.
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
cudaError_t noalloc_scratch(int device, void** ptr);

// mixed.cu
cudaError_t launch_residual(int64_t n, int nrhs, const int64_t* rp, const int32_t* ci, const int64_t* vmap,
                            const double* aval, const double* X, int64_t ldx, const double* B, int64_t ldb, double* R,
                            int64_t ldr, unsigned long long* colmax, cudaStream_t st);
cudaError_t launch_anorm(int64_t n, const int64_t* rp, const int64_t* vmap, const double* aval,
                         unsigned long long* out, cudaStream_t st);
cudaError_t launch_correct(const double* Y, int64_t ldy, double* X, int64_t ldx, const int32_t* perm, int64_t n,
                           int nrhs, cudaStream_t st);
// GMRES-IR: y = A x; out[j] = V_j . z (j < k, fixed-order reductions; partial
// holds kGmresBlocks * k doubles); z += alpha V h; y = alpha x.
constexpr int kGmresThreads = 256, kGmresBlocks = 304;
constexpr int kGmresRestart = 30;  // Krylov vectors per GMRES cycle
cudaError_t launch_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const int64_t* vmap, const double* aval,
                        const double* x, double* y, cudaStream_t st);
cudaError_t launch_dots(int64_t n, int k, const double* V, int64_t ldv, const double* z, double* partial,
                        double* out, cudaStream_t st);
cudaError_t launch_axpy_multi(int64_t n, int k, const double* V, int64_t ldv, const double* h, double alpha, double* z,
                              cudaStream_t st);
cudaError_t launch_scale(int64_t n, double alpha, const double* x, double* y, cudaStream_t st);

// sched.cu
cudaError_t launch_relpos(const UTask* ut, int n_u, const int32_t* rows, const int64_t* rowoff,
                          const int32_t* nrows, int32_t* relpos, cudaStream_t st);
cudaError_t launch_ring_reset(int* slots, int ntask, const int* seeds, int nseed, int* ctrl, int* c0,
                              const int* c0_init, int n0, int* c1, const int* c1_init, int n1, int* c2,
                              const int* c2_init, int n2, cudaStream_t st, int* c3 = nullptr,
                              const int* c3_init = nullptr, int n3 = 0, int seeds_hi = 0, int seed_off = 0);

}  // namespace spchol
