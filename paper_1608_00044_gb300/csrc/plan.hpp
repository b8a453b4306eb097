// Host-side analysis result: supernode partition, row structures, storage
// layout and the task graph of the factorization and the solves.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace spchol {

// FP64 tensor-core mode: every FP64 value of L below a diagonal block is split
// into this many 8-bit slices relative to its row's largest magnitude.
constexpr int kSlices = 7;
constexpr int kSliceBits = 8;

// One update tile U(s, t): rows [row0, row0 + rowlen) of source panel s (indices
// into s's row list) times the rows [seg0, seg0 + seglen) of s that fall inside
// target panel t's columns (Section III-A, task U; Section IV, task T_{s,t}).
struct UTask {
  int32_t s, t, seg0, seglen, row0, rowlen;
  int64_t rel;  // offset of the tile's relative row indices (rowlen of them) in the relative-index array
};

struct PlanParams {
  int max_width = 64;    // W (Section III-B caps supernodes at 150 columns)
  int relax_zeros = 4;   // amalgamation budget per column
  int tile_rows = 64;    // rows per update tile
  int trsm_rows = 128;   // rows per panel-solve tile
  int solve_rows = 128;  // rows per triangular-solve tile
  // Panels within top_depth of the root of the panel etree (the chains of the
  // top separators: the critical path) get smaller tiles, so that each step of
  // the chain spreads over more CTAs.
  int top_depth = 128;
  int top_tile_rows = 16;
  int top_trsm_rows = 16;
  int top_solve_rows = 32;  // rows per triangular-solve tile of those panels
  // Tensor-core update tiles: source panels at least tc_min_width wide (0 =
  // none) use tc_tile_rows-row tiles (one MMA M-tile) on the tensor cores.
  int tc_min_width = 0;
  int tc_tile_rows = 128;
  bool slice_fp64 = false;  // FP64 tensor-core mode: split those panels into BF16 digits
  // Subtree tasks: a maximal subtree of the panel etree whose factorization
  // costs at most min(subtree_flops, total flops / 4096) runs as one task
  // (0: none).
  double subtree_flops = 1e6;
  // Deterministic order (the static (target, source) order of Section IV-B):
  // see Plan::u_next.  Subtree tasks are off in this mode.
  bool deterministic = false;
  // Deterministic by fan-in aggregation (the fan-in family of Section II-C, restated
  // for one GPU) instead of the chains: see Plan::fan_ptr.  Implies
  // deterministic (the solves keep their chains).
  bool fanin = false;
  // One FIFO ready ring instead of the two priority rings (spchol_options.sched
  // = 1): the launch gives the high-priority ring no slots, and every push goes
  // to the other ring.  The plan itself is the same.
  bool fifo = false;
  // Panels within w_depth of the root of the panel etree (0: none), outside
  // subtree tasks, at most kWMaxWidth wide and with rows below their diagonal
  // block, also keep W = L21 L11^{-1} (Plan::woff), so that their solve steps
  // need no diagonal task on the chain: see Plan::woff.
  int w_depth = 0;
};

// Widest panel of a subtree task that runs on one warp (Plan::wsub).
constexpr int kWarpSubW = 32;

// Widest panel that keeps W = L21 L11^{-1} (its packed inverse is staged in
// shared memory by the panel-solve tiles that form W).
constexpr int kWMaxWidth = 64;

// Rows of a target panel are gathered in pieces of at most this many rows.
constexpr int kFanPieceRows = 32;

// One entry of a fan-in gather list: rows [i0, i1) of update tile u fall in the
// piece that owns the list.
struct FanEnt {
  int32_t u;
  int16_t i0, i1;
};

struct Plan {
  int64_t n = 0;
  int64_t nnz_a = 0;
  std::vector<int64_t> perm;  // final new -> old (input perm refined by a postorder)
  std::vector<int64_t> pinv;  // old -> new

  // exact structure (before amalgamation)
  int64_t nnz_l = 0;
  double flops = 0.0;  // sum of c_j^2
  std::vector<int64_t> colcount;
  std::vector<int32_t> etree;

  // panels (supernodes after amalgamation and the width cap)
  int32_t ns = 0;
  std::vector<int32_t> fcol;    // ns + 1
  std::vector<int32_t> nrows;   // rows incl. the diagonal block
  std::vector<int32_t> ld;      // leading dimension (nrows rounded up to 4)
  std::vector<int64_t> rowoff;  // ns + 1, into rows
  std::vector<int32_t> rows;    // concatenated sorted row lists
  std::vector<int64_t> valoff;  // ns + 1, into the value pool (elements)
  std::vector<int64_t> invoff;  // ns + 1, into the diagonal-block inverse buffer (w x w per panel)
  std::vector<int64_t> sliceoff;  // ns + 1, into the BF16 slice buffer (FP64 tensor-core mode)
  std::vector<int32_t> parent;  // panel etree, -1 at roots
  std::vector<int32_t> snode_of;  // column -> panel
  std::vector<int64_t> a_dest;  // entry e of A's lower CSC -> pool index
  int64_t nnz_l_stored = 0;
  int32_t max_w = 0, max_r = 0;

  // factorization tasks: [0, ns) diagonal factor, then panel-solve tiles, then updates
  std::vector<int32_t> trsm_first, ntrsm, trsm_sn, trsm_rows;  // trsm_rows: tile rows per panel
  std::vector<int32_t> u_first, nu;
  std::vector<UTask> ut;
  std::vector<int32_t> dep_f;  // update tiles targeting each panel
  int64_t n_rel = 0;           // relative row indices of all update tiles (sum of rowlen)
  // Scheduling priority: diagonal and panel-solve tasks, and the first nu_hi[s]
  // update tiles of panel s (those into its etree parent, for panels within
  // top_depth of the root), go to the high-priority ready ring; n_hi_tasks of
  // them in all.  The remaining update tiles go to the other ring.
  std::vector<int32_t> nu_hi;
  // Subtree tasks: task ns + n_trsm + n_u + k factors panels sub_lo[k] ..
  // sub_hi[k] (a whole subtree: panels are numbered in postorder) in order in
  // one CTA; the panel-level tasks of those panels are never scheduled.
  // in_sub[s]: the subtree task of panel s, or -1.
  std::vector<int32_t> sub_lo, sub_hi, in_sub;
  // The subtree tasks whose panels are all at most kWarpSubW columns wide:
  // the FP64 factorization runs each of them on one warp (see wsub in
  // FactorArgs), several side by side in a CTA.
  std::vector<int32_t> wsub;
  double sub_work_frac = 0.0;  // the subtree tasks' share of the factorization's work
  int32_t n_trsm = 0, n_u = 0, n_sub = 0;
  int32_t n_task_ids = 0;      // size of the task id space: ns + n_trsm + n_u + n_sub
  int32_t n_factor_tasks = 0;  // tasks that are scheduled (pushed to a ring) in one factorization
  int32_t n_hi_tasks = 0;

  // solve tasks
  std::vector<int32_t> st_first, nst, st_sn, st_rows;  // st_rows: solve tile rows per panel
  std::vector<int32_t> kid_ptr, kids;  // panel children, CSR
  // precise solve dependencies: the panels whose columns each solve tile's rows
  // fall in (tile -> targets, CSR), the same relation reversed (panel -> tiles),
  // forward counters (tiles touching each panel) and backward tile counters
  // (targets + 1 for "every forward tile of the tile's own panel is done")
  std::vector<int32_t> st_tptr, st_tgt, rt_ptr, rt_tile, fdep0, bdep0;
  int32_t n_st = 0, n_solve_tasks = 0;
  // W panels (PlanParams::w_depth): woff[s] >= 0 is the offset (elements) of
  // panel s's W = L21 L11^{-1} in the W buffer, stored like the panel itself
  // (column-major, leading dimension ld[s], rows w .. nrows-1 used); -1 for the
  // other panels.  The panel-solve tiles of the factorization write W after
  // their L21 rows.  The solves then take, for a W panel s, b_s = the
  // right-hand side rows of s once every forward tile into s has landed:
  //   forward tile k:  y[rows of k] -= W[k] b_s   (ready with b_s, no diagonal task first)
  //   diagonal task:   y_s <- L11^{-T} L11^{-1} b_s, after every forward tile of s has read b_s
  //   backward tile k: y_s -= W[k]^T x[rows of k], after the diagonal task
  // and x_s = y_s once the backward tiles are done (the last one releases the
  // dependents, the role of the backward diagonal task, which never runs):
  // x_s = L11^{-T} (L11^{-1} b_s - L21^T x_below) = A11^{-1} b_s - W^T x_below.
  std::vector<int64_t> woff;
  int64_t n_w = 0;      // elements of the W buffer
  int32_t n_wpan = 0;   // W panels (backward diagonal tasks that never run)

  // Deterministic order (params.deterministic; empty otherwise).  The update
  // tiles into each target panel form a chain in (source panel, row tile)
  // order, and a tile becomes ready only when its source's panel-solve tiles
  // and its predecessor in the chain are done, so the scatter-adds into every
  // entry land in one fixed order: u_next (next tile into the same target, -1
  // at the end) and u_dep0 (1 + 1 with a predecessor).  Likewise the forward
  // solve tiles that subtract from each panel's rows chain in tile order
  // (ft_sptr / ft_succ: each tile's successors, one per target panel chain;
  // ft_dep0: 1 for its panel's diagonal solve + its predecessors), and the
  // backward tiles of a panel, which all subtract from that panel's entries,
  // chain in tile order (bdep0 counts the predecessor).
  std::vector<int32_t> u_next, u_dep0, ft_sptr, ft_succ, ft_dep0;

  // Fan-in aggregation (params.fanin; empty otherwise).  Update tile u stores
  // its product, negated, densely (column-major, rowlen rows, seglen columns,
  // lower entries only) at fan_off[u] of a private buffer instead of adding
  // it into the target.  The rows of each target panel are split into pieces:
  // the diagonal block in steps of kFanPieceRows rows, then each panel-solve
  // tile's rows in such steps.  fan_task[k] (k < ns: the diagonal task of
  // panel k; k >= ns: panel-solve tile k - ns) is the first piece of that
  // task's rows, whose pieces are consecutive; fan_ptr / fan_ent list, for
  // every piece in update-tile order, the tiles with rows in it and which.
  // The task that owns a piece adds those buffers into its rows in list
  // order before it factors or solves them, so every entry of L receives
  // its updates in one fixed order, and the update tiles themselves need no
  // order among them.
  std::vector<int64_t> fan_off;   // n_u + 1
  std::vector<int32_t> fan_task;  // ns + n_trsm
  std::vector<int64_t> fan_ptr;   // pieces + 1
  std::vector<FanEnt> fan_ent;
  // The solves of the fan-in mode: forward tile k stores its product (its
  // rows x nrhs, negated) at st_zf[k] * nrhs of one buffer and backward tile k
  // its product (its panel's width x nrhs) at st_zb[k] * nrhs of another,
  // instead of adding them into the right-hand sides.  A panel's forward
  // diagonal task adds the forward buffers of the tiles with rows in its
  // columns first, in tile order (its rt_tile list read from the end; rt_rng:
  // those rows of the tile, i0 | i1 << 16; st_roff: the tile's first row in
  // the row lists), and its backward diagonal task adds its own tiles'
  // backward buffers in tile order: every entry of the solution receives its
  // updates in one fixed order -- the order of the static chains.
  // Gather tasks (fan-in mode): one per row piece that receives updates, task
  // id ns + n_trsm + n_u + n_sub + g for g in [gat_first[t], gat_first[t + 1])
  // of panel t, piece gat_pc[g], all made ready when the panel's last update
  // tile lands.  pc_owner[piece]: the task whose rows it holds (t: the
  // diagonal task, ns + k: panel-solve tile k).  The diagonal task waits for
  // its gathers (gdiag0[t] of them; none: it is ready with the updates), each
  // panel-solve tile for the diagonal task and its own gathers (tdep0[k]).
  std::vector<int32_t> gat_first, gat_pc, pc_owner, gdiag0, tdep0;
  int32_t n_gat = 0;
  std::vector<int64_t> st_zf, st_zb;  // n_st + 1
  // the forward gather's record of each rt_tile entry: the tile's buffer (in
  // rows: st_zf), its first listed row's place in the row lists, the tile's
  // rows, its first listed row and how many are listed
  struct SolveFanRec {
    int64_t z, ro;
    int32_t cnt;
    int16_t i0, ni;
  };
  std::vector<SolveFanRec> rt_rec;
  std::vector<int64_t> st_roff;       // n_st
  std::vector<int32_t> rt_rng;        // like rt_tile

  PlanParams params;
};

// Validation error: argument index (1-based) and message.
struct PlanError {
  int arg = 0;
  std::string msg;
};

// Builds the plan.  Returns 0, or -k with err filled for an invalid argument k
// (1 n, 2 colptr, 3 rowind, 4 perm).
int build_plan(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm,
               const PlanParams& params, Plan& plan, PlanError& err);

}  // namespace spchol
