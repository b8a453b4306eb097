// Option defaults and the mapping from spchol_options to plan parameters,
// shared by the GPU library and the host-only library.
#pragma once
#include <algorithm>
#include <cstring>

#include "../../include/spchol.h"
#include "plan.hpp"

namespace spchol {

constexpr int kSolveTileRows = 64;  // rows per solve tile below the near-root band (staged in 32-row chunks)
constexpr int kTrsmTileRows = 64;
constexpr int kFp64TcMinWidth = 16;
constexpr int kWDepth = 32;  // W panels (PlanParams::w_depth) of a single matrix, by default

inline void default_options(spchol_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->precision = SPCHOL_FP64;
  o->max_width = 64;
  o->relax_zeros = 4;
  o->tile_rows = 0;
  o->ctas_per_sm = 0;
  o->deterministic = 0;
  o->wait_budget_ns = 2000000000LL;
  o->ir_max_iter = 10;
  o->ir_tol = 1e-12;
  o->fault_inject = 0;
  o->profile = 0;
  o->solve_tile_rows = 0;
  o->sched = 0;
  o->dev_alloc = nullptr;
  o->dev_free = nullptr;
  o->alloc_ctx = nullptr;
  o->solve_w_depth = 0;
}

inline bool options_valid(const spchol_options& o) {
  const bool tc = o.precision == SPCHOL_TF32 || o.precision == SPCHOL_TF32X3 || o.precision == SPCHOL_FP64_TC;
  return o.precision >= SPCHOL_FP64 && o.precision <= SPCHOL_FP64_TC && o.max_width >= 1 &&
         o.max_width <= (tc ? 64 : 128) &&
         o.relax_zeros >= 0 && o.wait_budget_ns > 0 && o.ir_max_iter >= 0 && o.tile_rows >= 0 && o.tile_rows <= 64 &&
         o.ctas_per_sm >= 0 && o.fault_inject >= 0 && o.fault_inject <= 1 && o.deterministic >= 0 &&
         o.deterministic <= 2 &&
         o.profile >= 0 && o.profile <= 2 && o.sched >= 0 && o.sched <= 1 &&
         (o.solve_tile_rows == 0 || (o.solve_tile_rows >= 8 && o.solve_tile_rows <= 256)) &&
         (o.dev_alloc == nullptr) == (o.dev_free == nullptr) && o.solve_w_depth >= -1;
}

inline PlanParams params_from(const spchol_options& o) {
  PlanParams p;
  p.max_width = std::min(std::max(o.max_width, 1), 128);
  p.relax_zeros = std::max(o.relax_zeros, 0);
  p.tile_rows = o.tile_rows > 0 ? o.tile_rows : 64;
  if (o.precision == SPCHOL_TF32 || o.precision == SPCHOL_TF32X3) p.tc_min_width = 1;  // every tile on TF32
  if (o.precision == SPCHOL_FP64_TC) {
    // panels of at least 16 columns carry almost all update work and go to the
    // tensor cores (measured on the 64^3 Laplacian: 201 ms against 210 ms with
    // 32); narrower ones keep DFMA tiles, whose cost scales with size
    p.tc_min_width = kFp64TcMinWidth;
    p.tc_tile_rows = 64;  // the BF16-split tile keeps 64 rows of digits in shared memory
    p.slice_fp64 = true;
  }
  p.trsm_rows = kTrsmTileRows;
  p.fifo = o.sched == 1;
  p.solve_rows = o.solve_tile_rows > 0 ? o.solve_tile_rows : kSolveTileRows;
  p.w_depth = o.solve_w_depth > 0 ? o.solve_w_depth : o.solve_w_depth == 0 ? kWDepth : 0;
  if (o.deterministic) {
    p.deterministic = true;
    p.fanin = o.deterministic == 2;
    p.subtree_flops = 0.0;
    p.w_depth = 0;  // the solves keep the chains of diagonal tasks and tiles
  }
  return p;
}

}  // namespace spchol
