// Host-only plan inspection and task-protocol simulator (include/spchol_host.h).
//
// The simulator runs the same task graph as the persistent GPU kernels, with
// the same dependency counters, one task at a time in a seeded random order
// among the ready tasks.  Task semantics mirror the kernels: POTRF on the
// diagonal block, row-tile forward substitution for L21, update tiles
// scatter-subtracted at relative positions found by binary search, and the
// forward / backward solve tiles.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/spchol_host.h"
#include "options.hpp"
#include "plan.hpp"

using namespace spchol;

struct spchol_plan_s {
  Plan plan;
};

namespace {

struct Rng {
  uint64_t s;
  uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  size_t pick(size_t n) { return (size_t)(next() % n); }
};

// Ready list with random extraction (the order of a parallel run is arbitrary).
struct Ready {
  std::vector<int> v;
  void push(int t) { v.push_back(t); }
  bool empty() const { return v.empty(); }
  int pop(Rng& r) {
    size_t i = r.pick(v.size());
    int t = v[i];
    v[i] = v.back();
    v.pop_back();
    return t;
  }
};

struct Sim {
  const Plan& P;
  std::vector<double> pool;
  std::vector<double> fan;  // fan-in mode: the update tiles' private buffers
  int info = 0;
  explicit Sim(const Plan& p)
      : P(p), pool((size_t)p.valoff[p.ns], 0.0), fan(p.fan_off.empty() ? 0 : (size_t)p.fan_off.back(), 0.0) {}
  double* panel(int s) { return pool.data() + P.valoff[s]; }
  int width(int s) const { return P.fcol[s + 1] - P.fcol[s]; }

  // Fan-in mode: add the buffered updates into rows [r0, r1) of panel t, whose
  // pieces start at piece pc0, in the lists' order.
  void gather(int t, int pc0, int r0, int r1) {
    const int ft = P.fcol[t], ldt = P.ld[t], rt = P.nrows[t];
    const int32_t* Rt = P.rows.data() + P.rowoff[t];
    double* T = panel(t);
    for (int pc = pc0, p0 = r0; p0 < r1; ++pc, p0 += kFanPieceRows) {
      const int p1 = std::min(r1, p0 + kFanPieceRows);
      for (int64_t e = P.fan_ptr[pc]; e < P.fan_ptr[pc + 1]; ++e) {
        const FanEnt& fe = P.fan_ent[e];
        const UTask& u = P.ut[fe.u];
        const int32_t* Rs = P.rows.data() + P.rowoff[u.s];
        const double* F = fan.data() + P.fan_off[fe.u];
        if (u.t != t || fe.i0 < 0 || fe.i0 >= fe.i1 || fe.i1 > u.rowlen) {
          info = -1;  // inconsistent list
          return;
        }
        for (int i = fe.i0; i < fe.i1; ++i) {
          const int gi = Rs[u.row0 + i];
          const int pos = (int)(std::lower_bound(Rt, Rt + rt, gi) - Rt);
          if (pos < p0 || pos >= p1 || Rt[pos] != gi) {
            info = -1;  // the row is not in this piece
            return;
          }
          for (int j = 0; j < u.seglen; ++j) {
            const int gj = Rs[u.seg0 + j];
            if (gi >= gj) T[pos + (size_t)(gj - ft) * ldt] += F[i + (size_t)j * u.rowlen];
          }
        }
      }
    }
  }

  void potrf(int s) {
    const int w = width(s), ld = P.ld[s], f = P.fcol[s];
    double* A = panel(s);
    for (int j = 0; j < w; ++j) {
      double d = A[j + (size_t)j * ld];
      if (!(d > 0.0)) {
        if (info == 0 || f + j + 1 < info) info = f + j + 1;
        return;
      }
      const double ljj = std::sqrt(d);
      A[j + (size_t)j * ld] = ljj;
      for (int i = j + 1; i < w; ++i) A[i + (size_t)j * ld] = A[i + (size_t)j * ld] / ljj;
      for (int k = j + 1; k < w; ++k)
        for (int i = k; i < w; ++i) A[i + (size_t)k * ld] -= A[i + (size_t)j * ld] * A[k + (size_t)j * ld];
    }
  }
  void trsm(int s, int k) {
    const int w = width(s), ld = P.ld[s], r = P.nrows[s];
    const int row0 = w + k * P.trsm_rows[s], cnt = std::min(P.trsm_rows[s], r - row0);
    double* A = panel(s);
    for (int i = row0; i < row0 + cnt; ++i)
      for (int j = 0; j < w; ++j) {
        double x = A[i + (size_t)j * ld];
        for (int c = 0; c < j; ++c) x -= A[i + (size_t)c * ld] * A[j + (size_t)c * ld];
        A[i + (size_t)j * ld] = x / A[j + (size_t)j * ld];
      }
  }
  void update(const UTask& u, int ui) {
    double* F = P.params.fanin ? fan.data() + P.fan_off[ui] : nullptr;
    const int ws = width(u.s), lds = P.ld[u.s], ldt = P.ld[u.t], ft = P.fcol[u.t], rt = P.nrows[u.t];
    const int32_t* Rs = P.rows.data() + P.rowoff[u.s];
    const int32_t* Rt = P.rows.data() + P.rowoff[u.t];
    const double* S = panel(u.s);
    double* T = panel(u.t);
    for (int i = 0; i < u.rowlen; ++i) {
      const int gi = Rs[u.row0 + i];
      const int pos = (int)(std::lower_bound(Rt, Rt + rt, gi) - Rt);
      if (pos >= rt || Rt[pos] != gi) {
        info = -1;  // relative index missing: broken plan
        return;
      }
      for (int j = 0; j < u.seglen; ++j) {
        const int gj = Rs[u.seg0 + j];
        if (gi < gj) continue;
        double c = 0.0;
        for (int k = 0; k < ws; ++k) c += S[(u.row0 + i) + (size_t)k * lds] * S[(u.seg0 + j) + (size_t)k * lds];
        if (F)
          F[i + (size_t)j * u.rowlen] = -c;  // fan-in: the tile's private buffer
        else
          T[pos + (size_t)(gj - ft) * ldt] -= c;
      }
    }
  }
};

}  // namespace

extern "C" {

int spchol_plan_build(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm,
                      const spchol_options* opt, spchol_plan_t* out) {
  if (!out) return -6;
  *out = nullptr;
  spchol_options o;
  if (opt) {
    o = *opt;
    if (!options_valid(o)) return -5;
  } else {
    spchol::default_options(&o);
  }
  spchol_plan_t p = new (std::nothrow) spchol_plan_s();
  if (!p) return SPCHOL_ENOMEM;
  PlanError err;
  int rc = build_plan(n, colptr, rowind, perm, params_from(o), p->plan, err);
  if (rc) {
    delete p;
    return rc;
  }
  *out = p;
  return 0;
}

int64_t spchol_plan_len(spchol_plan_t p, int what) {
  if (!p) return -1;
  const Plan& P = p->plan;
  switch (what) {
    case SPCHOL_PLAN_PERM: case SPCHOL_PLAN_COLCOUNT: case SPCHOL_PLAN_ETREE: return P.n;
    case SPCHOL_PLAN_FCOL: case SPCHOL_PLAN_ROWOFF: return P.ns + 1;
    case SPCHOL_PLAN_NROWS: case SPCHOL_PLAN_PARENT: case SPCHOL_PLAN_DEPF: case SPCHOL_PLAN_NTRSM:
    case SPCHOL_PLAN_NU: case SPCHOL_PLAN_NST: case SPCHOL_PLAN_NUHI: return P.ns;
    case SPCHOL_PLAN_ROWS: return (int64_t)P.rows.size();
    case SPCHOL_PLAN_UTASKS: return 6 * (int64_t)P.ut.size();
    case SPCHOL_PLAN_SCALARS: return 12;
    case SPCHOL_PLAN_SUBLO: case SPCHOL_PLAN_SUBHI: return (int64_t)P.sub_lo.size();
    case SPCHOL_PLAN_ADEST: return (int64_t)P.a_dest.size();
    case SPCHOL_PLAN_FANOFF: return (int64_t)P.fan_off.size();
    case SPCHOL_PLAN_FANTASK: return (int64_t)P.fan_task.size();
    case SPCHOL_PLAN_FANPTR: return (int64_t)P.fan_ptr.size();
    case SPCHOL_PLAN_FANENT: return 3 * (int64_t)P.fan_ent.size();
    default: return -1;
  }
}

int spchol_plan_get(spchol_plan_t p, int what, int64_t* dst) {
  if (!p) return -1;
  if (!dst) return -3;
  const Plan& P = p->plan;
  auto cp = [&](const auto& v) {
    for (size_t i = 0; i < v.size(); ++i) dst[i] = (int64_t)v[i];
  };
  switch (what) {
    case SPCHOL_PLAN_PERM: cp(P.perm); break;
    case SPCHOL_PLAN_COLCOUNT: cp(P.colcount); break;
    case SPCHOL_PLAN_ETREE: cp(P.etree); break;
    case SPCHOL_PLAN_FCOL: cp(P.fcol); break;
    case SPCHOL_PLAN_NROWS: cp(P.nrows); break;
    case SPCHOL_PLAN_ROWOFF: cp(P.rowoff); break;
    case SPCHOL_PLAN_ROWS: cp(P.rows); break;
    case SPCHOL_PLAN_PARENT: cp(P.parent); break;
    case SPCHOL_PLAN_DEPF: cp(P.dep_f); break;
    case SPCHOL_PLAN_NTRSM: cp(P.ntrsm); break;
    case SPCHOL_PLAN_NU: cp(P.nu); break;
    case SPCHOL_PLAN_NST: cp(P.nst); break;
    case SPCHOL_PLAN_NUHI: cp(P.nu_hi); break;
    case SPCHOL_PLAN_SUBLO: cp(P.sub_lo); break;
    case SPCHOL_PLAN_SUBHI: cp(P.sub_hi); break;
    case SPCHOL_PLAN_ADEST: cp(P.a_dest); break;
    case SPCHOL_PLAN_FANOFF: cp(P.fan_off); break;
    case SPCHOL_PLAN_FANTASK: cp(P.fan_task); break;
    case SPCHOL_PLAN_FANPTR: cp(P.fan_ptr); break;
    case SPCHOL_PLAN_FANENT:
      for (size_t i = 0; i < P.fan_ent.size(); ++i) {
        dst[3 * i] = P.fan_ent[i].u;
        dst[3 * i + 1] = P.fan_ent[i].i0;
        dst[3 * i + 2] = P.fan_ent[i].i1;
      }
      break;
    case SPCHOL_PLAN_UTASKS:
      for (size_t i = 0; i < P.ut.size(); ++i) {
        const UTask& u = P.ut[i];
        int64_t* d = dst + 6 * i;
        d[0] = u.s; d[1] = u.t; d[2] = u.seg0; d[3] = u.seglen; d[4] = u.row0; d[5] = u.rowlen;
      }
      break;
    case SPCHOL_PLAN_SCALARS:
      dst[0] = P.n; dst[1] = P.nnz_l; dst[2] = P.ns; dst[3] = P.n_factor_tasks; dst[4] = P.n_solve_tasks;
      dst[5] = P.max_w; dst[6] = P.max_r; dst[7] = P.nnz_l_stored; dst[8] = P.n_trsm; dst[9] = P.n_u;
      dst[10] = P.n_hi_tasks; dst[11] = P.n_sub;
      break;
    default: return -2;
  }
  return 0;
}

double spchol_plan_flops(spchol_plan_t p) { return p ? p->plan.flops : -1.0; }

int64_t spchol_plan_pool_len(spchol_plan_t p) { return p ? p->plan.valoff[p->plan.ns] : -1; }

int spchol_plan_simulate(spchol_plan_t p, const double* values, double* B, int64_t ldb, int nrhs, uint64_t seed,
                         double* Lx) {
  if (!p) return -1;
  const Plan& P = p->plan;
  if (!values && P.nnz_a > 0) return -2;
  if (nrhs > 0 && (!B || ldb < P.n)) return -3;
  Sim sim(P);
  for (int64_t e = 0; e < P.nnz_a; ++e) sim.pool[P.a_dest[e]] = values[e];
  Rng rng{seed};
  const int ns = P.ns;

  // ---- factorization: same ids, counters and two ready rings as the GPU kernel
  // (high priority: diagonal and panel-solve tasks and the first nu_hi[s]
  // update tiles of each panel).  Every push is counted against its ring's
  // size, and each ring must receive exactly as many tasks as it holds.
  std::vector<int> dep(P.dep_f.begin(), P.dep_f.end()), tleft(P.ntrsm.begin(), P.ntrsm.end());
  // deterministic order: update tiles chained per target (Plan::u_next) and
  // the solve chains -- not in the fan-in mode, whose tiles need no order
  const bool uchain = !P.u_next.empty();
  const bool fan = P.params.fanin;
  const bool det = P.params.deterministic && !fan;
  std::vector<int> udep(P.u_dep0.begin(), P.u_dep0.end());
  // fan-in mode: gather tasks (Plan::gat_first) and the counters they feed
  std::vector<int> gd(P.gdiag0.begin(), P.gdiag0.end()), td(P.tdep0.begin(), P.tdep0.end());
  const int gat0 = ns + P.n_trsm + P.n_u + P.n_sub;  // first gather task id
  const int u0 = ns + P.n_trsm;  // first update tile id
  std::vector<char> ran(P.n_task_ids, 0);
  Ready hi, lo;
  const int64_t n_hi = P.n_hi_tasks, n_lo = (int64_t)P.n_factor_tasks - P.n_hi_tasks;
  int64_t hi_pushed = 0, lo_pushed = 0;
  bool overflow = false;
  auto push = [&](bool to_hi, int t) {
    if (to_hi) {
      hi.push(t);
      overflow |= ++hi_pushed > n_hi;
    } else {
      lo.push(t);
      overflow |= ++lo_pushed > n_lo;
    }
  };
  const int sub0 = ns + P.n_trsm + P.n_u;  // first subtree task id
  // the last update into panel t has landed: its gathers (fan-in mode) and, when
  // none holds rows of its diagonal block, its diagonal task
  auto landed = [&](int t) {
    if (fan) {
      for (int g = P.gat_first[t]; g < P.gat_first[t + 1]; ++g) push(true, gat0 + g);
      if (P.gdiag0[t] == 0) push(true, t);
    } else {
      push(true, t);
    }
  };
  for (int k = 0; k < P.n_sub; ++k) push(true, sub0 + k);
  for (int s = 0; s < ns; ++s)
    if (dep[s] == 0 && P.in_sub[s] < 0) push(true, s);
  int done = 0;
  while (!hi.empty() || !lo.empty()) {
    if (overflow) return SPCHOL_EINTERNAL;
    const bool from_hi = !hi.empty() && (lo.empty() || (rng.next() & 1));
    const int task = from_hi ? hi.pop(rng) : lo.pop(rng);
    if (task < 0 || task >= P.n_task_ids || ran[task]) return SPCHOL_EINTERNAL;
    ran[task] = 1;
    ++done;
    const bool skip = sim.info != 0;
    if (task >= gat0) {  // gather task (fan-in mode): one row piece of a panel
      const int pc = P.gat_pc[task - gat0], o = P.pc_owner[pc];
      const int t = o < ns ? o : P.trsm_sn[o - ns];
      const int w = sim.width(t);
      int p0, p1;
      if (o < ns) {
        p0 = (pc - P.fan_task[t]) * kFanPieceRows;
        p1 = std::min(w, p0 + kFanPieceRows);
      } else {
        const int k = o - ns - P.trsm_first[t], tr = P.trsm_rows[t], r0 = w + k * tr;
        p0 = r0 + (pc - P.fan_task[o]) * kFanPieceRows;
        p1 = std::min(std::min(P.nrows[t], r0 + tr), p0 + kFanPieceRows);
      }
      if (!skip) sim.gather(t, pc, p0, p1);
      if (o < ns) {
        if (--gd[t] < 0) return SPCHOL_EINTERNAL;
        if (gd[t] == 0) push(true, t);
      } else {
        if (--td[o - ns] < 0) return SPCHOL_EINTERNAL;
        if (td[o - ns] == 0) push(true, o);
      }
    } else if (task >= sub0) {  // subtree task: its panels in order; counters only for targets outside
      const int k = task - sub0, lo = P.sub_lo[k], hi = P.sub_hi[k];
      for (int s = lo; s <= hi; ++s) {
        if (P.in_sub[s] != k) return SPCHOL_EINTERNAL;
        if (sim.info == 0) sim.potrf(s);
        for (int kt = 0; kt < P.ntrsm[s]; ++kt)
          if (sim.info == 0) sim.trsm(s, kt);
        for (int j = 0; j < P.nu[s]; ++j) {
          const UTask& u = P.ut[P.u_first[s] + j];
          if (sim.info == 0) sim.update(u, P.u_first[s] + j);
          if (u.t > hi) {
            if (P.in_sub[u.t] >= 0) return SPCHOL_EINTERNAL;  // an outside target is never in another subtree
            if (--dep[u.t] < 0) return SPCHOL_EINTERNAL;
            if (dep[u.t] == 0) landed(u.t);
          }
        }
      }
    } else if (task < ns) {
      if (P.in_sub[task] >= 0) return SPCHOL_EINTERNAL;
      if (!skip) sim.potrf(task);
      for (int k = 0; k < P.ntrsm[task]; ++k) {
        const int kt = P.trsm_first[task] + k;
        if (fan && --td[kt] != 0) {  // also waits for its rows' gathers
          if (td[kt] < 0) return SPCHOL_EINTERNAL;
          continue;
        }
        push(true, ns + kt);
      }
    } else if (task < ns + P.n_trsm) {
      const int kt = task - ns, s = P.trsm_sn[kt];
      if (P.in_sub[s] >= 0) return SPCHOL_EINTERNAL;
      if (!skip) sim.trsm(s, kt - P.trsm_first[s]);
      if (--tleft[s] < 0) return SPCHOL_EINTERNAL;
      if (tleft[s] == 0)
        for (int k = 0; k < P.nu[s]; ++k) {
          const int u = P.u_first[s] + k;
          if (uchain && --udep[u] != 0) {
            if (udep[u] < 0) return SPCHOL_EINTERNAL;
            continue;  // waits for its predecessor into the same target
          }
          push(k < P.nu_hi[s], u0 + u);
        }
    } else {
      const int ui = task - u0;
      const UTask& u = P.ut[ui];
      if (P.in_sub[u.s] >= 0) return SPCHOL_EINTERNAL;
      if (!skip) sim.update(u, ui);
      if (--dep[u.t] < 0) return SPCHOL_EINTERNAL;
      if (dep[u.t] == 0) landed(u.t);
      if (uchain && P.u_next[ui] >= 0) {
        const int nx = P.u_next[ui], sx = P.ut[nx].s;
        if (--udep[nx] < 0) return SPCHOL_EINTERNAL;
        if (udep[nx] == 0) push(nx - P.u_first[sx] < P.nu_hi[sx], u0 + nx);
      }
    }
    if (sim.info < 0) return SPCHOL_EINTERNAL;
  }
  if (done != P.n_factor_tasks || overflow || hi_pushed != n_hi || lo_pushed != n_lo) return SPCHOL_EINTERNAL;
  if (Lx) std::memcpy(Lx, sim.pool.data(), sim.pool.size() * sizeof(double));
  if (sim.info != 0) return sim.info;
  if (nrhs <= 0 || P.n == 0) return 0;

  // ---- solves ---------------------------------------------------------------
  const int64_t n = P.n;
  std::vector<double> Y((size_t)n * nrhs);
  for (int r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < n; ++i) Y[i + (size_t)r * n] = B[P.perm[i] + (size_t)r * ldb];
  const int nst = P.n_st;
  std::vector<int> fdep(P.fdep0.begin(), P.fdep0.end()), bdep(P.bdep0.begin(), P.bdep0.end());
  std::vector<int> ft(P.nst.begin(), P.nst.end()), bt(P.nst.begin(), P.nst.end());
  std::vector<int> ftdep(P.ft_dep0.begin(), P.ft_dep0.end());  // deterministic order only
  // fan-in mode: the tiles' private buffers (Plan::st_zf)
  std::vector<double> Zf(fan ? (size_t)P.st_zf.back() * nrhs : 0), Zb(fan ? (size_t)P.st_zb.back() * nrhs : 0);
  std::vector<char> sran(P.n_solve_tasks, 0);
  // Two rings as in the GPU kernel: the seeds (panels with no incoming forward
  // tile) fill the normal-priority ring; a task made ready by another is kept
  // as the releasing CTA's next task when that slot is free (continuation),
  // else goes to the high-priority ring.  Kept and pushed tasks must together
  // be exactly the non-seed tasks.
  Ready q, qs;
  int64_t s_seeds = 0, s_pushed = 0, s_kept = 0;
  int next = -1;
  auto spush = [&](int t) {
    q.push(t);
    ++s_pushed;
  };
  auto skeep = [&](int t) {
    if (next < 0) {
      next = t;
      ++s_kept;
    } else {
      spush(t);
    }
  };
  // W panels (Plan::woff): W = L21 L11^{-1} is applied as L21 (L11^{-1} .)
  // and L11^{-T} (L21^T .), the same products
  auto wpan = [&](int s) { return P.woff[s] >= 0; };
  for (int s = 0; s < ns; ++s)
    if (fdep[s] == 0) {
      if (wpan(s)) {  // its forward tiles are ready with b_s
        for (int k = 0; k < P.nst[s]; ++k) qs.push(ns + P.st_first[s] + k);
        s_seeds += P.nst[s];
      } else {
        qs.push(s);
        ++s_seeds;
      }
    }
  // L11^{-1} y (lower) and L11^{-T} y (upper) by substitution, y of length w
  auto lsolve = [&](const double* L, int ld, int w, double* y) {
    for (int j = 0; j < w; ++j) {
      y[j] /= L[j + (size_t)j * ld];
      for (int i = j + 1; i < w; ++i) y[i] -= L[i + (size_t)j * ld] * y[j];
    }
  };
  auto ltsolve = [&](const double* L, int ld, int w, double* y) {
    for (int j = w - 1; j >= 0; --j) {
      y[j] /= L[j + (size_t)j * ld];
      for (int i = 0; i < j; ++i) y[i] -= L[j + (size_t)i * ld] * y[j];
    }
  };
  std::vector<double> tmp;
  int sdone = 0;
  while (next >= 0 || !q.empty() || !qs.empty()) {
    int task = next;
    if (task >= 0) {
      next = -1;
    } else {
      const bool from_hi = !q.empty() && (qs.empty() || (rng.next() & 1));
      task = from_hi ? q.pop(rng) : qs.pop(rng);
    }
    if (task < 0 || task >= P.n_solve_tasks || sran[task]) return SPCHOL_EINTERNAL;
    sran[task] = 1;
    ++sdone;
    if (task < ns && wpan(task)) {  // FWD_D of a W panel: y_s <- L11^{-T} L11^{-1} b_s
      const int s = task, f = P.fcol[s], w = sim.width(s), ld = P.ld[s];
      const double* L = sim.panel(s);
      if (ft[s] != 0) return SPCHOL_EINTERNAL;  // its forward tiles must have read b_s
      for (int r = 0; r < nrhs; ++r) {
        lsolve(L, ld, w, Y.data() + f + (size_t)r * n);
        ltsolve(L, ld, w, Y.data() + f + (size_t)r * n);
      }
      for (int k = 0; k < P.nst[s]; ++k) {
        const int tile = P.st_first[s] + k;
        if (--bdep[tile] < 0) return SPCHOL_EINTERNAL;
        if (bdep[tile] == 0) skeep(ns + nst + tile);
      }
    } else if (task < ns) {  // FWD_D
      const int s = task, f = P.fcol[s], w = sim.width(s), ld = P.ld[s];
      const double* L = sim.panel(s);
      if (fan)  // the forward tiles' products into these rows, in tile order
        for (int e = P.rt_ptr[s + 1] - 1; e >= P.rt_ptr[s]; --e) {
          const int tile = P.rt_tile[e], i0 = P.rt_rng[e] & 0xffff, i1 = P.rt_rng[e] >> 16;
          const int cnt = (int)(P.st_zf[tile + 1] - P.st_zf[tile]);
          const double* z = Zf.data() + (size_t)P.st_zf[tile] * nrhs;
          for (int i = i0; i < i1; ++i) {
            const int c = P.rows[P.st_roff[tile] + i] - f;
            if (c < 0 || c >= w) return SPCHOL_EINTERNAL;
            for (int r = 0; r < nrhs; ++r) Y[f + c + (size_t)r * n] += z[i + (size_t)r * cnt];
          }
        }
      for (int r = 0; r < nrhs; ++r) {
        double* y = Y.data() + f + (size_t)r * n;
        for (int j = 0; j < w; ++j) {
          y[j] /= L[j + (size_t)j * ld];
          for (int i = j + 1; i < w; ++i) y[i] -= L[i + (size_t)j * ld] * y[j];
        }
      }
      // the first forward tile (or the backward diagonal task) continues here
      if (P.nst[s] > 0) {
        for (int k = 0; k < P.nst[s]; ++k) {
          const int tile = P.st_first[s] + k;
          if (det) {  // also waits for its predecessors into the same panels
            if (--ftdep[tile] < 0) return SPCHOL_EINTERNAL;
            if (ftdep[tile] != 0) continue;
          }
          skeep(ns + tile);
        }
      } else {
        skeep(ns + 2 * nst + s);
      }
    } else if (task < ns + nst) {  // FWD_T
      const int kt = task - ns, s = P.st_sn[kt], k = kt - P.st_first[s];
      const int f = P.fcol[s], w = sim.width(s), ld = P.ld[s], rr = P.nrows[s];
      const int TS = P.st_rows[s], row0 = w + k * TS, cnt = std::min(TS, rr - row0);
      const double* L = sim.panel(s);
      const int32_t* R = P.rows.data() + P.rowoff[s];
      const bool wp = wpan(s);
      tmp.assign((size_t)w * nrhs, 0.0);  // y_s, or for a W panel L11^{-1} b_s
      for (int r = 0; r < nrhs; ++r) {
        for (int j = 0; j < w; ++j) tmp[j + (size_t)r * w] = Y[f + j + (size_t)r * n];
        if (wp) lsolve(L, ld, w, tmp.data() + (size_t)r * w);
      }
      for (int r = 0; r < nrhs; ++r)
        for (int i = row0; i < row0 + cnt; ++i) {
          double acc = 0.0;
          for (int j = 0; j < w; ++j) acc += L[i + (size_t)j * ld] * tmp[j + (size_t)r * w];
          if (fan)
            Zf[(size_t)P.st_zf[kt] * nrhs + (i - row0) + (size_t)r * cnt] = -acc;
          else
            Y[R[i] + (size_t)r * n] -= acc;
        }
      for (int e = P.st_tptr[kt]; e < P.st_tptr[kt + 1]; ++e) {
        const int t = P.st_tgt[e];
        if (--fdep[t] < 0) return SPCHOL_EINTERNAL;
        if (fdep[t] == 0) {
          if (wpan(t)) {  // all of t's forward tiles, the first as the continuation
            for (int k2 = 0; k2 < P.nst[t]; ++k2) skeep(ns + P.st_first[t] + k2);
          } else {
            skeep(t);
          }
        }
      }
      if (det)
        for (int q2 = P.ft_sptr[kt]; q2 < P.ft_sptr[kt + 1]; ++q2) {
          const int nx = P.ft_succ[q2];
          if (--ftdep[nx] < 0) return SPCHOL_EINTERNAL;
          if (ftdep[nx] == 0) skeep(ns + nx);
        }
      if (--ft[s] < 0) return SPCHOL_EINTERNAL;
      if (ft[s] == 0) {
        if (wp) {
          skeep(s);  // the W panel's diagonal task
        } else {
          for (int k2 = 0; k2 < P.nst[s]; ++k2) {
            const int tile = P.st_first[s] + k2;
            if (--bdep[tile] == 0) skeep(ns + nst + tile);
          }
        }
      }
    } else if (task < ns + 2 * nst) {  // BWD_T
      const int kt = task - ns - nst, s = P.st_sn[kt], k = kt - P.st_first[s];
      const int f = P.fcol[s], w = sim.width(s), ld = P.ld[s], rr = P.nrows[s];
      const int TS = P.st_rows[s], row0 = w + k * TS, cnt = std::min(TS, rr - row0);
      const double* L = sim.panel(s);
      const int32_t* R = P.rows.data() + P.rowoff[s];
      const bool wp = wpan(s);
      tmp.assign((size_t)w, 0.0);
      for (int r = 0; r < nrhs; ++r) {
        for (int j = 0; j < w; ++j) {
          double acc = 0.0;
          for (int i = row0; i < row0 + cnt; ++i) acc += L[i + (size_t)j * ld] * Y[R[i] + (size_t)r * n];
          tmp[j] = acc;
        }
        if (wp) ltsolve(L, ld, w, tmp.data());  // W^T x = L11^{-T} (L21^T x)
        for (int j = 0; j < w; ++j) {
          if (fan)
            Zb[(size_t)P.st_zb[kt] * nrhs + j + (size_t)r * w] = -tmp[j];
          else
            Y[f + j + (size_t)r * n] -= tmp[j];
        }
      }
      if (det && k + 1 < P.nst[s]) {  // the panel's next backward tile
        const int nx = P.st_first[s] + k + 1;
        if (--bdep[nx] < 0) return SPCHOL_EINTERNAL;
        if (bdep[nx] == 0) skeep(ns + nst + nx);
      }
      if (--bt[s] < 0) return SPCHOL_EINTERNAL;
      if (bt[s] == 0 && wp) {  // x_s = y_s is final: release its readers
        for (int e = P.rt_ptr[s]; e < P.rt_ptr[s + 1]; ++e) {
          const int tile = P.rt_tile[e];
          if (--bdep[tile] < 0) return SPCHOL_EINTERNAL;
          if (bdep[tile] == 0) skeep(ns + nst + tile);
        }
      } else if (bt[s] == 0) {
        skeep(ns + 2 * nst + s);
      }
    } else {  // BWD_D
      const int s = task - ns - 2 * nst, f = P.fcol[s], w = sim.width(s), ld = P.ld[s];
      const double* L = sim.panel(s);
      if (fan)  // the panel's backward tiles' products, in tile order
        for (int k = 0; k < P.nst[s]; ++k) {
          const double* z = Zb.data() + (size_t)P.st_zb[P.st_first[s] + k] * nrhs;
          for (int r = 0; r < nrhs; ++r)
            for (int j = 0; j < w; ++j) Y[f + j + (size_t)r * n] += z[j + (size_t)r * w];
        }
      for (int r = 0; r < nrhs; ++r) {
        double* y = Y.data() + f + (size_t)r * n;
        for (int j = w - 1; j >= 0; --j) {
          y[j] /= L[j + (size_t)j * ld];
          for (int i = 0; i < j; ++i) y[i] -= L[j + (size_t)i * ld] * y[j];
        }
      }
      for (int e = P.rt_ptr[s]; e < P.rt_ptr[s + 1]; ++e) {
        const int tile = P.rt_tile[e];
        if (--bdep[tile] < 0) return SPCHOL_EINTERNAL;
        if (bdep[tile] == 0) skeep(ns + nst + tile);
      }
    }
  }
  const int64_t n_run = P.n_solve_tasks - P.n_wpan;  // W panels have no backward diagonal task
  if (sdone != n_run || s_pushed + s_kept != n_run - s_seeds) return SPCHOL_EINTERNAL;
  for (int r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < n; ++i) B[P.perm[i] + (size_t)r * ldb] = Y[i + (size_t)r * n];
  return 0;
}

void spchol_plan_destroy(spchol_plan_t p) { delete p; }

}  // extern "C"
