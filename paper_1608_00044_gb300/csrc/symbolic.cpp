// Host symbolic analysis (Section II-B, III-B): elimination tree, postorder,
// column counts, supernodes, relaxed amalgamation, width cap, row structures,
// storage layout and the task graph.
#include <algorithm>
#include <iterator>
#include <cstring>
#include <numeric>

#include "plan.hpp"

namespace spchol {
namespace {

// Pattern of B = P A P^T (lower), both by columns (CSC) and by rows (strict
// lower part, CSR): the column form feeds the supernodal row structures, the
// row form the elimination tree and the column counts.
struct Pattern {
  std::vector<int64_t> cp;  // CSC lower, rows unsorted
  std::vector<int32_t> ci;
  std::vector<int64_t> rp;  // CSR strict lower: row i lists k < i
  std::vector<int32_t> ri;
};

void permuted_pattern(int64_t n, const int64_t* colptr, const int32_t* rowind,
                      const std::vector<int64_t>& pinv, Pattern& B) {
  const int64_t nnz = colptr[n];
  B.cp.assign(n + 1, 0);
  B.rp.assign(n + 1, 0);
  for (int64_t c = 0; c < n; ++c)
    for (int64_t p = colptr[c]; p < colptr[c + 1]; ++p) {
      int64_t a = pinv[rowind[p]], b = pinv[c];
      int64_t lo = std::min(a, b), hi = std::max(a, b);
      B.cp[lo + 1]++;
      if (hi != lo) B.rp[hi + 1]++;
    }
  for (int64_t j = 0; j < n; ++j) {
    B.cp[j + 1] += B.cp[j];
    B.rp[j + 1] += B.rp[j];
  }
  B.ci.resize(nnz);
  B.ri.resize(B.rp[n]);
  std::vector<int64_t> fc(B.cp.begin(), B.cp.end() - 1), fr(B.rp.begin(), B.rp.end() - 1);
  for (int64_t c = 0; c < n; ++c)
    for (int64_t p = colptr[c]; p < colptr[c + 1]; ++p) {
      int64_t a = pinv[rowind[p]], b = pinv[c];
      int64_t lo = std::min(a, b), hi = std::max(a, b);
      B.ci[fc[lo]++] = (int32_t)hi;
      if (hi != lo) B.ri[fr[hi]++] = (int32_t)lo;
    }
}

// Elimination tree by Liu's algorithm with path compression: row i's nonzeros
// b_ik (k < i) attach the root of k's current subtree to i.
void etree_liu(int64_t n, const Pattern& B, std::vector<int32_t>& parent) {
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = B.rp[i]; p < B.rp[i + 1]; ++p) {
      int32_t r = B.ri[p];
      while (r != -1 && r != i) {
        int32_t nx = anc[r];
        anc[r] = (int32_t)i;
        if (nx == -1) parent[r] = (int32_t)i;
        r = nx;
      }
    }
}

// Depth-first postorder with children visited in increasing order; the identity
// when the numbering already is such a postorder.
void postorder(int64_t n, const std::vector<int32_t>& parent, std::vector<int64_t>& post) {
  std::vector<int32_t> head(n, -1), next(n, -1);
  for (int64_t j = n - 1; j >= 0; --j)
    if (parent[j] != -1) {
      next[j] = head[parent[j]];
      head[parent[j]] = (int32_t)j;
    }
  post.clear();
  post.reserve(n);
  std::vector<int32_t> stack;
  for (int64_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back((int32_t)r);
    while (!stack.empty()) {
      int32_t v = stack.back();
      if (head[v] != -1) {
        int32_t c = head[v];
        head[v] = next[c];
        stack.push_back(c);
      } else {
        stack.pop_back();
        post.push_back(v);
      }
    }
  }
}

// Column counts without forming L (Gilbert, Ng and Peyton, "An efficient
// algorithm to compute row and column counts for sparse Cholesky
// factorization", SIAM J. Matrix Anal. Appl. 15, 1994), restated.  c_j is the
// number of row subtrees T(i) (the union of the etree paths from each k with
// b_ik != 0 up to i, and i itself) that contain j.  With the columns in
// postorder, a weight per node -- +1 at each leaf of each T(i), -1 at the
// least common ancestor of two consecutive leaves of the same T(i), -1 at
// parent(i) for every row i -- sums over the subtree of j to exactly c_j.
// Column j is a leaf of T(i) when no earlier column of row i lies in j's
// subtree (the columns of j's subtree are first(j) .. j); the common
// ancestors come from a disjoint-set forest in which every finished column
// is joined to its parent (for columns p < j, the root of p's set is then the
// least common ancestor of p and j).  O(nnz(A) alpha(n)); requires the
// postorder numbering, which build_plan establishes first.
void column_counts(int64_t n, const Pattern& B, const std::vector<int32_t>& parent,
                   std::vector<int64_t>& cc) {
  std::vector<int32_t> first(n, -1), prevnz(n, -1), prevleaf(n, -1), anc(n);
  cc.assign(n, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = j; k != -1 && first[k] == -1; k = parent[k]) first[k] = (int32_t)j;
  for (int64_t j = 0; j < n; ++j) {
    anc[j] = (int32_t)j;
    if (parent[j] != -1) cc[parent[j]]--;
  }
  auto find = [&](int32_t x) {
    int32_t r = x;
    while (anc[r] != r) r = anc[r];
    while (anc[x] != r) {  // path compression
      const int32_t nx = anc[x];
      anc[x] = r;
      x = nx;
    }
    return r;
  };
  // row i has a nonzero in column j <= i (columns visited in increasing order)
  auto visit = [&](int32_t i, int32_t j) {
    const bool leaf = first[j] > prevnz[i];
    prevnz[i] = j;
    if (!leaf) return;
    cc[j]++;
    if (prevleaf[i] != -1) cc[find(prevleaf[i])]--;
    prevleaf[i] = j;
  };
  for (int64_t j = 0; j < n; ++j) {
    visit((int32_t)j, (int32_t)j);  // the diagonal: T(j) contains j
    for (int64_t p = B.cp[j]; p < B.cp[j + 1]; ++p)
      if (B.ci[p] != j) visit(B.ci[p], (int32_t)j);
    if (parent[j] != -1) anc[j] = parent[j];
  }
  for (int64_t j = 0; j < n; ++j)
    if (parent[j] != -1) cc[parent[j]] += cc[j];
}

inline int64_t round4(int64_t x) { return (x + 3) & ~int64_t(3); }

}  // namespace

int build_plan(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm_in,
               const PlanParams& prm, Plan& P, PlanError& err) {
  // ---- validation --------------------------------------------------------
  if (n < 0 || n > INT32_MAX - 1) {
    err = {1, "n out of range"};
    return -1;
  }
  if (n > 0 && !colptr) { err = {2, "colptr is NULL"}; return -2; }
  if (n > 0 && colptr[0] != 0) { err = {2, "colptr[0] != 0"}; return -2; }
  for (int64_t j = 0; j < n; ++j)
    if (colptr[j + 1] < colptr[j]) {
      err = {2, "colptr not non-decreasing"};
      return -2;
    }
  const int64_t nnz = n > 0 ? colptr[n] : 0;
  if (nnz > 0 && !rowind) { err = {3, "rowind is NULL"}; return -3; }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      int32_t r = rowind[p];
      if (r < j || r >= n) {
        err = {3, "row index outside the lower triangle"};
        return -3;
      }
      if (p > colptr[j] && r <= rowind[p - 1]) {
        err = {3, "rows not strictly increasing within a column"};
        return -3;
      }
    }
  P = Plan();
  P.params = prm;
  P.n = n;
  P.nnz_a = nnz;
  P.perm.resize(n);
  P.pinv.assign(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = perm_in ? perm_in[i] : i;
    if (o < 0 || o >= n || P.pinv[o] != -1) {
      err = {4, "perm is not a permutation"};
      return -4;
    }
    P.perm[i] = o;
    P.pinv[o] = i;
  }

  // ---- etree and postorder --------------------------------------------------
  Pattern B;
  permuted_pattern(n, colptr, rowind, P.pinv, B);
  std::vector<int32_t> parent;
  etree_liu(n, B, parent);
  std::vector<int64_t> post;
  postorder(n, parent, post);
  bool identity = true;
  for (int64_t k = 0; k < n; ++k)
    if (post[k] != k) { identity = false; break; }
  if (!identity) {
    std::vector<int64_t> np(n);
    for (int64_t k = 0; k < n; ++k) np[k] = P.perm[post[k]];
    P.perm.swap(np);
    for (int64_t k = 0; k < n; ++k) P.pinv[P.perm[k]] = k;
    permuted_pattern(n, colptr, rowind, P.pinv, B);
    // a postorder is a topological order of the elimination tree, under which
    // the tree is unchanged: relabel it instead of computing it again
    std::vector<int32_t> newpos(n), relabeled(n);
    for (int64_t k = 0; k < n; ++k) newpos[post[k]] = (int32_t)k;
    for (int64_t k = 0; k < n; ++k) {
      const int32_t q = parent[post[k]];
      relabeled[k] = q < 0 ? -1 : newpos[q];
    }
    parent.swap(relabeled);
  }
  column_counts(n, B, parent, P.colcount);
  P.etree = parent;
  P.nnz_l = 0;
  P.flops = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    P.nnz_l += P.colcount[j];
    P.flops += (double)P.colcount[j] * (double)P.colcount[j];
  }

  // ---- supernodes (Section II-B definition) --------------------------------
  // Column j+1 continues j's supernode iff parent(j) = j+1 and
  // c_j = c_{j+1} + 1, i.e. S_j \ {j+1} = S_{j+1} given S_j \ {j+1} is a subset.
  std::vector<int32_t> sn_first;
  for (int64_t j = 0; j < n; ++j)
    if (j == 0 || !(parent[j - 1] == j && P.colcount[j - 1] == P.colcount[j] + 1))
      sn_first.push_back((int32_t)j);
  const int32_t ns0 = (int32_t)sn_first.size();
  sn_first.push_back((int32_t)n);
  std::vector<int32_t> sn0_of(n);
  for (int32_t s = 0; s < ns0; ++s)
    for (int32_t j = sn_first[s]; j < sn_first[s + 1]; ++j) sn0_of[j] = s;
  std::vector<int32_t> sn0_parent(ns0, -1);
  for (int32_t s = 0; s < ns0; ++s) {
    int32_t last = sn_first[s + 1] - 1;
    if (parent[last] != -1) sn0_parent[s] = sn0_of[parent[last]];
  }

  // ---- relaxed amalgamation -------------------------------------------------
  // Bottom-up: the merged supernode that ends just before s is merged into s
  // when it is a child of s, the width stays <= W, and every merged column
  // gains at most relax_zeros explicit zeros over its exact count.
  const int W = std::max(1, prm.max_width);
  struct MS {
    int32_t f, l, top;
  };
  std::vector<MS> stack;
  stack.reserve(ns0);
  for (int32_t s = 0; s < ns0; ++s) {
    MS cur{sn_first[s], sn_first[s + 1] - 1, s};
    const int64_t nbelow = P.colcount[cur.l] - 1;
    while (prm.relax_zeros > 0 && !stack.empty()) {
      const MS& q = stack.back();
      if (q.l != cur.f - 1 || sn0_parent[q.top] != s) break;
      if ((cur.l - q.f + 1) > W) break;
      bool ok = true;
      for (int32_t j = q.f; j <= q.l && ok; ++j) {
        int64_t merged = (int64_t)(cur.l - j + 1) + nbelow;
        if (merged - P.colcount[j] > prm.relax_zeros) ok = false;
      }
      if (!ok) break;
      cur.f = q.f;
      stack.pop_back();
    }
    stack.push_back(cur);
  }

  // ---- width cap: chains of panels of at most W columns ----------------------
  P.fcol.clear();
  for (const MS& m : stack) {
    int32_t w = m.l - m.f + 1;
    for (int32_t c = 0; c < w; c += W) P.fcol.push_back(m.f + c);
  }
  P.ns = (int32_t)P.fcol.size();
  P.fcol.push_back((int32_t)n);
  const int32_t ns = P.ns;
  P.snode_of.resize(n);
  for (int32_t s = 0; s < ns; ++s)
    for (int32_t j = P.fcol[s]; j < P.fcol[s + 1]; ++j) P.snode_of[j] = s;
  P.parent.assign(ns, -1);
  for (int32_t s = 0; s < ns; ++s) {
    int32_t last = P.fcol[s + 1] - 1;
    if (parent[last] != -1) P.parent[s] = P.snode_of[parent[last]];
  }

  // ---- row structures: the union of the panel's columns of B and its
  // children's structures, restricted to rows past the panel -----------------
  std::vector<int32_t> kid_head(ns, -1), kid_next(ns, -1);
  for (int32_t s = ns - 1; s >= 0; --s)
    if (P.parent[s] != -1) {
      kid_next[s] = kid_head[P.parent[s]];
      kid_head[P.parent[s]] = s;
    }
  std::vector<std::vector<int32_t>> below(ns);
  std::vector<int32_t> mark(n, -1);
  std::vector<int32_t> buf, tmp;
  for (int32_t s = 0; s < ns; ++s) {
    const int32_t f = P.fcol[s], l = P.fcol[s + 1] - 1;
    // B's own rows past the panel (a few per column), sorted ...
    buf.clear();
    for (int32_t j = f; j <= l; ++j)
      for (int64_t p = B.cp[j]; p < B.cp[j + 1]; ++p) {
        int32_t r = B.ci[p];
        if (r > l && mark[r] != s) {
          mark[r] = s;
          buf.push_back(r);
        }
      }
    std::sort(buf.begin(), buf.end());
    // ... merged with each child's sorted list past the panel (linear merges)
    for (int32_t c = kid_head[s]; c != -1; c = kid_next[c]) {
      const std::vector<int32_t>& bc = below[c];
      auto from = std::upper_bound(bc.begin(), bc.end(), l);
      tmp.clear();
      std::set_union(buf.begin(), buf.end(), from, bc.end(), std::back_inserter(tmp));
      buf.swap(tmp);
    }
    below[s] = buf;
    // a child's list is needed only by its parent
    for (int32_t c = kid_head[s]; c != -1; c = kid_next[c]) std::vector<int32_t>().swap(below[c]);
    // panels are built in order, so the row lists are appended in order
    P.nrows.push_back((l - f + 1) + (int32_t)buf.size());
    for (int32_t j = f; j <= l; ++j) P.rows.push_back(j);
    P.rows.insert(P.rows.end(), buf.begin(), buf.end());
  }
  P.rowoff.assign(ns + 1, 0);
  for (int32_t s = 0; s < ns; ++s) P.rowoff[s + 1] = P.rowoff[s] + P.nrows[s];

  // ---- storage layout ------------------------------------------------------
  P.ld.resize(ns);
  P.valoff.assign(ns + 1, 0);
  P.invoff.assign(ns + 1, 0);
  P.sliceoff.assign(ns + 1, 0);
  P.nnz_l_stored = 0;
  P.max_w = 0;
  P.max_r = 0;
  for (int32_t s = 0; s < ns; ++s) {
    int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s];
    P.ld[s] = (int32_t)round4(r);
    P.valoff[s + 1] = P.valoff[s] + (int64_t)P.ld[s] * w;
    P.invoff[s + 1] = P.invoff[s] + (int64_t)w * w;
    // BF16 slices of the rows below the diagonal block (panels on the tensor
    // cores in the FP64 tensor-core mode): kSlices x nb x kpad16
    const bool sliced = prm.slice_fp64 && w >= prm.tc_min_width;
    P.sliceoff[s + 1] = P.sliceoff[s] + (sliced ? (int64_t)kSlices * (r - w) * (((int64_t)w + 15) & ~int64_t(15)) : 0);
    P.nnz_l_stored += (int64_t)r * w - (int64_t)w * (w - 1) / 2;
    P.max_w = std::max(P.max_w, w);
    P.max_r = std::max(P.max_r, r);
  }

  // ---- where each entry of A lands in the pool --------------------------------
  P.a_dest.resize(nnz);
  for (int64_t c = 0; c < n; ++c)
    for (int64_t p = colptr[c]; p < colptr[c + 1]; ++p) {
      int64_t a = P.pinv[rowind[p]], b = P.pinv[c];
      int32_t lo = (int32_t)std::min(a, b), hi = (int32_t)std::max(a, b);
      int32_t s = P.snode_of[lo];
      const int32_t* R = P.rows.data() + P.rowoff[s];
      int32_t pos = (int32_t)(std::lower_bound(R, R + P.nrows[s], hi) - R);
      P.a_dest[p] = P.valoff[s] + pos + (int64_t)(lo - P.fcol[s]) * P.ld[s];
    }

  // ---- factorization tasks ------------------------------------------------------
  std::vector<int32_t> depth(ns, 0);
  for (int32_t s = ns - 1; s >= 0; --s) depth[s] = P.parent[s] < 0 ? 0 : depth[P.parent[s]] + 1;
  P.trsm_rows.assign(ns, 0);
  P.trsm_first.assign(ns, 0);
  P.ntrsm.assign(ns, 0);
  P.u_first.assign(ns, 0);
  P.nu.assign(ns, 0);
  P.dep_f.assign(ns, 0);
  P.nu_hi.assign(ns, 0);
  P.trsm_sn.clear();
  P.ut.clear();
  P.n_rel = 0;
  {
    // the tile count first (the same walk), so that the tile list is built in
    // place: millions of tiles on the large grids
    int64_t nt = 0, ntr = 0;
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s];
      const bool top = depth[s] < prm.top_depth;
      const bool tc = prm.tc_min_width > 0 && w >= prm.tc_min_width;
      const int TU = std::max(1, tc ? prm.tc_tile_rows : top ? std::min(prm.top_tile_rows, prm.tile_rows) : prm.tile_rows);
      const int TR = std::max(1, top ? std::min(prm.top_trsm_rows, prm.trsm_rows) : prm.trsm_rows);
      ntr += (r - w + TR - 1) / TR;
      const int32_t* R = P.rows.data() + P.rowoff[s];
      for (int32_t a = w; a < r;) {
        const int32_t t = P.snode_of[R[a]];
        int32_t e = a;
        while (e < r && R[e] < P.fcol[t + 1]) ++e;
        nt += (r - a + TU - 1) / TU;
        a = e;
      }
    }
    P.ut.reserve((size_t)nt);
    P.trsm_sn.reserve((size_t)ntr);
  }
  for (int32_t s = 0; s < ns; ++s) {
    const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s];
    const int32_t nb = r - w;
    const bool top = depth[s] < prm.top_depth;
    const bool tc = prm.tc_min_width > 0 && w >= prm.tc_min_width;
    const int TU = std::max(1, tc ? prm.tc_tile_rows : top ? std::min(prm.top_tile_rows, prm.tile_rows) : prm.tile_rows);
    const int TR = std::max(1, top ? std::min(prm.top_trsm_rows, prm.trsm_rows) : prm.trsm_rows);
    P.trsm_rows[s] = TR;
    P.trsm_first[s] = (int32_t)P.trsm_sn.size();
    P.ntrsm[s] = (nb + TR - 1) / TR;
    for (int32_t k = 0; k < P.ntrsm[s]; ++k) P.trsm_sn.push_back(s);
    P.u_first[s] = (int32_t)P.ut.size();
    const int32_t* R = P.rows.data() + P.rowoff[s];
    int32_t a = w;
    while (a < r) {
      int32_t t = P.snode_of[R[a]];
      int32_t e = a;
      while (e < r && R[e] < P.fcol[t + 1]) ++e;
      for (int32_t r0 = a; r0 < r; r0 += TU) {
        const int32_t len = std::min(TU, r - r0);
        P.ut.push_back(UTask{s, t, a, e - a, r0, len, P.n_rel});
        P.n_rel += len;
        P.dep_f[t]++;
      }
      // the first target is the etree parent (it holds the first row below the
      // diagonal block); near the root its tiles are on the critical path
      if (a == w && top) P.nu_hi[s] = (int32_t)P.ut.size() - P.u_first[s];
      a = e;
    }
    P.nu[s] = (int32_t)P.ut.size() - P.u_first[s];
  }
  P.n_trsm = (int32_t)P.trsm_sn.size();
  P.n_u = (int32_t)P.ut.size();
  P.u_next.clear();
  P.u_dep0.clear();
  if (prm.deterministic && !prm.fanin) {
    // tiles are numbered by source panel, then by target, then by row tile:
    // in that order each target's tiles form its chain
    P.u_next.assign(P.n_u, -1);
    P.u_dep0.assign(P.n_u, 1);
    std::vector<int32_t> last(ns, -1);
    for (int32_t u = 0; u < P.n_u; ++u) {
      const int32_t t = P.ut[u].t;
      if (last[t] >= 0) {
        P.u_next[last[t]] = u;
        P.u_dep0[u] = 2;
      }
      last[t] = u;
    }
  }

  // ---- fan-in gather lists (see Plan::fan_ptr) ---------------------------------
  P.fan_off.clear();
  P.fan_task.clear();
  P.fan_ptr.clear();
  P.fan_ent.clear();
  if (prm.fanin) {
    P.fan_off.assign((size_t)P.n_u + 1, 0);
    for (int32_t u = 0; u < P.n_u; ++u)
      P.fan_off[u + 1] = P.fan_off[u] + (int64_t)P.ut[u].rowlen * P.ut[u].seglen;
    auto npieces = [](int32_t rows) { return (rows + kFanPieceRows - 1) / kFanPieceRows; };
    P.fan_task.assign((size_t)ns + P.n_trsm, 0);
    int32_t npc = 0;
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s], tr = P.trsm_rows[s];
      P.fan_task[s] = npc;
      npc += npieces(w);
      for (int32_t k = 0; k < P.ntrsm[s]; ++k) {
        P.fan_task[ns + P.trsm_first[s] + k] = npc;
        npc += npieces(std::min(tr, r - w - k * tr));
      }
    }
    // the piece holding row position p of panel t, and the first position past it
    auto piece_of = [&](int32_t t, int32_t p, int32_t& end) -> int32_t {
      const int32_t w = P.fcol[t + 1] - P.fcol[t], r = P.nrows[t], tr = P.trsm_rows[t];
      if (p < w) {
        const int32_t m = p / kFanPieceRows;
        end = std::min(w, (m + 1) * kFanPieceRows);
        return P.fan_task[t] + m;
      }
      const int32_t k = (p - w) / tr, b0 = w + k * tr, m = (p - b0) / kFanPieceRows;
      end = std::min(std::min(r, b0 + tr), b0 + (m + 1) * kFanPieceRows);
      return P.fan_task[ns + P.trsm_first[t] + k] + m;
    };
    struct Item {
      int32_t pc;
      FanEnt e;
    };
    std::vector<Item> items;
    items.reserve((size_t)P.n_u * 2);
    int32_t hint_s = -1, hint_t = -1, hint = 0;  // the last position found for this (source, target)
    for (int32_t u = 0; u < P.n_u; ++u) {
      const UTask& U = P.ut[u];
      const int32_t* Rs = P.rows.data() + P.rowoff[U.s] + U.row0;
      const int32_t* Rt = P.rows.data() + P.rowoff[U.t];
      const int32_t rt = P.nrows[U.t];
      if (U.s != hint_s || U.t != hint_t) {
        hint_s = U.s;
        hint_t = U.t;
        hint = 0;
      }
      for (int32_t i = 0; i < U.rowlen;) {
        // a tile's rows are rows of its target (the structure of L is closed
        // under updates), so the search finds each exactly; the rows of one
        // (source, target) pair come in increasing order, so it gallops
        // forward from the last position found
        int32_t lo = hint, step = 1;
        while (lo + step < rt && Rt[lo + step] < Rs[i]) {
          lo += step;
          step *= 2;
        }
        const int32_t p =
            (int32_t)(std::lower_bound(Rt + lo, Rt + std::min(rt, lo + step + 1), Rs[i]) - Rt);
        hint = p;
        int32_t end = 0;
        const int32_t pc = piece_of(U.t, p, end);
        const int32_t i1 =
            end >= rt ? U.rowlen : (int32_t)(std::lower_bound(Rs + i, Rs + U.rowlen, Rt[end]) - Rs);
        items.push_back(Item{pc, FanEnt{u, (int16_t)i, (int16_t)i1}});
        i = i1;
      }
    }
    // a stable counting sort by piece keeps each list in update-tile order
    P.fan_ptr.assign((size_t)npc + 1, 0);
    for (const Item& it : items) P.fan_ptr[it.pc + 1]++;
    for (int32_t k = 0; k < npc; ++k) P.fan_ptr[k + 1] += P.fan_ptr[k];
    P.fan_ent.resize(items.size());
    std::vector<int64_t> fill(P.fan_ptr.begin(), P.fan_ptr.end() - 1);
    for (const Item& it : items) P.fan_ent[fill[it.pc]++] = it.e;
  }

  // ---- subtree tasks ------------------------------------------------------------
  // Flops of each panel's own tasks, summed over subtrees (children precede
  // their parents in the postorder); maximal subtrees within the budget become
  // one task each.  A subtree is the contiguous panel range from its first
  // descendant to its root.
  std::vector<double> sub_fl(ns, 0.0);
  for (int32_t s = 0; s < ns; ++s) {
    const double w = P.fcol[s + 1] - P.fcol[s], nb = P.nrows[s] - w;
    sub_fl[s] += w * w * w / 3.0 + nb * w * w;
  }
  for (const UTask& u : P.ut) sub_fl[u.s] += 2.0 * (P.fcol[u.s + 1] - P.fcol[u.s]) * u.rowlen * u.seglen;
  std::vector<int32_t> first_desc(ns);
  for (int32_t s = 0; s < ns; ++s) first_desc[s] = s;
  for (int32_t s = 0; s < ns; ++s)
    if (P.parent[s] >= 0) {
      sub_fl[P.parent[s]] += sub_fl[s];
      first_desc[P.parent[s]] = std::min(first_desc[P.parent[s]], first_desc[s]);
    }
  P.sub_lo.clear();
  P.sub_hi.clear();
  P.in_sub.assign(ns, -1);
  // A subtree task runs serially in one CTA, so the budget is also capped at
  // 1/4096 of the whole factorization: a small problem keeps enough
  // independent pieces of work to spread over the GPU.
  double total = 0.0;
  for (int32_t s = 0; s < ns; ++s)
    if (P.parent[s] < 0) total += sub_fl[s];
  const double budget = std::min(prm.subtree_flops, total / 4096.0);
  if (prm.subtree_flops > 0.0)
    for (int32_t s = 0; s < ns; ++s) {
      const bool small = sub_fl[s] <= budget;
      const bool root = small && (P.parent[s] < 0 || sub_fl[P.parent[s]] > budget);
      if (root && s > first_desc[s]) {  // a subtree of one panel gains nothing
        const int32_t k = (int32_t)P.sub_lo.size();
        P.sub_lo.push_back(first_desc[s]);
        P.sub_hi.push_back(s);
        for (int32_t q = first_desc[s]; q <= s; ++q) P.in_sub[q] = k;
      }
    }
  P.n_sub = (int32_t)P.sub_lo.size();
  {
    double in_sub = 0.0;
    for (int32_t k = 0; k < P.n_sub; ++k) in_sub += sub_fl[P.sub_hi[k]];
    P.sub_work_frac = total > 0.0 ? in_sub / total : 0.0;
  }
  P.wsub.clear();
  for (int32_t k = 0; k < P.n_sub; ++k) {
    int32_t wmax = 0;
    for (int32_t q = P.sub_lo[k]; q <= P.sub_hi[k]; ++q) wmax = std::max(wmax, P.fcol[q + 1] - P.fcol[q]);
    if (wmax <= kWarpSubW) P.wsub.push_back(k);
  }
  // the most work first: each warp takes the next, so the last to start are
  // the smallest (a large subtree started late would hold its launch open)
  std::stable_sort(P.wsub.begin(), P.wsub.end(),
                   [&](int32_t x, int32_t y) { return sub_fl[P.sub_hi[x]] > sub_fl[P.sub_hi[y]]; });
  P.n_task_ids = ns + P.n_trsm + P.n_u + P.n_sub;
  P.n_factor_tasks = P.n_sub;
  P.n_hi_tasks = P.n_sub;
  for (int32_t s = 0; s < ns; ++s)
    if (P.in_sub[s] < 0) {
      P.n_factor_tasks += 1 + P.ntrsm[s] + P.nu[s];
      P.n_hi_tasks += 1 + P.ntrsm[s] + P.nu_hi[s];
    }
  // ---- gather tasks of the fan-in mode (see Plan::gat_first) ---------------------
  P.gat_first.clear();
  P.gat_pc.clear();
  P.pc_owner.clear();
  P.gdiag0.clear();
  P.tdep0.clear();
  P.n_gat = 0;
  if (prm.fanin) {
    const int32_t npc = (int32_t)P.fan_ptr.size() - 1;
    auto npieces = [](int32_t rows) { return (rows + kFanPieceRows - 1) / kFanPieceRows; };
    P.pc_owner.assign(npc, -1);
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s], tr = P.trsm_rows[s];
      for (int32_t m = 0; m < npieces(w); ++m) P.pc_owner[P.fan_task[s] + m] = s;
      for (int32_t k = 0; k < P.ntrsm[s]; ++k) {
        const int32_t kt = P.trsm_first[s] + k;
        for (int32_t m = 0; m < npieces(std::min(tr, r - w - k * tr)); ++m) P.pc_owner[P.fan_task[ns + kt] + m] = ns + kt;
      }
    }
    P.gat_first.assign(ns + 1, 0);
    P.gdiag0.assign(ns, 0);
    P.tdep0.assign(P.n_trsm, 1);
    for (int32_t s = 0; s < ns; ++s) {
      // a panel's pieces are numbered consecutively, from its diagonal block's
      P.gat_first[s] = (int32_t)P.gat_pc.size();
      const int32_t pc_end = s + 1 < ns ? P.fan_task[s + 1] : npc;
      for (int32_t pc = P.fan_task[s]; pc < pc_end; ++pc)
        if (P.fan_ptr[pc + 1] > P.fan_ptr[pc]) {
          P.gat_pc.push_back(pc);
          const int32_t o = P.pc_owner[pc];
          if (o < ns)
            P.gdiag0[s]++;
          else
            P.tdep0[o - ns]++;
        }
    }
    P.gat_first[ns] = (int32_t)P.gat_pc.size();
    P.n_gat = (int32_t)P.gat_pc.size();
    P.n_task_ids += P.n_gat;
    P.n_factor_tasks += P.n_gat;
    P.n_hi_tasks += P.n_gat;
  }

  // ---- solve tasks ------------------------------------------------------------
  // near the root (the critical path of both sweeps) the tiles are shorter
  P.st_first.assign(ns, 0);
  P.nst.assign(ns, 0);
  P.st_rows.assign(ns, 0);
  P.st_sn.clear();
  for (int32_t s = 0; s < ns; ++s) {
    const int32_t nb = P.nrows[s] - (P.fcol[s + 1] - P.fcol[s]);
    const bool top = depth[s] < prm.top_depth;
    const int TS = std::max(1, top ? std::min(prm.top_solve_rows, prm.solve_rows) : prm.solve_rows);
    P.st_rows[s] = TS;
    P.st_first[s] = (int32_t)P.st_sn.size();
    P.nst[s] = (nb + TS - 1) / TS;
    for (int32_t k = 0; k < P.nst[s]; ++k) P.st_sn.push_back(s);
  }
  P.n_st = (int32_t)P.st_sn.size();
  P.n_solve_tasks = 2 * ns + 2 * P.n_st;
  P.woff.assign(ns, -1);
  P.n_w = 0;
  P.n_wpan = 0;
  if (prm.w_depth > 0 && !prm.deterministic)
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t w = P.fcol[s + 1] - P.fcol[s];
      if (depth[s] < prm.w_depth && P.in_sub[s] < 0 && P.nst[s] > 0 && w <= kWMaxWidth) {
        P.woff[s] = P.n_w;
        P.n_w += (int64_t)P.ld[s] * w;
        P.n_wpan++;
      }
    }
  P.st_tptr.assign(P.n_st + 1, 0);
  P.st_tgt.clear();
  std::vector<int32_t> st_rng;  // per st_tgt entry: the tile's rows in that panel, i0 | i1 << 16
  P.fdep0.assign(ns, 0);
  P.bdep0.assign(P.n_st, 0);
  for (int32_t s = 0; s < ns; ++s) {
    const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s];
    const int32_t* R = P.rows.data() + P.rowoff[s];
    const int32_t TS = P.st_rows[s];
    for (int32_t k = 0; k < P.nst[s]; ++k) {
      const int32_t tile = P.st_first[s] + k;
      const int32_t r0 = w + k * TS, r1 = std::min(r, r0 + TS);
      int32_t last = -1;
      for (int32_t i = r0; i < r1; ++i) {
        const int32_t t = P.snode_of[R[i]];
        if (t != last) {  // rows are sorted, so each target appears as one run
          if (last >= 0) st_rng.back() |= (i - r0) << 16;
          P.st_tgt.push_back(t);
          st_rng.push_back(i - r0);
          P.fdep0[t]++;
          last = t;
        }
      }
      if (last >= 0) st_rng.back() |= (r1 - r0) << 16;
      P.st_tptr[tile + 1] = (int32_t)P.st_tgt.size();
      P.bdep0[tile] = (P.st_tptr[tile + 1] - P.st_tptr[tile]) + 1;
    }
  }
  P.ft_sptr.clear();
  P.ft_succ.clear();
  P.ft_dep0.clear();
  if (prm.deterministic && !prm.fanin) {
    // forward tiles: one chain per target panel, in tile order
    P.ft_dep0.assign(P.n_st, 1);
    std::vector<int32_t> last(ns, -1), npred_of(P.n_st, 0);
    std::vector<std::pair<int32_t, int32_t>> edges;  // (predecessor, successor)
    for (int32_t tile = 0; tile < P.n_st; ++tile)
      for (int32_t q = P.st_tptr[tile]; q < P.st_tptr[tile + 1]; ++q) {
        const int32_t t = P.st_tgt[q];
        if (last[t] >= 0) {
          edges.push_back({last[t], tile});
          P.ft_dep0[tile]++;
        }
        last[t] = tile;
      }
    P.ft_sptr.assign(P.n_st + 1, 0);
    for (const auto& e : edges) P.ft_sptr[e.first + 1]++;
    for (int32_t i = 0; i < P.n_st; ++i) P.ft_sptr[i + 1] += P.ft_sptr[i];
    P.ft_succ.resize(edges.size());
    std::vector<int32_t> fill(P.ft_sptr.begin(), P.ft_sptr.end() - 1);
    for (const auto& e : edges) P.ft_succ[fill[e.first]++] = e.second;
    // backward tiles of a panel: a chain in tile order
    for (int32_t s = 0; s < ns; ++s)
      for (int32_t k = 1; k < P.nst[s]; ++k) P.bdep0[P.st_first[s] + k]++;
  }
  P.rt_ptr.assign(ns + 1, 0);
  for (int32_t t : P.st_tgt) P.rt_ptr[t + 1]++;
  for (int32_t s = 0; s < ns; ++s) P.rt_ptr[s + 1] += P.rt_ptr[s];
  P.rt_tile.resize(P.st_tgt.size());
  {
    // each panel's list in descending tile order: the tiles of the nearest
    // descendants -- the next steps of the backward chain -- are released
    // first (and the first becomes the releasing CTA's continuation)
    std::vector<int32_t> fill(P.rt_ptr.begin(), P.rt_ptr.end() - 1);
    P.rt_rng.clear();
    if (prm.fanin) P.rt_rng.resize(P.st_tgt.size());
    for (int32_t tile = P.n_st - 1; tile >= 0; --tile)
      for (int32_t q = P.st_tptr[tile]; q < P.st_tptr[tile + 1]; ++q) {
        const int32_t e = fill[P.st_tgt[q]]++;
        P.rt_tile[e] = tile;
        if (prm.fanin) P.rt_rng[e] = st_rng[q];
      }
  }
  // fan-in solves: the tiles' private buffers (Plan::st_zf)
  P.st_zf.clear();
  P.st_zb.clear();
  P.st_roff.clear();
  P.rt_rec.clear();
  if (prm.fanin) {
    P.st_zf.assign(P.n_st + 1, 0);
    P.st_zb.assign(P.n_st + 1, 0);
    P.st_roff.assign(P.n_st, 0);
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s], TS = P.st_rows[s];
      for (int32_t k = 0; k < P.nst[s]; ++k) {
        const int32_t tile = P.st_first[s] + k, r0 = w + k * TS;
        P.st_zf[tile + 1] = P.st_zf[tile] + std::min(TS, r - r0);
        P.st_zb[tile + 1] = P.st_zb[tile] + w;
        P.st_roff[tile] = P.rowoff[s] + r0;
      }
    }
    P.rt_rec.resize(P.rt_tile.size());
    for (size_t e = 0; e < P.rt_tile.size(); ++e) {
      const int32_t tile = P.rt_tile[e], i0 = P.rt_rng[e] & 0xffff, i1 = P.rt_rng[e] >> 16;
      P.rt_rec[e] = Plan::SolveFanRec{P.st_zf[tile], P.st_roff[tile] + i0, (int32_t)(P.st_zf[tile + 1] - P.st_zf[tile]),
                                       (int16_t)i0, (int16_t)(i1 - i0)};
    }
  }
  P.kid_ptr.assign(ns + 1, 0);
  for (int32_t s = 0; s < ns; ++s)
    if (P.parent[s] != -1) P.kid_ptr[P.parent[s] + 1]++;
  for (int32_t s = 0; s < ns; ++s) P.kid_ptr[s + 1] += P.kid_ptr[s];
  P.kids.resize(P.kid_ptr[ns]);
  {
    std::vector<int32_t> fill(P.kid_ptr.begin(), P.kid_ptr.end() - 1);
    for (int32_t s = 0; s < ns; ++s)
      if (P.parent[s] != -1) P.kids[fill[P.parent[s]]++] = s;
  }
  return 0;
}

}  // namespace spchol
