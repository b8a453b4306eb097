// Fill-reducing ordering for a general symmetric pattern.
//
// Section V applies a fill-reducing symmetric permutation before the
// factorization (the paper takes it from Scotch's nested dissection).  For
// inputs that come without one, this file computes a nested dissection by
// level structures (George, "Nested dissection of a regular finite element
// mesh", SIAM J. Numer. Anal. 10, 1973; George and Liu, "An automatic nested
// dissection algorithm for irregular finite element problems", SIAM J. Numer.
// Anal. 15, 1978):
//   * a connected vertex set is rooted at a pseudo-peripheral vertex (repeated
//     breadth-first search from the far end until the eccentricity stops
//     growing, Gibbs, Poole and Stockmeyer 1976), and its breadth-first level
//     structure is cut at its smallest level that leaves 35 to 65 % of the
//     set below it (the level holding the median vertex if none does);
//   * that level is the separator, less the vertices with no neighbour above
//     it (they separate nothing and join the lower part);
//   * the lower and upper parts are ordered first, recursively (each connected
//     component on its own), and the separator last;
//   * sets of at most kLeaf vertices are ordered by minimum degree on their
//     elimination graph (Tinney and Walker's scheme 2, restated: repeatedly
//     eliminate a vertex of least current degree, joining its neighbours).
// Host code only; it needs no GPU.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "spchol.h"

namespace spchol {
namespace {

constexpr int kLeaf = 64;  // vertex sets this small are ordered by minimum degree

struct Graph {
  std::vector<int64_t> xadj;  // symmetric adjacency, no self loops
  std::vector<int32_t> adj;
};

void build_graph(int64_t n, const int64_t* colptr, const int32_t* rowind, Graph& g) {
  g.xadj.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p)
      if (rowind[p] != j) {
        g.xadj[j + 1]++;
        g.xadj[rowind[p] + 1]++;
      }
  for (int64_t j = 0; j < n; ++j) g.xadj[j + 1] += g.xadj[j];
  g.adj.resize(g.xadj[n]);
  std::vector<int64_t> fill(g.xadj.begin(), g.xadj.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p)
      if (rowind[p] != j) {
        g.adj[fill[j]++] = rowind[p];
        g.adj[fill[rowind[p]]++] = (int32_t)j;
      }
}

struct Dissection {
  const Graph& g;
  std::vector<int64_t>& perm;       // new -> old, filled by position
  std::vector<int32_t> stamp;       // set id a vertex currently belongs to
  std::vector<int32_t> level;       // breadth-first level (scratch)
  int32_t next_stamp = 1;

  Dissection(const Graph& gr, int64_t n, std::vector<int64_t>& p) : g(gr), perm(p), stamp(n, 0), level(n, -1) {}

  int32_t mark(const std::vector<int32_t>& vs) {
    const int32_t s = next_stamp++;
    for (int32_t v : vs) stamp[v] = s;
    return s;
  }

  // Breadth-first search from root inside the set with stamp s; returns the
  // vertices in visiting order and sets level[] for them (and leaves level[]
  // of other vertices of the set at -1 if unreached: callers reset it).
  void bfs(int32_t root, int32_t s, std::vector<int32_t>& order) {
    order.clear();
    order.push_back(root);
    level[root] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
      const int32_t v = order[h];
      for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
        const int32_t u = g.adj[p];
        if (stamp[u] == s && level[u] < 0) {
          level[u] = level[v] + 1;
          order.push_back(u);
        }
      }
    }
  }

  void clear_levels(const std::vector<int32_t>& vs) {
    for (int32_t v : vs) level[v] = -1;
  }

  int32_t degree_in(int32_t v, int32_t s) const {
    int32_t d = 0;
    for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) d += stamp[g.adj[p]] == s;
    return d;
  }

  // Minimum-degree order of a small set (at most 64 vertices) on its induced
  // subgraph, written to perm[pos ...].
  void order_leaf(const std::vector<int32_t>& vs, int64_t pos) {
    const int m = (int)vs.size();
    const int32_t s = mark(vs);
    // local index of each vertex: reuse level[] as scratch
    for (int i = 0; i < m; ++i) level[vs[i]] = i;
    std::vector<uint64_t> nb(m, 0ull);
    for (int i = 0; i < m; ++i)
      for (int64_t p = g.xadj[vs[i]]; p < g.xadj[vs[i] + 1]; ++p) {
        const int32_t u = g.adj[p];
        if (stamp[u] == s) nb[i] |= 1ull << level[u];
      }
    for (int i = 0; i < m; ++i) level[vs[i]] = -1;
    uint64_t alive = m == 64 ? ~0ull : ((1ull << m) - 1);
    for (int k = 0; k < m; ++k) {
      int best = -1, bd = 1 << 30;
      for (int i = 0; i < m; ++i)
        if ((alive >> i) & 1ull) {
          const int d = __builtin_popcountll(nb[i] & alive);
          if (d < bd) {
            bd = d;
            best = i;
          }
        }
      perm[pos + k] = vs[best];
      alive &= ~(1ull << best);
      const uint64_t nbr = nb[best] & alive;
      for (int i = 0; i < m; ++i)
        if ((nbr >> i) & 1ull) nb[i] |= nbr & ~(1ull << i);
    }
  }

  struct Item {
    std::vector<int32_t> vs;
    int64_t pos;  // first position of this set in the ordering
  };

  void run(std::vector<int32_t> all) {
    std::vector<Item> stack;
    stack.push_back({std::move(all), 0});
    std::vector<int32_t> order;
    while (!stack.empty()) {
      Item it = std::move(stack.back());
      stack.pop_back();
      std::vector<int32_t>& vs = it.vs;
      if (vs.empty()) continue;
      if ((int)vs.size() <= kLeaf) {
        order_leaf(vs, it.pos);
        continue;
      }
      const int32_t s = mark(vs);
      // connected components: each becomes an item of its own
      bfs(vs[0], s, order);
      if (order.size() < vs.size()) {
        int64_t pos = it.pos;
        std::vector<Item> parts;
        for (int32_t v : vs) {
          if (level[v] >= 0) continue;
          std::vector<int32_t> more;
          bfs(v, s, more);
          parts.push_back({std::move(more), 0});
        }
        parts.push_back({order, 0});
        clear_levels(vs);
        for (Item& p : parts) {
          p.pos = pos;
          pos += (int64_t)p.vs.size();
          stack.push_back(std::move(p));
        }
        continue;
      }
      // pseudo-peripheral root: restart from a vertex of least degree in the
      // last level while the eccentricity grows
      int32_t root = vs[0];
      {
        int32_t bestd = degree_in(root, s);
        for (int32_t v : vs) {
          const int32_t d = degree_in(v, s);
          if (d < bestd) {
            bestd = d;
            root = v;
          }
        }
      }
      clear_levels(vs);
      bfs(root, s, order);
      int32_t ecc = level[order.back()];
      for (int round = 0; round < 8; ++round) {
        int32_t cand = order.back(), cd = degree_in(cand, s);
        for (size_t h = order.size(); h-- > 0 && level[order[h]] == ecc;) {
          const int32_t d = degree_in(order[h], s);
          if (d < cd) {
            cd = d;
            cand = order[h];
          }
        }
        clear_levels(vs);
        bfs(cand, s, order);
        const int32_t e2 = level[order.back()];
        if (e2 <= ecc) {
          clear_levels(vs);
          bfs(root, s, order);
          break;
        }
        root = cand;
        ecc = e2;
      }
      const int32_t h = level[order.back()];
      const int64_t m = (int64_t)vs.size();
      if (h < 2) {  // no level can separate (a clique-like set): any order fills it
        for (int64_t k = 0; k < m; ++k) perm[it.pos + k] = order[k];
        clear_levels(vs);
        continue;
      }
      // the separating level: the smallest level whose lower part holds 35 to
      // 65 % of the set (else the one holding the median vertex), kept
      // strictly inside (1 .. h-1) so that both parts are non-empty
      std::vector<int64_t> cnt(h + 1, 0);
      for (int32_t v : order) cnt[level[v]]++;
      int32_t k = 1;
      for (int64_t acc = cnt[0]; k < h - 1 && acc + cnt[k] < m / 2; ++k) acc += cnt[k];
      {
        int64_t below = 0;
        for (int32_t l = 0; l < h; ++l) {
          if (l >= 1 && 20 * below >= 7 * m && 20 * below <= 13 * m && cnt[l] < cnt[k]) k = l;
          below += cnt[l];
        }
      }
      std::vector<int32_t> lower, upper, sep;
      for (int32_t v : order) {
        const int32_t l = level[v];
        if (l < k) {
          lower.push_back(v);
        } else if (l > k) {
          upper.push_back(v);
        } else {
          bool touches_upper = false;
          for (int64_t p = g.xadj[v]; p < g.xadj[v + 1] && !touches_upper; ++p) {
            const int32_t u = g.adj[p];
            touches_upper = stamp[u] == s && level[u] == k + 1;
          }
          (touches_upper ? sep : lower).push_back(v);
        }
      }
      clear_levels(vs);
      const int64_t p0 = it.pos, p1 = p0 + (int64_t)lower.size(), p2 = p1 + (int64_t)upper.size();
      for (size_t i = 0; i < sep.size(); ++i) perm[p2 + (int64_t)i] = sep[i];
      stack.push_back({std::move(upper), p1});
      stack.push_back({std::move(lower), p0});
    }
  }
};

}  // namespace
}  // namespace spchol

extern "C" int spchol_order_nd(int64_t n, const int64_t* colptr, const int32_t* rowind, int64_t* perm_out) {
  if (n < 0 || n > INT32_MAX - 1) return -1;
  if (n > 0 && (!colptr || colptr[0] != 0)) return -2;
  for (int64_t j = 0; j < n; ++j)
    if (colptr[j + 1] < colptr[j]) return -2;
  const int64_t nnz = n > 0 ? colptr[n] : 0;
  if (nnz > 0 && !rowind) return -3;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      const int32_t r = rowind[p];
      if (r < j || r >= n) return -3;
      if (p > colptr[j] && r <= rowind[p - 1]) return -3;
    }
  if (n > 0 && !perm_out) return -4;
  if (n == 0) return 0;
  spchol::Graph g;
  spchol::build_graph(n, colptr, rowind, g);
  std::vector<int64_t> perm(n, -1);
  std::vector<int32_t> all(n);
  for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
  spchol::Dissection d(g, n, perm);
  d.run(std::move(all));
  std::memcpy(perm_out, perm.data(), (size_t)n * sizeof(int64_t));
  return 0;
}
