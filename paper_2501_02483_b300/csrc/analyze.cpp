// Host-side symbolic analysis: input validation, partial RCM ordering
// (Section III.A), the CTSF tile map (Section III.B), the tile-level symbolic
// factorization (Section II, step 2), task flop counts, and the device task
// graph of the factorization and of the solves.
//
// Nothing here touches the GPU; stiles_analyze can run on any host.

#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <thread>

#include "plan.h"

namespace stiles {

void default_opts(stiles_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->tile = 32;
  o->ordering = STILES_ORDER_AUTO;
  o->precision = STILES_PREC_F64;
  o->block = 0;
  o->tree_chunk = 32;
  o->tree_fanin = 16;
  o->max_refine = 20;
  o->refine_tol = 1e-10;
  o->spin_limit = int64_t(1) << 24;
}

namespace {

// ---------------------------------------------------------------------------
// Partial Reverse Cuthill-McKee on the body block [0, nb).
// Tie-breaks (the paper leaves them open): degree = number of distinct body
// neighbours; components in order of their smallest vertex; George-Liu
// pseudo-peripheral start found from the min-(degree, index) vertex of the
// component, moving to the min-(degree, index) vertex of the last BFS level
// while the level structure gets strictly deeper; neighbours enqueued in
// ascending (degree, index); the body sequence is reversed at the end.
// ---------------------------------------------------------------------------
struct Graph {
  int64_t nb = 0;
  std::vector<int64_t> ptr, adj;
  int64_t deg(int64_t v) const { return ptr[v + 1] - ptr[v]; }
};

Graph body_graph(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t nb) {
  Graph g;
  g.nb = nb;
  std::vector<int64_t> cnt(nb + 1, 0);
  for (int64_t j = 0; j < nb; ++j)
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      int64_t i = rowidx[e];
      if (i != j && i < nb) { ++cnt[i]; ++cnt[j]; }
    }
  g.ptr.assign(nb + 1, 0);
  for (int64_t v = 0; v < nb; ++v) g.ptr[v + 1] = g.ptr[v] + cnt[v];
  g.adj.resize(g.ptr[nb]);
  std::vector<int64_t> fill(g.ptr.begin(), g.ptr.end() - 1);
  for (int64_t j = 0; j < nb; ++j)
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      int64_t i = rowidx[e];
      if (i != j && i < nb) { g.adj[fill[i]++] = j; g.adj[fill[j]++] = i; }
    }
  for (int64_t v = 0; v < nb; ++v) std::sort(g.adj.begin() + g.ptr[v], g.adj.begin() + g.ptr[v + 1]);
  (void)n;
  return g;
}

struct Levels {
  std::vector<int64_t> verts;  // BFS visit order
  std::vector<int64_t> start;  // level l = verts[start[l] .. start[l+1])
  int64_t depth() const { return int64_t(start.size()) - 1; }
};

void bfs_levels(const Graph& g, int64_t root, std::vector<int64_t>& stamp, int64_t& mark, Levels& L) {
  ++mark;
  L.verts.clear();
  L.start.clear();
  L.verts.push_back(root);
  stamp[root] = mark;
  L.start.push_back(0);
  size_t b = 0;
  while (true) {
    size_t e = L.verts.size();
    for (size_t idx = b; idx < e; ++idx) {
      int64_t v = L.verts[idx];
      for (int64_t a = g.ptr[v]; a < g.ptr[v + 1]; ++a) {
        int64_t u = g.adj[a];
        if (stamp[u] != mark) { stamp[u] = mark; L.verts.push_back(u); }
      }
    }
    L.start.push_back(int64_t(e));
    if (L.verts.size() == e) break;
    b = e;
  }
}

int64_t min_deg_index(const Graph& g, const int64_t* v, size_t cnt) {
  int64_t best = v[0];
  for (size_t i = 1; i < cnt; ++i) {
    int64_t u = v[i];
    if (g.deg(u) < g.deg(best) || (g.deg(u) == g.deg(best) && u < best)) best = u;
  }
  return best;
}

std::vector<int64_t> partial_rcm(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow) {
  const int64_t nb = n - n_arrow;
  Graph g = body_graph(n, colptr, rowidx, nb);
  std::vector<int64_t> stamp(nb, 0);
  int64_t mark = 0;
  std::vector<char> visited(nb, 0);
  std::vector<int64_t> seq;
  seq.reserve(nb);
  Levels comp, lr, lx;
  std::vector<int64_t> tmp;
  for (int64_t v = 0; v < nb; ++v) {
    if (visited[v]) continue;
    bfs_levels(g, v, stamp, mark, comp);
    int64_t r = min_deg_index(g, comp.verts.data(), comp.verts.size());
    bfs_levels(g, r, stamp, mark, lr);
    while (true) {
      const int64_t* last = lr.verts.data() + lr.start[lr.depth() - 1];
      size_t nlast = lr.verts.size() - size_t(lr.start[lr.depth() - 1]);
      int64_t x = min_deg_index(g, last, nlast);
      bfs_levels(g, x, stamp, mark, lx);
      if (lx.depth() > lr.depth()) { r = x; std::swap(lr, lx); }
      else break;
    }
    // Cuthill-McKee from r
    size_t head = seq.size();
    seq.push_back(r);
    visited[r] = 1;
    while (head < seq.size()) {
      int64_t u = seq[head++];
      tmp.clear();
      for (int64_t a = g.ptr[u]; a < g.ptr[u + 1]; ++a)
        if (!visited[g.adj[a]]) tmp.push_back(g.adj[a]);
      std::sort(tmp.begin(), tmp.end(), [&](int64_t x, int64_t y) {
        return g.deg(x) < g.deg(y) || (g.deg(x) == g.deg(y) && x < y);
      });
      for (int64_t w : tmp) { visited[w] = 1; seq.push_back(w); }
    }
  }
  std::reverse(seq.begin(), seq.end());
  for (int64_t a = nb; a < n; ++a) seq.push_back(a);
  return seq;
}

// ---------------------------------------------------------------------------
// Adaptable nested dissection, one level (Section III.A): split the body at
// mid = nb / 2 rounded down to a multiple of the tile size, take as separator
// every row in [mid, nb) that a column left of mid reaches, and order [0, mid),
// then the rest of the body reversed, then the separator, then the arrow.
// Both parts meet the separator with their last rows, so they are independent
// elimination chains (also at the tile level, the split being tile-aligned).
// ---------------------------------------------------------------------------
std::vector<int64_t> adaptable_nd(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                                  int64_t align) {
  const int64_t nb = n - n_arrow;
  std::vector<int64_t> perm;
  perm.reserve(n);
  // split at nb / 2 rounded down to a tile boundary: a tile holding rows of
  // both parts would join the two elimination chains again at the tile level
  const int64_t mid = (nb / 2) / align * align;
  if (nb < 2 || mid == 0) {
    for (int64_t i = 0; i < n; ++i) perm.push_back(i);
    return perm;
  }
  int64_t s_end = mid;
  for (int64_t j = 0; j < mid; ++j)
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      const int64_t i = rowidx[e];
      if (i >= mid && i < nb) s_end = std::max(s_end, i + 1);
    }
  for (int64_t i = 0; i < mid; ++i) perm.push_back(i);
  for (int64_t i = nb - 1; i >= s_end; --i) perm.push_back(i);
  for (int64_t i = mid; i < s_end; ++i) perm.push_back(i);
  for (int64_t i = nb; i < n; ++i) perm.push_back(i);
  return perm;
}

// ---------------------------------------------------------------------------
// Tile map and tile-level symbolic factorization.  cols[J] = sorted rows I > J
// of the present lower tiles of column J.  The closure follows the elimination
// tree: the structure of tile column k (minus its first row p) is merged into
// column p, which yields the same map as adding every pair of S_k.
// ---------------------------------------------------------------------------
// Tile row/column of every original index under the permutation: tile of
// position iperm[i] (avoids a division per entry in the O(nnz) passes).
std::vector<int32_t> tile_of_index(int64_t n, const std::vector<int64_t>& iperm, int64_t T) {
  std::vector<int32_t> t(n);
  for (int64_t i = 0; i < n; ++i) t[i] = int32_t(iperm[i] / T);
  return t;
}

std::vector<std::vector<int32_t>> tile_columns(int64_t n, const int64_t* colptr, const int32_t* rowidx,
                                               const std::vector<int64_t>& iperm, int64_t T, int64_t nt) {
  const std::vector<int32_t> tile = tile_of_index(n, iperm, T);
  // bucket the entries of P A P^T (flipped to the lower triangle) by tile column
  std::vector<int64_t> cnt(nt + 1, 0);
  for (int64_t j = 0; j < n; ++j) {
    const int32_t tq = tile[j];
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      const int32_t tp = tile[rowidx[e]];
      if (tp != tq) ++cnt[std::min(tp, tq) + 1];
    }
  }
  for (int64_t J = 0; J < nt; ++J) cnt[J + 1] += cnt[J];
  std::vector<int32_t> rows(cnt[nt]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t j = 0; j < n; ++j) {
    const int32_t tq = tile[j];
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      const int32_t tp = tile[rowidx[e]];
      if (tp != tq) rows[fill[std::min(tp, tq)]++] = std::max(tp, tq);
    }
  }
  std::vector<std::vector<int32_t>> cols(nt);
  std::vector<int64_t> stamp(nt, -1);
  for (int64_t J = 0; J < nt; ++J) {
    auto& cj = cols[J];
    for (int64_t e = cnt[J]; e < cnt[J + 1]; ++e) {
      int32_t I = rows[e];
      if (stamp[I] != J) { stamp[I] = J; cj.push_back(I); }
    }
    std::sort(cj.begin(), cj.end());
  }
  // symbolic closure along the elimination tree
  std::vector<int32_t> merged;
  for (int64_t k = 0; k < nt; ++k) {
    const auto& s = cols[k];
    if (s.size() < 2) continue;
    int32_t par = s[0];
    auto& cp = cols[par];
    merged.clear();
    std::set_union(cp.begin(), cp.end(), s.begin() + 1, s.end(), std::back_inserter(merged));
    cp.swap(merged);
  }
  return cols;
}

int64_t count_tiles(const std::vector<std::vector<int32_t>>& cols) {
  int64_t c = int64_t(cols.size());
  for (const auto& v : cols) c += int64_t(v.size());
  return c;
}

// Tree split of an accumulation list (Algorithm 3): the first chunks of
// `chunk` terms become leaves, leaves are summed by nodes of `fanin`
// children until at most `fanin` remain; the owning task keeps the last
// chunk and subtracts the remaining tree roots.
struct TreeNode {
  int32_t type;        // leaf or combine
  int32_t scratch;     // output scratch index
  int64_t pb, pe;      // leaf: range in the pair list
  std::vector<int32_t> children;  // combine: indices into the node list
  int64_t release;     // leaf: primary position of the last producer
  int64_t owner;       // leaf: primary task whose pairs it sums
};

constexpr int kTargetShift = 30;  // bit of a pair/partial index naming the CHAIN accumulator
constexpr int64_t kChainKeep = 3;  // newest terms a diagonal-chain task applies itself
constexpr int64_t kSweepKeep = 8;  // newest terms a sweep task keeps when its list is split into leaves
constexpr double kSplitFlopsPerStep = 1e7;  // below: the chain runs on reserved SMs
constexpr int32_t kIndexMask = (1 << 30) - 1;

inline void set_col(DevTask& t, int32_t c) { t.col = c; }
inline void set_col(SolveTask& t, int32_t c) { t.pad0 = c; }
// row and column block of the tile a factor task's first accumulator updates
inline void set_target(DevTask& t, int32_t row, int32_t col) {
  t.trow = row;
  t.tcol = col;
}
inline void set_target(SolveTask&, int32_t, int32_t) {}

}  // namespace

// ---------------------------------------------------------------------------
// Task graph builder shared by the factorization and the two solve sweeps.
// Primary tasks come in a fixed order; each has a list of pairs whose
// producers are earlier primary tasks.  Leaves are emitted right after their
// last producer, combines right after their last child, so every task's
// dependencies carry smaller tickets.
// ---------------------------------------------------------------------------
namespace {

struct PairList {
  std::vector<int32_t> pairs;      // 2 per pair
  std::vector<int64_t> producers;  // per pair: max primary position of the two producers
};

struct Primary {
  int32_t type, out, diag, col;
  int32_t row = -1;                // block row of `out` (factorization)
  int32_t out2 = -1, col2 = -1;    // CHAIN: second output
  PairList list[2];                // list[1] only for CHAIN
};

inline void set_second(DevTask& t, const Primary& p, int32_t pb, int32_t pe, int32_t qb, int32_t qe) {
  t.out2 = p.out2;
  t.col2 = p.col2;
  t.pb2 = pb;
  t.pe2 = pe;
  t.qb2 = qb;
  t.qe2 = qe;
}
inline void set_second(SolveTask&, const Primary&, int32_t, int32_t, int32_t, int32_t) {}
inline void clear_second(DevTask& t) {
  t.out2 = t.col2 = -1;
  t.pb2 = t.pe2 = t.qb2 = t.qe2 = 0;
}
inline void clear_second(SolveTask&) {}

// keep_types / keep: primaries of a type in keep_types (a bit mask) keep only
// their last `keep` terms; every earlier term goes to tree leaves.  Used for
// the diagonal chain of the factorization: its tasks are the critical path,
// so the sums of the old band terms are formed ahead of time by other CTAs
// (Algorithm 3 applied to band rows) and the chain task applies only the
// newest terms plus one partial.
// min_own: a primary whose list is split into leaves by the chunk rule keeps at
// least its newest min_own terms.  Used for the sweeps: a leaf holding one of a
// chain block's newest inputs is finished one step before its owner at best, so
// the chain would cross SMs twice per block (leaf, then owner).  With min_own > 0
// every list is first stably sorted by producer position, so the kept tail holds
// the newest terms whatever the order the list was built in (under nested
// dissection a block's index order is not its producers' order).
template <class Task>
void build_graph(std::vector<Primary>& prim, int64_t chunk, int64_t fanin, int32_t leaf_type, int32_t comb_type,
                 std::vector<Task>& tasks, std::vector<int32_t>& pairs, std::vector<int32_t>& parts,
                 int64_t& nscratch, uint32_t keep_types = 0, int64_t keep = 0, int64_t min_own = 0) {
  const int64_t np = int64_t(prim.size());
  if (min_own > 0) {
    std::vector<int64_t> idx;
    std::vector<int32_t> pairs_s;
    std::vector<int64_t> prod_s;
    for (Primary& pr : prim)
      for (PairList& pl : pr.list) {
        const size_t n = pl.producers.size();
        if (n < 2 || std::is_sorted(pl.producers.begin(), pl.producers.end())) continue;
        idx.resize(n);
        for (size_t q = 0; q < n; ++q) idx[q] = int64_t(q);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int64_t a, int64_t b) { return pl.producers[a] < pl.producers[b]; });
        pairs_s.resize(2 * n);
        prod_s.resize(n);
        for (size_t q = 0; q < n; ++q) {
          pairs_s[2 * q] = pl.pairs[2 * idx[q]];
          pairs_s[2 * q + 1] = pl.pairs[2 * idx[q] + 1];
          prod_s[q] = pl.producers[idx[q]];
        }
        pl.pairs.swap(pairs_s);
        pl.producers.swap(prod_s);
      }
  }
  std::vector<TreeNode> nodes;
  std::vector<int32_t> node_list;                     // which list of its owner a node belongs to
  std::vector<std::vector<int32_t>> roots(2 * np);    // per (primary, list): top-level tree nodes
  std::vector<std::vector<int32_t>> by_release(np);   // leaves by release position
  std::vector<int32_t> parent;
  std::vector<int32_t> pending;
  std::vector<int64_t> own_begin(2 * np, 0);
  for (int64_t t = 0; t < np; ++t)
    for (int l = 0; l < 2; ++l) {
      const PairList& pl = prim[t].list[l];
      const int64_t npairs = int64_t(pl.pairs.size() / 2);
      // terms [0, split) go to leaves of at most `chunk` terms, the owner keeps the rest
      int64_t split = 0;
      if (keep > 0 && ((keep_types >> prim[t].type) & 1u)) {
        if (npairs > keep + 1) split = npairs - keep;
      } else if (npairs > chunk) {
        split = ((npairs + chunk - 1) / chunk - 1) * chunk;
        if (npairs - split < min_own) split = std::max<int64_t>(0, npairs - min_own);
      }
      if (split == 0) continue;
      const int64_t nleaves = (split + chunk - 1) / chunk;
      std::vector<int32_t> level;
      for (int64_t c = 0; c < nleaves; ++c) {
        TreeNode nd;
        nd.type = leaf_type;
        nd.scratch = int32_t(nscratch++);
        nd.pb = c * chunk;
        nd.pe = std::min(split, (c + 1) * chunk);
        int64_t rel = 0;
        for (int64_t q = nd.pb; q < nd.pe; ++q) rel = std::max(rel, pl.producers[q]);
        nd.release = rel;
        nd.owner = t;
        level.push_back(int32_t(nodes.size()));
        by_release[rel].push_back(int32_t(nodes.size()));
        nodes.push_back(nd);
        node_list.push_back(l);
        parent.push_back(-1);
        pending.push_back(0);
      }
      own_begin[2 * t + l] = split;
      while (int64_t(level.size()) > fanin) {
        std::vector<int32_t> next;
        for (size_t g = 0; g < level.size(); g += size_t(fanin)) {
          TreeNode nd;
          nd.type = comb_type;
          nd.scratch = int32_t(nscratch++);
          nd.pb = nd.pe = 0;
          nd.release = -1;
          nd.owner = t;
          const size_t e = std::min(level.size(), g + size_t(fanin));
          const int32_t id = int32_t(nodes.size());
          for (size_t q = g; q < e; ++q) {
            nd.children.push_back(level[q]);
            parent[level[q]] = id;
          }
          nodes.push_back(nd);
          node_list.push_back(l);
          parent.push_back(-1);
          pending.push_back(int32_t(e - g));
          next.push_back(id);
        }
        level.swap(next);
      }
      roots[2 * t + l] = level;
    }
  // emission
  tasks.clear();
  pairs.clear();
  parts.clear();
  std::vector<int64_t> ticket_of_node(nodes.size(), -1);
  std::vector<int32_t> stack;
  auto emit_node = [&](int32_t id) {
    TreeNode& nd = nodes[id];
    Task tk{};
    tk.type = nd.type;
    tk.out = nd.scratch;
    tk.diag = -1;
    clear_second(tk);
    {
      const Primary& ow = prim[nd.owner];
      if (node_list[id] == 0) set_target(tk, ow.row, ow.col);
      else set_target(tk, ow.col2, ow.col2);
    }
    if (nd.type == leaf_type) {
      const PairList& pl = prim[nd.owner].list[node_list[id]];
      tk.pb = int32_t(pairs.size() / 2);
      pairs.insert(pairs.end(), pl.pairs.begin() + 2 * nd.pb, pl.pairs.begin() + 2 * nd.pe);
      tk.pe = int32_t(pairs.size() / 2);
      tk.qb = tk.qe = int32_t(parts.size());
    } else {
      tk.pb = tk.pe = int32_t(pairs.size() / 2);
      tk.qb = int32_t(parts.size());
      for (int32_t c : nd.children) parts.push_back(nodes[c].scratch);
      tk.qe = int32_t(parts.size());
    }
    ticket_of_node[id] = int64_t(tasks.size());
    tasks.push_back(tk);
  };
  // The primary's own terms of both lists are merged in the order their producers
  // run, each tagged with its target accumulator (bit 30 of the first index), so a
  // late term never holds back terms that are ready; tree roots (older sums) and
  // own terms share that encoding.
  struct OwnItem {
    int64_t prod;
    int32_t a, b;
  };
  std::vector<OwnItem> own;
  for (int64_t t = 0; t < np; ++t) {
    Primary& pr = prim[t];
    Task tk{};
    tk.type = pr.type;
    tk.out = pr.out;
    tk.diag = pr.diag;
    own.clear();
    const int nl = pr.out2 >= 0 ? 2 : 1;
    for (int l = 0; l < nl; ++l) {
      const PairList& pl = pr.list[l];
      for (size_t q = size_t(own_begin[2 * t + l]); q < pl.producers.size(); ++q)
        own.push_back(OwnItem{pl.producers[q], pl.pairs[2 * q] | (l << kTargetShift), pl.pairs[2 * q + 1]});
    }
    if (nl == 2)
      std::stable_sort(own.begin(), own.end(), [](const OwnItem& x, const OwnItem& y) { return x.prod < y.prod; });
    tk.pb = int32_t(pairs.size() / 2);
    for (const OwnItem& it : own) {
      pairs.push_back(it.a);
      pairs.push_back(it.b);
    }
    tk.pe = int32_t(pairs.size() / 2);
    tk.qb = int32_t(parts.size());
    for (int l = 0; l < nl; ++l)
      for (int32_t r : roots[2 * t + l]) {
        if (ticket_of_node[r] < 0) throw std::logic_error("tree root emitted after its owner");
        parts.push_back(nodes[r].scratch | (l << kTargetShift));
      }
    tk.qe = int32_t(parts.size());
    if (pr.out2 >= 0) set_second(tk, pr, 0, 0, 0, 0);
    else clear_second(tk);
    set_col(tk, pr.col);
    set_target(tk, pr.row, pr.col);
    tasks.push_back(tk);
    // leaves released by this primary, then any combine that became complete
    for (int32_t leaf : by_release[t]) {
      stack.assign(1, leaf);
      while (!stack.empty()) {
        const int32_t id = stack.back();
        stack.pop_back();
        emit_node(id);
        const int32_t p = parent[id];
        if (p >= 0 && --pending[p] == 0) stack.push_back(p);
      }
    }
  }
  for (size_t i = 0; i < nodes.size(); ++i)
    if (ticket_of_node[i] < 0) throw std::logic_error("tree node never emitted");
}

}  // namespace

namespace {

bool validate(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow, std::string* err) {
  if (n < 1 || n > (int64_t(1) << 31) - 1) { *err = "n must be in [1, 2^31)"; return false; }
  if (!colptr || !rowidx) { *err = "null colptr/rowidx"; return false; }
  if (n_arrow < 0 || n_arrow > n) { *err = "n_arrow must be in [0, n]"; return false; }
  if (colptr[0] != 0) { *err = "colptr[0] != 0"; return false; }
  for (int64_t j = 0; j < n; ++j) {
    if (colptr[j + 1] < colptr[j]) { *err = "colptr not nondecreasing at column " + std::to_string(j); return false; }
    if (colptr[j + 1] == colptr[j] || rowidx[colptr[j]] != j) {
      *err = "missing diagonal (or upper-triangle entry) in column " + std::to_string(j);
      return false;
    }
    for (int64_t e = colptr[j] + 1; e < colptr[j + 1]; ++e) {
      if (rowidx[e] <= rowidx[e - 1] || rowidx[e] >= n) {
        *err = "rows not strictly ascending / out of range in column " + std::to_string(j);
        return false;
      }
    }
  }
  return true;
}

std::vector<int64_t> invert(const std::vector<int64_t>& perm) {
  std::vector<int64_t> inv(perm.size());
  for (size_t i = 0; i < perm.size(); ++i) inv[perm[i]] = int64_t(i);
  return inv;
}

struct Second {
  int32_t out = -1, pb = 0, pe = 0, qb = 0, qe = 0;
};
inline Second second_of(const DevTask& t) { return Second{t.out2, t.pb2, t.pe2, t.qb2, t.qe2}; }
inline Second second_of(const SolveTask&) { return Second{}; }

// Ticket-order check: the producer of every tile (or block) a task reads must
// have a smaller ticket.  For solve graphs the second member of a pair is a
// block index; for the factorization both members are sub-tile indices.
template <class Task>
bool check_order(const std::vector<Task>& tasks, const std::vector<int32_t>& pairs, const std::vector<int32_t>& parts,
                 int64_t nout, int64_t nscratch, int32_t leaf, int32_t comb, bool solve, std::string* err) {
  std::vector<int64_t> tout(nout, -1), tscr(nscratch, -1);
  for (size_t t = 0; t < tasks.size(); ++t) {
    const Task& tk = tasks[t];
    if (tk.type == leaf || tk.type == comb) {
      if (tk.out < 0 || tk.out >= nscratch || tscr[tk.out] >= 0) { *err = "internal: bad scratch output"; return false; }
      tscr[tk.out] = int64_t(t);
    } else {
      if (tk.out < 0 || tk.out >= nout || tout[tk.out] >= 0) { *err = "internal: bad task output"; return false; }
      tout[tk.out] = int64_t(t);
      const Second s2 = second_of(tk);
      if (s2.out >= 0) {
        if (s2.out >= nout || tout[s2.out] >= 0) { *err = "internal: bad second output"; return false; }
        tout[s2.out] = int64_t(t);
      }
    }
  }
  auto check_range = [&](size_t t, int32_t pb, int32_t pe, int32_t qb, int32_t qe) {
    for (int32_t q = pb; q < pe; ++q) {
      const int64_t a = pairs[2 * size_t(q)] & kIndexMask, b = pairs[2 * size_t(q) + 1];
      const int64_t ta = solve ? -2 : tout[a];
      const int64_t tb = tout[b];
      if ((!solve && (ta < 0 || ta >= int64_t(t))) || tb < 0 || tb >= int64_t(t)) {
        *err = "internal: task " + std::to_string(t) + " reads a tile produced later";
        return false;
      }
    }
    for (int32_t q = qb; q < qe; ++q) {
      const int64_t ts = tscr[parts[q] & kIndexMask];
      if (ts < 0 || ts >= int64_t(t)) {
        *err = "internal: partial produced later";
        return false;
      }
    }
    return true;
  };
  for (size_t t = 0; t < tasks.size(); ++t) {
    const Task& tk = tasks[t];
    if (!check_range(t, tk.pb, tk.pe, tk.qb, tk.qe)) return false;
    const Second s2 = second_of(tk);
    if (s2.out >= 0 && !check_range(t, s2.pb, s2.pe, s2.qb, s2.qe)) return false;
    if (!solve && tk.diag >= 0 && (tout[tk.diag] < 0 || tout[tk.diag] >= int64_t(t))) {
      *err = "internal: diagonal tile produced later";
      return false;
    }
  }
  return true;
}

struct SubEntry {
  int32_t idx;  // sub-row (in a column list) or sub-column (in a row list)
  int32_t sub;  // sub-tile index
};

}  // namespace

stiles_status build_plan(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                         const stiles_opts& opts_in, stiles_plan* p, std::string* err) {
  stiles_opts o = opts_in;
  if (o.tile < 1) { *err = "tile must be >= 1"; return STILES_ERR_INVALID; }
  if (o.ordering < 0 || o.ordering > 3) { *err = "unknown ordering"; return STILES_ERR_INVALID; }
  if (o.precision < 0 || o.precision > 3) { *err = "unknown precision"; return STILES_ERR_INVALID; }
  if (o.tree_chunk <= 0) o.tree_chunk = 32;
  if (o.tree_fanin <= 1) o.tree_fanin = 16;
  if (o.max_refine <= 0) o.max_refine = 20;
  if (!(o.refine_tol > 0)) o.refine_tol = 1e-10;
  if (o.spin_limit <= 0) o.spin_limit = int64_t(1) << 24;
  if (o.block != 0 && o.block != 16 && o.block != 32 && o.block != 64) {
    *err = "block must be 0, 16, 32 or 64";
    return STILES_ERR_INVALID;
  }
  if (!validate(n, colptr, rowidx, n_arrow, err)) return STILES_ERR_INVALID;
  const int64_t nnz = colptr[n];
  const int64_t T = o.tile;
  p->opts = o;
  p->n = n;
  p->n_arrow = n_arrow;
  p->nnz = nnz;
  p->T = int32_t(T);
  p->colptr.assign(colptr, colptr + n + 1);
  p->rowidx.assign(rowidx, rowidx + nnz);
  // CSR index of the strict lower part (the residual y = A x gathers row i's
  // entries j < i from it and column i's entries from the CSC)
  p->rptr.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e)
      if (rowidx[e] != j) ++p->rptr[rowidx[e] + 1];
  for (int64_t i = 0; i < n; ++i) p->rptr[i + 1] += p->rptr[i];
  p->rcol.resize(p->rptr[n]);
  p->rval.resize(p->rptr[n]);
  {
    std::vector<int64_t> fill(p->rptr.begin(), p->rptr.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
        const int64_t i = rowidx[e];
        if (i == j) continue;
        p->rcol[fill[i]] = int32_t(j);
        p->rval[fill[i]++] = e;
      }
  }
  const int64_t nt = (n + T - 1) / T;
  p->nt = nt;

  // ordering (Section III.A) and tile map + symbolic closure per candidate
  std::vector<int64_t> ident(n);
  std::iota(ident.begin(), ident.end(), 0);
  std::vector<std::vector<int32_t>> best_cols;
  if (o.ordering == STILES_ORDER_NONE || o.ordering == STILES_ORDER_AUTO) {
    best_cols = tile_columns(n, colptr, rowidx, ident, T, nt);
    p->perm = ident;
    p->ordering_used = STILES_ORDER_NONE;
  }
  if (o.ordering == STILES_ORDER_ND) {
    // chosen for parallelism (two independent chains), not by the fill rule
    p->perm = adaptable_nd(n, colptr, rowidx, n_arrow, T);
    best_cols = tile_columns(n, colptr, rowidx, invert(p->perm), T, nt);
    p->ordering_used = STILES_ORDER_ND;
  }
  if (o.ordering == STILES_ORDER_RCM || o.ordering == STILES_ORDER_AUTO) {
    std::vector<int64_t> perm = partial_rcm(n, colptr, rowidx, n_arrow);
    std::vector<int64_t> inv = invert(perm);
    auto cols = tile_columns(n, colptr, rowidx, inv, T, nt);
    if (o.ordering == STILES_ORDER_RCM || count_tiles(cols) < count_tiles(best_cols)) {
      best_cols.swap(cols);
      p->perm.swap(perm);
      p->ordering_used = STILES_ORDER_RCM;
    }
  }
  p->iperm = invert(p->perm);

  // tile-CSC of L, diagonal first
  p->tcolptr.assign(nt + 1, 0);
  p->trowidx.clear();
  for (int64_t k = 0; k < nt; ++k) {
    p->trowidx.push_back(int32_t(k));
    p->trowidx.insert(p->trowidx.end(), best_cols[k].begin(), best_cols[k].end());
    p->tcolptr[k + 1] = int64_t(p->trowidx.size());
  }
  p->nnzt = int64_t(p->trowidx.size());
  best_cols.clear();
  best_cols.shrink_to_fit();

  // exact task flops at tile size T (actual ragged dimensions)
  auto dim = [&](int64_t I) { return std::min<int64_t>(T, n - I * T); };
  std::vector<std::vector<int32_t>> trows(nt);
  for (int64_t k = 0; k < nt; ++k)
    for (int64_t e = p->tcolptr[k]; e < p->tcolptr[k + 1]; ++e) trows[p->trowidx[e]].push_back(int32_t(k));
  p->flops_potrf = p->flops_syrk = p->flops_gemm = p->flops_trsm = 0;
  for (int64_t k = 0; k < nt; ++k) {
    const int64_t b = dim(k);
    p->flops_potrf += b * (b + 1) * (2 * b + 1) / 6;
    for (int32_t nn : trows[k])
      if (nn < k) p->flops_syrk += dim(nn) * b * (b + 1);
    for (int64_t e = p->tcolptr[k] + 1; e < p->tcolptr[k + 1]; ++e) {
      const int64_t m = p->trowidx[e];
      p->flops_trsm += dim(m) * b * b;
      const auto& rm = trows[m];
      const auto& rk = trows[k];
      size_t a = 0, c = 0;
      while (a < rm.size() && c < rk.size()) {
        if (rm[a] < rk[c]) ++a;
        else if (rk[c] < rm[a]) ++c;
        else {
          if (rm[a] < k) p->flops_gemm += 2 * dim(m) * b * dim(rm[a]);
          ++a;
          ++c;
        }
      }
    }
  }
  trows.clear();
  trows.shrink_to_fit();

  // device sub-tile size (the mixed-precision kernel works on 64-wide sub-tiles,
  // the sliced-update kernel on 32-wide ones)
  int64_t B = o.block;
  if (o.precision == STILES_PREC_SLICED) {
    B = (o.block == 0 || o.block == 32) ? 32 : 0;
  } else if (o.precision != STILES_PREC_F64) {
    B = (o.block == 0 || o.block == 64) ? 64 : 0;
  } else if (B == 0) {
    B = (T % 32 == 0) ? 32 : (T % 16 == 0 ? 16 : 0);
  }
  p->executable = (B == 16 || B == 32 || B == 64) && (T % B == 0);
  if (!p->executable) {
    p->B = int32_t(B);
    p->R = 0;
    return STILES_OK;
  }
  const int64_t R = T / B;
  p->B = int32_t(B);
  p->R = int32_t(R);
  const int64_t nsb = (n + B - 1) / B;
  p->nsb = nsb;
  p->nsub = p->nnzt * R * R;
  if (p->nsub >= (int64_t(1) << 30)) { *err = "too many sub-tiles"; return STILES_ERR_UNSUPPORTED; }

  auto tile_index = [&](int64_t I, int64_t J) -> int64_t {
    if (I == J) return p->tcolptr[J];
    const int32_t* b0 = p->trowidx.data() + p->tcolptr[J] + 1;
    const int32_t* e0 = p->trowidx.data() + p->tcolptr[J + 1];
    const int32_t* it = std::lower_bound(b0, e0, int32_t(I));
    if (it == e0 || *it != I) return -1;
    return int64_t(it - p->trowidx.data());
  };

  // present lower sub-tiles by sub-column and by sub-row (ascending)
  std::vector<std::vector<SubEntry>> scol(nsb), srow(nsb);
  for (int64_t J = 0; J < nt; ++J)
    for (int64_t e = p->tcolptr[J]; e < p->tcolptr[J + 1]; ++e) {
      const int64_t I = p->trowidx[e];
      for (int64_t q = 0; q < R; ++q) {
        const int64_t jj = J * R + q;
        if (jj >= nsb) break;
        for (int64_t pp = 0; pp < R; ++pp) {
          const int64_t ii = I * R + pp;
          if (ii >= nsb) break;
          if (ii < jj) continue;
          const int32_t s = int32_t(e * R * R + q * R + pp);
          scol[jj].push_back({int32_t(ii), s});
          srow[ii].push_back({int32_t(jj), s});
        }
      }
    }
  p->diag_sub.assign(nsb, -1);
  for (int64_t k = 0; k < nsb; ++k) p->diag_sub[k] = scol[k].front().sub;

  // scatter map of every input entry into the tile buffer; B is a power of two
  // and per-index tables give each permuted index's tile and offset, so the
  // O(nnz) pass does no division, and consecutive entries usually hit the tile
  // looked up last
  p->scatter.resize(nnz);
  {
    const int lb = (B == 16) ? 4 : (B == 32 ? 5 : 6);
    std::vector<int32_t> tile(n), off(n);
    for (int64_t i = 0; i < n; ++i) {
      tile[i] = int32_t(p->iperm[i] / T);
      off[i] = int32_t(p->iperm[i] % T);
    }
    int64_t lastI = -1, lastJ = -1, lastT = -1;
    for (int64_t j = 0; j < n; ++j) {
      for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
        const int64_t i = rowidx[e];
        // lower-triangle orientation of the permuted entry: (row r, column c) with r >= c
        const bool flip = p->iperm[i] < p->iperm[j];
        const int64_t tr = flip ? tile[j] : tile[i], tc = flip ? tile[i] : tile[j];
        const int64_t orr = flip ? off[j] : off[i], oc = flip ? off[i] : off[j];
        if (tr != lastI || tc != lastJ) {
          lastI = tr;
          lastJ = tc;
          lastT = tile_index(tr, tc);
          if (lastT < 0) { *err = "internal: entry outside the tile map"; return STILES_ERR_INVALID; }
        }
        const int64_t sub = lastT * R * R + (oc >> lb) * R + (orr >> lb);
        p->scatter[e] = (sub << (2 * lb)) + ((oc & (B - 1)) << lb) + (orr & (B - 1));
      }
    }
  }
  p->pad.clear();
  for (int64_t g = n; g < nsb * B; ++g)
    p->pad.push_back(int64_t(p->diag_sub[nsb - 1]) * B * B + (g % B) * B + (g % B));

  // Sub-columns in order of their elimination-tree level (leaves first), ties by
  // index: a topological order in which independent subtrees (e.g. the two parts
  // of a nested dissection) interleave, so their chains run at the same time.
  std::vector<int64_t> level(nsb, 0), corder(nsb);
  for (int64_t k = 0; k < nsb; ++k)
    if (scol[k].size() > 1) {
      const int64_t par = scol[k][1].idx;
      level[par] = std::max(level[par], level[k] + 1);
    }
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(), [&](int64_t a, int64_t b) { return level[a] < level[b]; });

  // factorization task graph: columns in level order, DIAG then OFF
  std::vector<Primary> prim;
  prim.reserve(size_t(nsb) * 4);
  std::vector<int64_t> pos(p->nsub, -1);
  for (int64_t k : corder) {
    const auto& rk = srow[k];
    // Chain step: when tile (k, k-1) exists, its TRSM and the SYRK term it feeds
    // into (k, k) run in the same task as POTRF(k) (no flag handoff in between).
    const bool chained = k > 0 && rk.size() >= 2 && rk[rk.size() - 2].idx == k - 1;
    if (chained) {
      const auto& rp = srow[k - 1];
      Primary c;
      c.type = TASK_CHAIN;
      c.out = rk[rk.size() - 2].sub;  // (k, k-1)
      c.diag = p->diag_sub[k - 1];
      c.col = int32_t(k - 1);
      c.out2 = p->diag_sub[k];
      c.col2 = int32_t(k);
      c.row = int32_t(k);
      size_t a2 = 0, b2 = 0;  // OFF part: n < k-1 common to rows k and k-1
      while (a2 < rk.size() && b2 < rp.size()) {
        if (rk[a2].idx >= k - 1 || rp[b2].idx >= k - 1) break;
        if (rk[a2].idx < rp[b2].idx) ++a2;
        else if (rp[b2].idx < rk[a2].idx) ++b2;
        else {
          c.list[0].pairs.push_back(rk[a2].sub);
          c.list[0].pairs.push_back(rp[b2].sub);
          c.list[0].producers.push_back(std::max(pos[rk[a2].sub], pos[rp[b2].sub]));
          ++a2;
          ++b2;
        }
      }
      for (const SubEntry& en : rk) {  // DIAG part: n < k-1 (n = k-1 is applied in the task)
        if (en.idx >= k - 1) break;
        c.list[1].pairs.push_back(en.sub);
        c.list[1].pairs.push_back(en.sub);
        c.list[1].producers.push_back(pos[en.sub]);
      }
      pos[c.out] = pos[c.out2] = int64_t(prim.size());
      prim.push_back(std::move(c));
    } else {
      Primary d;
      d.type = TASK_DIAG;
      d.out = p->diag_sub[k];
      d.diag = -1;
      d.col = int32_t(k);
      d.row = int32_t(k);
      for (const SubEntry& en : rk) {
        if (en.idx >= k) break;
        d.list[0].pairs.push_back(en.sub);
        d.list[0].pairs.push_back(en.sub);
        d.list[0].producers.push_back(pos[en.sub]);
      }
      pos[d.out] = int64_t(prim.size());
      prim.push_back(std::move(d));
    }
    for (size_t e = 1; e < scol[k].size(); ++e) {
      const int64_t i = scol[k][e].idx;
      if (i == k + 1) continue;  // tile (k+1, k) belongs to the chain step of column k+1
      Primary o2;
      o2.type = TASK_OFF;
      o2.out = scol[k][e].sub;
      o2.diag = p->diag_sub[k];
      o2.col = int32_t(k);
      o2.row = int32_t(i);
      const auto& ri = srow[i];
      size_t a = 0, c = 0;
      while (a < ri.size() && c < rk.size()) {
        if (ri[a].idx >= k || rk[c].idx >= k) break;
        if (ri[a].idx < rk[c].idx) ++a;
        else if (rk[c].idx < ri[a].idx) ++c;
        else {
          o2.list[0].pairs.push_back(ri[a].sub);
          o2.list[0].pairs.push_back(rk[c].sub);
          o2.list[0].producers.push_back(std::max(pos[ri[a].sub], pos[rk[c].sub]));
          ++a;
          ++c;
        }
      }
      pos[o2.out] = int64_t(prim.size());
      prim.push_back(std::move(o2));
    }
  }
  for (const auto& pr : prim)
    for (int l = 0; l < 2; ++l)
      for (int64_t q : pr.list[l].producers)
        if (q < 0) { *err = "internal: producer missing"; return STILES_ERR_INVALID; }
  try {
    build_graph(prim, o.tree_chunk, o.tree_fanin, TASK_PARTIAL, TASK_COMBINE, p->graph.tasks, p->graph.pairs,
                p->graph.parts, p->graph.nscratch, (1u << TASK_DIAG) | (1u << TASK_CHAIN), kChainKeep);
  } catch (const std::exception& ex) {
    *err = ex.what();
    return STILES_ERR_INVALID;
  }
  prim.clear();

  // forward sweep: one task per sub-row, ascending
  {
    std::vector<int64_t> rank(nsb);  // position of each block's task in the sweep
    for (int64_t q = 0; q < nsb; ++q) rank[corder[q]] = q;
    std::vector<Primary> fp(nsb);
    for (int64_t q = 0; q < nsb; ++q) {
      const int64_t k = corder[q];
      fp[q].type = SOLVE_FINAL;
      fp[q].out = int32_t(k);
      fp[q].diag = p->diag_sub[k];
      fp[q].col = int32_t(k);
      for (const SubEntry& en : srow[k]) {
        if (en.idx >= k) break;
        fp[q].list[0].pairs.push_back(en.sub);
        fp[q].list[0].pairs.push_back(en.idx);
        fp[q].list[0].producers.push_back(rank[en.idx]);
      }
    }
    build_graph(fp, o.tree_chunk, o.tree_fanin, SOLVE_PARTIAL, SOLVE_COMBINE, p->fwd.tasks, p->fwd.pairs,
                p->fwd.parts, p->fwd.nscratch, 0u, 0, kSweepKeep);
  }
  // backward sweep: one task per sub-column, descending
  {
    std::vector<int64_t> rank(nsb);  // backward sweep: reverse level order
    for (int64_t q = 0; q < nsb; ++q) rank[corder[nsb - 1 - q]] = q;
    std::vector<Primary> bp(nsb);
    for (int64_t q = 0; q < nsb; ++q) {
      const int64_t k = corder[nsb - 1 - q];
      bp[q].type = SOLVE_FINAL;
      bp[q].out = int32_t(k);
      bp[q].diag = p->diag_sub[k];
      bp[q].col = int32_t(k);
      // farthest block first: x_{k+1}, produced last, is consumed last
      for (size_t e = scol[k].size(); e-- > 1;) {
        bp[q].list[0].pairs.push_back(scol[k][e].sub);
        bp[q].list[0].pairs.push_back(scol[k][e].idx);
        bp[q].list[0].producers.push_back(rank[scol[k][e].idx]);
      }
    }
    build_graph(bp, o.tree_chunk, o.tree_fanin, SOLVE_PARTIAL, SOLVE_COMBINE, p->bwd.tasks, p->bwd.pairs,
                p->bwd.parts, p->bwd.nscratch, 0u, 0, kSweepKeep);
  }
  if (p->graph.nscratch >= (int64_t(1) << 30)) { *err = "too many tree partials"; return STILES_ERR_UNSUPPORTED; }
  // the two queues of a split launch (critical diagonal chain / everything else)
  p->chain_order.clear();
  p->bulk_order.clear();
  for (size_t t = 0; t < p->graph.tasks.size(); ++t) {
    const int32_t ty = p->graph.tasks[t].type;
    (ty == TASK_DIAG || ty == TASK_CHAIN ? p->chain_order : p->bulk_order).push_back(int32_t(t));
  }
  // Reserving SMs for the chain pays when the chain is the bottleneck: when the
  // tile work per chain step is small next to what the machine does during one
  // step (a thin band); on a wide band the reserved SMs would idle.
  const double flops_total = double(p->flops_potrf + p->flops_syrk + p->flops_gemm + p->flops_trsm);
  p->split_queues = !p->chain_order.empty() && flops_total / double(p->chain_order.size()) < kSplitFlopsPerStep;
  // every dependency must carry a smaller ticket, or the persistent kernels could wait forever
  if (!check_order(p->graph.tasks, p->graph.pairs, p->graph.parts, p->nsub, p->graph.nscratch, TASK_PARTIAL,
                   TASK_COMBINE, false, err) ||
      !check_order(p->fwd.tasks, p->fwd.pairs, p->fwd.parts, nsb, p->fwd.nscratch, SOLVE_PARTIAL, SOLVE_COMBINE,
                   true, err) ||
      !check_order(p->bwd.tasks, p->bwd.pairs, p->bwd.parts, nsb, p->bwd.nscratch, SOLVE_PARTIAL, SOLVE_COMBINE,
                   true, err))
    return STILES_ERR_INVALID;
  return STILES_OK;
}

// The factorization with the forward sweep folded in.  With block k's
// right-hand sides stored transposed as a tile (Y_k^T, a row per right-hand
// side), the forward step Y_k^T = (b_k^T - sum_j Y_j^T L_kj^T) L_kk^{-T} is an
// OFF task of the factor kernel: its pair loop forms acc -= A B^T with
// A = Y_j^T (tile nsub + j) and B = L_kj, and its row TRSM applies L_kk.  The
// forward solve graph's tasks are mapped one to one (tree partials to
// PARTIAL/COMBINE tasks on scratch tiles after the factor's) and each is
// placed right after the last producer of its inputs, so the forward chain
// follows the factorization instead of running after it.
stiles_status build_fused(stiles_plan* p, std::string* err) {
  if (p->fused_built) return STILES_OK;
  if (!p->executable) { *err = "the plan has no sub-tile executor"; return STILES_ERR_UNSUPPORTED; }
  const TaskGraph& fg = p->graph;
  const SolveGraph& sg = p->fwd;
  const int64_t nsub = p->nsub, nsb = p->nsb, nf = int64_t(fg.tasks.size());
  // ticket of the factor task that produces each sub-tile
  std::vector<int64_t> tout(size_t(nsub), -1);
  for (int64_t t = 0; t < nf; ++t) {
    const DevTask& tk = fg.tasks[size_t(t)];
    if (tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE) continue;
    tout[size_t(tk.out)] = t;
    if (tk.out2 >= 0) tout[size_t(tk.out2)] = t;
  }
  // forward tasks: mapped task and the factor ticket it must follow
  const int64_t ns = int64_t(sg.tasks.size());
  std::vector<int64_t> key(size_t(ns), -1), kblk(size_t(nsb), -1), kscr(size_t(std::max<int64_t>(sg.nscratch, 1)), -1);
  TaskGraph out;
  std::vector<DevTask> ftask(static_cast<size_t>(ns));
  std::vector<int32_t> fpairs, fparts;
  for (int64_t t = 0; t < ns; ++t) {
    const SolveTask& st = sg.tasks[size_t(t)];
    int64_t k = -1;
    DevTask d{};
    d.out2 = -1;
    d.col2 = -1;
    d.diag = -1;
    d.pb2 = d.pe2 = d.qb2 = d.qe2 = 0;
    d.trow = d.tcol = -1;  // forward blocks are not tile targets
    const int64_t pb = int64_t(fpairs.size()) / 2;
    for (int32_t q = st.pb; q < st.pe; ++q) {
      const int32_t ls = sg.pairs[2 * size_t(q)], bk = sg.pairs[2 * size_t(q) + 1];
      if (ls < 0 || ls >= nsub || bk < 0 || bk >= nsb || tout[size_t(ls)] < 0 || kblk[size_t(bk)] < 0) {
        *err = "internal: forward operand without a producer";
        return STILES_ERR_INVALID;
      }
      fpairs.push_back(int32_t(nsub + bk));
      fpairs.push_back(ls);
      k = std::max({k, tout[size_t(ls)], kblk[size_t(bk)]});
    }
    const int64_t qb = int64_t(fparts.size());
    for (int32_t q = st.qb; q < st.qe; ++q) {
      const int32_t sc = sg.parts[size_t(q)];
      if (sc < 0 || sc >= sg.nscratch || kscr[size_t(sc)] < 0) { *err = "internal: forward partial order"; return STILES_ERR_INVALID; }
      fparts.push_back(int32_t(fg.nscratch + sc));
      k = std::max(k, kscr[size_t(sc)]);
    }
    d.pb = int32_t(pb);
    d.pe = int32_t(fpairs.size() / 2);
    d.qb = int32_t(qb);
    d.qe = int32_t(fparts.size());
    if (st.type == SOLVE_FINAL) {
      if (st.diag < 0 || st.diag >= nsub || tout[size_t(st.diag)] < 0) { *err = "internal: forward diagonal"; return STILES_ERR_INVALID; }
      d.type = TASK_OFF;
      d.out = int32_t(nsub + st.out);
      d.diag = st.diag;
      d.col = st.out;
      k = std::max(k, tout[size_t(st.diag)]);
      kblk[size_t(st.out)] = k;
    } else {
      d.type = (st.type == SOLVE_PARTIAL) ? TASK_PARTIAL : TASK_COMBINE;
      d.out = int32_t(fg.nscratch + st.out);
      d.col = -1;
      kscr[size_t(st.out)] = k;
    }
    if (k < 0) { *err = "internal: forward task without inputs"; return STILES_ERR_INVALID; }
    key[size_t(t)] = k;
    ftask[size_t(t)] = d;
  }
  // merged ticket order: factor task i, then the forward tasks keyed to i (solve order)
  std::vector<std::vector<int32_t>> after(static_cast<size_t>(nf));
  for (int64_t t = 0; t < ns; ++t) after[size_t(key[size_t(t)])].push_back(int32_t(t));
  out.pairs = fg.pairs;
  out.parts = fg.parts;
  const int64_t pshift = int64_t(out.pairs.size()) / 2, qshift = int64_t(out.parts.size());
  out.pairs.insert(out.pairs.end(), fpairs.begin(), fpairs.end());
  out.parts.insert(out.parts.end(), fparts.begin(), fparts.end());
  out.nscratch = fg.nscratch + sg.nscratch;
  out.tasks.reserve(size_t(nf + ns));
  for (int64_t i = 0; i < nf; ++i) {
    out.tasks.push_back(fg.tasks[size_t(i)]);
    for (int32_t t : after[size_t(i)]) {
      DevTask d = ftask[size_t(t)];
      d.pb += int32_t(pshift);
      d.pe += int32_t(pshift);
      d.qb += int32_t(qshift);
      d.qe += int32_t(qshift);
      out.tasks.push_back(d);
    }
  }
  if (!check_order(out.tasks, out.pairs, out.parts, nsub + nsb, std::max<int64_t>(out.nscratch, 1), TASK_PARTIAL,
                   TASK_COMBINE, false, err))
    return STILES_ERR_INVALID;
  p->fused_chain.clear();
  p->fused_bulk.clear();
  for (size_t t = 0; t < out.tasks.size(); ++t) {
    const int32_t ty = out.tasks[t].type;
    const bool fwd = out.tasks[t].out >= nsub && ty != TASK_PARTIAL && ty != TASK_COMBINE;
    ((ty == TASK_DIAG || ty == TASK_CHAIN) && !fwd ? p->fused_chain : p->fused_bulk).push_back(int32_t(t));
  }
  p->fused = std::move(out);
  p->fused_built = true;
  return STILES_OK;
}

// Task graph of the selected inverse (Sigma L = L^{-T}, every column block
// after its ancestors).  For sub-column k with sub-rows S_k (p = min S_k, its
// parent in the sub-column elimination tree) and U_jk = L_jk L_kk^{-1}:
//   Sigma_mk = -sum_{j in S_k} Sigma_mj U_jk   (m in S_k),
//   Sigma_kk = L_kk^{-T} L_kk^{-1} - sum_{j in S_k} Sigma_jk^T U_jk.
// Sigma_mj (m, j > k) lies on the filled map (the tile closure makes S_k a
// clique); it is stored as (max, min) and read transposed when m < j.  For the
// parent row m = p every term but Sigma_pp U_pk comes from column p itself, so
// those terms X(j, k) = Sigma_jp^T U_jk are formed by the tasks of column p
// (their X products) and the task of Sigma_pk only loads them; likewise the
// task of Sigma_jk forms W(j, k) = Sigma_jk^T U_jk and the diagonal task loads
// the W terms.  Products run from the oldest producer (largest j) to the
// newest.  Every operand and every loaded term is published by a task with a
// smaller ticket (checked below), so the persistent kernel cannot wait on
// work that has not started.
stiles_status build_selinv(stiles_plan* p, std::string* err) {
  if (p->selinv_built) return STILES_OK;
  if (!p->executable) { *err = "the plan has no sub-tile executor"; return STILES_ERR_UNSUPPORTED; }
  const int64_t nsb = p->nsb, R = p->R, nt = p->nt;
  auto tile_index = [&](int64_t I, int64_t J) -> int64_t {
    if (I == J) return p->tcolptr[J];
    const int32_t* b0 = p->trowidx.data() + p->tcolptr[J] + 1;
    const int32_t* e0 = p->trowidx.data() + p->tcolptr[J + 1];
    const int32_t* it = std::lower_bound(b0, e0, int32_t(I));
    if (it == e0 || *it != I) return -1;
    return int64_t(it - p->trowidx.data());
  };
  auto sub_index = [&](int64_t ii, int64_t jj) -> int64_t {  // ii >= jj
    const int64_t e = tile_index(ii / R, jj / R);
    return e < 0 ? -1 : e * R * R + (jj % R) * R + (ii % R);
  };
  // sub-rows below the diagonal of every sub-column, ascending
  std::vector<std::vector<int32_t>> below(nsb);
  for (int64_t J = 0; J < nt; ++J)
    for (int64_t e = p->tcolptr[J]; e < p->tcolptr[J + 1]; ++e) {
      const int64_t I = p->trowidx[e];
      for (int64_t q = 0; q < R; ++q) {
        const int64_t jj = J * R + q;
        if (jj >= nsb) break;
        for (int64_t pp = 0; pp < R; ++pp) {
          const int64_t ii = I * R + pp;
          if (ii >= nsb) break;
          if (ii > jj) below[jj].push_back(int32_t(ii));
        }
      }
    }
  // Column order: by depth in the sub-column elimination tree (parent = first
  // sub-row below the diagonal), root first, ties by descending index.  Every
  // sub-row of S_k is an ancestor of k, so it comes earlier; independent
  // branches (the two halves of a nested dissection) interleave instead of
  // running one after the other.
  std::vector<int64_t> depth(nsb, 0), parent(nsb, -1), order(nsb);
  std::vector<std::vector<int32_t>> children(nsb);
  for (int64_t k = nsb - 1; k >= 0; --k) {
    std::vector<int32_t>& S = below[k];
    std::sort(S.begin(), S.end());
    parent[k] = S.empty() ? -1 : S[0];
    depth[k] = S.empty() ? 0 : depth[S[0]] + 1;
  }
  for (int64_t c = 0; c < nsb; ++c)
    if (parent[c] >= 0) children[parent[c]].push_back(int32_t(c));
  for (int64_t r = 0; r < nsb; ++r) order[r] = nsb - 1 - r;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return depth[x] < depth[y]; });
  // Per column (s = |S_k|): s + 1 tasks, 1 + (s - 1) s products, 2 s - 1 loads,
  // sum over the children c of (|S_c| - 1) X products, s U products.  Every
  // column is filled independently on host threads (the largest graphs hold a
  // few hundred million products).
  std::vector<int64_t> t_off(nsb + 1, 0), p_off(nsb + 1, 0), l_off(nsb + 1, 0), x_off(nsb + 1, 0),
      u_off(nsb + 1, 0);
  for (int64_t r = 0; r < nsb; ++r) {  // r-th column in depth order is order[r]
    const int64_t k = order[r];
    const int64_t sk = int64_t(below[k].size());
    int64_t nx = 0;
    for (int32_t c : children[k]) nx += int64_t(below[c].size()) - 1;
    t_off[r + 1] = t_off[r] + sk + 1;
    p_off[r + 1] = p_off[r] + (sk ? 1 + (sk - 1) * sk : 0);
    l_off[r + 1] = l_off[r] + (sk ? 2 * sk - 1 : 0);
    x_off[r + 1] = x_off[r] + nx;
    u_off[r + 1] = u_off[r] + sk;
  }
  if (p_off[nsb] >= (int64_t(1) << 31) || t_off[nsb] >= (int64_t(1) << 31) || l_off[nsb] >= (int64_t(1) << 31)) {
    *err = "selected inverse too large";
    return STILES_ERR_UNSUPPORTED;
  }
  const int64_t ntasks = t_off[nsb];
  std::vector<int64_t> producer(size_t(p->nsub), -1);  // ticket of the task that publishes a sub-tile
  SelinvGraph g;
  g.tasks.resize(size_t(8 * ntasks));
  g.pairs.resize(size_t(2 * p_off[nsb]));
  g.loads.resize(size_t(3 * l_off[nsb]));
  g.posts.resize(size_t(x_off[nsb]));
  g.ulist.resize(size_t(2 * u_off[nsb]));
  std::atomic<int> bad{0};
  const int64_t WBIT = int64_t(1) << 30;  // term index flag: the term lives in W (else X)
  auto fill = [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1 && !bad.load(std::memory_order_relaxed); ++r) {
      const int64_t k = order[r];
      const std::vector<int32_t>& S = below[k];
      int64_t u = u_off[r];
      for (int32_t j : S) {
        const int64_t sj = sub_index(j, k);
        if (sj < 0) { bad = 1; return; }
        g.ulist[2 * u] = int32_t(sj);
        g.ulist[2 * u + 1] = int32_t(k);
        ++u;
      }
      int64_t t = t_off[r], q = p_off[r], l = l_off[r], x = x_off[r];
      auto load = [&](int64_t flag, int64_t want, int64_t term) {
        g.loads[3 * l] = int32_t(flag);
        g.loads[3 * l + 1] = int32_t(want);
        g.loads[3 * l + 2] = int32_t(term);
        ++l;
      };
      // opens task t; close() records its ranges' ends
      auto open = [&](int64_t out, int32_t kind) -> int32_t* {
        int32_t* tk = &g.tasks[8 * t];
        tk[0] = int32_t(out);
        tk[1] = kind;
        tk[2] = int32_t(q);
        tk[4] = int32_t(l);
        tk[6] = int32_t(x);
        producer[size_t(out)] = t;
        return tk;
      };
      auto close = [&](int32_t* tk) {
        tk[3] = int32_t(q);
        tk[5] = int32_t(l);
        tk[7] = int32_t(x);
        ++t;
      };
      auto posts = [&](int64_t m) -> bool {
        // X(m, c) = Sigma_mk^T U_mc for every child c of k whose column holds row m
        for (int32_t c : children[k]) {
          const std::vector<int32_t>& Sc = below[c];
          if (std::binary_search(Sc.begin() + 1, Sc.end(), int32_t(m))) {
            const int64_t xs = sub_index(m, c);
            if (xs < 0) return false;
            g.posts[x++] = int32_t(xs);
          }
        }
        return true;
      };
      for (int32_t m : S) {
        const int64_t out = sub_index(m, k);
        if (out < 0) { bad = 2; return; }
        if (m == S[0]) {
          // the parent row: Sigma_pk = -(Sigma_pp U_pk + sum_{j > p} X(j, k)),
          // X(j, k) = Sigma_jp^T U_jk formed by the task of Sigma_jp
          const int64_t pp = sub_index(m, m);
          if (pp < 0) { bad = 2; return; }
          int32_t* tk = open(out, -1);
          g.pairs[2 * q] = int32_t(pp);
          g.pairs[2 * q + 1] = int32_t(sub_index(m, k));
          ++q;
          for (size_t c = 1; c < S.size(); ++c) {
            const int64_t fj = sub_index(S[c], m), xj = sub_index(S[c], k);
            if (fj < 0 || xj < 0) { bad = 2; return; }
            load(fj, 1, xj);
          }
          if (!posts(m)) { bad = 2; return; }
          close(tk);
          continue;
        }
        // products, oldest producer (largest j) first
        int32_t* tk = open(out, -1);
        for (size_t c = S.size(); c-- > 0;) {
          const int64_t j = S[c];
          int64_t sig;
          bool tr;
          if (m >= j) { sig = sub_index(m, j); tr = false; }
          else { sig = sub_index(j, m); tr = true; }
          if (sig < 0) { bad = 2; return; }
          g.pairs[2 * q] = int32_t(sig | (tr ? WBIT : 0));
          g.pairs[2 * q + 1] = int32_t(sub_index(j, k));
          ++q;
        }
        if (!posts(m)) { bad = 2; return; }
        close(tk);
      }
      // Sigma_kk = G_k - sum_j W(j, k), each behind the flag of Sigma_jk
      const int64_t outd = sub_index(k, k);
      if (outd < 0) { bad = 2; return; }
      int32_t* tk = open(outd, int32_t(k));
      for (int32_t j : S) load(sub_index(j, k), 1, sub_index(j, k) | WBIT);
      close(tk);
      if (t != t_off[r + 1] || q != p_off[r + 1] || l != l_off[r + 1] || x != x_off[r + 1]) { bad = 4; return; }
    }
  };
  const int64_t nthreads =
      std::max<int64_t>(1, std::min<int64_t>({int64_t(std::thread::hardware_concurrency()), 32, p_off[nsb] / 100000 + 1}));
  auto run = [&](auto&& fn) {
    if (nthreads == 1) {
      fn(0, nsb);
      return;
    }
    // chunks of about equal product counts
    std::vector<std::thread> pool;
    int64_t r0 = 0;
    for (int64_t w = 0; w < nthreads; ++w) {
      const int64_t target = p_off[nsb] * (w + 1) / nthreads;
      int64_t r1 = (w + 1 == nthreads) ? nsb
                                        : int64_t(std::lower_bound(p_off.begin(), p_off.end(), target) - p_off.begin());
      r1 = std::min<int64_t>(std::max<int64_t>(r1, r0), nsb);
      pool.emplace_back(fn, r0, r1);
      r0 = r1;
    }
    for (auto& th : pool) th.join();
  };
  run(fill);
  if (bad == 1) { *err = "internal: missing sub-tile"; return STILES_ERR_INVALID; }
  if (bad == 2) { *err = "internal: selected-inverse operand off the filled map"; return STILES_ERR_INVALID; }
  if (bad == 4) { *err = "internal: selected-inverse counts"; return STILES_ERR_INVALID; }
  // every operand and every loaded term must come from a task with a smaller ticket
  auto check = [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const int32_t* tk = &g.tasks[8 * i];
      for (int64_t q = tk[2]; q < tk[3]; ++q) {
        const int64_t pt = producer[size_t(g.pairs[2 * q] & ((1 << 30) - 1))];
        if (pt < 0 || pt >= i) { bad = 3; return; }
      }
      for (int64_t l = tk[4]; l < tk[5]; ++l) {
        const int64_t pt = producer[size_t(g.loads[3 * l])];
        if (pt < 0 || pt >= i || g.loads[3 * l + 1] != 1) { bad = 3; return; }
      }
    }
  };
  {
    std::vector<std::thread> pool;
    for (int64_t w = 0; w < nthreads; ++w) pool.emplace_back(check, ntasks * w / nthreads, ntasks * (w + 1) / nthreads);
    for (auto& th : pool) th.join();
  }
  if (bad == 3) { *err = "internal: selected-inverse operand not produced earlier"; return STILES_ERR_INVALID; }
  p->selinv = std::move(g);
  p->selinv_built = true;
  return STILES_OK;
}

}  // namespace stiles
