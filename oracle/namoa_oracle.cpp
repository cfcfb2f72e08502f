// Sequential NAMOA* oracle: TEST INFRASTRUCTURE ONLY.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
// load this library. It shares no code, header, table or helper with the CUDA
// library; the only thing both consume is the arrays produced by the seeded
// input generators.
//
// What it computes: the cost-unique set of non-dominated start->goal path cost
// vectors of a graph with non-negative d-vector arc costs (problem statement,
// Sec. 3), by Algorithm 1 (Sequential NAMOA*) executed step by step in the
// paper's order, with these readings where the text is silent or garbled:
//   * dominance a >- b: a[i] <= b[i] for all i and a[i] < b[i] for some i (Sec. 3);
//   * PruneOPEN(l) removes OPEN labels l* with g(l) <= F(l*) componentwise
//     (the parenthetical in Sec. 3 prints the inequality reversed);
//   * NotDominated against P (Algorithm 1, all three uses) is taken as "no p in P
//     weakly dominates", which keeps P cost-unique as Sec. 3 requires;
//   * OPEN ties in F are broken by label creation order;
//   * Visited(v) := a label was ever inserted at v;
//   * a candidate whose node has no path to the goal (h = infinity) is dropped;
//   * goal labels are not expanded (Algorithm 1: the goal branch ends the iteration).
// Arithmetic is uint64; results that do not fit uint32 are reported as overflow.
// The heuristic is the ideal point: h_k(v) = single-objective shortest distance
// from v to the goal under objective k (Sec. 4), by reverse Dijkstra.
//
// Parity status: pinned. The tests check this file against brute-force
// enumeration of simple paths (graphs up to 12 nodes, d = 1..8), textbook
// Dijkstra (d = 1, per-objective minima, lexicographic minimum) and the
// structural invariants of Sec. 3. Mistakes planted in copies of this file
// are rejected by those pins (tests/test_oracle_mutants.py). On the large
// benchmark graphs only the per-objective minima, the lexicographic minimum
// and the invariants are pinned. The rest of those fronts is parity
// unpinned: it rests on the agreement of two independent implementations.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <functional>
#include <new>
#include <queue>
#include <set>
#include <utility>
#include <vector>

namespace {

constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr uint64_t kInf64 = ~0ull;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxD = 16;

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_OVERFLOW = 2, ORC_BUDGET = 3, ORC_NOMEM = 4 };

struct GraphView {
  uint32_t n;
  uint64_t m;
  uint32_t d;
  const uint64_t* rowptr;
  const uint32_t* col;
  const uint32_t* cost;  // cost[k*m + e]
  uint32_t c(uint32_t k, uint64_t e) const { return cost[k * m + e]; }
};

int validate(const GraphView& G) {
  if (G.n == 0 || G.d == 0 || G.d > kMaxD) return ORC_INVALID;
  if (G.rowptr[0] != 0 || G.rowptr[G.n] != G.m) return ORC_INVALID;
  for (uint32_t v = 0; v < G.n; ++v)
    if (G.rowptr[v + 1] < G.rowptr[v]) return ORC_INVALID;
  for (uint64_t e = 0; e < G.m; ++e)
    if (G.col[e] >= G.n) return ORC_INVALID;
  return ORC_OK;
}

// h_k(v): shortest distance from v to goal under objective k, by Dijkstra on
// the reversed arcs. kInf32 where the goal cannot be reached.
int reverse_dijkstra(const GraphView& G, uint32_t goal, uint32_t* h) {
  // reversed adjacency: for each node v, the arcs e = (u -> v)
  std::vector<uint64_t> rstart(G.n + 1, 0);
  for (uint64_t e = 0; e < G.m; ++e) rstart[G.col[e] + 1]++;
  for (uint32_t v = 0; v < G.n; ++v) rstart[v + 1] += rstart[v];
  std::vector<uint64_t> fill(rstart.begin(), rstart.end() - 1);
  std::vector<uint64_t> rarc(G.m);
  std::vector<uint32_t> rsrc(G.m);
  for (uint32_t u = 0; u < G.n; ++u)
    for (uint64_t e = G.rowptr[u]; e < G.rowptr[u + 1]; ++e) {
      uint64_t slot = fill[G.col[e]]++;
      rarc[slot] = e;
      rsrc[slot] = u;
    }
  std::vector<uint64_t> dist(G.n);
  for (uint32_t k = 0; k < G.d; ++k) {
    std::fill(dist.begin(), dist.end(), kInf64);
    using Item = std::pair<uint64_t, uint32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    dist[goal] = 0;
    pq.push({0, goal});
    while (!pq.empty()) {
      auto [dv, v] = pq.top();
      pq.pop();
      if (dv != dist[v]) continue;
      for (uint64_t i = rstart[v]; i < rstart[v + 1]; ++i) {
        uint32_t u = rsrc[i];
        uint64_t nd = dv + G.c(k, rarc[i]);
        if (nd < dist[u]) {
          dist[u] = nd;
          pq.push({nd, u});
        }
      }
    }
    for (uint32_t v = 0; v < G.n; ++v) {
      if (dist[v] == kInf64) {
        h[(uint64_t)k * G.n + v] = kInf32;
      } else {
        if (dist[v] >= kInf32) return ORC_OVERFLOW;
        h[(uint64_t)k * G.n + v] = (uint32_t)dist[v];
      }
    }
  }
  return ORC_OK;
}

// Label pool, structure of arrays: label id i has node[i], parent[i],
// edge[i] (the arc that created it), g[i*d .. i*d+d) and F[i*d .. i*d+d).
struct Pool {
  int d = 0;
  std::vector<uint32_t> node, parent;
  std::vector<uint64_t> edge, gv, Fv;
  size_t size() const { return node.size(); }
  const uint64_t* g(uint32_t i) const { return gv.data() + (size_t)i * d; }
  const uint64_t* F(uint32_t i) const { return Fv.data() + (size_t)i * d; }
};

struct Counters {
  uint64_t extracted = 0;        // OPEN.popmin calls (Algorithm 1)
  uint64_t goal_extracted = 0;   // of which at the goal
  uint64_t expanded = 0;         // labels whose neighbours were generated
  uint64_t candidates = 0;       // l' generated
  uint64_t inserted = 0;         // OPEN inserts, including l_s
  uint64_t pruned_open = 0;      // OPEN labels removed by Prune(G_OP(v'), l')
  uint64_t pruned_open_goal = 0; // OPEN labels removed by PruneOPEN(l)
  uint64_t pruned_closed = 0;    // G_CL labels removed by Prune(G_CL(v'), l')
  uint64_t pruned_p = 0;         // P labels removed by Prune(P, l)
  uint64_t comparisons = 0;      // vector dominance/equality tests
  uint64_t max_open = 0;
  uint64_t ns = 0;               // main loop wall time, steady clock
};

// a weakly dominates b: a[i] <= b[i] for all i.
inline bool weakly(const uint64_t* a, const uint64_t* b, int d) {
  for (int i = 0; i < d; ++i)
    if (a[i] > b[i]) return false;
  return true;
}
// a dominates b in the sense of Sec. 3: weakly, and strictly in some i.
inline bool dominates(const uint64_t* a, const uint64_t* b, int d) {
  bool less = false;
  for (int i = 0; i < d; ++i) {
    if (a[i] > b[i]) return false;
    if (a[i] < b[i]) less = true;
  }
  return less;
}
inline bool equal(const uint64_t* a, const uint64_t* b, int d) {
  for (int i = 0; i < d; ++i)
    if (a[i] != b[i]) return false;
  return true;
}

struct Namoa {
  const GraphView& G;
  const uint32_t* h;
  uint32_t start, goal;
  int d;
  uint64_t budget;
  Pool pool;
  // OPEN order: F lexicographically, ties by label id (creation order).
  struct Lex {
    const Pool* pool;
    int d;
    bool operator()(uint32_t a, uint32_t b) const {
      const uint64_t* A = pool->F(a);
      const uint64_t* B = pool->F(b);
      for (int i = 0; i < d; ++i)
        if (A[i] != B[i]) return A[i] < B[i];
      return a < b;
    }
  };
  std::set<uint32_t, Lex> open;
  std::vector<std::vector<uint32_t>> gop, gcl;
  std::vector<uint8_t> visited;
  std::vector<uint32_t> P;
  Counters cnt;

  Namoa(const GraphView& g, const uint32_t* hh, uint32_t s, uint32_t t, uint64_t b)
      : G(g), h(hh), start(s), goal(t), d((int)g.d), budget(b), open(Lex{&pool, (int)g.d}),
        gop(g.n), gcl(g.n), visited(g.n, 0) {
    pool.d = d;
  }

  uint32_t hv(uint32_t k, uint32_t v) const { return h[(uint64_t)k * G.n + v]; }
  bool h_inf(uint32_t v) const { return hv(0, v) == kInf32; }

  static void erase_id(std::vector<uint32_t>& s, uint32_t id) {
    auto it = std::find(s.begin(), s.end(), id);
    if (it != s.end()) s.erase(it);
  }

  // NotDominated(x, P) in the weak reading: no p in P with g(p) <= x.
  bool not_dominated_by_P(const uint64_t* x) {
    for (uint32_t p : P) {
      cnt.comparisons++;
      if (weakly(pool.g(p), x, d)) return false;
    }
    return true;
  }

  std::chrono::steady_clock::time_point t0;

  int new_label(uint32_t v, uint32_t parent, uint64_t edge, const uint64_t* g, const uint64_t* F,
                uint32_t* id) {
    if (pool.size() >= budget) {
      cnt.ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now() - t0).count();
      return ORC_BUDGET;
    }
    pool.node.push_back(v);
    pool.parent.push_back(parent);
    pool.edge.push_back(edge);
    pool.gv.insert(pool.gv.end(), g, g + d);
    pool.Fv.insert(pool.Fv.end(), F, F + d);
    *id = (uint32_t)(pool.size() - 1);
    return ORC_OK;
  }

  void open_insert(uint32_t id) {
    open.insert(id);
    gop[pool.node[id]].push_back(id);
    visited[pool.node[id]] = 1;
    cnt.inserted++;
    if (open.size() > cnt.max_open) cnt.max_open = open.size();
  }

  int run() {
    t0 = std::chrono::steady_clock::now();
    // initialisation: l_s = (v_s, 0), into OPEN and G_OP(v_s)
    uint64_t zero[kMaxD] = {0}, Fs[kMaxD];
    for (int i = 0; i < d; ++i) Fs[i] = h_inf(start) ? kInf64 : hv(i, start);
    uint32_t ls;
    if (int rc = new_label(start, kNone, ~0ull, zero, Fs, &ls)) return rc;
    open_insert(ls);
    // main loop: while OPEN is not empty
    while (!open.empty()) {
      // l <- OPEN.popmin()
      uint32_t l = *open.begin();
      open.erase(open.begin());
      cnt.extracted++;
      const uint32_t v = pool.node[l];
      // move l from G_OP(v) to G_CL(v)
      erase_id(gop[v], l);
      gcl[v].push_back(l);
      if (v == goal) {
        cnt.goal_extracted++;
        // goal branch: PruneOPEN(l) over the whole OPEN
        for (auto it = open.begin(); it != open.end();) {
          cnt.comparisons++;
          if (weakly(pool.g(l), pool.F(*it), d)) {
            erase_id(gop[pool.node[*it]], *it);
            it = open.erase(it);
            cnt.pruned_open_goal++;
          } else {
            ++it;
          }
        }
        // Prune(P, l)
        for (size_t i = 0; i < P.size();) {
          cnt.comparisons++;
          if (dominates(pool.g(l), pool.g(P[i]), d)) {
            P.erase(P.begin() + i);
            cnt.pruned_p++;
          } else {
            ++i;
          }
        }
        // insert l into P unless a member weakly dominates it
        if (not_dominated_by_P(pool.g(l))) P.push_back(l);
        continue;
      }
      // expansion of l along the out-arcs of v
      cnt.expanded++;
      for (uint64_t e = G.rowptr[v]; e < G.rowptr[v + 1]; ++e) {
        const uint32_t vp = G.col[e];
        // l' = (v', g + c(e)), F(l') = g(l') + h(v')
        cnt.candidates++;
        if (h_inf(vp)) continue;
        uint64_t g2[kMaxD], F2[kMaxD];
        for (int i = 0; i < d; ++i) {
          g2[i] = pool.g(l)[i] + G.c(i, e);
          F2[i] = g2[i] + hv(i, vp);
        }
        if (!visited[vp]) {
          // v' never visited: insert l' unless P dominates F(l')
          if (not_dominated_by_P(F2)) {
            uint32_t id;
            if (int rc = new_label(vp, l, e, g2, F2, &id)) return rc;
            open_insert(id);
          }
          continue;
        }
        // Duplicate(l')
        bool dup = false;
        for (const auto* S : {&gop[vp], &gcl[vp]})
          for (uint32_t x : *S) {
            cnt.comparisons++;
            if (equal(pool.g(x), g2, d)) dup = true;
          }
        if (dup) continue;
        // NotDominated(l', G_OP(v')) and NotDominated(l', G_CL(v'))
        bool dominated = false;
        for (const auto* S : {&gop[vp], &gcl[vp]})
          for (uint32_t x : *S) {
            cnt.comparisons++;
            if (dominates(pool.g(x), g2, d)) dominated = true;
          }
        if (dominated) continue;
        // Prune(G_CL(v'), l')
        for (size_t i = 0; i < gcl[vp].size();) {
          cnt.comparisons++;
          if (dominates(g2, pool.g(gcl[vp][i]), d)) {
            gcl[vp].erase(gcl[vp].begin() + i);
            cnt.pruned_closed++;
          } else {
            ++i;
          }
        }
        // Prune(G_OP(v'), l') and remove the pruned labels from OPEN
        for (size_t i = 0; i < gop[vp].size();) {
          cnt.comparisons++;
          if (dominates(g2, pool.g(gop[vp][i]), d)) {
            open.erase(gop[vp][i]);
            gop[vp].erase(gop[vp].begin() + i);
            cnt.pruned_open++;
          } else {
            ++i;
          }
        }
        // insert l' unless P dominates F(l')
        if (not_dominated_by_P(F2)) {
          uint32_t id;
          if (int rc = new_label(vp, l, e, g2, F2, &id)) return rc;
          open_insert(id);
        }
      }
    }
    cnt.ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                 std::chrono::steady_clock::now() - t0).count();
    for (uint32_t p : P)
      for (int i = 0; i < d; ++i)
        if (pool.g(p)[i] >= kInf32) return ORC_OVERFLOW;
    return ORC_OK;
  }
};

}  // namespace

struct oracle_result {
  uint32_t d = 0;
  uint32_t partial = 0;                       // 1: stopped by the label budget
  uint32_t partial_pad = 0;
  std::vector<uint32_t> costs;                // count*d, lexicographically sorted
  std::vector<std::vector<uint32_t>> nodes;   // per solution, start..goal
  std::vector<std::vector<uint64_t>> edges;   // per solution, arc ids
  Counters cnt;
  uint64_t labels = 0;
};

extern "C" {

// h_out[k*n + v] = min cost_k of a v->goal path, 0xFFFFFFFF if none.
int oracle_heuristic(uint32_t n, uint64_t m, uint32_t d, const uint64_t* rowptr,
                     const uint32_t* col, const uint32_t* cost, uint32_t goal, uint32_t* h_out) {
  GraphView G{n, m, d, rowptr, col, cost};
  if (int rc = validate(G)) return rc;
  if (goal >= n) return ORC_INVALID;
  return reverse_dijkstra(G, goal, h_out);
}

// Runs Algorithm 1. h may be NULL (computed here). label_budget = 0 means
// unlimited. On success *out owns the front. When the budget stops the run the
// return code is ORC_BUDGET and *out holds the counters only (count 0); on any
// other failure *out is NULL.
int oracle_solve(uint32_t n, uint64_t m, uint32_t d, const uint64_t* rowptr, const uint32_t* col,
                 const uint32_t* cost, const uint32_t* h, uint32_t start, uint32_t goal,
                 uint64_t label_budget, oracle_result** out) {
  *out = nullptr;
  GraphView G{n, m, d, rowptr, col, cost};
  if (int rc = validate(G)) return rc;
  if (start >= n || goal >= n) return ORC_INVALID;
  try {
    std::vector<uint32_t> hbuf;
    if (!h) {
      hbuf.resize((size_t)d * n);
      if (int rc = reverse_dijkstra(G, goal, hbuf.data())) return rc;
      h = hbuf.data();
    }
    Namoa S(G, h, start, goal, label_budget ? label_budget : ~0ull);
    const int rc = S.run();
    if (rc && rc != ORC_BUDGET) return rc;
    auto* r = new oracle_result;
    r->d = d;
    r->cnt = S.cnt;
    r->labels = S.pool.size();
    if (rc == ORC_BUDGET) {
      // stopped by the budget: counters only (the front is not final)
      r->partial = 1;
      *out = r;
      return ORC_BUDGET;
    }
    std::vector<uint32_t> P = S.P;
    std::sort(P.begin(), P.end(), [&](uint32_t a, uint32_t b) {
      for (uint32_t i = 0; i < d; ++i)
        if (S.pool.g(a)[i] != S.pool.g(b)[i]) return S.pool.g(a)[i] < S.pool.g(b)[i];
      return a < b;
    });
    for (uint32_t p : P) {
      for (uint32_t i = 0; i < d; ++i) r->costs.push_back((uint32_t)S.pool.g(p)[i]);
      std::vector<uint32_t> nodes;
      std::vector<uint64_t> edges;
      for (uint32_t x = p; x != kNone; x = S.pool.parent[x]) {
        nodes.push_back(S.pool.node[x]);
        if (S.pool.parent[x] != kNone) edges.push_back(S.pool.edge[x]);
      }
      std::reverse(nodes.begin(), nodes.end());
      std::reverse(edges.begin(), edges.end());
      r->nodes.push_back(std::move(nodes));
      r->edges.push_back(std::move(edges));
    }
    *out = r;
    return ORC_OK;
  } catch (const std::bad_alloc&) {
    return ORC_NOMEM;
  }
}

uint32_t oracle_result_count(const oracle_result* r) { return r ? (uint32_t)r->nodes.size() : 0; }

int oracle_result_costs(const oracle_result* r, uint32_t* out) {
  if (!r) return ORC_INVALID;
  std::memcpy(out, r->costs.data(), r->costs.size() * sizeof(uint32_t));
  return ORC_OK;
}

uint32_t oracle_result_path_len(const oracle_result* r, uint32_t i) {
  return (r && i < r->nodes.size()) ? (uint32_t)r->nodes[i].size() : 0;
}

// nodes: path_len entries; edges: path_len - 1 entries.
int oracle_result_path(const oracle_result* r, uint32_t i, uint32_t* nodes, uint64_t* edges) {
  if (!r || i >= r->nodes.size()) return ORC_INVALID;
  std::memcpy(nodes, r->nodes[i].data(), r->nodes[i].size() * sizeof(uint32_t));
  if (!r->edges[i].empty())
    std::memcpy(edges, r->edges[i].data(), r->edges[i].size() * sizeof(uint64_t));
  return ORC_OK;
}

// out[0..12]: extracted, goal_extracted, expanded, candidates, inserted, pruned_open,
// pruned_open_goal, pruned_closed, pruned_p, comparisons, max_open, ns, labels
int oracle_result_stats(const oracle_result* r, uint64_t* out) {
  if (!r) return ORC_INVALID;
  const Counters& c = r->cnt;
  uint64_t v[13] = {c.extracted, c.goal_extracted, c.expanded, c.candidates, c.inserted,
                    c.pruned_open, c.pruned_open_goal, c.pruned_closed, c.pruned_p,
                    c.comparisons, c.max_open, c.ns, r->labels};
  std::memcpy(out, v, sizeof(v));
  return ORC_OK;
}

void oracle_result_free(oracle_result* r) { delete r; }

}  // extern "C"
