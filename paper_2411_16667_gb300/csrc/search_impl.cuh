// Ordered-parallel multi-objective label-setting search (Sec. 5, Algorithm 2)
// on one GPU, pipelined as in Sec. 5.1. One "team" of threads works on one
// query: the whole cooperative grid for a single query, or a share of the
// grid's blocks per query in the multi-query kernel.
//
// Step i of the search is ONE phase between two team barriers, in which two
// things run side by side on the team's warps (Sec. 5.1: the next batch is
// extracted while the current one is processed):
//
//   merge (window i)     the candidates produced by expanding window i are
//                        merged node by node, one warp per target node (a
//                        whole block when candidates x frontier entries are
//                        many, split into parts of one block each when they
//                        are very many):
//                        resolved against each other (in-batch dominance and
//                        duplicates), against the node's frontier alpha(v')
//                        (Algorithm 1: weakly dominated candidates are dropped,
//                        strictly dominated frontier labels are pruned), then
//                        against P on F (Algorithm 1); survivors become labels,
//                        join alpha(v') and the next OPEN. Extracted goal
//                        labels reach a virtual node n standing for P, whose
//                        merge applies the goal branch of Algorithm 1 and
//                        appends survivors to the P log.
//   extract (window i+1) OPEN_i is scanned once: the window is every live entry
//                        in the lowest histogram bins of (F[0], F[1]) whose
//                        cumulative count stays within W (the NUM_POP of
//                        Sec. 5); pruned entries are dropped (lazy OPEN delete,
//                        Sec. 5.1) and so are entries whose F a logged solution
//                        weakly dominates (PruneOPEN of Algorithm 1, applied
//                        lazily); window labels are expanded at once along
//                        their out-arcs (g' = g + c(e), dropped when h(v') is
//                        infinite) into the other candidate set; all other
//                        entries are carried to OPEN_{i+1}.
//
// Labels created by merge i therefore become extractable from window i+2 on:
// the same one-step lag as the paper's asynchronous scheme, which leaves the
// result exact (only the amount of work changes).
//
// The histogram of OPEN_{i+1} is built while its entries are written (carried
// entries and new labels), on bins fixed at the start of step i. Its F[0]
// origin is a lower bound on every key OPEN_{i+1} can hold: with a consistent
// heuristic a child's F is at least its parent's, so min F[0] over OPEN plus
// the window in flight never decreases. A bin holds 2^s2 consecutive cells
// q * 256 + x, q the F[0] bucket and x the F[1] cell of a key, so that every
// bin prefix is a lexicographic prefix of OPEN.
//
// Determinism: a label pruned in step j is still extractable in step j (its
// ldead word records j, and extraction drops labels with ldead < i), equal
// candidates at a node keep the smallest arc id, a label created in step i
// that an equal candidate with a smaller arc id meets takes that candidate's
// parent and arc, and a label created and pruned within one step is taken
// back out of the histogram. Given the launch parameters, the windows, the
// fronts and the paths do not depend on the timing of the threads.
//
// The F-against-P tests use an index of P rebuilt once P has grown by 32 +
// a fraction of its indexed count: P sorted along a Z-order curve over
// objectives 1..3 in tiles of 32, each with its componentwise minimum, plus
// the goal costs logged since; a rebuild runs over three steps (rank,
// scatter, tiles) and is then published.
//
// A node is only ever merged by one warp (or block) per step, so frontier
// updates need no locks. All waits are bounded (see GridTeam::sync).
#pragma once

#include "opmos_dev.cuh"
#include "search.cuh"

namespace opmos {
namespace detail {

__device__ __forceinline__ unsigned warp_min(unsigned x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ unsigned warp_max(unsigned x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ void flush_stats(QCtl* C, unsigned long long (&st)[kNStat]) {
#pragma unroll
  for (int i = 0; i < kNStat; ++i) {
    unsigned long long v = st[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0 && v) atomicAdd(&C->stats[i], v);
    st[i] = 0;
  }
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ inline unsigned block_exclusive_scan(unsigned x, unsigned* s_warp, unsigned& total) {
  const unsigned lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned v = lane < nw ? s_warp[lane] : 0;
    unsigned vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= (unsigned)o) vi += y;
    }
    if (lane < nw) s_warp[lane] = vi - v;
    if (lane == nw - 1) s_warp[32] = vi;
  }
  __syncthreads();
  const unsigned r = s_warp[w] + incl - x;
  total = s_warp[32];
  __syncthreads();
  return r;
}

constexpr unsigned kHC = 256;  // candidates a block merge holds at once

struct Shared {
  alignas(16) unsigned hist[kNB];  // this block's share of the next OPEN's histogram
  unsigned warp[33];
  unsigned f_min, b1_max, bstar;
  unsigned pmax[3];
  unsigned claim;
  PIdx pd;             // the P index as this step sees it
  // the candidates of a block-merged node (up to kHC at a time)
  uint32_t hc[OPMOS_MAX_D][kHC];
  int hcid[kHC];
  uint32_t hedge[kHC], hpar[kHC];
  unsigned halive[kHC / 32], hkill[kHC / 32], hpkill[kHC / 32];
  int hlist[32];       // cursors of the block-merged node's lists
  unsigned mq_ncand, mq_next, m_nb, m_ok, m_lb, m_cap, m_plen, m_more;
  unsigned long long m_fb;
  unsigned tmax[5];    // this block's longest heavy merge, light merge, extraction item (ns);
                       // most candidates and largest frontier of its heavy merges
};

// Histogram bin of an OPEN key (F0 << 32 | F1): the key's cell is
// q * kSub + x, q = (F0 - b0) / delta its F[0] bucket and x = (F1 - b1) >> s1
// (at most kSub - 1) its F[1] cell; a bin is 2^s2 consecutive cells, and the
// last bin collects every key beyond. Monotone in lexicographic (F0, F1)
// order for F0 >= b0, so every prefix of bins is a lexicographic prefix of
// OPEN.
struct BinParams {
  uint32_t b0, b1, s1, delta, s2;
};
__device__ __forceinline__ unsigned bin_of(uint64_t key, const BinParams& bp) {
  const uint32_t F0 = (uint32_t)(key >> 32), F1 = (uint32_t)key;
  const uint64_t q = F0 > bp.b0 ? (F0 - bp.b0) / bp.delta : 0u;
  const uint32_t x = F1 > bp.b1 ? min((F1 - bp.b1) >> bp.s1, (unsigned)kSub - 1) : 0u;
  return (unsigned)min((q * kSub + x) >> bp.s2, (uint64_t)(kNB - 1));
}

// Z-order ("Morton") comparison without interleaving: the dimension whose
// values differ in the highest bit decides.
__device__ __forceinline__ bool msb_less(uint32_t a, uint32_t b) { return a < b && a < (a ^ b); }
template <int MD>
__device__ __forceinline__ bool z_less(const uint32_t (&a)[MD], const uint32_t (&b)[MD]) {
  int dim = 0;
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < MD; ++k) {
    const uint32_t y = a[k] ^ b[k];
    if (msb_less(x, y)) {
      dim = k;
      x = y;
    }
  }
  return a[dim] < b[dim];
}

template <int D>
struct Search {
  // frontier tiles loaded per round of a scan: fewer at high d (registers)
  static constexpr int kU = D <= 4 ? 4 : (D <= 8 ? 2 : 1);
  static constexpr int kUH = D <= 8 ? 2 : 1;
  static constexpr int kPT = D <= 4 ? 4 : (D <= 8 ? 2 : 1);  // P-index tiles loaded per round

  const GraphDev& G;
  const QArena& A;
  QCtl* C;
  const QParams& P;
  const OutPool& O;
  Shared& S;
  unsigned long long st[kNStat];
  // fixed for one step
  unsigned cyc = 0;    // step number i
  unsigned psnap = 0;  // P-log prefix every F-against-P test of step i uses
  unsigned lbase = 0;  // labels that existed when step i began
  unsigned fifo_head = 0;  // FIFO: the oldest ring position still in use in step i
  BinParams bpn{};     // bins of the next OPEN's histogram

  __device__ Search(const GraphDev& g, const QArena& a, QCtl* c, const QParams& p, const OutPool& o,
                    Shared& s)
      : G(g), A(a), C(c), P(p), O(o), S(s) {
#pragma unroll
    for (int i = 0; i < kNStat; ++i) st[i] = 0;
  }

  // h_k(v) and c_k(e); objectives the query does not use read as 0, which
  // leaves every dominance relation of the used ones unchanged
  __device__ __forceinline__ uint32_t hk(int k, uint32_t v) const {
    return (uint32_t)k < P.qd ? __ldg(P.h + (size_t)k * G.n + v) : 0u;
  }
  __device__ __forceinline__ uint32_t ck(int k, uint32_t e) const {
    return (uint32_t)k < P.qd ? __ldg(G.cost + (size_t)k * G.m + e) : 0u;
  }
  __device__ __forceinline__ uint64_t key_of(const uint32_t (&g)[D], uint32_t v) const {
    return ((uint64_t)(g[0] + hk(0, v)) << 32) | (D > 1 ? g[1 % D] + hk(1 % D, v) : 0u);
  }
  __device__ __forceinline__ bool dead_now(uint32_t id) const { return A.ldead[id] < cyc; }

  // ---------------- initialisation (Algorithm 1) ----------------
  // Empty frontiers, candidate sets and histograms (the empty sets Algorithm
  // 1 starts from). The team must pass a barrier before init_seed.
  template <class Team>
  __device__ void init_zero(const Team& T) {
    for (unsigned v = T.tid(); v <= G.n; v += T.nthreads()) {  // n real nodes + P
      A.fcount[v] = 0;
      A.fcap[v] = 0;
      A.fbase[v] = 0;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        for (unsigned j = 0; j < (1u << A.lsub); ++j) A.cs[b].node_head[((size_t)v << A.lsub) + j] = kNil;
        A.cs[b].ncand[v] = 0;
        A.cs[b].hflag[v] = 0;
        A.cs[b].hcnt[v] = 0;
      }
    }
    for (unsigned i = T.tid(); i < 3u * kNB; i += T.nthreads()) A.hist[i] = 0;
    for (unsigned i = T.tid(); i < kPSMax; i += T.nthreads()) A.prank[i] = 0;
  }

  __device__ static void clear_cycle(CycleCtl& K) {
    K.open_count.v = 0;
    K.min_key.v = ~0ull;
    K.win_count.v = 0;
    K.win_min.v = kInf;
    K.win_max.v = 0;
    K.cand_count.v = 0;
    K.touched_count.v = 0;
    K.heavy_count.v = 0;
    K.work_next.v = 0;
    K.heavy_next.v = 0;
    K.part_count.v = 0;
    K.f1lo.v = kInf;
    K.f1hi.v = 0;
    K.plen.v = 0;
    K.lbase.v = 0;
    for (int j = 0; j < 5; ++j) K.tmax[j] = 0;
    K.head = 0;
  }

  // l_s = (v_s, 0) into OPEN_0 and G_OP(v_s) (Algorithm 1), control reset.
  template <class Team>
  __device__ void init_seed(const Team& T, bool reset_ctl) {
    if (!T.leader()) return;
    if (reset_ctl) {
      C->error = 0;
      C->done = 0;
      C->res_count = C->res_status = 0;
      C->res_off = C->res_path = C->res_total = 0;
      for (int i = 0; i < kNStat; ++i) C->stats[i] = 0;
    }
    C->step = 0;
    C->t_start = globaltimer();
    const uint32_t s = P.start, t = P.goal, tile = P.tile;
#pragma unroll
    for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap] = 0;
    A.lnode[0] = s;
    A.lparent[0] = kInf;
    A.ledge[0] = kInf;
    A.lpver[0] = 0;
    A.ldead[0] = kAlive;
    const uint32_t fs = (s == t) ? G.n : s;  // start == goal: l_s is the solution
    A.fbase[fs] = 0;
    A.fcap[fs] = tile;
    A.fcount[fs] = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) A.fpool[(size_t)k * tile] = 0;
    A.fpool[(size_t)D * tile] = 0;
    C->f_words.v = (unsigned long long)(D + 1) * tile;
    C->n_labels.v = 1;
    for (int r = 0; r < 3; ++r) {
      clear_cycle(C->cyc[r]);
      C->cyc[r].win_min_prev = kInf;
    }
    for (int b = 0; b < 2; ++b) C->pidx[b] = PIdx{};
    const uint32_t h0 = hk(0, s);
    const uint64_t key = ((uint64_t)h0 << 32) | (D > 1 ? hk(1, s) : 0u);
    CycleCtl& K = C->cyc[0];
    K.lbase.v = 1;
    // the bins of OPEN_0's histogram put l_s in bin 0
    C->bins[0] = BinLimits{h0, (uint32_t)key, 0u, P.delta, 0u};
    if (s != t && h0 != kInf) {  // start == goal: P = {l_s}; h(s) = inf: goal unreachable
      A.okey[0][0] = key;
      A.oid[0][0] = 0;
      K.open_count.v = 1;
      K.min_key.v = key;
      K.f1lo.v = K.f1hi.v = (uint32_t)key;
      A.hist[0] = 1;
    }
    if (s == t) {
#pragma unroll
      for (int k = 0; k < D; ++k) A.plog[(size_t)k * A.plog_cap] = 0;
    }
    C->fifo_tail.v = K.open_count.v;
    C->plog_len.v = (s == t) ? 1u : 0u;
    K.plen.v = C->plog_len.v;
    st[S_INSERTED] += 1;
  }

  // ---------------- window selection (Algorithm 2: NUM_POP lowest labels) ----------------
  // Bins [0, b*] where b* is the largest bin whose cumulative count is <= W,
  // but at least the first non-empty bin (the overflow bin is never taken).
  // Every block computes the same b* into S.bstar. all: OPEN holds at most W
  // entries, so every bin but the last has a cumulative count within W and
  // b* is kNB - 2 without reading the histogram.
  __device__ void select_window(const unsigned* gh, bool all = false) {
    constexpr unsigned kPer = kNB / 256;  // bins per thread: blocks have 256 threads or more
    static_assert(kGridThreads >= 256 && kGridWideThreads >= 256 && kMultiThreads >= 256, "kPer");
    if (all) {
      if (threadIdx.x == 0) S.bstar = kNB - 2;
      for (unsigned x = threadIdx.x; x < kNB; x += blockDim.x) S.hist[x] = 0;
      __syncthreads();
      return;
    }
    const unsigned per = (kNB + blockDim.x - 1) / blockDim.x;
    // the histogram (other SMs added to it: read past L1) staged in shared
    // memory with 16-byte loads, then each thread takes `per` consecutive bins
    {
      const uint4* g4 = reinterpret_cast<const uint4*>(gh);
      uint4* s4 = reinterpret_cast<uint4*>(S.hist);
      for (unsigned x = threadIdx.x; x < kNB / 4; x += blockDim.x) s4[x] = __ldcg(g4 + x);
    }
    if (threadIdx.x == 0) {
      S.f_min = kNB;
      S.b1_max = 0;
    }
    __syncthreads();
    const unsigned b0 = threadIdx.x * per;
    unsigned loc[kPer];
    unsigned sum = 0;
#pragma unroll
    for (unsigned j = 0; j < kPer; ++j) {
      loc[j] = (j < per && b0 + j < (unsigned)kNB) ? S.hist[b0 + j] : 0u;
      sum += loc[j];
    }
    unsigned total;
    unsigned run = block_exclusive_scan(sum, S.warp, total);
    unsigned fmin = kNB, b1 = 0;
    bool any_b1 = false;
#pragma unroll
    for (unsigned j = 0; j < kPer; ++j) {
      const unsigned b = b0 + j;
      run += loc[j];
      if (j < per && b < (unsigned)kNB - 1) {
        if (loc[j] && b < fmin) fmin = b;
        if (run <= P.window) {
          b1 = b;
          any_b1 = true;
        }
      }
    }
    if (fmin < kNB) atomicMin(&S.f_min, fmin);
    if (any_b1) atomicMax(&S.b1_max, b1);
    __syncthreads();
    if (threadIdx.x == 0) S.bstar = max(S.b1_max, S.f_min == (unsigned)kNB ? 0u : S.f_min);
    // S.hist starts the next OPEN's histogram empty
    for (unsigned x = threadIdx.x; x < kNB; x += blockDim.x) S.hist[x] = 0;
    __syncthreads();
  }

  // Bins of the histogram of OPEN_{i+1}, from what step i-1 measured (the
  // same on every block). F[0] origin: the smallest F[0] among the entries
  // carried into OPEN_i, window i (whose children merge i creates) and window
  // i-1 (whose children are OPEN_i's other entries). F[1] cells: the F[1]
  // range of the entries carried into OPEN_i in 256 cells. Cells per bin: the
  // bins cover the F[0] buckets from the origin to window i's largest F[0]
  // and three times window i's F[0] extent beyond.
  __device__ BinParams next_bins(const CycleCtl& K) const {
    const unsigned long long mk = ld_volatile64(&K.min_key.v);
    const unsigned lo = ld_volatile(&K.f1lo.v), hi = ld_volatile(&K.f1hi.v);
    BinParams b;
    b.b0 = min(min((uint32_t)(mk >> 32), ld_volatile(&K.win_min.v)), ld_volatile(&K.win_min_prev));
    if (b.b0 == kInf) b.b0 = 0;
    b.b1 = lo <= hi ? lo : (mk != ~0ull ? (uint32_t)mk : 0u);
    const unsigned span = lo <= hi ? hi - lo : 0u;
    b.s1 = 0;
    while ((span >> b.s1) >= (unsigned)kSub) ++b.s1;
    b.delta = P.delta;
    const uint32_t wmax = ld_volatile(&K.win_max.v), wmin = min(ld_volatile(&K.win_min.v), wmax);
    const uint64_t rows = (wmax > b.b0 ? (wmax - b.b0) / b.delta : 0u) + 1 + 3ull * ((wmax - wmin) / b.delta + 1);
    b.s2 = 0;
    while (b.s2 < 30 && ((uint64_t)(kNB - 1) << b.s2) / kSub < rows) ++b.s2;
    return b;
  }

  // n-th (0-based) set bit of m, 32 if there is none.
  __device__ __forceinline__ unsigned nth_bit(unsigned m, unsigned n) {
    for (unsigned i = 0; i < n && m; ++i) m &= m - 1;
    return m ? __ffs(m) - 1 : 32u;
  }

  // ---------------- expansion (Algorithm 1) ----------------
  __device__ __forceinline__ void add_candidate(const CandSet& cs, CycleCtl& K1, uint32_t v2, uint32_t parent,
                                                uint32_t e, const uint32_t (&g2)[D]) {
    const unsigned c = agg_inc(&K1.cand_count.v);
    cs.cnode[c] = v2;
    cs.cparent[c] = parent;
    cs.cedge[c] = e;
    cs.cflag[c] = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) cs.cg[(size_t)k * A.cand_cap + c] = g2[k];
    const unsigned pos = atomicAdd(&cs.ncand[v2], 1u);
    if (pos < A.nslots) {
      cs.cslot[(size_t)v2 * A.nslots + pos] = (int)c;
    } else {  // list (pos - nslots) mod 2^lsub of the node, so all its lists grow evenly
      const unsigned j = (pos - A.nslots) & ((1u << A.lsub) - 1u);
      cs.cnext[c] = atomicExch(&cs.node_head[((size_t)v2 << A.lsub) + j], (int)c);
      st[S_OVF]++;
    }
    // Every node is listed among the light ones (one warp each) on its
    // first candidate. A node with a large frontier, or reached by many
    // candidates, is also listed once at the far end of the touched array
    // (hflag decides; the array holds 2 * cand_cap entries) and merged by
    // whole blocks; its light item then only clears hflag. Only light items
    // touch hflag during the merge, so a block merge never races a warp.
    if (pos == 0) cs.touched[agg_inc(&K1.touched_count.v)] = v2;
    // A node is merged by a whole block once its candidates x frontier
    // entries reach P.heavy_work (checked at 1, 4, 8 and 16 candidates: the
    // work of a one-warp merge grows with that product; at the goal node n,
    // with candidates x P), and always past kHeavyCands candidates (a warp
    // would take them in two batches).
    const unsigned nc = pos + 1u;
    const bool list = pos == kHeavyCands ||
                      ((nc == 1u || nc == 4u || nc == 8u || nc == 16u) &&
                       (unsigned long long)nc * A.fcount[v2] >= P.heavy_work);
    // at 64, 128, 256, ... candidates the merge may be split further
    const bool grow = A.kparts > 1u && pos > kHeavyCands && ((pos + 1u) & pos) == 0u;
    // (the P test of a goal candidate skips most of P through the index tiles)
    if (list || grow) heavy_list(cs, K1, v2, parts_for(pos + 1u, A.fcount[v2] >> (v2 == G.n ? 3 : 0)), list);
  }

  // Parts a block merge of nc candidates against F frontier entries is split
  // into: a power of two, each part about P.part_work comparisons or fewer.
  __device__ unsigned parts_for(unsigned nc, unsigned F) const {
    const unsigned long long w = (unsigned long long)nc * F;
    unsigned k = 1;
    while (k < A.kparts && w > (unsigned long long)P.part_work * k) k <<= 1;
    return k;
  }

  // Lists node v as a heavy node (list), or raises the parts of its merge to
  // want as its candidates grow. The lister holds hflag at kHeavyBusy until
  // the node's index h and part count are written, then publishes h + 1; a
  // raise that finds the node not yet published is dropped (the next one, at
  // twice the candidates, tries again). Every new part is recorded in xpart;
  // parts already recorded keep their numbers.
  __device__ void heavy_list(const CandSet& cs, CycleCtl& K1, uint32_t v, unsigned want, bool list) {
    unsigned h, r0;
    if (list) {
      if (atomicCAS(&cs.hflag[v], 0u, kHeavyBusy) != 0u) return;  // listed already
      h = atomicAdd(&K1.heavy_count.v, 1u);
      cs.touched[2u * A.cand_cap - 1u - h] = v;
      cs.hsplit[h] = want;
      r0 = 0;
    } else {
      const unsigned f = ld_volatile(&cs.hflag[v]);
      if (f == 0u || f == kHeavyBusy) return;
      h = f - 1u;
      unsigned old = ld_volatile(&cs.hsplit[h]);
      for (;;) {
        if (want <= old) return;
        const unsigned seen = atomicCAS(&cs.hsplit[h], old, want);
        if (seen == old) break;
        old = seen;
      }
      r0 = old > 1u ? old : 0u;  // parts [old, want), or all of them when the merge was not split
    }
    if (want > 1u) {
      const unsigned j = atomicAdd(&K1.part_count.v, want - r0);
      if (j + (want - r0) > A.xcap)
        set_error(C, OPMOS_ERR_CAPACITY);
      else
        for (unsigned r = r0; r < want; ++r) cs.xpart[j + r - r0] = h << 4 | r;
    }
    if (list) {
      __threadfence();
      atomicExch(&cs.hflag[v], h + 1u);
    }
  }

  // Expansion of up to 32 / L window labels, one per lane group of L lanes
  // (has: the lane's group holds label lid), one round of out-arcs at a time
  // with every lane of the warp taking part: g' = g + c(e), dropped when h(v')
  // is infinite (Algorithm 1). A goal label is not expanded (Algorithm 1); it
  // becomes a candidate at the virtual node n.
  __device__ void expand_labels(uint32_t lid, bool has, unsigned gl, unsigned L, const CandSet& cs, CycleCtl& K1,
                                unsigned long long& pcmp) {
    uint32_t v = 0, e0 = 0, e1 = 0;
    uint32_t g[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = 0;
    if (has) {
      v = A.lnode[lid];
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = A.lg[(size_t)k * A.label_cap + lid];
    }
    const bool goal = has && v == P.goal;
    if (goal && gl == 0) add_candidate(cs, K1, G.n, A.lparent[lid], A.ledge[lid], g);
    if (has && !goal) {
      e0 = __ldg(G.rowptr + v);
      e1 = __ldg(G.rowptr + v + 1);
    }
    const PIdx& pd = S.pd;
    for (uint32_t r = 0;; r += L) {
      const uint32_t e = e0 + gl + r;
      const bool valid = has && !goal && e < e1;
      if (!__any_sync(0xffffffffu, valid)) break;
      uint32_t v2 = 0, g2[D];
      bool alive = false;
      if (valid) {
        v2 = __ldg(G.col + e);
        st[S_CAND]++;
        alive = hk(0, v2) != kInf;  // else the goal is unreachable from v2
      }
#pragma unroll
      for (int k = 0; k < D; ++k) g2[k] = alive ? g[k] + ck(k, e) : 0u;
      if (alive) add_candidate(cs, K1, v2, lid, e, g2);
    }
  }

  // ---------------- extraction of window i+1 from OPEN_i ----------------
  // One warp, the kChunk entries chunk, chunk + nchunks, chunk + 2 nchunks,
  // ... (a merge appends a node's new labels side by side and they tend to
  // fall in the same window, so strided chunks spread the window's labels
  // over the work items): dead entries are dropped (lazy OPEN delete), window
  // entries whose F a logged solution weakly dominates are dropped (lazy
  // PruneOPEN), the other window entries are taken and expanded at once by
  // lane groups; every other entry is carried to OPEN_{i+1} and counted in
  // its histogram.
  __device__ void extract_chunk(unsigned chunk, unsigned n_in, const BinParams& bp, CycleCtl& K1) {
    const unsigned cur = cyc & 1u, nxt = cur ^ 1u;
    const uint64_t* in = A.okey[cur];
    const uint32_t* in_id = A.oid[cur];
    uint64_t* out = A.okey[nxt];
    uint32_t* out_id = A.oid[nxt];
    const CandSet& cs = A.cs[nxt];
    const PIdx& pd = S.pd;
    const unsigned bstar = S.bstar;
    const unsigned lane = lane_id();
    const unsigned L = P.lanes, G_per = 32 / L, grp = lane / L, gl = lane % L;
    unsigned long long kmin = ~0ull, pcmp = 0;
    unsigned wmin = kInf, wmax = 0, f1lo = kInf, f1hi = 0;
    const unsigned nchunks = (n_in + kChunk - 1) / kChunk;
    for (unsigned r = 0; r < kChunk; r += 32) {
      const unsigned i = chunk + (r + lane) * nchunks;
      const bool valid = i < n_in;
      uint64_t key = 0;
      uint32_t id = 0;
      bool keep = false, want = false;
      if (valid) {
        key = in[i];
        id = in_id[i];
        st[S_OSCAN]++;
        if (dead_now(id))
          st[S_DEAD]++;
        else if (bin_of(key, bp) <= bstar)
          want = true;
        else
          keep = true;
      }
      // lazy PruneOPEN: F against the goal costs logged since the label's
      // last check (through the P index when that check predates it)
      uint32_t F[D];
      unsigned since = kInf;
      if (want) {
        const uint32_t v = A.lnode[id];
#pragma unroll
        for (int k = 0; k < D; ++k) F[k] = A.lg[(size_t)k * A.label_cap + id] + hk(k, v);
        since = A.lpver[id];
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) F[k] = 0;
      }
      since = warp_min(since);
      bool alive = want;
      if (since < psnap) {
        if (pd.count && since < pd.mark)
          p_filter(alive, F, pd.mark, psnap, pd.count, pd.ntiles, pd.cur, pcmp);
        else
          p_filter(alive, F, since, psnap, 0, 0, 0, pcmp);
      }
      bool take = false;
      if (want && !alive) {
        st[S_GOALPRUNED]++;
      } else if (want) {
        if (agg_inc(&K1.win_count.v) < A.win_cap) {
          st[S_EXTRACTED]++;
          take = true;
          wmin = min(wmin, (uint32_t)(key >> 32));
          wmax = max(wmax, (uint32_t)(key >> 32));
        } else {
          keep = true;  // window full: stays in OPEN for the next step
        }
      }
      if (keep) {
        const unsigned o = agg_inc(&K1.open_count.v);
        if (o < A.open_cap) {
          out[o] = key;
          out_id[o] = id;
          st[S_OKEEP]++;
          kmin = min(kmin, (unsigned long long)key);
          const unsigned b = bin_of(key, bpn);
          atomicAdd(&S.hist[b], 1u);
          if (b < (unsigned)kNB - 1) {
            f1lo = min(f1lo, (uint32_t)key);
            f1hi = max(f1hi, (uint32_t)key);
          }
        } else {
          set_error(C, OPMOS_ERR_CAPACITY);
        }
      }
      unsigned hits = __ballot_sync(0xffffffffu, take);
      while (hits) {
        const unsigned src = nth_bit(hits, grp);
        const uint32_t lid = __shfl_sync(0xffffffffu, id, src < 32 ? src : 0);
        expand_labels(lid, src < 32, gl, L, cs, K1, pcmp);
        for (unsigned r = 0; r < G_per && hits; ++r) hits &= hits - 1;
      }
    }
    st[S_PCMP] += pcmp;
    kmin = warp_min64(kmin);
    wmin = warp_min(wmin);
    wmax = warp_max(wmax);
    f1lo = warp_min(f1lo);
    f1hi = warp_max(f1hi);
    if (lane == 0) {
      if (kmin != ~0ull) atomicMin(&K1.min_key.v, kmin);
      if (wmin != kInf) {
        atomicMin(&K1.win_min.v, wmin);
        atomicMax(&K1.win_max.v, wmax);
      }
      if (f1lo != kInf) {
        atomicMin(&K1.f1lo.v, f1lo);
        atomicMax(&K1.f1hi.v, f1hi);
      }
    }
  }

  // FIFO order (OPMOS_FLAG_FIFO): one warp takes the ring positions
  // [p0, p1) of window i+1 -- the oldest entries -- and expands every one
  // that is alive and not dominated by a logged solution on F. Nothing is
  // carried: the rest of the ring stays where it is.
  __device__ void extract_fifo(unsigned p0, unsigned p1, CycleCtl& K1) {
    const CandSet& cs = A.cs[(cyc & 1u) ^ 1u];
    const PIdx& pd = S.pd;
    const unsigned lane = lane_id();
    const unsigned L = P.lanes, G_per = 32 / L, grp = lane / L, gl = lane % L;
    unsigned long long pcmp = 0;
    const unsigned pos = p0 + lane;
    const bool valid = pos < p1;
    uint32_t id = 0;
    bool want = false;
    if (valid) {
      id = A.oid[0][pos % A.open_cap];
      st[S_OSCAN]++;
      if (dead_now(id))
        st[S_DEAD]++;
      else
        want = true;
    }
    uint32_t F[D];
    unsigned since = kInf;
    if (want) {
      const uint32_t v = A.lnode[id];
#pragma unroll
      for (int k = 0; k < D; ++k) F[k] = A.lg[(size_t)k * A.label_cap + id] + hk(k, v);
      since = A.lpver[id];
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) F[k] = 0;
    }
    since = warp_min(since);
    bool alive = want;
    if (since < psnap) {
      if (pd.count && since < pd.mark)
        p_filter(alive, F, pd.mark, psnap, pd.count, pd.ntiles, pd.cur, pcmp);
      else
        p_filter(alive, F, since, psnap, 0, 0, 0, pcmp);
    }
    if (want && !alive) st[S_GOALPRUNED]++;
    if (alive) {
      st[S_EXTRACTED]++;
      agg_inc(&K1.win_count.v);
    }
    unsigned hits = __ballot_sync(0xffffffffu, alive);
    while (hits) {
      const unsigned src = nth_bit(hits, grp);
      const uint32_t lid = __shfl_sync(0xffffffffu, id, src < 32 ? src : 0);
      expand_labels(lid, src < 32, gl, L, cs, K1, pcmp);
      for (unsigned r = 0; r < G_per && hits; ++r) hits &= hits - 1;
    }
    st[S_PCMP] += pcmp;
  }

  // F against the P index + the logged goal costs log[t0, t1): clears alive
  // for candidates a solution weakly dominates (Algorithm 1). Every lane of
  // the warp calls it; pcmp counts vector comparisons (lane 0's count is the
  // warp's).
  __device__ __forceinline__ void p_filter(bool& alive, const uint32_t (&F)[D], unsigned t0, unsigned t1,
                                           unsigned pcount, unsigned pntiles, unsigned pbuf,
                                           unsigned long long& pcmp) {
    p_filter(alive, F, t0, t1, pcount, 0u, pntiles, pntiles, pbuf, pcmp);
  }

  // The same over the index tiles [tg_lo, tg_hi) of pntiles only (tg_lo a
  // multiple of 32): the slice one warp of a block takes.
  __device__ void p_filter(bool& alive, const uint32_t (&F)[D], unsigned t0, unsigned t1, unsigned pcount,
                           unsigned tg_lo, unsigned tg_hi, unsigned pntiles, unsigned pbuf,
                           unsigned long long& pcmp) {
    const unsigned lane = lane_id();
    unsigned long long cnt = 0;
    constexpr int UT = kU;  // tail tiles loaded per round
    for (unsigned r0 = t0; r0 < t1; r0 += 32 * UT) {
      if (!__any_sync(0xffffffffu, alive)) break;
      uint32_t pt[UT][D];
#pragma unroll
      for (int u = 0; u < UT; ++u) {
        const unsigned jj = r0 + u * 32 + lane;
#pragma unroll
        for (int k = 0; k < D; ++k) pt[u][k] = jj < t1 ? A.plog[(size_t)k * A.plog_cap + jj] : kInf;
      }
#pragma unroll
      for (int u = 0; u < UT; ++u) {
        const unsigned j0 = r0 + u * 32;
        unsigned amask = __ballot_sync(0xffffffffu, alive);
        if (j0 >= t1 || !amask) break;
        const bool vp = j0 + lane < t1;
        cnt += (unsigned long long)__popc(amask) * min(32u, t1 - j0);
        while (amask) {
          const unsigned j = __ffs(amask) - 1;
          amask &= amask - 1;
          uint32_t Fj[D];
#pragma unroll
          for (int k = 0; k < D; ++k) Fj[k] = __shfl_sync(0xffffffffu, F[k], j);
          const bool wd = vp && weakly_le<D>(pt[u], Fj);
          if (__ballot_sync(0xffffffffu, wd) && lane == j) alive = false;
        }
      }
    }
    if (pcount) {
      const uint32_t* ps = A.ps[pbuf];
      const uint32_t* pst = A.pst[pbuf];
      const size_t tcap = A.plog_cap / 32 + 1;
      constexpr int U = kU;  // tile-minimum groups loaded per round
      for (unsigned tg0 = tg_lo; tg0 < tg_hi; tg0 += 32 * U) {
        if (!__any_sync(0xffffffffu, alive)) break;
        uint32_t tm[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned tl = tg0 + u * 32 + lane;
#pragma unroll
          for (int k = 0; k < D; ++k) tm[u][k] = tl < tg_hi ? pst[(size_t)k * tcap + tl] : kInf;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned tg = tg0 + u * 32;
          unsigned amask = __ballot_sync(0xffffffffu, alive);
          if (tg >= tg_hi || !amask) break;
          const bool vt = tg + lane < tg_hi;
          while (amask) {
            const unsigned j = __ffs(amask) - 1;
            amask &= amask - 1;
            uint32_t Fj[D];
#pragma unroll
            for (int k = 0; k < D; ++k) Fj[k] = __shfl_sync(0xffffffffu, F[k], j);
            unsigned pm = __ballot_sync(0xffffffffu, vt && weakly_le<D>(tm[u], Fj));
            cnt += min(32u, tg_hi - tg);
            bool dead = false;
            while (pm && !dead) {
              // up to kPT passing tiles per round: their loads overlap
              unsigned tt[kPT];
#pragma unroll
              for (int q = 0; q < kPT; ++q) {
                tt[q] = pm ? __ffs(pm) - 1 : 32u;
                pm &= pm - 1;
              }
              uint32_t p[kPT][D];
              bool ve[kPT];
#pragma unroll
              for (int q = 0; q < kPT; ++q) {
                const unsigned e = (tg + tt[q]) * 32 + lane;
                ve[q] = tt[q] < 32u && e < pcount;
#pragma unroll
                for (int k = 0; k < D; ++k) p[q][k] = ve[q] ? ps[(size_t)k * A.plog_cap + e] : kInf;
              }
#pragma unroll
              for (int q = 0; q < kPT; ++q) {
                dead |= __ballot_sync(0xffffffffu, ve[q] && weakly_le<D>(p[q], Fj)) != 0;
                cnt += tt[q] < 32u ? 32 : 0;
              }
            }
            if (dead && lane == j) alive = false;
          }
        }
      }
    }
    if (lane == 0) pcmp += cnt;
  }

  // ---------------- merge of window i's candidates (Algorithm 1: frontier checks, goal branch) ----------------
  // (a) in-batch: lanes holding candidates; a candidate another one strictly
  // dominates, or that equals one with a smaller arc id, is dropped.
  __device__ __forceinline__ bool in_batch_alive(const uint32_t (&c)[D], uint32_t my_edge, bool valid, unsigned nb) {
    const unsigned lane = lane_id();
    bool alive = valid;
    for (unsigned j = 0; j < nb; ++j) {
      uint32_t cj[D];
#pragma unroll
      for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
      const uint32_t ej = __shfl_sync(0xffffffffu, my_edge, j);
      if (alive && lane != j &&
          (dominates<D>(cj, c) || (equal<D>(cj, c) && (ej < my_edge || (ej == my_edge && j < lane)))))
        alive = false;
    }
    return alive;
  }

  // A frontier entry m created in this step (id >= lbase) that candidate j
  // equals takes j's parent and arc if j's arc id is smaller, so the path kept
  // for a cost does not depend on the order in which candidates arrived.
  __device__ __forceinline__ void adopt_smaller_arc(unsigned eqmask, unsigned j, uint32_t mid, uint32_t my_edge,
                                                    uint32_t my_par) {
    const uint32_t ej = __shfl_sync(0xffffffffu, my_edge, j);
    const uint32_t pj = __shfl_sync(0xffffffffu, my_par, j);
    if ((eqmask >> lane_id()) & 1u) {
      if (ej < A.ledge[mid]) {
        A.ledge[mid] = ej;
        A.lparent[mid] = pj;
      }
    }
  }

  // A label created in this step and pruned in it is taken back out of the
  // next OPEN's histogram (its OPEN entry is dropped at the next extraction).
  __device__ __forceinline__ void unhist(const uint32_t (&g)[D], uint32_t v, uint32_t id) {
    if (id >= lbase && v != G.n) atomicSub(&S.hist[bin_of(key_of(g, v), bpn)], 1u);
  }

  __device__ void merge_batch(uint32_t v, int mine, unsigned nb, CycleCtl& K1) {
    const CandSet& cs = A.cs[cyc & 1u];
    const unsigned lane = lane_id();
    const bool is_goal = (v == G.n);  // the virtual node standing for P
    uint32_t c[D];
    const bool valid = lane < nb;
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = valid ? cs.cg[(size_t)k * A.cand_cap + mine] : 0u;
    const uint32_t my_edge = valid ? cs.cedge[mine] : kInf;
    const uint32_t my_par = valid ? cs.cparent[mine] : kInf;
    bool alive = in_batch_alive(c, my_edge, valid, nb);
    uint64_t fb = A.fbase[v];
    unsigned cap = A.fcap[v];
    const unsigned fc = A.fcount[v];
    unsigned out = fc;
    unsigned long long fcmp = 0, pcmp = 0;
    if (is_goal) {
      // (b') at the goal alpha(v_g) is P: one weak-dominance test against the
      // P index and every goal cost logged since it was built (this warp is
      // the only writer of the log in this step). P members a new solution
      // dominates are dropped once, at output (Prune(P, l) of Algorithm 1).
      const unsigned plen = ld_volatile(&C->plog_len.v);
      const PIdx& pd = S.pd;
      p_filter(alive, c, pd.count ? pd.mark : 0u, plen, pd.count, pd.ntiles, pd.cur, pcmp);
    } else {
      // (b) against the frontier alpha(v), compacting it in place; kU tiles
      // of 32 entries are loaded per round
      out = 0;
      constexpr int U = kU;
      bool done = false;
      for (unsigned r0 = 0; r0 < fc && !done; r0 += 32 * U) {
        uint32_t m[U][D];
        uint32_t mid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i = r0 + u * 32 + lane;
          const bool vm = i < fc;
#pragma unroll
          for (int k = 0; k < D; ++k) m[u][k] = vm ? A.fpool[fb + (size_t)k * cap + i] : kInf;
          mid[u] = vm ? A.fpool[fb + (size_t)D * cap + i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i0 = r0 + u * 32;
          if (i0 >= fc) {
            done = true;
            break;
          }
          const unsigned i = i0 + lane;
          const bool vm = i < fc;
          bool pruned = false;
          unsigned amask = __ballot_sync(0xffffffffu, alive);
          if (amask == 0 && out == i0) {
            // nothing left to test and nothing moved: the rest stays in place
            out = fc;
            done = true;
            break;
          }
          fcmp += (unsigned long long)__popc(amask) * min(32u, fc - i0);
          const bool fresh = vm && mid[u] >= lbase;
          while (amask) {
            const unsigned j = __ffs(amask) - 1;
            amask &= amask - 1;
            uint32_t cj[D];
#pragma unroll
            for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
            const bool le_mc = vm && weakly_le<D>(m[u], cj);
            const bool le_cm = vm && weakly_le<D>(cj, m[u]);
            if (__ballot_sync(0xffffffffu, le_mc) && lane == j) alive = false;
            const unsigned eqm = __ballot_sync(0xffffffffu, fresh && le_mc && le_cm);
            if (eqm) adopt_smaller_arc(eqm, j, mid[u], my_edge, my_par);
            pruned |= le_cm && !le_mc;
          }
          const bool keep = vm && !pruned;
          if (vm && pruned) {
            A.ldead[mid[u]] = cyc;
            unhist(m[u], v, mid[u]);
            st[S_PRUNED]++;
          }
          const unsigned km = __ballot_sync(0xffffffffu, keep);
          const unsigned pos = out + __popc(km & lanemask_lt());
          __syncwarp();
          if (keep && pos != i) {
#pragma unroll
            for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + pos] = m[u][k];
            A.fpool[fb + (size_t)D * cap + pos] = mid[u];
          }
          __syncwarp();
          out += __popc(km);
        }
      }
    }
    merge_finish(v, mine, c, valid, alive, out, fb, cap, K1, fcmp, pcmp);
  }

  // The end of a batch's merge, by one warp, lane j holding candidate j:
  // (c) F against P (Algorithm 1) at an ordinary node, then (d) survivors
  // become labels and join alpha(v) and the next OPEN (or the P log at the
  // goal). A candidate P rejects has still pruned the frontier entries it
  // dominates (as in Algorithm 1, where Prune precedes the P test). out =
  // live frontier entries left after (b); fb, cap = the frontier block.
  __device__ void merge_finish(uint32_t v, int mine, const uint32_t (&c)[D], bool valid, bool alive, unsigned out,
                               uint64_t fb, unsigned cap, CycleCtl& K1, unsigned long long fcmp,
                               unsigned long long pcmp, bool p_done = false) {
    const CandSet& cs = A.cs[cyc & 1u];
    const unsigned lane = lane_id();
    const bool is_goal = (v == G.n);
    if (!is_goal && !p_done && __any_sync(0xffffffffu, alive)) {
      uint32_t F[D];
#pragma unroll
      for (int k = 0; k < D; ++k) F[k] = c[k] + (valid ? hk(k, v) : 0u);
      const PIdx& pd = S.pd;
      p_filter(alive, F, pd.count ? pd.mark : 0u, psnap, pd.count, pd.ntiles, pd.cur, pcmp);
    }
    // (d) survivors become labels, join alpha(v), OPEN (or the P log at the goal)
    const unsigned smask = __ballot_sync(0xffffffffu, alive);
    const unsigned ns = __popc(smask);
    if (ns) {
      unsigned lb = 0;
      if (lane == 0) lb = atomicAdd(&C->n_labels.v, ns);
      lb = __shfl_sync(0xffffffffu, lb, 0);
      const bool over_budget = lb + ns > P.label_budget;
      if (lb + ns > A.label_cap || over_budget) {
        if (lane == 0) set_error(C, (lb + ns > A.label_cap) ? OPMOS_ERR_CAPACITY : OPMOS_ERR_BUDGET);
      } else {
        if (lane == 0) atomicMax(&K1.lbase.v, lb + ns);
        const unsigned need = out + ns;
        if (need > cap) {
          // grow: new block of twice the size, copy the live entries
          const unsigned tile = P.tile;
          unsigned ncap = max(2u * need, tile);
          ncap = (ncap + tile - 1) / tile * tile;
          unsigned long long nb0 = 0;
          if (lane == 0) nb0 = atomicAdd(&C->f_words.v, (unsigned long long)(D + 1) * ncap);
          nb0 = __shfl_sync(0xffffffffu, nb0, 0);
          if (nb0 + (unsigned long long)(D + 1) * ncap > A.fpool_words) {
            if (lane == 0) set_error(C, OPMOS_ERR_CAPACITY);
            return;
          }
          for (unsigned i = lane; i < out; i += 32) {
#pragma unroll
            for (int k = 0; k <= D; ++k) A.fpool[nb0 + (size_t)k * ncap + i] = A.fpool[fb + (size_t)k * cap + i];
          }
          fb = nb0;
          cap = ncap;
          if (lane == 0) {
            A.fbase[v] = fb;
            A.fcap[v] = cap;
          }
        }
        unsigned plen = 0;
        if (is_goal) {
          plen = ld_volatile(&C->plog_len.v);
          if (plen + ns > A.plog_cap) {
            if (lane == 0) set_error(C, OPMOS_ERR_CAPACITY);
            return;
          }
        }
        if (alive) {
          const unsigned r = __popc(smask & lanemask_lt());
          const unsigned id = lb + r;
#pragma unroll
          for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap + id] = c[k];
          A.lnode[id] = is_goal ? P.goal : v;
          A.lparent[id] = cs.cparent[mine];
          A.ledge[id] = cs.cedge[mine];
          A.lpver[id] = psnap;
          A.ldead[id] = kAlive;
#pragma unroll
          for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + out + r] = c[k];
          A.fpool[fb + (size_t)D * cap + out + r] = id;
          if (is_goal) {
#pragma unroll
            for (int k = 0; k < D; ++k) A.plog[(size_t)k * A.plog_cap + plen + r] = c[k];
          } else {
            push_open(id, c, v, K1);
          }
        }
        if (is_goal && lane == 0) {
          __threadfence();
          *reinterpret_cast<volatile unsigned*>(&C->plog_len.v) = plen + ns;
          atomicMax(&K1.plen.v, plen + ns);
        }
        out += ns;
      }
    }
    if (lane == 0) {
      A.fcount[v] = out;
      st[S_INSERTED] += ns;
      st[S_FCMP] += fcmp;
      st[S_PCMP] += pcmp;
    }
  }

  // A new label joins the next OPEN: the array of step i+1 (counted in its
  // histogram) or, with OPMOS_FLAG_FIFO, the ring's tail (positions
  // [head, tail) of this step are never written over).
  __device__ __forceinline__ void push_open(uint32_t id, const uint32_t (&c)[D], uint32_t v, CycleCtl& K1) {
    if (P.flags & OPMOS_FLAG_FIFO) {
      const unsigned o = agg_inc(&C->fifo_tail.v);
      if (o - fifo_head < A.open_cap) {
        A.oid[0][o % A.open_cap] = id;
        atomicMax(&K1.open_count.v, o + 1u);
      } else {
        set_error(C, OPMOS_ERR_CAPACITY);
      }
      return;
    }
    const uint64_t key = key_of(c, v);
    const unsigned o = agg_inc(&K1.open_count.v);
    if (o < A.open_cap) {
      const unsigned nxt = (cyc & 1u) ^ 1u;
      A.okey[nxt][o] = key;
      A.oid[nxt][o] = id;
      atomicAdd(&S.hist[bin_of(key, bpn)], 1u);
    } else {
      set_error(C, OPMOS_ERR_CAPACITY);
    }
  }

  // A warp's cursor over node v's candidates of one step: the slots 32 at a
  // time, then the node's 2^lsub lists, lane j walking list j. Opening it
  // reads and clears the node's count and list heads (the set is reused two
  // steps later).
  struct Cursor {
    unsigned ncand;  // candidates of the node this step
    unsigned next;   // next slot index to read
    int lcur;        // lane j < 2^lsub: its position in list j (kNil at the end)
  };
  __device__ __forceinline__ Cursor open_cursor(const CandSet& cs, uint32_t v) {
    const unsigned lane = lane_id();
    Cursor q;
    q.ncand = cs.ncand[v];
    q.next = 0;
    // lists holding something: min(candidates beyond the slots, 2^lsub)
    const unsigned nl = q.ncand > A.nslots ? min(q.ncand - A.nslots, 1u << A.lsub) : 0u;
    int32_t* heads = cs.node_head + ((size_t)v << A.lsub);
    q.lcur = lane < nl ? heads[lane] : kNil;
    __syncwarp();
    if (lane == 0) cs.ncand[v] = 0;
    if (lane < nl) heads[lane] = kNil;
    return q;
  }
  __device__ __forceinline__ bool cursor_more(const Cursor& q) const {
    return q.next < min(q.ncand, A.nslots) || __any_sync(0xffffffffu, q.lcur != kNil);
  }
  // Next batch (up to 32): the lane's candidate (kNil if none) and the batch
  // size in *nb; the batch's candidates sit in lanes 0 .. *nb - 1.
  __device__ __forceinline__ int next_batch(const CandSet& cs, uint32_t v, Cursor& q, unsigned* nb) {
    const unsigned lane = lane_id();
    int mine = kNil;
    const unsigned in_slots = min(q.ncand, A.nslots);
    if (q.next < in_slots) {
      const unsigned n = min(32u, in_slots - q.next);
      if (lane < n) mine = cs.cslot[(size_t)v * A.nslots + q.next + lane];
      q.next += n;
      *nb = n;
    } else {
      // rounds over the lists side by side: the lanes still inside a list
      // hand their candidates to lanes n, n+1, ... and step on
      unsigned n = 0;
      for (;;) {
        const unsigned bal = __ballot_sync(0xffffffffu, q.lcur != kNil);
        if (bal == 0u || n >= 32u) break;
        const unsigned cnt = __popc(bal);
        const unsigned t = lane - n;  // this lane receives the t-th candidate of the round
        const bool recv = lane >= n && t < cnt;
        const int got = __shfl_sync(0xffffffffu, q.lcur, recv ? nth_bit(bal, t) : 0u);
        if (recv) mine = got;
        if (q.lcur != kNil && n + __popc(bal & lanemask_lt()) < 32u) q.lcur = cs.cnext[q.lcur];
        n = min(32u, n + cnt);
      }
      *nb = n;
    }
    return mine;
  }

  // One node's merge by one warp.
  __device__ void merge_node(uint32_t v, CycleCtl& K1) {
    const CandSet& cs = A.cs[cyc & 1u];
    Cursor q = open_cursor(cs, v);
    do {
      unsigned nb = 0;
      const int mine = next_batch(cs, v, q, &nb);
      merge_batch(v, mine, nb, K1);
    } while (cursor_more(q));
  }

  // Merge of a node with a large frontier, or many candidates, by the whole
  // block (every thread calls it). Up to kHC candidates at a time sit in
  // shared memory (the node's slots, then its list):
  //  (a) every thread resolves one candidate against all the others (strict
  //      dominance; of equal ones the smallest arc id stays);
  //  (b) all warps scan the frontier in rounds of nwarps * 32 * kUH entries,
  //      each warp kUH tiles of 32 against every live candidate, and compact
  //      it in place: a round's reads all precede the first barrier, its
  //      writes land below the round's start, so they never overwrite an
  //      entry another warp still has to read. Candidates killed by one warp
  //      are dropped by the others from the next round on; a candidate that a
  //      frontier entry weakly dominates never dominates another entry (the
  //      frontier is an antichain), so the entries each candidate prunes do
  //      not depend on when its death is seen;
  //  (c) F against P, 32 candidates per warp, the P log tail and the index
  //      tiles split between the warps that hold the same candidates;
  //  (d) survivors become labels, join alpha(v) and the next OPEN.
  __device__ void merge_heavy(uint32_t v, CycleCtl& K1) {
    open_block_cursor(A.cs[cyc & 1u], v, false);
    __syncthreads();
    heavy_groups(v, K1, false);
  }

  // Warp 0 opens node v's cursor for a block merge in shared memory:
  // S.mq_ncand candidates, slots from S.mq_next (past the slots if
  // slots_done), list positions in S.hlist. A block barrier must follow.
  __device__ void open_block_cursor(const CandSet& cs, uint32_t v, bool slots_done) {
    if (threadIdx.x < 32) {
      const Cursor q = open_cursor(cs, v);
      S.hlist[threadIdx.x] = q.lcur;
      if (threadIdx.x == 0) {
        S.mq_ncand = q.ncand;
        S.mq_next = slots_done ? min(q.ncand, A.nslots) : 0u;
      }
    }
  }

  // The next group (up to kHC, one per thread) of a block merge's candidates, into S.hcid;
  // returns its size (every thread), 0 once none is left. First the slot
  // rows S.mq_next, S.mq_next + 1, ... below nrows, row j being slot
  // first + j * stride, then the lists whose cursors sit in S.hlist, walked
  // side by side by warp 0. With filtered, candidates a part of a split merge
  // dropped are skipped (and the group still fills while any are left).
  __device__ unsigned gather_group(const CandSet& cs, uint32_t v, unsigned nrows, unsigned first, unsigned stride,
                                   bool filtered) {
    const unsigned tid = threadIdx.x;
    const unsigned hcap = min(kHC, blockDim.x);  // one candidate per thread
    unsigned s0 = S.mq_next, n0 = 0;
    if (!filtered) {  // every slot below the count holds a candidate
      n0 = s0 < nrows ? min(hcap, nrows - s0) : 0u;
      if (tid < n0) S.hcid[tid] = cs.cslot[(size_t)v * A.nslots + first + (s0 + tid) * stride];
      s0 += n0;
    }
    while (s0 < nrows && n0 < hcap) {  // (uniform: s0 and n0 are the same in every thread)
      const unsigned take = min(hcap - n0, nrows - s0);
      int c = kNil;
      if (tid < take) c = cs.cslot[(size_t)v * A.nslots + first + (s0 + tid) * stride];
      const bool keep = c != kNil && __ldcg(cs.cflag + c) == 0u;
      unsigned cnt;
      const unsigned pos = block_exclusive_scan(keep ? 1u : 0u, S.warp, cnt);  // (every thread has read mq_next)
      if (keep) S.hcid[n0 + pos] = c;
      n0 += cnt;
      s0 += take;
    }
    __syncthreads();
    if (tid < 32) {
      int cur = S.hlist[tid];
      unsigned n = n0;
      for (;;) {
        const bool live = cur != kNil;
        if (!__any_sync(0xffffffffu, live) || n >= hcap) break;
        const bool kp = live && (!filtered || __ldcg(cs.cflag + cur) == 0u);
        const unsigned bal = __ballot_sync(0xffffffffu, kp);
        const unsigned rk = __popc(bal & lanemask_lt());
        const bool put = kp && n + rk < hcap;
        if (put) S.hcid[n + rk] = cur;
        if (put || (live && !kp)) cur = cs.cnext[cur];
        n = min(hcap, n + __popc(bal));
      }
      S.hlist[tid] = cur;
      const bool more = s0 < nrows || __any_sync(0xffffffffu, cur != kNil);
      if (tid == 0) {
        S.mq_next = s0;
        S.m_nb = n;
        S.m_more = more;
      }
    }
    __syncthreads();
    return S.m_nb;
  }

  // A gathered group's costs, arcs and parents into shared memory; the
  // group's kill words cleared. A block barrier must follow.
  __device__ void load_group(const CandSet& cs, unsigned nb) {
    const unsigned tid = threadIdx.x;
    if (tid < nb) {
      const int c = S.hcid[tid];
#pragma unroll
      for (int k = 0; k < D; ++k) S.hc[k][tid] = cs.cg[(size_t)k * A.cand_cap + c];
      S.hedge[tid] = cs.cedge[c];
      S.hpar[tid] = cs.cparent[c];
    }
    if (tid < kHC / 32) {
      S.halive[tid] = 0;
      S.hkill[tid] = 0;
      S.hpkill[tid] = 0;
    }
  }

  // In-set resolution of a group (Sec. 5's Dup&Dom): candidate tid dies when
  // another strictly dominates it or equals it with a smaller (arc, index);
  // the survivors' words go to S.halive. A block barrier must follow.
  __device__ void group_inset(unsigned nb) {
    const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    bool alive = tid < nb;
    if (alive) {
      uint32_t ct[D];
#pragma unroll
      for (int k = 0; k < D; ++k) ct[k] = S.hc[k][tid];
      const uint32_t et = S.hedge[tid];
      for (unsigned j = 0; j < nb && alive; ++j) {
        if (j == tid) continue;
        uint32_t cj[D];
#pragma unroll
        for (int k = 0; k < D; ++k) cj[k] = S.hc[k][j];
        const uint32_t ej = S.hedge[j];
        if (dominates<D>(cj, ct) || (equal<D>(cj, ct) && (ej < et || (ej == et && j < tid)))) alive = false;
      }
    }
    const unsigned am = __ballot_sync(0xffffffffu, alive);
    if (lane == 0 && w < kHC / 32) S.halive[w] = am;
  }

  // F against P for the live candidates of group word q, this warp taking
  // slice sl of nsl of the P log entries [t0, t1) and of the first nt index
  // tiles; the ones P dominates are flagged in S.hpkill. At the goal node n,
  // F = g (h(n) = 0).
  __device__ void group_ptest(uint32_t v, unsigned q, unsigned nsl, unsigned sl, unsigned t0, unsigned t1,
                              unsigned nt) {
    const unsigned lane = lane_id();
    const unsigned word = S.halive[q] & ~S.hkill[q];
    if (!word || sl >= nsl) return;
    const PIdx& pd = S.pd;
    const unsigned jj = q * 32 + lane;
    uint32_t F[D];
#pragma unroll
    for (int k = 0; k < D; ++k) F[k] = S.hc[k][jj] + (v == G.n ? 0u : hk(k, v));
    bool alive = (word >> lane) & 1u;
    const unsigned tper = ((t1 - min(t0, t1) + nsl - 1) / nsl + 31) / 32 * 32;
    const unsigned lo = min(t1, t0 + sl * tper), hi = min(t1, lo + tper);
    const unsigned gper = ((nt + nsl - 1) / nsl + 31) / 32 * 32;
    const unsigned glo = min(nt, sl * gper), ghi = min(nt, glo + gper);
    unsigned long long pcmp = 0;
    p_filter(alive, F, lo, hi, pd.count, glo, ghi, nt, pd.cur, pcmp);
    st[S_PCMP] += pcmp;
    const unsigned pk = __ballot_sync(0xffffffffu, !alive) & word;
    if (lane == 0 && pk) atomicOr(&S.hpkill[q], pk);
  }

  // The group loop of a block merge, from the cursor in shared memory
  // (S.mq_ncand candidates, slots from S.mq_next, then the lists at
  // S.hlist). filtered: the survivors of a split merge's parts (the ones
  // without cflag), already checked against the frontier's first `old`
  // entries, so only the entries the loop itself inserts are scanned. At the
  // goal node n there is no frontier scan: alpha(n) is P, and candidates meet
  // P through the P index and log, up to the entries this merge appended
  // (from entry pfrom on only, when filtered: the parts tested the rest).
  __device__ void heavy_groups(uint32_t v, CycleCtl& K1, bool filtered, unsigned old = 0, unsigned pfrom = 0) {
    const bool goal = v == G.n;
    constexpr int U = kUH;
    constexpr unsigned NW = kHC / 32;  // candidate words
    const CandSet& cs = A.cs[cyc & 1u];
    const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
    const unsigned in_slots = min(S.mq_ncand, A.nslots);
    for (;;) {
      const unsigned nb = gather_group(cs, v, in_slots, 0u, 1u, filtered);
      if (nb == 0) break;
      const unsigned nwords = (nb + 31) / 32;
      load_group(cs, nb);
      __syncthreads();
      // (a) in-set resolution
      group_inset(nb);
      __syncthreads();
      // (b) the frontier
      const uint64_t fb = A.fbase[v];
      const unsigned cap = A.fcap[v];
      const unsigned fc = A.fcount[v];
      unsigned out = goal ? fc : old;
      unsigned long long fcmp = 0;
      const unsigned R = nw * 32u * U;
      for (unsigned r0 = out; r0 < fc; r0 += R) {
        const unsigned base = r0 + w * 32u * U;
        uint32_t m[U][D];
        uint32_t mid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i = base + u * 32 + lane;
          const bool vm = i < fc;
#pragma unroll
          for (int k = 0; k < D; ++k) m[u][k] = vm ? A.fpool[fb + (size_t)k * cap + i] : kInf;
          mid[u] = vm ? A.fpool[fb + (size_t)D * cap + i] : 0u;
        }
        unsigned kill[NW], km[U], wtot = 0;
#pragma unroll
        for (unsigned q = 0; q < NW; ++q) kill[q] = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i0 = base + u * 32;
          const unsigned i = i0 + lane;
          const bool vm = i < fc;
          const bool fresh = vm && mid[u] >= lbase;
          bool pruned = false;
          if (i0 < fc) {
#pragma unroll
            for (unsigned q = 0; q < NW; ++q) {
              if (q >= nwords) break;
              unsigned am = S.halive[q] & ~S.hkill[q] & ~kill[q];
              fcmp += (unsigned long long)__popc(am) * min(32u, fc - i0);
              while (am) {
                const unsigned j = __ffs(am) - 1;
                am &= am - 1;
                const unsigned jj = q * 32 + j;
                uint32_t cj[D];
#pragma unroll
                for (int k = 0; k < D; ++k) cj[k] = S.hc[k][jj];
                const bool le_mc = vm && weakly_le<D>(m[u], cj);
                const bool le_cm = vm && weakly_le<D>(cj, m[u]);
                if (__ballot_sync(0xffffffffu, le_mc)) kill[q] |= 1u << j;
                if (fresh && le_mc && le_cm && S.hedge[jj] < A.ledge[mid[u]]) {
                  A.ledge[mid[u]] = S.hedge[jj];
                  A.lparent[mid[u]] = S.hpar[jj];
                }
                pruned |= le_cm && !le_mc;
              }
            }
          }
          if (vm && pruned) {
            A.ldead[mid[u]] = cyc;
            unhist(m[u], v, mid[u]);
            st[S_PRUNED]++;
          }
          km[u] = __ballot_sync(0xffffffffu, vm && !pruned);
          wtot += __popc(km[u]);
        }
        if (lane == 0) {
          S.warp[w] = wtot;
#pragma unroll
          for (unsigned q = 0; q < NW; ++q)
            if (kill[q]) atomicOr(&S.hkill[q], kill[q]);
        }
        __syncthreads();  // (1) all reads of this round are done
        const unsigned x = lane < nw ? S.warp[lane] : 0u;
        unsigned incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= (unsigned)o) incl += y;
        }
        const unsigned wpre = __shfl_sync(0xffffffffu, incl - x, w);
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned pos = out + wpre;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i = base + u * 32 + lane;
          const bool keep = (km[u] >> lane) & 1u;
          const unsigned p = pos + __popc(km[u] & lanemask_lt());
          if (keep && p != i) {
#pragma unroll
            for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + p] = m[u][k];
            A.fpool[fb + (size_t)D * cap + p] = mid[u];
          }
          pos += __popc(km[u]);
        }
        bool any = false;
#pragma unroll
        for (unsigned q = 0; q < NW; ++q) any |= (S.halive[q] & ~S.hkill[q]) != 0;
        __syncthreads();  // (2) S.warp and S.hkill read by every warp
        const unsigned seen = min(r0 + R, fc);
        out += total;
        if (!any && out == seen) {
          // no candidate left to test and nothing moved: the rest stays in place
          out = fc;
          break;
        }
      }
      if (lane == 0) st[S_FCMP] += fcmp;
      // (c) F against P: warp w takes candidate word w % nwords and one of the
      // nw / nwords slices of the P log tail and of the index tiles
      {
        const unsigned pl = goal ? ld_volatile(&C->plog_len.v) : psnap;
        if (goal && filtered)
          group_ptest(v, w % nwords, nw / nwords, w / nwords, pfrom, pl, 0u);
        else
          group_ptest(v, w % nwords, nw / nwords, w / nwords, S.pd.count ? S.pd.mark : 0u, pl,
                      S.pd.count ? S.pd.ntiles : 0u);
      }
      __syncthreads();
      // (d) survivors become labels, join alpha(v) and the next OPEN
      const bool surv = tid < nb && (((S.halive[w % NW] & ~S.hkill[w % NW] & ~S.hpkill[w % NW]) >> lane) & 1u);
      heavy_insert(v, K1, surv, out, fb, cap);
      const bool more = S.m_more;
      __syncthreads();  // the next group reuses the shared candidate arrays
      if (!more) break;
    }
  }

  // Survivors of a block merge (thread tid holds candidate tid in shared
  // memory; surv tells whether it survived) become labels, join alpha(v) --
  // out live entries at fb, cap, grown when full -- and the next OPEN, or at
  // the goal node n the P log. Returns alpha(v)'s new size (the block must
  // pass a barrier before the shared candidate arrays are reused).
  __device__ unsigned heavy_insert(uint32_t v, CycleCtl& K1, bool surv, unsigned out, uint64_t fb, unsigned cap) {
    const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
    const bool goal = v == G.n;
    const unsigned smask = __ballot_sync(0xffffffffu, surv);
    if (lane == 0) S.warp[w] = __popc(smask);
    __syncthreads();
    unsigned pre = 0, ntot = 0;
    for (unsigned q = 0; q < nw; ++q) {
      const unsigned c = S.warp[q];
      pre += q < w ? c : 0u;
      ntot += c;
    }
    const unsigned rank = pre + __popc(smask & lanemask_lt());
    if (tid == 0) {
      S.m_ok = 0;
      S.m_fb = fb;
      S.m_cap = cap;
      if (ntot) {
        const unsigned lb = atomicAdd(&C->n_labels.v, ntot);
        S.m_lb = lb;
        if (lb + ntot > A.label_cap || lb + ntot > P.label_budget) {
          set_error(C, (lb + ntot > A.label_cap) ? OPMOS_ERR_CAPACITY : OPMOS_ERR_BUDGET);
        } else if (goal && ld_volatile(&C->plog_len.v) + ntot > A.plog_cap) {
          set_error(C, OPMOS_ERR_CAPACITY);
        } else {
          atomicMax(&K1.lbase.v, lb + ntot);
          S.m_ok = 1;
          S.m_plen = goal ? ld_volatile(&C->plog_len.v) : 0u;  // this block is the log's only writer
          if (out + ntot > cap) {  // grow: a new block of twice the size
            const unsigned tile = P.tile;
            unsigned ncap = max(2u * (out + ntot), tile);
            ncap = (ncap + tile - 1) / tile * tile;
            const unsigned long long nb0 = atomicAdd(&C->f_words.v, (unsigned long long)(D + 1) * ncap);
            if (nb0 + (unsigned long long)(D + 1) * ncap > A.fpool_words) {
              set_error(C, OPMOS_ERR_CAPACITY);
              S.m_ok = 0;
            } else {
              S.m_fb = nb0;
              S.m_cap = ncap;
            }
          }
        }
      }
    }
    __syncthreads();
    const unsigned ok = S.m_ok;
    if (ok) {
      const uint64_t nfb = S.m_fb;
      const unsigned ncap = S.m_cap;
      if (nfb != fb) {
        for (unsigned x = tid; x < out; x += blockDim.x)
#pragma unroll
          for (int k = 0; k <= D; ++k) A.fpool[nfb + (size_t)k * ncap + x] = A.fpool[fb + (size_t)k * cap + x];
      }
      if (surv) {
        const unsigned id = S.m_lb + rank;
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = S.hc[k][tid];
#pragma unroll
        for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap + id] = c[k];
        A.lnode[id] = goal ? P.goal : v;
        A.lparent[id] = S.hpar[tid];
        A.ledge[id] = S.hedge[tid];
        A.lpver[id] = psnap;
        A.ldead[id] = kAlive;
#pragma unroll
        for (int k = 0; k < D; ++k) A.fpool[nfb + (size_t)k * ncap + out + rank] = c[k];
        A.fpool[nfb + (size_t)D * ncap + out + rank] = id;
        if (goal) {
#pragma unroll
          for (int k = 0; k < D; ++k) A.plog[(size_t)k * A.plog_cap + S.m_plen + rank] = c[k];
        } else {
          push_open(id, c, v, K1);
        }
      }
      if (goal) {
        __syncthreads();  // the log entries are written before they are published
        if (tid == 0) {
          __threadfence();
          *reinterpret_cast<volatile unsigned*>(&C->plog_len.v) = S.m_plen + ntot;
          atomicMax(&K1.plen.v, S.m_plen + ntot);
        }
      }
      if (tid == 0) {
        A.fbase[v] = nfb;
        A.fcap[v] = ncap;
        A.fcount[v] = out + ntot;
        st[S_INSERTED] += ntot;
      }
    } else if (tid == 0) {
      A.fcount[v] = out;
    }
    return ok ? out + ntot : out;
  }

  // Compaction of a frontier after a split merge: the entries whose label
  // was pruned in this step (ldead == cyc, written by other blocks: read past
  // L1) are removed; returns the live count. Rounds as in heavy_groups (b).
  __device__ unsigned compact_pruned(uint64_t fb, unsigned cap, unsigned F) {
    constexpr int U = kUH;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned R = nw * 32u * U;
    unsigned out = 0;
    for (unsigned r0 = 0; r0 < F; r0 += R) {
      const unsigned base = r0 + w * 32u * U;
      uint32_t m[U][D];
      uint32_t mid[U];
      unsigned km[U], wtot = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned i = base + u * 32 + lane;
        const bool vm = i < F;
#pragma unroll
        for (int k = 0; k < D; ++k) m[u][k] = vm ? A.fpool[fb + (size_t)k * cap + i] : 0u;
        mid[u] = vm ? A.fpool[fb + (size_t)D * cap + i] : 0u;
        km[u] = __ballot_sync(0xffffffffu, vm && __ldcg(A.ldead + mid[u]) != cyc);
        wtot += __popc(km[u]);
      }
      if (lane == 0) S.warp[w] = wtot;
      __syncthreads();  // (1) all reads of this round are done
      const unsigned x = lane < nw ? S.warp[lane] : 0u;
      unsigned incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += y;
      }
      const unsigned wpre = __shfl_sync(0xffffffffu, incl - x, w);
      const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned pos = out + wpre;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned i = base + u * 32 + lane;
        const bool keep = (km[u] >> lane) & 1u;
        const unsigned p = pos + __popc(km[u] & lanemask_lt());
        if (keep && p != i) {
#pragma unroll
          for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + p] = m[u][k];
          A.fpool[fb + (size_t)D * cap + p] = mid[u];
        }
        pos += __popc(km[u]);
      }
      __syncthreads();  // (2) S.warp read by every warp
      out += total;
    }
    return out;
  }

  // Shape of a merge split into k parts: ka shares of the candidates (ka
  // divides k, each share kPartCands candidates or more) times kb = k / ka
  // ranges of the frontier. Splitting the candidates keeps each candidate's
  // early exit in one scan, so it is preferred.
  __device__ static void part_shape(unsigned k, unsigned nc, unsigned& ka, unsigned& kb) {
    const unsigned amax = max(1u, nc / kPartCands);
    ka = 1;
    for (unsigned x = 2; x <= k; ++x)
      if (k % x == 0 && x <= amax) ka = x;
    kb = k / ka;
  }

  // Part r of a block merge split into k parts (k >= 2; decided while the
  // node's candidates arrived). With the shape (ka, kb), part r = b * ka + a
  // takes share a of the candidates -- slots a, a + ka, ... and lists a,
  // a + ka, ... -- kHC at a time, and frontier entries [b F / kb,
  // (b+1) F / kb), read only:
  //  (a) in-set resolution within each group;
  //  (b) frontier entries a candidate strictly dominates are marked pruned
  //      (ldead = cyc); candidates an entry weakly dominates die;
  // and the candidates that died get cflag set. Each dies only when a
  // candidate of its group or a frontier entry dominates it, and every entry
  // some candidate strictly dominates is marked (dominance is transitive and
  // the frontier is an antichain). The last part to finish (a counter per
  // node; nobody waits) compacts the frontier if a part pruned, then merges
  // the surviving candidates as one block merge does -- against each other,
  // the entries it inserts and P -- so P tests only the survivors. At the goal
  // node n, whose alpha is P, the parts split the candidates only and test
  // them against P; the last part tests the survivors against the log
  // entries it appends itself.
  __device__ void merge_part(uint32_t v, unsigned r, unsigned k, CycleCtl& K1) {
    constexpr int U = kUH;
    constexpr unsigned NW = kHC / 32;
    const CandSet& cs = A.cs[cyc & 1u];
    const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
    const unsigned F = A.fcount[v];
    const unsigned nc = cs.ncand[v];
    const uint64_t fb = A.fbase[v];
    const unsigned cap = A.fcap[v];
    const bool goal = v == G.n;  // no frontier ranges: the parts test their shares against P
    unsigned ka = k, kb = 1;
    if (!goal) part_shape(k, nc, ka, kb);
    const unsigned a = r % ka, b = r / ka;
    const unsigned lo = (unsigned)((uint64_t)F * b / kb), hi = goal ? 0u : (unsigned)((uint64_t)F * (b + 1) / kb);
    const unsigned ns = min(nc, A.nslots), nl = nc - ns;
    if (tid < 32) {  // this share's lists (the node's heads stay until the last part resets them)
      const unsigned j = a + tid * ka;
      S.hlist[tid] = (j < (1u << A.lsub) && j < nl) ? cs.node_head[((size_t)v << A.lsub) + j] : kNil;
      if (tid == 0) S.mq_next = 0;
    }
    __syncthreads();
    const unsigned nrows = ns > a ? (ns - a + ka - 1) / ka : 0u;
    unsigned long long fcmp = 0;
    bool any_pruned = false;
    for (;;) {
      const unsigned nb = gather_group(cs, v, nrows, a, ka, false);
      if (nb == 0) break;
      const unsigned nwords = (nb + 31) / 32;
      load_group(cs, nb);
      __syncthreads();
      group_inset(nb);
      __syncthreads();
      // (b) the frontier range, read only, until no candidate of the group lives
      for (unsigned r0 = lo + w * 32u * U; r0 < hi; r0 += nw * 32u * U) {
        bool any = false;
#pragma unroll
        for (unsigned q = 0; q < NW; ++q) any |= q < nwords && (S.halive[q] & ~S.hkill[q]) != 0u;
        if (!any) break;
        uint32_t m[U][D];
        uint32_t mid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i = r0 + u * 32 + lane;
          const bool vm = i < hi;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) m[u][kk] = vm ? A.fpool[fb + (size_t)kk * cap + i] : kInf;
          mid[u] = vm ? A.fpool[fb + (size_t)D * cap + i] : 0u;
        }
        unsigned kill[NW];
#pragma unroll
        for (unsigned q = 0; q < NW; ++q) kill[q] = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i0 = r0 + u * 32;
          const bool vm = i0 + lane < hi;
          bool pruned = false;
          if (i0 < hi) {
#pragma unroll
            for (unsigned q = 0; q < NW; ++q) {
              if (q >= nwords) break;
              unsigned am = S.halive[q] & ~S.hkill[q] & ~kill[q];
              fcmp += (unsigned long long)__popc(am) * min(32u, hi - i0);
              while (am) {
                const unsigned j = __ffs(am) - 1;
                am &= am - 1;
                uint32_t cj[D];
#pragma unroll
                for (int kk = 0; kk < D; ++kk) cj[kk] = S.hc[kk][q * 32 + j];
                const bool le_mc = vm && weakly_le<D>(m[u], cj);
                const bool le_cm = vm && weakly_le<D>(cj, m[u]);
                if (__ballot_sync(0xffffffffu, le_mc)) kill[q] |= 1u << j;
                pruned |= le_cm && !le_mc;
              }
            }
          }
          if (vm && pruned) {
            A.ldead[mid[u]] = cyc;
            st[S_PRUNED]++;
            any_pruned = true;
          }
        }
        if (lane == 0) {
#pragma unroll
          for (unsigned q = 0; q < NW; ++q)
            if (kill[q]) atomicOr(&S.hkill[q], kill[q]);
        }
      }
      __syncthreads();
      if (goal) {  // P as the parts see it: no part appends to the log
        group_ptest(v, w % nwords, nw / nwords, w / nwords, S.pd.count ? S.pd.mark : 0u,
                    ld_volatile(&C->plog_len.v), S.pd.count ? S.pd.ntiles : 0u);
        __syncthreads();
      }
      if (tid < nb) {
        const unsigned q = tid >> 5, bit = 1u << (tid & 31);
        if (((S.hkill[q] | S.hpkill[q]) & bit) || !(S.halive[q] & bit)) cs.cflag[S.hcid[tid]] = 1u;
      }
      const bool more = S.m_more;
      __syncthreads();  // the next group reuses the shared arrays
      if (!more) break;
    }
    if (lane == 0) st[S_FCMP] += fcmp;
    // the part counter's low 16 bits count finished parts; kPartPruned is
    // added by a part that pruned a frontier entry
    const unsigned pr = __syncthreads_or(any_pruned) ? kPartPruned : 0u;
    __threadfence();
    if (tid == 0) {
      const unsigned c = atomicAdd(&cs.hcnt[v], 1u + pr) + 1u + pr;
      S.m_ok = (c & (kPartPruned - 1u)) == k ? (c >= kPartPruned ? 2u : 1u) : 0u;
    }
    __syncthreads();
    const unsigned ok = S.m_ok;
    if (!ok) return;
    // the last part of the node: the survivors of every share
    __threadfence();
    open_block_cursor(cs, v, false);
    if (tid == 0) cs.hcnt[v] = 0;
    unsigned out = F;
    if (ok == 2u) {  // some part pruned an entry: compact
      out = compact_pruned(fb, cap, F);
      if (tid == 0) A.fcount[v] = out;
    }
    __syncthreads();
    heavy_groups(v, K1, true, out, ld_volatile(&C->plog_len.v));
  }

  // ---------------- P index rebuild (three steps, then published) ----------------
  // Rank item: the Z-order rank contributions of 32 logged goal costs (one
  // per lane) from kRankQ others, added into prank.
  __device__ void rank_item(unsigned item) {
    if constexpr (D >= 2) {
      constexpr int MD = D - 1 < 3 ? D - 1 : 3;
      const PIdx& pd = S.pd;
      const unsigned k = pd.k;
      const unsigned nq = (k + kRankQ - 1) / kRankQ;
      const unsigned eb = item / nq, qc = item % nq;
      const unsigned lane = lane_id();
      const unsigned i = eb * 32 + lane;
      const bool vi = i < k;
      const size_t pc = A.plog_cap;
      uint32_t lo[MD], zi[MD];
#pragma unroll
      for (int j = 0; j < MD; ++j) {
        lo[j] = hk(j + 1, P.start);
        zi[j] = vi ? (A.plog[(size_t)(j + 1) * pc + i] - lo[j]) >> pd.shift[j] : 0u;
      }
      unsigned rank = 0;
      const unsigned q1 = min(k, (qc + 1) * kRankQ);
      for (unsigned q = qc * kRankQ; q < q1; ++q) {
        uint32_t zq[MD];
#pragma unroll
        for (int j = 0; j < MD; ++j) zq[j] = (A.plog[(size_t)(j + 1) * pc + q] - lo[j]) >> pd.shift[j];
        rank += z_less<MD>(zq, zi) || (q < i && !z_less<MD>(zi, zq));
      }
      if (vi && rank) atomicAdd(&A.prank[i], rank);
    }
  }

  template <class Team>
  __device__ void index_strided_work(const Team& T) {
    if constexpr (D >= 2) {
      const PIdx& pd = S.pd;
      const unsigned k = pd.k, nb = pd.nb;
      const size_t pc = A.plog_cap;
      if (pd.state == 2) {  // scatter every logged cost to its rank
        for (unsigned x = T.tid(); x < k; x += T.nthreads()) {
          const unsigned r = A.prank[x];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) A.ps[nb][(size_t)kk * pc + r] = A.plog[(size_t)kk * pc + x];
        }
      } else if (pd.state == 3) {  // tile minima; ranks cleared for the next rebuild
        const unsigned nt = (k + 31) / 32;
        const size_t tcap = pc / 32 + 1;
        for (unsigned t = T.tid(); t < nt; t += T.nthreads()) {
          uint32_t mn[D];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) mn[kk] = kInf;
          for (unsigned e = t * 32; e < min(k, t * 32 + 32); ++e)
#pragma unroll
            for (int kk = 0; kk < D; ++kk) mn[kk] = min(mn[kk], A.ps[nb][(size_t)kk * pc + e]);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) A.pst[nb][(size_t)kk * tcap + t] = mn[kk];
        }
        for (unsigned x = T.tid(); x < k; x += T.nthreads()) A.prank[x] = 0;
      }
    }
  }

  // The P index as step i+1 will see it (leader block, all threads): a
  // rebuild advances rank -> scatter -> tiles -> published; with none in
  // progress, one starts once the log has outgrown the index by 32 + its
  // count >> ps_grow (each F-against-P test also scans the unindexed tail).
  __device__ void index_transition(unsigned i) {
    PIdx nd = S.pd;
    bool plan = false;
    if (nd.state == 1) {
      nd.state = 2;
    } else if (nd.state == 2) {
      nd.state = 3;
    } else if (nd.state == 3) {
      nd.cur = nd.nb;
      nd.count = nd.k;
      nd.mark = nd.k;
      nd.ntiles = (nd.k + 31) / 32;
      nd.state = 0;
    } else if (D >= 2) {
      plan = psnap - nd.mark > 32u + (nd.count >> P.ps_grow) && psnap <= kPSMax;
    }
    if (plan) {
      constexpr int MD = D - 1 < 3 ? D - 1 : 3;
      if (threadIdx.x == 0) S.pmax[0] = S.pmax[1] = S.pmax[2] = 0;
      __syncthreads();
      unsigned mx[3] = {0, 0, 0};
      for (unsigned x = threadIdx.x; x < psnap; x += blockDim.x)
#pragma unroll
        for (int j = 0; j < MD; ++j)
          mx[j] = max(mx[j], A.plog[(size_t)(j + 1) * A.plog_cap + x] - hk(j + 1, P.start));
#pragma unroll
      for (int j = 0; j < MD; ++j) atomicMax(&S.pmax[j], mx[j]);
      __syncthreads();
      int bl[3] = {0, 0, 0}, mn = 32;
#pragma unroll
      for (int j = 0; j < MD; ++j) {
        bl[j] = 32 - __clz(S.pmax[j]);
        mn = min(mn, bl[j]);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) nd.shift[j] = j < MD ? (unsigned)(bl[j] - mn) : 0u;
      nd.state = 1;
      nd.nb = nd.cur ^ 1u;
      nd.k = psnap;
    }
    if (threadIdx.x == 0) C->pidx[(i + 1) & 1u] = nd;
  }

  // ---------------- one step ----------------
  // Returns false (on every block alike) when the search is over: OPEN_i
  // holds no entry and window i produced no candidate.
  template <class Team>
  __device__ bool step(const Team& T, unsigned i, unsigned long long* tlap) {
    const unsigned r0 = i % 3, r1 = (i + 1) % 3, r2 = (i + 2) % 3;
    const unsigned cur = i & 1u;
    CycleCtl& K0 = C->cyc[r0];
    CycleCtl& K1 = C->cyc[r1];
    CycleCtl& K2 = C->cyc[r2];
    const bool fifo = (P.flags & OPMOS_FLAG_FIFO) != 0;
    const unsigned head = ld_volatile(&K0.head);
    const unsigned n_in = min(ld_volatile(&K0.open_count.v) - head, A.open_cap);  // FIFO: ring tail - head
    const unsigned nt = ld_volatile(&K0.touched_count.v);
    const unsigned nh = ld_volatile(&K0.heavy_count.v);
    if (n_in == 0 && nt == 0 && nh == 0) return false;
    cyc = i;
    fifo_head = head;
    const unsigned fwin = min(n_in, P.window);  // FIFO: ring positions window i+1 takes
    psnap = ld_volatile(&K0.plen.v);
    lbase = ld_volatile(&K0.lbase.v);
    const BinLimits bl = C->bins[r0];
    const BinParams bp{bl.b0, bl.b1, bl.s1, bl.delta, bl.s2};  // bins OPEN_i's histogram was built on
    bpn = next_bins(K0);
    if (threadIdx.x == 0) {
      for (int j = 0; j < 5; ++j) S.tmax[j] = 0;
      const volatile PIdx* src = &C->pidx[cur];
      S.pd.cur = src->cur;
      S.pd.count = src->count;
      S.pd.mark = src->mark;
      S.pd.ntiles = src->ntiles;
      S.pd.state = src->state;
      S.pd.nb = src->nb;
      S.pd.k = src->k;
      for (int j = 0; j < 3; ++j) S.pd.shift[j] = src->shift[j];
    }
    select_window(A.hist + r0 * kNB, n_in <= P.window);  // has block barriers: S.pd is visible after it
    for (unsigned x = T.tid(); x < kNB; x += T.nthreads()) A.hist[r2 * kNB + x] = 0;
    if (T.leader_block()) {
      if (threadIdx.x == 0) {
        // the longest tasks of step i-1 (its slot is K2)
        st[S_MAXH] += K2.tmax[0];
        st[S_MAXL] += K2.tmax[1];
        st[S_MAXX] += K2.tmax[2];
        st[S_MAXNC] += K2.tmax[3];
        st[S_MAXF] += K2.tmax[4];
        clear_cycle(K2);
        // values step i+1 starts from; the writers of this step raise them
        atomicMax(&K1.plen.v, psnap);
        atomicMax(&K1.lbase.v, lbase);
        K1.win_min_prev = ld_volatile(&K0.win_min.v);
        C->bins[r1] = BinLimits{bpn.b0, bpn.b1, bpn.s1, bpn.delta, bpn.s2};
        if (fifo) {
          K1.head = head + fwin;
          atomicMax(&K1.open_count.v, head + n_in);
        }
      }
      index_transition(i);
    }
    __syncthreads();
    if (T.leader() && tlap) {
      const unsigned long long t = globaltimer();
      st[S_TSEL] += t - *tlap;
      *tlap = t;
    }
    // block merges first (the longest single tasks): the parts of split
    // merges (recorded in xpart while the candidates arrived), then one item
    // per heavy node, skipped when the node's merge is split
    const unsigned np = ld_volatile(&K0.part_count.v);
    for (const unsigned nhi = np + nh; nhi;) {
      if (threadIdx.x == 0) S.claim = atomicAdd(&K0.heavy_next.v, 1u);
      __syncthreads();
      const unsigned t = S.claim;
      __syncthreads();
      if (t >= nhi) break;
      const unsigned x = t < np ? A.cs[cur].xpart[t] : (t - np) << 4;
      const unsigned h = x >> 4, r = x & 15u;
      const unsigned k = A.cs[cur].hsplit[h];
      if (t >= np && k > 1u) continue;
      const uint32_t v = A.cs[cur].touched[2u * A.cand_cap - 1u - h];
      if (threadIdx.x == 0 && r == 0) {  // read before the merge clears them
        S.tmax[3] = max(S.tmax[3], A.cs[cur].ncand[v]);
        S.tmax[4] = max(S.tmax[4], A.fcount[v]);
      }
      const unsigned long long t0 = globaltimer();
      if constexpr (Team::kSplitMerges) {
        if (k > 1u)
          merge_part(v, r, k, K1);
        else
          merge_heavy(v, K1);
      } else {
        merge_heavy(v, K1);
      }
      if (threadIdx.x == 0) {
        const unsigned long long dt = globaltimer() - t0;
        S.tmax[0] = max(S.tmax[0], (unsigned)min(dt, 0xFFFFFFFFull));
        st[S_NHEAVY] += r == 0;
        st[S_SUMH] += dt;
      }
    }
    // warp items: index-rank items, light merges, extraction chunks
    const PIdx& pd = S.pd;
    const unsigned nrank = (D >= 2 && pd.state == 1) ? ((pd.k + 31) / 32) * ((pd.k + kRankQ - 1) / kRankQ) : 0u;
    const unsigned nchunks = ((fifo ? fwin : n_in) + kChunk - 1) / kChunk;
    const unsigned nitems = nrank + nt + nchunks;
    const unsigned lane = lane_id();
    for (;;) {
      unsigned t = 0;
      if (lane == 0) t = atomicAdd(&K0.work_next.v, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= nitems) break;
      const unsigned long long t0 = globaltimer();
      if (t < nrank) {
        rank_item(t);
      } else if (t < nrank + nt) {
        const uint32_t v = A.cs[cur].touched[t - nrank];
        uint32_t* hf = A.cs[cur].hflag + v;
        if (*hf) {
          if (lane == 0) *hf = 0;  // merged by a block this step
        } else {
          merge_node(v, K1);
        }
        if (lane == 0) {
          const unsigned long long dt = globaltimer() - t0;
          atomicMax(&S.tmax[1], (unsigned)min(dt, 0xFFFFFFFFull));
          st[S_SUML] += dt;
        }
      } else {
        const unsigned c = t - nrank - nt;
        if (fifo)
          extract_fifo(head + c * kChunk, head + min(fwin, (c + 1) * kChunk), K1);
        else
          extract_chunk(c, n_in, bp, K1);
        if (lane == 0) {
          const unsigned long long dt = globaltimer() - t0;
          atomicMax(&S.tmax[2], (unsigned)min(dt, 0xFFFFFFFFull));
          st[S_SUMX] += dt;
        }
      }
    }
    index_strided_work(T);
    __syncthreads();
    if (threadIdx.x < 5) atomicMax(&K0.tmax[threadIdx.x], S.tmax[threadIdx.x]);
    for (unsigned x = threadIdx.x; x < kNB; x += blockDim.x)
      if (S.hist[x]) atomicAdd(&A.hist[r1 * kNB + x], S.hist[x]);
    if (T.leader() && tlap) {
      const unsigned long long t = globaltimer();
      st[S_TWORK] += t - *tlap;
      *tlap = t;
    }
    return true;
  }

  // ---------------- output: P without dominated members, sorted, with paths ----------------
  // Four parts separated by team barriers (single query) or by iterations of
  // the multi-query kernel: filter | rank | scan | paths. Regions of the
  // output pool: res_off holds k'*D costs then k'+1 path offsets; res_path
  // holds the path nodes then their arcs.

  // (1) Prune(P, l) deferred from the search: drop members another member
  // dominates; C->res_count must be 0 beforehand.
  template <class Team>
  __device__ void out_filter(const Team& T) {
    const uint32_t t = G.n;  // P
    const unsigned k = A.fcount[t];
    const uint64_t fb = A.fbase[t];
    const unsigned cap = A.fcap[t];
    unsigned kept = 0;
    for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
      uint32_t ci[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) ci[kk] = A.fpool[fb + (size_t)kk * cap + i];
      bool dom = false;
      for (unsigned j = 0; j < k && !dom; ++j) {
        uint32_t cj[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) cj[kk] = A.fpool[fb + (size_t)kk * cap + j];
        dom = dominates<D>(cj, ci);
      }
      if (dom) {
        A.ldead[A.fpool[fb + (size_t)D * cap + i]] = 0;
        st[S_PRUNED]++;
      } else {
        ++kept;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane_id() == 0 && kept) atomicAdd(&C->res_count, kept);
  }

  // (2a) region 1 allocation, one thread.
  __device__ void out_alloc1() {
    const unsigned kk_live = ld_volatile(&C->res_count);
    const unsigned long long words = (unsigned long long)kk_live * D + kk_live + 1;
    const unsigned long long off = atomicAdd(O.used, words);
    if (off + words > O.cap) set_error(C, OPMOS_ERR_CAPACITY);
    C->res_off = off;
  }

  // (2b) lexicographic rank of every kept member; costs and path lengths.
  template <class Team>
  __device__ void out_rank(const Team& T) {
    const uint32_t t = G.n;  // P
    const unsigned k = A.fcount[t];
    const uint64_t fb = A.fbase[t];
    const unsigned cap = A.fcap[t];
    const bool paths = !(P.flags & OPMOS_FLAG_NO_PATHS);
    const unsigned kk_live = ld_volatile(&C->res_count);
    const unsigned long long off = C->res_off;
    for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
      const uint32_t idi = A.fpool[fb + (size_t)D * cap + i];
      if (A.ldead[idi] != kAlive) continue;
      uint32_t ci[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) ci[kk] = A.fpool[fb + (size_t)kk * cap + i];
      unsigned rank = 0;
      for (unsigned j = 0; j < k; ++j) {
        uint32_t cj[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) cj[kk] = A.fpool[fb + (size_t)kk * cap + j];
        if ((lex_less<D>(cj, ci) || (j < i && equal<D>(cj, ci))) &&
            A.ldead[A.fpool[fb + (size_t)D * cap + j]] == kAlive)
          ++rank;
      }
      if (rank >= kk_live || off + (unsigned long long)kk_live * D + kk_live + 1 > O.cap) {
        set_error(C, OPMOS_ERR_CAPACITY);  // never write outside the allocated region
        continue;
      }
#pragma unroll
      for (int kk = 0; kk < D; ++kk) O.words[off + (size_t)rank * D + kk] = ci[kk];
      unsigned len = 0;
      if (paths)
        for (uint32_t x = idi; x != kInf; x = A.lparent[x]) ++len;
      O.words[off + (size_t)kk_live * D + rank] = len;
      A.lpver[idi] = rank;  // remembered for the path pass
    }
  }

  // (3) exclusive scan of the path lengths and region 2 allocation; one block.
  __device__ void out_scan() {
    const bool paths = !(P.flags & OPMOS_FLAG_NO_PATHS);
    const unsigned kk_live = ld_volatile(&C->res_count);
    const unsigned long long off = C->res_off;
    uint32_t* lens = O.words + off + (size_t)kk_live * D;
    unsigned carry = 0;
    for (unsigned b0 = 0; b0 < kk_live + 1; b0 += blockDim.x) {
      const unsigned i = b0 + threadIdx.x;
      const unsigned x = i < kk_live ? lens[i] : 0;
      unsigned total;
      const unsigned ex = block_exclusive_scan(x, S.warp, total);
      if (i <= kk_live) lens[i] = carry + ex;
      carry += total;
    }
    if (threadIdx.x == 0) {
      const unsigned long long total = carry;
      const unsigned long long words = paths ? 2 * total - kk_live : 0;
      unsigned long long p0 = 0;
      if (words) {
        p0 = atomicAdd(O.used, words);
        if (p0 + words > O.cap) set_error(C, OPMOS_ERR_CAPACITY);
      }
      C->res_path = p0;
      C->res_total = total;
    }
  }

  // (4) parent-chain walks: nodes start..goal and the arcs between them.
  template <class Team>
  __device__ void out_paths(const Team& T) {
    if (P.flags & OPMOS_FLAG_NO_PATHS) return;
    const uint32_t t = G.n;  // P
    const unsigned k = A.fcount[t];
    const uint64_t fb = A.fbase[t];
    const unsigned cap = A.fcap[t];
    const unsigned kk_live = ld_volatile(&C->res_count);
    const unsigned long long off = C->res_off, p0 = C->res_path, total = C->res_total;
    const uint32_t* offs = O.words + off + (size_t)kk_live * D;
    if (p0 + 2 * total > O.cap + kk_live) return;  // region 2 was not granted
    for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
      const uint32_t idi = A.fpool[fb + (size_t)D * cap + i];
      if (A.ldead[idi] != kAlive) continue;
      const unsigned rank = A.lpver[idi];
      if (rank >= kk_live) continue;
      const unsigned a = offs[rank], b = offs[rank + 1];
      // nodes at p0 + [a, b); arcs at p0 + total + [a - rank, b - rank - 1)
      unsigned pos = b;
      for (uint32_t x = idi; x != kInf && pos > a; x = A.lparent[x]) {
        --pos;
        O.words[p0 + pos] = A.lnode[x];
        if (A.lparent[x] != kInf) O.words[p0 + total + pos - rank - 1] = A.ledge[x];
      }
    }
  }

  template <class Team>
  __device__ bool output(const Team& T) {
    out_filter(T);
    if (!T.sync(C)) return false;
    if (T.leader()) out_alloc1();
    if (!T.sync(C)) return false;
    out_rank(T);
    if (!T.sync(C)) return false;
    if (T.leader_block()) out_scan();
    if (!T.sync(C)) return false;
    out_paths(T);
    return true;
  }
};

// ---------------------------------------------------------------------------
// Single query on the whole cooperative grid
// ---------------------------------------------------------------------------
template <int D>
__device__ void run_grid(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P, const OutPool& O,
                         QResult* R) {
  __shared__ Shared S;
  const GridTeam T;
  Search<D> X(G, A, C, P, O, S);
  X.init_zero(T);
  bool ok = T.sync(C);
  X.init_seed(T, false);
  ok = ok && T.sync(C);
  unsigned step = 0;
  unsigned long long tph = globaltimer();
  while (ok) {
    if (T.leader() && globaltimer() - C->t_start > P.time_limit_ns) set_error(C, OPMOS_ERR_TIMEOUT);
    if (!X.step(T, step, &tph)) break;
    ok = T.sync(C);
    if (T.leader()) {
      const unsigned long long t = globaltimer();
      X.st[S_TSYNC] += t - tph;
      tph = t;
    }
    ++step;
  }
  if (ok) {
    if (T.leader()) C->res_count = 0;
    ok = T.sync(C) && X.output(T);
    if (T.leader()) X.st[S_TOUT] += globaltimer() - tph;
  }
  X.st[S_STEPS] = T.leader() ? step : 0;
  X.st[S_GOALINS] = T.leader() ? ld_volatile(&C->plog_len.v) : 0;
  flush_stats(C, X.st);
  T.sync(C);
  if (T.leader()) {
    __threadfence();
    R->status = *reinterpret_cast<volatile unsigned*>(&C->error);
    R->count = C->res_count;
    R->off = C->res_off;
    R->path = C->res_path;
    R->total = C->res_total;
    R->labels = C->n_labels.v;
    R->f_words = C->f_words.v;
    for (int i = 0; i < kNStat; ++i) R->stats[i] = C->stats[i];
  }
}

template <int D, unsigned NT, unsigned NB>
__global__ void __launch_bounds__(NT, NB) search_grid_kernel(GraphDev G, QArena A, QCtl* C, QParams P, OutPool O,
                                                             QResult* R) {
  run_grid<D>(G, A, C, P, O, R);
}

// ---------------------------------------------------------------------------
// Multi-query persistent kernel (batch and serving): continuous batching of
// many independent queries, each a slot. Every iteration:
//   P0  block 0 retires finished slots and admits queued queries into free
//       slots (FREE -> INIT -> RUN -> OUT -> FREE), and advances every
//       running slot by one step;
//   P1  INIT slots are initialised, OUT slots write one part of their
//       result, RUN slots run one search step (merge of window i beside the
//       extraction of window i+1).
// In P1 each block derives the same assignment of "virtual blocks" to slots
// (a running slot gets a share of the grid in proportion to its work, at
// least one block), so large and small queries advance side by side.
// ---------------------------------------------------------------------------
struct SubTeam {
  static constexpr bool kSplitMerges = false;  // a query's arena has kparts = 1
  unsigned j, nb;
  __device__ __forceinline__ unsigned tid() const { return j * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ unsigned nthreads() const { return nb * blockDim.x; }
  __device__ __forceinline__ unsigned wid() const { return tid() >> 5; }
  __device__ __forceinline__ unsigned nwarps() const { return nthreads() >> 5; }
  __device__ __forceinline__ bool leader_block() const { return j == 0; }
  __device__ __forceinline__ bool leader() const { return j == 0 && threadIdx.x == 0; }
};

__device__ inline bool mq_barrier(MCtl* M) {
  __shared__ unsigned s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_volatile(&M->bar_gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&M->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&M->bar_count, 0u);
      __threadfence();
      atomicAdd(&M->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_volatile(&M->bar_gen) == gen) {
        if (++spins > 64) __nanosleep(64);
        if ((spins & 255u) == 0) {
          if (ld_volatile(&M->error) != 0) break;
          if (globaltimer() - t0 > kBarrierTimeoutNs) {
            atomicCAS(&M->error, 0u, (unsigned)OPMOS_ERR_TIMEOUT);
            break;
          }
        }
      }
    }
    __threadfence();
    s_ok = ld_volatile(&M->error) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ inline void mq_write_result(const MSlot& sl, unsigned slot, QCtl* C, QResult* results,
                                       unsigned* done_flags, unsigned qcap) {
  const unsigned ri = sl.qidx % qcap;
  QResult* R = &results[ri];
  R->status = ld_volatile(&C->error);
  R->slot = slot;
  R->count = C->res_count;
  R->off = C->res_off;
  R->path = C->res_path;
  R->total = C->res_total;
  R->labels = C->n_labels.v;
  R->f_words = C->f_words.v;
  C->stats[S_STEPS] = C->step;
  C->stats[S_GOALINS] = C->plog_len.v;
  for (int i = 0; i < kNStat; ++i) R->stats[i] = C->stats[i];
  if (done_flags) {
    __threadfence_system();  // the record is visible before its completion flag
    *reinterpret_cast<volatile unsigned*>(&done_flags[ri]) = 1u;
    __threadfence_system();
  }
}

template <int D>
__device__ void mq_alloc_region1(const MSlot& sl, QCtl* C) {
  const OutPool& O = sl.O;
  const unsigned kk_live = ld_volatile(&C->res_count);
  const unsigned long long words = (unsigned long long)kk_live * D + kk_live + 1;
  const unsigned long long off = atomicAdd(O.used, words);
  if (off + words > O.cap) atomicCAS(&C->error, 0u, (unsigned)OPMOS_ERR_CAPACITY);
  C->res_off = off;
}

__device__ __forceinline__ bool step_empty(const QCtl* C, unsigned i) {
  const CycleCtl& K = C->cyc[i % 3];
  return ld_volatile(&K.open_count.v) == ld_volatile(&K.head) && ld_volatile(&K.touched_count.v) == 0 &&
         ld_volatile(&K.heavy_count.v) == 0;
}

// P0: slot transitions and admission (block 0).
template <int D>
__device__ void mq_schedule(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                            const GraphDev* graphs, MCtl* M, QResult* results, unsigned* done_flags) {
  __shared__ unsigned s_busy;
  if (threadIdx.x == 0) s_busy = 0;
  __syncthreads();
  const unsigned q_count = ld_volatile(&hctl[HC_TAIL]);
  const unsigned qcap = M->qcap;
  const unsigned after_out = M->hold ? SL_HELD : SL_FREE;
  for (unsigned q = threadIdx.x; q < nslots; q += blockDim.x) {
    MSlot& sl = slots[q];
    QCtl* C = &ctls[q];
    unsigned st = sl.state;
    if (st == SL_RUN) {
      const unsigned step = C->step + 1;
      C->step = step;
      if (ld_volatile(&C->error) || step_empty(C, step))
        st = SL_OUT1;
      else if (globaltimer() - C->t_start > sl.P.time_limit_ns) {
        atomicCAS(&C->error, 0u, (unsigned)OPMOS_ERR_TIMEOUT);
        st = SL_OUT1;
      }
      if (st == SL_OUT1) C->res_count = 0;
    } else if (st == SL_INIT) {
      st = (ld_volatile(&C->error) || step_empty(C, 0)) ? SL_OUT1 : SL_RUN;
      if (st == SL_OUT1) C->res_count = 0;
    } else if (st == SL_OUT1 || st == SL_OUT2 || st == SL_OUT3 || st == SL_OUT4) {
      // one output part per iteration; an error ends the output early
      if (ld_volatile(&C->error) || st == SL_OUT4) {
        mq_write_result(sl, q, C, results, done_flags, qcap);
        st = after_out;
      } else if (st == SL_OUT1) {
        mq_alloc_region1<D>(sl, C);
        if (ld_volatile(&C->error)) {  // no room for the result: report, never write
          mq_write_result(sl, q, C, results, done_flags, qcap);
          st = after_out;
        } else {
          st = SL_OUT2;
        }
      } else {
        st = st + 1;
      }
    } else if (st == SL_HELD && ld_volatile(&hctl[HC_RELEASE + q])) {
      hctl[HC_RELEASE + q] = 0;  // the host has collected the result
      st = SL_FREE;
    }
    if (st == SL_FREE) {
      unsigned qn = ld_volatile(&M->q_next);
      while (qn < q_count) {
        const unsigned got = atomicCAS(&M->q_next, qn, qn + 1);
        if (got == qn) break;
        qn = got;
      }
      if (qn < q_count) {
        MQuery Q;
        {
          const volatile MQuery* src = &queue[qn % qcap];
          Q.graph = src->graph;
          Q.start = src->start;
          Q.goal = src->goal;
          Q.d = src->d;
          Q.h = src->h;
        }
        sl.P.start = Q.start;
        sl.P.goal = Q.goal;
        sl.P.h = Q.h;
        sl.P.qd = Q.d;
        sl.G = graphs[Q.graph];
        sl.d = Q.d;
        sl.qidx = qn;
        if (M->hold) *sl.O.used = 0;  // serving: the slot's own pool starts empty (batch pools are shared)
        st = SL_INIT;
      }
    }
    sl.state = st;
    if (st != SL_FREE) atomicAdd(&s_busy, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    M->iter++;
    const unsigned closing = ld_volatile(&hctl[HC_CLOSING]);
    if (closing >= 2 || (closing && s_busy == 0 && ld_volatile(&M->q_next) >= ld_volatile(&hctl[HC_TAIL])))
      M->done = 1;  // 1: drain then stop; 2: stop now
  }
}

template <int D>
__device__ void mq_work(MSlot* slots, QCtl* ctls, unsigned q, unsigned j, unsigned nb, Shared& S) {
  const QArena A = slots[q].A;
  const QParams P = slots[q].P;
  const GraphDev G = slots[q].G;
  const OutPool O = slots[q].O;
  const unsigned st = slots[q].state;
  QCtl* C = &ctls[q];
  Search<D> X(G, A, C, P, O, S);
  if (st == SL_INIT) {
    const BlockTeam T;
    X.init_zero(T);
    if (threadIdx.x == 0) C->error = 0;
    __syncthreads();
    X.init_seed(T, true);
    __syncthreads();
  } else if (st == SL_OUT1) {
    X.out_filter(SubTeam{j, nb});
  } else if (st == SL_OUT2) {
    X.out_rank(SubTeam{j, nb});
  } else if (st == SL_OUT3) {
    X.out_scan();
  } else if (st == SL_OUT4) {
    X.out_paths(SubTeam{j, nb});
  } else if (st == SL_RUN) {
    X.step(SubTeam{j, nb}, C->step, nullptr);
  }
  flush_stats(C, X.st);
}

__device__ __forceinline__ unsigned A_fcount_goal(const MSlot& sl) { return sl.A.fcount[sl.G.n]; }

// Work units of a slot (0: none). INIT and the scan part of the output get
// one block; the other output parts a share like search steps.
__device__ __forceinline__ unsigned mq_weight(const MSlot& sl, QCtl* C, bool& single) {
  single = false;
  const unsigned st = sl.state;
  if (st == SL_FREE || st == SL_HELD) return 0;
  if (st == SL_INIT || st == SL_OUT3) {
    single = true;
    return 1u;
  }
  if (st >= SL_OUT1) return max(1u, ld_volatile(&C->res_count) + A_fcount_goal(sl));
  const CycleCtl& K = C->cyc[C->step % 3];
  const unsigned w = (ld_volatile(&K.open_count.v) - ld_volatile(&K.head)) + ld_volatile(&K.touched_count.v) +
                     8u * ld_volatile(&K.heavy_count.v);
  return w ? w : 1u;  // a running slot always gets a block
}

template <int D>
__device__ void mq_phase(MSlot* slots, QCtl* ctls, unsigned nslots, Shared& S, unsigned* s_pref) {
  // total weight of the multi-block slots
  __shared__ unsigned long long s_wtot;
  if (threadIdx.x == 0) s_wtot = 0;
  __syncthreads();
  unsigned long long wloc = 0;
  for (unsigned q = threadIdx.x; q < nslots; q += blockDim.x) {
    bool single;
    const unsigned w = mq_weight(slots[q], &ctls[q], single);
    if (!single) wloc += w;
  }
  atomicAdd(&s_wtot, wloc);
  __syncthreads();
  const unsigned long long wtot = s_wtot > 0 ? s_wtot : 1;
  const unsigned B = gridDim.x;
  // virtual blocks per slot, then their prefix sums (chunked block scan)
  unsigned carry = 0;
  for (unsigned c0 = 0; c0 < nslots; c0 += blockDim.x) {
    const unsigned q = c0 + threadIdx.x;
    unsigned nbq = 0;
    if (q < nslots) {
      bool single;
      const unsigned w = mq_weight(slots[q], &ctls[q], single);
      if (single)
        nbq = 1;
      else if (w)
        nbq = (unsigned)min((unsigned long long)B, max(1ull, (w * (unsigned long long)B + wtot - 1) / wtot));
    }
    unsigned total;
    const unsigned ex = block_exclusive_scan(nbq, S.warp, total);
    if (q < nslots) s_pref[q] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) s_pref[nslots] = carry;
  __syncthreads();
  const unsigned VB = s_pref[nslots];
  for (unsigned v = blockIdx.x; v < VB; v += B) {
    unsigned lo = 0, hi = nslots;  // last q with s_pref[q] <= v
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) / 2;
      if (s_pref[mid] <= v) lo = mid; else hi = mid;
    }
    const unsigned q = lo;
    const unsigned j = v - s_pref[q], nb = s_pref[q + 1] - s_pref[q];
    mq_work<D>(slots, ctls, q, j, nb, S);
    __syncthreads();
  }
}

template <int D>
__global__ void __launch_bounds__(kMultiThreads, 2)
    multi_kernel(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                 const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M) {
  __shared__ Shared S;
  __shared__ unsigned s_pref[kMaxSlots + 1];
  for (;;) {
    if (blockIdx.x == 0) mq_schedule<D>(slots, ctls, nslots, queue, hctl, graphs, M, results, done_flags);
    if (!mq_barrier(M)) return;
    if (ld_volatile(&M->done)) return;
    mq_phase<D>(slots, ctls, nslots, S, s_pref);
    if (!mq_barrier(M)) return;
  }
}

}  // namespace detail

// ---------------------------------------------------------------------------
// host launchers, explicitly instantiated per objective count
// ---------------------------------------------------------------------------
template <int D>
cudaError_t launch_grid(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P, const OutPool& O,
                        QResult* R, bool wide, unsigned blocks, cudaStream_t s) {
  void* args[] = {(void*)&G, (void*)&A, (void*)&C, (void*)&P, (void*)&O, (void*)&R};
  if (wide)
    return cudaLaunchCooperativeKernel(
        (void*)detail::search_grid_kernel<D, kGridWideThreads, kGridWideBlocksPerSM>, dim3(blocks),
        dim3(kGridWideThreads), args, 0, s);
  return cudaLaunchCooperativeKernel((void*)detail::search_grid_kernel<D, kGridThreads, 1>, dim3(blocks),
                                     dim3(kGridThreads), args, 0, s);
}

template <int D>
int grid_occupancy(bool wide) {
  int nb = 0;
  if (wide)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, detail::search_grid_kernel<D, kGridWideThreads, kGridWideBlocksPerSM>, kGridWideThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, detail::search_grid_kernel<D, kGridThreads, 1>,
                                                  kGridThreads, 0);
  return nb;
}

template <int D>
cudaError_t launch_multi_d(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                           const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M, unsigned blocks,
                           cudaStream_t s) {
  void* args[] = {(void*)&slots, (void*)&ctls, (void*)&nslots, (void*)&queue, (void*)&hctl,
                  (void*)&graphs, (void*)&results, (void*)&done_flags, (void*)&M};
  return cudaLaunchCooperativeKernel((void*)detail::multi_kernel<D>, dim3(blocks), dim3(kMultiThreads), args, 0, s);
}

template <int D>
int multi_occupancy_d() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, detail::multi_kernel<D>, kMultiThreads, 0);
  return nb;
}

}  // namespace opmos
