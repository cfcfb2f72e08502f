// Ordered-parallel multi-objective label-setting search (Sec. 5, Algorithm 2)
// on one GPU. One "team" of threads works on one query: the whole cooperative
// grid for a single query, or one thread block per query in batch mode. A step
// of the search is four phases separated by team barriers:
//
//   1. histogram   the open entries by lexicographic bucket of (F[0], F[1])
//                  (Algorithm 2: OPEN is a lexicographic priority queue):
//                  one bucket per F[0] value, the lowest one split by F[1]
//   2. extract     the window = every live entry in the lowest buckets whose
//                  cumulative count stays within W (the NUM_POP of Sec. 5);
//                  entries whose label was pruned are dropped here (lazy OPEN
//                  delete, Sec. 5.1 and Algorithm 2) and so are labels whose F is
//                  weakly dominated by a solution (PruneOPEN of Algorithm 1,
//                  applied lazily at extraction)
//   3. expand      every window label along its out-arcs, L lanes per label:
//                  g' = g + c(e), dropped if h(v') is infinite (Algorithm 1)
//   4. merge       one warp per target node: the node's candidates of this step
//                  are resolved against each other (in-batch dominance and
//                  duplicates), then against the node's frontier alpha(v')
//                  (Algorithm 1: weakly dominated candidates are dropped,
//                  strictly dominated frontier labels are pruned), then against
//                  P on F (Algorithm 1); survivors become labels, join alpha(v')
//                  and OPEN. Goal labels are ordinary labels until they are
//                  extracted (Algorithm 1); an extracted goal label is sent
//                  to a virtual node n that stands for P, whose merge applies
//                  the goal branch of Algorithm 1 and appends survivors to the P log.
//
// The F-against-P test of phase 4 uses an index of P rebuilt every time P has
// grown by 32 + 1/64 of its indexed count: P sorted along a Z-order curve over
// objectives 1..3 in tiles of 32, each with its componentwise minimum; a
// candidate only scans the tiles whose minimum weakly dominates it, plus the
// goal costs found since the last rebuild (the rebuild is split over phases
// 1-3 of a step).
//
// A node is only ever touched by one warp per step, so frontier updates need
// no locks. All waits are bounded (see GridTeam::sync).
#include "opmos_dev.cuh"
#include "search.cuh"

namespace opmos {

namespace {

__device__ __forceinline__ unsigned warp_min(unsigned x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

template <class Team>
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
__device__ unsigned block_exclusive_scan(unsigned x, unsigned* s_warp, unsigned& total) {
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

struct Shared {
  unsigned hist[kNB];
  unsigned warp[33];
  unsigned f_min, b1_max;
  unsigned span;
  unsigned pmax[3];
  // one batch of a heavy node's candidates, merged by the whole block
  uint32_t mc[OPMOS_MAX_D][32];
  int mmine[32];
  int m_next;
  unsigned m_nb, m_alive, m_kill, m_claim;
};

// Histogram bucket of an OPEN key (F0 << 32 | F1): buckets [0, kNB1) split the
// lowest F0 bucket by F1 >> s1, buckets [kNB1, kNB-1) are whole F0 buckets of
// width delta, kNB-1 collects everything beyond. Monotone in lexicographic
// (F0, F1) order, so every prefix of buckets is a lexicographic prefix of OPEN.
struct BinParams {
  uint32_t b0, b1, s1, delta;
};
__device__ __forceinline__ unsigned bin_of(uint64_t key, const BinParams& bp) {
  const uint32_t F0 = (uint32_t)(key >> 32), F1 = (uint32_t)key;
  const uint32_t q = F0 > bp.b0 ? (F0 - bp.b0) / bp.delta : 0u;
  if (q == 0) {
    const uint32_t x = F1 > bp.b1 ? (F1 - bp.b1) >> bp.s1 : 0u;
    return min(x, (unsigned)kNB1 - 1);
  }
  return kNB1 + min(q - 1, (unsigned)(kNB - kNB1 - 1));
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
  const GraphDev& G;
  const QArena& A;
  QCtl* C;
  const QParams& P;
  const OutPool& O;
  Shared& S;
  unsigned long long st[kNStat];

  __device__ Search(const GraphDev& g, const QArena& a, QCtl* c, const QParams& p, const OutPool& o,
                    Shared& s)
      : G(g), A(a), C(c), P(p), O(o), S(s) {
#pragma unroll
    for (int i = 0; i < kNStat; ++i) st[i] = 0;
  }

  __device__ __forceinline__ uint32_t hk(int k, uint32_t v) const {
    return __ldg(P.h + (size_t)k * G.n + v);
  }

  // ---------------- initialisation (Algorithm 1) ----------------
  // Empty frontiers and histograms (the empty sets Algorithm 1 starts from). The team must pass a
  // barrier before init_seed writes the start node's frontier.
  template <class Team>
  __device__ void init_zero(const Team& T) {
    for (unsigned v = T.tid(); v <= G.n; v += T.nthreads()) {  // n real nodes + P
      A.fcount[v] = 0;
      A.fcap[v] = 0;
      A.fbase[v] = 0;
      A.node_head[v] = kNil;
      A.ncand[v] = 0;
    }
    for (unsigned i = T.tid(); i < 2u * kNB; i += T.nthreads()) A.hist[i] = 0;
  }

  // l_s = (v_s, 0) into OPEN and G_OP(v_s) (Algorithm 1), control block reset.
  template <class Team>
  __device__ void init_seed(const Team& T, bool reset_ctl) {
    if (T.leader()) {
      if (reset_ctl) {
        C->error = 0;
        C->done = 0;
        C->step = 0;
        C->win_count.v = C->cand_count.v = C->touched_count.v = 0;
        C->heavy_count.v = C->heavy_next.v = 0;
        C->theta = 0;
        C->plog_snap = 0;
        C->res_count = C->res_status = 0;
        C->res_off = C->res_path = C->res_total = 0;
        for (int i = 0; i < kNStat; ++i) C->stats[i] = 0;
      }
      C->t_start = globaltimer();
      const uint32_t s = P.start, t = P.goal, tile = P.tile;
      // l_s = (v_s, 0): label 0, frontier of v_s, OPEN
#pragma unroll
      for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap] = 0;
      A.lnode[0] = s;
      A.lparent[0] = kInf;
      A.ledge[0] = kInf;
      A.lpver[0] = 0;
      A.lstatus[0] = (s == t) ? ST_CLOSED : ST_OPEN;
      const uint32_t fs = (s == t) ? G.n : s;  // start == goal: l_s is the solution
      A.fbase[fs] = 0;
      A.fcap[fs] = tile;
      A.fcount[fs] = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) A.fpool[(size_t)k * tile] = 0;
      A.fpool[(size_t)D * tile] = 0;
      C->f_words.v = (unsigned long long)(D + 1) * tile;
      C->n_labels.v = 1;
      C->plog_len.v = 0;
      const uint32_t h0 = hk(0, s);
      const uint64_t key = ((uint64_t)h0 << 32) | (D > 1 ? hk(1, s) : 0u);
      // start == goal: P = {l_s}, nothing to search. h(s) = inf: goal unreachable.
      if (s != t && h0 != kInf) {
        A.okey[0][0] = key;
        A.oid[0][0] = 0;
        C->open_count[0].v = 1;
        C->min_key[0].v = key;
      } else {
        C->open_count[0].v = 0;
        C->min_key[0].v = ~0ull;
      }
      if (s == t) {
#pragma unroll
        for (int k = 0; k < D; ++k) A.plog[(size_t)k * A.plog_cap] = 0;
        C->plog_len.v = 1;
      }
      C->open_count[1].v = 0;
      C->min_key[1].v = ~0ull;
      C->f1span[0] = C->f1span[1] = 0;
      C->ps_cur = C->ps_count = C->ps_mark = C->ps_ntiles = 0;
      C->ps_build = C->ps_src = C->ps_mark_new = C->ps_nbuild = C->ps_nb = 0;
      st[S_INSERTED] += 1;
    }
  }

  // ---------------- phase 1: bucket histogram of the live OPEN entries ----------------
  template <class Team>
  __device__ void phase_hist(const Team& T, unsigned cur, unsigned n_in, const BinParams& bp) {
    for (unsigned i = threadIdx.x; i < kNB; i += blockDim.x) S.hist[i] = 0;
    if (threadIdx.x == 0) S.span = 0;
    if (T.leader_block()) publish_p_index();
    __syncthreads();
    const uint64_t* in = A.okey[cur];
    const uint32_t* in_id = A.oid[cur];
    unsigned span = 0;
    for (unsigned i = T.tid(); i < n_in; i += T.nthreads()) {
      if (A.lstatus[in_id[i]] == ST_DEAD) continue;  // pruned while open: not counted
      const uint64_t key = in[i];
      const unsigned b = bin_of(key, bp);
      atomicAdd(&S.hist[b], 1u);
      if (b < (unsigned)kNB1) span = max(span, (uint32_t)key - min((uint32_t)key, bp.b1));
    }
    span = ~warp_min(~span);  // warp maximum
    if (lane_id() == 0 && span) atomicMax(&S.span, span);
    __syncthreads();
    unsigned* gh = A.hist + cur * kNB;
    for (unsigned i = threadIdx.x; i < kNB; i += blockDim.x)
      if (S.hist[i]) atomicAdd(&gh[i], S.hist[i]);
    const unsigned nxt = cur ^ 1u;
    if (threadIdx.x == 0 && S.span) atomicMax(&C->f1span[nxt], S.span);
    if (T.leader()) {
      C->open_count[nxt].v = 0;
      C->min_key[nxt].v = ~0ull;
      C->win_count.v = 0;
      C->cand_count.v = 0;
      C->touched_count.v = 0;
      C->merge_next.v = 0;
      C->heavy_count.v = 0;
      C->heavy_next.v = 0;
    }
    if (T.leader_block()) plan_p_index();
  }

  // A rebuild planned in step s is ranked in phase 2 and tiled in phase 4 of
  // step s; it becomes the live index here, at the start of step s+1.
  __device__ void publish_p_index() {
    if (threadIdx.x == 0 && C->ps_build) {
      C->ps_cur = C->ps_nb;
      C->ps_count = C->ps_src;
      C->ps_ntiles = (C->ps_src + 31) / 32;
      C->ps_mark = C->ps_mark_new;
      C->ps_nbuild++;
      C->ps_build = 0;
    }
  }

  // Decide whether this step rebuilds the P index (the P log grew by 32 +
  // 1/64 of the indexed count since the last build: every candidate scans
  // the unindexed tail, a rebuild costs one O(k^2) rank pass) and fix the per-objective shifts that balance the
  // Z-order. The index covers log[0, mark); the rest is scanned directly.
  __device__ void plan_p_index() {
    __syncthreads();
    if (D < 2) return;
    const unsigned plen = ld_volatile(&C->plog_len.v);
    const bool build = plen - C->ps_mark > 32u + C->ps_count / 64u && plen <= kPSMax;
    if (threadIdx.x == 0) S.pmax[0] = S.pmax[1] = S.pmax[2] = 0;
    __syncthreads();
    if (!build) return;
    constexpr int MD = D - 1 < 3 ? D - 1 : 3;
    unsigned mx[3] = {0, 0, 0};
    for (unsigned i = threadIdx.x; i < plen; i += blockDim.x)
#pragma unroll
      for (int j = 0; j < MD; ++j)
        mx[j] = max(mx[j], A.plog[(size_t)(j + 1) * A.plog_cap + i] - hk(j + 1, P.start));
#pragma unroll
    for (int j = 0; j < MD; ++j) atomicMax(&S.pmax[j], mx[j]);
    __syncthreads();
    if (threadIdx.x == 0) {
      int bl[3] = {0, 0, 0}, mn = 32;
#pragma unroll
      for (int j = 0; j < MD; ++j) {
        bl[j] = 32 - __clz(S.pmax[j]);
        mn = min(mn, bl[j]);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) C->ps_shift[j] = j < MD ? (unsigned)(bl[j] - mn) : 0u;
      C->ps_src = plen;
      C->ps_mark_new = plen;
      C->ps_nb = C->ps_cur ^ 1u;
      C->ps_build = 1;
    }
  }

  // Phase 2 part of a rebuild: rank every logged goal cost in Z-order and
  // scatter it into the idle index buffer.
  template <class Team>
  __device__ void build_p_rank(const Team& T) {
    if constexpr (D >= 2) {
      constexpr int MD = D - 1 < 3 ? D - 1 : 3;
      if (!ld_volatile(&C->ps_build)) return;
      const unsigned k = C->ps_src;
      const unsigned nb = C->ps_nb;
      uint32_t lo[MD], sh[MD];
#pragma unroll
      for (int j = 0; j < MD; ++j) {
        lo[j] = hk(j + 1, P.start);
        sh[j] = C->ps_shift[j];
      }
      const size_t pc = A.plog_cap;
      for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
        uint32_t zi[MD];
#pragma unroll
        for (int j = 0; j < MD; ++j) zi[j] = (A.plog[(size_t)(j + 1) * pc + i] - lo[j]) >> sh[j];
        unsigned rank = 0;
        for (unsigned q = 0; q < k; ++q) {
          uint32_t zq[MD];
#pragma unroll
          for (int j = 0; j < MD; ++j) zq[j] = (A.plog[(size_t)(j + 1) * pc + q] - lo[j]) >> sh[j];
          rank += z_less<MD>(zq, zi) || (q < i && !z_less<MD>(zi, zq));
        }
#pragma unroll
        for (int kk = 0; kk < D; ++kk) A.ps[nb][(size_t)kk * pc + rank] = A.plog[(size_t)kk * pc + i];
      }
    }
  }

  // Phase 4 part of a rebuild: tile minima of the idle buffer.
  template <class Team>
  __device__ void build_p_tiles(const Team& T) {
    if constexpr (D >= 2) {
      if (!ld_volatile(&C->ps_build)) return;
      const unsigned k = C->ps_src;
      const unsigned nb = C->ps_nb;
      const unsigned nt = (k + 31) / 32;
      const size_t tcap = A.plog_cap / 32 + 1;
      for (unsigned t = T.tid(); t < nt; t += T.nthreads()) {
        uint32_t mn[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) mn[kk] = kInf;
        for (unsigned e = t * 32; e < min(k, t * 32 + 32); ++e)
#pragma unroll
          for (int kk = 0; kk < D; ++kk) mn[kk] = min(mn[kk], A.ps[nb][(size_t)kk * A.plog_cap + e]);
#pragma unroll
        for (int kk = 0; kk < D; ++kk) A.pst[nb][(size_t)kk * tcap + t] = mn[kk];
      }
    }
  }

  // Window: buckets [0, b*] where b* is the largest bucket whose cumulative
  // count is <= W, but at least the first non-empty bucket (the overflow bucket
  // is never taken). Every block computes the same b*.
  __device__ unsigned select_bucket(unsigned cur) {
    const unsigned* gh = A.hist + cur * kNB;
    const unsigned per = (kNB + blockDim.x - 1) / blockDim.x;  // blockDim >= 64
    const unsigned b0 = threadIdx.x * per;
    unsigned loc[kNB / 64 > 0 ? kNB / 64 : 1];
    unsigned sum = 0;
    for (unsigned j = 0; j < per; ++j) {
      loc[j] = b0 + j < (unsigned)kNB ? *reinterpret_cast<const volatile unsigned*>(&gh[b0 + j]) : 0u;
      sum += loc[j];
    }
    if (threadIdx.x == 0) {
      S.f_min = kNB;
      S.b1_max = 0;
    }
    unsigned total;
    unsigned run = block_exclusive_scan(sum, S.warp, total);
    unsigned fmin = kNB, b1 = 0;
    bool any_b1 = false;
    for (unsigned j = 0; j < per; ++j) {
      const unsigned b = b0 + j;
      run += loc[j];
      if (b < (unsigned)kNB - 1) {
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
    const unsigned bstar = max(S.b1_max, S.f_min == (unsigned)kNB ? 0u : S.f_min);
    __syncthreads();
    return bstar;
  }

  // n-th (0-based) set bit of m, 32 if there is none.
  __device__ __forceinline__ unsigned nth_bit(unsigned m, unsigned n) {
    for (unsigned i = 0; i < n && m; ++i) m &= m - 1;
    return m ? __ffs(m) - 1 : 32u;
  }

  // Expansion of one window label by the L lanes of a lane group (Algorithm
  // 1): g' = g + c(e) for every out-arc, dropped when h(v') is infinite.
  __device__ void expand_label(uint32_t id, unsigned gl, unsigned L) {
    const uint32_t v = A.lnode[id];
    uint32_t g[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = A.lg[(size_t)k * A.label_cap + id];
    if (v == P.goal) {
      // Algorithm 1: a goal label is not expanded; it goes to P (virtual node n)
      if (gl == 0) {
        const uint32_t vp = G.n;
        const unsigned c = agg_inc(&C->cand_count.v);
        A.cnode[c] = vp;
        A.cparent[c] = A.lparent[id];
        A.cedge[c] = A.ledge[id];
#pragma unroll
        for (int k = 0; k < D; ++k) A.cg[(size_t)k * A.cand_cap + c] = g[k];
        const unsigned pos = atomicAdd(&A.ncand[vp], 1u);
        if (pos < kNodeSlots)
          A.cslot[(size_t)vp * kNodeSlots + pos] = (int)c;
        else
          A.cnext[c] = atomicExch(&A.node_head[vp], (int)c);
        if (pos == 0) A.touched[agg_inc(&C->touched_count.v)] = vp;
      }
      return;
    }
    const uint32_t e0 = __ldg(G.rowptr + v), e1 = __ldg(G.rowptr + v + 1);
    for (uint32_t e = e0 + gl; e < e1; e += L) {
      const uint32_t v2 = __ldg(G.col + e);
      st[S_CAND]++;
      if (hk(0, v2) == kInf) continue;  // goal unreachable from v2
      const unsigned c = agg_inc(&C->cand_count.v);
      A.cnode[c] = v2;
      A.cparent[c] = id;
      A.cedge[c] = e;
#pragma unroll
      for (int k = 0; k < D; ++k) A.cg[(size_t)k * A.cand_cap + c] = g[k] + __ldg(G.cost + (size_t)k * G.m + e);
      const unsigned pos = atomicAdd(&A.ncand[v2], 1u);
      if (pos < kNodeSlots)
        A.cslot[(size_t)v2 * kNodeSlots + pos] = (int)c;
      else
        A.cnext[c] = atomicExch(&A.node_head[v2], (int)c);
      if (pos == 0) {
        // a node with a large frontier is merged by a whole block; it is kept at
        // the far end of the touched array (touched + heavy <= candidates <= cand_cap)
        if (A.fcount[v2] >= kHeavyFrontier)
          A.touched[A.cand_cap - 1u - atomicAdd(&C->heavy_count.v, 1u)] = v2;
        else
          A.touched[agg_inc(&C->touched_count.v)] = v2;
      }
    }
  }

  // ---------------- phase 2: extraction + expansion (Algorithm 2) ----------------
  // A warp reads 32 OPEN entries at a time: dead entries are dropped (lazy OPEN
  // delete), entries in the window whose F a solution weakly dominates are
  // dropped (lazy PruneOPEN), the other window entries are closed and expanded
  // at once by lane groups; the rest is copied to the next OPEN.
  template <class Team>
  __device__ void phase_extract_expand(const Team& T, unsigned cur, unsigned n_in, const BinParams& bp) {
    const unsigned bstar = select_bucket(cur);
    const unsigned nxt = cur ^ 1u;
    for (unsigned i = T.tid(); i < kNB; i += T.nthreads()) A.hist[nxt * kNB + i] = 0;
    if (T.leader()) {
      C->theta = bstar;
      C->plog_snap = ld_volatile(&C->plog_len.v);
      C->f1span[cur] = 0;  // measured again by the next step's phase 1
    }
    const uint64_t* in = A.okey[cur];
    const uint32_t* in_id = A.oid[cur];
    uint64_t* out = A.okey[nxt];
    uint32_t* out_id = A.oid[nxt];
    const unsigned plen = ld_volatile(&C->plog_len.v);
    const unsigned pcount = ld_volatile(&C->ps_count);
    const unsigned pmark = ld_volatile(&C->ps_mark);
    const unsigned pntiles = ld_volatile(&C->ps_ntiles);
    const unsigned pbuf = ld_volatile(&C->ps_cur);
    const unsigned lane = lane_id();
    const unsigned L = P.lanes, G_per = 32 / L, grp = lane / L, gl = lane % L;
    unsigned long long kmin = ~0ull, pcmp = 0;
    for (unsigned base = T.wid() * 32; base < n_in; base += T.nwarps() * 32) {
      const unsigned i = base + lane;
      const bool valid = i < n_in;
      uint64_t key = 0;
      uint32_t id = 0;
      bool keep = false, want = false;
      if (valid) {
        key = in[i];
        id = in_id[i];
        if (A.lstatus[id] == ST_DEAD)
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
      if (since < plen) {
        if (pcount && since < pmark)
          p_filter(alive, F, pmark, plen, pcount, pntiles, pbuf, pcmp);
        else
          p_filter(alive, F, since, plen, 0, 0, 0, pcmp);
      }
      bool take = false;
      if (want && !alive) {
        A.lstatus[id] = ST_DEAD;
        st[S_GOALPRUNED]++;
      } else if (want) {
        if (agg_inc(&C->win_count.v) < A.win_cap) {
          A.lstatus[id] = ST_CLOSED;
          st[S_EXTRACTED]++;
          take = true;
        } else {
          keep = true;  // window full: stays in OPEN for the next step
        }
      }
      if (keep) {
        const unsigned o = agg_inc(&C->open_count[nxt].v);
        if (o < A.open_cap) {
          out[o] = key;
          out_id[o] = id;
          kmin = min(kmin, (unsigned long long)key);
        } else {
          set_error(C, OPMOS_ERR_CAPACITY);
        }
      }
      unsigned hits = __ballot_sync(0xffffffffu, take);
      while (hits) {
        const unsigned src = nth_bit(hits, grp);
        const uint32_t lid = __shfl_sync(0xffffffffu, id, src < 32 ? src : 0);
        if (src < 32) expand_label(lid, gl, L);
        for (unsigned r = 0; r < G_per && hits; ++r) hits &= hits - 1;
      }
    }
    if (lane == 0) st[S_PCMP] += pcmp;
    kmin = warp_min64(kmin);
    if (lane == 0 && kmin != ~0ull) atomicMin(&C->min_key[nxt].v, kmin);
    build_p_rank(T);
  }

  // F against the P index + the recent goal costs log[t0, t1): clears alive
  // for candidates a solution weakly dominates (Algorithm 1).
  __device__ void p_filter(bool& alive, const uint32_t (&F)[D], unsigned t0, unsigned t1, unsigned pcount,
                           unsigned pntiles, unsigned pbuf, unsigned long long& pcmp) {
    const unsigned lane = lane_id();
    constexpr int UT = 4;  // tail tiles loaded per round
    for (unsigned r0 = t0; r0 < t1; r0 += 32 * UT) {
      if (!__any_sync(0xffffffffu, alive)) return;
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
        pcmp += (unsigned long long)__popc(amask) * min(32u, t1 - j0);
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
    if (!pcount) return;
    const uint32_t* ps = A.ps[pbuf];
    const uint32_t* pst = A.pst[pbuf];
    const size_t tcap = A.plog_cap / 32 + 1;
    constexpr int U = 4;  // tile-minimum groups loaded per round
    for (unsigned tg0 = 0; tg0 < pntiles; tg0 += 32 * U) {
      if (!__any_sync(0xffffffffu, alive)) return;
      uint32_t tm[U][D];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned tl = tg0 + u * 32 + lane;
#pragma unroll
        for (int k = 0; k < D; ++k) tm[u][k] = tl < pntiles ? pst[(size_t)k * tcap + tl] : kInf;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned tg = tg0 + u * 32;
        unsigned amask = __ballot_sync(0xffffffffu, alive);
        if (tg >= pntiles || !amask) break;
        const bool vt = tg + lane < pntiles;
        while (amask) {
          const unsigned j = __ffs(amask) - 1;
          amask &= amask - 1;
          uint32_t Fj[D];
#pragma unroll
          for (int k = 0; k < D; ++k) Fj[k] = __shfl_sync(0xffffffffu, F[k], j);
          unsigned pm = __ballot_sync(0xffffffffu, vt && weakly_le<D>(tm[u], Fj));
          pcmp += min(32u, pntiles - tg);
          bool dead = false;
          while (pm && !dead) {
            const unsigned tt = __ffs(pm) - 1;
            pm &= pm - 1;
            const unsigned e = (tg + tt) * 32 + lane;
            const bool ve = e < pcount;
            uint32_t p[D];
#pragma unroll
            for (int k = 0; k < D; ++k) p[k] = ve ? ps[(size_t)k * A.plog_cap + e] : kInf;
            dead = __ballot_sync(0xffffffffu, ve && weakly_le<D>(p, Fj)) != 0;
            pcmp += 32;
          }
          if (dead && lane == j) alive = false;
        }
      }
    }
  }

  // ---------------- phase 4: merge (Algorithm 1: frontier checks and goal branch) ----------------
  __device__ void merge_batch(uint32_t v, int mine, unsigned nb, unsigned cur, unsigned psnap, unsigned pmark,
                              unsigned pcount, unsigned pntiles, unsigned pbuf) {
    const unsigned lane = lane_id();
    const bool is_goal = (v == G.n);  // the virtual node standing for P
    uint32_t c[D];
    const bool valid = lane < nb;
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = valid ? A.cg[(size_t)k * A.cand_cap + mine] : 0u;
    bool alive = valid;
    // (a) in-batch: dominated by, or a duplicate of an earlier, candidate
    for (unsigned j = 0; j < nb; ++j) {
      uint32_t cj[D];
#pragma unroll
      for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
      if (alive && lane != j && (dominates<D>(cj, c) || (j < lane && equal<D>(cj, c)))) alive = false;
    }
    uint64_t fb = A.fbase[v];
    unsigned cap = A.fcap[v];
    const unsigned fc = A.fcount[v];
    unsigned out = fc;
    unsigned long long fcmp = 0, pruned_n = 0, pcmp = 0;
    if (is_goal) {
      // (b') at the goal alpha(v_g) is P: one weak-dominance test against the
      // P index and every goal cost logged since it was built (this warp is
      // the only writer of the log in this phase). P members a new solution
      // dominates are dropped once, at output (Prune(P, l) of Algorithm 1).
      const unsigned plen = ld_volatile(&C->plog_len.v);
      p_filter(alive, c, pcount ? pmark : 0u, plen, pcount, pntiles, pbuf, pcmp);
    } else {
      // (b) against the frontier alpha(v), compacting it in place; four
      // tiles of 32 entries are loaded per round
      out = 0;
      constexpr int U = 4;
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
          while (amask) {
            const unsigned j = __ffs(amask) - 1;
            amask &= amask - 1;
            uint32_t cj[D];
#pragma unroll
            for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
            const bool wd = vm && weakly_le<D>(m[u], cj);
            if (__ballot_sync(0xffffffffu, wd) && lane == j) alive = false;
            pruned |= vm && dominates<D>(cj, m[u]);
          }
          const bool keep = vm && !pruned;
          if (vm && pruned) {
            A.lstatus[mid[u]] = ST_DEAD;
            pruned_n++;
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
    merge_finish(v, mine, c, valid, alive, out, fb, cap, cur, psnap, pmark, pcount, pntiles, pbuf, fcmp, pruned_n,
                 pcmp);
  }

  // The end of a batch's merge, by one warp, lane j holding candidate j:
  // (c) F against P (Algorithm 1) at an ordinary node, then (d) survivors
  // become labels and join alpha(v) and OPEN (or the P log at the goal).
  // out = live frontier entries left after (b); fb, cap = the frontier block.
  __device__ void merge_finish(uint32_t v, int mine, const uint32_t (&c)[D], bool valid, bool alive, unsigned out,
                               uint64_t fb, unsigned cap, unsigned cur, unsigned psnap, unsigned pmark,
                               unsigned pcount, unsigned pntiles, unsigned pbuf, unsigned long long fcmp,
                               unsigned long long pruned_n, unsigned long long pcmp) {
    const unsigned lane = lane_id();
    const unsigned nxt = cur ^ 1u;
    const bool is_goal = (v == G.n);
    if (!is_goal && __any_sync(0xffffffffu, alive)) {
      uint32_t F[D];
#pragma unroll
      for (int k = 0; k < D; ++k) F[k] = c[k] + (valid ? hk(k, v) : 0u);
      p_filter(alive, F, pcount ? pmark : 0u, psnap, pcount, pntiles, pbuf, pcmp);
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
        unsigned long long my_key = ~0ull;
        if (alive) {
          const unsigned r = __popc(smask & lanemask_lt());
          const unsigned id = lb + r;
#pragma unroll
          for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap + id] = c[k];
          A.lnode[id] = is_goal ? P.goal : v;
          A.lparent[id] = A.cparent[mine];
          A.ledge[id] = A.cedge[mine];
          A.lpver[id] = psnap;
          A.lstatus[id] = is_goal ? ST_CLOSED : ST_OPEN;
#pragma unroll
          for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + out + r] = c[k];
          A.fpool[fb + (size_t)D * cap + out + r] = id;
          if (is_goal) {
#pragma unroll
            for (int k = 0; k < D; ++k) A.plog[(size_t)k * A.plog_cap + plen + r] = c[k];
          } else {
            const uint64_t key = ((uint64_t)(c[0] + hk(0, v)) << 32) | (D > 1 ? c[1 % D] + hk(1 % D, v) : 0u);
            const unsigned o = agg_inc(&C->open_count[nxt].v);
            if (o < A.open_cap) {
              A.okey[nxt][o] = key;
              A.oid[nxt][o] = id;
              my_key = key;
            } else {
              set_error(C, OPMOS_ERR_CAPACITY);
            }
          }
        }
        my_key = warp_min64(my_key);
        if (lane == 0 && my_key != ~0ull) atomicMin(&C->min_key[nxt].v, my_key);
        if (is_goal && lane == 0) {
          __threadfence();
          *reinterpret_cast<volatile unsigned*>(&C->plog_len.v) = plen + ns;
        }
        out += ns;
      }
    }
    if (lane == 0) {
      A.fcount[v] = out;
      st[S_INSERTED] += ns;
      st[S_PRUNED] += pruned_n;
      st[S_FCMP] += fcmp;
      st[S_PCMP] += pcmp;
    }
  }

  // Merge of a node with a large frontier by the whole block (every thread
  // calls it). Batches of up to 32 candidates as in merge_batch; warp 0
  // gathers a batch and resolves it in itself (a), then all warps scan the
  // frontier (b) in rounds of nwarps * 32 * U entries, each warp U tiles of
  // 32, and compact it in place: a round's reads all precede the first
  // barrier, its writes land below the round's start, so they never overwrite
  // an entry another warp still has to read. Candidates killed by one warp
  // are dropped by the others from the next round on. A candidate that a
  // frontier entry weakly dominates never dominates another entry (the
  // frontier is an antichain), so the entries each candidate prunes do not
  // depend on when its death is seen. Warp 0 then runs (c)-(d).
  __device__ void merge_heavy(uint32_t v, unsigned cur, unsigned psnap, unsigned pmark, unsigned pcount,
                              unsigned pntiles, unsigned pbuf) {
    constexpr int U = 2;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) S.m_next = -2;  // first batch: the node's slots
    for (;;) {
      __syncthreads();
      if (S.m_next == kNil) break;
      __syncthreads();  // every thread has read m_next before warp 0 moves it
      if (w == 0) {
        int cur_c = S.m_next;
        int mine = kNil;
        unsigned nb = 0;
        if (cur_c == -2) {
          const unsigned ncand = A.ncand[v];
          const int slot = A.cslot[(size_t)v * kNodeSlots + lane];
          cur_c = ncand > kNodeSlots ? A.node_head[v] : kNil;
          __syncwarp();
          if (lane == 0) {
            A.ncand[v] = 0;
            if (ncand > kNodeSlots) A.node_head[v] = kNil;
          }
          nb = min(ncand, kNodeSlots);
          if (lane < nb) mine = slot;
        } else {
          while (cur_c != kNil && nb < 32) {
            if (lane == nb) mine = cur_c;
            cur_c = A.cnext[cur_c];
            ++nb;
          }
        }
        const bool valid = lane < nb;
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = valid ? A.cg[(size_t)k * A.cand_cap + mine] : 0u;
        bool alive = valid;
        for (unsigned j = 0; j < nb; ++j) {
          uint32_t cj[D];
#pragma unroll
          for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
          if (alive && lane != j && (dominates<D>(cj, c) || (j < lane && equal<D>(cj, c)))) alive = false;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) S.mc[k][lane] = c[k];
        S.mmine[lane] = mine;
        const unsigned a0 = __ballot_sync(0xffffffffu, alive);
        if (lane == 0) {
          S.m_next = cur_c;
          S.m_nb = nb;
          S.m_alive = a0;
          S.m_kill = 0;
        }
      }
      __syncthreads();
      unsigned a = S.m_alive;
      const uint64_t fb = A.fbase[v];
      const unsigned cap = A.fcap[v];
      const unsigned fc = A.fcount[v];
      unsigned out = 0;
      unsigned long long fcmp = 0, pruned_n = 0;
      const unsigned R = nw * 32u * U;
      for (unsigned r0 = 0; r0 < fc; r0 += R) {
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
        unsigned kill = 0, km[U], wtot = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned i0 = base + u * 32;
          const unsigned i = i0 + lane;
          const bool vm = i < fc;
          bool pruned = false;
          unsigned am = i0 < fc ? (a & ~kill) : 0u;
          if (i0 < fc) fcmp += (unsigned long long)__popc(am) * min(32u, fc - i0);
          while (am) {
            const unsigned j = __ffs(am) - 1;
            am &= am - 1;
            uint32_t cj[D];
#pragma unroll
            for (int k = 0; k < D; ++k) cj[k] = S.mc[k][j];
            if (__ballot_sync(0xffffffffu, vm && weakly_le<D>(m[u], cj))) kill |= 1u << j;
            pruned |= vm && dominates<D>(cj, m[u]);
          }
          if (vm && pruned) {
            A.lstatus[mid[u]] = ST_DEAD;
            pruned_n++;
          }
          km[u] = __ballot_sync(0xffffffffu, vm && !pruned);
          wtot += __popc(km[u]);
        }
        if (lane == 0) {
          S.warp[w] = wtot;
          if (kill) atomicOr(&S.m_kill, kill);
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
        a &= ~S.m_kill;
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
        __syncthreads();  // (2) S.warp and S.m_kill read by every warp
        const unsigned seen = min(r0 + R, fc);
        out += total;
        if (a == 0 && out == seen) {
          // no candidate left to test and nothing moved: the rest stays in place
          out = fc;
          break;
        }
      }
      if (lane == 0) {
        st[S_PRUNED] += pruned_n;
        st[S_FCMP] += fcmp;
      }
      if (w == 0) {
        const unsigned nb = S.m_nb;
        const bool valid = lane < nb;
        uint32_t c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = S.mc[k][lane];
        const bool alive = valid && ((a >> lane) & 1u);
        merge_finish(v, S.mmine[lane], c, valid, alive, out, fb, cap, cur, psnap, pmark, pcount, pntiles, pbuf,
                     0ull, 0ull, 0ull);
      }
    }
  }

  template <class Team>
  __device__ void phase_merge(const Team& T, unsigned cur) {
    const unsigned nt = ld_volatile(&C->touched_count.v);
    const unsigned psnap = ld_volatile(&C->plog_snap);
    const unsigned pcount = ld_volatile(&C->ps_count);
    const unsigned pmark = ld_volatile(&C->ps_mark);
    const unsigned pntiles = ld_volatile(&C->ps_ntiles);
    const unsigned pbuf = ld_volatile(&C->ps_cur);
    const unsigned lane = lane_id();
    // heavy nodes first, one block each
    const unsigned nh = ld_volatile(&C->heavy_count.v);
    while (nh) {
      if (threadIdx.x == 0) S.m_claim = atomicAdd(&C->heavy_next.v, 1u);
      __syncthreads();
      const unsigned h = S.m_claim;
      __syncthreads();
      if (h >= nh) break;
      merge_heavy(A.touched[A.cand_cap - 1u - h], cur, psnap, pmark, pcount, pntiles, pbuf);
    }
    for (;;) {
      unsigned t = 0;
      if (lane == 0) t = atomicAdd(&C->merge_next.v, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= nt) break;
      const uint32_t v = A.touched[t];
      // the first kNodeSlots candidates sit in the node's slots (one load), the
      // rest in a list
      const unsigned ncand = A.ncand[v];
      const int slot = A.cslot[(size_t)v * kNodeSlots + lane];
      int cur_c = ncand > kNodeSlots ? A.node_head[v] : kNil;
      __syncwarp();
      if (lane == 0) {
        A.ncand[v] = 0;
        if (ncand > kNodeSlots) A.node_head[v] = kNil;
      }
      const unsigned n0 = min(ncand, kNodeSlots);
      merge_batch(v, lane < n0 ? slot : kNil, n0, cur, psnap, pmark, pcount, pntiles, pbuf);
      while (cur_c != kNil) {
        int mine = kNil;
        unsigned nb = 0;
        while (cur_c != kNil && nb < 32) {
          if (lane == nb) mine = cur_c;
          cur_c = A.cnext[cur_c];
          ++nb;
        }
        merge_batch(v, mine, nb, cur, psnap, pmark, pcount, pntiles, pbuf);
      }
    }
    build_p_tiles(T);
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
        A.lstatus[A.fpool[fb + (size_t)D * cap + i]] = ST_DEAD;
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
      if (A.lstatus[idi] == ST_DEAD) continue;
      uint32_t ci[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) ci[kk] = A.fpool[fb + (size_t)kk * cap + i];
      unsigned rank = 0;
      for (unsigned j = 0; j < k; ++j) {
        uint32_t cj[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) cj[kk] = A.fpool[fb + (size_t)kk * cap + j];
        if ((lex_less<D>(cj, ci) || (j < i && equal<D>(cj, ci))) &&
            A.lstatus[A.fpool[fb + (size_t)D * cap + j]] != ST_DEAD)
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
      if (A.lstatus[idi] == ST_DEAD) continue;
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

}  // namespace

template <int D, class Team>
__device__ void run_query(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                          const OutPool& O, const Team& T, QResult* R, bool reset_ctl) {
  __shared__ Shared S;
  Search<D> X(G, A, C, P, O, S);
  X.init_zero(T);
  if (reset_ctl && T.leader()) C->error = 0;
  bool ok = T.sync(C);
  X.init_seed(T, reset_ctl);
  ok = ok && T.sync(C);
  unsigned step = 0;
  unsigned long long tph = globaltimer();
  auto lap = [&](int idx) {
    if (T.leader()) {
      const unsigned long long t = globaltimer();
      X.st[idx] += t - tph;
      tph = t;
    }
  };
  while (ok) {
    const unsigned cur = step & 1u;
    const unsigned n_in = ld_volatile(&C->open_count[cur].v);
    if (n_in == 0) break;
    if (T.leader() && globaltimer() - C->t_start > P.time_limit_ns) set_error(C, OPMOS_ERR_TIMEOUT);
    const unsigned long long base = ld_volatile64(&C->min_key[cur].v);
    BinParams bp;
    bp.b0 = (uint32_t)(base >> 32);
    bp.b1 = (uint32_t)base;
    bp.delta = P.delta;
    bp.s1 = 0;
    for (unsigned sp = ld_volatile(&C->f1span[cur]); (sp >> bp.s1) >= (unsigned)kNB1; ++bp.s1) {
    }
    X.phase_hist(T, cur, n_in, bp);
    if (!(ok = T.sync(C))) break;
    lap(S_THIST);
    X.phase_extract_expand(T, cur, n_in, bp);
    if (!(ok = T.sync(C))) break;
    lap(S_TEXPAND);
    X.phase_merge(T, cur);
    if (!(ok = T.sync(C))) break;
    lap(S_TMERGE);
    ++step;
  }
  if (ok) {
    if (T.leader()) C->res_count = 0;
    ok = T.sync(C) && X.output(T);
    lap(S_TOUT);
  }
  X.st[S_STEPS] = T.leader() ? step : 0;
  X.st[S_GOALINS] = T.leader() ? ld_volatile(&C->plog_len.v) : 0;
  flush_stats<Team>(C, X.st);
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

template <int D>
__global__ void __launch_bounds__(kGridThreads, 1) search_grid_kernel(GraphDev G, QArena A, QCtl* C, QParams P,
                                                          OutPool O, QResult* R) {
  run_query<D>(G, A, C, P, O, GridTeam{}, R, false);
}

// ---------------------------------------------------------------------------
// Multi-query persistent kernel (batch and serving): continuous batching of
// many independent queries. Every iteration:
//   P0  block 0 retires finished slots and admits queued queries into free
//       slots (FREE -> INIT -> RUN -> OUT -> FREE);
//   P1  INIT slots are initialised, OUT slots write their result, RUN slots
//       build their OPEN histogram;
//   P2  RUN slots extract and expand;  P3  RUN slots merge.
// In P1-P3 each block derives the same assignment of "virtual blocks" to slots
// (a running slot gets a share of the grid in proportion to its work, at
// least one block), so large and small queries advance side by side.
// ---------------------------------------------------------------------------
struct SubTeam {
  unsigned j, nb;
  __device__ __forceinline__ unsigned tid() const { return j * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ unsigned nthreads() const { return nb * blockDim.x; }
  __device__ __forceinline__ unsigned wid() const { return tid() >> 5; }
  __device__ __forceinline__ unsigned nwarps() const { return nthreads() >> 5; }
  __device__ __forceinline__ bool leader_block() const { return j == 0; }
  __device__ __forceinline__ bool leader() const { return j == 0 && threadIdx.x == 0; }
};

__device__ bool mq_barrier(MCtl* M) {
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

// P0: slot transitions and admission (block 0).
__device__ void mq_write_result(const MSlot& sl, unsigned slot, QCtl* C, QResult* results, unsigned* done_flags,
                                unsigned qcap) {
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

__device__ void mq_alloc_region1(const MSlot& sl, QCtl* C) {
  const OutPool& O = sl.O;
  const unsigned kk_live = ld_volatile(&C->res_count);
  const unsigned long long words = (unsigned long long)kk_live * sl.d + kk_live + 1;
  const unsigned long long off = atomicAdd(O.used, words);
  if (off + words > O.cap) atomicCAS(&C->error, 0u, (unsigned)OPMOS_ERR_CAPACITY);
  C->res_off = off;
}

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
      if (ld_volatile(&C->error) || ld_volatile(&C->open_count[step & 1u].v) == 0)
        st = SL_OUT1;
      else if (globaltimer() - C->t_start > sl.P.time_limit_ns) {
        atomicCAS(&C->error, 0u, (unsigned)OPMOS_ERR_TIMEOUT);
        st = SL_OUT1;
      }
      if (st == SL_OUT1) C->res_count = 0;
    } else if (st == SL_INIT) {
      st = (ld_volatile(&C->error) || ld_volatile(&C->open_count[0].v) == 0) ? SL_OUT1 : SL_RUN;
      if (st == SL_OUT1) C->res_count = 0;
    } else if (st == SL_OUT1 || st == SL_OUT2 || st == SL_OUT3 || st == SL_OUT4) {
      // one output part per iteration; an error ends the output early
      if (ld_volatile(&C->error) || st == SL_OUT4) {
        mq_write_result(sl, q, C, results, done_flags, qcap);
        st = after_out;
      } else if (st == SL_OUT1) {
        mq_alloc_region1(sl, C);
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
__device__ void mq_work(MSlot* slots, QCtl* ctls, unsigned q, unsigned j, unsigned nb, unsigned ph, Shared& S) {
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
    flush_stats<BlockTeam>(C, X.st);
  } else if (st == SL_OUT1) {
    X.out_filter(SubTeam{j, nb});
    flush_stats<SubTeam>(C, X.st);
  } else if (st == SL_OUT2) {
    X.out_rank(SubTeam{j, nb});
  } else if (st == SL_OUT3) {
    X.out_scan();
  } else if (st == SL_OUT4) {
    X.out_paths(SubTeam{j, nb});
  } else if (st == SL_RUN) {
    const SubTeam T{j, nb};
    const unsigned cur = C->step & 1u;
    const unsigned n_in = ld_volatile(&C->open_count[cur].v);
    const unsigned long long base = ld_volatile64(&C->min_key[cur].v);
    BinParams bp;
    bp.b0 = (uint32_t)(base >> 32);
    bp.b1 = (uint32_t)base;
    bp.delta = P.delta;
    bp.s1 = 0;
    for (unsigned sp = ld_volatile(&C->f1span[cur]); (sp >> bp.s1) >= (unsigned)kNB1; ++bp.s1) {
    }
    if (ph == 1)
      X.phase_hist(T, cur, n_in, bp);
    else if (ph == 2)
      X.phase_extract_expand(T, cur, n_in, bp);
    else
      X.phase_merge(T, cur);
    flush_stats<SubTeam>(C, X.st);
  }
}

__device__ __forceinline__ unsigned A_fcount_goal(const MSlot& sl) { return sl.A.fcount[sl.G.n]; }

// Work units of a slot in phase ph (0: none). INIT and the scan part of the
// output get one block; the other output parts a share like search phases.
__device__ __forceinline__ unsigned mq_weight(const MSlot& sl, QCtl* C, unsigned ph, bool& single) {
  single = false;
  const unsigned st = sl.state;
  if (st == SL_FREE) return 0;
  if (st == SL_INIT || st == SL_OUT3) {
    single = ph == 1;
    return ph == 1 ? 1u : 0u;
  }
  if (st >= SL_OUT1) return ph == 1 ? max(1u, ld_volatile(&C->res_count) + A_fcount_goal(sl)) : 0u;
  const unsigned cur = C->step & 1u;
  const unsigned w = ph == 3 ? ld_volatile(&C->touched_count.v) + 8u * ld_volatile(&C->heavy_count.v)
                             : ld_volatile(&C->open_count[cur].v);
  return w ? w : 1u;  // a running slot always gets a block (index builds run in every phase)
}

__device__ void mq_phase(unsigned ph, MSlot* slots, QCtl* ctls, unsigned nslots, Shared& S, unsigned* s_pref) {
  // total weight of the multi-block slots
  __shared__ unsigned long long s_wtot;
  if (threadIdx.x == 0) s_wtot = 0;
  __syncthreads();
  unsigned long long wloc = 0;
  for (unsigned q = threadIdx.x; q < nslots; q += blockDim.x) {
    bool single;
    const unsigned w = mq_weight(slots[q], &ctls[q], ph, single);
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
      const unsigned w = mq_weight(slots[q], &ctls[q], ph, single);
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
    switch (slots[q].d) {
#define MQ_CASE(DD) \
  case DD:          \
    mq_work<DD>(slots, ctls, q, j, nb, ph, S); \
    break;
      MQ_CASE(1) MQ_CASE(2) MQ_CASE(3) MQ_CASE(4) MQ_CASE(5) MQ_CASE(6) MQ_CASE(7) MQ_CASE(8)
#undef MQ_CASE
      default:
        break;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMultiThreads, 2)
    multi_kernel(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                 const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M) {
  __shared__ Shared S;
  __shared__ unsigned s_pref[kMaxSlots + 1];
  for (;;) {
    if (blockIdx.x == 0) mq_schedule(slots, ctls, nslots, queue, hctl, graphs, M, results, done_flags);
    if (!mq_barrier(M)) return;
    if (ld_volatile(&M->done)) return;
    for (unsigned ph = 1; ph <= 3; ++ph) {
      mq_phase(ph, slots, ctls, nslots, S, s_pref);
      if (!mq_barrier(M)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int D>
static cudaError_t launch_grid_d(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                                 const OutPool& O, QResult* R, unsigned blocks, cudaStream_t s) {
  void* args[] = {(void*)&G, (void*)&A, (void*)&C, (void*)&P, (void*)&O, (void*)&R};
  return cudaLaunchCooperativeKernel((void*)search_grid_kernel<D>, dim3(blocks), dim3(kGridThreads), args, 0, s);
}

template <int D>
static int occupancy_d(int) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_grid_kernel<D>, kGridThreads, 0);
  return nb;
}

#define OPMOS_DISPATCH_D(d, CALL) \
  switch (d) {                    \
    case 1: return CALL(1);       \
    case 2: return CALL(2);       \
    case 3: return CALL(3);       \
    case 4: return CALL(4);       \
    case 5: return CALL(5);       \
    case 6: return CALL(6);       \
    case 7: return CALL(7);       \
    case 8: return CALL(8);       \
    default: break;               \
  }

cudaError_t launch_search_grid(unsigned d, const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                               const OutPool& O, QResult* R, unsigned blocks, cudaStream_t s) {
#define CALL(D) launch_grid_d<D>(G, A, C, P, O, R, blocks, s)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_multi(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                         const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M,
                         unsigned blocks, cudaStream_t s) {
  void* args[] = {(void*)&slots, (void*)&ctls, (void*)&nslots, (void*)&queue, (void*)&hctl,
                  (void*)&graphs, (void*)&results, (void*)&done_flags, (void*)&M};
  return cudaLaunchCooperativeKernel((void*)multi_kernel, dim3(blocks), dim3(kMultiThreads), args, 0, s);
}

int multi_occupancy() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, multi_kernel, kMultiThreads, 0);
  return nb;
}

int search_occupancy(unsigned d, int batch) {
#define CALL(D) occupancy_d<D>(batch)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return 0;
}

}  // namespace opmos
