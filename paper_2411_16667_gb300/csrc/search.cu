// Ordered-parallel multi-objective label-setting search (Sec. 5, Algorithm 2)
// on one GPU. One "team" of threads works on one query: the whole cooperative
// grid for a single query, or one thread block per query in batch mode. A step
// of the search is four phases separated by team barriers:
//
//   1. histogram   the open entries by bucket of F[0] (Algorithm 2 l.9, OPEN is
//                  a lexicographic priority queue; F[0] is its first key)
//   2. extract     the window = every live entry in the lowest buckets whose
//                  cumulative count stays within W (the NUM_POP of Sec. 5);
//                  entries whose label was pruned are dropped here (lazy OPEN
//                  delete, Sec. 5.1 / Alg. 2 l.11) and so are labels whose F is
//                  weakly dominated by a solution (PruneOPEN, Alg. 1 l.9-10,
//                  applied lazily at extraction)
//   3. expand      every window label along its out-arcs, L lanes per label:
//                  g' = g + c(e), dropped if h(v') is infinite (Alg. 1 l.15-17)
//   4. merge       one warp per target node: the node's candidates of this step
//                  are resolved against each other (in-batch dominance and
//                  duplicates), then against the node's frontier alpha(v')
//                  (Alg. 1 l.22-28: weakly dominated candidates are dropped,
//                  strictly dominated frontier labels are pruned), then against
//                  P on F (Alg. 1 l.29); survivors become labels, join alpha(v')
//                  and OPEN. At the goal node alpha(v_g) is P itself (Alg. 1
//                  l.11-13) and survivors are appended to the P log.
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
};

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

  // ---------------- initialisation (Algorithm 1 l.1-4) ----------------
  template <class Team>
  __device__ void init(const Team& T, bool reset_ctl) {
    for (unsigned v = T.tid(); v < G.n; v += T.nthreads()) {
      A.fcount[v] = 0;
      A.fcap[v] = 0;
      A.fbase[v] = 0;
      A.node_head[v] = kNil;
    }
    for (unsigned i = T.tid(); i < 2u * kNB; i += T.nthreads()) A.hist[i] = 0;
    if (T.leader()) {
      if (reset_ctl) {
        C->error = 0;
        C->done = 0;
        C->step = 0;
        C->win_count = C->cand_count = C->touched_count = 0;
        C->theta = 0;
        C->plog_snap = 0;
        C->res_count = C->res_status = 0;
        C->res_off = C->res_path = C->res_total = 0;
        for (int i = 0; i < kNStat; ++i) C->stats[i] = 0;
      }
      C->t_start = globaltimer();
      const uint32_t s = P.start, t = P.goal, tile = P.tile;
      // l_s = (v_s, 0): label 0, frontier of v_s, OPEN (lines 3-4)
#pragma unroll
      for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap] = 0;
      A.lnode[0] = s;
      A.lparent[0] = kInf;
      A.ledge[0] = kInf;
      A.lpver[0] = 0;
      A.lstatus[0] = (s == t) ? ST_CLOSED : ST_OPEN;
      A.fbase[s] = 0;
      A.fcap[s] = tile;
      A.fcount[s] = 1;
#pragma unroll
      for (int k = 0; k < D; ++k) A.fpool[(size_t)k * tile] = 0;
      A.fpool[(size_t)D * tile] = 0;
      C->f_words = (unsigned long long)(D + 1) * tile;
      C->n_labels = 1;
      C->plog_len = 0;
      const uint32_t key = hk(0, s);
      // start == goal: P = {l_s}, nothing to search. h(s) = inf: goal unreachable.
      if (s != t && key != kInf) {
        A.open[0][0] = ((uint64_t)key << 32) | 0u;
        C->open_count[0] = 1;
        C->min_key[0] = key;
      } else {
        C->open_count[0] = 0;
        C->min_key[0] = kInf;
      }
      C->open_count[1] = 0;
      C->min_key[1] = kInf;
      st[S_INSERTED] += 1;
    }
  }

  // ---------------- phase 1: bucket histogram of OPEN ----------------
  template <class Team>
  __device__ void phase_hist(const Team& T, unsigned cur, unsigned n_in, unsigned base) {
    for (unsigned i = threadIdx.x; i < kNB; i += blockDim.x) S.hist[i] = 0;
    __syncthreads();
    const uint64_t* in = A.open[cur];
    const unsigned delta = P.delta;
    for (unsigned i = T.tid(); i < n_in; i += T.nthreads()) {
      const unsigned key = (unsigned)(in[i] >> 32);
      unsigned b = key <= base ? 0u : (key - base) / delta;
      b = min(b, (unsigned)kNB - 1);
      atomicAdd(&S.hist[b], 1u);
    }
    __syncthreads();
    unsigned* gh = A.hist + cur * kNB;
    for (unsigned i = threadIdx.x; i < kNB; i += blockDim.x)
      if (S.hist[i]) atomicAdd(&gh[i], S.hist[i]);
    if (T.leader()) {
      const unsigned nxt = cur ^ 1u;
      C->open_count[nxt] = 0;
      C->min_key[nxt] = kInf;
      C->win_count = 0;
      C->cand_count = 0;
      C->touched_count = 0;
    }
  }

  // Threshold of the window: largest bucket b whose cumulative count is <= W,
  // but at least the first non-empty bucket. Every block computes the same.
  __device__ unsigned select_theta(unsigned cur, unsigned base) {
    const unsigned* gh = A.hist + cur * kNB;
    const unsigned per = kNB / blockDim.x;  // blockDim divides kNB
    const unsigned b0 = threadIdx.x * per;
    unsigned loc[kNB / 64 > 0 ? kNB / 64 : 1];
    unsigned sum = 0;
    for (unsigned j = 0; j < per; ++j) {
      loc[j] = *reinterpret_cast<const volatile unsigned*>(&gh[b0 + j]);
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
    unsigned bstar = max(S.b1_max, S.f_min == (unsigned)kNB ? 0u : S.f_min);
    __syncthreads();
    const unsigned long long th = (unsigned long long)base + (unsigned long long)(bstar + 1) * P.delta - 1;
    return th >= kInf ? kInf - 1 : (unsigned)th;
  }

  // ---------------- phase 2: extraction (Algorithm 2 l.9-16) ----------------
  template <class Team>
  __device__ void phase_extract(const Team& T, unsigned cur, unsigned n_in, unsigned base) {
    const unsigned theta = select_theta(cur, base);
    if (T.leader()) C->theta = theta;
    const unsigned nxt = cur ^ 1u;
    const uint64_t* in = A.open[cur];
    uint64_t* out = A.open[nxt];
    const unsigned plen = *reinterpret_cast<const volatile unsigned*>(&C->plog_len);
    unsigned kmin = kInf;
    for (unsigned i = T.tid(); i < n_in; i += T.nthreads()) {
      const uint64_t e = in[i];
      const unsigned key = (unsigned)(e >> 32);
      const unsigned id = (unsigned)e;
      bool keep = true;
      if (key <= theta) {
        keep = false;
        const uint8_t s = A.lstatus[id];
        if (s == ST_DEAD) {
          st[S_DEAD]++;
        } else {
          const uint32_t v = A.lnode[id];
          uint32_t F[D];
#pragma unroll
          for (int k = 0; k < D; ++k) F[k] = A.lg[(size_t)k * A.label_cap + id] + hk(k, v);
          bool dom = false;
          for (unsigned j = A.lpver[id]; j < plen && !dom; ++j) {
            uint32_t p[D];
#pragma unroll
            for (int k = 0; k < D; ++k) p[k] = A.plog[(size_t)k * A.plog_cap + j];
            dom = weakly_le<D>(p, F);
            st[S_PCMP]++;
          }
          if (dom) {
            A.lstatus[id] = ST_DEAD;
            st[S_GOALPRUNED]++;
          } else {
            const unsigned w = agg_inc(&C->win_count);
            if (w < A.win_cap) {
              A.window[w] = id;
              A.lstatus[id] = ST_CLOSED;
              st[S_EXTRACTED]++;
            } else {
              keep = true;  // window full: stays in OPEN for the next step
            }
          }
        }
      }
      if (keep) {
        const unsigned o = agg_inc(&C->open_count[nxt]);
        if (o < A.open_cap) {
          out[o] = e;
          kmin = min(kmin, key);
        } else {
          set_error(C, OPMOS_ERR_CAPACITY);
        }
      }
    }
    kmin = warp_min(kmin);
    if (lane_id() == 0 && kmin != kInf) atomicMin(&C->min_key[nxt], kmin);
  }

  // ---------------- phase 3: expansion (Algorithm 1 l.15-17) ----------------
  template <class Team>
  __device__ void phase_expand(const Team& T, unsigned nxt) {
    // the histogram of the next step starts from zero
    for (unsigned i = T.tid(); i < kNB; i += T.nthreads()) A.hist[nxt * kNB + i] = 0;
    if (T.leader()) C->plog_snap = *reinterpret_cast<const volatile unsigned*>(&C->plog_len);
    const unsigned nw = min(*reinterpret_cast<const volatile unsigned*>(&C->win_count), A.win_cap);
    const unsigned L = P.lanes;
    const unsigned gl = T.tid() % L;
    const unsigned ngroups = T.nthreads() / L;
    for (unsigned w = T.tid() / L; w < nw; w += ngroups) {
      const uint32_t id = A.window[w];
      const uint32_t v = A.lnode[id];
      uint32_t g[D];
#pragma unroll
      for (int k = 0; k < D; ++k) g[k] = A.lg[(size_t)k * A.label_cap + id];
      const uint32_t e0 = __ldg(G.rowptr + v), e1 = __ldg(G.rowptr + v + 1);
      for (uint32_t e = e0 + gl; e < e1; e += L) {
        const uint32_t v2 = __ldg(G.col + e);
        st[S_CAND]++;
        if (hk(0, v2) == kInf) continue;  // goal unreachable from v2
        const unsigned c = agg_inc(&C->cand_count);
        A.cnode[c] = v2;
        A.cparent[c] = id;
        A.cedge[c] = e;
#pragma unroll
        for (int k = 0; k < D; ++k)
          A.cg[(size_t)k * A.cand_cap + c] = g[k] + __ldg(G.cost + (size_t)k * G.m + e);
        const int old = atomicExch(&A.node_head[v2], (int)c);
        A.cnext[c] = old;
        if (old == kNil) A.touched[agg_inc(&C->touched_count)] = v2;
      }
    }
  }

  // ---------------- phase 4: merge (Algorithm 1 l.18-31, l.8-13) ----------------
  __device__ void merge_batch(uint32_t v, int mine, unsigned nb, unsigned cur, unsigned psnap) {
    const unsigned lane = lane_id();
    const unsigned nxt = cur ^ 1u;
    const bool is_goal = (v == P.goal);
    uint32_t c[D];
    const bool valid = lane < nb;
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = valid ? A.cg[(size_t)k * A.cand_cap + mine] : 0u;
    bool alive = valid;
    // (a) in-batch: dominated or duplicate of an earlier candidate
    for (unsigned j = 0; j < nb; ++j) {
      uint32_t cj[D];
#pragma unroll
      for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
      if (alive && lane != j && (dominates<D>(cj, c) || (j < lane && equal<D>(cj, c)))) alive = false;
    }
    // (b) against the frontier alpha(v), compacting it in place
    uint64_t fb = A.fbase[v];
    unsigned cap = A.fcap[v];
    const unsigned fc = A.fcount[v];
    unsigned out = 0;
    unsigned long long fcmp = 0, pruned_n = 0;
    for (unsigned i0 = 0; i0 < fc; i0 += 32) {
      const unsigned i = i0 + lane;
      const bool vm = i < fc;
      uint32_t m[D];
      uint32_t mid = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) m[k] = vm ? A.fpool[fb + (size_t)k * cap + i] : kInf;
      if (vm) mid = A.fpool[fb + (size_t)D * cap + i];
      bool pruned = false;
      unsigned amask = __ballot_sync(0xffffffffu, alive);
      if (amask == 0) {
        // nothing left to test: the rest of the frontier is kept as is
        if (out == i0) {
          out = fc;
          break;
        }
      }
      fcmp += (unsigned long long)__popc(amask) * min(32u, fc - i0);
      while (amask) {
        const unsigned j = __ffs(amask) - 1;
        amask &= amask - 1;
        uint32_t cj[D];
#pragma unroll
        for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(0xffffffffu, c[k], j);
        const bool wd = vm && weakly_le<D>(m, cj);
        if (__ballot_sync(0xffffffffu, wd) && lane == j) alive = false;
        pruned |= vm && dominates<D>(cj, m);
      }
      const bool keep = vm && !pruned;
      if (vm && pruned) {
        A.lstatus[mid] = ST_DEAD;
        pruned_n++;
      }
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      const unsigned pos = out + __popc(km & lanemask_lt());
      __syncwarp();
      if (keep && pos != i) {
#pragma unroll
        for (int k = 0; k < D; ++k) A.fpool[fb + (size_t)k * cap + pos] = m[k];
        A.fpool[fb + (size_t)D * cap + pos] = mid;
      }
      __syncwarp();
      out += __popc(km);
    }
    // (c) F against P (Algorithm 1 l.29); at the goal alpha(v_g) is P already
    unsigned long long pcmp = 0;
    if (!is_goal && __any_sync(0xffffffffu, alive)) {
      uint32_t F[D];
#pragma unroll
      for (int k = 0; k < D; ++k) F[k] = c[k] + (valid ? hk(k, v) : 0u);
      for (unsigned j0 = 0; j0 < psnap; j0 += 32) {
        unsigned amask = __ballot_sync(0xffffffffu, alive);
        if (!amask) break;
        const unsigned jj = j0 + lane;
        const bool vp = jj < psnap;
        uint32_t p[D];
#pragma unroll
        for (int k = 0; k < D; ++k) p[k] = vp ? A.plog[(size_t)k * A.plog_cap + jj] : kInf;
        pcmp += (unsigned long long)__popc(amask) * min(32u, psnap - j0);
        while (amask) {
          const unsigned j = __ffs(amask) - 1;
          amask &= amask - 1;
          uint32_t Fj[D];
#pragma unroll
          for (int k = 0; k < D; ++k) Fj[k] = __shfl_sync(0xffffffffu, F[k], j);
          const bool wd = vp && weakly_le<D>(p, Fj);
          if (__ballot_sync(0xffffffffu, wd) && lane == j) alive = false;
        }
      }
    }
    // (d) survivors become labels, join alpha(v), OPEN (or the P log at the goal)
    const unsigned smask = __ballot_sync(0xffffffffu, alive);
    const unsigned ns = __popc(smask);
    if (ns) {
      unsigned lb = 0;
      if (lane == 0) lb = atomicAdd(&C->n_labels, ns);
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
          if (lane == 0) nb0 = atomicAdd(&C->f_words, (unsigned long long)(D + 1) * ncap);
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
          plen = *reinterpret_cast<volatile unsigned*>(&C->plog_len);
          if (plen + ns > A.plog_cap) {
            if (lane == 0) set_error(C, OPMOS_ERR_CAPACITY);
            return;
          }
        }
        unsigned my_key = kInf;
        if (alive) {
          const unsigned r = __popc(smask & lanemask_lt());
          const unsigned id = lb + r;
#pragma unroll
          for (int k = 0; k < D; ++k) A.lg[(size_t)k * A.label_cap + id] = c[k];
          A.lnode[id] = v;
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
            const uint32_t key = c[0] + hk(0, v);
            const unsigned o = agg_inc(&C->open_count[nxt]);
            if (o < A.open_cap) {
              A.open[nxt][o] = ((uint64_t)key << 32) | id;
              my_key = key;
            } else {
              set_error(C, OPMOS_ERR_CAPACITY);
            }
          }
        }
        my_key = warp_min(my_key);
        if (lane == 0 && my_key != kInf) atomicMin(&C->min_key[nxt], my_key);
        if (is_goal && lane == 0) {
          __threadfence();
          *reinterpret_cast<volatile unsigned*>(&C->plog_len) = plen + ns;
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

  template <class Team>
  __device__ void phase_merge(const Team& T, unsigned cur) {
    const unsigned nt = *reinterpret_cast<const volatile unsigned*>(&C->touched_count);
    const unsigned psnap = *reinterpret_cast<const volatile unsigned*>(&C->plog_snap);
    const unsigned lane = lane_id();
    for (unsigned t = T.wid(); t < nt; t += T.nwarps()) {
      const uint32_t v = A.touched[t];
      int cur_c = A.node_head[v];
      __syncwarp();
      if (lane == 0) A.node_head[v] = kNil;
      while (cur_c != kNil) {
        int mine = kNil;
        unsigned nb = 0;
        while (cur_c != kNil && nb < 32) {
          if (lane == nb) mine = cur_c;
          cur_c = A.cnext[cur_c];
          ++nb;
        }
        merge_batch(v, mine, nb, cur, psnap);
      }
    }
  }

  // ---------------- output: sorted P and its paths ----------------
  template <class Team>
  __device__ void output(const Team& T, QResult* R) {
    const uint32_t t = P.goal;
    const unsigned k = A.fcount[t];
    const uint64_t fb = A.fbase[t];
    const unsigned cap = A.fcap[t];
    const bool paths = !(P.flags & OPMOS_FLAG_NO_PATHS);
    // region 1: costs (k*D, lexicographic) then path offsets (k+1)
    if (T.leader()) {
      const unsigned long long words = (unsigned long long)k * D + k + 1;
      const unsigned long long off = atomicAdd(O.used, words);
      if (off + words > O.cap) {
        set_error(C, OPMOS_ERR_CAPACITY);
      }
      C->res_off = off;
      C->res_count = k;
    }
    if (!T.sync(C)) return;
    const unsigned long long off = C->res_off;
    for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
      uint32_t ci[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) ci[kk] = A.fpool[fb + (size_t)kk * cap + i];
      unsigned rank = 0;
      for (unsigned j = 0; j < k; ++j) {
        uint32_t cj[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) cj[kk] = A.fpool[fb + (size_t)kk * cap + j];
        rank += lex_less<D>(cj, ci);
      }
#pragma unroll
      for (int kk = 0; kk < D; ++kk) O.words[off + (size_t)rank * D + kk] = ci[kk];
      unsigned len = 0;
      if (paths) {
        for (uint32_t x = A.fpool[fb + (size_t)D * cap + i]; x != kInf; x = A.lparent[x]) ++len;
      }
      O.words[off + (size_t)k * D + rank] = len;
    }
    if (!T.sync(C)) return;
    // exclusive scan of path lengths by the leader block, then allocate region 2
    if (T.leader_block()) {
      uint32_t* lens = O.words + off + (size_t)k * D;
      unsigned carry = 0;
      for (unsigned b0 = 0; b0 < k + 1; b0 += blockDim.x) {
        const unsigned i = b0 + threadIdx.x;
        const unsigned x = i < k ? lens[i] : 0;
        unsigned total;
        const unsigned ex = block_exclusive_scan(x, S.warp, total);
        if (i <= k) lens[i] = carry + ex;
        carry += total;
      }
      if (threadIdx.x == 0) {
        const unsigned long long total = carry;
        const unsigned long long words = paths ? 2 * total - k : 0;
        unsigned long long p0 = 0;
        if (words) {
          p0 = atomicAdd(O.used, words);
          if (p0 + words > O.cap) set_error(C, OPMOS_ERR_CAPACITY);
        }
        C->res_path = p0;
        C->res_total = total;
      }
    }
    if (!T.sync(C)) return;
    if (paths) {
      const unsigned long long p0 = C->res_path, total = C->res_total;
      const uint32_t* offs = O.words + off + (size_t)k * D;
      for (unsigned i = T.tid(); i < k; i += T.nthreads()) {
        uint32_t ci[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) ci[kk] = A.fpool[fb + (size_t)kk * cap + i];
        unsigned rank = 0;
        for (unsigned j = 0; j < k; ++j) {
          uint32_t cj[D];
#pragma unroll
          for (int kk = 0; kk < D; ++kk) cj[kk] = A.fpool[fb + (size_t)kk * cap + j];
          rank += lex_less<D>(cj, ci);
        }
        const unsigned a = offs[rank], b = offs[rank + 1];
        // nodes at p0 + [a, b); arcs at p0 + total + [a - rank, b - rank - 1)
        unsigned pos = b;
        for (uint32_t x = A.fpool[fb + (size_t)D * cap + i]; x != kInf; x = A.lparent[x]) {
          --pos;
          O.words[p0 + pos] = A.lnode[x];
          if (A.lparent[x] != kInf) O.words[p0 + total + pos - rank - 1] = A.ledge[x];
        }
      }
    }
  }
};

}  // namespace

template <int D, class Team>
__device__ void run_query(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                          const OutPool& O, const Team& T, QResult* R, bool reset_ctl) {
  __shared__ Shared S;
  Search<D> X(G, A, C, P, O, S);
  X.init(T, reset_ctl);
  bool ok = T.sync(C);
  unsigned step = 0;
  while (ok) {
    const unsigned cur = step & 1u, nxt = cur ^ 1u;
    const unsigned n_in = *reinterpret_cast<const volatile unsigned*>(&C->open_count[cur]);
    if (n_in == 0) break;
    if (T.leader() && globaltimer() - C->t_start > P.time_limit_ns) set_error(C, OPMOS_ERR_TIMEOUT);
    const unsigned base = *reinterpret_cast<const volatile unsigned*>(&C->min_key[cur]);
    X.phase_hist(T, cur, n_in, base);
    if (!(ok = T.sync(C))) break;
    X.phase_extract(T, cur, n_in, base);
    if (!(ok = T.sync(C))) break;
    X.phase_expand(T, nxt);
    if (!(ok = T.sync(C))) break;
    X.phase_merge(T, cur);
    if (!(ok = T.sync(C))) break;
    ++step;
  }
  if (ok) X.output(T, R);
  X.st[S_STEPS] = T.leader() ? step : 0;
  flush_stats<Team>(C, X.st);
  T.sync(C);
  if (T.leader()) {
    __threadfence();
    R->status = *reinterpret_cast<volatile unsigned*>(&C->error);
    R->count = C->res_count;
    R->off = C->res_off;
    R->path = C->res_path;
    R->total = C->res_total;
    R->labels = C->n_labels;
    R->f_words = C->f_words;
    for (int i = 0; i < kNStat; ++i) R->stats[i] = C->stats[i];
  }
}

template <int D>
__global__ void __launch_bounds__(256) search_grid_kernel(GraphDev G, QArena A, QCtl* C, QParams P,
                                                          OutPool O, QResult* R) {
  run_query<D>(G, A, C, P, O, GridTeam{}, R, false);
}

template <int D>
__global__ void __launch_bounds__(256) search_batch_kernel(GraphDev G, const QArena* arenas, QCtl* ctls,
                                                           const BatchQuery* qs, unsigned nq,
                                                           unsigned* next_q, QParams base, OutPool O,
                                                           QResult* results) {
  __shared__ unsigned s_q;
  const QArena A = arenas[blockIdx.x];
  QCtl* C = &ctls[blockIdx.x];
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(next_q, 1u);
    __syncthreads();
    const unsigned q = s_q;
    __syncthreads();
    if (q >= nq) break;
    QParams P = base;
    P.start = qs[q].start;
    P.goal = qs[q].goal;
    P.h = qs[q].h;
    run_query<D>(G, A, C, P, O, BlockTeam{}, &results[q], true);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int D>
static cudaError_t launch_grid_d(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                                 const OutPool& O, QResult* R, unsigned blocks, cudaStream_t s) {
  void* args[] = {(void*)&G, (void*)&A, (void*)&C, (void*)&P, (void*)&O, (void*)&R};
  return cudaLaunchCooperativeKernel((void*)search_grid_kernel<D>, dim3(blocks), dim3(256), args, 0, s);
}

template <int D>
static cudaError_t launch_batch_d(const GraphDev& G, const QArena* arenas, QCtl* ctls, const BatchQuery* qs,
                                  unsigned nq, unsigned* next_q, const QParams& P, const OutPool& O,
                                  QResult* R, unsigned blocks, cudaStream_t s) {
  search_batch_kernel<D><<<blocks, 256, 0, s>>>(G, arenas, ctls, qs, nq, next_q, P, O, R);
  return cudaGetLastError();
}

template <int D>
static int occupancy_d(int which) {
  int nb = 0;
  if (which == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_grid_kernel<D>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_batch_kernel<D>, 256, 0);
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

cudaError_t launch_search_batch(unsigned d, const GraphDev& G, const QArena* arenas, QCtl* ctls,
                                const BatchQuery* qs, unsigned nq, unsigned* next_q, const QParams& P,
                                const OutPool& O, QResult* R, unsigned blocks, cudaStream_t s) {
#define CALL(D) launch_batch_d<D>(G, arenas, ctls, qs, nq, next_q, P, O, R, blocks, s)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

int search_occupancy(unsigned d, int batch) {
#define CALL(D) occupancy_d<D>(batch)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return 0;
}

}  // namespace opmos
