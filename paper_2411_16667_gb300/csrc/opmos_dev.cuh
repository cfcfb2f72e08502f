// Device-side building blocks of the GB300 multi-objective search.
//
// Data layout (all device-resident, structure of arrays):
//   graph      rowptr[n+1], col[m], cost[k*m + e]; reversed CSR rrowptr/rsrc/rcost
//   heuristic  h[k*n + v]                      (Sec. 4 ideal point)
//   labels     lg[k*label_cap + id], lnode, lparent, ledge, lstatus, lpver
//   frontier   per node v: a contiguous block at fpool[fbase[v]] of capacity
//              fcap[v]: costs [k*cap + i] then label ids [d*cap + i]; fcount[v]
//              live entries (alpha(v) = G_OP(v) u G_CL(v), Sec. 3)
//   OPEN       two unsorted arrays of 64-bit keys (F[0] << 32 | F[1]) with
//              label ids beside them, bucketed through a per-step histogram
//              (the batch extraction of Algorithm 2): the lowest F[0] bucket is split by F[1]
//   P log      append-only list of every goal cost vector ever accepted; its
//              prefix is a valid filter for "F dominated by P" (Algorithm 1)
//   P index    a snapshot of P sorted along a Z-order curve over objectives
//              1..3, tiled by 32 with each tile's componentwise minimum
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "opmos.h"

namespace opmos {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr int32_t kNil = -1;
constexpr int kNB = 2048;   // open-list histogram buckets per step
constexpr int kNB1 = 1024;  // of which sub-buckets (by F[1]) of the lowest F[0] bucket
constexpr unsigned kPSMax = 32768;  // largest P indexed by the sorted snapshot
constexpr unsigned kHeavyFrontier = 512;  // frontiers this large are merged by a whole block
constexpr unsigned kNodeSlots = 32;  // candidates a node holds in slots per step; more go to a list

enum : uint8_t { ST_OPEN = 0, ST_CLOSED = 1, ST_DEAD = 2 };

enum StatIdx {
  S_EXTRACTED = 0,
  S_DEAD,
  S_GOALPRUNED,
  S_CAND,
  S_INSERTED,
  S_PRUNED,
  S_STEPS,
  S_FCMP,
  S_PCMP,
  S_THIST,    // device ns spent in phase 1 (leader's view, barrier included)
  S_TEXPAND,  // phase 2
  S_TMERGE,   // phase 4
  S_TOUT,     // output
  S_GOALINS,  // goal labels accepted into P during the search (P log length)
  kNStat
};

constexpr unsigned kGridThreads = 512;  // threads per block of the single-query grid

struct GraphDev {
  uint32_t n, m, d, maxdeg;
  const uint32_t* rowptr;   // n+1
  const uint32_t* col;      // m
  const uint32_t* cost;     // d*m
  const uint32_t* rrowptr;  // n+1, in-arcs grouped by head node
  const uint32_t* rsrc;     // m, tail node of each reversed arc
  const uint32_t* rcost;    // d*m, cost of each reversed arc
};

// A counter alone in its 128-byte line: the hot counters of a query are hit
// by atomics from every warp each step, and counters sharing a line would
// serialise on it.
template <class T>
struct alignas(128) Hot {
  T v;
};

// Per-query control block (global memory). Counters that the team reads after
// a barrier are plain words; concurrent updates use atomics.
struct QCtl {
  unsigned error;
  unsigned done;
  unsigned step;
  unsigned theta;
  unsigned plog_snap;
  unsigned res_count;
  unsigned res_status;
  unsigned f1span[2];     // F[1] spread of the lowest F[0] bucket, measured per step
  unsigned ps_cur, ps_count, ps_mark, ps_ntiles;   // live P index
  unsigned ps_build, ps_src, ps_mark_new, ps_nbuild;
  unsigned ps_shift[3];
  unsigned ps_nb;         // index buffer being built this step
  unsigned long long res_off;    // costs (count*d) then path offsets (count+1)
  unsigned long long res_path;   // nodes (total) then arc ids (total - count)
  unsigned long long res_total;  // total path nodes
  unsigned long long t_start;
  unsigned long long stats[kNStat];
  Hot<unsigned> n_labels;
  Hot<unsigned> open_count[2];
  Hot<unsigned> win_count;
  Hot<unsigned> cand_count;
  Hot<unsigned> touched_count;
  Hot<unsigned> merge_next;    // next touched node to merge (dynamic scheduling)
  Hot<unsigned> heavy_count;   // touched nodes with a large frontier, merged by a whole block
  Hot<unsigned> heavy_next;    // next heavy node to merge
  Hot<unsigned> plog_len;
  Hot<unsigned long long> min_key[2];  // lexicographic minimum (F0 << 32 | F1) of OPEN
  Hot<unsigned long long> f_words;
  Hot<unsigned> bar_count;
  Hot<unsigned> bar_gen;
};

// Pointers into one query's arena (one slot).
struct QArena {
  uint64_t* fbase;     // n
  uint32_t* fcount;    // n
  uint32_t* fcap;      // n
  int32_t* node_head;  // n: this step's candidates beyond the slots (linked by cnext)
  uint32_t* ncand;     // n: candidates that reached the node this step
  int32_t* cslot;      // n * kNodeSlots: the first kNodeSlots of them
  uint32_t* lg;        // d * label_cap
  uint32_t* lnode;
  uint32_t* lparent;
  uint32_t* ledge;
  uint32_t* lpver;
  uint8_t* lstatus;
  uint32_t* fpool;
  uint64_t* okey[2];   // OPEN keys (F0 << 32 | F1)
  uint32_t* oid[2];    // OPEN label ids
  uint32_t* ps[2];     // P index: d * plog_cap costs, Z-order
  uint32_t* pst[2];    // P index tile minima: d * (plog_cap / 32 + 1)
  uint32_t* window;
  uint32_t* cnode;
  uint32_t* cparent;
  uint32_t* cedge;
  int32_t* cnext;
  uint32_t* cg;        // d * cand_cap
  uint32_t* touched;
  uint32_t* plog;      // d * plog_cap
  uint32_t* hist;      // 2 * kNB
  uint32_t label_cap;
  uint32_t open_cap;
  uint32_t win_cap;
  uint32_t cand_cap;
  uint32_t plog_cap;
  uint32_t pad;
  unsigned long long fpool_words;
};

struct QParams {
  uint32_t start, goal;
  const uint32_t* h;      // d * n
  uint32_t window;        // target W
  uint32_t lanes;         // lanes per label
  uint32_t delta;         // F[0] bucket width
  uint32_t tile;          // frontier growth granule
  uint32_t label_budget;  // max labels (<= label_cap)
  uint32_t flags;
  unsigned long long time_limit_ns;
};

struct OutPool {
  uint32_t* words;
  unsigned long long cap;
  unsigned long long* used;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Warp-aggregated atomic increment: one atomicAdd per group of converged lanes.
__device__ __forceinline__ unsigned agg_inc(unsigned* ctr) {
  const unsigned mask = __activemask();
  const unsigned leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane_id() == leader) base = atomicAdd(ctr, __popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & lanemask_lt());
}

__device__ __forceinline__ void set_error(QCtl* C, unsigned code) { atomicCAS(&C->error, 0u, code); }

// ---------------------------------------------------------------------------
// Dominance on d-vectors (Sec. 3): a dominates b iff a <= b componentwise and
// a < b in some component; "weakly" drops the strictness (covers Duplicate).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ bool weakly_le(const uint32_t (&a)[D], const uint32_t (&b)[D]) {
  bool r = true;
#pragma unroll
  for (int k = 0; k < D; ++k) r &= (a[k] <= b[k]);
  return r;
}
template <int D>
__device__ __forceinline__ bool dominates(const uint32_t (&a)[D], const uint32_t (&b)[D]) {
  bool le = true, lt = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    le &= (a[k] <= b[k]);
    lt |= (a[k] < b[k]);
  }
  return le && lt;
}
template <int D>
__device__ __forceinline__ bool equal(const uint32_t (&a)[D], const uint32_t (&b)[D]) {
  bool r = true;
#pragma unroll
  for (int k = 0; k < D; ++k) r &= (a[k] == b[k]);
  return r;
}
template <int D>
__device__ __forceinline__ bool lex_less(const uint32_t (&a)[D], const uint32_t (&b)[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (a[k] != b[k]) return a[k] < b[k];
  return false;
}

// ---------------------------------------------------------------------------
// Teams: the set of threads that cooperates on one query.
// ---------------------------------------------------------------------------
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;  // 20 s

// Whole cooperative grid on one query; the barrier is a generation counter
// with a bounded wait (gives up with OPMOS_ERR_TIMEOUT, never hangs).
struct GridTeam {
  __device__ __forceinline__ unsigned tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ unsigned nthreads() const { return gridDim.x * blockDim.x; }
  __device__ __forceinline__ unsigned wid() const { return tid() >> 5; }
  __device__ __forceinline__ unsigned nwarps() const { return nthreads() >> 5; }
  __device__ __forceinline__ bool leader_block() const { return blockIdx.x == 0; }
  __device__ __forceinline__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
  // Returns false when the query has an error set; the decision is read once
  // per block so every thread of a block takes the same branch.
  __device__ __forceinline__ bool sync(QCtl* C) const {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned gen = ld_volatile(&C->bar_gen.v);
      __threadfence();
      const unsigned arrived = atomicAdd(&C->bar_count.v, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(&C->bar_count.v, 0u);
        __threadfence();
        atomicAdd(&C->bar_gen.v, 1u);
      } else {
        const unsigned long long t0 = globaltimer();
        unsigned spins = 0;
        while (ld_volatile(&C->bar_gen.v) == gen) {
          if (++spins > 64) __nanosleep(64);
          if ((spins & 255u) == 0) {
            if (ld_volatile(&C->error) != 0) break;
            if (globaltimer() - t0 > kBarrierTimeoutNs) {
              set_error(C, OPMOS_ERR_TIMEOUT);
              break;
            }
          }
        }
      }
      __threadfence();
      s_ok = ld_volatile(&C->error) == 0;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// One thread block on one query (batch mode).
struct BlockTeam {
  __device__ __forceinline__ unsigned tid() const { return threadIdx.x; }
  __device__ __forceinline__ unsigned nthreads() const { return blockDim.x; }
  __device__ __forceinline__ unsigned wid() const { return threadIdx.x >> 5; }
  __device__ __forceinline__ unsigned nwarps() const { return blockDim.x >> 5; }
  __device__ __forceinline__ bool leader_block() const { return true; }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
  __device__ __forceinline__ bool sync(QCtl* C) const {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) s_ok = ld_volatile(&C->error) == 0;
    __syncthreads();
    return s_ok != 0;
  }
};

}  // namespace opmos
