// Device-side building blocks of the GB300 multi-objective search.
//
// Data layout (all device-resident, structure of arrays):
//   graph      rowptr[n+1], col[m], cost[k*m + e]; reversed CSR rrowptr/rsrc/rcost
//   heuristic  h[k*n + v]                      (Sec. 4 ideal point)
//   labels     lg[k*label_cap + id], lnode, lparent, ledge, lpver, ldead (the
//              step in which the label was pruned, kAlive while it is not)
//   frontier   per node v: a contiguous block at fpool[fbase[v]] of capacity
//              fcap[v]: costs [k*cap + i] then label ids [d*cap + i]; fcount[v]
//              live entries (alpha(v) = G_OP(v) u G_CL(v), Sec. 3)
//   OPEN       two unsorted arrays of 64-bit keys (F[0] << 32 | F[1]) with
//              label ids beside them (the step's OPEN and the next one), and a
//              histogram of each by lexicographic cell of (F[0], F[1]) (the
//              ordered batch extraction of Algorithm 2); with OPMOS_FLAG_FIFO
//              the first array is a ring read oldest first instead
//   candidates two sets (step parity): the candidates of one window, grouped by
//              target node (the first nslots per node in slots, the rest in a
//              per-node list)
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
constexpr uint32_t kAlive = 0xFFFFFFFFu;  // ldead of a label that has not been pruned
constexpr int32_t kNil = -1;
constexpr int kNB = 4096;    // histogram bins of one OPEN array (the last one collects the rest)
constexpr int kSub = 256;    // F[1] cells per F[0] bucket; a bin is 2^s2 consecutive cells
constexpr unsigned kChunk = 32;       // OPEN entries per extraction work item
constexpr unsigned kRankQ = 1024;     // P entries per rank work item of an index rebuild
constexpr unsigned kPSMax = 32768;    // largest P indexed by the sorted snapshot
// candidates x frontier entries from which a node's merge takes a whole block:
// lower for small windows (a step is short, its longest one-warp merge sets
// its length), higher for large windows and batches (block merges are most
// of the work)
constexpr unsigned kHeavyWorkSmallWindow = 512;
constexpr unsigned kHeavyWork = 2048;
constexpr unsigned kSmallWindow = 16384;
constexpr unsigned kHeavyCands = 32;      // ... and so are nodes reached by more candidates in a step
// A block merge whose candidates x frontier entries exceed the part work is
// split into parts (up to kPartsMax, each a whole block), each part holding
// at least kPartCands candidates when the candidates are split; the part
// work is larger on the wide grid, whose blocks are three to an SM.
constexpr unsigned kPartWork = 1u << 17;
constexpr unsigned kPartWorkWide = 1u << 18;
constexpr unsigned kPartsMax = 16;
constexpr unsigned kPartCands = 64;
constexpr unsigned kPartPruned = 1u << 16;  // added to a node's part counter by a part that pruned
constexpr unsigned kHeavyBusy = 0xFFFFFFFFu;  // hflag while the node is being listed
constexpr unsigned kNodeSlots = 64;       // candidate slots per node and step in batch mode
constexpr unsigned kNodeSlotsGrid = 128;  // ... for a single query (whole-grid search)
// Lists per node for the candidates beyond the slots (log2): the lanes of a
// warp walk them side by side, so gathering k of them costs about
// k / 2^lsub dependent loads instead of k.
constexpr unsigned kLSubBatch = 3;
constexpr unsigned kLSubGrid = 5;

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
  S_TSEL,     // device ns, leader's view: window selection and step control
  S_TWORK,    // merge of window i overlapped with extraction + expansion of window i+1
  S_TSYNC,    // end of step: histogram flush and grid barrier wait
  S_TOUT,     // output
  S_GOALINS,  // goal labels accepted into P during the search (P log length)
  S_OSCAN,    // OPEN entries read by the extraction scans
  S_OKEEP,    // OPEN entries copied to the next step's OPEN array
  S_OVF,      // candidates beyond a node's slots (merged through the node's list)
  S_MAXH,     // sum over steps of the longest heavy (block) merge of the step, ns
  S_MAXL,     // ... of the longest light (warp) merge
  S_MAXX,     // ... of the longest extraction work item
  S_NHEAVY,   // heavy merges
  S_MAXNC,    // sum over steps of the most candidates a block-merged node of the step had
  S_MAXF,     // ... of the largest frontier a block-merged node of the step had
  S_SUMH,     // summed durations of block merges (one block each), ns
  S_SUML,     // ... of one-warp merges (one warp each)
  S_SUMX,     // ... of extraction work items (one warp each)
  kNStat
};

// Two shapes of the single-query grid: one 512-thread block per SM for short
// steps (windows below kSmallWindow), three 256-thread blocks per SM for large
// windows, where block merges are most of a step and the merges of three
// blocks overlap on one SM (registers are capped at 85 a thread then, and
// some spill; two blocks with 128 registers were 9% slower, four with 64
// no faster).
constexpr unsigned kGridThreads = 512;
constexpr unsigned kGridWideThreads = 256;
constexpr unsigned kGridWideBlocksPerSM = 3;

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

// Counters of one search step i, kept in a ring of three indexed by i % 3.
// They are written during step i-1 (the OPEN array, window and candidates
// step i works on are produced then) and read during step i; step i clears
// the slot of step i+2.
struct CycleCtl {
  Hot<unsigned> open_count;         // entries of step i's OPEN array (FIFO: the ring's tail)
  Hot<unsigned long long> min_key;  // smallest key among the entries carried over by extraction
  Hot<unsigned> win_count;          // labels of window i
  Hot<unsigned> win_min;            // smallest F[0] among them
  Hot<unsigned> win_max;            // largest F[0] among them
  Hot<unsigned> cand_count;         // candidates of window i (merged in step i)
  Hot<unsigned> touched_count;      // nodes they reach with a small frontier (one warp each)
  Hot<unsigned> heavy_count;        // ... with a large frontier (one block each)
  Hot<unsigned> work_next;          // dynamic claims: index-rank items, light merges, extraction chunks
  Hot<unsigned> heavy_next;         // dynamic claims of heavy merges (parts first)
  Hot<unsigned> part_count;         // parts of split heavy merges listed in xpart
  Hot<unsigned> f1lo;               // F[1] range of the carried entries the histogram's bins cover
  Hot<unsigned> f1hi;
  Hot<unsigned> plen;               // P-log length every reader uses in step i
  Hot<unsigned> lbase;              // labels that existed when step i began
  unsigned win_min_prev;            // win_min of window i-1
  unsigned head;                    // FIFO: the ring position window i+1 starts at (0 otherwise)
  unsigned tmax[5];                 // longest heavy merge, light merge, extraction item of step i (ns);
                                    // most candidates and largest frontier of a heavy merge
};

// Bins of one OPEN array's histogram: F[0] origin, F[1] origin and shift,
// F[0] bucket width, cells per bin (2^s2).
struct BinLimits {
  uint32_t b0, b1, s1, delta, s2;
};

// The P index as one step sees it (a pair indexed by step parity; step i
// reads entry i & 1 and writes entry (i+1) & 1).
struct PIdx {
  unsigned cur, count, mark, ntiles;  // live buffer, entries (the log prefix [0, mark)), tiles
  unsigned state;                     // rebuild in progress: 0 none, 1 rank, 2 scatter, 3 tiles
  unsigned nb, k;                     // its target buffer and log prefix
  unsigned shift[3];                  // per-objective shifts balancing the Z-order
};

// Per-query control block (global memory).
struct QCtl {
  unsigned error;
  unsigned done;
  unsigned step;
  unsigned res_count;
  unsigned res_status;
  unsigned pad0;
  unsigned long long res_off;    // costs (count*d) then path offsets (count+1)
  unsigned long long res_path;   // nodes (total) then arc ids (total - count)
  unsigned long long res_total;  // total path nodes
  unsigned long long t_start;
  unsigned long long stats[kNStat];
  PIdx pidx[2];
  BinLimits bins[3];             // bins of step i's histogram at bins[i % 3]
  CycleCtl cyc[3];
  Hot<unsigned> n_labels;
  Hot<unsigned> plog_len;        // the P log's length (written by the goal node's merge only)
  Hot<unsigned> fifo_tail;       // FIFO: ring positions handed out so far
  Hot<unsigned long long> f_words;
  Hot<unsigned> bar_count;
  Hot<unsigned> bar_gen;
};

// The candidates of one window, grouped by target node.
struct CandSet {
  uint32_t* ncand;     // n+1: candidates that reached the node
  int32_t* cslot;      // (n+1) * nslots: the first nslots of them
  int32_t* node_head;  // (n+1) << lsub: the rest, in 2^lsub lists per node linked by cnext (the
                       // j-th candidate beyond the slots joins list j mod 2^lsub)
  uint32_t* hflag;     // n+1: 0, or h + 1 once the node is listed as the h-th heavy node (merged by
                       // whole blocks), kHeavyBusy while it is being listed
  uint32_t* hcnt;      // n+1: parts of a split block merge finished so far (low 16 bits), plus
                       // kPartPruned for each part that pruned a frontier entry
  uint32_t* hsplit;    // cand_cap: parts the h-th heavy node's merge is split into (1: not split)
  uint32_t* xpart;     // parts of split merges, h << 4 | part (kPartsMax per heavy node at most)
  uint32_t* cflag;     // cand_cap: candidate dropped by a part of a split merge
  uint32_t* cnode;
  uint32_t* cparent;
  uint32_t* cedge;
  int32_t* cnext;
  uint32_t* cg;        // d * cand_cap
  uint32_t* touched;   // 2 * cand_cap: every node reached from the front, block-merged ones from the back
};

// Pointers into one query's arena (one slot).
struct QArena {
  uint64_t* fbase;     // n+1
  uint32_t* fcount;    // n+1
  uint32_t* fcap;      // n+1
  CandSet cs[2];
  uint32_t* lg;        // d * label_cap
  uint32_t* lnode;
  uint32_t* lparent;
  uint32_t* ledge;
  uint32_t* lpver;     // P-log length at the label's last F-against-P test
  uint32_t* ldead;     // step in which the label was pruned, kAlive if never
  uint32_t* fpool;
  uint64_t* okey[2];   // OPEN keys (F0 << 32 | F1)
  uint32_t* oid[2];    // OPEN label ids
  uint32_t* ps[2];     // P index: d * plog_cap costs, Z-order
  uint32_t* pst[2];    // P index tile minima: d * (plog_cap / 32 + 1)
  uint32_t* prank;     // kPSMax: ranks of a rebuild in progress
  uint32_t* plog;      // d * plog_cap
  uint32_t* hist;      // 3 * kNB (step i: hist + (i % 3) * kNB)
  uint32_t label_cap;
  uint32_t open_cap;
  uint32_t win_cap;
  uint32_t cand_cap;
  uint32_t plog_cap;
  uint32_t pad;
  unsigned long long fpool_words;
  uint32_t nslots;     // candidate slots per node and step (the rest go to the node's lists)
  uint32_t lsub;       // log2 of the lists per node
  uint32_t kparts;     // most parts a block merge is split into (1: never split)
  uint32_t xcap;       // entries of each candidate set's xpart
};

struct QParams {
  uint32_t start, goal;
  const uint32_t* h;      // qd * n (objective k of node v at h[k*n + v])
  uint32_t window;        // target W
  uint32_t lanes;         // lanes per label
  uint32_t delta;         // F[0] bucket width
  uint32_t tile;          // frontier growth granule
  uint32_t label_budget;  // max labels (<= label_cap)
  uint32_t flags;
  uint32_t qd;            // objectives the query uses (<= the kernel's D; the rest read as 0)
  uint32_t ps_grow;       // the P index is rebuilt once the log outgrows it by 32 + count >> ps_grow
  uint32_t heavy_work;    // candidates x frontier entries from which a node is merged by a whole block
  uint32_t part_work;     // ... per part of a split block merge
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
  static constexpr bool kSplitMerges = true;  // block merges may be split into parts
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
