// Host-visible declarations shared by the search kernels and the C ABI layer.
#pragma once

#include "opmos_dev.cuh"

namespace opmos {

// Multi-query kernel (batch and serving) --------------------------------------
constexpr unsigned kMultiThreads = 256;  // threads per block
constexpr unsigned kMaxSlots = 1024;     // concurrent queries
enum SlotState : unsigned {
  SL_FREE = 0, SL_INIT = 1, SL_RUN = 2, SL_OUT1 = 3, SL_OUT2 = 4, SL_OUT3 = 5, SL_OUT4 = 6,
  SL_HELD = 7  // result written, waiting for the host to collect it (serving)
};

struct MSlot {     // one concurrent query: its arena and current parameters
  QArena A;
  QParams P;
  GraphDev G;
  OutPool O;       // where its result goes (shared in batch mode, its own when serving)
  unsigned d, state, qidx, pad;  // d: objectives the query uses (<= the kernel's)
};

struct MQuery {    // a queued query
  uint32_t graph, start, goal, d;
  const uint32_t* h;  // d * n heuristic toward goal (device)
};

struct MCtl {      // grid-wide control of the multi-query kernel
  unsigned bar_count, bar_gen, error, done;
  unsigned q_next, iter, qcap, hold;  // hold: keep slots until the host releases them
};

// Host control words (host-mapped memory when serving): [0] queries queued
// so far, [1] closing (no more queries will come), [2 + slot] release flag.
enum { HC_TAIL = 0, HC_CLOSING = 1, HC_RELEASE = 2 };

// Result descriptor of one query, written by the team leader at the end.
// Output words (in the OutPool): at off, count*d costs (lexicographic) then
// count+1 path offsets; at path, total node ids then total-count arc ids.
struct QResult {
  unsigned status;
  unsigned slot;    // slot whose output pool holds the result
  unsigned count;
  unsigned pad;
  unsigned long long off;
  unsigned long long path;
  unsigned long long total;
  unsigned long long labels;
  unsigned long long f_words;
  unsigned long long stats[kNStat];
};

// Kernel launchers of one objective count D (search_inst.cu instantiates them,
// one object per group of D values); the kernel of a query with qd < D
// objectives reads objectives qd..D-1 as 0.
// wide: the grid of three 256-thread blocks per SM (large windows) instead
// of one 512-thread block per SM.
template <int D>
cudaError_t launch_grid(const GraphDev& G, const QArena& A, QCtl* C, const QParams& P, const OutPool& O,
                        QResult* R, bool wide, unsigned blocks, cudaStream_t s);
template <int D>
int grid_occupancy(bool wide);
template <int D>
cudaError_t launch_multi_d(MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue, unsigned* hctl,
                           const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M, unsigned blocks,
                           cudaStream_t s);
template <int D>
int multi_occupancy_d();

// Dispatch on the objective count, 1..OPMOS_MAX_D (search_dispatch.cu).
cudaError_t launch_search_grid(unsigned d, const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                               const OutPool& O, QResult* R, bool wide, unsigned blocks, cudaStream_t s);
int search_occupancy(unsigned d, bool wide);
cudaError_t launch_multi(unsigned d, MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue,
                         unsigned* hctl, const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M,
                         unsigned blocks, cudaStream_t s);
int multi_occupancy(unsigned d);

// Ideal-point heuristic jobs: h_out[v] = shortest v->goal distance under
// objective k (Sec. 4), one thread block per job.
struct HJob {
  uint32_t goal, k;
  uint32_t* h_out;  // n entries
};
// Sets the calling thread's opmos_last_error() message; returns code.
int record_error(int code, const char* msg);

cudaError_t launch_heuristic(const GraphDev& G, const HJob* jobs, unsigned njobs, uint32_t* scratch,
                             size_t scratch_words_per_block, unsigned blocks, const uint32_t* delta,
                             unsigned* next_job, unsigned* err, cudaStream_t s);

}  // namespace opmos
