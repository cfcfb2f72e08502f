// Dispatch of the search kernels on the objective count (1..OPMOS_MAX_D); the
// kernels themselves are instantiated in search_inst.cu.
#include "search.cuh"

namespace opmos {

static_assert(OPMOS_MAX_D == 16, "the dispatch below lists 1..16");

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
    case 9: return CALL(9);       \
    case 10: return CALL(10);     \
    case 11: return CALL(11);     \
    case 12: return CALL(12);     \
    case 13: return CALL(13);     \
    case 14: return CALL(14);     \
    case 15: return CALL(15);     \
    case 16: return CALL(16);     \
    default: break;               \
  }

cudaError_t launch_search_grid(unsigned d, const GraphDev& G, const QArena& A, QCtl* C, const QParams& P,
                               const OutPool& O, QResult* R, bool wide, unsigned blocks, cudaStream_t s) {
#define CALL(D) launch_grid<D>(G, A, C, P, O, R, wide, blocks, s)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

int search_occupancy(unsigned d, bool wide) {
#define CALL(D) grid_occupancy<D>(wide)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return 0;
}

cudaError_t launch_multi(unsigned d, MSlot* slots, QCtl* ctls, unsigned nslots, const MQuery* queue,
                         unsigned* hctl, const GraphDev* graphs, QResult* results, unsigned* done_flags, MCtl* M,
                         unsigned blocks, cudaStream_t s) {
#define CALL(D) launch_multi_d<D>(slots, ctls, nslots, queue, hctl, graphs, results, done_flags, M, blocks, s)
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

int multi_occupancy(unsigned d) {
#define CALL(D) multi_occupancy_d<D>()
  OPMOS_DISPATCH_D(d, CALL)
#undef CALL
  return 0;
}

}  // namespace opmos
