// Kernel instantiations for the objective counts OPMOS_D_FIRST..OPMOS_D_LAST.
// The build compiles this file once per group of counts (in parallel), so
// each object holds the single-query and multi-query kernels of a few D.
#include "search_impl.cuh"

#if !defined(OPMOS_D_FIRST) || !defined(OPMOS_D_LAST)
#error "compile with -DOPMOS_D_FIRST=a -DOPMOS_D_LAST=b (1 <= a <= b <= OPMOS_MAX_D)"
#endif

namespace opmos {

#define OPMOS_INSTANTIATE(D)                                                                                     \
  template cudaError_t launch_grid<D>(const GraphDev&, const QArena&, QCtl*, const QParams&, const OutPool&,    \
                                      QResult*, bool, unsigned, cudaStream_t);                                   \
  template int grid_occupancy<D>(bool);                                                                         \
  template cudaError_t launch_multi_d<D>(MSlot*, QCtl*, unsigned, const MQuery*, unsigned*, const GraphDev*,     \
                                         QResult*, unsigned*, MCtl*, unsigned, cudaStream_t);                   \
  template int multi_occupancy_d<D>();

#define OPMOS_IN_GROUP(D) (OPMOS_D_FIRST <= (D) && (D) <= OPMOS_D_LAST)
#if OPMOS_IN_GROUP(1)
OPMOS_INSTANTIATE(1)
#endif
#if OPMOS_IN_GROUP(2)
OPMOS_INSTANTIATE(2)
#endif
#if OPMOS_IN_GROUP(3)
OPMOS_INSTANTIATE(3)
#endif
#if OPMOS_IN_GROUP(4)
OPMOS_INSTANTIATE(4)
#endif
#if OPMOS_IN_GROUP(5)
OPMOS_INSTANTIATE(5)
#endif
#if OPMOS_IN_GROUP(6)
OPMOS_INSTANTIATE(6)
#endif
#if OPMOS_IN_GROUP(7)
OPMOS_INSTANTIATE(7)
#endif
#if OPMOS_IN_GROUP(8)
OPMOS_INSTANTIATE(8)
#endif
#if OPMOS_IN_GROUP(9)
OPMOS_INSTANTIATE(9)
#endif
#if OPMOS_IN_GROUP(10)
OPMOS_INSTANTIATE(10)
#endif
#if OPMOS_IN_GROUP(11)
OPMOS_INSTANTIATE(11)
#endif
#if OPMOS_IN_GROUP(12)
OPMOS_INSTANTIATE(12)
#endif
#if OPMOS_IN_GROUP(13)
OPMOS_INSTANTIATE(13)
#endif
#if OPMOS_IN_GROUP(14)
OPMOS_INSTANTIATE(14)
#endif
#if OPMOS_IN_GROUP(15)
OPMOS_INSTANTIATE(15)
#endif
#if OPMOS_IN_GROUP(16)
OPMOS_INSTANTIATE(16)
#endif

}  // namespace opmos
