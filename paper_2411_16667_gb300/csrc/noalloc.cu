// opmos_heuristic_noalloc: the ideal-point heuristic without any device
// allocation inside the call.
//
// Who needs it: callers that cannot call cudaMalloc while they run -- for
// example a process whose device memory is entirely reserved up front by its
// own pool allocator (an allocation outside that pool fails or breaks its
// accounting), or a latency-sensitive service that must not pay for the
// allocation and the implicit device synchronisation cudaMalloc/cudaFree can
// bring. They allocate the output once, elsewhere, and pass it in.
//
// How: the heuristic kernel of heuristic.cu is launched unchanged, but its
// worklists, job table and counters live in one file-scope __device__ array
// (g_noalloc_scratch, kNoAllocWords words, about 10.5 MB, held by every device
// that loads this library until the process exits). Its device address is
// looked up once per device with cudaGetSymbolAddress -- the host-side name of
// the array is only a stand-in and must never be passed to a kernel.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <new>

#include "graph.cuh"
#include "opmos.h"
#include "search.cuh"

using namespace opmos;

namespace {

constexpr uint32_t kNoAllocMaxNodes = 1u << 18;  // largest graph (nodes) served
constexpr unsigned kNoAllocBlocks = 2;           // thread blocks sharing the jobs
constexpr size_t kNoAllocCtrWords = 64;          // [0] next job, [1] error code
constexpr size_t kNoAllocJobWords = 64;          // up to OPMOS_MAX_D HJob records
constexpr size_t kNoAllocBlockWords = 5ull * kNoAllocMaxNodes + 64;
constexpr size_t kNoAllocWords = kNoAllocCtrWords + kNoAllocJobWords + kNoAllocBlocks * kNoAllocBlockWords;
static_assert(sizeof(HJob) * OPMOS_MAX_D <= kNoAllocJobWords * 4, "job table does not fit");

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];  // device address of g_noalloc_scratch, per device ordinal

// Reported through opmos_last_error(), like every other entry point.
int noalloc_fail(int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return record_error(code, buf);
}

// No C++ exception crosses the C ABI (see opmos.h).
template <class F>
int noalloc_guarded(const char* what, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return noalloc_fail(OPMOS_ERR_OUT_OF_MEMORY, "%s: host allocation failed", what);
  } catch (...) {
    return noalloc_fail(OPMOS_ERR_CUDA, "%s: unexpected exception", what);
  }
}

// One-time set-up per device (with that device current): the device address
// of the scratch array.
int scratch_address(int dev, uint32_t** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= 64) return noalloc_fail(OPMOS_ERR_CUDA, "device ordinal %d out of range", dev);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(OPMOS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    }
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<uint32_t*>(g_noalloc_addr[dev]);
  return OPMOS_OK;
}

__global__ void fill_jobs_kernel(HJob* jobs, uint32_t goal, uint32_t d, uint32_t* h_out, uint32_t n) {
  const uint32_t k = threadIdx.x;
  if (k < d) jobs[k] = HJob{goal, k, h_out + (size_t)k * n};
}

}  // namespace

extern "C" {

int opmos_heuristic_noalloc(const opmos_graph* g, uint32_t goal, uint32_t d_used, uint32_t* h_out_device,
                            void* stream) {
  return noalloc_guarded("opmos_heuristic_noalloc", [&]() -> int {
    if (!g || !h_out_device) return noalloc_fail(OPMOS_ERR_INVALID_ARG, "NULL graph or output");
    if (goal >= g->n) return noalloc_fail(OPMOS_ERR_INVALID_ARG, "goal %u >= n = %u", goal, g->n);
    const uint32_t D = d_used ? d_used : g->d;
    if (D > g->d) return noalloc_fail(OPMOS_ERR_INVALID_ARG, "d_used %u > d %u", D, g->d);
    if (g->n > kNoAllocMaxNodes)
      return noalloc_fail(OPMOS_ERR_CAPACITY,
                          "graph has %u nodes; the allocation-free heuristic handles at most %u "
                          "(use opmos_heuristic)",
                          g->n, kNoAllocMaxNodes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(OPMOS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    uint32_t* base = nullptr;
    if (int rc = scratch_address(dev, &base)) return rc;
    unsigned* ctr = base;
    HJob* jobs = reinterpret_cast<HJob*>(base + kNoAllocCtrWords);
    uint32_t* work = base + kNoAllocCtrWords + kNoAllocJobWords;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the counters must restart
    // at zero (worklists and flags are re-initialised by the kernel itself)
    e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return noalloc_fail(OPMOS_ERR_CUDA, "clear counters: %s", cudaGetErrorString(e));
    fill_jobs_kernel<<<1, 32, 0, s>>>(jobs, goal, D, h_out_device, g->n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(OPMOS_ERR_CUDA, "job table: %s", cudaGetErrorString(e));
    const unsigned blocks = D < kNoAllocBlocks ? D : kNoAllocBlocks;
    e = launch_heuristic(g->dev, jobs, D, work, kNoAllocBlockWords, blocks, g->delta, ctr, ctr + 1, s);
    if (e != cudaSuccess) return noalloc_fail(OPMOS_ERR_CUDA, "heuristic launch: %s", cudaGetErrorString(e));
    unsigned err = 0;
    e = cudaMemcpyAsync(&err, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(OPMOS_ERR_CUDA, "heuristic kernel: %s", cudaGetErrorString(e));
    if (err) return noalloc_fail((int)err, "heuristic kernel reported error %u", err);
    return OPMOS_OK;
  });
}

}  // extern "C"
