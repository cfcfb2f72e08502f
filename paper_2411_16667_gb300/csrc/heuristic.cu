// Ideal-point heuristic (Sec. 4; the "heuristics H" input of Algorithms 1-2):
// h_k(v) = length of the shortest v -> goal path under objective k alone.
//
// One thread block computes one (goal, k) pair by a bucketed label-correcting
// single-source shortest-path search from the goal over the reversed arcs
// (near/far variant of delta-stepping): nodes whose tentative distance is
// below the current threshold are relaxed in rounds until none improves, the
// threshold then jumps to the smallest pending distance plus delta. Worklists
// are deduplicated with per-node flag bits so each holds at most n entries.
// The distances are exact shortest distances (label-correcting converges to
// them); unreachable nodes keep 0xFFFFFFFF.
//
// Scratch per resident block: near, next, far, far2 (n each) and flags (n).
#include "opmos_dev.cuh"
#include "search.cuh"

namespace opmos {

namespace {

constexpr unsigned kHeurThreads = 512;

__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }

__global__ void __launch_bounds__(kHeurThreads)
    heuristic_kernel(GraphDev G, const HJob* jobs, unsigned njobs, uint32_t* scratch, size_t spb,
                     const uint32_t* delta, unsigned* next_job, unsigned* err) {
  __shared__ unsigned s_job, s_near_n, s_next_n, s_far_n, s_far2_n, s_min;
  const unsigned n = G.n, tid = threadIdx.x, nt = blockDim.x;
  uint32_t* base = scratch + (size_t)blockIdx.x * spb;
  uint32_t* bufA = base;
  uint32_t* bufB = base + n;
  uint32_t* farA = base + 2 * (size_t)n;
  uint32_t* farB = base + 3 * (size_t)n;
  uint32_t* flags = base + 4 * (size_t)n;
  for (;;) {
    if (tid == 0) s_job = atomicAdd(next_job, 1u);
    __syncthreads();
    const unsigned job = s_job;
    __syncthreads();
    if (job >= njobs) return;
    const unsigned k = jobs[job].k, goal = jobs[job].goal;
    uint32_t* dist = jobs[job].h_out;
    const uint32_t* rc = G.rcost + (size_t)k * G.m;
    const unsigned long long dk = delta[k] ? delta[k] : 1u;
    for (unsigned v = tid; v < n; v += nt) {
      dist[v] = kInf;
      flags[v] = 0;
    }
    __syncthreads();
    if (tid == 0) {
      dist[goal] = 0;
      bufA[0] = goal;
      flags[goal] = 1;
      s_near_n = 1;
      s_far_n = 0;
    }
    __syncthreads();
    uint32_t* near = bufA;
    uint32_t* next = bufB;
    uint32_t* far = farA;
    uint32_t* far2 = farB;
    unsigned long long thr = dk;     // near holds distances < thr
    unsigned long long settled = 0;  // distances < settled are final
    unsigned long long rounds = 0;
    const unsigned long long max_rounds = 64ull * n + 4096;
    for (;;) {
      while (s_near_n > 0) {
        const unsigned nn = s_near_n;
        if (++rounds > max_rounds) {
          if (tid == 0) atomicCAS(err, 0u, (unsigned)OPMOS_ERR_TIMEOUT);
          return;
        }
        for (unsigned i = tid; i < nn; i += nt) atomicAnd(&flags[near[i]], ~1u);
        if (tid == 0) s_next_n = 0;
        __syncthreads();
        for (unsigned i = tid; i < nn; i += nt) {
          const uint32_t u = near[i];
          const uint32_t du = ld_cg(&dist[u]);
          const uint32_t j0 = __ldg(G.rrowptr + u), j1 = __ldg(G.rrowptr + u + 1);
          for (uint32_t j = j0; j < j1; ++j) {
            const uint32_t w = __ldg(G.rsrc + j);
            const uint32_t nd = du + __ldg(rc + j);
            if (nd < ld_cg(&dist[w])) {
              const uint32_t old = atomicMin(&dist[w], nd);
              if (nd < old) {
                if (nd < thr) {
                  if (!(atomicOr(&flags[w], 1u) & 1u)) next[atomicAdd(&s_next_n, 1u)] = w;
                } else {
                  if (!(atomicOr(&flags[w], 2u) & 2u)) far[atomicAdd(&s_far_n, 1u)] = w;
                }
              }
            }
          }
        }
        __syncthreads();
        uint32_t* t = near;
        near = next;
        next = t;
        if (tid == 0) s_near_n = s_next_n;
        __syncthreads();
      }
      settled = thr;
      const unsigned fn = s_far_n;
      if (fn == 0) break;
      if (tid == 0) s_min = kInf;
      __syncthreads();
      for (unsigned i = tid; i < fn; i += nt) {
        const uint32_t dw = ld_cg(&dist[far[i]]);
        if (dw >= settled) atomicMin(&s_min, dw);
      }
      __syncthreads();
      const unsigned mn = s_min;
      if (mn == kInf) break;
      thr = (unsigned long long)mn + dk;
      if (tid == 0) {
        s_near_n = 0;
        s_far2_n = 0;
      }
      __syncthreads();
      for (unsigned i = tid; i < fn; i += nt) {
        const uint32_t w = far[i];
        const uint32_t dw = ld_cg(&dist[w]);
        if (dw < settled) {
          flags[w] &= ~2u;  // already final
        } else if (dw < thr) {
          flags[w] = 1u;
          near[atomicAdd(&s_near_n, 1u)] = w;
        } else {
          flags[w] = 2u;
          far2[atomicAdd(&s_far2_n, 1u)] = w;
        }
      }
      __syncthreads();
      uint32_t* t = far;
      far = far2;
      far2 = t;
      if (tid == 0) s_far_n = s_far2_n;
      __syncthreads();
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_heuristic(const GraphDev& G, const HJob* jobs, unsigned njobs, uint32_t* scratch,
                             size_t scratch_words_per_block, unsigned blocks, const uint32_t* delta,
                             unsigned* next_job, unsigned* err, cudaStream_t s) {
  heuristic_kernel<<<blocks, kHeurThreads, 0, s>>>(G, jobs, njobs, scratch, scratch_words_per_block, delta,
                                                    next_job, err);
  return cudaGetLastError();
}

}  // namespace opmos
