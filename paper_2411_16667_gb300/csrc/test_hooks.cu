// Test hooks (include/opmos_test.h): single routines of a search step run on
// caller-given inputs, through the same device code the search kernels use.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "opmos_test.h"
#include "search_impl.cuh"

using namespace opmos;
using namespace opmos::detail;

namespace {

int hook_fail(int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return record_error(code, buf);
}

// Device buffer freed on scope exit.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

template <class T>
T* take(char*& p, size_t count) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  a = (a + 255) / 256 * 256;
  p = reinterpret_cast<char*>(a + count * sizeof(T));
  return reinterpret_cast<T*>(a);
}

// One node (node 0) merged as in step 0: one warp or the whole block.
template <int D>
__global__ void __launch_bounds__(kGridThreads, 1) merge_hook_kernel(GraphDev G, QArena A, QCtl* C, QParams P,
                                                                     OutPool O, unsigned lbase, unsigned block) {
  __shared__ Shared S;
  Search<D> X(G, A, C, P, O, S);
  X.cyc = 0;
  X.psnap = 0;
  X.lbase = lbase;
  X.bpn = BinParams{0u, 0u, 0u, 1u, 0u};
  if (threadIdx.x == 0) {
    S.pd = PIdx{};
    for (int i = 0; i < kNB; ++i) S.hist[i] = 0;
  }
  __syncthreads();
  if (block >= 2) {  // a merge split into `block` parts, one after the other (the last one finishes)
    for (unsigned r = 0; r < block; ++r) {
      X.merge_part(0u, r, block, C->cyc[1]);
      __syncthreads();
    }
  } else if (block) {
    X.merge_heavy(0u, C->cyc[1]);
  } else if (threadIdx.x < 32) {
    X.merge_node(0u, C->cyc[1]);
  }
}

template <int D>
int merge_hook(uint32_t nfront, const uint32_t* front, uint32_t ncand, const uint32_t* cand, const uint32_t* arc,
               uint32_t block, uint32_t slots, uint32_t lsub, uint32_t* out_cost, uint32_t* out_origin,
               uint32_t* out_count) {
  const uint32_t n = 1;  // node 0, and node 1 standing for P
  const uint32_t label_cap = nfront + ncand + 64, cand_cap = ncand + 64, open_cap = ncand + 64;
  const uint32_t fcap0 = (nfront + 31) / 32 * 32 + 32;
  const size_t fpool_words = (size_t)(D + 1) * (fcap0 + 4 * (nfront + ncand) + 256);
  size_t bytes = 64 * 256 + sizeof(QCtl) + (size_t)D * 4 * (n + 1) + 8 * 4 * (n + 1) +
                 2 * (4 * (n + 1) * (3 + slots + (1u << lsub))) +
                 2 * (size_t)cand_cap * (32 + 4 * D) + 2 * 4 * (n + 1) + (size_t)label_cap * (4 * D + 20) + fpool_words * 4 +
                 2 * (size_t)open_cap * 12 + 3 * kNB * 4 + kPSMax * 4 + 64 * 4 * D * 6;
  DevBuf mem;
  cudaError_t e = cudaMalloc(&mem.p, bytes);
  if (e != cudaSuccess) return hook_fail(OPMOS_ERR_OUT_OF_MEMORY, "test hook: %s", cudaGetErrorString(e));
  char* base = static_cast<char*>(mem.p);
  char* p = base;
  QCtl* C = take<QCtl>(p, 1);
  uint32_t* h = take<uint32_t>(p, (size_t)D * (n + 1));
  QArena A{};
  A.fbase = take<uint64_t>(p, n + 1);
  A.fcount = take<uint32_t>(p, n + 1);
  A.fcap = take<uint32_t>(p, n + 1);
  for (int b = 0; b < 2; ++b) {
    CandSet& cs = A.cs[b];
    cs.ncand = take<uint32_t>(p, n + 1);
    cs.node_head = take<int32_t>(p, (size_t)(n + 1) << lsub);
    cs.hflag = take<uint32_t>(p, n + 1);
    cs.hcnt = take<uint32_t>(p, n + 1);
    cs.hsplit = take<uint32_t>(p, cand_cap);
    cs.cflag = take<uint32_t>(p, cand_cap);
    cs.cslot = take<int32_t>(p, (size_t)(n + 1) * slots);
    cs.cnode = take<uint32_t>(p, cand_cap);
    cs.cparent = take<uint32_t>(p, cand_cap);
    cs.cedge = take<uint32_t>(p, cand_cap);
    cs.cnext = take<int32_t>(p, cand_cap);
    cs.touched = take<uint32_t>(p, 2 * (size_t)cand_cap);
    cs.cg = take<uint32_t>(p, (size_t)cand_cap * D);
  }
  A.lg = take<uint32_t>(p, (size_t)label_cap * D);
  A.lnode = take<uint32_t>(p, label_cap);
  A.lparent = take<uint32_t>(p, label_cap);
  A.ledge = take<uint32_t>(p, label_cap);
  A.lpver = take<uint32_t>(p, label_cap);
  A.ldead = take<uint32_t>(p, label_cap);
  A.fpool = take<uint32_t>(p, fpool_words);
  for (int b = 0; b < 2; ++b) {
    A.okey[b] = take<uint64_t>(p, open_cap);
    A.oid[b] = take<uint32_t>(p, open_cap);
    A.ps[b] = take<uint32_t>(p, 64 * D);
    A.pst[b] = take<uint32_t>(p, 64 * D);
  }
  A.prank = take<uint32_t>(p, kPSMax);
  A.plog = take<uint32_t>(p, 64 * D);
  A.hist = take<uint32_t>(p, 3 * kNB);
  A.label_cap = label_cap;
  A.open_cap = open_cap;
  A.win_cap = cand_cap;
  A.cand_cap = cand_cap;
  A.plog_cap = 64;
  A.fpool_words = fpool_words;
  A.nslots = slots;
  A.lsub = lsub;
  if ((size_t)(p - base) > bytes) return hook_fail(OPMOS_ERR_CAPACITY, "test hook: layout exceeds its buffer");
  e = cudaMemset(mem.p, 0, bytes);
  // host images of what a step finds: frontier of node 0 (labels 0..nfront-1)
  // and the candidates of node 0 in set 0 (slots, then the lists)
  std::vector<uint32_t> fimg((size_t)(D + 1) * fcap0, 0), lg((size_t)label_cap * D, 0), lnode(label_cap, 0),
      lpar(label_cap, kInf), ledge(label_cap, kInf), ldead(label_cap, kAlive);
  for (uint32_t i = 0; i < nfront; ++i) {
    for (int k = 0; k < D; ++k) {
      fimg[(size_t)k * fcap0 + i] = front[(size_t)i * D + k];
      lg[(size_t)k * label_cap + i] = front[(size_t)i * D + k];
    }
    fimg[(size_t)D * fcap0 + i] = i;
  }
  std::vector<uint32_t> cnode(cand_cap, 0), cpar(cand_cap, 0), cedge(cand_cap, 0), cg((size_t)cand_cap * D, 0);
  std::vector<int32_t> cnext(cand_cap, kNil), cslot((size_t)(n + 1) * slots, kNil),
      head((size_t)(n + 1) << lsub, kNil);
  for (uint32_t j = 0; j < ncand; ++j) {
    cpar[j] = j;
    cedge[j] = arc[j];
    for (int k = 0; k < D; ++k) cg[(size_t)k * cand_cap + j] = cand[(size_t)j * D + k];
    if (j < slots) {
      cslot[j] = (int32_t)j;
    } else {  // list (j - slots) mod 2^lsub, newest first, as the expansion's exchanges leave it
      const uint32_t l = (j - slots) & ((1u << lsub) - 1u);
      cnext[j] = head[l];
      head[l] = (int32_t)j;
    }
  }
  const uint32_t ncand_v[2] = {ncand, 0};
  const uint64_t fbase0 = 0;
  const uint32_t fcount0 = nfront, fcap0v = fcap0;
  QCtl hc;
  std::memset(&hc, 0, sizeof(hc));
  hc.n_labels.v = nfront;
  hc.f_words.v = (unsigned long long)(D + 1) * fcap0;
  for (int r = 0; r < 3; ++r) {
    hc.cyc[r].min_key.v = ~0ull;
    hc.cyc[r].win_min.v = kInf;
    hc.cyc[r].f1lo.v = kInf;
  }
  auto up = [&](void* dst, const void* src, size_t b) {
    if (e == cudaSuccess && b) e = cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice);
  };
  up(C, &hc, sizeof(hc));
  up(A.fbase, &fbase0, 8);
  up(A.fcount, &fcount0, 4);
  up(A.fcap, &fcap0v, 4);
  up(A.fpool, fimg.data(), fimg.size() * 4);
  up(A.lg, lg.data(), lg.size() * 4);
  up(A.lnode, lnode.data(), lnode.size() * 4);
  up(A.lparent, lpar.data(), lpar.size() * 4);
  up(A.ledge, ledge.data(), ledge.size() * 4);
  up(A.ldead, ldead.data(), ldead.size() * 4);
  const CandSet& cs = A.cs[0];
  up(cs.ncand, ncand_v, 8);
  up(cs.node_head, head.data(), head.size() * 4);
  up(cs.cslot, cslot.data(), cslot.size() * 4);
  up(cs.cnode, cnode.data(), cnode.size() * 4);
  up(cs.cparent, cpar.data(), cpar.size() * 4);
  up(cs.cedge, cedge.data(), cedge.size() * 4);
  up(cs.cnext, cnext.data(), cnext.size() * 4);
  up(cs.cg, cg.data(), cg.size() * 4);
  std::vector<int32_t> nil1((size_t)(n + 1) << lsub, kNil);
  up(A.cs[1].node_head, nil1.data(), nil1.size() * 4);
  if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook upload: %s", cudaGetErrorString(e));
  GraphDev G{};
  G.n = n;
  G.d = D;
  QParams P{};
  P.goal = n;  // no real goal: node 0 is an ordinary node
  P.h = h;
  P.window = 1;
  P.lanes = 8;
  P.delta = 1;
  P.tile = 32;
  P.label_budget = label_cap;
  P.qd = D;
  P.ps_grow = 6;
  P.heavy_work = kHeavyWork;
  P.part_work = kPartWork;
  OutPool O{nullptr, 0, nullptr};
  merge_hook_kernel<D><<<1, kGridThreads>>>(G, A, C, P, O, nfront, block);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook kernel: %s", cudaGetErrorString(e));
  unsigned err = 0;
  uint64_t fb = 0;
  uint32_t fc = 0, cap = 0;
  e = cudaMemcpy(&err, &C->error, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&fb, A.fbase, 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&fc, A.fcount, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&cap, A.fcap, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook download: %s", cudaGetErrorString(e));
  if (err) return hook_fail((int)err, "test hook: the merge reported error %u", err);
  std::vector<uint32_t> blk((size_t)(D + 1) * cap);
  e = cudaMemcpy(blk.data(), A.fpool + fb, blk.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(lpar.data(), A.lparent, lpar.size() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook download: %s", cudaGetErrorString(e));
  if (fc > nfront + ncand) return hook_fail(OPMOS_ERR_CUDA, "test hook: frontier grew past its inputs");
  for (uint32_t i = 0; i < fc; ++i) {
    for (int k = 0; k < D; ++k) out_cost[(size_t)i * D + k] = blk[(size_t)k * cap + i];
    const uint32_t id = blk[(size_t)D * cap + i];
    out_origin[i] = id < nfront ? id : nfront + lpar[id];
  }
  *out_count = fc;
  return OPMOS_OK;
}

// The window of step 1 over OPEN_1 = the given entries (labels at a node
// without out-arcs, heuristic 0, two objectives).
__global__ void window_hist_kernel(QArena A, unsigned n, BinParams bp, unsigned* hist) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (A.ldead[A.oid[1][i]] == kAlive) atomicAdd(&hist[bin_of(A.okey[1][i], bp)], 1u);
}

__global__ void __launch_bounds__(kGridThreads, 1) window_hook_kernel(GraphDev G, QArena A, QCtl* C, QParams P,
                                                                      OutPool O, unsigned n, BinParams bp,
                                                                      unsigned* bstar) {
  __shared__ Shared S;
  Search<2> X(G, A, C, P, O, S);
  X.cyc = 1;
  X.psnap = 0;
  X.lbase = n;
  X.bpn = bp;
  if (threadIdx.x == 0) S.pd = PIdx{};
  __syncthreads();
  X.select_window(A.hist + 1 * kNB);  // leaves S.hist empty for the extraction
  if (threadIdx.x == 0) *bstar = S.bstar;
  const unsigned nchunks = (n + kChunk - 1) / kChunk;
  for (unsigned c = threadIdx.x >> 5; c < nchunks; c += blockDim.x >> 5) X.extract_chunk(c, n, bp, C->cyc[2]);
}

}  // namespace

extern "C" {

int opmos_test_merge(uint32_t d, uint32_t nfront, const uint32_t* front, uint32_t ncand, const uint32_t* cand,
                     const uint32_t* cand_arc, uint32_t block, uint32_t slots, uint32_t lists,
                     uint32_t* out_cost, uint32_t* out_origin, uint32_t* out_count) {
  try {
    if (!out_cost || !out_origin || !out_count || (nfront && !front) || (ncand && (!cand || !cand_arc)))
      return hook_fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    if (slots == 0 || slots > 4096) return hook_fail(OPMOS_ERR_INVALID_ARG, "slots must be in [1, 4096]");
    if (block > kPartsMax) return hook_fail(OPMOS_ERR_INVALID_ARG, "block must be 0..%u", kPartsMax);
    if (nfront > (1u << 20) || ncand > (1u << 20)) return hook_fail(OPMOS_ERR_INVALID_ARG, "inputs too large");
    unsigned lsub = 0;
    while ((1u << lsub) < lists && lsub < 5) ++lsub;
    if (lists == 0 || lists != (1u << lsub))
      return hook_fail(OPMOS_ERR_INVALID_ARG, "lists must be 1, 2, 4, 8, 16 or 32");
    switch (d) {
      case 1:
        return merge_hook<1>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 2:
        return merge_hook<2>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 3:
        return merge_hook<3>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 4:
        return merge_hook<4>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 5:
        return merge_hook<5>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 8:
        return merge_hook<8>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 12:
        return merge_hook<12>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      case 16:
        return merge_hook<16>(nfront, front, ncand, cand, cand_arc, block, slots, lsub, out_cost, out_origin, out_count);
      default:
        return hook_fail(OPMOS_ERR_INVALID_ARG, "d = %u has no merge test hook", d);
    }
  } catch (...) {
    return hook_fail(OPMOS_ERR_OUT_OF_MEMORY, "test hook: host allocation failed");
  }
}

int opmos_test_window(uint32_t n, const uint32_t* f0, const uint32_t* f1, const uint8_t* dead, uint32_t window,
                      const uint32_t* bins, uint8_t* taken, uint32_t* bstar) {
  try {
    if (!taken || !bstar || !bins || (n && (!f0 || !f1 || !dead))) return hook_fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    if (bins[3] == 0 || bins[2] >= 32 || bins[4] > 30 || window == 0 || n > (1u << 22))
      return hook_fail(OPMOS_ERR_INVALID_ARG, "bad window, bins or size");
    constexpr int D = 2;
    const uint32_t cap = n + 64;
    size_t bytes = 64 * 256 + sizeof(QCtl) + 4 * 2 * 3 + 4 * 3 * 16 + 2 * (size_t)cap * 12 + (size_t)cap * (4 * D + 20) +
                   3 * kNB * 4 + 2 * ((size_t)cap * (32 + 4 * D) + 4 * 3 * 44) + 64 * 4 * D * 6 + kPSMax * 4;
    DevBuf mem;
    cudaError_t e = cudaMalloc(&mem.p, bytes);
    if (e != cudaSuccess) return hook_fail(OPMOS_ERR_OUT_OF_MEMORY, "test hook: %s", cudaGetErrorString(e));
    e = cudaMemset(mem.p, 0, bytes);
    char* p = static_cast<char*>(mem.p);
    QCtl* C = take<QCtl>(p, 1);
    uint32_t* h = take<uint32_t>(p, 2 * 3);
    uint32_t* rowptr = take<uint32_t>(p, 4);
    unsigned* d_bstar = take<unsigned>(p, 1);
    QArena A{};
    A.fbase = take<uint64_t>(p, 3);
    A.fcount = take<uint32_t>(p, 3);
    A.fcap = take<uint32_t>(p, 3);
    for (int b = 0; b < 2; ++b) {
      CandSet& cs = A.cs[b];
      cs.ncand = take<uint32_t>(p, 3);
      cs.node_head = take<int32_t>(p, 3);
      cs.hflag = take<uint32_t>(p, 3);
      cs.hcnt = take<uint32_t>(p, 3);
      cs.hsplit = take<uint32_t>(p, cap);
      cs.cflag = take<uint32_t>(p, cap);
      cs.cslot = take<int32_t>(p, 3 * 32);
      cs.cnode = take<uint32_t>(p, cap);
      cs.cparent = take<uint32_t>(p, cap);
      cs.cedge = take<uint32_t>(p, cap);
      cs.cnext = take<int32_t>(p, cap);
      cs.touched = take<uint32_t>(p, 2 * (size_t)cap);
      cs.cg = take<uint32_t>(p, (size_t)cap * D);
    }
    A.lg = take<uint32_t>(p, (size_t)cap * D);
    A.lnode = take<uint32_t>(p, cap);
    A.lparent = take<uint32_t>(p, cap);
    A.ledge = take<uint32_t>(p, cap);
    A.lpver = take<uint32_t>(p, cap);
    A.ldead = take<uint32_t>(p, cap);
    for (int b = 0; b < 2; ++b) {
      A.okey[b] = take<uint64_t>(p, cap);
      A.oid[b] = take<uint32_t>(p, cap);
      A.ps[b] = take<uint32_t>(p, 64 * D);
      A.pst[b] = take<uint32_t>(p, 64 * D);
    }
    A.prank = take<uint32_t>(p, kPSMax);
    A.plog = take<uint32_t>(p, 64 * D);
    A.hist = take<uint32_t>(p, 3 * kNB);
    A.fpool = take<uint32_t>(p, 64);
    A.label_cap = cap;
    A.open_cap = cap;
    A.win_cap = cap;  // no cap on the window here: the bins alone decide
    A.cand_cap = cap;
    A.plog_cap = 64;
    A.fpool_words = 64;
    A.nslots = 32;
    if ((size_t)(p - static_cast<char*>(mem.p)) > bytes) return hook_fail(OPMOS_ERR_CAPACITY, "test hook layout");
    std::vector<uint64_t> keys(n);
    std::vector<uint32_t> ids(n), lg((size_t)cap * D, 0), ld(cap, kAlive);
    for (uint32_t i = 0; i < n; ++i) {
      keys[i] = ((uint64_t)f0[i] << 32) | f1[i];
      ids[i] = i;
      lg[i] = f0[i];
      lg[(size_t)cap + i] = f1[i];
      if (dead[i]) ld[i] = 0;
    }
    QCtl hc;
    std::memset(&hc, 0, sizeof(hc));
    for (int r = 0; r < 3; ++r) {
      hc.cyc[r].min_key.v = ~0ull;
      hc.cyc[r].win_min.v = kInf;
      hc.cyc[r].f1lo.v = kInf;
    }
    hc.n_labels.v = n;
    const int32_t nil3[3] = {kNil, kNil, kNil};
    auto up = [&](void* dst, const void* src, size_t b) {
      if (e == cudaSuccess && b) e = cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice);
    };
    up(C, &hc, sizeof(hc));
    up(A.okey[1], keys.data(), keys.size() * 8);
    up(A.oid[1], ids.data(), ids.size() * 4);
    up(A.lg, lg.data(), lg.size() * 4);
    up(A.ldead, ld.data(), ld.size() * 4);
    up(A.cs[0].node_head, nil3, sizeof(nil3));
    up(A.cs[1].node_head, nil3, sizeof(nil3));
    if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook upload: %s", cudaGetErrorString(e));
    GraphDev G{};
    G.n = 2;
    G.d = D;
    G.rowptr = rowptr;  // no arcs: window labels produce no candidates
    QParams P{};
    P.goal = 1;
    P.h = h;
    P.window = window;
    P.lanes = 8;
    P.delta = bins[3];
    P.tile = 32;
    P.label_budget = cap;
    P.qd = D;
    P.ps_grow = 6;
    P.heavy_work = kHeavyWork;
    P.part_work = kPartWork;
    const BinParams bp{bins[0], bins[1], bins[2], bins[3], bins[4]};
    OutPool O{nullptr, 0, nullptr};
    window_hist_kernel<<<64, 256>>>(A, n, bp, A.hist + 1 * kNB);
    window_hook_kernel<<<1, kGridThreads>>>(G, A, C, P, O, n, bp, d_bstar);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook kernel: %s", cudaGetErrorString(e));
    unsigned kept = 0, err = 0;
    e = cudaMemcpy(&kept, &C->cyc[2].open_count.v, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, &C->error, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(bstar, d_bstar, 4, cudaMemcpyDeviceToHost);
    std::vector<uint32_t> kid(kept);
    if (e == cudaSuccess && kept) e = cudaMemcpy(kid.data(), A.oid[0], kept * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return hook_fail(OPMOS_ERR_CUDA, "test hook download: %s", cudaGetErrorString(e));
    if (err) return hook_fail((int)err, "test hook: extraction reported error %u", err);
    for (uint32_t i = 0; i < n; ++i) taken[i] = dead[i] ? 0 : 1;
    for (uint32_t x : kid)
      if (x < n) taken[x] = 0;
    return OPMOS_OK;
  } catch (...) {
    return hook_fail(OPMOS_ERR_OUT_OF_MEMORY, "test hook: host allocation failed");
  }
}

}  // extern "C"
