// C ABI (include/opmos.h): argument checking, device memory, launches and
// result marshalling. Every step of the search runs in the kernels of
// search.cu and heuristic.cu; this file only moves data and sizes arenas.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "opmos.h"
#include "graph.cuh"
#include "search.cuh"

using namespace opmos;

namespace {

thread_local std::string g_err;
std::mutex g_mu;  // the library runs one call at a time per process

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// No C++ exception crosses the C ABI: every entry point that returns a code
// runs its body here and turns an exception into an error code.
template <class F>
int guarded(const char* what, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(OPMOS_ERR_OUT_OF_MEMORY, "%s: host allocation failed", what);
  } catch (const std::exception& e) {
    return fail(OPMOS_ERR_CUDA, "%s: %s", what, e.what());
  } catch (...) {
    return fail(OPMOS_ERR_CUDA, "%s: unexpected exception", what);
  }
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(OPMOS_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(OPMOS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct DevInfo {
  bool ok = false;
  int sms = 0;
  int dev = 0;
};

DevInfo device_info() {
  DevInfo di;
  int cnt = 0;
  if (cudaGetDeviceCount(&cnt) != cudaSuccess || cnt == 0) {
    cudaGetLastError();
    return di;
  }
  cudaGetDevice(&di.dev);
  cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, di.dev);
  di.ok = di.sms > 0;
  return di;
}

// A grow-only device buffer reused across calls.
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
  int get(size_t want, void** out) {
    if (want > bytes) {
      if (ptr) cudaFree(ptr);
      ptr = nullptr;
      bytes = 0;
      cudaError_t e = cudaMalloc(&ptr, want);
      if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
      }
      bytes = want;
    }
    *out = ptr;
    return OPMOS_OK;
  }
};

Workspace g_arena, g_out, g_scratch, g_misc;

// A grow-only pinned host buffer (staging for captured launches).
struct PinnedWorkspace {
  void* ptr = nullptr;
  size_t bytes = 0;
  int get(size_t want, void** out) {
    if (want > bytes) {
      if (ptr) cudaFreeHost(ptr);
      ptr = nullptr;
      bytes = 0;
      cudaError_t e = cudaHostAlloc(&ptr, want, cudaHostAllocDefault);
      if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_fail(e, "cudaHostAlloc(staging)");
      }
      bytes = want;
    }
    *out = ptr;
    return OPMOS_OK;
  }
};
PinnedWorkspace g_pinned;

template <class T>
T* carve(char*& p, size_t count, size_t align = 256) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  a = (a + align - 1) / align * align;
  T* r = reinterpret_cast<T*>(a);
  p = reinterpret_cast<char*>(a + count * sizeof(T));
  return r;
}

}  // namespace

int opmos::record_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

struct opmos_heur {
  const opmos_graph* g = nullptr;
  uint32_t goal = 0, d = 0;
  uint32_t* h = nullptr;
  uint64_t ns = 0;
};

struct opmos_result {
  uint32_t count = 0, d = 0;
  bool has_paths = false;
  std::vector<uint32_t> costs, offs, nodes;
  std::vector<uint64_t> edges;
  opmos_stats stats{};
};

namespace {

void free_graph(opmos_graph* g) {
  if (!g) return;
  for (uint32_t* p : {g->rowptr, g->col, g->cost, g->rrowptr, g->rsrc, g->rcost, g->delta})
    if (p) cudaFree(p);
  delete g;
}

opmos_options resolve(const opmos_options* in, bool batch) {
  opmos_options o;
  opmos_default_options(&o);
  if (batch) {
    o.window = 256;
    o.mem_budget_bytes = 160ull << 30;
  }
  if (!in) return o;
  if (in->window) o.window = in->window;
  if (in->lanes_per_label) o.lanes_per_label = in->lanes_per_label;
  if (in->tile) o.tile = in->tile;
  if (in->delta) o.delta = in->delta;
  if (in->label_budget) o.label_budget = in->label_budget;
  if (in->mem_budget_bytes) o.mem_budget_bytes = in->mem_budget_bytes;
  if (in->d_used) o.d_used = in->d_used;
  if (in->alone_labels) o.alone_labels = in->alone_labels;
  if (in->alone_window) o.alone_window = in->alone_window;
  o.flags = in->flags;
  o.stream = in->stream;
  return o;
}

int check_options(const opmos_options& o, const opmos_graph* g, uint32_t* d_used) {
  const uint32_t du = o.d_used ? o.d_used : g->d;
  if (du < 1 || du > g->d) return fail(OPMOS_ERR_INVALID_ARG, "d_used %u not in [1, %u]", du, g->d);
  if (o.lanes_per_label != 4 && o.lanes_per_label != 8 && o.lanes_per_label != 16 && o.lanes_per_label != 32)
    return fail(OPMOS_ERR_INVALID_ARG, "lanes_per_label must be 4, 8, 16 or 32");
  if (o.tile % 32 || o.tile == 0) return fail(OPMOS_ERR_INVALID_ARG, "tile must be a positive multiple of 32");
  if (o.window == 0 || o.window > (1u << 22)) return fail(OPMOS_ERR_INVALID_ARG, "window out of range");
  if (o.alone_window > (1u << 22)) return fail(OPMOS_ERR_INVALID_ARG, "alone_window out of range");
  *d_used = du;
  return OPMOS_OK;
}

constexpr uint32_t kWindowCapMin = 16384;  // labels a window may hold at least

// Sizes of one query arena for a given byte budget.
struct ArenaPlan {
  uint32_t label_cap, open_cap, win_cap, cand_cap, plog_cap, nslots, lsub, kparts, xcap;
  unsigned long long fpool_words;
  size_t bytes;
  size_t fixed;  // the part that does not grow with the labels
};

int plan_arena(const opmos_graph* g, uint32_t D, uint32_t window, size_t budget, bool batch, ArenaPlan* pl) {
  const size_t n = g->n;
  // a step takes whole histogram bins, so it may take more than W when the
  // lowest bin alone holds more; beyond win_cap the part it takes would
  // depend on thread timing (the front would not), hence the generous cap
  pl->win_cap = std::max<uint32_t>(4 * window, kWindowCapMin);
  pl->cand_cap = pl->win_cap * std::max<uint32_t>(g->maxdeg, 1);
  pl->plog_cap = batch ? (1u << 16) : (1u << 20);
  const size_t ptiles = pl->plog_cap / 32 + 1;
  // per node: fbase, fcount, fcap, then per candidate set ncand, list heads, heavy flag,
  // part count, slots; per candidate (two sets): node, parent, arc, list link, two touched
  // entries, part count, flag, cost vector; the parts of split merges (two sets)
  pl->lsub = batch ? kLSubBatch : kLSubGrid;
  pl->nslots = kNodeSlots;
  pl->kparts = 1;
  pl->xcap = 0;
  if (!batch) {
    pl->nslots = kNodeSlotsGrid;
    pl->kparts = kPartsMax;
    pl->xcap = kPartsMax * (uint32_t)std::min<size_t>(n + 1, pl->cand_cap);
  }
  size_t fixed = (n + 1) * (8 + 4 + 4 + 2 * (4 + (4u << pl->lsub) + 4 + 4 + 4 * (size_t)pl->nslots)) + 3 * kNB * 4 +
                 2 * (size_t)pl->cand_cap * (32 + 4 * D) + 2 * (size_t)pl->xcap * 4 + (size_t)pl->plog_cap * 4 * D +
                 2 * ((size_t)pl->plog_cap + ptiles) * 4 * D + kPSMax * 4 + 96 * 256;
  pl->fixed = fixed;
  if (budget < fixed + (8u << 20))
    return fail(OPMOS_ERR_CAPACITY, "arena budget %zu too small (fixed part %zu)", budget, fixed);
  const size_t rem = budget - fixed;
  const size_t per_label = 4 * D + 20;  // cost vector, node, parent, arc, P-log mark, death step
  size_t labels = rem * 30 / 100 / per_label;
  labels = std::min<size_t>(labels, 0xFFFFFF00u);
  pl->label_cap = (uint32_t)labels;
  pl->fpool_words = rem * 55 / 100 / 4;
  size_t open = rem * 15 / 100 / 24;
  pl->open_cap = (uint32_t)std::min<size_t>(open, 0xFFFFFF00u);
  pl->bytes = budget;
  return OPMOS_OK;
}

void layout_arena(const opmos_graph* g, uint32_t D, const ArenaPlan& pl, char* base, QArena* A) {
  char* p = base;
  const size_t n = g->n + 1;  // the last node stands for P (extracted goal labels)
  A->fbase = carve<uint64_t>(p, n);
  A->fcount = carve<uint32_t>(p, n);
  A->fcap = carve<uint32_t>(p, n);
  for (int b = 0; b < 2; ++b) {
    CandSet& cs = A->cs[b];
    cs.ncand = carve<uint32_t>(p, n);
    cs.node_head = carve<int32_t>(p, n << pl.lsub);
    cs.hflag = carve<uint32_t>(p, n);
    cs.hcnt = carve<uint32_t>(p, n);
    cs.hsplit = carve<uint32_t>(p, pl.cand_cap);
    cs.xpart = carve<uint32_t>(p, std::max<uint32_t>(pl.xcap, 1));
    cs.cflag = carve<uint32_t>(p, pl.cand_cap);
    cs.cslot = carve<int32_t>(p, n * pl.nslots);
    cs.cnode = carve<uint32_t>(p, pl.cand_cap);
    cs.cparent = carve<uint32_t>(p, pl.cand_cap);
    cs.cedge = carve<uint32_t>(p, pl.cand_cap);
    cs.cnext = carve<int32_t>(p, pl.cand_cap);
    cs.touched = carve<uint32_t>(p, 2 * (size_t)pl.cand_cap);
    cs.cg = carve<uint32_t>(p, (size_t)pl.cand_cap * D);
  }
  A->hist = carve<uint32_t>(p, 3 * kNB);
  A->prank = carve<uint32_t>(p, kPSMax);
  A->plog = carve<uint32_t>(p, (size_t)pl.plog_cap * D);
  A->lg = carve<uint32_t>(p, (size_t)pl.label_cap * D);
  A->lnode = carve<uint32_t>(p, pl.label_cap);
  A->lparent = carve<uint32_t>(p, pl.label_cap);
  A->ledge = carve<uint32_t>(p, pl.label_cap);
  A->lpver = carve<uint32_t>(p, pl.label_cap);
  A->ldead = carve<uint32_t>(p, pl.label_cap);
  for (int b = 0; b < 2; ++b) {
    A->okey[b] = carve<uint64_t>(p, pl.open_cap);
    A->oid[b] = carve<uint32_t>(p, pl.open_cap);
    A->ps[b] = carve<uint32_t>(p, (size_t)pl.plog_cap * D);
    A->pst[b] = carve<uint32_t>(p, ((size_t)pl.plog_cap / 32 + 1) * D);
  }
  A->fpool = carve<uint32_t>(p, pl.fpool_words);
  A->label_cap = pl.label_cap;
  A->open_cap = pl.open_cap;
  A->win_cap = pl.win_cap;
  A->cand_cap = pl.cand_cap;
  A->plog_cap = pl.plog_cap;
  A->fpool_words = pl.fpool_words;
  A->nslots = pl.nslots;
  A->lsub = pl.lsub;
  A->kparts = pl.kparts;
  A->xcap = pl.xcap;
}

int compute_heuristic(const opmos_graph* g, uint32_t D, const uint32_t* goals, uint32_t ngoals, uint32_t* h,
                      cudaStream_t s, uint64_t* ns) {
  const DevInfo di = device_info();
  if (!di.ok) return fail(OPMOS_ERR_CUDA, "no CUDA device");
  const unsigned njobs = ngoals * D;
  std::vector<HJob> jobs(njobs);
  for (uint32_t q = 0; q < ngoals; ++q)
    for (uint32_t k = 0; k < D; ++k) jobs[q * D + k] = HJob{goals[q], k, h + ((size_t)q * D + k) * g->n};
  const unsigned blocks = std::min<unsigned>(njobs, (unsigned)di.sms * 2);
  const size_t spb = 5 * (size_t)g->n + 64;
  void* scratch = nullptr;
  if (int rc = g_scratch.get(spb * blocks * 4, &scratch)) return rc;
  void* misc = nullptr;
  const size_t jobs_bytes = njobs * sizeof(HJob);
  if (int rc = g_misc.get(jobs_bytes + 1024, &misc)) return rc;
  char* mp = (char*)misc;
  unsigned* ctr = carve<unsigned>(mp, 2);
  HJob* djobs = carve<HJob>(mp, njobs);
  CK(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s));
  CK(cudaMemcpyAsync(djobs, jobs.data(), jobs_bytes, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t e = launch_heuristic(g->dev, djobs, njobs, (uint32_t*)scratch, spb, blocks, g->delta, ctr,
                                   ctr + 1, s);
  cudaEventRecord(e1, s);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(e, "heuristic launch");
  }
  unsigned herr = 0;
  cudaError_t e2 = cudaMemcpyAsync(&herr, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e2 != cudaSuccess) return cuda_fail(e2, "heuristic status copy");
  if (e3 != cudaSuccess) return cuda_fail(e3, "heuristic kernel");
  if (herr) return fail((int)herr, "heuristic kernel reported error %u", herr);
  if (ns) *ns = (uint64_t)(ms * 1e6);
  return OPMOS_OK;
}

void fill_stats(opmos_stats* s, const QResult& R, uint32_t D) {
  s->extracted = R.stats[S_EXTRACTED];
  s->dead_skipped = R.stats[S_DEAD];
  s->goal_pruned = R.stats[S_GOALPRUNED];
  s->candidates = R.stats[S_CAND];
  s->inserted = R.stats[S_INSERTED];
  s->pruned = R.stats[S_PRUNED];
  s->steps = R.stats[S_STEPS];
  s->frontier_cmp = R.stats[S_FCMP];
  s->p_cmp = R.stats[S_PCMP];
  s->phase_ns[0] = R.stats[S_TSEL];
  s->phase_ns[1] = R.stats[S_TWORK];
  s->phase_ns[2] = R.stats[S_TSYNC];
  s->phase_ns[3] = R.stats[S_TOUT];
  s->goal_inserted = R.stats[S_GOALINS];
  s->open_scanned = R.stats[S_OSCAN];
  s->open_rewritten = R.stats[S_OKEEP];
  s->list_candidates = R.stats[S_OVF];
  s->longest_task_ns[0] = R.stats[S_MAXH];
  s->longest_task_ns[1] = R.stats[S_MAXL];
  s->longest_task_ns[2] = R.stats[S_MAXX];
  s->heavy_merges = R.stats[S_NHEAVY];
  s->heavy_max_candidates = R.stats[S_MAXNC];
  s->heavy_max_frontier = R.stats[S_MAXF];
  s->task_ns[0] = R.stats[S_SUMH];
  s->task_ns[1] = R.stats[S_SUML];
  s->task_ns[2] = R.stats[S_SUMX];
  // algorithmic bytes: per extracted label 8d+12 (g, node, rowptr pair, F key),
  // per candidate 4+8d (col, cost, h), per compared frontier/P entry 4d, per
  // inserted label 4d+24 (label record, frontier slot, OPEN entry), per prune 4.
  const uint64_t d = D;
  s->bytes = s->extracted * (8 * d + 12) + s->candidates * (4 + 8 * d) + (s->frontier_cmp + s->p_cmp) * 4 * d +
             s->inserted * (4 * d + 24) + s->pruned * 4;
}

// Copy one query's output region to a host result. The kernel wrote Dk
// columns per cost vector; the query uses the first D of them (the rest are
// the zero objectives a query with fewer objectives than its kernel carries).
int take_result(const QResult& R, uint32_t D, bool paths, const uint32_t* words, cudaStream_t s,
                opmos_result** out, uint32_t Dk = 0) {
  if (Dk == 0) Dk = D;
  auto* r = new (std::nothrow) opmos_result;
  if (!r) return fail(OPMOS_ERR_OUT_OF_MEMORY, "host allocation");
  r->count = R.count;
  r->d = D;
  r->has_paths = paths;
  const size_t k = R.count;
  r->costs.resize(k * D);
  r->offs.resize(k + 1);
  std::vector<uint32_t> tmp(k * Dk + k + 1);
  if (!tmp.empty()) {
    cudaError_t e = cudaMemcpyAsync(tmp.data(), words + R.off, tmp.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
      delete r;
      return cuda_fail(e, "result copy");
    }
  }
  std::vector<uint32_t> pw;
  if (paths && R.total) {
    pw.resize(2 * R.total - k);
    cudaError_t e = cudaMemcpyAsync(pw.data(), words + R.path, pw.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
      delete r;
      return cuda_fail(e, "path copy");
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete r;
    return cuda_fail(e, "result copy");
  }
  for (size_t i = 0; i < k; ++i)
    std::copy(tmp.begin() + i * Dk, tmp.begin() + i * Dk + D, r->costs.begin() + i * D);
  std::copy(tmp.begin() + k * Dk, tmp.end(), r->offs.begin());
  if (paths && R.total) {
    r->nodes.assign(pw.begin(), pw.begin() + R.total);
    r->edges.resize(R.total - k);
    for (size_t i = 0; i < R.total - k; ++i) r->edges[i] = pw[R.total + i];
  }
  *out = r;
  return OPMOS_OK;
}

int search_status(unsigned st) {
  switch (st) {
    case 0:
      return OPMOS_OK;
    case OPMOS_ERR_CAPACITY:
      return fail(OPMOS_ERR_CAPACITY, "query arena full (labels, frontier pool, open list or output)");
    case OPMOS_ERR_BUDGET:
      return fail(OPMOS_ERR_BUDGET, "label budget exceeded");
    case OPMOS_ERR_TIMEOUT:
      return fail(OPMOS_ERR_TIMEOUT, "device-side wait or time limit expired");
    default:
      return fail((int)st, "search kernel error %u", st);
  }
}

constexpr unsigned long long kTimeLimitNs = 300ull * 1000 * 1000 * 1000;

// Device time a search may take before it stops with OPMOS_ERR_TIMEOUT: 300 s,
// or OPMOS_TIME_LIMIT_MS from the environment (read at each call) when that
// is a positive integer.
unsigned long long time_limit_ns() {
  if (const char* e = std::getenv("OPMOS_TIME_LIMIT_MS")) {
    char* end = nullptr;
    const unsigned long long ms = std::strtoull(e, &end, 10);
    if (end != e && *end == '\0' && ms > 0 && ms < (1ull << 40)) return ms * 1000000ull;
  }
  return kTimeLimitNs;
}
constexpr unsigned kBatchSlots = 192;  // concurrent queries of a batch
constexpr uint64_t kAloneLabels = 1000000;  // default alone_labels
// P-index rebuild thresholds (log growth beyond 32 + count >> grow): the
// whole grid ranks a single query's index fast; a multi-query slot has only
// its share of the blocks, so it rebuilds less often.
constexpr uint32_t kGridIndexGrow = 6;
constexpr uint32_t kMultiIndexGrow = 4;
constexpr size_t kOutWords = 64ull << 20;

int solve_one(const opmos_graph* g, const opmos_heur* heur, uint32_t start, uint32_t goal, const opmos_options& o,
              uint32_t D, opmos_result** out) {
  const auto t0 = std::chrono::steady_clock::now();
  const DevInfo di = device_info();
  if (!di.ok) return fail(OPMOS_ERR_CUDA, "no CUDA device");
  cudaStream_t s = (cudaStream_t)o.stream;
  uint64_t hns = 0;
  const uint32_t* h = nullptr;
  opmos_heur tmp{};
  if (heur) {
    if (heur->g != g || heur->goal != goal || heur->d < D)
      return fail(OPMOS_ERR_INVALID_ARG, "heuristic belongs to another graph, goal or objective count");
    if (heur->d != D) return fail(OPMOS_ERR_INVALID_ARG, "heuristic computed for d=%u, query uses d=%u", heur->d, D);
    h = heur->h;
  } else {
    CK(cudaMalloc(&tmp.h, (size_t)D * g->n * 4));
    if (int rc = compute_heuristic(g, D, &goal, 1, tmp.h, s, &hns)) {
      cudaFree(tmp.h);
      return rc;
    }
    h = tmp.h;
  }
  struct Free {
    uint32_t* p;
    ~Free() {
      if (p) cudaFree(p);
    }
  } free_h{tmp.h};

  ArenaPlan pl;
  if (int rc = plan_arena(g, D, o.window, o.mem_budget_bytes, false, &pl)) return rc;
  void* arena = nullptr;
  if (int rc = g_arena.get(pl.bytes, &arena)) return rc;
  QArena A{};
  layout_arena(g, D, pl, (char*)arena, &A);
  void* outp = nullptr;
  const size_t header = 4 * 256 + sizeof(QCtl) + sizeof(QResult);  // counters, control block, result
  if (int rc = g_out.get(kOutWords * 4 + header, &outp)) return rc;
  char* op = (char*)outp;
  unsigned long long* used = carve<unsigned long long>(op, 1);
  QCtl* C = carve<QCtl>(op, 1);
  QResult* R = carve<QResult>(op, 1);
  uint32_t* words = carve<uint32_t>(op, kOutWords);
  OutPool O{words, kOutWords, used};
  CK(cudaMemsetAsync(outp, 0, (size_t)((char*)words - (char*)outp), s));

  QParams P{};
  P.start = start;
  P.goal = goal;
  P.h = h;
  P.window = o.window;
  P.lanes = o.lanes_per_label;
  P.delta = o.delta;
  P.tile = o.tile;
  P.label_budget = (uint32_t)std::min<uint64_t>(o.label_budget ? o.label_budget : ~0ull, A.label_cap);
  P.flags = o.flags;
  P.qd = D;
  P.ps_grow = kGridIndexGrow;
  P.heavy_work = o.window < kSmallWindow ? kHeavyWorkSmallWindow : kHeavyWork;
  P.part_work = o.window < kSmallWindow ? kPartWork : kPartWorkWide;
  P.time_limit_ns = time_limit_ns();

  // large windows take the wide grid (three 256-thread blocks per SM)
  const bool wide = o.window >= kSmallWindow;
  int occ = search_occupancy(D, wide);
  if (occ <= 0) return fail(OPMOS_ERR_CUDA, "search kernel cannot be resident");
  const unsigned blocks = (unsigned)di.sms * (unsigned)std::min(occ, wide ? (int)kGridWideBlocksPerSM : 1);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t e = launch_search_grid(D, g->dev, A, C, P, O, R, wide, blocks, s);
  cudaEventRecord(e1, s);
  QResult hr{};
  cudaError_t e2 = e == cudaSuccess ? cudaMemcpyAsync(&hr, R, sizeof(QResult), cudaMemcpyDeviceToHost, s) : e;
  cudaError_t e3 = cudaStreamSynchronize(s);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "search launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "search status copy");
  if (e3 != cudaSuccess) return cuda_fail(e3, "search kernel");
  if (int rc = search_status(hr.status)) return rc;
  const bool paths = !(o.flags & OPMOS_FLAG_NO_PATHS);
  opmos_result* r = nullptr;
  if (int rc = take_result(hr, D, paths, words, s, &r)) return rc;
  fill_stats(&r->stats, hr, D);
  r->stats.heuristic_ns = heur ? 0 : hns;
  r->stats.search_ns = (uint64_t)(ms * 1e6);
  r->stats.total_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now() - t0).count();
  *out = r;
  return OPMOS_OK;
}

// h_0(start) of every query (its distance under objective 0), for ordering.
__global__ void gather_h0_kernel(const MQuery* qs, unsigned nq, unsigned n, uint32_t* out) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nq) out[i] = qs[i].h[qs[i].start];
}

// One launch of the multi-query kernel over the queries in qlist, `slots` at a
// time with `slot_budget` bytes each. Results go to out/status; queries that
// outgrew their slot are listed in *overflow.
int run_multi(const opmos_graph* g, uint32_t D, const opmos_options& o, const std::vector<uint32_t>& qlist,
              const uint32_t* starts, const uint32_t* goals, uint32_t* hall, std::map<uint32_t, uint32_t>& gidx,
              unsigned slots, size_t slot_budget, uint64_t hns, std::chrono::steady_clock::time_point t0,
              opmos_result** out, int* status, std::vector<uint32_t>* overflow) {
  const DevInfo di = device_info();
  cudaStream_t s = (cudaStream_t)o.stream;
  const uint32_t nq = (uint32_t)qlist.size();
  const int occ = multi_occupancy(D);
  if (occ <= 0) return fail(OPMOS_ERR_CUDA, "multi-query kernel cannot be resident");
  const unsigned blocks = (unsigned)di.sms * (unsigned)std::min(occ, 2);
  ArenaPlan pl;
  if (int rc = plan_arena(g, D, o.window, slot_budget, true, &pl)) return rc;
  const size_t slot_bytes = (pl.bytes + 255) / 256 * 256;
  void* arena = nullptr;
  if (int rc = g_arena.get(slot_bytes * slots, &arena)) return rc;
  QParams P{};
  P.window = o.window;
  P.lanes = o.lanes_per_label;
  P.delta = o.delta;
  P.tile = o.tile;
  // the slot's label budget: the query's own, or the point past which it is
  // solved alone instead (a lower one), within what the slot holds
  const uint64_t own = o.label_budget ? o.label_budget : ~0ull;
  P.label_budget = (uint32_t)std::min<uint64_t>(std::min<uint64_t>(own, o.alone_labels), pl.label_cap);
  P.flags = o.flags;
  P.qd = D;
  P.ps_grow = kMultiIndexGrow;
  P.heavy_work = kHeavyWork;
  P.part_work = kPartWork;
  P.time_limit_ns = time_limit_ns();
  std::vector<MSlot> hslots(slots);
  for (unsigned i = 0; i < slots; ++i) {
    MSlot& sl = hslots[i];
    std::memset(&sl, 0, sizeof(sl));
    layout_arena(g, D, pl, (char*)arena + i * slot_bytes, &sl.A);
    sl.P = P;
    sl.G = g->dev;
    sl.d = D;
    sl.state = SL_FREE;
  }
  std::vector<MQuery> qs(nq);
  for (uint32_t i = 0; i < nq; ++i) {
    const uint32_t q = qlist[i];
    qs[i] = MQuery{0, starts[q], goals[q], D, hall + (size_t)gidx[goals[q]] * D * g->n};
  }
  // Longest first: admit queries in decreasing h_0(start) so that the large
  // searches start early and overlap with many small ones.
  std::vector<uint32_t> order(nq);
  {
    void* tmp = nullptr;
    if (int rc = g_misc.get(nq * (sizeof(MQuery) + 4) + 512, &tmp)) return rc;
    char* tp = (char*)tmp;
    MQuery* tq = carve<MQuery>(tp, nq);
    uint32_t* th = carve<uint32_t>(tp, nq);
    std::vector<uint32_t> h0(nq);
    CK(cudaMemcpyAsync(tq, qs.data(), nq * sizeof(MQuery), cudaMemcpyHostToDevice, s));
    gather_h0_kernel<<<(nq + 255) / 256, 256, 0, s>>>(tq, nq, g->n, th);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h0.data(), th, nq * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < nq; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return h0[a] > h0[b]; });
    std::vector<MQuery> sorted(nq);
    for (uint32_t i = 0; i < nq; ++i) sorted[i] = qs[order[i]];
    qs.swap(sorted);
  }
  // result pool: costs, offsets and paths of every query of this launch; a
  // query that finds it full is reported as a capacity overflow and re-run
  const size_t out_words = std::max<size_t>(kOutWords, std::min<size_t>((size_t)nq << 18, 1ull << 30));
  void* outp = nullptr;
  const size_t misc_bytes = slots * (sizeof(MSlot) + sizeof(QCtl) + 4) + nq * (sizeof(MQuery) + sizeof(QResult)) +
                            sizeof(GraphDev) + sizeof(MCtl) + 16 * 256;
  if (int rc = g_out.get(out_words * 4 + misc_bytes, &outp)) return rc;
  char* op = (char*)outp;
  unsigned long long* used = carve<unsigned long long>(op, 1);
  unsigned* hctl = carve<unsigned>(op, HC_RELEASE + slots);
  MCtl* M = carve<MCtl>(op, 1);
  GraphDev* dgraphs = carve<GraphDev>(op, 1);
  QCtl* ctls = carve<QCtl>(op, slots);
  MSlot* dslots = carve<MSlot>(op, slots);
  MQuery* dqs = carve<MQuery>(op, nq);
  QResult* dres = carve<QResult>(op, nq);
  uint32_t* words = carve<uint32_t>(op, out_words);
  for (auto& sl : hslots) sl.O = OutPool{words, out_words, used};  // one pool shared by all slots
  MCtl hM{};
  hM.qcap = nq;
  hM.hold = 0;
  std::vector<unsigned> hc(HC_RELEASE + slots, 0);
  hc[HC_TAIL] = nq;     // every query is queued up front
  hc[HC_CLOSING] = 1;   // and no more will come
  std::vector<QResult> hres(nq);
  MCtl hM2{};
  float ms = 0;
  if (o.flags & OPMOS_FLAG_GRAPH) {
    // stage the inputs in pinned memory, capture uploads + kernel + downloads
    const size_t b_hc = hc.size() * 4, b_sl = slots * sizeof(MSlot), b_q = nq * sizeof(MQuery),
                 b_r = nq * sizeof(QResult);
    void* pin = nullptr;
    if (int rc = g_pinned.get(b_hc + sizeof(MCtl) * 2 + sizeof(GraphDev) + b_sl + b_q + b_r + 8 * 256, &pin))
      return rc;
    char* pp = (char*)pin;
    unsigned* p_hc = carve<unsigned>(pp, hc.size());
    MCtl* p_M = carve<MCtl>(pp, 1);
    MCtl* p_M2 = carve<MCtl>(pp, 1);
    GraphDev* p_g = carve<GraphDev>(pp, 1);
    MSlot* p_sl = carve<MSlot>(pp, slots);
    MQuery* p_q = carve<MQuery>(pp, nq);
    QResult* p_r = carve<QResult>(pp, nq);
    std::memcpy(p_hc, hc.data(), b_hc);
    *p_M = hM;
    *p_g = g->dev;
    std::memcpy(p_sl, hslots.data(), b_sl);
    std::memcpy(p_q, qs.data(), b_q);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the legacy default stream cannot be captured: use a stream of our own
    static cudaStream_t own = nullptr;
    if (!s) {
      if (!own) CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
      CK(cudaDeviceSynchronize());  // earlier default-stream work is complete
      s = own;
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(used, 0, 8, s);
      cudaMemcpyAsync(hctl, p_hc, b_hc, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(M, p_M, sizeof(MCtl), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(dgraphs, p_g, sizeof(GraphDev), cudaMemcpyHostToDevice, s);
      cudaMemsetAsync(ctls, 0, slots * sizeof(QCtl), s);
      cudaMemsetAsync(dres, 0, b_r, s);
      cudaMemcpyAsync(dslots, p_sl, b_sl, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(dqs, p_q, b_q, cudaMemcpyHostToDevice, s);
      const cudaError_t el = launch_multi(D, dslots, ctls, slots, dqs, hctl, dgraphs, dres, nullptr, M, blocks, s);
      cudaMemcpyAsync(p_r, dres, b_r, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(p_M2, M, sizeof(MCtl), cudaMemcpyDeviceToHost, s);
      e = cudaStreamEndCapture(s, &graph);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (e == cudaSuccess) {
      cudaEventRecord(e0, s);
      e = cudaGraphLaunch(exec, s);
      cudaEventRecord(e1, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "captured multi-query launch");
    }
    std::memcpy(hres.data(), p_r, b_r);
    hM2 = *p_M2;
  } else {
    CK(cudaMemsetAsync(used, 0, 8, s));
    CK(cudaMemcpyAsync(hctl, hc.data(), hc.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(M, &hM, sizeof(MCtl), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dgraphs, &g->dev, sizeof(GraphDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctls, 0, slots * sizeof(QCtl), s));
    CK(cudaMemsetAsync(dres, 0, nq * sizeof(QResult), s));
    CK(cudaMemcpyAsync(dslots, hslots.data(), slots * sizeof(MSlot), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dqs, qs.data(), nq * sizeof(MQuery), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = launch_multi(D, dslots, ctls, slots, dqs, hctl, dgraphs, dres, nullptr, M, blocks, s);
    cudaEventRecord(e1, s);
    cudaError_t e2 =
        e == cudaSuccess ? cudaMemcpyAsync(hres.data(), dres, nq * sizeof(QResult), cudaMemcpyDeviceToHost, s) : e;
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&hM2, M, sizeof(MCtl), cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "multi-query launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "batch status copy");
    if (e3 != cudaSuccess) return cuda_fail(e3, "multi-query kernel");
  }
  if (hM2.error) return fail((int)hM2.error, "multi-query kernel stopped with error %u", hM2.error);
  const bool paths = !(o.flags & OPMOS_FLAG_NO_PATHS);
  const uint64_t total_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t0).count();
  for (uint32_t i = 0; i < nq; ++i) {
    const uint32_t q = qlist[order[i]];
    const unsigned st = hres[i].status;
    if (st == OPMOS_ERR_CAPACITY || (st == OPMOS_ERR_BUDGET && P.label_budget < own)) {
      overflow->push_back(q);  // outgrew its slot or the shared launch: solved alone
      continue;
    }
    if (st != 0) {
      status[q] = (int)st;
      continue;
    }
    opmos_result* r = nullptr;
    int rc = take_result(hres[i], D, paths, words, s, &r);
    status[q] = rc;
    if (rc) continue;
    fill_stats(&r->stats, hres[i], D);
    r->stats.heuristic_ns = hns;
    r->stats.search_ns = (uint64_t)(ms * 1e6);
    r->stats.total_ns = total_ns;
    out[q] = r;
  }
  return OPMOS_OK;
}

}  // namespace

extern "C" {

void opmos_default_options(opmos_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->window = 1024;
  o->lanes_per_label = 8;
  o->tile = 32;
  o->delta = 1;
  o->label_budget = 0;
  o->mem_budget_bytes = 8ull << 30;
  o->d_used = 0;
  o->flags = 0;
  o->alone_labels = kAloneLabels;
  o->stream = nullptr;
}

int opmos_device_count(void) {
  int c = 0;
  if (cudaGetDeviceCount(&c) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return c;
}

const char* opmos_last_error(void) { return g_err.c_str(); }

int opmos_graph_create(uint32_t n, uint64_t m, uint32_t d, const uint64_t* rowptr, const uint32_t* col,
                       const uint32_t* cost, opmos_graph** out) {
  return guarded("opmos_graph_create", [&]() -> int {
    if (!out) return fail(OPMOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!rowptr || (m && (!col || !cost))) return fail(OPMOS_ERR_INVALID_ARG, "NULL array");
    if (n == 0 || n >= (1u << 31)) return fail(OPMOS_ERR_INVALID_ARG, "n=%u out of range", n);
    if (d < 1 || d > OPMOS_MAX_D) return fail(OPMOS_ERR_INVALID_ARG, "d=%u not in [1, %d]", d, OPMOS_MAX_D);
    if (m >= 0xFFFFFFFFull) return fail(OPMOS_ERR_INVALID_ARG, "m too large");
    if (rowptr[0] != 0 || rowptr[n] != m) return fail(OPMOS_ERR_INVALID_ARG, "rowptr[0] != 0 or rowptr[n] != m");
    uint32_t maxdeg = 0;
    for (uint32_t v = 0; v < n; ++v) {
      if (rowptr[v + 1] < rowptr[v]) return fail(OPMOS_ERR_INVALID_ARG, "rowptr not monotone at %u", v);
      maxdeg = std::max<uint32_t>(maxdeg, (uint32_t)(rowptr[v + 1] - rowptr[v]));
    }
    for (uint64_t e = 0; e < m; ++e)
      if (col[e] >= n) return fail(OPMOS_ERR_INVALID_ARG, "col[%llu] = %u >= n", (unsigned long long)e, col[e]);
    std::vector<uint32_t> delta(d);
    for (uint32_t k = 0; k < d; ++k) {
      uint64_t mx = 0, sum = 0;
      for (uint64_t e = 0; e < m; ++e) {
        mx = std::max<uint64_t>(mx, cost[k * m + e]);
        sum += cost[k * m + e];
      }
      // g and F = g + h must fit uint32 on every simple path
      if ((unsigned __int128)2 * (n - 1) * mx >= ((unsigned __int128)1 << 32))
        return fail(OPMOS_ERR_OVERFLOW, "objective %u: 2*(n-1)*max cost does not fit uint32", k);
      const uint64_t mean = m ? (sum + m - 1) / m : 1;
      delta[k] = (uint32_t)std::max<uint64_t>(1, 2 * mean);
    }
    const DevInfo di = device_info();
    if (!di.ok) return fail(OPMOS_ERR_CUDA, "no CUDA device");
    // reversed CSR (in-arcs grouped by head node), costs carried along
    std::vector<uint32_t> rp32(n + 1), rrp(n + 1, 0), rsrc(m), rcost((size_t)d * m);
    for (uint32_t v = 0; v <= n; ++v) rp32[v] = (uint32_t)rowptr[v];
    for (uint64_t e = 0; e < m; ++e) rrp[col[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v) rrp[v + 1] += rrp[v];
    {
      std::vector<uint32_t> fill(rrp.begin(), rrp.end() - 1);
      for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
          const uint32_t slot = fill[col[e]]++;
          rsrc[slot] = u;
          for (uint32_t k = 0; k < d; ++k) rcost[(size_t)k * m + slot] = cost[k * m + e];
        }
    }
    auto* g = new (std::nothrow) opmos_graph;
    if (!g) return fail(OPMOS_ERR_OUT_OF_MEMORY, "host allocation");
    g->n = n;
    g->m = m;
    g->d = d;
    g->maxdeg = maxdeg;
    const size_t mb = std::max<size_t>(m, 1);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](uint32_t** p, size_t words) {
      if (e == cudaSuccess) e = cudaMalloc(p, words * 4);
    };
    alloc(&g->rowptr, n + 1);
    alloc(&g->col, mb);
    alloc(&g->cost, (size_t)d * mb);
    alloc(&g->rrowptr, n + 1);
    alloc(&g->rsrc, mb);
    alloc(&g->rcost, (size_t)d * mb);
    alloc(&g->delta, d);
    if (e == cudaSuccess) e = cudaMemcpy(g->rowptr, rp32.data(), (n + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(g->col, col, m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(g->cost, cost, (size_t)d * m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->rrowptr, rrp.data(), (n + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(g->rsrc, rsrc.data(), m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(g->rcost, rcost.data(), (size_t)d * m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->delta, delta.data(), d * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_graph(g);
      return cuda_fail(e, "graph upload");
    }
    g->dev = GraphDev{n, (uint32_t)m, d, maxdeg, g->rowptr, g->col, g->cost, g->rrowptr, g->rsrc, g->rcost};
    *out = g;
    return OPMOS_OK;
  });
}

void opmos_graph_destroy(opmos_graph* g) {
  std::lock_guard<std::mutex> lk(g_mu);
  free_graph(g);
}

int opmos_heuristic(const opmos_graph* g, uint32_t goal, uint32_t d_used, opmos_heur** out) {
  return guarded("opmos_heuristic", [&]() -> int {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!out) return fail(OPMOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g) return fail(OPMOS_ERR_INVALID_ARG, "graph is NULL");
    if (goal >= g->n) return fail(OPMOS_ERR_INVALID_ARG, "goal %u >= n", goal);
    const uint32_t D = d_used ? d_used : g->d;
    if (D > g->d) return fail(OPMOS_ERR_INVALID_ARG, "d_used %u > d %u", D, g->d);
    auto* h = new (std::nothrow) opmos_heur;
    if (!h) return fail(OPMOS_ERR_OUT_OF_MEMORY, "host allocation");
    h->g = g;
    h->goal = goal;
    h->d = D;
    cudaError_t e = cudaMalloc(&h->h, (size_t)D * g->n * 4);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaMalloc(heuristic)");
    }
    if (int rc = compute_heuristic(g, D, &goal, 1, h->h, nullptr, &h->ns)) {
      cudaFree(h->h);
      delete h;
      return rc;
    }
    *out = h;
    return OPMOS_OK;
  });
}

int opmos_heuristic_copy(const opmos_heur* h, uint32_t* h_out) {
  return guarded("opmos_heuristic_copy", [&]() -> int {
    if (!h || !h_out) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaMemcpy(h_out, h->h, (size_t)h->d * h->g->n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "heuristic copy");
    return OPMOS_OK;
  });
}

void opmos_heuristic_destroy(opmos_heur* h) {
  if (!h) return;
  if (h->h) cudaFree(h->h);
  delete h;
}

int opmos_solve(const opmos_graph* g, const opmos_heur* heur, uint32_t start, uint32_t goal,
                const opmos_options* opt, opmos_result** out) {
  return guarded("opmos_solve", [&]() -> int {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!out) return fail(OPMOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g) return fail(OPMOS_ERR_INVALID_ARG, "graph is NULL");
    if (start >= g->n || goal >= g->n) return fail(OPMOS_ERR_INVALID_ARG, "start/goal out of range");
    const opmos_options o = resolve(opt, false);
    uint32_t D;
    if (int rc = check_options(o, g, &D)) return rc;
    return solve_one(g, heur, start, goal, o, D, out);
  });
}

int opmos_solve_batch(const opmos_graph* g, uint32_t nq, const uint32_t* starts, const uint32_t* goals,
                      const opmos_options* opt, opmos_result** out, int* status) {
  return guarded("opmos_solve_batch", [&]() -> int {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g || !out || !status || (nq && (!starts || !goals))) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    for (uint32_t q = 0; q < nq; ++q) {
      out[q] = nullptr;
      status[q] = OPMOS_ERR_INVALID_ARG;
    }
    for (uint32_t q = 0; q < nq; ++q)
      if (starts[q] >= g->n || goals[q] >= g->n) return fail(OPMOS_ERR_INVALID_ARG, "query %u out of range", q);
    const opmos_options o = resolve(opt, true);
    uint32_t D;
    if (int rc = check_options(o, g, &D)) return rc;
    if (nq == 0) return OPMOS_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const DevInfo di = device_info();
    if (!di.ok) return fail(OPMOS_ERR_CUDA, "no CUDA device");
    cudaStream_t s = (cudaStream_t)o.stream;
    // heuristics, one per distinct goal
    std::map<uint32_t, uint32_t> gidx;
    std::vector<uint32_t> ugoals;
    for (uint32_t q = 0; q < nq; ++q)
      if (gidx.emplace(goals[q], (uint32_t)ugoals.size()).second) ugoals.push_back(goals[q]);
    uint32_t* hall = nullptr;
    CK(cudaMalloc(&hall, (size_t)ugoals.size() * D * g->n * 4));
    struct Free {
      void* p;
      ~Free() {
        if (p) cudaFree(p);
      }
    } free_h{hall};
    uint64_t hns = 0;
    if (int rc = compute_heuristic(g, D, ugoals.data(), (uint32_t)ugoals.size(), hall, s, &hns)) return rc;
    // One launch of the multi-query kernel for all queries; those that
    // outgrow their slot, or pass alone_labels, are solved alone afterwards.
    std::vector<uint32_t> todo(nq);
    for (uint32_t q = 0; q < nq; ++q) todo[q] = q;
    {
      const unsigned slots = std::max(1u, std::min<unsigned>(nq, std::min<unsigned>(kMaxSlots, kBatchSlots)));
      std::vector<uint32_t> overflow;
      if (int rc = run_multi(g, D, o, todo, starts, goals, hall, gidx, slots, o.mem_budget_bytes / slots, hns, t0, out,
                             status, &overflow))
        return rc;
      todo.swap(overflow);
    }
    if (!todo.empty()) {
      opmos_options so = resolve(opt, false);
      so.flags = o.flags;
      so.stream = o.stream;
      if (o.alone_window) so.window = o.alone_window;
      if (opt && opt->mem_budget_bytes) so.mem_budget_bytes = std::max<uint64_t>(opt->mem_budget_bytes, 1ull << 30);
      for (uint32_t q : todo) {
        opmos_result* r = nullptr;
        opmos_heur hh{g, goals[q], D, hall + (size_t)gidx[goals[q]] * D * g->n, 0};
        const int rc = solve_one(g, &hh, starts[q], goals[q], so, D, &r);
        status[q] = rc;
        if (rc == OPMOS_OK) {
          r->stats.heuristic_ns = hns;
          out[q] = r;
        }
      }
    }
    return OPMOS_OK;
  });
}


uint32_t opmos_result_count(const opmos_result* r) { return r ? r->count : 0; }
uint32_t opmos_result_d(const opmos_result* r) { return r ? r->d : 0; }

int opmos_result_costs(const opmos_result* r, uint32_t* out) {
  return guarded("opmos_result_costs", [&]() -> int {
    if (!r || (!out && r->count)) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    if (r->count) std::memcpy(out, r->costs.data(), r->costs.size() * 4);
    return OPMOS_OK;
  });
}

int opmos_result_path(const opmos_result* r, uint32_t i, uint32_t* nodes, uint64_t* edges, uint32_t cap,
                      uint32_t* len) {
  return guarded("opmos_result_path", [&]() -> int {
    if (!r || !len) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    if (!r->has_paths) return fail(OPMOS_ERR_INVALID_ARG, "result was solved without paths");
    if (i >= r->count) return fail(OPMOS_ERR_INVALID_ARG, "solution index %u >= count %u", i, r->count);
    const uint32_t a = r->offs[i], b = r->offs[i + 1];
    *len = b - a;
    if (b - a > cap) return fail(OPMOS_ERR_CAPACITY, "path of %u nodes exceeds cap %u", b - a, cap);
    if (!nodes || (b - a > 1 && !edges)) return fail(OPMOS_ERR_INVALID_ARG, "NULL output array");
    std::memcpy(nodes, r->nodes.data() + a, (size_t)(b - a) * 4);
    if (b - a > 1) std::memcpy(edges, r->edges.data() + (a - i), (size_t)(b - a - 1) * 8);
    return OPMOS_OK;
  });
}

int opmos_result_paths(const opmos_result* r, uint32_t* offsets, uint32_t* nodes, uint64_t* edges) {
  return guarded("opmos_result_paths", [&]() -> int {
    if (!r || !offsets || (!nodes != !edges)) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    if (!r->has_paths) return fail(OPMOS_ERR_INVALID_ARG, "result was solved without paths");
    std::memcpy(offsets, r->offs.data(), ((size_t)r->count + 1) * 4);
    if (nodes) {
      std::memcpy(nodes, r->nodes.data(), (size_t)r->offs[r->count] * 4);
      std::memcpy(edges, r->edges.data(), ((size_t)r->offs[r->count] - r->count) * 8);
    }
    return OPMOS_OK;
  });
}

int opmos_result_stats(const opmos_result* r, opmos_stats* out) {
  return guarded("opmos_result_stats", [&]() -> int {
    if (!r || !out) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    *out = r->stats;
    return OPMOS_OK;
  });
}

void opmos_result_free(opmos_result* r) { delete r; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Continuous-batching server: one persistent multi-query kernel stays
// resident; queries are queued through host-mapped memory and admitted as
// slots (arena + result pool, within the memory budget) free up; results are
// kept in their slot until the host collects them.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kServeSlotBytes = 512ull << 20;   // search arena per slot
constexpr size_t kServeOutWords = 8ull << 20;      // result pool per slot (32 MiB)
constexpr unsigned kServeHeurBlocks = 16;          // heuristic blocks left room beside the kernel
}  // namespace

struct opmos_server {
  std::mutex mu;
  std::vector<const opmos_graph*> graphs;
  opmos_graph shape{};  // largest n / degree, for arena planning
  uint32_t dmax = 0;
  unsigned nslots = 0, qcap = 0, blocks = 0;
  opmos_options o{};
  cudaStream_t kstream = nullptr, hstream = nullptr;
  char* dmem = nullptr;
  char* hmem = nullptr;
  uint32_t* hring = nullptr;  // heuristics of queued/running queries, qcap x dmax x nmax
  uint32_t* hscratch = nullptr;
  HJob* djobs = nullptr;
  unsigned* hkctr = nullptr;
  std::vector<uint32_t*> pool_words;  // per slot, device
  MQuery* hq = nullptr;               // host views of the mapped rings
  QResult* hres = nullptr;
  unsigned* hdone = nullptr;
  unsigned* hctl = nullptr;
  std::vector<uint8_t> inuse;
  std::vector<uint32_t> qd;  // objectives of each ring entry
  uint64_t next_ticket = 0;
  bool running = false;
};

namespace {

void server_free(opmos_server* sv) {
  if (sv->running) {
    *reinterpret_cast<volatile unsigned*>(&sv->hctl[HC_CLOSING]) = 2;  // stop now
    for (unsigned i = 0; i < sv->nslots; ++i) *reinterpret_cast<volatile unsigned*>(&sv->hctl[HC_RELEASE + i]) = 1;
    cudaStreamSynchronize(sv->kstream);
  }
  if (sv->dmem) cudaFree(sv->dmem);
  if (sv->hmem) cudaFreeHost(sv->hmem);
  if (sv->kstream) cudaStreamDestroy(sv->kstream);
  if (sv->hstream) cudaStreamDestroy(sv->hstream);
  delete sv;
}

}  // namespace

extern "C" {

int opmos_server_create(const opmos_graph* const* graphs, uint32_t ngraphs, const opmos_options* opt,
                        opmos_server** out) {
  return guarded("opmos_server_create", [&]() -> int {
    if (!out) return fail(OPMOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs == 0) return fail(OPMOS_ERR_INVALID_ARG, "no graphs");
    const DevInfo di = device_info();
    if (!di.ok) return fail(OPMOS_ERR_CUDA, "no CUDA device");
    auto* sv = new (std::nothrow) opmos_server;
    if (!sv) return fail(OPMOS_ERR_OUT_OF_MEMORY, "host allocation");
    opmos_options o = resolve(opt, true);
    if (!opt || !opt->mem_budget_bytes) o.mem_budget_bytes = 64ull << 30;
    sv->o = o;
    for (uint32_t i = 0; i < ngraphs; ++i) {
      if (!graphs[i]) {
        delete sv;
        return fail(OPMOS_ERR_INVALID_ARG, "graph %u is NULL", i);
      }
      sv->graphs.push_back(graphs[i]);
      sv->shape.n = std::max(sv->shape.n, graphs[i]->n);
      sv->shape.maxdeg = std::max(sv->shape.maxdeg, graphs[i]->maxdeg);
      sv->dmax = std::max(sv->dmax, graphs[i]->d);
    }
    uint32_t Dchk;
    {
      opmos_options oc = o;
      oc.d_used = 0;
      opmos_graph tmp = sv->shape;
      tmp.d = sv->dmax;
      if (int rc = check_options(oc, &tmp, &Dchk)) {
        delete sv;
        return rc;
      }
    }
    // a slot's search arena: 512 MiB, or what a query of label_budget labels
    // needs (labels take 30% of the part that grows) when that is more
    ArenaPlan pl;
    size_t slot_budget = kServeSlotBytes;
    if (o.label_budget) {
      if (int rc = plan_arena(&sv->shape, sv->dmax, o.window, 1ull << 40, true, &pl)) {
        delete sv;
        return rc;
      }
      const size_t per_label = 4 * (size_t)sv->dmax + 20;
      slot_budget = std::max<size_t>(slot_budget, pl.fixed + (8u << 20) + o.label_budget * per_label * 10 / 3);
    }
    if (int rc = plan_arena(&sv->shape, sv->dmax, o.window, slot_budget, true, &pl)) {
      delete sv;
      return rc;
    }
    const size_t slot_bytes = (pl.bytes + 255) / 256 * 256;
    const size_t pool_bytes = kServeOutWords * 4 + 256;
    const size_t per_slot = slot_bytes + pool_bytes;
    sv->nslots = (unsigned)std::min<size_t>(kMaxSlots, std::max<size_t>(1, o.mem_budget_bytes / per_slot));
    sv->qcap = std::max(64u, 2 * sv->nslots);
    const size_t hstride = (size_t)sv->dmax * sv->shape.n;
    const size_t spb = 5 * (size_t)sv->shape.n + 64;
    const size_t misc = sizeof(MCtl) + sv->graphs.size() * sizeof(GraphDev) + sv->nslots * (sizeof(MSlot) + sizeof(QCtl)) +
                        OPMOS_MAX_D * sizeof(HJob) + 64 + 32 * 256;
    const size_t dbytes = sv->nslots * per_slot + sv->qcap * hstride * 4 + kServeHeurBlocks * spb * 4 + misc;
    cudaError_t e = cudaMalloc(&sv->dmem, dbytes);
    if (e != cudaSuccess) {
      sv->dmem = nullptr;
      server_free(sv);
      return cuda_fail(e, "server device memory");
    }
    const size_t hbytes = sv->qcap * (sizeof(MQuery) + sizeof(QResult) + 4) + (HC_RELEASE + sv->nslots) * 4 + 8 * 256;
    e = cudaHostAlloc(&sv->hmem, hbytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
      sv->hmem = nullptr;
      server_free(sv);
      return cuda_fail(e, "server mapped host memory");
    }
    std::memset(sv->hmem, 0, hbytes);
    char* hp = sv->hmem;
    sv->hq = carve<MQuery>(hp, sv->qcap);
    sv->hres = carve<QResult>(hp, sv->qcap);
    sv->hdone = carve<unsigned>(hp, sv->qcap);
    sv->hctl = carve<unsigned>(hp, HC_RELEASE + sv->nslots);
    auto dev_of = [&](void* h) {
      void* d = nullptr;
      cudaHostGetDevicePointer(&d, h, 0);
      return d;
    };
    char* dp = sv->dmem;
    MCtl* M = carve<MCtl>(dp, 1);
    GraphDev* dgraphs = carve<GraphDev>(dp, sv->graphs.size());
    QCtl* ctls = carve<QCtl>(dp, sv->nslots);
    MSlot* dslots = carve<MSlot>(dp, sv->nslots);
    sv->djobs = carve<HJob>(dp, OPMOS_MAX_D);
    sv->hkctr = carve<unsigned>(dp, 16);
    sv->hscratch = carve<uint32_t>(dp, kServeHeurBlocks * spb);
    sv->hring = carve<uint32_t>(dp, sv->qcap * hstride);
    std::vector<MSlot> hslots(sv->nslots);
    for (unsigned i = 0; i < sv->nslots; ++i) {
      char* base = carve<char>(dp, per_slot);
      MSlot& sl = hslots[i];
      std::memset(&sl, 0, sizeof(sl));
      layout_arena(&sv->shape, sv->dmax, pl, base, &sl.A);
      char* pp = base + slot_bytes;
      unsigned long long* used = carve<unsigned long long>(pp, 1);
      uint32_t* words = carve<uint32_t>(pp, kServeOutWords);
      sl.O = OutPool{words, kServeOutWords, used};
      sv->pool_words.push_back(words);
      sl.P.window = o.window;
      sl.P.lanes = o.lanes_per_label;
      sl.P.delta = o.delta;
      sl.P.tile = o.tile;
      sl.P.label_budget = (uint32_t)std::min<uint64_t>(o.label_budget ? o.label_budget : ~0ull, pl.label_cap);
      sl.P.flags = o.flags;
      sl.P.qd = sv->dmax;
      sl.P.ps_grow = kMultiIndexGrow;
      sl.P.heavy_work = kHeavyWork;
      sl.P.part_work = kPartWork;
      sl.P.time_limit_ns = time_limit_ns();
      sl.state = SL_FREE;
    }
    std::vector<GraphDev> gd;
    for (auto* g : sv->graphs) gd.push_back(g->dev);
    MCtl hM{};
    hM.qcap = sv->qcap;
    hM.hold = 1;
    sv->inuse.assign(sv->qcap, 0);
    sv->qd.assign(sv->qcap, 0);
    e = cudaStreamCreateWithFlags(&sv->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->hstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpy(M, &hM, sizeof(MCtl), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dgraphs, gd.data(), gd.size() * sizeof(GraphDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctls, 0, sv->nslots * sizeof(QCtl));
    if (e == cudaSuccess) e = cudaMemcpy(dslots, hslots.data(), sv->nslots * sizeof(MSlot), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      server_free(sv);
      return cuda_fail(e, "server set-up");
    }
    const int occ = multi_occupancy(sv->dmax);
    const unsigned full = (unsigned)di.sms * (unsigned)std::min(occ, 2);
    sv->blocks = full > 2 * kServeHeurBlocks ? full - 2 * kServeHeurBlocks : std::max(1u, full / 2);
    e = launch_multi(sv->dmax, dslots, ctls, sv->nslots, (MQuery*)dev_of(sv->hq), (unsigned*)dev_of(sv->hctl), dgraphs,
                     (QResult*)dev_of(sv->hres), (unsigned*)dev_of(sv->hdone), M, sv->blocks, sv->kstream);
    if (e != cudaSuccess) {
      server_free(sv);
      return cuda_fail(e, "server kernel launch");
    }
    sv->running = true;
    *out = sv;
    return OPMOS_OK;
  });
}

int opmos_server_submit(opmos_server* sv, uint32_t graph, uint32_t d, uint32_t start, uint32_t goal,
                        uint64_t* ticket) {
  return guarded("opmos_server_submit", [&]() -> int {
    if (!sv || !ticket) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (graph >= sv->graphs.size()) return fail(OPMOS_ERR_INVALID_ARG, "graph %u out of range", graph);
    const opmos_graph* g = sv->graphs[graph];
    const uint32_t D = d ? d : g->d;
    if (D < 1 || D > g->d) return fail(OPMOS_ERR_INVALID_ARG, "d %u not in [1, %u]", D, g->d);
    if (start >= g->n || goal >= g->n) return fail(OPMOS_ERR_INVALID_ARG, "start/goal out of range");
    const uint64_t t = sv->next_ticket;
    const unsigned idx = (unsigned)(t % sv->qcap);
    if (sv->inuse[idx]) return fail(OPMOS_ERR_CAPACITY, "server queue full (%u outstanding queries)", sv->qcap);
    // the heuristic of this query, on the SMs the resident kernel leaves free
    uint32_t* h = sv->hring + (size_t)idx * sv->dmax * sv->shape.n;
    HJob jobs[OPMOS_MAX_D];
    for (uint32_t k = 0; k < D; ++k) jobs[k] = HJob{goal, k, h + (size_t)k * g->n};
    cudaStream_t s = sv->hstream;
    CK(cudaMemsetAsync(sv->hkctr, 0, 2 * sizeof(unsigned), s));
    CK(cudaMemcpyAsync(sv->djobs, jobs, D * sizeof(HJob), cudaMemcpyHostToDevice, s));
    CK(launch_heuristic(g->dev, sv->djobs, D, sv->hscratch, 5 * (size_t)sv->shape.n + 64,
                        std::min<unsigned>(D, kServeHeurBlocks), g->delta, sv->hkctr, sv->hkctr + 1, s));
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, sv->hkctr + 1, 4, cudaMemcpyDeviceToHost, s));
    // bounded wait: the heuristic runs on SMs the resident kernel leaves free
    const auto tw = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t q = cudaStreamQuery(s);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return cuda_fail(q, "server heuristic");
      if (std::chrono::steady_clock::now() - tw > std::chrono::seconds(30))
        return fail(OPMOS_ERR_TIMEOUT, "server heuristic did not finish within 30 s");
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (herr) return fail((int)herr, "heuristic kernel reported error %u", herr);
    MQuery q{graph, start, goal, D, h};
    sv->hq[idx] = q;
    sv->hdone[idx] = 0;
    sv->inuse[idx] = 1;
    sv->qd[idx] = D;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *reinterpret_cast<volatile unsigned*>(&sv->hctl[HC_TAIL]) = (unsigned)(t + 1);
    sv->next_ticket = t + 1;
    *ticket = t;
    return OPMOS_OK;
  });
}

int opmos_server_poll(opmos_server* sv, uint64_t ticket, opmos_result** out) {
  return guarded("opmos_server_poll", [&]() -> int {
    if (!sv || !out) return fail(OPMOS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(sv->mu);
    const unsigned idx = (unsigned)(ticket % sv->qcap);
    if (ticket >= sv->next_ticket || !sv->inuse[idx]) return fail(OPMOS_ERR_INVALID_ARG, "unknown ticket");
    if (!*reinterpret_cast<volatile unsigned*>(&sv->hdone[idx])) return OPMOS_PENDING;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    QResult R;
    std::memcpy(&R, (const void*)&sv->hres[idx], sizeof(R));
    const unsigned slot = R.slot;
    int rc = (int)R.status;
    if (rc == OPMOS_OK) {
      opmos_result* r = nullptr;
      rc = take_result(R, sv->qd[idx], !(sv->o.flags & OPMOS_FLAG_NO_PATHS), sv->pool_words[slot], sv->hstream, &r,
                       sv->dmax);
      if (rc == OPMOS_OK) {
        fill_stats(&r->stats, R, sv->qd[idx]);
        *out = r;
      }
    } else {
      search_status((unsigned)rc);
    }
    // the result has been copied: the slot may take the next query
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *reinterpret_cast<volatile unsigned*>(&sv->hctl[HC_RELEASE + slot]) = 1;
    sv->hdone[idx] = 0;
    sv->inuse[idx] = 0;
    return rc;
  });
}

void opmos_server_destroy(opmos_server* sv) {
  if (!sv) return;
  server_free(sv);
}

}  // extern "C"
