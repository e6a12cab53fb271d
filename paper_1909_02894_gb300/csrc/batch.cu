// Batched stepping of many independent simulations (contexts) of uneven sizes.
//
// Contexts of the same grid size and precision form a class. One tick advances every
// active context by up to K steps through a device table of per-instance pointers
// [K steps][2 passes][capacity]. Each class launches, for each step, one x-pass and one
// y-pass over all its active contexts; with DIRAC_BATCH_TICK=1, a class of square
// complex64 grids whose passes run the persistent pass takes the whole tick in one
// persistent launch instead (work items with per-instance dependencies,
// line_pass_persistent's TICK mode). The classes run on parallel branches of a CUDA graph
// so that their work overlaps on the device. The graph of a tick is captured once per
// class layout (classes present and their table capacities) and replayed; between
// ticks only the tables and the active counts (device memory) change, so contexts are
// admitted and retired without re-capturing. Within a step, contexts are ordered by
// the number of steps they have left, so the contexts still running at step k of a
// tick are a prefix of the table.
//
// The trailing half-step of one step and the leading one of the next merge into U^2
// exactly as in dirac_step: a context's first step reads U at the x pass, its last step
// stores with U, all others store with U^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dirac.h"
#include "ctx.h"
#include "internal.h"

using namespace dgb;

namespace {

struct Class {
  int nx = 0, ny = 0;
  int capacity = 0;
  std::vector<int> members;  // slots of active contexts
  void* h_tab = nullptr;     // pinned host tables
  void* d_tab = nullptr;     // device tables
  int* h_count = nullptr;
  int* d_count = nullptr;
  cudaStream_t stream = nullptr;
  void* tw_x = nullptr;  // twiddle tables owned by the class (contexts come and go)
  void* tw_y = nullptr;
  void* tw_x_alt = nullptr;  // the same for the alternative radix schedule (if any)
  void* tw_y_alt = nullptr;
  int opt[2] = {-1, -1};  // CTA shape of the x / y pass chosen by the autotuner (-1: default)
  int* d_sync = nullptr;  // batched tick launch: per-slot done counters [capacity], queue
};

struct Slot {
  dirac_ctx* ctx = nullptr;
  long left = 0;
  long total = 0;
  double dt = 0.0;
  bool started = false;
  bool failed = false;  // a bounded device wait ran out while it was in the batch
  int state = 0;  // 0 free, 1 active, 2 finished (until released)
  unsigned long long finish_tick = 0;
};

}  // namespace

struct dirac_batch {
  dirac_precision prec = DIRAC_C64;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int steps_per_tick = 32;
  std::vector<Slot> slots;
  std::map<std::pair<int, int>, Class> classes;
  cudaGraphExec_t graph = nullptr;
  std::vector<std::pair<std::pair<int, int>, int>> graph_key;  // (class, capacity) list
  int graph_k = 0;
  long graph_kernels = 0;  // kernel nodes in the captured tick
  cudaEvent_t fork = nullptr, tick_done = nullptr;
  std::vector<cudaEvent_t> tick_events;  // per tick, recycled
  unsigned long long ticks = 0, ticks_done_seen = 0;
  int* d_err = nullptr;
  long launches = 0;
  // DIRAC_BATCH_TICK=1: one persistent launch per tick for the eligible classes (measured
  // 4-8% slower per class than per-step launches on the 256-instance mix, so not the
  // default)
  bool tick_launch = false;
  std::string err;
};

static dirac_status bfail(dirac_batch* b, dirac_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define BCK(call, where)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? DIRAC_ENOMEM : DIRAC_ECUDA,   \
                   std::string(where) + ": " + cudaGetErrorString(e_));               \
  } while (0)

template <typename T>
static size_t table_bytes(int K, int cap) {
  return (size_t)K * 2 * cap * sizeof(InstPtrs<T>);
}

static size_t tab_bytes(const dirac_batch* b, int cap) {
  return b->prec == DIRAC_C64 ? table_bytes<float>(b->steps_per_tick, cap)
                              : table_bytes<double>(b->steps_per_tick, cap);
}

static void free_class(Class& c) {
  if (c.h_tab) cudaFreeHost(c.h_tab);
  if (c.d_tab) cudaFree(c.d_tab);
  if (c.h_count) cudaFreeHost(c.h_count);
  if (c.d_count) cudaFree(c.d_count);
  if (c.stream) cudaStreamDestroy(c.stream);
  if (c.tw_x) cudaFree(c.tw_x);
  if (c.tw_y) cudaFree(c.tw_y);
  if (c.tw_x_alt) cudaFree(c.tw_x_alt);
  if (c.tw_y_alt) cudaFree(c.tw_y_alt);
  if (c.d_sync) cudaFree(c.d_sync);
  c = Class();
}

static dirac_status grow_class(dirac_batch* b, Class& c, int need) {
  if (c.capacity >= need) return DIRAC_OK;
  int cap = c.capacity ? c.capacity : 4;
  while (cap < need) cap *= 2;
  void *h = nullptr, *d = nullptr;
  int *hc = nullptr, *dc = nullptr, *ds = nullptr;
  BCK(cudaMallocHost(&h, tab_bytes(b, cap)), "batch tables");
  BCK(cudaMalloc(&d, tab_bytes(b, cap)), "batch tables");
  BCK(cudaMallocHost((void**)&hc, b->steps_per_tick * sizeof(int)), "batch counts");
  BCK(cudaMalloc((void**)&dc, b->steps_per_tick * sizeof(int)), "batch counts");
  BCK(cudaMalloc((void**)&ds, (cap + 1) * sizeof(int)), "batch tick counters");
  // the previous tables may still be read by an enqueued tick
  BCK(cudaStreamSynchronize(b->stream), "batch grow");
  if (c.h_tab) cudaFreeHost(c.h_tab);
  if (c.d_tab) cudaFree(c.d_tab);
  if (c.h_count) cudaFreeHost(c.h_count);
  if (c.d_count) cudaFree(c.d_count);
  if (c.d_sync) cudaFree(c.d_sync);
  c.h_tab = h;
  c.d_tab = d;
  c.h_count = hc;
  c.d_count = dc;
  c.d_sync = ds;
  c.capacity = cap;
  return DIRAC_OK;
}

// Fill the host tables of a class for one tick; returns the number of steps any of its
// contexts takes in this tick.
// Reads the device error flag (after the work it covers has completed). A bounded wait
// that ran out leaves every context then in the batch without a valid state: they are
// marked failed and stop stepping (poll reports DIRAC_ETIMEOUT until they are released),
// and the flag is cleared so that contexts submitted afterwards step normally.
static dirac_status batch_device_error(dirac_batch* b, const char* where) {
  int flag = 0;
  BCK(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
  if (DIRAC_DEBUG && dgb_debug_bounds())
    return bfail(b, DIRAC_ECUDA, "debug build: an index check of a line pass failed");
  if (!flag) return DIRAC_OK;
  BCK(cudaMemset(b->d_err, 0, sizeof(int)), "error flag");
  for (Slot& sl : b->slots) {
    if (sl.state == 0) continue;
    sl.failed = true;
    if (sl.state == 1) {
      sl.left = 0;
      sl.state = 2;
      sl.finish_tick = b->ticks ? b->ticks : 1;
    }
  }
  return bfail(b, DIRAC_ETIMEOUT, where);
}

template <typename T>
static int fill_class(dirac_batch* b, Class& c, int K) {
  std::vector<int>& m = c.members;
  std::stable_sort(m.begin(), m.end(),
                   [&](int x, int y) { return b->slots[x].left > b->slots[y].left; });
  InstPtrs<T>* tab = (InstPtrs<T>*)c.h_tab;
  int steps_used = 0;
  for (int k = 0; k < K; ++k) {
    int cnt = 0;
    for (int s : m) {
      const Slot& sl = b->slots[s];
      if (sl.left <= k) break;
      dirac_ctx* x = sl.ctx;
      InstPtrs<T>& px = tab[((size_t)k * 2 + 0) * c.capacity + cnt];
      InstPtrs<T>& py = tab[((size_t)k * 2 + 1) * c.capacity + cnt];
      px.in = (const Q4<T>*)x->psi;
      px.out = (Q4<T>*)x->psiT;
      px.beta = (const T*)x->beta1;
      px.u_load = (!x->u_identity && !sl.started && k == 0) ? (const Q4<T>*)x->u_n : nullptr;
      px.u_store = nullptr;
      px.mult = (const Q4<T>*)x->mult_x;
      px.mult_perm = (const Q4<T>*)x->mult_px;
      py.in = (const Q4<T>*)x->psiT;
      py.out = (Q4<T>*)x->psi;
      py.beta = (const T*)x->beta2T;
      py.u_load = nullptr;
      py.u_store = x->u_identity ? nullptr
                                 : (const Q4<T>*)(k + 1 == sl.left ? x->u_t : x->u2_t);
      py.mult = (const Q4<T>*)x->mult_y;
      py.mult_perm = (const Q4<T>*)x->mult_py;
      // failure-detection test hook (dirac_test_timeout_next_step): the first x pass of
      // the context in this tick waits for bytes that never arrive
      px.test_extra_tx = k == 0 ? x->test_timeout_next : 0u;
      py.test_extra_tx = 0u;
      if (k == 0) x->test_timeout_next = 0;
      ++cnt;
    }
    c.h_count[k] = cnt;
    if (cnt) steps_used = k + 1;
  }
  return steps_used;
}

template <typename T>
static dirac_status launch_class_step(dirac_batch* b, Class& c, int k, cudaStream_t st) {
  for (int pass = 0; pass < 2; ++pass) {
    LinePassArgs<T> a{};
    a.L = pass == 0 ? c.nx : c.ny;
    a.n_lines = pass == 0 ? c.ny : c.nx;
    a.sigma = pass;
    a.tw = (const Cx<T>*)(pass == 0 ? c.tw_x : c.tw_y);
    a.tw_alt = (const Cx<T>*)(pass == 0 ? c.tw_x_alt : c.tw_y_alt);
    a.err = b->d_err;
    a.inst = (const InstPtrs<T>*)c.d_tab + ((size_t)k * 2 + pass) * c.capacity;
    a.n_inst = c.d_count + k;
    a.inst_capacity = c.capacity;
    // the autotuner's choice, else: complex64 lines of 256 points or more the persistent
    // pass (its grid does not depend on the number of active instances), otherwise the
    // larger shape
    const int opt = c.opt[pass] >= 0 ? c.opt[pass] : (sizeof(T) == 4 && a.L >= 256) ? 2 : 1;
    BCK(launch_line_pass<T>(a, MODE_STEP, opt, st), "batched pass");
    b->launches += 1;
  }
  return DIRAC_OK;
}

// A class whose passes both run the persistent pass on square complex64 grids of
// 256..2048-point lines takes the whole tick in one persistent launch (work items with
// per-instance dependencies); the others launch each step's x and y passes.
template <typename T>
static bool class_tick_launch(const dirac_batch* b, const Class& c) {
  if (sizeof(T) != 4 || !b->tick_launch || c.nx != c.ny) return false;
  if (c.nx < 256 || c.nx > 2048) return false;
  for (int p = 0; p < 2; ++p)
    if (c.opt[p] != -1 && c.opt[p] != 2) return false;
  return true;
}

template <typename T>
static dirac_status launch_class_tick(dirac_batch* b, Class& c, int K, cudaStream_t st) {
  BCK(cudaMemsetAsync(c.d_sync, 0, (c.capacity + 1) * sizeof(int), st), "tick counters");
  LinePassArgs<T> a{};
  a.L = c.nx;
  a.n_lines = c.ny;
  a.sigma = 0;  // per work item
  a.tw = (const Cx<T>*)c.tw_x;  // the same table serves both passes (nx == ny)
  a.err = b->d_err;
  a.inst = (const InstPtrs<T>*)c.d_tab;
  a.n_inst = c.d_count;
  a.inst_capacity = c.capacity;
  a.tick_k = K;
  a.tick_done = c.d_sync;
  a.tick_queue = c.d_sync + c.capacity;
  BCK(launch_line_pass_tick<T>(a, st), "batched tick");
  b->launches += 1;
  return DIRAC_OK;
}

// Capture (or reuse) the graph of one tick for the current class layout.
template <typename T>
static dirac_status tick_graph(dirac_batch* b, int K) {
  std::vector<std::pair<std::pair<int, int>, int>> key;
  for (auto& kv : b->classes) key.push_back({kv.first, kv.second.capacity});
  if (b->graph && key == b->graph_key && K == b->graph_k) return DIRAC_OK;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  const long launches_before = b->launches;
  BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture");
  dirac_status st = DIRAC_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  std::vector<cudaEvent_t> joins;
  for (auto& kv : b->classes) {
    Class& c = kv.second;
    if (e != cudaSuccess || st != DIRAC_OK) break;
    e = cudaStreamWaitEvent(c.stream, b->fork, 0);
    if (e == cudaSuccess && class_tick_launch<T>(b, c)) {
      st = launch_class_tick<T>(b, c, K, c.stream);
    } else {
      for (int k = 0; k < K && e == cudaSuccess && st == DIRAC_OK; ++k)
        st = launch_class_step<T>(b, c, k, c.stream);
    }
    cudaEvent_t j = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, j, 0);
    if (j) joins.push_back(j);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  for (cudaEvent_t j : joins) cudaEventDestroy(j);
  if (st != DIRAC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, DIRAC_ECUDA, std::string("capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, DIRAC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  b->graph_key = key;
  b->graph_k = K;
  b->graph_kernels = b->launches - launches_before;
  b->launches = launches_before;  // counted when the graph runs
  return DIRAC_OK;
}

template <typename T>
static dirac_status run_tick(dirac_batch* b, int K) {
  // the pinned tables of the previous tick must have been copied before they are
  // rewritten: wait for the previous tick's copies (not its kernels)
  BCK(cudaEventSynchronize(b->tick_done), "batch tick");
  bool any = false;
  for (auto& kv : b->classes) {
    Class& c = kv.second;
    // drop finished members
    std::vector<int> keep;
    for (int s : c.members)
      if (b->slots[s].state == 1 && b->slots[s].left > 0) keep.push_back(s);
    c.members.swap(keep);
    dirac_status st = grow_class(b, c, (int)c.members.size() > 0 ? (int)c.members.size() : 1);
    if (st != DIRAC_OK) return st;
    const int used = fill_class<T>(b, c, K);
    if (used) any = true;
  }
  if (!any) return DIRAC_OK;
  dirac_status st = tick_graph<T>(b, K);
  if (st != DIRAC_OK) return st;
  for (auto& kv : b->classes) {
    Class& c = kv.second;
    BCK(cudaMemcpyAsync(c.d_tab, c.h_tab, tab_bytes(b, c.capacity), cudaMemcpyHostToDevice,
                        b->stream),
        "tables");
    BCK(cudaMemcpyAsync(c.d_count, c.h_count, K * sizeof(int), cudaMemcpyHostToDevice, b->stream),
        "counts");
  }
  BCK(cudaEventRecord(b->tick_done, b->stream), "tick");
  BCK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
  b->launches += b->graph_kernels;
  ++b->ticks;
  // bookkeeping: contexts finishing in this tick complete when the tick does
  cudaEvent_t ev = nullptr;
  BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "tick event");
  BCK(cudaEventRecord(ev, b->stream), "tick event");
  b->tick_events.push_back(ev);
  for (auto& kv : b->classes) {
    for (int s : kv.second.members) {
      Slot& sl = b->slots[s];
      const long n = sl.left < K ? sl.left : K;
      sl.left -= n;
      sl.started = true;
      if (sl.left == 0) {
        sl.state = 2;
        sl.finish_tick = b->ticks;  // 1-based index into tick_events
      }
    }
  }
  return DIRAC_OK;
}

// Shapes worth timing for a pass over lines of L points (the launcher maps the others onto
// these): complex64 256..4096 points also the persistent pass; lines of 32 points or
// fewer and 4096-point lines have one non-persistent shape.
template <typename T>
static std::vector<int> shape_candidates(int L) {
  std::vector<int> o;
  if (L >= 64 && L < 4096) o.push_back(0);
  o.push_back(1);
  if (sizeof(T) == 4 && L >= 256) o.push_back(2);
  if (line_pass_radix_alt<T>(L)) {  // the other radix schedule (3 smaller, 4 larger CTA)
    o.push_back(3);
    if ((sizeof(T) == 4 && L < 4096) || (sizeof(T) == 8 && L < 2048)) o.push_back(4);
  }
  return o;
}

// Times every candidate shape of both passes of one class over its stepping contexts.
// The launches read the states and write the contexts' second state buffers only (scratch
// between steps): the x pass as in a step, the y pass reading the state as if transposed
// (the same number of points), so no state changes.
template <typename T>
static dirac_status autotune_class(dirac_batch* b, Class& c, int reps, bool* changed) {
  std::vector<int> m;
  for (int s : c.members)
    if (b->slots[s].state == 1 && b->slots[s].left > 0) m.push_back(s);
  if (m.empty()) return DIRAC_OK;
  const int n = (int)m.size();
  std::vector<InstPtrs<T>> h(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const dirac_ctx* x = b->slots[m[i]].ctx;
    InstPtrs<T>& px = h[i];
    InstPtrs<T>& py = h[(size_t)n + i];
    px = InstPtrs<T>{};
    py = InstPtrs<T>{};
    px.in = py.in = (const Q4<T>*)x->psi;
    px.out = py.out = (Q4<T>*)x->psiT;
    px.beta = (const T*)x->beta1;
    py.beta = (const T*)x->beta2T;
    px.mult = (const Q4<T>*)x->mult_x;
    py.mult = (const Q4<T>*)x->mult_y;
    px.mult_perm = (const Q4<T>*)x->mult_px;
    py.mult_perm = (const Q4<T>*)x->mult_py;
    py.u_store = x->u_identity ? nullptr : (const Q4<T>*)x->u2_t;
  }
  InstPtrs<T>* d_tab = nullptr;
  int* d_cnt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dirac_status st = DIRAC_OK;
  auto cleanup = [&]() {
    if (d_tab) cudaFree(d_tab);
    if (d_cnt) cudaFree(d_cnt);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = cudaMalloc((void**)&d_tab, h.size() * sizeof(InstPtrs<T>));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_cnt, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(d_tab, h.data(), h.size() * sizeof(InstPtrs<T>), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_cnt, &n, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    LinePassArgs<T> a{};
    a.L = pass == 0 ? c.nx : c.ny;
    a.n_lines = pass == 0 ? c.ny : c.nx;
    a.sigma = pass;
    a.tw = (const Cx<T>*)(pass == 0 ? c.tw_x : c.tw_y);
    a.tw_alt = (const Cx<T>*)(pass == 0 ? c.tw_x_alt : c.tw_y_alt);
    a.err = b->d_err;
    a.inst = d_tab + (size_t)pass * n;
    a.n_inst = d_cnt;
    a.inst_capacity = n;
    float best = 0.f;
    int best_opt = -1;
    for (int o : shape_candidates<T>(a.L)) {
      e = launch_line_pass<T>(a, MODE_STEP, o, b->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = launch_line_pass<T>(a, MODE_STEP, o, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      b->launches += reps + 1;
      if (best_opt < 0 || ms < best) {
        best = ms;
        best_opt = o;
      }
    }
    if (e == cudaSuccess && best_opt != c.opt[pass]) {
      c.opt[pass] = best_opt;
      *changed = true;
    }
  }
  if (e != cudaSuccess)
    st = bfail(b, e == cudaErrorMemoryAllocation ? DIRAC_ENOMEM : DIRAC_ECUDA,
               std::string("batch autotune: ") + cudaGetErrorString(e));
  cleanup();
  return st;
}

extern "C" {

dirac_status dirac_batch_create(size_t hbm_budget_bytes, dirac_precision precision,
                                void* cuda_stream, int steps_per_tick, dirac_batch** out) {
  if (!out) return DIRAC_EINVAL;
  *out = nullptr;
  if (precision != DIRAC_C64 && precision != DIRAC_C128) return DIRAC_EINVAL;
  if (steps_per_tick < 1 || steps_per_tick > 1024) return DIRAC_EINVAL;
  dirac_batch* b = new (std::nothrow) dirac_batch();
  if (!b) return DIRAC_ENOMEM;
  b->prec = precision;
  b->budget = hbm_budget_bytes;
  {
    const char* t = getenv("DIRAC_BATCH_TICK");
    b->tick_launch = t && t[0] == '1' && t[1] == '\0';
  }
  b->steps_per_tick = steps_per_tick;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->tick_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(b->tick_done, b->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    dirac_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? DIRAC_ENOMEM : DIRAC_ECUDA;
  }
  *out = b;
  return DIRAC_OK;
}

dirac_status dirac_batch_submit(dirac_batch* b, dirac_ctx* inst, long n_steps, double dt,
                                int* slot) {
  if (!b) return DIRAC_EINVAL;
  if (!inst || !slot) return bfail(b, DIRAC_EINVAL, "inst and slot are required");
  *slot = -1;
  if (inst->prec != b->prec) return bfail(b, DIRAC_EINVAL, "precision differs from the batch");
  if (!inst->state_set) return bfail(b, DIRAC_ESTATE, "set_state must come before submit");
  if (inst->scheme != DIRAC_SCHEME_II)
    return bfail(b, DIRAC_EUNSUPPORTED, "the batch runs the printed sub-step order only");
  if (inst->has_pot || inst->beta1_im)
    return bfail(b, DIRAC_EUNSUPPORTED,
                 "the batch runs without static potentials and complex stretching");
  if (n_steps < 1) return bfail(b, DIRAC_EINVAL, "n_steps must be >= 1");
  if (!(dt > 0.0)) return bfail(b, DIRAC_EINVAL, "dt must be positive");
  for (const Slot& s : b->slots)
    if (s.state && s.ctx == inst) return bfail(b, DIRAC_ESTATE, "context already submitted");
  const size_t need = dgb_footprint_bytes(inst->nx, inst->ny, inst->prec);
  if (b->used + need > b->budget)
    return bfail(b, DIRAC_ENOMEM, "device-memory budget of the batch exhausted");
  // the context's work so far must be ordered before the batch's
  BCK(cudaStreamSynchronize(inst->stream), "submit");
  if (dt != inst->dt_cached) {
    dirac_status st = dgb_tables_for_dt(inst, dt);
    if (st != DIRAC_OK) return bfail(b, st, inst->err);
    BCK(cudaStreamSynchronize(inst->stream), "submit");
  }
  int s = -1;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (b->slots[i].state == 0) {
      s = i;
      break;
    }
  if (s < 0) {
    b->slots.push_back(Slot());
    s = (int)b->slots.size() - 1;
  }
  Slot& sl = b->slots[s];
  sl = Slot();
  sl.ctx = inst;
  sl.left = sl.total = n_steps;
  sl.dt = dt;
  sl.state = 1;
  b->used += need;
  auto key = std::make_pair(inst->nx, inst->ny);
  Class& c = b->classes[key];
  if (!c.stream) {
    c.nx = inst->nx;
    c.ny = inst->ny;
    BCK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "class stream");
    const size_t cx = b->prec == DIRAC_C64 ? sizeof(Cx<float>) : sizeof(Cx<double>);
    BCK(cudaMalloc(&c.tw_x, c.nx * cx), "class twiddles");
    BCK(cudaMalloc(&c.tw_y, c.ny * cx), "class twiddles");
    if (b->prec == DIRAC_C64) {
      BCK(launch_twiddles<float>(c.nx, line_pass_radix<float>(c.nx), (Cx<float>*)c.tw_x, b->stream), "twiddles");
      BCK(launch_twiddles<float>(c.ny, line_pass_radix<float>(c.ny), (Cx<float>*)c.tw_y, b->stream), "twiddles");
    } else {
      BCK(launch_twiddles<double>(c.nx, line_pass_radix<double>(c.nx), (Cx<double>*)c.tw_x, b->stream), "twiddles");
      BCK(launch_twiddles<double>(c.ny, line_pass_radix<double>(c.ny), (Cx<double>*)c.tw_y, b->stream), "twiddles");
    }
    const int ax = b->prec == DIRAC_C64 ? line_pass_radix_alt<float>(c.nx) : line_pass_radix_alt<double>(c.nx);
    const int ay = b->prec == DIRAC_C64 ? line_pass_radix_alt<float>(c.ny) : line_pass_radix_alt<double>(c.ny);
    if (ax) BCK(cudaMalloc(&c.tw_x_alt, c.nx * cx), "class twiddles");
    if (ay) BCK(cudaMalloc(&c.tw_y_alt, c.ny * cx), "class twiddles");
    if (b->prec == DIRAC_C64) {
      if (ax) BCK(launch_twiddles<float>(c.nx, ax, (Cx<float>*)c.tw_x_alt, b->stream), "twiddles");
      if (ay) BCK(launch_twiddles<float>(c.ny, ay, (Cx<float>*)c.tw_y_alt, b->stream), "twiddles");
    } else {
      if (ax) BCK(launch_twiddles<double>(c.nx, ax, (Cx<double>*)c.tw_x_alt, b->stream), "twiddles");
      if (ay) BCK(launch_twiddles<double>(c.ny, ay, (Cx<double>*)c.tw_y_alt, b->stream), "twiddles");
    }
    BCK(cudaStreamSynchronize(b->stream), "class twiddles");
  }
  c.members.push_back(s);
  *slot = s;
  return DIRAC_OK;
}

dirac_status dirac_batch_run(dirac_batch* b, int n_ticks) {
  if (!b) return DIRAC_EINVAL;
  for (int t = 0; t < n_ticks; ++t) {
    dirac_status st = b->prec == DIRAC_C64 ? run_tick<float>(b, b->steps_per_tick)
                                           : run_tick<double>(b, b->steps_per_tick);
    if (st != DIRAC_OK) return st;
  }
  return DIRAC_OK;
}

dirac_status dirac_batch_poll(dirac_batch* b, int slot, int* done) {
  if (!b || !done) return DIRAC_EINVAL;
  if (slot < 0 || slot >= (int)b->slots.size() || b->slots[slot].state == 0)
    return bfail(b, DIRAC_EINVAL, "no such slot");
  const Slot& sl = b->slots[slot];
  *done = 0;
  if (sl.state != 2) return DIRAC_OK;
  if (sl.finish_tick >= 1 && sl.finish_tick <= b->tick_events.size()) {
    cudaError_t e = cudaEventQuery(b->tick_events[sl.finish_tick - 1]);
    if (e == cudaErrorNotReady) return DIRAC_OK;
    if (e != cudaSuccess) return bfail(b, DIRAC_ECUDA, cudaGetErrorString(e));
  }
  if (sl.failed)
    return bfail(b, DIRAC_ETIMEOUT, "a bounded device wait ran out while this context was "
                                    "in the batch; its state is not valid");
  dirac_status st = batch_device_error(b, "a bounded device wait ran out in a batched pass; "
                                          "the contexts in the batch have no valid state");
  if (st != DIRAC_OK) return st;
  *done = 1;
  return DIRAC_OK;
}

dirac_status dirac_batch_release(dirac_batch* b, int slot) {
  if (!b) return DIRAC_EINVAL;
  if (slot < 0 || slot >= (int)b->slots.size() || b->slots[slot].state == 0)
    return bfail(b, DIRAC_EINVAL, "no such slot");
  Slot& sl = b->slots[slot];
  if (sl.state == 1) {
    // cancel: drop from its class before the next tick (steps already enqueued run)
    sl.left = 0;
  }
  BCK(cudaStreamSynchronize(b->stream), "release");
  b->used -= dgb_footprint_bytes(sl.ctx->nx, sl.ctx->ny, sl.ctx->prec);
  auto it = b->classes.find(std::make_pair(sl.ctx->nx, sl.ctx->ny));
  if (it != b->classes.end()) {
    std::vector<int>& m = it->second.members;
    m.erase(std::remove(m.begin(), m.end(), slot), m.end());
  }
  sl = Slot();
  return DIRAC_OK;
}

dirac_status dirac_batch_synchronize(dirac_batch* b) {
  if (!b) return DIRAC_EINVAL;
  BCK(cudaStreamSynchronize(b->stream), "synchronize");
  return batch_device_error(b, "a bounded device wait ran out in a batched pass; the "
                               "contexts in the batch have no valid state");
}

int dirac_batch_active(const dirac_batch* b) {
  if (!b) return 0;
  int n = 0;
  for (const Slot& s : b->slots) n += s.state == 1;
  return n;
}

long dirac_batch_launch_count(const dirac_batch* b) { return b ? b->launches : 0; }

const char* dirac_batch_last_error(const dirac_batch* b) { return b ? b->err.c_str() : ""; }

dirac_status dirac_batch_autotune(dirac_batch* b, int reps) {
  if (!b) return DIRAC_EINVAL;
  if (reps < 1) return bfail(b, DIRAC_EINVAL, "reps must be >= 1");
  BCK(cudaStreamSynchronize(b->stream), "batch autotune");
  bool changed = false;
  for (auto& kv : b->classes) {
    dirac_status st = b->prec == DIRAC_C64 ? autotune_class<float>(b, kv.second, reps, &changed)
                                           : autotune_class<double>(b, kv.second, reps, &changed);
    if (st != DIRAC_OK) return st;
  }
  {
    dirac_status st = batch_device_error(b, "a bounded device wait ran out in a timed pass");
    if (st != DIRAC_OK) return st;
  }
  if (changed && b->graph) {  // the next tick captures a graph with the new shapes
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_key.clear();
  }
  return DIRAC_OK;
}

dirac_status dirac_batch_launch_shape(const dirac_batch* b, int nx, int ny, int* threads_x,
                                      int* threads_y) {
  if (!b || !threads_x || !threads_y) return DIRAC_EINVAL;
  auto it = b->classes.find(std::make_pair(nx, ny));
  if (it == b->classes.end()) return DIRAC_EINVAL;
  static const int th[5] = {256, 512, 1024, 256 | DIRAC_LAUNCH_ALT_RADIX,
                            512 | DIRAC_LAUNCH_ALT_RADIX};
  const int L[2] = {nx, ny};
  int* out[2] = {threads_x, threads_y};
  for (int p = 0; p < 2; ++p) {
    const int o = it->second.opt[p];
    *out[p] = th[o >= 0 ? o : (b->prec == DIRAC_C64 && L[p] >= 256) ? 2 : 1];
  }
  return DIRAC_OK;
}

void dirac_batch_destroy(dirac_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& kv : b->classes) free_class(kv.second);
  for (cudaEvent_t e : b->tick_events) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->tick_done) cudaEventDestroy(b->tick_done);
  if (b->d_err) cudaFree(b->d_err);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
