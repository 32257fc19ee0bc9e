// Serving: continuous batching of single-pattern probability requests.
//
// A host thread owns the device state. Requests wait in a bounded queue and
// are admitted into resident slots while a slot is free and the partial-sum
// arena (the device memory budget) has room for the request's work items.
// Every step takes a quota of work items from each resident request (round
// robin), runs them in one subset-kernel launch per precision, and finalises
// the requests whose last items are in that step; their results come back in
// the same step. Partial sums stay on the device between steps, so a large
// request is spread over several steps while small ones that arrive meanwhile
// are admitted, run beside it and finish first.
//
// A request's work items, their partial-sum slots and the order in which its
// partials are added depend only on its own n and precision, so its result is
// bit-for-bit the same whether it runs alone or among others.
//
// Steps are double-buffered (the host builds step k+1 while step k runs) and,
// by default, replayed as one instantiated CUDA graph per buffer. The graphs
// never change: a step's item and finalisation counts travel in a small header
// copied by the graph, the kernels read the step's items in place from the
// buffer's pinned (device-mapped) memory and exit at once when a count is
// zero, and the grids are the largest a step can use. A step is one graph
// launch, and its last copy writes the step's number into pinned host memory,
// which the server polls without a driver call. Every wait on the device is a
// bounded poll: past wait_timeout_s the server fails the outstanding requests
// with GBS_ETIMEDOUT and stops.
//
// A request with n >= kPairingMinN first waits for the ordering probe of the
// batched calls (run on a side stream, several waiting requests in one
// launch): its index list is stored in the chosen ordering, so its subset sum
// has the same cancellation, and so the same accuracy, as in gbs_prob_batch.
// The choice depends only on the request, so results stay the same alone and
// in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gbs_api_internal.h"

using namespace gbs;

namespace {

struct Request {
  int64_t ticket;
  int n;
  int prec;
  bool probed;  // the list is in its chosen ordering (n >= kPairingMinN)
  int idx[GBS_MAX_N];
};

constexpr int kProbeMax = 64;  // requests in one probe launch

struct Result {
  int rc;
  double p, hr, hi, err;
};

// First-fit allocator over the partial-sum arena [0, cap).
class Arena {
 public:
  void init(int cap) {
    cap_ = cap;
    free_.clear();
    free_.push_back({0, cap});
  }
  int capacity() const { return cap_; }
  int alloc(int len) {
    for (size_t i = 0; i < free_.size(); ++i)
      if (free_[i].len >= len) {
        const int s = free_[i].start;
        free_[i].start += len;
        free_[i].len -= len;
        if (free_[i].len == 0) free_.erase(free_.begin() + i);
        return s;
      }
    return -1;
  }
  void release(int start, int len) {
    size_t i = 0;
    while (i < free_.size() && free_[i].start < start) ++i;
    free_.insert(free_.begin() + i, {start, len});
    // coalesce neighbours
    if (i + 1 < free_.size() && free_[i].start + free_[i].len == free_[i + 1].start) {
      free_[i].len += free_[i + 1].len;
      free_.erase(free_.begin() + i + 1);
    }
    if (i > 0 && free_[i - 1].start + free_[i - 1].len == free_[i].start) {
      free_[i - 1].len += free_[i].len;
      free_.erase(free_.begin() + i);
    }
  }

 private:
  struct R {
    int start, len;
  };
  std::vector<R> free_;
  int cap_ = 0;
};

struct Slot {
  bool used = false;
  int64_t ticket = 0;
  int n = 0, prec = 0;
  std::vector<WorkItem> items;  // part = arena base + i, pat = slot index
  size_t next = 0;              // next item to dispatch
  int part_base = 0;
  bool finalize_sent = false;
  bool cancelled = false;  // its ticket is answered; the slot frees once no step in flight uses it
  int64_t last_step = 0;   // the last step that carried its items or its finalisation
  int pt = -1;             // FP64: element offset of its pair sums in the pool (-1: none)
  bool pt_ready = false;   // its pair sums are computed (by an earlier step)
};

constexpr int kStepCap = 65536;  // work items per precision per step
constexpr size_t kPtPoolBytes = (size_t)256 << 20;  // FP64 pair-sum pool

// The GPU's global nanosecond timer, for the step graph's start and end stamps.
__global__ void stamp_kernel(unsigned long long* out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

struct Stage {
  // pinned host: slot tables, items (2 precisions), selection list, step
  // header (item counts, finalisation count); results
  unsigned char* h_up = nullptr;
  unsigned char* h_up_dev = nullptr;  // the same memory as the device sees it
  double* h_res = nullptr;  // 5 S results, 2 timer stamps, the completion word (graph path)
  // device
  WorkItem* d_items[2] = {nullptr, nullptr};
  int* d_sel = nullptr;
  int* d_ctr = nullptr;  // [0..1] queue heads, [2..5] the step header (graph path)
  double* d_res = nullptr;
  cudaEvent_t ev = nullptr;   // the step's end
  cudaEvent_t ev0 = nullptr;  // its start on the stream (device time = ev - ev0)
  bool busy = false;
  int64_t id = 0;
  int n_items[2] = {0, 0};
  int n_pt_new = 0;      // slots whose pair sums this step computes
  std::vector<int> fin;  // slots finalised in this step, in selection order
  std::chrono::steady_clock::time_point t_launch;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t nd_t0 = nullptr, nd_t1 = nullptr, nd_pats = nullptr, nd_idx = nullptr, nd_hdr = nullptr, nd_ctr = nullptr,
                  nd_k[2] = {nullptr, nullptr}, nd_pt = nullptr, nd_ptk = nullptr, nd_sel = nullptr,
                  nd_fin = nullptr, nd_res = nullptr,
                  nd_done = nullptr, nd_ev = nullptr;
};

}  // namespace

struct gbs_server {
  const gbs_kernel* k = nullptr;
  int device = 0;
  gbs_serve_opts o;
  double log_norm = 0.0;
  cudaStream_t st = nullptr;
  TuneCfg cfg[2];
  int blocks_max[2] = {0, 0};
  // host state
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  bool failed = false;
  int fail_rc = GBS_ECUDA;  // why the server stopped (GBS_ETIMEDOUT or GBS_ECUDA)
  std::deque<Request> queue;
  // Results have their own lock (taken after mu, never before it), so that a
  // client polling in a tight loop contends only for the result table and
  // never holds up the server thread, which keeps mu while it admits, builds
  // and completes steps.
  std::mutex rmu;
  std::condition_variable rcv;                 // a result was added to done
  std::unordered_set<int64_t> pending;         // under rmu
  std::unordered_map<int64_t, Result> done;   // under rmu
  int64_t next_ticket = 1;
  std::vector<Slot> slots;
  Arena arena;
  int rr = 0;  // round-robin start
  int64_t step_id = 0;
  // device tables
  PatDesc* d_pats = nullptr;
  int* d_idx = nullptr;
  // FP64 pair sums (R_2 of every subset in one addition per entry, as in the
  // batched path): every FP64 request of order >= 6 holds its pair sums in a
  // pool (first fit, in complex elements) and is admitted only when they fit,
  // so its result never depends on the load; the step tables give each
  // slot's offset (-1: none) to the subset kernel and, for the slots whose
  // pair sums the step computes first, to the pair-term kernel
  double* d_pt = nullptr;
  Arena pt_arena;
  int64_t* d_pttab = nullptr;   // [0, S): all, [S, 2S): computed in this step
  Partial* d_parts = nullptr;
  std::vector<PatDesc> h_pats;
  std::vector<int> h_idx;
  size_t off_pats = 0, off_idx = 0, off_items[2] = {0, 0}, off_sel = 0, off_hdr = 0, off_pt = 0, up_bytes = 0;
  Stage stage[2];
  // ordering probe of requests with n >= kPairingMinN (side stream)
  cudaStream_t st_probe = nullptr;
  std::deque<Request> probe_wait;
  std::vector<Request> probing;  // in the probe launch in flight
  OrderProbe probe;
  bool probe_busy = false;
  std::chrono::steady_clock::time_point probe_t0;
  std::unordered_set<int64_t> probe_cancelled;  // cancelled while in the probe launch
  int64_t last_done_step = 0;  // the newest step whose completion was handled
  int fault_allocs = 0;        // injected allocation failures still to report
  std::thread th;
  gbs_serve_stats_t stats;
  // server-thread only (no lock): the last time the thread ran its loop or a
  // completion poll, and the longest interval between two such times
  std::chrono::steady_clock::time_point last_tick;
  double tick_gap_max = 0.0;
};

namespace {

int64_t binom64(int a, int b) {
  if (b < 0 || b > a) return 0;
  int64_t r = 1;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

// Work items of one request (slot index `si`), largest subsets first so the
// longest items start earliest: one lane-group round each in FP64; in the
// float kernel, whose rounds are short next to an item's fixed cost (series
// flush and double-double reduction), up to 4 rounds where a round holds 8 or
// more subsets and 2 where it holds 4 (at 78K req/s that kept the mixed
// stream's p99 at 6 ms instead of 55; in FP64 it only raised latency).
void request_items(const gbs_server* s, int si, int n, int prec, std::vector<WorkItem>& out) {
  out.clear();
  const int h = n / 2;
  const int cb = complex_bytes(prec);
  for (int sz = h; sz >= 1; --sz) {
    const int G = 32 / lanes_for(2 * sz, h, s->cfg[prec].warp_bytes, s->o.max_n / 2, cb);
    const int R = (prec == GBS_FP64) ? 1 : (G >= 8 ? 4 : (G >= 4 ? 2 : 1));
    const int64_t cnt = binom64(h, sz), cap = (int64_t)G * R;
    for (int64_t r0 = 0; r0 < cnt; r0 += cap) {
      WorkItem w;
      w.pat = si;
      w.s = sz;
      w.rank0 = (int)r0;
      w.count = (int)std::min<int64_t>(cap, cnt - r0);
      w.part = 0;
      w.stride = 1;
      w.s_last = 0;
      w.aux = 0;
      out.push_back(w);
    }
  }
}

// Launch arguments of a stage's subset kernel. In the step graph the kernel
// reads its items in place from the stage's pinned buffer and their count from
// the step header, so the graph's parameters never change between steps;
// direct launches pass the uploaded items and the count itself.
HafLaunch make_launch(gbs_server* s, Stage& g, int prec, bool graph) {
  HafLaunch L;
  memset(&L, 0, sizeof(L));
  L.src = s->k->B;
  L.src32 = (prec == GBS_MIXED) ? s->k->B32 : nullptr;
  L.idx = s->d_idx;
  L.pats = s->d_pats;
  if (graph) {
    L.items = (const WorkItem*)(g.h_up_dev + s->off_items[prec]);
    L.n_items_dev = g.d_ctr + 2 + prec;
  } else {
    L.items = g.d_items[prec];
    L.n_items = g.n_items[prec];
  }
  L.m_bound = 0;  // indices are checked on submit
  L.counter = g.d_ctr + prec;
  L.status = nullptr;
  L.parts = s->d_parts;
  L.warp_bytes = s->cfg[prec].warp_bytes;
  L.stage_h = s->o.max_n / 2;
  if (prec == GBS_FP64 && s->d_pt != nullptr) {
    L.pt = s->d_pt;
    L.pt_off = s->d_pttab;
  }
  return L;
}

// Launch arguments of the pair-term kernel: the slots whose offsets the
// step's second table gives (their first step); in the step graph it reads
// their count from the step header and returns at once when it is 0.
HafLaunch make_pt_launch(gbs_server* s, Stage& g, bool graph) {
  HafLaunch L;
  memset(&L, 0, sizeof(L));
  L.src = s->k->B;
  L.idx = s->d_idx;
  L.pats = s->d_pats;
  L.pt = s->d_pt;
  L.pt_off = s->d_pttab + s->o.max_slots;
  L.batch = s->o.max_slots;
  L.stage_h = s->o.max_n / 2;
  if (graph) L.n_items_dev = g.d_ctr + 6;
  return L;
}

FinalizeLaunch make_finalize(gbs_server* s, Stage& g, bool graph) {
  const int S = s->o.max_slots;
  FinalizeLaunch F;
  memset(&F, 0, sizeof(F));
  F.sel = g.d_sel;
  F.pats = s->d_pats;
  F.parts = s->d_parts;
  F.idx = s->d_idx;
  F.status = nullptr;
  if (graph)
    F.batch_dev = g.d_ctr + 4;
  else
    F.batch = (int)g.fin.size();
  F.precision = GBS_FP64;
  F.log_norm = s->k->dscal;
  F.p_out = g.d_res;
  F.logp_out = g.d_res + S;
  F.haf_out = g.d_res + 2 * S;
  F.kappa_out = g.d_res + 4 * S;
  F.err_out = nullptr;
  return F;
}

int grid_for(gbs_server* s, int prec, int n_items) {
  const int wpb = s->cfg[prec].warps_per_block;
  int b = (n_items + wpb - 1) / wpb;
  if (b > s->blocks_max[prec]) b = s->blocks_max[prec];
  return b < 1 ? 1 : b;
}

// Build the graph of one stage. Every node is fixed: the per-step counts
// travel in the step header (copied into d_ctr[2..4]), the kernels read their
// items from the stage's pinned buffer and exit at once when a count is zero,
// and the grids are the largest a step can use. A step is then one graph
// launch, with no parameter update.
cudaError_t build_graph(gbs_server* s, Stage& g) {
  cudaError_t e = cudaGraphCreate(&g.graph, 0);
  if (e != cudaSuccess) return e;
  const int S = s->o.max_slots;
  cudaGraphNode_t prev = nullptr;
  auto dep = [&](cudaGraphNode_t* deps) -> size_t {
    if (prev) {
      deps[0] = prev;
      return 1;
    }
    return 0;
  };
  cudaGraphNode_t deps[1];
  size_t nd;
  // the step's start and end are stamped with the GPU's timer by the graph
  // itself (device time without a driver call); its end event remains for
  // the error check of a long wait
  unsigned long long* d_stamp = (unsigned long long*)(g.d_res + 5 * S);
  auto add_stamp = [&](cudaGraphNode_t* node, unsigned long long* out) -> cudaError_t {
    void* args[1] = {&out};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)stamp_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    nd = dep(deps);
    return cudaGraphAddKernelNode(node, g.graph, deps, nd, &kp);
  };
  e = add_stamp(&g.nd_t0, d_stamp);
  if (e != cudaSuccess) return e;
  prev = g.nd_t0;
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_pats, g.graph, deps, nd, s->d_pats, g.h_up + s->off_pats,
                               sizeof(PatDesc) * S, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  prev = g.nd_pats;
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_idx, g.graph, deps, nd, s->d_idx, g.h_up + s->off_idx,
                               sizeof(int) * GBS_MAX_N * S, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  prev = g.nd_idx;
  cudaMemsetParams mp;
  memset(&mp, 0, sizeof(mp));
  mp.dst = g.d_ctr;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  nd = dep(deps);
  e = cudaGraphAddMemsetNode(&g.nd_ctr, g.graph, deps, nd, &mp);
  if (e != cudaSuccess) return e;
  prev = g.nd_ctr;
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_hdr, g.graph, deps, nd, g.d_ctr + 2, g.h_up + s->off_hdr, sizeof(int) * 5,
                               cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  prev = g.nd_hdr;
  if (s->d_pt != nullptr) {
    nd = dep(deps);
    e = cudaGraphAddMemcpyNode1D(&g.nd_pt, g.graph, deps, nd, s->d_pttab, g.h_up + s->off_pt,
                                 sizeof(int64_t) * 2 * S, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    prev = g.nd_pt;
    HafLaunch Lp = make_pt_launch(s, g, true);
    void* args[1] = {&Lp};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)pair_terms_kernel_fn();
    kp.gridDim = dim3(pair_terms_grid(Lp));
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    nd = dep(deps);
    e = cudaGraphAddKernelNode(&g.nd_ptk, g.graph, deps, nd, &kp);
    if (e != cudaSuccess) return e;
    prev = g.nd_ptk;
  }
  for (int p = 0; p < 2; ++p) {
    HafLaunch L = make_launch(s, g, p, true);
    void* args[1] = {&L};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)haf_kernel_fn(p);
    kp.gridDim = dim3(s->blocks_max[p]);
    kp.blockDim = dim3(s->cfg[p].warps_per_block * 32);
    kp.sharedMemBytes = s->cfg[p].warps_per_block * s->cfg[p].warp_bytes;
    kp.kernelParams = args;
    nd = dep(deps);
    e = cudaGraphAddKernelNode(&g.nd_k[p], g.graph, deps, nd, &kp);
    if (e != cudaSuccess) return e;
    prev = g.nd_k[p];
  }
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_sel, g.graph, deps, nd, g.d_sel, g.h_up + s->off_sel,
                               sizeof(int) * S, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  prev = g.nd_sel;
  {
    FinalizeLaunch F = make_finalize(s, g, true);
    void* args[1] = {&F};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)finalize_kernel_fn();
    kp.gridDim = dim3((unsigned)((S + 3) / 4));
    kp.blockDim = dim3(128);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    nd = dep(deps);
    e = cudaGraphAddKernelNode(&g.nd_fin, g.graph, deps, nd, &kp);
    if (e != cudaSuccess) return e;
    prev = g.nd_fin;
  }
  e = add_stamp(&g.nd_t1, d_stamp + 1);
  if (e != cudaSuccess) return e;
  prev = g.nd_t1;
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_res, g.graph, deps, nd, g.h_res, g.d_res, sizeof(double) * 5 * S + 16,
                               cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  prev = g.nd_res;
  nd = dep(deps);
  e = cudaGraphAddEventRecordNode(&g.nd_ev, g.graph, deps, nd, g.ev);
  if (e != cudaSuccess) return e;
  prev = g.nd_ev;
  // the completion word last: the step's number, copied back after its results
  // and its end event, so that the server sees a finished step without a
  // driver call
  nd = dep(deps);
  e = cudaGraphAddMemcpyNode1D(&g.nd_done, g.graph, deps, nd, g.h_res + 5 * S + 2, g.d_ctr + 5, sizeof(int),
                               cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&g.exec, g.graph, 0);
}

// Launch one prepared stage: the step header and one graph launch, or direct
// copies and launches.
// The longest parameter update (graph path) and the longest submission are
// kept in the stats.
void note_max(double& m, std::chrono::steady_clock::time_point t0) {
  const double d = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (d > m) m = d;
}

cudaError_t launch_stage(gbs_server* s, Stage& g) {
  const int S = s->o.max_slots;
  auto t0 = std::chrono::steady_clock::now();
  cudaError_t e;
  if (s->o.use_graphs) {
    // the whole step, its two events included, is one graph launch
    int* hdr = (int*)(g.h_up + s->off_hdr);
    hdr[0] = g.n_items[0];
    hdr[1] = g.n_items[1];
    hdr[2] = (int)g.fin.size();
    hdr[3] = (int)(g.id & 0x7fffffff);  // comes back in the completion word
    hdr[4] = g.n_pt_new;
    note_max(s->stats.update_max_s, t0);
    t0 = std::chrono::steady_clock::now();
    e = cudaGraphLaunch(g.exec, s->st);
    note_max(s->stats.submit_max_s, t0);
    return e;
  }
  e = cudaEventRecord(g.ev0, s->st);
  if (e != cudaSuccess) return e;
  {
    e = cudaMemcpyAsync(s->d_pats, g.h_up + s->off_pats, sizeof(PatDesc) * S, cudaMemcpyHostToDevice, s->st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(s->d_idx, g.h_up + s->off_idx, sizeof(int) * GBS_MAX_N * S, cudaMemcpyHostToDevice,
                        s->st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(g.d_ctr, 0, 2 * sizeof(int), s->st);
    if (e != cudaSuccess) return e;
    if (s->d_pt != nullptr) {
      e = cudaMemcpyAsync(s->d_pttab, g.h_up + s->off_pt, sizeof(int64_t) * 2 * S, cudaMemcpyHostToDevice, s->st);
      if (e != cudaSuccess) return e;
      if (g.n_pt_new > 0) {
        e = launch_pair_terms(make_pt_launch(s, g, false), s->st);
        if (e != cudaSuccess) return e;
      }
    }
    for (int p = 0; p < 2; ++p) {
      if (g.n_items[p] == 0) continue;
      e = cudaMemcpyAsync(g.d_items[p], g.h_up + s->off_items[p], sizeof(WorkItem) * g.n_items[p],
                          cudaMemcpyHostToDevice, s->st);
      if (e != cudaSuccess) return e;
      e = launch_haf_subsets(make_launch(s, g, p, false), p, grid_for(s, p, g.n_items[p]),
                             s->cfg[p].warps_per_block, s->st);
      if (e != cudaSuccess) return e;
    }
    if (!g.fin.empty()) {
      e = cudaMemcpyAsync(g.d_sel, g.h_up + s->off_sel, sizeof(int) * g.fin.size(), cudaMemcpyHostToDevice,
                          s->st);
      if (e != cudaSuccess) return e;
      e = launch_finalize(make_finalize(s, g, false), s->st);
      if (e != cudaSuccess) return e;
      e = cudaMemcpyAsync(g.h_res, g.d_res, sizeof(double) * 5 * S, cudaMemcpyDeviceToHost, s->st);
      if (e != cudaSuccess) return e;
    }
    note_max(s->stats.submit_max_s, t0);
  }
  return cudaEventRecord(g.ev, s->st);
}

void fail_all(gbs_server* s, int rc);

// Fail the given tickets with rc (lock held).
void fail_tickets(gbs_server* s, const std::vector<Request>& reqs, int rc) {
  std::lock_guard<std::mutex> rl(s->rmu);
  for (const Request& q : reqs) {
    Result r;
    r.rc = rc;
    r.p = r.hr = r.hi = r.err = NAN;
    s->done[q.ticket] = r;
    s->pending.erase(q.ticket);
  }
  s->rcv.notify_all();
}

// Ordering probe (lock held): collect a finished probe launch, whose requests
// go back to the front of the queue with their lists in the chosen ordering,
// and start the next one for the requests waiting. Returns false after a
// failure that stops the server.
bool probe_step(gbs_server* s) {
  if (s->probe_busy) {
    if (!order_probe_ready(s->probe)) {
      // no driver call while it runs (a probe takes well under a
      // millisecond); past 5 ms its event tells a failed launch from a slow one
      const double el =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - s->probe_t0).count();
      if (el < 5e-3) return true;
      const cudaError_t e = cudaEventQuery(s->probe.done);
      if (e != cudaSuccess && e != cudaErrorNotReady) {
        cudaGetLastError();
        fail_all(s, GBS_ECUDA);
        s->fail_rc = GBS_ECUDA;
        return false;
      }
      if (el <= s->o.wait_timeout_s) return true;
      fail_all(s, GBS_ETIMEDOUT);
      s->fail_rc = GBS_ETIMEDOUT;
      return false;
    }
    int pos[GBS_MAX_N];
    for (int i = (int)s->probing.size() - 1; i >= 0; --i) {
      Request& q = s->probing[i];
      if (s->probe_cancelled.erase(q.ticket)) continue;  // answered already
      if (order_probe_result(s->probe, i, pos)) {
        // the kernel reads position p of the list at default_pos(p, h): store
        // the list so that this gives source position pos[p]
        int y[GBS_MAX_N];
        for (int p = 0; p < q.n; ++p) y[default_pos(p, q.n / 2)] = q.idx[pos[p]];
        memcpy(q.idx, y, sizeof(int) * q.n);
      }
      q.probed = true;
      s->queue.push_front(q);
    }
    s->probing.clear();
    order_probe_release(&s->probe, s->st_probe);
    s->probe_busy = false;
  }
  if (!s->probe_busy && !s->probe_wait.empty()) {
    const int cnt = (int)std::min<size_t>(s->probe_wait.size(), kProbeMax);
    s->probing.assign(s->probe_wait.begin(), s->probe_wait.begin() + cnt);
    s->probe_wait.erase(s->probe_wait.begin(), s->probe_wait.begin() + cnt);
    const int* lists[kProbeMax];
    int ns[kProbeMax];
    for (int i = 0; i < cnt; ++i) {
      lists[i] = s->probing[i].idx;
      ns[i] = s->probing[i].n;
    }
    const int rc = order_probe_launch(s->k, lists, ns, cnt, s->o.max_n / 2, s->cfg[GBS_MIXED], s->st_probe,
                                      &s->probe);
    if (rc != GBS_OK) {
      fail_tickets(s, s->probing, rc);
      s->probing.clear();
      return true;
    }
    s->probe_busy = true;
    s->probe_t0 = std::chrono::steady_clock::now();
    s->stats.probed += cnt;
  }
  return true;
}

// Admit queued requests into free slots while the arena has room (lock held).
// A request that still needs the ordering probe moves to its waiting list.
void admit(gbs_server* s) {
  while (!s->queue.empty()) {
    if (s->queue.front().n >= kPairingMinN && !s->queue.front().probed) {
      s->probe_wait.push_back(s->queue.front());
      s->queue.pop_front();
      continue;
    }
    int si = -1;
    for (int i = 0; i < s->o.max_slots; ++i)
      if (!s->slots[i].used) {
        si = i;
        break;
      }
    if (si < 0) return;
    const Request& r = s->queue.front();
    Slot& sl = s->slots[si];
    request_items(s, si, r.n, r.prec, sl.items);
    if ((int64_t)sl.items.size() > s->arena.capacity()) {
      // more partial sums than the whole memory budget holds: it can never
      // be admitted, so it fails now instead of waiting forever
      fail_tickets(s, std::vector<Request>(1, r), GBS_ENOMEM);
      sl.items.clear();
      s->queue.pop_front();
      continue;
    }
    int base = -1;
    if (s->fault_allocs > 0) {
      --s->fault_allocs;  // injected failure: as if the budget were used up
    } else {
      base = s->arena.alloc((int)sl.items.size());
    }
    if (base < 0) {  // wait for memory to free up
      s->stats.alloc_waits++;
      sl.items.clear();
      return;
    }
    int pto = -1;
    if (r.prec == GBS_FP64 && s->d_pt != nullptr && pair_terms_elems(r.n) > 0) {
      pto = s->pt_arena.alloc((int)pair_terms_elems(r.n));
      if (pto < 0) {  // wait for pair-sum room to free up
        s->arena.release(base, (int)sl.items.size());
        s->stats.alloc_waits++;
        sl.items.clear();
        return;
      }
    }
    for (size_t i = 0; i < sl.items.size(); ++i) sl.items[i].part = base + (int)i;
    sl.used = true;
    sl.ticket = r.ticket;
    sl.n = r.n;
    sl.prec = r.prec;
    sl.next = 0;
    sl.part_base = base;
    sl.finalize_sent = false;
    sl.cancelled = false;
    sl.last_step = 0;
    sl.pt = pto;
    sl.pt_ready = false;
    PatDesc& d = s->h_pats[si];
    d.src_off = 0;
    d.idx_off = (int64_t)si * GBS_MAX_N;
    d.ld = s->k->m;
    d.n = r.n;
    d.item_begin = base;
    d.item_end = base + (int)sl.items.size();
    memcpy(&s->h_idx[(size_t)si * GBS_MAX_N], r.idx, sizeof(int) * r.n);
    s->queue.pop_front();
  }
}

// Fill a stage with this step's work (lock held). Returns true if it has work.
bool build_step(gbs_server* s, Stage& g) {
  const int S = s->o.max_slots;
  g.n_items[0] = g.n_items[1] = 0;
  g.fin.clear();
  memcpy(g.h_up + s->off_pats, s->h_pats.data(), sizeof(PatDesc) * S);
  memcpy(g.h_up + s->off_idx, s->h_idx.data(), sizeof(int) * GBS_MAX_N * S);
  WorkItem* it[2] = {(WorkItem*)(g.h_up + s->off_items[0]), (WorkItem*)(g.h_up + s->off_items[1])};
  int* sel = (int*)(g.h_up + s->off_sel);
  const int quota = s->o.subsets_per_step;
  const int64_t id = s->step_id + 1;
  // pair-sum offsets: every FP64 slot that has a region, and those whose pair
  // sums this step computes before its subset kernel (their first items)
  int64_t* pt_all = (int64_t*)(g.h_up + s->off_pt);
  int64_t* pt_new = pt_all + S;
  g.n_pt_new = 0;
  for (int q = 0; q < S; ++q) {
    const Slot& sl = s->slots[q];
    pt_all[q] = (sl.used && sl.pt >= 0) ? (int64_t)sl.pt : -1;
    pt_new[q] = -1;
  }
  for (int q = 0; q < S; ++q) {
    const int si = (s->rr + q) % S;
    Slot& sl = s->slots[si];
    if (!sl.used || sl.finalize_sent || sl.cancelled) continue;
    sl.last_step = id;
    if (sl.pt >= 0 && !sl.pt_ready && sl.next < sl.items.size()) {
      pt_new[si] = pt_all[si];
      sl.pt_ready = true;  // steps run in order on one stream
      ++g.n_pt_new;
    }
    int taken = 0;
    int& cnt = g.n_items[sl.prec];
    while (sl.next < sl.items.size() && taken < quota && cnt < kStepCap) {
      it[sl.prec][cnt++] = sl.items[sl.next];
      taken += sl.items[sl.next].count;
      ++sl.next;
    }
    if (sl.next == sl.items.size()) {
      sel[g.fin.size()] = si;
      g.fin.push_back(si);
      sl.finalize_sent = true;
    }
  }
  s->rr = (s->rr + 1) % S;
  g.id = ++s->step_id;  // == id
  return g.n_items[0] > 0 || g.n_items[1] > 0 || !g.fin.empty();
}

// Return a slot's partial sums and pair-sum region (no step in flight uses them).
void free_slot(gbs_server* s, Slot& sl) {
  s->arena.release(sl.part_base, (int)sl.items.size());
  if (sl.pt >= 0) s->pt_arena.release(sl.pt, (int)pair_terms_elems(sl.n));
  sl.pt = -1;
  sl.pt_ready = false;
  sl.used = false;
  sl.cancelled = false;
  sl.items.clear();
}

// Publish the results of a completed stage and free its finished slots (lock held).
void complete(gbs_server* s, Stage& g) {
  const int S = s->o.max_slots;
  std::lock_guard<std::mutex> rl(s->rmu);
  for (size_t b = 0; b < g.fin.size(); ++b) {
    Slot& sl = s->slots[g.fin[b]];
    if (sl.cancelled) {  // answered at cancellation: drop the result
      free_slot(s, sl);
      continue;
    }
    Result r;
    r.rc = GBS_OK;
    r.p = g.h_res[b];
    r.hr = g.h_res[2 * S + 2 * b];
    r.hi = g.h_res[2 * S + 2 * b + 1];
    const double kappa = g.h_res[4 * S + b];
    r.err = err_estimate(sl.prec, sl.n, kappa);
    s->done[sl.ticket] = r;
    s->pending.erase(sl.ticket);
    free_slot(s, sl);
  }
  s->rcv.notify_all();
  g.fin.clear();
  g.busy = false;
  s->last_done_step = std::max(s->last_done_step, g.id);
}

// Free the slots of cancelled requests that no step in flight uses (lock held).
void reap_cancelled(gbs_server* s) {
  for (Slot& sl : s->slots)
    if (sl.used && sl.cancelled && !sl.finalize_sent && sl.last_step <= s->last_done_step) free_slot(s, sl);
}

void fail_all(gbs_server* s, int rc) {
  std::lock_guard<std::mutex> rl(s->rmu);
  for (int64_t t : s->pending) {
    Result r;
    r.rc = rc;
    r.p = r.hr = r.hi = r.err = NAN;
    s->done[t] = r;
  }
  s->pending.clear();
  s->rcv.notify_all();
  s->queue.clear();
  s->probe_wait.clear();
  s->probing.clear();
  s->probe_cancelled.clear();
  for (auto& sl : s->slots) {
    if (sl.pt >= 0) s->pt_arena.release(sl.pt, (int)pair_terms_elems(sl.n));
    sl.pt = -1;
    sl.pt_ready = false;
    sl.used = false;
    sl.cancelled = false;
  }
}

// Bounded wait for a stage's event; false on timeout or error. The first
// half millisecond polls with yields only (a step takes ~0.1-1 ms, and a short
// sleep lasts tens of microseconds on Linux, which would add to every
// request's latency); after that it sleeps between polls.
// The server thread's responsiveness: the longest interval between two of its
// loop iterations or completion polls while a step is in flight (a
// descheduled or blocked thread shows here; a step that is slow on the device
// does not, nor does an idle server waiting for requests).
void tick(gbs_server* s) {
  const auto now = std::chrono::steady_clock::now();
  const double gap = std::chrono::duration<double>(now - s->last_tick).count();
  if ((s->stage[0].busy || s->stage[1].busy) && gap > s->tick_gap_max) s->tick_gap_max = gap;
  s->last_tick = now;
}

bool wait_stage(gbs_server* s, Stage& g, bool block) {
  const auto t0 = std::chrono::steady_clock::now();
  const int S = s->o.max_slots;
  for (;;) {
    tick(s);
    if (s->o.use_graphs) {
      // the graph's last copy writes the step's number: no driver call here
      if (*(volatile int*)(g.h_res + 5 * S + 2) == (int)(g.id & 0x7fffffff)) {
        std::atomic_thread_fence(std::memory_order_acquire);  // results before the word
        return true;
      }
      // a step still running after 5 ms (most take well under 1 ms) is also
      // checked with the driver, so that a failed step is reported at once
      if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > 5e-3) {
        const cudaError_t e = cudaEventQuery(g.ev);
        if (e != cudaSuccess && e != cudaErrorNotReady) return false;
      }
    } else {
      const cudaError_t e = cudaEventQuery(g.ev);
      if (e == cudaSuccess) return true;
      if (e != cudaErrorNotReady) return false;
    }
    if (!block) return false;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > s->o.wait_timeout_s) return false;
    if (el < 5e-4)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void serve_loop(gbs_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  s->last_tick = std::chrono::steady_clock::now();
  for (;;) {
    tick(s);
    s->stats.poll_gap_max_s = s->tick_gap_max;
    admit(s);
    if (!probe_step(s)) {
      s->failed = true;
      break;
    }
    reap_cancelled(s);
    admit(s);  // requests whose probe just finished, or whose slot freed
    bool any_work = false;
    for (const Slot& sl : s->slots)
      if (sl.used && !sl.finalize_sent && !sl.cancelled) any_work = true;
    Stage* free_stage = !s->stage[0].busy ? &s->stage[0] : (!s->stage[1].busy ? &s->stage[1] : nullptr);
    if (s->stop && !any_work && !s->stage[0].busy && !s->stage[1].busy && s->queue.empty() && !s->probe_busy &&
        s->probe_wait.empty())
      break;
    bool launched = false;
    if (any_work && free_stage && build_step(s, *free_stage)) {
      const auto tl0 = std::chrono::steady_clock::now();
      const cudaError_t e = launch_stage(s, *free_stage);
      const double tl = std::chrono::duration<double>(std::chrono::steady_clock::now() - tl0).count();
      if (tl > s->stats.launch_max_s) s->stats.launch_max_s = tl;
      if (e != cudaSuccess) {
        cudaGetLastError();
        fail_all(s, GBS_ECUDA);
        s->failed = true;
        break;
      }
      free_stage->busy = true;
      free_stage->t_launch = std::chrono::steady_clock::now();
      s->stats.steps++;
      for (int p = 0; p < 2; ++p) {
        s->stats.items += free_stage->n_items[p];
        const WorkItem* it = (const WorkItem*)(free_stage->h_up + s->off_items[p]);
        for (int q = 0; q < free_stage->n_items[p]; ++q) s->stats.subsets += it[q].count;
      }
      launched = true;
    }
    Stage* old = nullptr;
    for (int i = 0; i < 2; ++i)
      if (s->stage[i].busy && (!old || s->stage[i].id < old->id)) old = &s->stage[i];
    if (old) {
      // block on the oldest step when nothing new could be launched
      const bool block = !launched || (s->stage[0].busy && s->stage[1].busy);
      lk.unlock();
      const bool ok = wait_stage(s, *old, block);
      lk.lock();
      if (ok) {
        const double w = std::chrono::duration<double>(std::chrono::steady_clock::now() - old->t_launch).count();
        s->stats.step_wall_s += w;
        if (w > s->stats.step_wall_max_s) s->stats.step_wall_max_s = w;
        double dev_s = -1.0;
        if (s->o.use_graphs) {
          const unsigned long long* st = (const unsigned long long*)(old->h_res + 5 * s->o.max_slots);
          if (st[1] >= st[0]) dev_s = 1e-9 * (double)(st[1] - st[0]);
        } else {
          float dev_ms = 0.f;
          if (cudaEventElapsedTime(&dev_ms, old->ev0, old->ev) == cudaSuccess) dev_s = 1e-3 * dev_ms;
          else cudaGetLastError();
        }
        if (dev_s >= 0.0) {
          s->stats.step_device_s += dev_s;
          if (dev_s > s->stats.step_device_max_s) s->stats.step_device_max_s = dev_s;
        }
        s->stats.completed += (int64_t)old->fin.size();
        complete(s, *old);
        s->cv.notify_all();
      } else if (block) {
        // the wait gave up: a step that has finished meanwhile is taken
        // normally on the next pass; one still running, or failed, stops the
        // server
        const cudaError_t e = cudaEventQuery(old->ev);
        if (e != cudaSuccess) {
          cudaGetLastError();
          s->fail_rc = (e == cudaErrorNotReady) ? GBS_ETIMEDOUT : GBS_ECUDA;
          fail_all(s, s->fail_rc);
          s->failed = true;
          break;
        }
      }
    } else if (!launched) {
      if (s->probe_busy)  // a probe is in flight: poll it soon
        s->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
  s->cv.notify_all();
}

void destroy_resources(gbs_server* s) {
  for (int i = 0; i < 2; ++i) {
    Stage& g = s->stage[i];
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.ev) cudaEventDestroy(g.ev);
    if (g.ev0) cudaEventDestroy(g.ev0);
    if (g.h_up) cudaFreeHost(g.h_up);
    if (g.h_res) cudaFreeHost(g.h_res);
    if (g.d_items[0]) cudaFree(g.d_items[0]);
    if (g.d_sel) cudaFree(g.d_sel);
    if (g.d_ctr) cudaFree(g.d_ctr);
    if (g.d_res) cudaFree(g.d_res);
  }
  if (s->d_pats) cudaFree(s->d_pats);
  if (s->d_idx) cudaFree(s->d_idx);
  if (s->d_parts) cudaFree(s->d_parts);
  if (s->d_pt) cudaFree(s->d_pt);
  if (s->d_pttab) cudaFree(s->d_pttab);
  if (s->st_probe) {
    cudaStreamSynchronize(s->st_probe);
    order_probe_release(&s->probe, s->st_probe);
    order_probe_destroy(&s->probe);
    cudaStreamDestroy(s->st_probe);
  }
  if (s->st) cudaStreamDestroy(s->st);
}

}  // namespace

extern "C" int gbs_serve_create(const gbs_kernel* k, const gbs_serve_opts* opts, gbs_server** out) {
  clear_error();
  if (!k || !out) return fail(GBS_EINVAL, "null argument");
  *out = nullptr;
  gbs_server* s = new (std::nothrow) gbs_server();
  if (!s) return fail(GBS_ENOMEM, "host allocation");
  memset(&s->o, 0, sizeof(s->o));
  memset(&s->stats, 0, sizeof(s->stats));
  if (opts) s->o = *opts;
  if (s->o.max_slots <= 0) s->o.max_slots = 256;
  if (s->o.mem_budget == 0) s->o.mem_budget = (size_t)64 << 20;
  if (s->o.queue_capacity <= 0) s->o.queue_capacity = 65536;
  if (s->o.subsets_per_step <= 0) s->o.subsets_per_step = 8192;
  if (s->o.wait_timeout_s <= 0) s->o.wait_timeout_s = 10.0;
  if (s->o.max_n <= 0 || s->o.max_n > GBS_MAX_N) s->o.max_n = GBS_MAX_N;
  s->fault_allocs = s->o.fault_alloc_failures > 0 ? s->o.fault_alloc_failures : 0;
  s->o.use_graphs = (s->o.use_graphs >= 0) ? 1 : 0;
  s->k = k;
  s->device = k->device;
  int ret = GBS_OK;
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaSetDevice");
  }
  const int S = s->o.max_slots;
  do {
    e = cudaMemcpy(&s->log_norm, k->dscal, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { ret = cuda_fail(e, "log_norm"); break; }
    e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ret = cuda_fail(e, "stream"); break; }
    e = cudaStreamCreateWithFlags(&s->st_probe, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe stream"); break; }
    for (int p = 0; p < 2; ++p) {
      s->cfg[p] = default_cfg(p, s->o.max_n);
      const int smem = s->cfg[p].warps_per_block * s->cfg[p].warp_bytes;
      e = prepare_haf_kernel(p, smem);
      if (e != cudaSuccess) { ret = cuda_fail(e, "kernel attribute"); break; }
      s->blocks_max[p] = device_sm_count() * std::max(1, max_blocks_per_sm(p, s->cfg[p].warps_per_block, smem));
    }
    if (ret) break;
    // memory budget: slot tables, per-stage buffers, then the partial arena
    const size_t tables = sizeof(PatDesc) * S + sizeof(int) * GBS_MAX_N * S;
    const size_t stage_b = 2 * (2 * sizeof(WorkItem) * kStepCap + sizeof(int) * S + 256 + 5 * sizeof(double) * S);
    if (s->o.mem_budget <= tables + stage_b + 1024 * sizeof(Partial)) {
      ret = fail(GBS_EINVAL, "mem_budget %zu bytes is too small", s->o.mem_budget);
      break;
    }
    const size_t arena_items = std::min<size_t>((s->o.mem_budget - tables - stage_b) / sizeof(Partial),
                                                (size_t)1 << 30);
    s->arena.init((int)arena_items);
    s->stats.arena_slots = (int64_t)arena_items;
    if ((e = cudaMalloc(&s->d_pats, sizeof(PatDesc) * S)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_idx, sizeof(int) * GBS_MAX_N * S)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_parts, sizeof(Partial) * arena_items)) != cudaSuccess) {
      cudaGetLastError();
      ret = fail(GBS_ENOMEM, "device buffers: %s", cudaGetErrorString(e));
      break;
    }
    // FP64 pair-sum pool: kPtPoolBytes, or less when every slot holding a
    // request of the largest even order the server accepts needs less
    const int64_t pt_max = pair_terms_elems(s->o.max_n & ~1);
    if (pt_max > 0) {
      const int64_t elems = std::min<int64_t>((int64_t)S * pt_max, (int64_t)(kPtPoolBytes / 16));
      if ((e = cudaMalloc(&s->d_pt, 16 * (size_t)elems)) != cudaSuccess ||
          (e = cudaMalloc(&s->d_pttab, sizeof(int64_t) * 2 * S)) != cudaSuccess) {
        cudaGetLastError();
        ret = fail(GBS_ENOMEM, "pair-sum pool: %s", cudaGetErrorString(e));
        break;
      }
      s->pt_arena.init((int)elems);
    }
    s->h_pats.assign(S, PatDesc());
    memset(s->h_pats.data(), 0, sizeof(PatDesc) * S);
    s->h_idx.assign((size_t)GBS_MAX_N * S, 0);
    s->slots.assign(S, Slot());
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    s->off_pats = 0;
    s->off_idx = al(sizeof(PatDesc) * S);
    s->off_items[0] = s->off_idx + al(sizeof(int) * GBS_MAX_N * S);
    s->off_items[1] = s->off_items[0] + al(sizeof(WorkItem) * kStepCap);
    s->off_sel = s->off_items[1] + al(sizeof(WorkItem) * kStepCap);
    s->off_hdr = s->off_sel + al(sizeof(int) * S);
    s->off_pt = s->off_hdr + al(sizeof(int) * 8);
    s->up_bytes = s->off_pt + al(sizeof(int64_t) * 2 * S);
    for (int i = 0; i < 2 && ret == GBS_OK; ++i) {
      Stage& g = s->stage[i];
      if ((e = cudaMallocHost(&g.h_up, s->up_bytes)) != cudaSuccess ||
          (e = cudaMallocHost(&g.h_res, 5 * sizeof(double) * S + 32)) != cudaSuccess ||
          (e = cudaMalloc(&g.d_items[0], 2 * al(sizeof(WorkItem) * kStepCap))) != cudaSuccess ||
          (e = cudaMalloc(&g.d_sel, sizeof(int) * S)) != cudaSuccess ||
          (e = cudaMalloc(&g.d_ctr, 256)) != cudaSuccess ||
          (e = cudaMalloc(&g.d_res, 5 * sizeof(double) * S + 16)) != cudaSuccess ||
          (e = cudaEventCreate(&g.ev)) != cudaSuccess || (e = cudaEventCreate(&g.ev0)) != cudaSuccess) {
        cudaGetLastError();
        ret = fail(GBS_ENOMEM, "stage buffers: %s", cudaGetErrorString(e));
        break;
      }
      memset(g.h_up, 0, s->up_bytes);
      memset(g.h_res, 0, 5 * sizeof(double) * S + 32);  // completion word 0: no step has number 0
      g.d_items[1] = (WorkItem*)((unsigned char*)g.d_items[0] + al(sizeof(WorkItem) * kStepCap));
      if ((e = cudaHostGetDevicePointer((void**)&g.h_up_dev, g.h_up, 0)) != cudaSuccess) {
        cudaGetLastError();
        ret = fail(GBS_ECUDA, "pinned step buffer not mapped: %s", cudaGetErrorString(e));
        break;
      }
      if (s->o.use_graphs) {
        e = build_graph(s, g);
        if (e != cudaSuccess) {
          cudaGetLastError();
          ret = cuda_fail(e, "step graph");
          break;
        }
      }
    }
  } while (0);
  if (ret != GBS_OK) {
    destroy_resources(s);
    delete s;
    return ret;
  }
  s->th = std::thread(serve_loop, s);
  *out = s;
  return GBS_OK;
}

extern "C" int gbs_serve_submit(gbs_server* s, const int* idx, int n, int precision, int64_t* ticket) {
  clear_error();
  if (!s || !ticket || (n > 0 && !idx)) return fail(GBS_EINVAL, "null argument");
  if (precision != GBS_FP64 && precision != GBS_MIXED) return fail(GBS_EINVAL, "bad precision");
  if (n < 0 || n > s->o.max_n) return fail(GBS_ERANGE, "n = %d outside [0, %d]", n, s->o.max_n);
  for (int i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= s->k->m)
      return fail(GBS_ERANGE, "index %d = %d is outside [0, %d)", i, idx[i], s->k->m);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->failed)
    return fail(s->fail_rc, "server stopped after %s",
                s->fail_rc == GBS_ETIMEDOUT ? "a device wait timed out" : "an error");
  if (s->stop) return fail(GBS_EINVAL, "server is stopping");
  if (n == 0 || (n & 1)) {
    const int64_t t = s->next_ticket++;
    *ticket = t;
    // answered without device work: n = 0 is the vacuum (Haf = 1); odd n has
    // no perfect matching (Haf = 0)
    Result r;
    r.rc = GBS_OK;
    r.hr = (n == 0) ? 1.0 : 0.0;
    r.hi = 0.0;
    r.p = (n == 0) ? exp(-s->log_norm) : 0.0;
    r.err = 0.0;
    std::lock_guard<std::mutex> rl(s->rmu);
    s->done[t] = r;
    s->rcv.notify_all();
    return GBS_OK;
  }
  if ((int)s->queue.size() >= s->o.queue_capacity) return fail(GBS_EAGAIN, "queue full");
  const int64_t t = s->next_ticket++;
  *ticket = t;
  Request r;
  r.ticket = t;
  r.n = n;
  r.prec = precision;
  r.probed = false;
  memcpy(r.idx, idx, sizeof(int) * n);
  s->queue.push_back(r);
  {
    std::lock_guard<std::mutex> rl(s->rmu);
    s->pending.insert(t);
  }
  s->cv.notify_all();
  return GBS_OK;
}

extern "C" int gbs_serve_cancel(gbs_server* s, int64_t ticket) {
  clear_error();
  if (!s) return fail(GBS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  {
    std::lock_guard<std::mutex> rl(s->rmu);
    if (s->done.count(ticket)) return 1;  // finished (or failed): collect it with gbs_serve_poll
    if (!s->pending.count(ticket))
      return fail(GBS_ENOENT, "unknown or already collected ticket %lld", (long long)ticket);
  }
  bool found = false;
  for (auto it = s->queue.begin(); it != s->queue.end() && !found; ++it)
    if (it->ticket == ticket) {
      s->queue.erase(it);
      found = true;
      break;
    }
  for (auto it = s->probe_wait.begin(); it != s->probe_wait.end() && !found; ++it)
    if (it->ticket == ticket) {
      s->probe_wait.erase(it);
      found = true;
      break;
    }
  for (const Request& q : s->probing)
    if (!found && q.ticket == ticket) {
      s->probe_cancelled.insert(ticket);  // dropped when its probe launch returns
      found = true;
    }
  for (Slot& sl : s->slots)
    if (!found && sl.used && !sl.cancelled && sl.ticket == ticket) {
      // its steps in flight finish; no more are built, and the slot frees
      // once none is left
      sl.cancelled = true;
      found = true;
    }
  std::lock_guard<std::mutex> rl(s->rmu);
  Result r;
  r.rc = GBS_ECANCELED;
  r.p = r.hr = r.hi = r.err = NAN;
  s->done[ticket] = r;
  s->pending.erase(ticket);
  s->stats.cancelled++;
  s->rcv.notify_all();
  s->cv.notify_all();
  return GBS_OK;
}

extern "C" int gbs_serve_poll(gbs_server* s, int64_t ticket, double* p, double* haf_ri, double* err_est) {
  clear_error();
  if (!s) return fail(GBS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->rmu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (s->pending.count(ticket)) return 1;
    return fail(GBS_ENOENT, "unknown or already collected ticket %lld", (long long)ticket);
  }
  const Result r = it->second;
  s->done.erase(it);
  if (r.rc != GBS_OK)
    return fail(r.rc, "request failed (%s)",
                r.rc == GBS_ETIMEDOUT   ? "device wait timed out"
                : r.rc == GBS_ECANCELED ? "cancelled"
                : r.rc == GBS_ENOMEM    ? "needs more partial sums than the memory budget holds"
                                        : "CUDA error");
  if (p) *p = r.p;
  if (haf_ri) {
    haf_ri[0] = r.hr;
    haf_ri[1] = r.hi;
  }
  if (err_est) *err_est = r.err;
  return 0;
}

extern "C" int gbs_serve_wait_any(gbs_server* s, double timeout_s, int max, int64_t* tickets, double* p,
                                  double* haf_ri, double* err_est, int* rc, int* count) {
  clear_error();
  if (!s || !tickets || !count || max < 0 || !(timeout_s >= 0.0)) return fail(GBS_EINVAL, "invalid argument");
  *count = 0;
  std::unique_lock<std::mutex> lk(s->rmu);
  if (s->done.empty() && !s->pending.empty() && timeout_s > 0.0) {
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(std::min(timeout_s, 1e6)));
    s->rcv.wait_until(lk, until, [s] { return !s->done.empty() || s->pending.empty(); });
  }
  int k = 0;
  for (auto it = s->done.begin(); it != s->done.end() && k < max; ++k) {
    const Result& r = it->second;
    tickets[k] = it->first;
    if (p) p[k] = r.p;
    if (haf_ri) {
      haf_ri[2 * k] = r.hr;
      haf_ri[2 * k + 1] = r.hi;
    }
    if (err_est) err_est[k] = r.err;
    if (rc) rc[k] = r.rc;
    it = s->done.erase(it);
  }
  *count = k;
  return GBS_OK;
}

extern "C" int gbs_serve_stats(gbs_server* s, gbs_serve_stats_t* out) {
  clear_error();
  if (!s || !out) return fail(GBS_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return GBS_OK;
}

extern "C" int gbs_serve_destroy(gbs_server* s) {
  clear_error();
  if (!s) return GBS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->st);
  const bool failed = s->failed;
  const int frc = s->fail_rc;
  destroy_resources(s);
  delete s;
  return failed ? fail(frc, "server had stopped after %s",
                       frc == GBS_ETIMEDOUT ? "a device wait timed out" : "an error")
                : GBS_OK;
}
