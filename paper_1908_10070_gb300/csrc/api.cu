// C ABI entry points: kernel matrix, batched Hafnians and probabilities, and
// the launch planner shared with the serving loop and the autotuner.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gbs_api_internal.h"

namespace gbs {

// ------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------
static thread_local std::string t_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

void clear_error() { t_err.clear(); }

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GBS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------------
// device memory: one stream-ordered pool per device, kept warm
// ------------------------------------------------------------------------
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaError_t get_pool(int dev, cudaMemPool_t* out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  cudaError_t e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return e;
  uint64_t thr = ~0ull;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e != cudaSuccess) return e;
  g_pools[dev] = pool;
  *out = pool;
  return cudaSuccess;
}

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  e = get_pool(dev, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes < 256 ? 256 : bytes, pool, st);
}

cudaError_t scratch_free(void* p, cudaStream_t st) { return p ? cudaFreeAsync(p, st) : cudaSuccess; }

// ------------------------------------------------------------------------
// pinned host staging: a small ring of buffers, each reused once the copy
// that last read it has completed on the device
// ------------------------------------------------------------------------
struct PinnedSlot {
  void* ptr = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool busy = false;
};
static std::mutex g_pin_mu;
static std::vector<PinnedSlot> g_pin;

int pinned_acquire(size_t bytes, void** ptr, int* slot) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  int pick = -1;
  for (size_t i = 0; i < g_pin.size(); ++i) {
    PinnedSlot& s = g_pin[i];
    if (s.busy) continue;
    if (s.ev && cudaEventQuery(s.ev) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (s.cap >= bytes) {
      pick = (int)i;
      break;
    }
  }
  if (pick < 0) {
    // grow a free slot, or add one (at most 32; then wait for slot 0)
    for (size_t i = 0; i < g_pin.size() && pick < 0; ++i) {
      PinnedSlot& s = g_pin[i];
      if (s.busy) continue;
      if (s.ev && cudaEventQuery(s.ev) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      pick = (int)i;
    }
    if (pick < 0 && g_pin.size() < 32) {
      g_pin.push_back(PinnedSlot());
      pick = (int)g_pin.size() - 1;
    }
    if (pick < 0) {
      for (size_t i = 0; i < g_pin.size() && pick < 0; ++i)
        if (!g_pin[i].busy) pick = (int)i;
      if (pick < 0) return fail(GBS_EAGAIN, "all pinned staging buffers are in use");
      cudaEventSynchronize(g_pin[pick].ev);
    }
    PinnedSlot& s = g_pin[pick];
    if (s.cap < bytes) {
      if (s.ptr) cudaFreeHost(s.ptr);
      s.ptr = nullptr;
      s.cap = 0;
      size_t cap = 1 << 20;
      while (cap < bytes) cap <<= 1;
      cudaError_t e = cudaMallocHost(&s.ptr, cap);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
      s.cap = cap;
    }
    if (!s.ev) {
      cudaError_t e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
  }
  g_pin[pick].busy = true;
  *ptr = g_pin[pick].ptr;
  *slot = pick;
  return GBS_OK;
}

void pinned_release(int slot, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (slot < 0 || slot >= (int)g_pin.size()) return;
  cudaEventRecord(g_pin[slot].ev, st);
  g_pin[slot].busy = false;
}

// ------------------------------------------------------------------------
// launch shapes
// ------------------------------------------------------------------------
static std::mutex g_tune_mu;
bool shape_fits(int precision, int warp_bytes, int maxn);
static std::map<std::pair<int, int>, TuneCfg> g_tuned;  // (precision, n) -> cfg

// Default launch shape for photon number n: the most warps per block (6 down
// to 2, one block per SM) whose per-warp shared memory still holds every lane
// group that n can need.
TuneCfg default_cfg(int precision, int n) {
  static const int optin = [] {  // thread-safe one-time initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 232448;  // 227 KB, the GB300 opt-in limit
    }
    return v;
  }();
  TuneCfg c;
  c.rounds = (n >= 24) ? 2 : 4;
  for (int wpb = 6; wpb >= 2; --wpb) {
    c.warps_per_block = wpb;
    c.warp_bytes = ((optin - 4096) / wpb) & ~127;
    if (shape_fits(precision, c.warp_bytes, n < 2 ? 2 : n)) break;
  }
  return c;
}

// default_cfg per (precision, n), computed once (g_tune_mu held)
static const TuneCfg& default_cfg_cached(int precision, int n) {
  static TuneCfg table[2][kMaxN + 1];
  static bool ready[2] = {false, false};
  const int p = precision == GBS_FP64 ? 0 : 1;
  if (!ready[p]) {
    for (int v = 0; v <= kMaxN; ++v) table[p][v] = default_cfg(precision, v);
    ready[p] = true;
  }
  return table[p][n < 0 ? 0 : (n > kMaxN ? kMaxN : n)];
}

TuneCfg get_cfg(int precision, int n) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_pair(precision, n));
  if (it != g_tuned.end()) return it->second;
  return default_cfg_cached(precision, n);
}

// Rounds per item for every order 0..kMaxN (one lock for all of them).
static void get_rounds(int precision, int* rounds) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int v = 0; v <= kMaxN; ++v) {
    auto it = g_tuned.find(std::make_pair(precision, v));
    rounds[v] = (it != g_tuned.end()) ? it->second.rounds : default_cfg_cached(precision, v).rounds;
  }
}

void set_cfg(int precision, int n, const TuneCfg& c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[std::make_pair(precision, n)] = c;
}

int complex_bytes(int precision) { return precision == GBS_FP64 ? 16 : 8; }

// Every order that a batch with largest photon number maxn can need fits the
// warp's shared bytes (the largest group is N = n, h = n/2 for each n).
bool shape_fits(int precision, int warp_bytes, int maxn) {
  const int cb = complex_bytes(precision);
  for (int n = 2; n <= maxn; n += 2)
    if (lanes_for(n, n / 2, warp_bytes, maxn / 2, cb) == 0) return false;
  return true;
}

int64_t binom64(int a, int b) {
  if (b < 0 || b > a) return 0;
  int64_t r = 1;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

// Work-item planning in two passes over per-n templates. Every matrix of order
// n gets the same list of items (subset size s, first colex rank, count); items
// of one matrix take consecutive partial slots (pattern order), and the
// schedule lists the most expensive items first (longest-first list
// scheduling) by bucketing on (s, rounds), whose cost is rounds * (2s)^3.


// Estimated cost of a bucket key: size s * 65 + rounds for per-size items
// (rounds * s^3), 0 * 65 + h for whole-matrix items (sum_s C(h, s) s^3).
static int64_t key_cost(int key) {
  const int64_t sz = key / 65, r = key % 65;
  if (sz > 0) return r * sz * sz * sz;
  int64_t c = 0;
  for (int s = 1; s <= r; ++s) c += binom64((int)r, s) * s * s * s;
  return c;
}

void Planner::init(const int* n, int batch, int precision, int warp_bytes, const int* rounds_for_n,
                   int64_t whole_reserve) {
  n_ = n;
  batch_ = batch;
  const int cb = complex_bytes(precision);
  int maxn = 0;
  for (int b = 0; b < batch; ++b) maxn = std::max(maxn, n[b]);
  const int stage_h = maxn / 2;
  for (int v = 0; v <= kMaxN; ++v) {
    tmpl_[v].clear();
    npat_[v] = 0;
    nwhole_[v] = 0;
  }
  for (int b = 0; b < batch; ++b) npat_[n[b]]++;
  std::fill(bucket_, bucket_ + kKeys, 0);
  total_ = 0;
  for (int v = 2; v <= kMaxN; v += 2) {
    if (!npat_[v]) continue;
    const int h = v / 2, R = rounds_for_n[v];
    if (whole_reserve > 0 && v >= 4 && v <= kWholeMaxN && npat_[v] >= 2 * whole_reserve)
      nwhole_[v] = npat_[v] - whole_reserve;
    const int64_t nsplit = npat_[v] - nwhole_[v];
    if (nwhole_[v]) {
      bucket_[h] += nwhole_[v];  // size 0 row of the key table: whole-matrix items of half order h
      total_ += nwhole_[v];
    }
    for (int sz = 1; sz <= h; ++sz) {
      const int G = 32 / lanes_for(2 * sz, h, warp_bytes, stage_h, cb);
      const int64_t cnt = binom64(h, sz), cap = (int64_t)G * R;
      for (int64_t r0 = 0; r0 < cnt; r0 += cap) {
        ItemTemplate t;
        t.s = sz;
        t.s_last = sz;
        t.rank0 = (int)r0;
        t.count = (int)std::min<int64_t>(cap, cnt - r0);
        const int rnds = std::min((t.count + G - 1) / G, 64);
        t.key = sz * 65 + rnds;
        tmpl_[v].push_back(t);
        bucket_[t.key] += nsplit;
      }
    }
    total_ += (int64_t)tmpl_[v].size() * nsplit;
  }
  whole_.assign(batch, 0);
  int64_t seen[kMaxN + 1] = {0};
  for (int b = 0; b < batch; ++b) {
    const int v = n[b];
    if (v < 4 || (v & 1)) continue;
    whole_[b] = (seen[v]++ < nwhole_[v]) ? 1 : 0;
  }
  // bucket start offsets, most expensive key first
  int order[kKeys];
  int nk = 0;
  for (int k = 0; k < kKeys; ++k)
    if (bucket_[k]) order[nk++] = k;
  std::sort(order, order + nk, [](int x, int y) {
    const int64_t cx = key_cost(x), cy = key_cost(y);
    return cx != cy ? cx > cy : x < y;
  });
  int64_t acc = 0;
  for (int q = 0; q < nk; ++q) {
    start_[order[q]] = acc;
    acc += bucket_[order[q]];
  }
}

void Planner::fill(PatDesc* pats, WorkItem* items) {
  int64_t next[kKeys];
  std::copy(start_, start_ + kKeys, next);
  int q = 0;
  for (int b = 0; b < batch_; ++b) {
    PatDesc& d = pats[b];
    const int v = n_[b];
    d.n = v;
    d.item_begin = q;
    if (whole_[b]) {
      const int h = v / 2;
      WorkItem& w = items[next[h]++];
      w.pat = b;
      w.s = 1;
      w.rank0 = 0;
      w.count = (1 << h) - 1;
      w.part = q++;
      w.stride = 1;
      w.s_last = h;  // every subset of the matrix
      w.aux = 0;
    } else if (v >= 2 && !(v & 1)) {
      for (const ItemTemplate& t : tmpl_[v]) {
        WorkItem& w = items[next[t.key]++];
        w.pat = b;
        w.s = t.s;
        w.rank0 = t.rank0;
        w.count = t.count;
        w.part = q++;
        w.stride = 1;
        w.s_last = 0;
        w.aux = 0;
      }
    }
    d.item_end = q;
  }
}

// ------------------------------------------------------------------------
// pairing probe
// ------------------------------------------------------------------------
// The subset sum pairs positions (2t, 2t+1) of each matrix; the Hafnian does
// not depend on that choice, but the size of the signed terms does, and with
// it the rounding error of the sum, which grows with sum |f| / |Haf|. For
// matrices with n >= kPairingMinN the library tries kPairingCands orderings
// (the default one and seeded random ones, the same for every matrix of an
// order) on a systematic sample of kProbePerSize subsets of each size from
// ceil(h/2) to h-3 (where most of sum |f| lies), and runs the full sum in the
// ordering with the smallest estimate. The sample costs a few per cent of
// the full sum at these orders.
constexpr int kPairingCands = 16;
constexpr int kProbePerSize = 8;
static_assert(kProbePerSize < kMaxProbeSample, "probe sample count must index the reciprocal table");

struct PairingPlan {
  std::vector<int> sel;             // probed matrices (batch indices)
  std::vector<int> perm;            // candidate orderings, per order n
  std::vector<PatDesc> pats;        // probe matrices (source fields filled later)
  std::vector<WorkItem> items;      // their sampled items, part slot = index
  std::vector<int> perm_off;        // ordering of each probe matrix
};

static uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Probe items hold one round of lane groups each (G subsets of one size), so
// that the samples of one matrix run in parallel warps.
static void plan_pairing(const int* n, int batch, int precision, int warp_bytes, int stage_h,
                         PairingPlan* pp) {
  const int cb = complex_bytes(precision);
  int base[kMaxN + 1];
  for (int v = 0; v <= kMaxN; ++v) base[v] = -1;
  for (int b = 0; b < batch; ++b)
    if (n[b] >= kPairingMinN && !(n[b] & 1)) pp->sel.push_back(b);
  if (pp->sel.empty()) return;
  for (int b : pp->sel) {
    const int v = n[b];
    if (base[v] >= 0) continue;
    base[v] = (int)pp->perm.size();
    for (int c = 0; c < kPairingCands; ++c) {
      const size_t o = pp->perm.size();
      for (int i = 0; i < v; ++i) pp->perm.push_back(default_pos(i, v / 2));
      uint64_t state = 0x5eedull * 1000003ull + (uint64_t)v * 1009ull + (uint64_t)c;
      for (int i = v - 1; c > 0 && i > 0; --i) {  // Fisher-Yates; candidate 0 stays the default order
        const int j = (int)(splitmix64(state) % (uint64_t)(i + 1));
        std::swap(pp->perm[o + i], pp->perm[o + j]);
      }
    }
  }
  for (size_t k = 0; k < pp->sel.size(); ++k) {
    const int v = n[pp->sel[k]], h = v / 2;
    for (int c = 0; c < kPairingCands; ++c) {
      PatDesc d;
      memset(&d, 0, sizeof(d));
      d.n = v;
      d.item_begin = (int)pp->items.size();
      const int q = (int)pp->pats.size();
      for (int sz = (h + 1) / 2; sz <= h - 3; ++sz) {
        const int64_t cs = binom64(h, sz);
        const int K = (int)std::min<int64_t>(cs, kProbePerSize);
        const int stride = (int)(cs / K);
        const int G = 32 / lanes_for(2 * sz, h, warp_bytes, stage_h, cb);
        for (int j = 0; j < K; j += G) {
          WorkItem w;
          w.pat = q;
          w.s = sz;
          w.rank0 = stride / 2 + j * stride;
          w.count = std::min(G, K - j);
          w.part = (int)pp->items.size();
          w.stride = stride;
          w.s_last = 0;
          w.aux = K;  // the sample stands for C(h, s) / K times its kappa
          pp->items.push_back(w);
        }
      }
      d.item_end = (int)pp->items.size();
      pp->pats.push_back(d);
      pp->perm_off.push_back(base[v] + c * v);
    }
  }
}

// ------------------------------------------------------------------------
// route choice: subset sum or repeated-row terms
// ------------------------------------------------------------------------
// FP64 operations of the subset sum for order n (products and traces of every
// subset, the schedule's product count per h).
static double subset_cost(int n) {
  static const int kProducts[kMaxH + 1] = {0, 0, 0, 1, 1, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 5, 6};
  const int h = n / 2;
  double c = 0.0;
  for (int s = 1; s <= h; ++s) {
    const double N = 2.0 * s;
    c += (double)binom64(h, s) * (kProducts[h] + 1) * 2.0 * N * N * (N + 1);
  }
  return c;
}

// Most distinct modes with which the repeated-row route can still win at
// order n: T >= 2^d, so beyond it the route never does (collision-free lists,
// the common case, stop their scan after about n/2 entries).
static int rep_d_max(int n) {
  static const std::vector<int> d_max = [] {  // thread-safe one-time initialisation
    std::vector<int> t(kMaxN + 1, 0);
    for (int v = 4; v <= kMaxN; v += 2) {
      const double pc = subset_cost(v);
      for (int d = 1; d <= kRepMaxDistinct; ++d)
        if (4.0 * std::ldexp(1.0, d - 1) * (double)(d * d + 3 * d + 60) < pc) t[v] = d;
    }
    return t;
  }();
  return (n >= 0 && n <= kMaxN) ? d_max[n] : 0;
}

// Largest number of repeated-row partials (term chunks) that a pattern of
// order n can need under the rule below: T = prod (c_j + 1) is largest for
// balanced multiplicities, and the cost condition bounds ceil(T / 2) too.
static int64_t rep_max_chunks(int n) {
  static const std::vector<int64_t> table = [] {  // thread-safe one-time initialisation
    std::vector<int64_t> t(kMaxN + 1, 0);
    for (int v = 4; v <= kMaxN; v += 2) {
      const double pc = subset_cost(v);
      int64_t best = 0;
      for (int d = 1; d <= rep_d_max(v) && d < v; ++d) {
        const int q = v / d, r = v % d;
        const double T = std::min(std::pow(q + 2.0, r) * std::pow(q + 1.0, d - r), 0x1p30);
        const double lim = std::ceil(pc / (4.0 * (double)(d * d + 3 * d + 60)));
        best = std::max(best, (int64_t)std::min(std::ceil(T / 2), lim));
      }
      t[v] = (best + kRepTermsPerItem - 1) / kRepTermsPerItem;
    }
    return t;
  }();
  return (n >= 0 && n <= kMaxN) ? table[n] : 0;
}

static cudaEvent_t g_time_start = nullptr, g_time_stop = nullptr;

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------------
// the batched path shared by gbs_hafnian_batch and gbs_prob_batch
// ------------------------------------------------------------------------
// Sizes and counts of a batch's plan: the plan block (descriptors, work
// items, pair-sum offsets, probe tables, chunk tables) and what the launches
// need to know about it. The inputs themselves are not part of it.
struct BatchLayout {
  int maxn = 0;
  TuneCfg cfg, pcfg;
  int pprec = GBS_FP64;
  bool probe32 = false;
  int64_t n_items = 0, src_elems = 0, idx_elems = 0, pt_elems = 0, dev_rep_cap = 0;
  int n_sel = 0, n_probe = 0, n_pitems = 0, n_chunks = 0;
  size_t pats_b = 0, items_b = 0, ptoff_b = 0;
  size_t perm_b = 0, ppats_b = 0, pitems_b = 0, pperm_b = 0, selpat_b = 0, probe_up_b = 0;
  size_t choff_b = 0, chpat_b = 0, up_b = 0;
  size_t probe_at = 0, chunk_at = 0;
};

// Plans of repeated batch shapes. The plan block depends only on the orders,
// offsets, m and launch shapes (never on the index lists or matrices), so a
// call whose n[] and offs[] match a kept plan skips the planning and its
// upload and reads the kept block (read-only on the device; the probe's
// per-call choice lives in the call's own scratch). Entries are
// evicted least recently used, never while a call is using them, and only
// after the device has finished every launch that read them.
struct PlanKey {
  int mode, precision, batch, maxn, m, device, sms, probe32;
  int wpb, warp_bytes, pwpb, pwarp_bytes;
  int rounds[kMaxN + 1];
  bool operator==(const PlanKey& o) const { return memcmp(this, &o, sizeof(PlanKey)) == 0; }
};
struct PlanEntry {
  PlanKey key;
  std::vector<int> n;
  std::vector<int64_t> offs;
  BatchLayout lay;
  void* d_up = nullptr;          // the upload block (cudaMalloc)
  cudaEvent_t ready = nullptr;   // recorded after its upload
  bool uploaded = false;         // `ready` recorded: other calls may use it
  bool bad = false;              // its upload failed: never used again
  int in_use = 0;
  uint64_t last_use = 0;
};
constexpr int kPlanCacheEntries = 8;
constexpr size_t kPlanCacheBytes = (size_t)256 << 20;
static std::mutex g_plan_mu;
static std::vector<PlanEntry*> g_plans;
static uint64_t g_plan_clock = 0;

// Free a kept plan's device memory once its device has finished every launch
// that may read it (on any stream); the caller's current device is kept.
static cudaError_t plan_free(PlanEntry* v) {
  int cur = 0;
  cudaGetDevice(&cur);
  if (v->key.device != cur) cudaSetDevice(v->key.device);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(v->d_up);
  if (v->ready) cudaEventDestroy(v->ready);
  if (v->key.device != cur) cudaSetDevice(cur);
  delete v;
  return e;
}

static PlanEntry* plan_lookup(const PlanKey& key, const int* n, const int64_t* offs) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (PlanEntry* p : g_plans)
    if (p->uploaded && !p->bad && p->key == key && memcmp(p->n.data(), n, sizeof(int) * key.batch) == 0 &&
        memcmp(p->offs.data(), offs, sizeof(int64_t) * key.batch) == 0) {
      p->in_use++;
      p->last_use = ++g_plan_clock;
      return p;
    }
  return nullptr;
}

// A new entry (in use by the caller) with room for the layout's upload block,
// or null when none can be made (the call then uploads into its own scratch).
static PlanEntry* plan_insert(const PlanKey& key, const int* n, const int64_t* offs, const BatchLayout& lay) {
  if (lay.up_b > kPlanCacheBytes / 4) return nullptr;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  size_t used = 0;
  for (PlanEntry* p : g_plans) used += p->lay.up_b;
  while ((int)g_plans.size() >= kPlanCacheEntries || used + lay.up_b > kPlanCacheBytes) {
    int victim = -1;
    for (int i = 0; i < (int)g_plans.size(); ++i)
      if (g_plans[i]->in_use == 0 && (victim < 0 || g_plans[i]->last_use < g_plans[victim]->last_use)) victim = i;
    if (victim < 0) return nullptr;
    PlanEntry* v = g_plans[victim];
    used -= v->lay.up_b;
    plan_free(v);
    g_plans.erase(g_plans.begin() + victim);
  }
  PlanEntry* p = new (std::nothrow) PlanEntry();
  if (!p) return nullptr;
  if (cudaMalloc(&p->d_up, lay.up_b) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (p->d_up) cudaFree(p->d_up);
    delete p;
    return nullptr;
  }
  p->key = key;
  p->n.assign(n, n + key.batch);
  p->offs.assign(offs, offs + key.batch);
  p->lay = lay;
  p->in_use = 1;
  p->last_use = ++g_plan_clock;
  g_plans.push_back(p);
  return p;
}

// The upload into a new entry was issued (and `ready` recorded), or failed.
static void plan_uploaded(PlanEntry* p, bool ok) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  p->uploaded = ok;
  p->bad = !ok;
}

static void plan_release(PlanEntry* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  p->in_use--;
}

static int clear_plans() {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < g_plans.size();) {
    PlanEntry* v = g_plans[i];
    if (v->in_use) {
      ++i;
      continue;
    }
    const cudaError_t ev = plan_free(v);
    if (e == cudaSuccess) e = ev;
    g_plans.erase(g_plans.begin() + i);
  }
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "synchronize before freeing kept plans");
}


int run_batch(const BatchArgs& a) {
  cudaStream_t st = a.stream;
  const int batch = a.batch;
  if (batch == 0) return GBS_OK;
  if (a.precision != GBS_FP64 && a.precision != GBS_MIXED)
    return fail(GBS_EINVAL, "precision must be GBS_FP64 or GBS_MIXED");
  BatchLayout U;
  // checks, the largest order and the extent of the inputs (elements)
  const bool hmode = (a.mode == BatchArgs::HAFNIAN);
  int64_t elems = 0;
  for (int b = 0; b < batch; ++b) {
    const int v = a.n[b];
    if (v < 0) return fail(GBS_EINVAL, "n[%d] = %d is negative", b, v);
    if (v > GBS_MAX_N) return fail(GBS_ERANGE, "n[%d] = %d exceeds GBS_MAX_N", b, v);
    if (a.offs[b] < 0) return fail(GBS_EINVAL, "offs[%d] is negative", b);
    U.maxn = std::max(U.maxn, v);
    elems = std::max<int64_t>(elems, a.offs[b] + (hmode ? (int64_t)v * v : (int64_t)v));
  }
  (hmode ? U.src_elems : U.idx_elems) = elems;
  const int maxn = U.maxn;
  // launch shape from the largest n (it dominates the cost); rounds per n
  U.cfg = a.cfg_override ? *a.cfg_override : get_cfg(a.precision, maxn);
  const TuneCfg& cfg = U.cfg;
  int rounds_for_n[kMaxN + 1];
  if (a.cfg_override)
    for (int v = 0; v <= kMaxN; ++v) rounds_for_n[v] = a.cfg_override->rounds;
  else
    get_rounds(a.precision, rounds_for_n);
  const bool src_dev = (a.mode == BatchArgs::HAFNIAN) ? is_device_ptr(a.src) : true;
  const bool idx_dev = (a.mode == BatchArgs::PROB) ? is_device_ptr(a.idx) : true;
  // host inputs are checked and staged on every call
  if (a.mode == BatchArgs::HAFNIAN && U.src_elems > 0 && a.src == nullptr)
    return fail(GBS_EINVAL, "A_ri is null");
  if (a.mode == BatchArgs::PROB && U.idx_elems > 0 && a.idx == nullptr)
    return fail(GBS_EINVAL, "idx is null");
  if (a.mode == BatchArgs::PROB && !idx_dev) {
    for (int b = 0; b < batch; ++b)
      for (int i = 0; i < a.n[b]; ++i) {
        const int v = a.idx[a.offs[b] + i];
        if (v < 0 || v >= a.m)
          return fail(GBS_ERANGE, "pattern %d index %d = %d is outside [0, %d)", b, i, v, a.m);
      }
  }
  const int64_t src_elems = U.src_elems, idx_elems = U.idx_elems;
  // host inputs: staged per call into the call's own device block
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t data_b = (a.mode == BatchArgs::PROB && !idx_dev) ? al(sizeof(int) * idx_elems)
                      : (a.mode == BatchArgs::HAFNIAN && !src_dev) ? al(16 * (size_t)src_elems) : 0;
  // The probe only ranks candidate orderings by their estimated sum |f|, which
  // float arithmetic does as well as FP64; so FP64 probability calls run it on
  // the float kernel over the kernel's float copy of B (about a quarter of the
  // time), with the float kernel's launch shape.
  U.probe32 = (a.precision == GBS_FP64 && a.mode == BatchArgs::PROB && a.B32 != nullptr);
  U.pprec = U.probe32 ? GBS_MIXED : a.precision;
  U.pcfg = (U.probe32 && !a.cfg_override) ? get_cfg(GBS_MIXED, maxn) : cfg;

  // a kept plan of the same shape (untuned calls)
  const bool cacheable = !a.cfg_override;
  PlanKey key;
  memset(&key, 0, sizeof(key));
  PlanEntry* pe = nullptr;
  bool hit = false;
  if (cacheable) {
    key.mode = (int)a.mode;
    key.precision = a.precision;
    key.batch = batch;
    key.maxn = maxn;
    key.m = a.m;
    cudaGetDevice(&key.device);
    key.sms = device_sm_count();
    key.probe32 = U.probe32;
    key.wpb = cfg.warps_per_block;
    key.warp_bytes = cfg.warp_bytes;
    key.pwpb = U.pcfg.warps_per_block;
    key.pwarp_bytes = U.pcfg.warp_bytes;
    for (int v = 0; v <= kMaxN; ++v) key.rounds[v] = rounds_for_n[v];
    pe = plan_lookup(key, a.n, a.offs);
    if (pe) {
      U = pe->lay;
      hit = true;
    }
  }

  // FP64: pair terms of each matrix with n >= 6, up to kPairTermBudget bytes
  // (later matrices form A_S X A_S by the product)
  constexpr int64_t kPairTermBudget = (int64_t)2 << 30;
  void* host_stage = nullptr;
  int slot = -1;
  unsigned char* hs = nullptr;
  if (!hit) {
    // (a kept plan's shape was checked when it was made)
    if (!shape_fits(a.precision, cfg.warp_bytes, maxn))
      return fail(GBS_EINVAL, "warp_bytes %d too small for n = %d", cfg.warp_bytes, maxn);
    Planner plan;
    // a few items per resident warp balance the load over all SMs; whole-matrix
    // items for all but a reserve of an order, whose per-size items fill the
    // schedule's tail: one matrix per two resident warps in FP64 (one per warp
    // was 0.8 % slower at 10 warps per SM, one per four warps 9 % slower), one
    // per warp for the float kernel (half that was 5 % slower); tuning runs keep
    // per-size items, whose rounds they choose
    const int64_t want = 4LL * device_sm_count() * cfg.warps_per_block;
    const int64_t reserve = a.cfg_override ? 0
                          : (int64_t)device_sm_count() * cfg.warps_per_block / (a.precision == GBS_FP64 ? 2 : 1);
    plan.init(a.n, batch, a.precision, cfg.warp_bytes, rounds_for_n, reserve);
    if (!a.cfg_override) {
      // A small batch gets smaller work items (fewer rounds each) for the same reason.
      for (int iter = 0; iter < 6 && plan.total() < want; ++iter) {
        bool shrunk = false;
        for (int v = 0; v <= kMaxN; ++v)
          if (rounds_for_n[v] > 1) {
            rounds_for_n[v] /= 2;
            shrunk = true;
          }
        if (!shrunk) break;
        plan.init(a.n, batch, a.precision, cfg.warp_bytes, rounds_for_n, reserve);
      }
    }
    U.n_items = plan.total();
    if (U.n_items > ((int64_t)1 << 30))
      return fail(GBS_ENOMEM, "too many work items (%lld)", (long long)U.n_items);

    // FP64 probabilities: the route choice (repeated-row sum for bunched
    // patterns) is made on the device (route_plan_kernel) before the subset
    // sum; repeated-row partial slots are reserved for the most each pattern's
    // order can need, up to kDevRepCap in all (patterns past that in batch
    // order keep the subset sum)
    constexpr int64_t kDevRepCap = (int64_t)1 << 20;
    if (a.mode == BatchArgs::PROB && a.precision == GBS_FP64 && U.idx_elems > 0) {
      for (int b = 0; b < batch; ++b) U.dev_rep_cap += rep_max_chunks(a.n[b]);
      U.dev_rep_cap = std::min(U.dev_rep_cap, kDevRepCap);
    }

    // plan block: pats | items | (pair-sum offsets) | (probe tables) | (chunk
    // tables)
    U.pats_b = al(sizeof(PatDesc) * batch);
    U.items_b = al(sizeof(WorkItem) * std::max<int64_t>(U.n_items, 1));
    if (a.precision == GBS_FP64)
      for (int b = 0; b < batch; ++b) {
        const int64_t q = pair_terms_elems(a.n[b]);
        if (q > 0 && 16 * (U.pt_elems + q) <= kPairTermBudget) U.pt_elems += q;
      }
    U.ptoff_b = (U.pt_elems > 0) ? al(sizeof(int64_t) * batch) : 0;
    // pairing probe of the largest matrices
    PairingPlan pp;
    if (U.n_items > 0) plan_pairing(a.n, batch, U.pprec, U.pcfg.warp_bytes, maxn / 2, &pp);
    U.n_sel = (int)pp.sel.size();
    U.n_probe = (int)pp.pats.size();
    U.n_pitems = (int)pp.items.size();
    U.perm_b = U.n_sel ? al(sizeof(int) * pp.perm.size()) : 0;
    U.ppats_b = U.n_sel ? al(sizeof(PatDesc) * U.n_probe) : 0;
    U.pitems_b = U.n_sel ? al(sizeof(WorkItem) * U.n_pitems) : 0;
    U.pperm_b = U.n_sel ? al(sizeof(int) * U.n_probe) : 0;
    U.selpat_b = U.n_sel ? al(sizeof(int) * U.n_sel) : 0;
    U.probe_up_b = U.perm_b + U.ppats_b + U.pitems_b + U.pperm_b + U.selpat_b;
    // two-stage finalisation when some matrix has more than kChunkItems items
    std::vector<int> chunk_off, chunk_pat;
    int max_items = 0;
    for (int b = 0; b < batch; ++b) max_items = std::max(max_items, plan.items_for(b));
    if (max_items > kChunkItems) {
      chunk_off.resize(batch + 1);
      for (int b = 0; b < batch; ++b) {
        chunk_off[b] = (int)chunk_pat.size();
        const int cnt = plan.items_for(b);
        for (int c = 0; c * kChunkItems < cnt; ++c) chunk_pat.push_back(b);
      }
      chunk_off[batch] = (int)chunk_pat.size();
    }
    U.n_chunks = (int)chunk_pat.size();
    U.choff_b = U.n_chunks ? al(sizeof(int) * (batch + 1)) : 0;
    U.chpat_b = U.n_chunks ? al(sizeof(int) * U.n_chunks) : 0;
    U.up_b = U.pats_b + U.items_b + U.ptoff_b + U.probe_up_b + U.choff_b + U.chpat_b;
    U.probe_at = U.pats_b + U.items_b + U.ptoff_b;
    U.chunk_at = U.probe_at + U.probe_up_b;

    int rc = pinned_acquire(U.up_b + data_b, &host_stage, &slot);
    if (rc) return rc;
    hs = (unsigned char*)host_stage;
    PatDesc* h_pats = (PatDesc*)hs;
    plan.fill(h_pats, (WorkItem*)(hs + U.pats_b));
    for (int b = 0; b < batch; ++b) {
      PatDesc& d = h_pats[b];
      if (a.mode == BatchArgs::HAFNIAN) {
        d.src_off = a.offs[b];
        d.idx_off = -1;
        d.ld = a.n[b];
      } else {
        d.src_off = 0;
        d.idx_off = a.offs[b];
        d.ld = a.m;
      }
    }
    if (U.ptoff_b) {
      int64_t* h_ptoff = (int64_t*)(hs + U.pats_b + U.items_b);
      int64_t off = 0;
      for (int b = 0; b < batch; ++b) {
        const int64_t q = pair_terms_elems(a.n[b]);
        if (q > 0 && 16 * (off + q) <= kPairTermBudget) {
          h_ptoff[b] = off;
          off += q;
        } else {
          h_ptoff[b] = -1;
        }
      }
    }
    if (U.n_sel) {
      unsigned char* q = hs + U.probe_at;
      memcpy(q, pp.perm.data(), sizeof(int) * pp.perm.size());
      q += U.perm_b;
      PatDesc* h_ppats = (PatDesc*)q;
      for (int k = 0; k < U.n_sel; ++k)
        for (int c = 0; c < kPairingCands; ++c) {
          PatDesc d = pp.pats[k * kPairingCands + c];
          const PatDesc& m = h_pats[pp.sel[k]];
          d.src_off = m.src_off;
          d.idx_off = m.idx_off;
          d.ld = m.ld;
          h_ppats[k * kPairingCands + c] = d;
        }
      q += U.ppats_b;
      memcpy(q, pp.items.data(), sizeof(WorkItem) * U.n_pitems);
      q += U.pitems_b;
      memcpy(q, pp.perm_off.data(), sizeof(int) * U.n_probe);
      q += U.pperm_b;
      memcpy(q, pp.sel.data(), sizeof(int) * U.n_sel);
    }
    if (U.n_chunks) {
      memcpy(hs + U.chunk_at, chunk_off.data(), sizeof(int) * (batch + 1));
      memcpy(hs + U.chunk_at + U.choff_b, chunk_pat.data(), sizeof(int) * U.n_chunks);
    }
    if (cacheable) pe = plan_insert(key, a.n, a.offs, U);
  } else if (data_b) {
    int rc = pinned_acquire(data_b, &host_stage, &slot);
    if (rc) {
      plan_release(pe);
      return rc;
    }
    hs = (unsigned char*)host_stage;
  }
  // host inputs after the plan in the staging buffer
  unsigned char* hdata = data_b ? hs + (hit ? 0 : U.up_b) : nullptr;
  if (data_b) {
    if (a.mode == BatchArgs::PROB) memcpy(hdata, a.idx, sizeof(int) * idx_elems);
    else memcpy(hdata, a.src, 16 * (size_t)src_elems);
  }
  const int64_t n_items = U.n_items, dev_rep_cap = U.dev_rep_cap;
  const int n_sel = U.n_sel, n_probe = U.n_probe, n_pitems = U.n_pitems, n_chunks = U.n_chunks;
  const TuneCfg& pcfg = U.pcfg;
  const int pprec = U.pprec;
  const bool probe32 = U.probe32;

  // the call's device block: (staged inputs) | parts | counter | status |
  // probe status | output staging | float copy | pair sums | probe partials |
  // chunk sums | the probe's choice | route choice; preceded by the plan
  // block unless a kept plan holds it
  const size_t parts_b = al(sizeof(Partial) * std::max<int64_t>(n_items, 1));
  const size_t ctr_b = 256;
  const size_t status_b = al(sizeof(int) * batch);
  const size_t pstatus_b = n_sel ? al(sizeof(int) * n_probe) : 0;  // zeroed with ctr and status
  // outputs in host memory (any of them sends all through device staging)
  bool out_hmem[4];
  {
    const double* outs[4] = {a.out0, a.out1, a.out2, a.out3};
    for (int i = 0; i < 4; ++i) out_hmem[i] = outs[i] != nullptr && !is_device_ptr(outs[i]);
  }
  const bool out_host = out_hmem[0] || out_hmem[1] || out_hmem[2] || out_hmem[3];
  const size_t outs_b = out_host ? al(sizeof(double) * 5 * batch) : 0;
  // FP32 path on explicit matrices: one rounded copy per call, gathered by the kernel
  const size_t a32_b = (a.mode == BatchArgs::HAFNIAN && a.precision == GBS_MIXED) ? al(8 * (size_t)src_elems) : 0;
  const size_t pt_b = U.ptoff_b ? al(16 * (size_t)U.pt_elems) : 0;
  const size_t pparts_b = n_sel ? al(sizeof(Partial) * n_pitems) : 0;
  const size_t chparts_b = n_chunks ? al(sizeof(Partial) * n_chunks) : 0;
  const size_t mperm_b = n_sel ? al(sizeof(int) * batch) : 0;  // written by the probe's choice
  // route choice on the device: rep_half | rep_end | repeated-row partials
  const size_t droute_b = dev_rep_cap ? 2 * al(sizeof(int) * batch) + al(sizeof(Partial) * dev_rep_cap) : 0;
  const size_t dev_b = data_b + parts_b + ctr_b + status_b + pstatus_b + outs_b + a32_b + pt_b + pparts_b + chparts_b + mperm_b + droute_b;
  const size_t own_up_b = pe ? 0 : U.up_b;

  void* dmem = nullptr;
  cudaError_t e = scratch_alloc(&dmem, own_up_b + dev_b, st);
  if (e != cudaSuccess) {
    pinned_release(slot, st);
    if (!hit && pe) plan_uploaded(pe, false);
    plan_release(pe);
    cudaGetLastError();
    return fail(GBS_ENOMEM, "device scratch of %zu bytes: %s", own_up_b + dev_b, cudaGetErrorString(e));
  }
  unsigned char* up = pe ? (unsigned char*)pe->d_up : (unsigned char*)dmem;
  unsigned char* dv = (unsigned char*)dmem + own_up_b;
  PatDesc* d_pats = (PatDesc*)up;
  WorkItem* d_items = (WorkItem*)(up + U.pats_b);
  const int* d_idx = (data_b && a.mode == BatchArgs::PROB) ? (const int*)dv : a.idx;
  const double* d_src = (data_b && a.mode == BatchArgs::HAFNIAN) ? (const double*)dv : a.src;
  const int64_t* d_ptoff = U.ptoff_b ? (const int64_t*)(up + U.pats_b + U.items_b) : nullptr;
  const int* d_perm = n_sel ? (const int*)(up + U.probe_at) : nullptr;
  const PatDesc* d_ppats = n_sel ? (const PatDesc*)(up + U.probe_at + U.perm_b) : nullptr;
  const WorkItem* d_pitems = n_sel ? (const WorkItem*)(up + U.probe_at + U.perm_b + U.ppats_b) : nullptr;
  const int* d_pperm = n_sel ? (const int*)(up + U.probe_at + U.perm_b + U.ppats_b + U.pitems_b) : nullptr;
  const int* d_selpat = n_sel ? (const int*)(up + U.probe_at + U.perm_b + U.ppats_b + U.pitems_b + U.pperm_b) : nullptr;
  const int* d_choff = n_chunks ? (const int*)(up + U.chunk_at) : nullptr;
  const int* d_chpat = n_chunks ? (const int*)(up + U.chunk_at + U.choff_b) : nullptr;
  size_t o = data_b;
  Partial* d_parts = (Partial*)(dv + o);
  o += parts_b;
  int* d_ctr = (int*)(dv + o);
  o += ctr_b;
  int* d_status = (int*)(dv + o);
  o += status_b;
  int* d_pstatus = n_sel ? (int*)(dv + o) : nullptr;
  o += pstatus_b;
  double* d_outs = outs_b ? (double*)(dv + o) : nullptr;
  o += outs_b;
  float* d_a32 = a32_b ? (float*)(dv + o) : nullptr;
  o += a32_b;
  double* d_pt = pt_b ? (double*)(dv + o) : nullptr;
  o += pt_b;
  Partial* d_pparts = n_sel ? (Partial*)(dv + o) : nullptr;
  o += pparts_b;
  Partial* d_chparts = n_chunks ? (Partial*)(dv + o) : nullptr;
  o += chparts_b;
  int* d_mperm = n_sel ? (int*)(dv + o) : nullptr;
  o += mperm_b;
  int* d_rephalf = dev_rep_cap ? (int*)(dv + o) : nullptr;
  int* d_repend = dev_rep_cap ? (int*)(dv + o + al(sizeof(int) * batch)) : nullptr;
  Partial* d_repparts = dev_rep_cap ? (Partial*)(dv + o + 2 * al(sizeof(int) * batch)) : nullptr;

  HafLaunch L;
  memset(&L, 0, sizeof(L));
  int ret = GBS_OK;
  void* h_outs = nullptr;  // pinned copy of the output staging (host outputs)
  int oslot = -1;
  const size_t out_sz[4] = {sizeof(double) * batch, sizeof(double) * batch, 2 * sizeof(double) * batch,
                            sizeof(double) * batch};
  do {
    if (!hit) {
      e = cudaMemcpyAsync(up, hs, U.up_b, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "upload"); break; }
      if (pe && (e = cudaEventRecord(pe->ready, st)) != cudaSuccess) { ret = cuda_fail(e, "plan event"); break; }
    } else {
      // the kept block was uploaded on some stream: order this one after it
      e = cudaStreamWaitEvent(st, pe->ready, 0);
      if (e != cudaSuccess) { ret = cuda_fail(e, "plan wait"); break; }
    }
    if (data_b) {
      e = cudaMemcpyAsync(dv, hdata, data_b, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "input upload"); break; }
    }
    e = cudaMemsetAsync(d_ctr, 0, ctr_b + status_b + pstatus_b, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "memset"); break; }
    if (d_mperm) {  // -1: the default ordering until the probe's choice replaces it
      e = cudaMemsetAsync(d_mperm, 0xff, sizeof(int) * batch, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "memset"); break; }
    }
    if (d_a32) {
      e = launch_to_float(d_src, d_a32, 2 * src_elems, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "float copy"); break; }
    }
    if (n_items > 0) {
      L.src = (a.mode == BatchArgs::HAFNIAN) ? d_src : a.B;
      L.src32 = (a.precision == GBS_MIXED) ? ((a.mode == BatchArgs::HAFNIAN) ? d_a32 : a.B32) : nullptr;
      L.idx = (a.mode == BatchArgs::PROB) ? d_idx : nullptr;
      L.pats = d_pats;
      L.items = d_items;
      L.n_items = (int)n_items;
      L.m_bound = (a.mode == BatchArgs::PROB) ? a.m : 0;
      L.counter = d_ctr;
      L.status = d_status;
      L.parts = d_parts;
      L.warp_bytes = cfg.warp_bytes;
      L.stage_h = maxn / 2;
      L.pt = d_pt;
      L.pt_off = d_ptoff;
      L.batch = batch;
      L.perm = d_perm;
      L.perm_off = d_mperm;
      const int smem = cfg.warps_per_block * cfg.warp_bytes;
      int per_sm = max_blocks_per_sm(a.precision, cfg.warps_per_block, smem);
      if (per_sm < 1) { ret = fail(GBS_EINVAL, "launch shape does not fit an SM"); break; }
      int blocks = device_sm_count() * per_sm;
      const int64_t need = (n_items + cfg.warps_per_block - 1) / cfg.warps_per_block;
      if (need < blocks) blocks = (int)need;
      const bool timed = g_time_start && g_time_stop && !a.cfg_override;
      if (timed) cudaEventRecord(g_time_start, st);
      if (dev_rep_cap) {
        RoutePlan RP;
        memset(&RP, 0, sizeof(RP));
        RP.idx = d_idx;
        RP.pats = d_pats;
        RP.batch = batch;
        RP.m_bound = a.m;
        RP.cap = (int)dev_rep_cap;
        for (int v = 0; v <= kMaxN; ++v) {
          RP.subset_cost[v] = (v >= 4 && !(v & 1)) ? subset_cost(v) : 0.0;
          RP.d_max[v] = rep_d_max(v);
        }
        RP.rep_half = d_rephalf;
        RP.rep_end = d_repend;
        RP.rep_total = d_ctr + 56;
        RP.blocks_done = (unsigned*)(d_ctr + 57);
        RP.n_chosen = d_ctr + 59;
        e = launch_route_plan(RP, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "route choice launch"); break; }
        L.skip = d_rephalf;
      }
      if (n_sel) {
        // probe launch over the candidate orderings, then the choice per matrix
        HafLaunch Lp = L;
        Lp.skip = nullptr;  // probe matrices are numbered differently
        Lp.pats = d_ppats;
        Lp.items = d_pitems;
        Lp.n_items = n_pitems;
        Lp.counter = d_ctr + 32;
        Lp.status = d_pstatus;
        Lp.parts = d_pparts;
        Lp.pt = nullptr;
        Lp.pt_off = nullptr;
        Lp.batch = n_probe;
        Lp.perm_off = d_pperm;
        if (probe32) Lp.src32 = a.B32;
        Lp.warp_bytes = pcfg.warp_bytes;
        // few items (one or a few matrices): fewer warps per block, so that
        // the samples spread over every SM instead of sharing FP64 units
        const int sms = device_sm_count();
        int pwpb = (n_pitems + sms - 1) / sms;
        pwpb = std::max(1, std::min(pwpb, pcfg.warps_per_block));
        const int pper_sm = max_blocks_per_sm(pprec, pwpb, pwpb * pcfg.warp_bytes);
        if (pper_sm < 1) { ret = fail(GBS_EINVAL, "probe shape does not fit an SM"); break; }
        int pblocks = sms * pper_sm;
        const int pneed = (n_pitems + pwpb - 1) / pwpb;
        if (pneed < pblocks) pblocks = pneed;
        e = launch_haf_subsets(Lp, pprec, pblocks, pwpb, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "probe launch"); break; }
        PairingSelect S;
        S.probe_pats = d_ppats;
        S.probe_items = d_pitems;
        S.probe_parts = d_pparts;
        S.probe_perm_off = d_pperm;
        S.sel_pat = d_selpat;
        S.n_sel = n_sel;
        S.n_cand = kPairingCands;
        S.main_perm_off = d_mperm;
        e = launch_pairing_select(S, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "pairing choice launch"); break; }
      }
      e = launch_pair_terms(L, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "pair-term kernel launch"); break; }
      if (n_items > 0) {
        e = launch_haf_subsets(L, a.precision, blocks, cfg.warps_per_block, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "subset kernel launch"); break; }
      }
      if (dev_rep_cap) {
        // the patterns the device chose for the repeated-row sum (the item
        // count is read on the device; the grid covers the reservation)
        RepLaunch R;
        R.B = a.B;
        R.idx = d_idx;
        R.pats = d_pats;
        R.n_items = (int)dev_rep_cap;
        R.n_items_dev = d_ctr + 56;
        R.m_bound = L.m_bound;
        R.counter = d_ctr + 58;
        R.status = d_status;
        R.parts = d_repparts;
        R.rep_half = d_rephalf;
        R.rep_end = d_repend;
        R.batch = batch;
        e = launch_haf_repeated(R, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "repeated-row kernel launch"); break; }
      }
      if (timed) cudaEventRecord(g_time_stop, st);
    }
    if (n_chunks && n_items > 0) {
      ChunkLaunch C;
      C.pats = d_pats;
      C.parts = d_parts;
      C.chunk_pat = d_chpat;
      C.chunk_off = d_choff;
      C.n_chunks = n_chunks;
      C.out = d_chparts;
      e = launch_chunk_sums(C, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "chunk-sum launch"); break; }
    }
    FinalizeLaunch F;
    memset(&F, 0, sizeof(F));
    F.pats = d_pats;
    F.parts = d_parts;
    if (n_chunks && n_items > 0) {
      F.chunk_parts = d_chparts;
      F.chunk_off = d_choff;
    }
    F.idx = (a.mode == BatchArgs::PROB) ? d_idx : nullptr;
    F.status = d_status;
    if (dev_rep_cap && n_items > 0) {
      F.rep_half = d_rephalf;
      F.rep_end = d_repend;
      F.rep_parts = d_repparts;
    }
    F.batch = batch;
    F.precision = a.precision;
    F.log_norm = a.log_norm_dev;
    double* o[4] = {a.out0, a.out1, a.out2, a.out3};
    double* dst[4];
    for (int i = 0; i < 4; ++i) dst[i] = o[i];
    if (out_host) {
      // all outputs go to device staging: p | logp | haf (2) | err
      dst[0] = a.out0 ? d_outs : nullptr;
      dst[1] = a.out1 ? d_outs + batch : nullptr;
      dst[2] = a.out2 ? d_outs + 2 * batch : nullptr;
      dst[3] = a.out3 ? d_outs + 4 * batch : nullptr;
    }
    if (a.mode == BatchArgs::PROB) {
      F.p_out = dst[0];
      F.logp_out = dst[1];
      F.haf_out = dst[2];
      F.err_out = dst[3];
    } else {
      F.haf_out = dst[2];
      F.kappa_out = dst[3];
    }
    e = launch_finalize(F, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "finalize launch"); break; }
    if (out_host) {
      // device outputs straight from the staging; host ones by one copy of
      // the staging block into pinned memory, spread after the synchronisation
      for (int i = 0; i < 4 && ret == GBS_OK; ++i)
        if (o[i] && !out_hmem[i]) {
          e = cudaMemcpyAsync(o[i], dst[i], out_sz[i], cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) ret = cuda_fail(e, "result copy");
        }
      if (ret != GBS_OK) break;
      const int prc = pinned_acquire(sizeof(double) * 5 * batch, &h_outs, &oslot);
      if (prc != GBS_OK) {
        ret = prc;
        break;
      }
      e = cudaMemcpyAsync(h_outs, d_outs, sizeof(double) * 5 * batch, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) ret = cuda_fail(e, "result copy");
    }
  } while (0);
  pinned_release(slot, st);
  if (!hit && pe) plan_uploaded(pe, ret == GBS_OK);
  plan_release(pe);
  e = scratch_free(dmem, st);
  if (e != cudaSuccess && ret == GBS_OK) ret = cuda_fail(e, "scratch free");
  if (ret == GBS_OK && out_host) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) ret = cuda_fail(e, "stream synchronize");
    if (ret == GBS_OK) {
      const double* ho = (const double*)h_outs;
      const size_t off[4] = {0, (size_t)batch, 2 * (size_t)batch, 4 * (size_t)batch};
      double* o[4] = {a.out0, a.out1, a.out2, a.out3};
      for (int i = 0; i < 4; ++i)
        if (out_hmem[i]) memcpy(o[i], ho + off[i], out_sz[i]);
    }
  }
  if (oslot >= 0) pinned_release(oslot, st);
  return ret;
}

// ------------------------------------------------------------------------
// the ordering probe on its own (serving loop)
// ------------------------------------------------------------------------
int order_probe_launch(const gbs_kernel* k, const int* const* lists, const int* n, int count, int stage_h,
                       const TuneCfg& cfg, cudaStream_t st, OrderProbe* out) {
  out->n_lists = count;
  out->n.assign(n, n + count);
  PairingPlan pp;
  plan_pairing(n, count, GBS_MIXED, cfg.warp_bytes, stage_h, &pp);
  out->perm = pp.perm;
  out->sel = pp.sel;
  const int n_sel = (int)pp.sel.size();
  if (n_sel == 0) return GBS_OK;
  const int n_probe = (int)pp.pats.size();
  const int n_pitems = (int)pp.items.size();
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // upload: idx (kMaxN per list) | probe pats | items | perm | probe perm offsets | sel
  const size_t idx_b = al(sizeof(int) * kMaxN * count), ppats_b = al(sizeof(PatDesc) * n_probe);
  const size_t items_b = al(sizeof(WorkItem) * n_pitems), perm_b = al(sizeof(int) * pp.perm.size());
  const size_t pperm_b = al(sizeof(int) * n_probe), sel_b = al(sizeof(int) * n_sel);
  const size_t up_b = idx_b + ppats_b + items_b + perm_b + pperm_b + sel_b;
  // device only: partials | counter, completion word | status | chosen offsets
  const size_t parts_b = al(sizeof(Partial) * n_pitems), ctr_b = 256, status_b = al(sizeof(int) * n_probe);
  const size_t mperm_b = al(sizeof(int) * count);
  const size_t total_b = up_b + parts_b + ctr_b + status_b + mperm_b;
  void* hv = nullptr;
  // pinned: the uploads, then the results and the completion word
  int rc = pinned_acquire(up_b + mperm_b + 256, &hv, &out->pin_slot);
  if (rc) return rc;
  unsigned char* hs = (unsigned char*)hv;
  int* h_idx = (int*)hs;
  for (int i = 0; i < count; ++i) memcpy(h_idx + (size_t)i * kMaxN, lists[i], sizeof(int) * n[i]);
  PatDesc* h_ppats = (PatDesc*)(hs + idx_b);
  for (int q = 0; q < n_probe; ++q) {
    PatDesc d = pp.pats[q];
    d.src_off = 0;
    d.idx_off = (int64_t)pp.sel[q / kPairingCands] * kMaxN;
    d.ld = k->m;
    h_ppats[q] = d;
  }
  memcpy(hs + idx_b + ppats_b, pp.items.data(), sizeof(WorkItem) * n_pitems);
  memcpy(hs + idx_b + ppats_b + items_b, pp.perm.data(), sizeof(int) * pp.perm.size());
  memcpy(hs + idx_b + ppats_b + items_b + perm_b, pp.perm_off.data(), sizeof(int) * n_probe);
  memcpy(hs + idx_b + ppats_b + items_b + perm_b + pperm_b, pp.sel.data(), sizeof(int) * n_sel);
  out->res = (int*)(hs + up_b);
  out->flag = (volatile int*)(hs + up_b + mperm_b);
  *out->flag = 0;
  static std::atomic<unsigned> seq{0};
  const unsigned byte = 1u + seq.fetch_add(1u) % 255u;  // the word's four bytes, never 0
  out->expect = (int)(byte * 0x01010101u);
  cudaError_t e = scratch_alloc(&out->dmem, total_b, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pinned_release(out->pin_slot, st);
    out->pin_slot = -1;
    out->dmem = nullptr;
    return fail(GBS_ENOMEM, "probe scratch of %zu bytes: %s", total_b, cudaGetErrorString(e));
  }
  unsigned char* dm = (unsigned char*)out->dmem;
  int ret = GBS_OK;
  do {
    e = cudaMemcpyAsync(dm, hs, up_b, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe upload"); break; }
    int* d_ctr = (int*)(dm + up_b + parts_b);
    e = cudaMemsetAsync(d_ctr, 0, ctr_b + status_b, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe memset"); break; }
    HafLaunch Lp;
    memset(&Lp, 0, sizeof(Lp));
    Lp.src = k->B;
    Lp.src32 = k->B32;
    Lp.idx = (const int*)dm;
    Lp.pats = (const PatDesc*)(dm + idx_b);
    Lp.items = (const WorkItem*)(dm + idx_b + ppats_b);
    Lp.n_items = n_pitems;
    Lp.counter = d_ctr;
    Lp.status = (int*)(dm + up_b + parts_b + ctr_b);
    Lp.parts = (Partial*)(dm + up_b);
    Lp.warp_bytes = cfg.warp_bytes;
    Lp.stage_h = stage_h;
    Lp.perm = (const int*)(dm + idx_b + ppats_b + items_b);
    Lp.perm_off = (const int*)(dm + idx_b + ppats_b + items_b + perm_b);
    Lp.batch = n_probe;
    const int sms = device_sm_count();
    const int pwpb = std::max(1, std::min((n_pitems + sms - 1) / sms, cfg.warps_per_block));
    const int per_sm = max_blocks_per_sm(GBS_MIXED, pwpb, pwpb * cfg.warp_bytes);
    if (per_sm < 1) { ret = fail(GBS_EINVAL, "probe shape does not fit an SM"); break; }
    const int blocks = std::min(sms * per_sm, (n_pitems + pwpb - 1) / pwpb);
    e = launch_haf_subsets(Lp, GBS_MIXED, blocks, pwpb, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe launch"); break; }
    int* d_mperm = (int*)(dm + up_b + parts_b + ctr_b + status_b);
    PairingSelect S;
    S.probe_pats = Lp.pats;
    S.probe_items = Lp.items;
    S.probe_parts = Lp.parts;
    S.probe_perm_off = Lp.perm_off;
    S.sel_pat = (const int*)(dm + idx_b + ppats_b + items_b + perm_b + pperm_b);
    S.n_sel = n_sel;
    S.n_cand = kPairingCands;
    S.main_perm_off = d_mperm;
    e = launch_pairing_select(S, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "pairing choice launch"); break; }
    e = cudaMemcpyAsync(out->res, d_mperm, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe result copy"); break; }
    // the completion word after the results (stream order)
    e = cudaMemsetAsync(d_ctr + 32, (int)byte, sizeof(int), st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)out->flag, d_ctr + 32, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe completion word"); break; }
    if (!out->done) {
      e = cudaEventCreateWithFlags(&out->done, cudaEventDisableTiming);
      if (e != cudaSuccess) { ret = cuda_fail(e, "probe event"); break; }
    }
    e = cudaEventRecord(out->done, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "probe event record"); break; }
  } while (0);
  scratch_free(out->dmem, st);
  out->dmem = nullptr;
  if (ret != GBS_OK) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    order_probe_release(out, st);
  }
  return ret;
}

bool order_probe_ready(const OrderProbe& pr) {
  if (pr.flag == nullptr || *pr.flag != pr.expect) return false;
  std::atomic_thread_fence(std::memory_order_acquire);  // the results before the word
  return true;
}

bool order_probe_result(const OrderProbe& pr, int i, int* positions) {
  if (i < 0 || i >= pr.n_lists || pr.res == nullptr) return false;
  if (std::find(pr.sel.begin(), pr.sel.end(), i) == pr.sel.end()) return false;
  const int off = pr.res[i], v = pr.n[i];
  if (off < 0 || off + v > (int)pr.perm.size()) return false;
  memcpy(positions, pr.perm.data() + off, sizeof(int) * v);
  return true;
}

void order_probe_release(OrderProbe* pr, cudaStream_t st) {
  if (pr->pin_slot >= 0) pinned_release(pr->pin_slot, st);
  pr->pin_slot = -1;
  pr->res = nullptr;
  pr->flag = nullptr;
  pr->sel.clear();
  pr->perm.clear();
  pr->n.clear();
  pr->n_lists = 0;
}

void order_probe_destroy(OrderProbe* pr) {
  if (pr->done) cudaEventDestroy(pr->done);
  pr->done = nullptr;
}

}  // namespace gbs

using namespace gbs;

// ------------------------------------------------------------------------
// kernel matrix
// ------------------------------------------------------------------------
extern "C" int gbs_build_kernel(const double* U_ri, const double* r, int m, void* stream,
                                gbs_kernel** out) {
  clear_error();
  if (!U_ri || !r || !out) return fail(GBS_EINVAL, "null argument");
  if (m < 1) return fail(GBS_EINVAL, "m = %d must be >= 1", m);
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  gbs_kernel* k = new (std::nothrow) gbs_kernel();
  if (!k) return fail(GBS_ENOMEM, "host allocation");
  cudaError_t e = cudaGetDevice(&k->device);
  if (e != cudaSuccess) { delete k; return cuda_fail(e, "cudaGetDevice"); }
  k->m = m;
  const size_t mm = (size_t)m * m;
  e = cudaMalloc(&k->B, 16 * mm);
  if (e != cudaSuccess) { delete k; cudaGetLastError(); return fail(GBS_ENOMEM, "B: %s", cudaGetErrorString(e)); }
  e = cudaMalloc(&k->dscal, 256);
  if (e != cudaSuccess) { cudaFree(k->B); delete k; cudaGetLastError(); return fail(GBS_ENOMEM, "scalars"); }
  e = cudaMalloc(&k->B32, 8 * mm);
  if (e == cudaSuccess) e = cudaMalloc(&k->t, 8 * (size_t)m);
  if (e != cudaSuccess) {
    cudaFree(k->B); cudaFree(k->B32); cudaFree(k->dscal); delete k; cudaGetLastError();
    return fail(GBS_ENOMEM, "B32: %s", cudaGetErrorString(e));
  }
  // stage U and r on the device when they are host memory
  const bool u_dev = is_device_ptr(U_ri), r_dev = is_device_ptr(r);
  void* tmp = nullptr;
  const size_t u_b = u_dev ? 0 : 16 * mm, r_b = r_dev ? 0 : 8 * (size_t)m;
  e = scratch_alloc(&tmp, u_b + r_b + 256, st);
  if (e != cudaSuccess) {
    cudaFree(k->B); cudaFree(k->dscal); delete k; cudaGetLastError();
    return fail(GBS_ENOMEM, "staging: %s", cudaGetErrorString(e));
  }
  unsigned char* tb = (unsigned char*)tmp;
  const double* dU = U_ri;
  const double* dr = r;
  int ret = GBS_OK;
  {
    // identical squeezing (needed by the marginals of the chain-rule sampler)
    std::vector<double> hr(m);
    if (cudaMemcpy(hr.data(), r, 8 * (size_t)m, cudaMemcpyDefault) == cudaSuccess) {
      k->r_uniform = 1;
      for (int i = 1; i < m; ++i)
        if (hr[i] != hr[0]) k->r_uniform = 0;
      k->t_uniform = tanh(hr[0]);
    } else {
      cudaGetLastError();
    }
  }
  if (!u_dev) {
    e = cudaMemcpyAsync(tb, U_ri, u_b, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) ret = cuda_fail(e, "U upload");
    dU = (const double*)tb;
  }
  if (ret == GBS_OK && !r_dev) {
    e = cudaMemcpyAsync(tb + u_b, r, r_b, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) ret = cuda_fail(e, "r upload");
    dr = (const double*)(tb + u_b);
  }
  if (ret == GBS_OK) {
    e = launch_build_B(dU, dr, m, k->B, k->dscal, k->t, st);
    if (e != cudaSuccess) ret = cuda_fail(e, "build_B launch");
  }
  if (ret == GBS_OK) {
    e = launch_to_float(k->B, k->B32, 2 * (int64_t)mm, st);
    if (e != cudaSuccess) ret = cuda_fail(e, "B32 launch");
  }
  scratch_free(tmp, st);
  if (ret == GBS_OK && (!u_dev || !r_dev)) {
    // host sources were copied from pageable memory; nothing else to wait for
  }
  if (ret != GBS_OK) {
    cudaStreamSynchronize(st);
    cudaFree(k->B);
    cudaFree(k->B32);
    cudaFree(k->t);
    cudaFree(k->dscal);
    delete k;
    return ret;
  }
  *out = k;
  return GBS_OK;
}

extern "C" int gbs_free_kernel(gbs_kernel* k) {
  clear_error();
  if (!k) return GBS_OK;
  cudaError_t e1 = cudaFree(k->B);
  cudaError_t e2 = cudaFree(k->dscal);
  cudaFree(k->B32);
  cudaFree(k->t);
  delete k;
  if (e1 != cudaSuccess) return cuda_fail(e1, "cudaFree(B)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFree(scalars)");
  return GBS_OK;
}

extern "C" int gbs_kernel_info(const gbs_kernel* k, int* m, double* log_norm) {
  clear_error();
  if (!k) return fail(GBS_EINVAL, "null kernel");
  if (m) *m = k->m;
  if (log_norm) {
    cudaError_t e = cudaMemcpy(log_norm, k->dscal, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "log_norm copy");
  }
  return GBS_OK;
}

extern "C" int gbs_kernel_copy_B(const gbs_kernel* k, double* dst, void* stream) {
  clear_error();
  if (!k || !dst) return fail(GBS_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(dst);
  cudaError_t e = cudaMemcpyAsync(dst, k->B, 16 * (size_t)k->m * k->m,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "B copy");
  if (!dev) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  }
  return GBS_OK;
}

// ------------------------------------------------------------------------
// batches
// ------------------------------------------------------------------------
extern "C" int gbs_hafnian_batch(const double* A_ri, const int* n, const int64_t* offs, int batch,
                                 int precision, void* stream, double* haf_ri_out, double* kappa_out) {
  clear_error();
  if (batch < 0) return fail(GBS_EINVAL, "batch = %d is negative", batch);
  if (batch > 0 && (!n || !offs || !haf_ri_out)) return fail(GBS_EINVAL, "null argument");
  BatchArgs a;
  a.mode = BatchArgs::HAFNIAN;
  a.src = A_ri;
  a.n = n;
  a.offs = offs;
  a.batch = batch;
  a.precision = precision;
  a.stream = (cudaStream_t)stream;
  a.out2 = haf_ri_out;
  a.out3 = kappa_out;
  return run_batch(a);
}

extern "C" int gbs_prob_batch(const gbs_kernel* k, const int* idx, const int* n, const int64_t* offs,
                              int batch, int precision, void* stream, double* p_out, double* logp_out,
                              double* haf_ri_out, double* err_est_out) {
  clear_error();
  if (!k) return fail(GBS_EINVAL, "null kernel");
  if (batch < 0) return fail(GBS_EINVAL, "batch = %d is negative", batch);
  if (batch > 0 && (!n || !offs)) return fail(GBS_EINVAL, "null argument");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != k->device) return fail(GBS_EINVAL, "kernel lives on device %d, current is %d", k->device, dev);
  BatchArgs a;
  a.mode = BatchArgs::PROB;
  a.B = k->B;
  a.B32 = k->B32;
  a.m = k->m;
  a.log_norm_dev = k->dscal;
  a.idx = idx;
  a.n = n;
  a.offs = offs;
  a.batch = batch;
  a.precision = precision;
  a.stream = (cudaStream_t)stream;
  a.out0 = p_out;
  a.out1 = logp_out;
  a.out2 = haf_ri_out;
  a.out3 = err_est_out;
  return run_batch(a);
}

extern "C" int gbs_set_timing_events(void* start, void* stop) {
  clear_error();
  g_time_start = (cudaEvent_t)start;
  g_time_stop = (cudaEvent_t)stop;
  return GBS_OK;
}

extern "C" int gbs_clear_plans(void) {
  clear_error();
  return clear_plans();
}

extern "C" const char* gbs_last_error(void) { return t_err.c_str(); }
