// Host-side internals shared by the C ABI, the serving loop and the autotuner.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gbs_internal.cuh"

namespace gbs {
struct ItemTemplate {
  int s, rank0, count, key;
  int s_last;  // > s: the item covers every subset of sizes s..s_last (whole matrix)
};
}  // namespace gbs

struct gbs_kernel {
  int device = 0;
  int m = 0;
  double* B = nullptr;      // m*m complex128, device
  float* B32 = nullptr;     // the same rounded to complex64 (gathered by the FP32 path)
  double* t = nullptr;      // tanh r_i, m doubles, device
  int r_uniform = 0;        // 1 if every r_i is the same
  double t_uniform = 0.0;   // tanh r when r_uniform
  double* dscal = nullptr;  // [0] = L = sum_i log cosh r_i, [1] = exp(-L), device
};

namespace gbs {

// Launch shape of the subset kernel.
struct TuneCfg {
  int warps_per_block = 6;
  int warp_bytes = 36864;  // dynamic shared memory per warp
  int rounds = 4;          // lane-group rounds per work item (subsets per item = G * rounds)
};

struct BatchArgs {
  enum Mode { HAFNIAN, PROB } mode = PROB;
  const double* src = nullptr;  // Hafnian mode: concatenated matrices
  const double* B = nullptr;    // probability mode: kernel matrix (device)
  const float* B32 = nullptr;   // probability mode: kernel matrix as complex64
  int m = 0;
  const double* log_norm_dev = nullptr;
  const int* idx = nullptr;
  const int* n = nullptr;
  const int64_t* offs = nullptr;
  int batch = 0;
  int precision = GBS_FP64;
  cudaStream_t stream = nullptr;
  double* out0 = nullptr;  // p
  double* out1 = nullptr;  // log p
  double* out2 = nullptr;  // Haf (2 per entry)
  double* out3 = nullptr;  // err estimate (probabilities) or kappa (Hafnians)
  const TuneCfg* cfg_override = nullptr;
};

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
bool is_device_ptr(const void* p);
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);
cudaError_t scratch_free(void* p, cudaStream_t st);
int pinned_acquire(size_t bytes, void** ptr, int* slot);
void pinned_release(int slot, cudaStream_t st);

TuneCfg default_cfg(int precision, int n);
TuneCfg get_cfg(int precision, int n);
void set_cfg(int precision, int n, const TuneCfg& c);
int complex_bytes(int precision);
bool shape_fits(int precision, int warp_bytes, int maxn);
int64_t binom64(int a, int b);

struct ItemTemplate;
// Largest order whose matrices may be one whole-matrix work item each
// (2^12 - 1 subsets at n = 24).
constexpr int kWholeMaxN = 24;
// Work items of a batch: init() counts them, fill() writes the descriptors'
// item ranges and the items (in schedule order) into caller memory.
class Planner {
 public:
  // whole_reserve (0 = never): of an order n <= kWholeMaxN with at least
  // 2 * whole_reserve matrices, all but whole_reserve get one item each that
  // covers all their subsets (sizes staged and reduced together); the
  // remaining ones keep one item per size and rank range, which fill the tail
  // of the schedule (whole items go first, as the largest).
  void init(const int* n, int batch, int precision, int warp_bytes, const int* rounds_for_n,
            int64_t whole_reserve = 0);
  void fill(PatDesc* pats, WorkItem* items);
  int64_t total() const { return total_; }
  // work items of one matrix of order v (0 for odd v or v < 2)
  // work items (= partial slots) of matrix b
  int items_for(int b) const {
    if (!whole_.empty() && whole_[b]) return 1;
    const int v = n_[b];
    return (v >= 2 && !(v & 1)) ? (int)tmpl_[v].size() : 0;
  }

 private:
  static constexpr int kKeys = (kMaxN / 2 + 1) * 65;
  const int* n_ = nullptr;
  int batch_ = 0;
  int64_t total_ = 0;
  int npat_[kMaxN + 1];
  int64_t nwhole_[kMaxN + 1];
  std::vector<char> whole_;  // per matrix: one whole-matrix item
  std::vector<ItemTemplate> tmpl_[kMaxN + 1];
  int64_t bucket_[kKeys];
  int64_t start_[kKeys];
};
int device_sm_count();
int run_batch(const BatchArgs& a);

// Smallest order whose subset sum runs in an ordering chosen by the probe.
constexpr int kPairingMinN = 26;

// The ordering probe of the batched calls, on its own, for index lists held
// on the host (the serving loop): for every list with n >= kPairingMinN it
// runs the sampled subset sums of the candidate orderings on the float kernel
// over k's float copy of B and picks the one with the smallest estimated
// sum |f|, asynchronously on `st`. Lists never probe each other: a list's
// choice depends only on the list, the launch shape cfg and stage_h.
struct OrderProbe {
  int n_lists = 0;
  std::vector<int> n;          // order of each list
  std::vector<int> perm;       // candidate orderings (source positions), per order
  std::vector<int> sel;        // probed lists
  void* dmem = nullptr;        // device scratch (freed stream-ordered at launch)
  int pin_slot = -1;           // pinned staging, holding the results at `res`
  int* res = nullptr;          // per list: chosen ordering's offset into perm
  volatile int* flag = nullptr;  // pinned: equals `expect` once res has arrived
  int expect = 0;
  cudaEvent_t done = nullptr;  // recorded after the results (for error checks); kept across launches
};
// Enqueue the probe of `count` host index lists (lists[i] has n[i] entries,
// all < k->m). On success the caller waits for order_probe_ready (or
// out->done) and then calls order_probe_result for each list, then
// order_probe_release (order_probe_destroy once the object is not reused).
int order_probe_launch(const gbs_kernel* k, const int* const* lists, const int* n, int count, int stage_h,
                       const TuneCfg& cfg, cudaStream_t st, OrderProbe* out);
// After out->done: positions[p] = the source position that position p of list
// i reads in the chosen ordering, p < n[i]; false if list i was not probed.
bool order_probe_result(const OrderProbe& pr, int i, int* positions);
// True once the launch's results are in host memory (reads a pinned word that
// the stream writes after them; no driver call).
bool order_probe_ready(const OrderProbe& pr);
void order_probe_release(OrderProbe* pr, cudaStream_t st);
void order_probe_destroy(OrderProbe* pr);

}  // namespace gbs
