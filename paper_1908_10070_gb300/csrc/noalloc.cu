// gbs_hafnian_batch_noalloc: the batched Hafnian call for callers that must
// not allocate memory.
//
// Some callers cannot allocate device memory while they run: code that runs
// inside a host callback or a framework's memory-accounting scope, processes
// that reserve all device memory up front for other work, or embedded
// deployments that forbid cudaMalloc after start-up. For them this entry point
// takes its working space (pattern descriptors, work items, per-item partial
// sums, the work-queue counter and status flags) from one fixed array compiled
// into the library, and its host-side plan from fixed host arrays, so it calls
// no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine. It
// launches the same subset-sum and finalisation kernels as gbs_hafnian_batch.
//
// Costs of that choice: the array (kNoAllocBytes, about 1.6 MB) is reserved
// on every GPU that loads the library, until the process exits; batches are
// limited to kNoAllocMaxBatch matrices and kNoAllocMaxItems work items; and
// all calls share the one array, so calls whose GPU work overlaps (on two
// streams, or from two host threads without ordering) race on it.
#include <string.h>

#include <mutex>

#include "gbs_api_internal.h"

namespace gbs {
namespace {

constexpr int kNoAllocMaxBatch = 1024;
constexpr int kNoAllocMaxItems = 16384;
constexpr size_t kPatsBytes = sizeof(PatDesc) * kNoAllocMaxBatch;
constexpr size_t kItemsBytes = sizeof(WorkItem) * kNoAllocMaxItems;
constexpr size_t kPartsBytes = sizeof(Partial) * kNoAllocMaxItems;
constexpr size_t kCtrBytes = 256;
constexpr size_t kStatusBytes = sizeof(int) * kNoAllocMaxBatch;
constexpr size_t kNoAllocBytes = kPatsBytes + kItemsBytes + kPartsBytes + kCtrBytes + kStatusBytes;

// The shared working space. In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;                          // guards the host plan arrays and the address table
void* g_dev_addr[kMaxDevices] = {nullptr};  // device address of the array, per device
PatDesc g_host_pats[kNoAllocMaxBatch];
WorkItem g_host_items[kNoAllocMaxItems];

int64_t binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  int64_t r = 1;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_hafnian_batch_noalloc(const double* A_ri, const int* n, const int64_t* offs,
                                         int batch, int precision, void* stream, double* haf_ri_out,
                                         double* kappa_out) {
  clear_error();
  if (batch < 0) return fail(GBS_EINVAL, "batch = %d is negative", batch);
  if (batch == 0) return GBS_OK;
  if (!n || !offs || !A_ri || !haf_ri_out) return fail(GBS_EINVAL, "null argument");
  if (batch > kNoAllocMaxBatch)
    return fail(GBS_ERANGE, "batch of %d matrices exceeds the %d this entry point holds", batch,
                kNoAllocMaxBatch);
  if (precision != GBS_FP64 && precision != GBS_MIXED)
    return fail(GBS_EINVAL, "precision must be GBS_FP64 or GBS_MIXED");
  if (!is_device_ptr(A_ri) || !is_device_ptr(haf_ri_out) || (kappa_out && !is_device_ptr(kappa_out)))
    return fail(GBS_EINVAL, "A_ri, haf_ri_out and kappa_out must be device memory");
  int maxn = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 0) return fail(GBS_EINVAL, "n[%d] = %d is negative", b, n[b]);
    if (n[b] > GBS_MAX_N) return fail(GBS_ERANGE, "n[%d] = %d exceeds GBS_MAX_N", b, n[b]);
    if (offs[b] < 0) return fail(GBS_EINVAL, "offs[%d] is negative", b);
    if (n[b] > maxn) maxn = n[b];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(GBS_EINVAL, "device %d out of range", dev);

  std::lock_guard<std::mutex> lk(g_mu);
  // One-time set-up per device (the current device): look up the array's
  // device address. Make the first call on a device before any stream capture.
  if (!g_dev_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_dev_addr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_dev_addr[dev];

  // Plan into the fixed host arrays: the same items, in pattern order, as the
  // allocating entry point builds (its order of execution does not change any
  // result, which is summed per pattern in item order).
  const TuneCfg cfg = get_cfg(precision, maxn);
  if (!shape_fits(precision, cfg.warp_bytes, maxn))
    return fail(GBS_EINVAL, "warp_bytes %d too small for n = %d", cfg.warp_bytes, maxn);
  const int cb = complex_bytes(precision);
  int q = 0;
  for (int b = 0; b < batch; ++b) {
    PatDesc& d = g_host_pats[b];
    d.src_off = offs[b];
    d.idx_off = -1;
    d.ld = n[b];
    d.n = n[b];
    d.item_begin = q;
    if (n[b] >= 2 && !(n[b] & 1)) {
      const int h = n[b] / 2;
      const int R = get_cfg(precision, n[b]).rounds;
      for (int s = 1; s <= h; ++s) {
        const int G = 32 / lanes_for(2 * s, h, cfg.warp_bytes, maxn / 2, cb);
        const int64_t cnt = binom(h, s);
        const int64_t cap = (int64_t)G * R;
        for (int64_t r0 = 0; r0 < cnt; r0 += cap) {
          if (q >= kNoAllocMaxItems)
            return fail(GBS_ERANGE, "batch needs more than the %d work items this entry point holds",
                        kNoAllocMaxItems);
          WorkItem& w = g_host_items[q];
          w.pat = b;
          w.s = s;
          w.rank0 = (int)r0;
          w.count = (int)((cnt - r0) < cap ? (cnt - r0) : cap);
          w.part = q;
          w.stride = 1;
          w.s_last = 0;
          w.aux = 0;
          ++q;
        }
      }
    }
    d.item_end = q;
  }
  const int n_items = q;

  PatDesc* d_pats = (PatDesc*)base;
  WorkItem* d_items = (WorkItem*)(base + kPatsBytes);
  Partial* d_parts = (Partial*)(base + kPatsBytes + kItemsBytes);
  int* d_ctr = (int*)(base + kPatsBytes + kItemsBytes + kPartsBytes);
  int* d_status = (int*)(base + kPatsBytes + kItemsBytes + kPartsBytes + kCtrBytes);

  // pageable copies: each returns once the host arrays have been read
  e = cudaMemcpyAsync(d_pats, g_host_pats, sizeof(PatDesc) * batch, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "descriptor upload");
  if (n_items > 0) {
    e = cudaMemcpyAsync(d_items, g_host_items, sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "work-item upload");
  }
  // the queue counter and status flags must start at zero on every call
  e = cudaMemsetAsync(d_ctr, 0, kCtrBytes + sizeof(int) * batch, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (n_items > 0) {
    HafLaunch L;
    memset(&L, 0, sizeof(L));
    L.src = A_ri;
    L.idx = nullptr;
    L.pats = d_pats;
    L.items = d_items;
    L.n_items = n_items;
    L.m_bound = 0;
    L.counter = d_ctr;
    L.status = d_status;
    L.parts = d_parts;
    L.warp_bytes = cfg.warp_bytes;
    L.stage_h = maxn / 2;
    const int smem = cfg.warps_per_block * cfg.warp_bytes;
    const int per_sm = max_blocks_per_sm(precision, cfg.warps_per_block, smem);
    if (per_sm < 1) return fail(GBS_EINVAL, "launch shape does not fit an SM");
    int blocks = device_sm_count() * per_sm;
    const int need = (n_items + cfg.warps_per_block - 1) / cfg.warps_per_block;
    if (need < blocks) blocks = need;
    e = launch_haf_subsets(L, precision, blocks, cfg.warps_per_block, st);
    if (e != cudaSuccess) return cuda_fail(e, "subset kernel launch");
  }
  FinalizeLaunch F;
  memset(&F, 0, sizeof(F));
  F.pats = d_pats;
  F.parts = d_parts;
  F.idx = nullptr;
  F.status = d_status;
  F.batch = batch;
  F.precision = precision;
  F.log_norm = nullptr;
  F.haf_out = haf_ri_out;
  F.kappa_out = kappa_out;
  e = launch_finalize(F, st);
  if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
  return GBS_OK;
}
