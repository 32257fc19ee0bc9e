// Autotuner: picks the subset kernel's launch shape for one photon number n.
//
// Candidates are (warps per block, shared bytes per warp, lane-group rounds per
// work item). Each is timed with CUDA events on synthetic symmetric complex
// matrices of order n (values from a fixed linear congruential sequence), one
// warm-up and three timed runs, and the fastest median is kept in the
// in-process table consulted by every later batch.
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_api_internal.h"

using namespace gbs;

namespace {

int max_dynamic_smem() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin - 4096;  // room for the kernel's static tables
}

}  // namespace

extern "C" int gbs_autotune(int n, int precision, void* stream, int* chosen_out) {
  clear_error();
  if (precision != GBS_FP64 && precision != GBS_MIXED) return fail(GBS_EINVAL, "bad precision");
  if (n < 0 || n > GBS_MAX_N) return fail(GBS_ERANGE, "n = %d outside [0, %d]", n, GBS_MAX_N);
  cudaStream_t st = (cudaStream_t)stream;
  if (n < 4 || (n & 1)) {
    const TuneCfg c = default_cfg(precision, n);
    set_cfg(precision, n, c);
    if (chosen_out) *chosen_out = c.rounds;
    return GBS_OK;
  }
  const int h = n / 2;
  int batch = (int)std::max<int64_t>(4, std::min<int64_t>(4096, ((int64_t)1 << 22) / ((int64_t)1 << h) / h));
  // synthetic matrices (host LCG, uploaded once)
  std::vector<double> A((size_t)batch * n * n * 2);
  uint64_t st64 = 0x9E3779B97F4A7C15ull;
  for (int b = 0; b < batch; ++b)
    for (int i = 0; i < n; ++i)
      for (int j = i; j < n; ++j) {
        double v[2];
        for (int q = 0; q < 2; ++q) {
          st64 = st64 * 6364136223846793005ull + 1442695040888963407ull;
          v[q] = ((double)(st64 >> 11) * 0x1p-53 - 0.5) * 0.5;
        }
        const size_t o1 = ((size_t)b * n * n + (size_t)i * n + j) * 2;
        const size_t o2 = ((size_t)b * n * n + (size_t)j * n + i) * 2;
        A[o1] = A[o2] = v[0];
        A[o1 + 1] = A[o2 + 1] = v[1];
      }
  std::vector<int> nv(batch, n);
  std::vector<int64_t> offs(batch);
  for (int b = 0; b < batch; ++b) offs[b] = (int64_t)b * n * n;
  void* dA = nullptr;
  void* dOut = nullptr;
  cudaError_t e = scratch_alloc(&dA, A.size() * 8, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "autotune input: %s", cudaGetErrorString(e));
  e = scratch_alloc(&dOut, (size_t)batch * 24, st);
  if (e != cudaSuccess) {
    scratch_free(dA, st);
    return fail(GBS_ENOMEM, "autotune output: %s", cudaGetErrorString(e));
  }
  int ret = GBS_OK;
  e = cudaMemcpyAsync(dA, A.data(), A.size() * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) ret = cuda_fail(e, "autotune upload");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ret == GBS_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  const int maxdyn = max_dynamic_smem();
  // 5 warps is the most that holds n = 28 and 30 (whose largest lane groups
  // take about 45 KB a warp)
  const int wpbs[] = {4, 5, 6, 8, 10, 12};
  const int n_wpbs = (int)(sizeof(wpbs) / sizeof(wpbs[0]));
  static_assert(12 <= kMaxWarpsPerBlock, "a tuner shape exceeds the kernel's launch bounds");
  const int rnds[] = {1, 2, 4, 8, 16};
  TuneCfg best = default_cfg(precision, n);
  float best_ms = 1e30f;
  for (int wi = 0; wi < n_wpbs && ret == GBS_OK; ++wi) {
    TuneCfg c;
    c.warps_per_block = wpbs[wi];
    c.warp_bytes = (maxdyn / c.warps_per_block) & ~127;
    if (!shape_fits(precision, c.warp_bytes, n)) continue;
    for (int ri = 0; ri < 5 && ret == GBS_OK; ++ri) {
      c.rounds = rnds[ri];
      BatchArgs a;
      a.mode = BatchArgs::HAFNIAN;
      a.src = (const double*)dA;
      a.n = nv.data();
      a.offs = offs.data();
      a.batch = batch;
      a.precision = precision;
      a.stream = st;
      a.out2 = (double*)dOut;
      a.out3 = (double*)dOut + 2 * batch;
      a.cfg_override = &c;
      float t[3];
      bool ok = true;
      for (int rep = 0; rep < 4 && ok; ++rep) {
        if (rep > 0) cudaEventRecord(e0, st);
        if (run_batch(a) != GBS_OK) ok = false;
        if (rep > 0) {
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
          cudaEventElapsedTime(&t[rep - 1], e0, e1);
        }
      }
      if (!ok) {
        cudaGetLastError();
        clear_error();
        continue;
      }
      std::sort(t, t + 3);
      if (t[1] < best_ms) {
        best_ms = t[1];
        best = c;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  scratch_free(dA, st);
  scratch_free(dOut, st);
  if (ret == GBS_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) ret = cuda_fail(e, "autotune synchronize");
  }
  if (ret == GBS_OK) {
    set_cfg(precision, n, best);
    if (chosen_out) *chosen_out = best.rounds;
  }
  return ret;
}
