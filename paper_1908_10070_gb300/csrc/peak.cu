// FP64 peak measurement: the denominator of the FP64 roofline fraction.
//
// The subset sum is bound by the FP64 pipe (DFMA), whose rate on this part is
// low and not published per clock with certainty, so it is measured: every
// thread of a grid that fills all SMs runs kChains independent DFMA chains
// (independent so that the pipe, not the latency of one chain, sets the rate)
// for a fixed number of iterations, timed with CUDA events on the caller's
// stream. Operands stay bounded (x <- x * a + b with |a| < 1), and the final
// values are stored so the work cannot be removed.
#include "gbs_api_internal.h"

namespace gbs {
namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) dfma_peak_kernel(int iters, double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_measure_fp64_peak(void* stream, double* tflops_out) {
  clear_error();
  if (!tflops_out) return fail(GBS_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_peak_kernel, kPeakThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  const int blocks = device_sm_count() * (per_sm > 4 ? 4 : (per_sm < 1 ? 1 : per_sm));
  void* out = nullptr;
  e = scratch_alloc(&out, sizeof(double) * blocks * kPeakThreads, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "peak output: %s", cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int ret = GBS_OK;
  const int iters = 4096;
  float best_ms = 1e30f;
  do {
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      ret = cuda_fail(e, "event");
      break;
    }
    for (int rep = 0; rep < 4 && ret == GBS_OK; ++rep) {  // the first is a warm-up
      cudaEventRecord(e0, st);
      dfma_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, 0.999999, 1e-7, (double*)out);
      if ((e = cudaGetLastError()) != cudaSuccess) { ret = cuda_fail(e, "peak launch"); break; }
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { ret = cuda_fail(e, "peak synchronize"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best_ms) best_ms = ms;
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  scratch_free(out, st);
  if (ret != GBS_OK) return ret;
  const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
  *tflops_out = flops / (best_ms * 1e-3) / 1e12;
  return GBS_OK;
}
