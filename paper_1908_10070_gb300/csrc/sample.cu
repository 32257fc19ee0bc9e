// Sampling on top of the probability path.
//
// Step 1 of the sampler (Sec. 3.1): the photon-number distribution
//   P_n = sum_{|s| = n} p(s) = [z^n] prod_i sech r_i (1 - tanh^2 r_i z^2)^{-1/2},
// which for identical r is the negative binomial of Eq. Eqdistribution, built
// on the device as a product of per-mode power series.
//
// Brute-force sampling (Appendix I): all C(m+n-1, n) configurations with n
// photons are enumerated on the device (index lists in colex order of the
// stars-and-bars combinations), their probabilities are computed by the
// batched probability path, a fixed-order prefix sum turns them into
// intervals, and each caller-supplied uniform number in [0, 1) selects the
// configuration whose interval contains u * (sum of all p).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_api_internal.h"

namespace gbs {
namespace {

// P_n for n = 0..n_max: coefficient k of prod_i (1 - t_i^2 z^2)^{-1/2}, times
// exp(-log_norm) = prod_i sech r_i. One block; thread k owns coefficient k.
// (1 - a z^2)^{-1/2} = sum_j C(2j, j) / 4^j a^j z^{2j}.
__global__ void photon_number_kernel(const double* __restrict__ t, int m, int n_max,
                                     const double* __restrict__ log_norm, double* __restrict__ out) {
  extern __shared__ double sh[];
  double* cur = sh;                // n_max + 1
  double* nxt = sh + (n_max + 1);  // n_max + 1
  for (int k = threadIdx.x; k <= n_max; k += blockDim.x) cur[k] = (k == 0) ? 1.0 : 0.0;
  __syncthreads();
  for (int i = 0; i < m; ++i) {
    const double a = t[i] * t[i];
    for (int k = threadIdx.x; k <= n_max; k += blockDim.x) {
      // sum over even j <= k of c_{j/2}(a) cur[k - j], c_q = C(2q, q) / 4^q a^q
      double acc = 0.0, c = 1.0;
      for (int q = 0; 2 * q <= k; ++q) {
        acc = fma(c, cur[k - 2 * q], acc);
        c *= a * (double)(2 * q + 1) / (double)(2 * q + 2);  // C(2q+2,q+1)/4^{q+1} / (C(2q,q)/4^q)
      }
      nxt[k] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= n_max; k += blockDim.x) cur[k] = nxt[k];
    __syncthreads();
  }
  const double norm = exp(-*log_norm);
  for (int k = threadIdx.x; k <= n_max; k += blockDim.x) out[k] = cur[k] * norm;
}

// Colex unranking of n-element multisets of {0..m-1}: the multiset
// x_1 <= ... <= x_n corresponds to the combination c_j = x_j + j - 1 of
// {0..m+n-2}, with rank = sum_j C(c_j, j).
__global__ void enumerate_kernel(int m, int n, int64_t first, int64_t count,
                                 const int64_t* __restrict__ binom,  // (m+n) x (n+1), row-major
                                 int* __restrict__ idx) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = first + q;
    int c = m + n - 2;
    for (int j = n; j >= 1; --j) {
      while (c >= 0 && binom[(int64_t)c * (n + 1) + j] > r) --c;
      r -= binom[(int64_t)c * (n + 1) + j];
      idx[q * n + (j - 1)] = c - (j - 1);
      --c;
    }
  }
}

// Inclusive prefix sum of count doubles in a fixed order (one block): thread
// t sums its contiguous chunk, the chunk totals are scanned by thread 0, and
// each thread rescans its chunk from its offset. Deterministic.
__global__ void prefix_kernel(const double* __restrict__ p, int64_t count, double* __restrict__ cum) {
  __shared__ double tot[1024];
  const int T = blockDim.x;
  const int64_t chunk = (count + T - 1) / T;
  const int64_t lo = threadIdx.x * chunk, hi = min(count, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo; i < hi; ++i) s += p[i];
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int i = 0; i < T; ++i) {
      const double v = tot[i];
      tot[i] = run;
      run += v;
    }
  }
  __syncthreads();
  double run = tot[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    run += p[i];
    cum[i] = run;
  }
}

// For each uniform u, the first configuration whose cumulative probability
// exceeds u * total; its index list is copied to the output.
__global__ void pick_kernel(const double* __restrict__ cum, int64_t count, const double* __restrict__ u,
                            int draws, const int* __restrict__ idx, int n, int* __restrict__ out) {
  const double total = cum[count - 1];
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < draws; d += gridDim.x * blockDim.x) {
    const double target = u[d] * total;
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cum[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    for (int j = 0; j < n; ++j) out[(int64_t)d * n + j] = idx[lo * n + j];
  }
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_photon_number_dist(const gbs_kernel* k, int n_max, void* stream, double* Pn_out) {
  clear_error();
  if (!k || !Pn_out) return fail(GBS_EINVAL, "null argument");
  if (n_max < 0 || n_max > 2048) return fail(GBS_ERANGE, "n_max = %d outside [0, 2048]", n_max);
  if (!k->t) return fail(GBS_EINVAL, "kernel has no squeezing parameters");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(Pn_out);
  void* tmp = nullptr;
  cudaError_t e = cudaSuccess;
  double* dst = Pn_out;
  if (!dev) {
    e = scratch_alloc(&tmp, sizeof(double) * (n_max + 1), st);
    if (e != cudaSuccess) return fail(GBS_ENOMEM, "P_n buffer: %s", cudaGetErrorString(e));
    dst = (double*)tmp;
  }
  photon_number_kernel<<<1, 256, 2 * sizeof(double) * (n_max + 1), st>>>(k->t, k->m, n_max, k->dscal, dst);
  e = cudaGetLastError();
  int ret = GBS_OK;
  if (e != cudaSuccess) ret = cuda_fail(e, "photon-number kernel");
  if (ret == GBS_OK && !dev) {
    e = cudaMemcpyAsync(Pn_out, dst, sizeof(double) * (n_max + 1), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) ret = cuda_fail(e, "P_n copy");
    if (ret == GBS_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) ret = cuda_fail(e, "synchronize");
  }
  if (tmp) scratch_free(tmp, st);
  return ret;
}

extern "C" int gbs_sample_bruteforce(const gbs_kernel* k, int n, const double* uniforms, int draws,
                                     int precision, void* stream, int* patterns_out, double* total_out) {
  clear_error();
  if (!k || (draws > 0 && (!uniforms || !patterns_out))) return fail(GBS_EINVAL, "null argument");
  if (n < 0 || n > GBS_MAX_N) return fail(GBS_ERANGE, "n = %d outside [0, %d]", n, GBS_MAX_N);
  if (draws < 0) return fail(GBS_EINVAL, "draws = %d is negative", draws);
  if (precision != GBS_FP64 && precision != GBS_MIXED) return fail(GBS_EINVAL, "bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = k->m;
  // C(m+n-1, n) configurations; binomials C(a, b) for a < m+n, b <= n
  std::vector<int64_t> binom((size_t)(m + n) * (n + 1), 0);
  const int64_t cap = (int64_t)1 << 26;
  for (int a = 0; a < m + n; ++a)
    for (int b = 0; b <= n; ++b) {
      int64_t v;
      if (b == 0) v = 1;
      else if (a == 0) v = 0;
      else v = binom[(size_t)(a - 1) * (n + 1) + b - 1] + binom[(size_t)(a - 1) * (n + 1) + b];
      binom[(size_t)a * (n + 1) + b] = std::min<int64_t>(v, cap + 1);
    }
  const int64_t count = (n == 0) ? 1 : binom[(size_t)(m + n - 1) * (n + 1) + n];
  if (count > cap)
    return fail(GBS_ERANGE, "C(m+n-1, n) configurations exceed the 2^26 this call enumerates");
  const bool u_dev = is_device_ptr(uniforms), o_dev = is_device_ptr(patterns_out);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t binom_b = al(sizeof(int64_t) * binom.size());
  const size_t idx_b = al(sizeof(int) * std::max<int64_t>(1, count * n));
  const size_t p_b = al(sizeof(double) * count);
  const size_t u_b = u_dev ? 0 : al(sizeof(double) * std::max(1, draws));
  const size_t o_b = o_dev ? 0 : al(sizeof(int) * std::max<int64_t>(1, (int64_t)draws * n));
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, binom_b + idx_b + 2 * p_b + u_b + o_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "sampler scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  int64_t* d_binom = (int64_t*)t;
  int* d_idx = (int*)(t + binom_b);
  double* d_p = (double*)(t + binom_b + idx_b);
  double* d_cum = (double*)(t + binom_b + idx_b + p_b);
  double* d_u = u_dev ? (double*)uniforms : (double*)(t + binom_b + idx_b + 2 * p_b);
  int* d_out = o_dev ? patterns_out : (int*)(t + binom_b + idx_b + 2 * p_b + u_b);
  int ret = GBS_OK;
  do {
    e = cudaMemcpyAsync(d_binom, binom.data(), sizeof(int64_t) * binom.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { ret = cuda_fail(e, "binomial upload"); break; }
    if (!u_dev && draws > 0) {
      e = cudaMemcpyAsync(d_u, uniforms, sizeof(double) * draws, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "uniform upload"); break; }
    }
    if (n > 0) {
      int64_t blocks = std::min<int64_t>(4096, (count + 255) / 256);
      enumerate_kernel<<<(int)blocks, 256, 0, st>>>(m, n, 0, count, d_binom, d_idx);
      if ((e = cudaGetLastError()) != cudaSuccess) { ret = cuda_fail(e, "enumerate"); break; }
    }
    // probabilities of every configuration, in chunks through the batched path
    const int64_t chunk = 1 << 20;
    std::vector<int> nv;
    std::vector<int64_t> offs;
    for (int64_t c0 = 0; c0 < count && ret == GBS_OK; c0 += chunk) {
      const int64_t c = std::min(chunk, count - c0);
      nv.assign((size_t)c, n);
      offs.resize((size_t)c);
      for (int64_t q = 0; q < c; ++q) offs[(size_t)q] = q * n;
      BatchArgs a;
      a.mode = BatchArgs::PROB;
      a.B = k->B;
      a.B32 = k->B32;
      a.m = m;
      a.log_norm_dev = k->dscal;
      a.idx = d_idx + c0 * n;
      a.n = nv.data();
      a.offs = offs.data();
      a.batch = (int)c;
      a.precision = precision;
      a.stream = st;
      a.out0 = d_p + c0;
      ret = run_batch(a);
    }
    if (ret) break;
    prefix_kernel<<<1, 1024, 0, st>>>(d_p, count, d_cum);
    if ((e = cudaGetLastError()) != cudaSuccess) { ret = cuda_fail(e, "prefix sum"); break; }
    if (total_out) {
      e = cudaMemcpyAsync(total_out, d_cum + count - 1, sizeof(double), cudaMemcpyDefault, st);
      if (e != cudaSuccess) { ret = cuda_fail(e, "total copy"); break; }
    }
    if (draws > 0) {
      pick_kernel<<<std::max(1, std::min(4096, (draws + 255) / 256)), 256, 0, st>>>(d_cum, count, d_u, draws,
                                                                                    d_idx, n, d_out);
      if ((e = cudaGetLastError()) != cudaSuccess) { ret = cuda_fail(e, "pick"); break; }
      if (!o_dev) {
        e = cudaMemcpyAsync(patterns_out, d_out, sizeof(int) * (size_t)draws * n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "sample copy"); break; }
      }
    }
  } while (0);
  scratch_free(tmp, st);
  if (ret == GBS_OK && ((!o_dev && draws > 0) || (total_out && !is_device_ptr(total_out)))) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) ret = cuda_fail(e, "synchronize");
  }
  return ret;
}
