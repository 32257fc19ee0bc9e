// Marginal probabilities q_n(x_1..x_k) of the position-basis distribution and
// the chain-rule sampler built on them (Sec. 3.3-3.4, Theorem 1, Algorithms 1
// and 2). Identical squeezing only: the theorem collapses the sums over the
// unsampled photons with the unitarity of W = U U^T (Rule 3:
// sum_i W(i, j) conj(W(i, j')) = delta_jj'); for B = U diag(tanh r_i) U^T with
// unequal r_i that sum is (U* diag(tanh^2 r) U^T)_{j'j}, not a multiple of
// delta, so the theorem does not apply (and q_n does not depend on r when the
// r_i are equal).
//
// Theorem 1, as used here (with the index sets of Algorithm 2):
//   q_n(x_1..x_k) = sum_{ja, jb} sum_{s in C([k], ja), s' in C([k], jb)}
//       Haf(W_s) conj(Haf(W_s')) sum_mu F(k, mu, ja, jb) / f_n
//       sum_{A in C([k] \ s, mu), B in C([k] \ s', mu)} Per(S_{A,B})
//       Haf(W_e) conj(Haf(W_e')),   e = [k] \ (s u A), e' = [k] \ (s' u B),
// ja, jb even in [max(0, 2k - n), k], mu in [max(0, 3k - ja - jb - n), k - max(ja, jb)],
// F = (n-k)! C((n-k+mu+m)/2 - 1, k - (ja+jb)/2 + m/2 - 1) (Appendix H),
// f_n = n! C((m+n)/2 - 1, n/2), S_{A,B}(i, j) = [x_{A_i} = x_{B_j}] (so Per is
// the product of c! over the values whose multiplicities c in A and B agree,
// and 0 if any disagree). W_T is W on the rows/columns x_T. (The pseudocode's
// e' uses s; the theorem's B ranges over [k] \ a. Both are read with s', which
// the brute-force marginal of Eq. marginal_definition confirms.)
//
// Evaluation order. The same sum, regrouped: W_T, and so Haf(W_T), depends
// only on the multiset of modes x_T, and Per(S_{A,B}) only on the multisets
// of A and B. Write alpha for the multiset of A (per distinct mode v of the
// prefix, alpha_v of its m_v copies) and rho = prefix - alpha for what is
// left. For fixed A and B the sums over s and s' separate, and each depends
// on A (or B) only through alpha, so
//   q_n = sum_alpha  prod_v alpha_v! (prod_v C(m_v, alpha_v))^2
//         sum_{ja, jb} F(k, |alpha|, ja, jb) / f_n  G(rho, ja) conj(G(rho, jb)),
//   G(rho, j) = sum_{sigma <= rho, |sigma| = j} prod_v C(rho_v, sigma_v)
//               Haf(W_sigma) Haf(W_{rho - sigma})
// (the binomials count the position sets with a given multiset). That is
// at most 3^k products per prefix, where the nested sums of the theorem take
// about 6^k; for a prefix without repeated modes the multisets are the
// position sets themselves and every count is 1.
//
// The sub-Hafnians Haf(W_T) for every even subset T of the prefix come from
// the batched subset-sum path (Haf(B_T) = tanh(r)^{|T|/2} Haf(W_T)); the
// regrouped sum runs one thread per rho, in fixed-order block and prefix
// reductions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_api_internal.h"

namespace gbs {
namespace {

constexpr int kMaxK = 20;  // prefix length limit (the regrouped sum takes up to 3^k products)
constexpr int kMargThreads = 256;

__device__ double lgbinom(double x, double y) { return lgamma(x + 1.0) - lgamma(y + 1.0) - lgamma(x - y + 1.0); }

// F(k, mu, ja, jb) / f_n for ja, jb in {0, 2, .., k}, mu in [0, k]; 0 outside
// the ranges of Theorem 1.
__global__ void fcoef_kernel(int k, int n, int m, double* __restrict__ F) {
  const int K2 = k / 2 + 1;
  const int total = K2 * K2 * (k + 1);
  const int lo = max(0, 2 * k - n);
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int ja = 2 * (q / (K2 * (k + 1)));
    const int jb = 2 * ((q / (k + 1)) % K2);
    const int mu = q % (k + 1);
    double v = 0.0;
    if (ja >= lo && jb >= lo && mu >= max(0, 3 * k - ja - jb - n) && mu <= k - max(ja, jb)) {
      const double lf = lgamma((double)(n - k) + 1.0) +
                        lgbinom(0.5 * (n - k + mu + m) - 1.0, k - 0.5 * (ja + jb) + 0.5 * m - 1.0) -
                        lgamma((double)n + 1.0) - lgbinom(0.5 * (m + n) - 1.0, 0.5 * n);
      v = exp(lf);
    }
    F[q] = v;
  }
}

__device__ __forceinline__ double binom_d(int a, int b) {
  double r = 1.0;
  for (int i = 1; i <= b; ++i) r = r * (double)(a - b + i) / (double)i;
  return r;
}

// The regrouped Theorem 1 sum (see the top of this file). Blocks cover the
// rho of one prefix (blockIdx.y = prefix, blockIdx.x = a run of kMargThreads
// indices); each thread forms G(rho, .) for its rho and the quadratic form
// with F, and the block writes the sum of its threads (fixed tree) to
// part[prefix * gridDim.x + blockIdx.x].
//   H: Haf(W_T) of every position set T (bitmask order, 0 for odd |T|), 2^k per prefix.
//   vmask, nv: per prefix, the position mask of each of its nv distinct modes.
// A prefix without repeated modes (nv == k) indexes rho by position masks; otherwise
// rho is a mixed-radix number over the distinct modes (digit v in [0, m_v]),
// and a multiset reads the sub-Hafnian of its representative position set (the
// first rho_v positions of each mode v).
__global__ void __launch_bounds__(kMargThreads) marginal_terms_kernel(int k, int n, const double2* __restrict__ H,
                                                                     const double* __restrict__ F,
                                                                     const int* __restrict__ vmask,
                                                                     const int* __restrict__ nv,
                                                                     double* __restrict__ part) {
  __shared__ double red[kMargThreads];
  __shared__ int s_pm[kMaxK][kMaxK + 1];  // first c positions of mode v
  __shared__ int s_mv[kMaxK], s_stride[kMaxK + 1];
  const int b = blockIdx.y;
  const double2* Hb = H + ((int64_t)b << k);
  const int nvals = nv[b];
  const int* vm = vmask + (int64_t)b * kMaxK;
  if (threadIdx.x == 0) {
    int stride = 1;
    for (int v = 0; v < nvals; ++v) {
      const int mk = vm[v];
      s_mv[v] = __popc(mk);
      s_stride[v] = stride;
      stride *= s_mv[v] + 1;
      int acc = 0, rest = mk;
      s_pm[v][0] = 0;
      for (int c = 1; c <= s_mv[v]; ++c) {
        acc |= rest & -rest;  // the next position of mode v
        rest &= rest - 1;
        s_pm[v][c] = acc;
      }
    }
    s_stride[nvals] = stride;
  }
  __syncthreads();
  const int K2 = k / 2 + 1;
  const int full = (1 << k) - 1;
  const int64_t idx = (int64_t)blockIdx.x * kMargThreads + threadIdx.x;
  double acc = 0.0;
  const bool distinct = (nvals == k);
  if (idx < (distinct ? (int64_t)1 << k : (int64_t)s_stride[nvals])) {
    double2 G[kMaxK / 2 + 1];
    for (int j = 0; j < K2; ++j) G[j] = make_double2(0.0, 0.0);
    int rsize;
    double w;  // prod alpha_v! (prod C(m_v, alpha_v))^2
    if (distinct) {
      const int rho = (int)idx;
      rsize = __popc(rho);
      if (!(rsize & 1)) {
        for (int sub = rho;; sub = (sub - 1) & rho) {
          const int c = __popc(sub);
          if (!(c & 1)) {
            const double2 a = Hb[sub], e = Hb[rho ^ sub];
            G[c >> 1].x += a.x * e.x - a.y * e.y;
            G[c >> 1].y += a.x * e.y + a.y * e.x;
          }
          if (sub == 0) break;
        }
      }
      w = 1.0;
      (void)full;
    } else {
      int rho_d[kMaxK];
      int rem = (int)idx;
      rsize = 0;
      w = 1.0;
      for (int v = 0; v < nvals; ++v) {
        rho_d[v] = rem % (s_mv[v] + 1);
        rem /= s_mv[v] + 1;
        rsize += rho_d[v];
        const int a = s_mv[v] - rho_d[v];
        const double cm = binom_d(s_mv[v], a);
        double fa = 1.0;
        for (int c = 2; c <= a; ++c) fa *= (double)c;
        w *= fa * cm * cm;
      }
      if (!(rsize & 1)) {
        // sigma <= rho in mixed radix (digit v in [0, rho_v])
        int sg[kMaxK];
        for (int v = 0; v < nvals; ++v) sg[v] = 0;
        for (;;) {
          int c = 0, ms = 0, mr = 0;
          double cnt = 1.0;
          for (int v = 0; v < nvals; ++v) {
            c += sg[v];
            ms |= s_pm[v][sg[v]];
            mr |= s_pm[v][rho_d[v] - sg[v]];
            cnt *= binom_d(rho_d[v], sg[v]);
          }
          if (!(c & 1)) {
            const double2 a = Hb[ms], e = Hb[mr];
            G[c >> 1].x = fma(cnt, a.x * e.x - a.y * e.y, G[c >> 1].x);
            G[c >> 1].y = fma(cnt, a.x * e.y + a.y * e.x, G[c >> 1].y);
          }
          int v = 0;
          while (v < nvals && sg[v] == rho_d[v]) sg[v++] = 0;
          if (v == nvals) break;
          ++sg[v];
        }
      }
    }
    if (!(rsize & 1)) {
      // the Hermitian form sum_{ja, jb} F(k, mu, ja, jb) G_ja conj(G_jb), mu = k - |rho|
      const int mu = k - rsize;
      double t = 0.0;
      for (int a = 0; a < K2; ++a)
        for (int c = 0; c < K2; ++c) {
          const double f = F[(a * K2 + c) * (k + 1) + mu];
          if (f != 0.0) t = fma(f, G[a].x * G[c].x + G[a].y * G[c].y, t);
        }
      acc = w * t;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = kMargThreads / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = red[0];
}

// q_out[b] = sum of the prefix's block sums, in block order (one warp per
// prefix: lane-strided, then a fixed butterfly).
__global__ void marginal_sum_kernel(const double* __restrict__ part, int nblk, int batch, double* __restrict__ q_out) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= batch) return;
  double s = 0.0;
  for (int i = lane; i < nblk; i += 32) s += part[(int64_t)b * nblk + i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) q_out[b] = s;
}

// H_W[b][T] = Haf(B_{x_T}) / t^{|T|/2} for even |T| (0 for odd |T|).
__global__ void rescale_kernel(const double* __restrict__ hafB, const int* __restrict__ slot, int count,
                               int k, double t, double2* __restrict__ H, int batch) {
  const int64_t total = (int64_t)batch << k;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int T = (int)(q & ((1 << k) - 1));
    const int c = __popc(T);
    double2 v = make_double2(0.0, 0.0);
    if (!(c & 1)) {
      const int j = slot[q];
      const double sc = pow(t, -0.5 * c);
      v.x = hafB[2 * j] * sc;
      v.y = hafB[2 * j + 1] * sc;
    }
    H[q] = v;
  }
}

// Exponential-space variant (Appendix D) for the chain sampler: the sampled
// prefix's sub-Hafnians Haf(B_T) are kept in `cache` (index = position mask
// over the prefix). For candidate l of step k (prefix x_1..x_{k-1}, l), T with
// position k-1 reads the step's new value newv[l][T minus that position], the
// rest the cache; H holds Haf(W_T) = Haf(B_T) / t^{|T|/2} (0 for odd |T|).
__global__ void chain_table_kernel(const double2* __restrict__ cache, const double2* __restrict__ newv, int k,
                                   double t, int m, double2* __restrict__ H) {
  const int64_t total = (int64_t)m << k;
  const int half = 1 << (k - 1);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(q >> k);
    const int T = (int)(q & ((1 << k) - 1));
    const int c = __popc(T);
    double2 v = make_double2(0.0, 0.0);
    if (!(c & 1)) {
      const double2 h = (T & half) ? newv[(int64_t)l * half + (T & (half - 1))] : cache[T];
      const double sc = pow(t, -0.5 * c);
      v.x = h.x * sc;
      v.y = h.y * sc;
    }
    H[q] = v;
  }
}

// The regrouped sum for `batch` prefixes of length k: block sums into
// part (batch * blocks doubles), then one total per prefix.
cudaError_t launch_marginals(int k, int n, const double2* H, const double* F, const int* vmask, const int* nv,
                             int batch, double* part, double* q_out, cudaStream_t st) {
  const int nblk = (int)((((int64_t)1 << k) + kMargThreads - 1) / kMargThreads);
  marginal_terms_kernel<<<dim3(nblk, batch), kMargThreads, 0, st>>>(k, n, H, F, vmask, nv, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  marginal_sum_kernel<<<(batch + 7) / 8, 256, 0, st>>>(part, nblk, batch, q_out);
  return cudaGetLastError();
}

size_t marginal_part_bytes(int k, int batch) {
  const int64_t nblk = (((int64_t)1 << k) + kMargThreads - 1) / kMargThreads;
  return sizeof(double) * (size_t)(nblk * batch);
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_marginal_batch(const gbs_kernel* k, const int* x, int kk, int batch, int n, void* stream,
                                  double* q_out) {
  clear_error();
  if (!k || (batch > 0 && (!q_out || (kk > 0 && !x)))) return fail(GBS_EINVAL, "null argument");
  if (batch < 0) return fail(GBS_EINVAL, "batch = %d is negative", batch);
  if (batch == 0) return GBS_OK;
  if (n < 0 || n > GBS_MAX_N || (n & 1)) return fail(GBS_ERANGE, "n = %d must be even and <= %d", n, GBS_MAX_N);
  if (kk < 0 || kk > n || kk > kMaxK) return fail(GBS_ERANGE, "prefix length %d outside [0, min(n, %d)]", kk, kMaxK);
  if (!k->r_uniform) return fail(GBS_EINVAL, "marginals need identical squeezing on every mode");
  if (!(k->t_uniform > 0.0)) return fail(GBS_EINVAL, "marginals need r > 0");
  cudaStream_t st = (cudaStream_t)stream;
  // prefixes on the host (small): check them and build the sub-Hafnian lists
  std::vector<int> hx((size_t)batch * std::max(kk, 1));
  if (kk > 0) {
    const cudaError_t e0 = cudaMemcpy(hx.data(), x, sizeof(int) * batch * kk, cudaMemcpyDefault);
    if (e0 != cudaSuccess) return cuda_fail(e0, "prefix copy");
  }
  for (size_t i = 0; i < (size_t)batch * kk; ++i)
    if (hx[i] < 0 || hx[i] >= k->m) return fail(GBS_ERANGE, "mode index %d outside [0, %d)", hx[i], k->m);
  const int nsub = 1 << kk;
  std::vector<int> idx, nv_list, slot((size_t)batch * nsub, 0), vmask((size_t)batch * kMaxK, 0), nv(batch, 0);
  std::vector<int64_t> offs;
  for (int b = 0; b < batch; ++b) {
    const int* xb = hx.data() + (size_t)b * kk;
    for (int T = 0; T < nsub; ++T) {
      if (__builtin_popcount(T) & 1) continue;
      slot[(size_t)b * nsub + T] = (int)nv_list.size();
      offs.push_back((int64_t)idx.size());
      int c = 0;
      for (int i = 0; i < kk; ++i)
        if (T >> i & 1) {
          idx.push_back(xb[i]);
          ++c;
        }
      nv_list.push_back(c);
    }
    // position masks of the distinct mode values (for Per(S_{A,B}))
    for (int i = 0; i < kk; ++i) {
      int v = 0;
      while (v < nv[b] && xb[__builtin_ctz(vmask[(size_t)b * kMaxK + v])] != xb[i]) ++v;
      if (v == nv[b]) nv[b]++;
      vmask[(size_t)b * kMaxK + v] |= 1 << i;
    }
  }
  if (idx.empty()) idx.push_back(0);
  const int nh = (int)nv_list.size();
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t hafB_b = al(16 * (size_t)nh), H_b = al(16 * ((size_t)batch << kk)), slot_b = al(4 * slot.size());
  const size_t F_b = al(8 * (size_t)(kk / 2 + 1) * (kk / 2 + 1) * (kk + 1)), vm_b = al(4 * vmask.size()),
               nv_b = al(4 * (size_t)batch), q_b = al(8 * (size_t)batch);
  const size_t part_b = al(marginal_part_bytes(kk, batch));
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, hafB_b + H_b + slot_b + F_b + vm_b + nv_b + q_b + part_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "marginal scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double* d_hafB = (double*)t;
  double2* d_H = (double2*)(t + hafB_b);
  int* d_slot = (int*)(t + hafB_b + H_b);
  double* d_F = (double*)(t + hafB_b + H_b + slot_b);
  int* d_vm = (int*)(t + hafB_b + H_b + slot_b + F_b);
  int* d_nv = (int*)(t + hafB_b + H_b + slot_b + F_b + vm_b);
  double* d_q = (double*)(t + hafB_b + H_b + slot_b + F_b + vm_b + nv_b);
  double* d_part = (double*)(t + hafB_b + H_b + slot_b + F_b + vm_b + nv_b + q_b);
  const bool q_dev = is_device_ptr(q_out);
  int ret = GBS_OK;
  do {
    BatchArgs a;
    a.mode = BatchArgs::PROB;
    a.B = k->B;
    a.B32 = k->B32;
    a.m = k->m;
    a.log_norm_dev = k->dscal;
    a.idx = idx.data();
    a.n = nv_list.data();
    a.offs = offs.data();
    a.batch = nh;
    a.precision = GBS_FP64;
    a.stream = st;
    a.out2 = d_hafB;
    if ((ret = run_batch(a)) != GBS_OK) break;
    if ((e = cudaMemcpyAsync(d_slot, slot.data(), 4 * slot.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_vm, vmask.data(), 4 * vmask.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_nv, nv.data(), 4 * (size_t)batch, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
      ret = cuda_fail(e, "marginal upload");
      break;
    }
    rescale_kernel<<<std::min(4096, (int)((((int64_t)batch << kk) + 255) / 256)), 256, 0, st>>>(
        d_hafB, d_slot, nh, kk, k->t_uniform, d_H, batch);
    fcoef_kernel<<<1, 256, 0, st>>>(kk, n, k->m, d_F);
    double* qd = q_dev ? q_out : d_q;
    const int nblk = (int)(marginal_part_bytes(kk, 1) / sizeof(double));
    for (int b0 = 0; b0 < batch && e == cudaSuccess; b0 += 65535)  // the grid's y extent
      e = launch_marginals(kk, n, d_H + ((int64_t)b0 << kk), d_F, d_vm + (int64_t)b0 * kMaxK, d_nv + b0,
                           std::min(65535, batch - b0), d_part + (int64_t)b0 * nblk, qd + b0, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      ret = cuda_fail(e, "marginal kernels");
      break;
    }
    if (!q_dev) {
      e = cudaMemcpyAsync(q_out, d_q, 8 * (size_t)batch, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        ret = cuda_fail(e, "marginal result copy");
        break;
      }
    }
  } while (0);
  scratch_free(tmp, st);
  return ret;
}

// Algorithm 1: x_k drawn from the m conditional weights q_n(x_1..x_{k-1}, l),
// l = 0..m-1, with the caller's uniform number u_k (inverse CDF in mode order).
// The exponential-space variant of Appendix D: the sub-Hafnians of the sampled
// prefix are kept on the device across steps, so step k computes only those
// of subsets that hold the new photon (for each candidate l, the odd subsets
// T' of positions 0..k-2 plus l), half of the step's table; the marginal
// kernels then read the cache for the rest. Candidates are taken in chunks
// of at most 2^22 new sub-Hafnians, so memory stays bounded at large k; the
// chosen candidate's new sub-Hafnians are then computed once more for the
// cache.
namespace {

// new sub-Hafnians of candidates [l0, l0 + cnt) at step kk into dst
// (cnt * 2^(kk-1) entries, candidate-major)
int chain_new_subhafnians(const gbs_kernel* k, const std::vector<int>& x, int kk, int l0, int cnt,
                          cudaStream_t st, double2* dst) {
  const int half = 1 << (kk - 1);
  std::vector<int> idx, nvl;
  std::vector<int64_t> offs;
  idx.reserve((size_t)cnt * half * kk / 2 + 1);
  for (int l = l0; l < l0 + cnt; ++l)
    for (int T = 0; T < half; ++T) {
      offs.push_back((int64_t)idx.size());
      for (int i = 0; i < kk - 1; ++i)
        if (T >> i & 1) idx.push_back(x[i]);
      idx.push_back(l);
      nvl.push_back(__builtin_popcount(T) + 1);
    }
  BatchArgs a;
  a.mode = BatchArgs::PROB;
  a.B = k->B;
  a.B32 = k->B32;
  a.m = k->m;
  a.log_norm_dev = k->dscal;
  a.idx = idx.data();
  a.n = nvl.data();
  a.offs = offs.data();
  a.batch = cnt * half;
  a.precision = GBS_FP64;
  a.stream = st;
  a.out2 = (double*)dst;
  return run_batch(a);
}

}  // namespace

extern "C" int gbs_sample_chain(const gbs_kernel* k, int n, const double* uniforms, void* stream, int* x_out) {
  clear_error();
  if (!k || (n > 0 && (!uniforms || !x_out))) return fail(GBS_EINVAL, "null argument");
  if (n < 0 || n > kMaxK || (n & 1)) return fail(GBS_ERANGE, "n = %d must be even and <= %d", n, kMaxK);
  if (n == 0) return GBS_OK;
  if (!k->r_uniform) return fail(GBS_EINVAL, "marginals need identical squeezing on every mode");
  if (!(k->t_uniform > 0.0)) return fail(GBS_EINVAL, "marginals need r > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = k->m;
  // candidates per pass at the last step (at most 2^22 new sub-Hafnians)
  const int chunk_max = std::max(1, std::min(m, (1 << 22) >> (n - 1)));
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t cache_b = al(16 * ((size_t)1 << n)), new_b = al(16 * ((size_t)chunk_max << (n - 1)));
  const size_t H_b = al(16 * ((size_t)chunk_max << n)), F_b = al(8 * (size_t)(n / 2 + 1) * (n / 2 + 1) * (n + 1));
  const size_t vm_b = al(4 * (size_t)m * kMaxK), nv_b = al(4 * (size_t)m), q_b = al(8 * (size_t)m);
  size_t part_b = 0;
  for (int kk = 1; kk <= n; ++kk) {
    const int ch = std::max(1, std::min(m, (1 << 22) >> (kk - 1)));
    part_b = std::max(part_b, al(marginal_part_bytes(kk, ch)));
  }
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, cache_b + new_b + H_b + F_b + vm_b + nv_b + q_b + part_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "chain scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double2* d_cache = (double2*)t;
  double2* d_new = (double2*)(t + cache_b);
  double2* d_H = (double2*)(t + cache_b + new_b);
  double* d_F = (double*)(t + cache_b + new_b + H_b);
  int* d_vm = (int*)(t + cache_b + new_b + H_b + F_b);
  int* d_nv = (int*)(t + cache_b + new_b + H_b + F_b + vm_b);
  double* d_q = (double*)(t + cache_b + new_b + H_b + F_b + vm_b + nv_b);
  double* d_part = (double*)(t + cache_b + new_b + H_b + F_b + vm_b + nv_b + q_b);
  std::vector<int> x;
  std::vector<double> w(m);
  std::vector<int> vmask((size_t)m * kMaxK), nvals(m);
  int ret = GBS_OK;
  do {
    const double2 one = make_double2(1.0, 0.0);  // Haf of the empty matrix
    if ((e = cudaMemcpyAsync(d_cache, &one, 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
      ret = cuda_fail(e, "cache init");
      break;
    }
    for (int kk = 1; kk <= n && ret == GBS_OK; ++kk) {
      const int half = 1 << (kk - 1);
      const int chunk = std::max(1, std::min(m, (1 << 22) >> (kk - 1)));
      // per candidate: position masks of the distinct values (for Per(S_{A,B}))
      std::fill(vmask.begin(), vmask.end(), 0);
      for (int l = 0; l < m; ++l) {
        int nvv = 0;
        for (int i = 0; i < kk; ++i) {
          const int xi = (i < kk - 1) ? x[i] : l;
          int v = 0;
          while (v < nvv) {
            const int p0 = __builtin_ctz(vmask[(size_t)l * kMaxK + v]);
            if (((p0 < kk - 1) ? x[p0] : l) == xi) break;
            ++v;
          }
          if (v == nvv) nvv++;
          vmask[(size_t)l * kMaxK + v] |= 1 << i;
        }
        nvals[l] = nvv;
      }
      if ((e = cudaMemcpyAsync(d_vm, vmask.data(), 4 * vmask.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(d_nv, nvals.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        ret = cuda_fail(e, "chain upload");
        break;
      }
      fcoef_kernel<<<1, 256, 0, st>>>(kk, n, m, d_F);
      for (int l0 = 0; l0 < m && ret == GBS_OK; l0 += chunk) {
        const int cnt = std::min(chunk, m - l0);
        if ((ret = chain_new_subhafnians(k, x, kk, l0, cnt, st, d_new)) != GBS_OK) break;
        chain_table_kernel<<<std::min(4096, (int)((((int64_t)cnt << kk) + 255) / 256)), 256, 0, st>>>(
            d_cache, d_new, kk, k->t_uniform, cnt, d_H);
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = launch_marginals(kk, n, d_H, d_F, d_vm + (size_t)l0 * kMaxK, d_nv + l0, cnt, d_part, d_q + l0, st);
        if (e != cudaSuccess) {
          ret = cuda_fail(e, "chain kernels");
          break;
        }
      }
      if (ret != GBS_OK) break;
      if ((e = cudaMemcpyAsync(w.data(), d_q, 8 * (size_t)m, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        ret = cuda_fail(e, "chain weights");
        break;
      }
      double tot = 0.0;
      for (int l = 0; l < m; ++l) tot += std::max(w[l], 0.0);
      const double target = uniforms[kk - 1] * tot;
      double run = 0.0;
      int pick = m - 1;
      for (int l = 0; l < m; ++l) {
        run += std::max(w[l], 0.0);
        if (run > target) {
          pick = l;
          break;
        }
      }
      x.push_back(pick);
      // keep the chosen candidate's new sub-Hafnians: masks with bit kk-1
      if (kk < n) {
        if (chunk >= m) {
          e = cudaMemcpyAsync(d_cache + half, d_new + (size_t)pick * half, 16 * (size_t)half,
                              cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) {
            ret = cuda_fail(e, "cache update");
            break;
          }
        } else {
          std::vector<int> xp(x.begin(), x.end() - 1);
          if ((ret = chain_new_subhafnians(k, xp, kk, pick, 1, st, d_cache + half)) != GBS_OK) break;
        }
      }
    }
  } while (0);
  scratch_free(tmp, st);
  if (ret == GBS_OK)
    for (int i = 0; i < n; ++i) x_out[i] = x[i];
  return ret;
}

// Steps 1-3 of Sec. 3: n from P_n (truncated at n_max, renormalised) by the
// inverse CDF with uniforms[0], then the chain rule for the n photons.
extern "C" int gbs_sample(const gbs_kernel* k, int n_max, const double* uniforms, void* stream, int* n_out,
                          int* x_out) {
  clear_error();
  if (!k || !uniforms || !n_out || (n_max > 0 && !x_out)) return fail(GBS_EINVAL, "null argument");
  if (n_max < 0 || n_max > kMaxK) return fail(GBS_ERANGE, "n_max = %d outside [0, %d]", n_max, kMaxK);
  if (!k->r_uniform) return fail(GBS_EINVAL, "sampling needs identical squeezing on every mode");
  std::vector<double> Pn((size_t)n_max + 1);
  int rc = gbs_photon_number_dist(k, n_max, stream, Pn.data());
  if (rc) return rc;
  double tot = 0.0;
  for (int v = 0; v <= n_max; v += 2) tot += std::max(Pn[v], 0.0);
  if (!(tot > 0.0)) return fail(GBS_EINVAL, "P_n vanishes for every n <= n_max");
  const double target = uniforms[0] * tot;
  double run = 0.0;
  int n = n_max & ~1;
  for (int v = 0; v <= n_max; v += 2) {
    run += std::max(Pn[v], 0.0);
    if (run > target) {
      n = v;
      break;
    }
  }
  *n_out = n;
  if (n == 0) return GBS_OK;
  return gbs_sample_chain(k, n, uniforms + 1, stream, x_out);
}
