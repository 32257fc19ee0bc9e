// Marginal probabilities q_n(x_1..x_k) of the position-basis distribution and
// the chain-rule sampler built on them (Sec. 3.3-3.4, Theorem 1, Algorithms 1
// and 2). Identical squeezing only: the theorem uses the unitarity of
// W = U U^T (Rule 3), and q_n does not depend on r.
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
// The sub-Hafnians Haf(W_T) for every even subset T of the prefix come from
// the batched subset-sum path (Haf(B_T) = tanh(r)^{|T|/2} Haf(W_T)); one block
// per prefix then adds the terms in a fixed order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_api_internal.h"

namespace gbs {
namespace {

constexpr int kMaxK = 10;  // prefix length limit (the term count grows like 9^k)

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

// One block per prefix. H: Haf(W_T) for all 2^k subsets T (bitmask order),
// F: coefficient table, vmask: for each distinct mode value of the prefix the
// bitmask of its positions (nv values). Terms are split over threads by
// (s, s') in a fixed order and reduced in a fixed tree.
__global__ void marginal_kernel(int k, int n, const double2* __restrict__ H, const double* __restrict__ F,
                                const int* __restrict__ vmask, const int* __restrict__ nv,
                                double* __restrict__ q_out) {
  __shared__ double red_re[256], red_im[256];
  const int b = blockIdx.x;
  const double2* Hb = H + ((int64_t)b << k);
  const int* vm = vmask + b * kMaxK;
  const int nvals = nv[b];
  const int full = (1 << k) - 1;
  const int K2 = k / 2 + 1;
  const int lo = max(0, 2 * k - n);
  double acc_re = 0.0, acc_im = 0.0;
  const int pairs = 1 << (2 * k);
  for (int ps = threadIdx.x; ps < pairs; ps += blockDim.x) {
    const int s = ps & full, sp = ps >> k;
    const int ja = __popc(s), jb = __popc(sp);
    if ((ja & 1) || (jb & 1) || ja < lo || jb < lo) continue;
    const double2 hs = Hb[s], hsp = Hb[sp];
    // Haf(W_s) conj(Haf(W_s'))
    const double pr = hs.x * hsp.x + hs.y * hsp.y, pi = hs.y * hsp.x - hs.x * hsp.y;
    if (pr == 0.0 && pi == 0.0) continue;
    const int cs = full & ~s, csp = full & ~sp;
    double t_re = 0.0, t_im = 0.0;
    const int mu_lo = max(0, 3 * k - ja - jb - n), mu_hi = k - max(ja, jb);
    // submasks A of cs and B of csp with |A| = |B| = mu
    for (int A = cs;; A = (A - 1) & cs) {
      const int mu = __popc(A);
      if (mu >= mu_lo && mu <= mu_hi && !((k - ja - mu) & 1)) {
        const double f = F[((ja >> 1) * K2 + (jb >> 1)) * (k + 1) + mu];
        if (f != 0.0 && nvals == k) {
          // Proposition (collision-free prefix): Per(S_{A,B}) is 1 for B = A
          // and 0 for every other B, so only B = A contributes
          if ((A & ~csp) == 0) {
            const double2 he = Hb[cs & ~A], hep = Hb[csp & ~A];
            const double er = he.x * hep.x + he.y * hep.y, ei = he.y * hep.x - he.x * hep.y;
            t_re = fma(f, er, t_re);
            t_im = fma(f, ei, t_im);
          }
        } else if (f != 0.0) {
          const double2 he = Hb[cs & ~A];
          for (int B = csp;; B = (B - 1) & csp) {
            if (__popc(B) == mu) {
              // Per(S_{A,B}) = prod_v c_v! when A and B hold each value equally often
              double per = 1.0;
              for (int v = 0; v < nvals; ++v) {
                const int ca = __popc(A & vm[v]), cb = __popc(B & vm[v]);
                if (ca != cb) {
                  per = 0.0;
                  break;
                }
                for (int c = 2; c <= ca; ++c) per *= (double)c;
              }
              if (per != 0.0) {
                const double2 hep = Hb[csp & ~B];
                // Haf(W_e) conj(Haf(W_e'))
                const double er = he.x * hep.x + he.y * hep.y, ei = he.y * hep.x - he.x * hep.y;
                t_re = fma(f * per, er, t_re);
                t_im = fma(f * per, ei, t_im);
              }
            }
            if (B == 0) break;
          }
        }
      }
      if (A == 0) break;
    }
    acc_re += pr * t_re - pi * t_im;
    acc_im += pr * t_im + pi * t_re;
  }
  red_re[threadIdx.x] = acc_re;
  red_im[threadIdx.x] = acc_im;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red_re[threadIdx.x] += red_re[threadIdx.x + w];
      red_im[threadIdx.x] += red_im[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) q_out[b] = red_re[0];  // the imaginary part cancels
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
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, hafB_b + H_b + slot_b + F_b + vm_b + nv_b + q_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "marginal scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double* d_hafB = (double*)t;
  double2* d_H = (double2*)(t + hafB_b);
  int* d_slot = (int*)(t + hafB_b + H_b);
  double* d_F = (double*)(t + hafB_b + H_b + slot_b);
  int* d_vm = (int*)(t + hafB_b + H_b + slot_b + F_b);
  int* d_nv = (int*)(t + hafB_b + H_b + slot_b + F_b + vm_b);
  double* d_q = (double*)(t + hafB_b + H_b + slot_b + F_b + vm_b + nv_b);
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
    marginal_kernel<<<batch, 256, 0, st>>>(kk, n, d_H, d_F, d_vm, d_nv, q_dev ? q_out : d_q);
    if ((e = cudaGetLastError()) != cudaSuccess) {
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
// kernel then reads the cache for the rest.
extern "C" int gbs_sample_chain(const gbs_kernel* k, int n, const double* uniforms, void* stream, int* x_out) {
  clear_error();
  if (!k || (n > 0 && (!uniforms || !x_out))) return fail(GBS_EINVAL, "null argument");
  if (n < 0 || n > kMaxK || (n & 1)) return fail(GBS_ERANGE, "n = %d must be even and <= %d", n, kMaxK);
  if (n == 0) return GBS_OK;
  if (!k->r_uniform) return fail(GBS_EINVAL, "marginals need identical squeezing on every mode");
  if (!(k->t_uniform > 0.0)) return fail(GBS_EINVAL, "marginals need r > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = k->m;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t cache_b = al(16 * ((size_t)1 << n)), new_b = al(16 * ((size_t)m << (n - 1)));
  const size_t H_b = al(16 * ((size_t)m << n)), F_b = al(8 * (size_t)(n / 2 + 1) * (n / 2 + 1) * (n + 1));
  const size_t vm_b = al(4 * (size_t)m * kMaxK), nv_b = al(4 * (size_t)m), q_b = al(8 * (size_t)m);
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, cache_b + new_b + H_b + F_b + vm_b + nv_b + q_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "chain scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double2* d_cache = (double2*)t;
  double2* d_new = (double2*)(t + cache_b);
  double2* d_H = (double2*)(t + cache_b + new_b);
  double* d_F = (double*)(t + cache_b + new_b + H_b);
  int* d_vm = (int*)(t + cache_b + new_b + H_b + F_b);
  int* d_nv = (int*)(t + cache_b + new_b + H_b + F_b + vm_b);
  double* d_q = (double*)(t + cache_b + new_b + H_b + F_b + vm_b + nv_b);
  std::vector<int> x;
  std::vector<double> w(m);
  std::vector<int> idx, nvl, vmask((size_t)m * kMaxK), nvals(m);
  std::vector<int64_t> offs;
  int ret = GBS_OK;
  do {
    const double2 one = make_double2(1.0, 0.0);  // Haf of the empty matrix
    if ((e = cudaMemcpyAsync(d_cache, &one, 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
      ret = cuda_fail(e, "cache init");
      break;
    }
    for (int kk = 1; kk <= n && ret == GBS_OK; ++kk) {
      const int half = 1 << (kk - 1);
      // new sub-Hafnians: candidate l, mask T' over positions 0..kk-2 (odd
      // |T'| gives an even list; even |T'| an odd one, whose Hafnian is 0 and
      // costs no work), list = x_{T'} followed by l
      idx.clear();
      nvl.clear();
      offs.clear();
      for (int l = 0; l < m; ++l)
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
      a.m = m;
      a.log_norm_dev = k->dscal;
      a.idx = idx.data();
      a.n = nvl.data();
      a.offs = offs.data();
      a.batch = m * half;
      a.precision = GBS_FP64;
      a.stream = st;
      a.out2 = (double*)d_new;
      if ((ret = run_batch(a)) != GBS_OK) break;
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
      chain_table_kernel<<<std::min(4096, (int)((((int64_t)m << kk) + 255) / 256)), 256, 0, st>>>(
          d_cache, d_new, kk, k->t_uniform, m, d_H);
      fcoef_kernel<<<1, 256, 0, st>>>(kk, n, m, d_F);
      marginal_kernel<<<m, 256, 0, st>>>(kk, n, d_H, d_F, d_vm, d_nv, d_q);
      if ((e = cudaGetLastError()) != cudaSuccess) {
        ret = cuda_fail(e, "chain kernels");
        break;
      }
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
      if (kk < n && (e = cudaMemcpyAsync(d_cache + half, d_new + (size_t)pick * half, 16 * (size_t)half,
                                         cudaMemcpyDeviceToDevice, st)) != cudaSuccess) {
        ret = cuda_fail(e, "cache update");
        break;
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
