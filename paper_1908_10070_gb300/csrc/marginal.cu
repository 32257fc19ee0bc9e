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
// Evaluation order. The same sum, regrouped by rho = [k] \ A: Per(S_{A,B})
// vanishes unless A and B hold the same multiset alpha of modes, and is then
// prod_v alpha_v!; rho_A and rho_B then hold equal multisets too, so their
// sub-Hafnians agree, and for fixed A the sum over s runs over s in rho_A:
//   q_n = sum_rho w(rho) sum_{ja, jb} F(k, k - |rho|, ja, jb) / f_n G(rho, ja) conj(G(rho, jb)),
//   G(rho, j) = sum_{sigma in rho, |sigma| = j} Haf(W_sigma) Haf(W_{rho \ sigma}),
//   w(rho) = prod_v alpha_v! C(m_v, alpha_v)
// (alpha_v = m_v - |rho cap positions of v|, m_v the multiplicity of mode v in
// the prefix; C(m_v, alpha_v) counts the sets B with A's multiset; w = 1
// without repeated modes, the Proposition). F is 0 outside the theorem's
// ranges, and the kernel forms no term there: a rho takes part only if some
// (ja, jb) is in range for mu = k - |rho|, and only the sizes ja in range are
// enumerated. At k = n only rho = [k], s = [k] remains; summed over the n
// steps of a 16-photon sample, about 29 thousand products per candidate mode
// (3^k each when every size is formed).
//
// The sub-Hafnians Haf(W_T) of the sizes read (Haf(B_T) = tanh(r)^{|T|/2}
// Haf(W_T)) come from the batched subset-sum path in gbs_marginal_batch and
// from the sampled prefix's cache in the chain sampler; the sum runs a team
// of lanes per rho, in fixed-order team, block and prefix reductions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_api_internal.h"

namespace gbs {
namespace {

constexpr int kMaxK = 20;  // prefix length limit (position masks in an int; the sum's sets up to 2^k)
constexpr int kMargThreads = 256;

// C(p, i) for p, i <= kMaxK (Pascal's rule, at compile time), in global
// memory; blocks copy it (coalesced) into shared memory, where lanes index it
// freely.
struct BinomTable {
  int v[kMaxK + 1][kMaxK + 1];
};
constexpr BinomTable make_binom_table() {
  BinomTable t{};
  for (int p = 0; p <= kMaxK; ++p)
    for (int i = 0; i <= kMaxK; ++i) t.v[p][i] = i == 0 ? 1 : p == 0 ? 0 : t.v[p - 1][i - 1] + t.v[p - 1][i];
  return t;
}
__device__ const BinomTable c_binom = make_binom_table();
static_assert(make_binom_table().v[20][10] == 184756, "Pascal table");

// Rows p <= rows of the table (a prefix of length k indexes p < k).
__device__ __forceinline__ void load_binom(int (*binom)[kMaxK + 1], int rows) {
  for (int q = threadIdx.x; q < (rows + 1) * (kMaxK + 1); q += blockDim.x)
    binom[q / (kMaxK + 1)][q % (kMaxK + 1)] = c_binom.v[q / (kMaxK + 1)][q % (kMaxK + 1)];
}

__device__ double lgbinom(double x, double y) { return lgamma(x + 1.0) - lgamma(y + 1.0) - lgamma(x - y + 1.0); }

// t^{-s/2} for s = 0..kMaxK photons (tanh r = t): the factor from Haf(B_T)
// to Haf(W_T). Computed once per call on the host.
struct SizeScale {
  double s[kMaxK + 1];
};

SizeScale size_scale(double t) {
  SizeScale sc;
  for (int i = 0; i <= kMaxK; ++i) sc.s[i] = pow(t, -0.5 * i);
  return sc;
}

// The ranges of Theorem 1: ja, jb (the even sizes of s and s') at least
// max(0, 2k - n), and mu = |A| in [max(0, 3k - ja - jb - n), k - max(ja, jb)].
// F vanishes outside them, so no term there is formed.
__host__ __device__ __forceinline__ bool theorem_range(int k, int n, int mu, int ja, int jb) {
  const int lo = 2 * k - n > 0 ? 2 * k - n : 0;
  const int hi = ja > jb ? ja : jb;
  return ja >= lo && jb >= lo && mu >= (3 * k - ja - jb - n > 0 ? 3 * k - ja - jb - n : 0) && mu <= k - hi;
}

// F(k, mu, ja, jb) / f_n for ja, jb in {0, 2, .., k}, mu in [0, k]; 0 outside
// the ranges above. Prefix length k = k0 + blockIdx.y, its table at
// F + blockIdx.y * stride (index (ja/2 * (k/2+1) + jb/2) * (k+1) + mu).
__global__ void fcoef_kernel(int k0, int n, int m, int64_t stride, double* __restrict__ F) {
  const int k = k0 + (int)blockIdx.y;
  double* Fk = F + blockIdx.y * stride;
  const int K2 = k / 2 + 1;
  const int total = K2 * K2 * (k + 1);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int ja = 2 * (q / (K2 * (k + 1)));
    const int jb = 2 * ((q / (k + 1)) % K2);
    const int mu = q % (k + 1);
    double v = 0.0;
    if (theorem_range(k, n, mu, ja, jb)) {
      const double lf = lgamma((double)(n - k) + 1.0) +
                        lgbinom(0.5 * (n - k + mu + m) - 1.0, k - 0.5 * (ja + jb) + 0.5 * m - 1.0) -
                        lgamma((double)n + 1.0) - lgbinom(0.5 * (m + n) - 1.0, 0.5 * n);
      v = exp(lf);
    }
    Fk[q] = v;
  }
}

// Entries of one F table for prefixes of up to k photons.
inline int64_t fcoef_stride(int k) { return (int64_t)(k / 2 + 1) * (k / 2 + 1) * (k + 1); }

// The sets rho of the sum that have some (ja, jb) in range: those of the
// even sizes c[i], count[i] of each. `part` selects them: 0 every such rho
// (C(k, c) of size c), 1 those that hold position k-1 (C(k-1, c-1)), 2 those
// that do not (C(k-1, c)). A team of team[i] lanes (a power of two up to a
// block, kMargThreads) shares each such rho; class i takes the threads from
// start[i], a multiple of 32 (of a block when its teams span several warps),
// so a warp never mixes classes and a block holds one class whenever that
// class's teams need the block's barrier.
struct RhoClasses {
  int part = 0;
  int ncls = 0;
  unsigned need[kMaxK + 1];  // per mu: bit a set if ja = 2a has some jb in range
  int c[kMaxK / 2 + 1];
  int team[kMaxK / 2 + 1];
  int64_t count[kMaxK / 2 + 1];
  int64_t start[kMaxK / 2 + 2];
  __host__ __device__ int64_t total() const { return start[ncls]; }
};

// Subsets per lane that size a team: 8 when a launch has little work (its
// longest team sets the time), more when the launch fills the GPU (the FP64
// pipe sets it, and fewer lanes per team need fewer butterfly adds): up to
// 128 where a step's largest sets hold 1024 subsets or more (measured better
// at 20 photons), else up to 32 (measured better at 12 and 16).
constexpr int kTeamWorkMin = 8, kTeamWorkMax = 32, kTeamWorkMaxLarge = 128;
constexpr int64_t kLargeSetWork = 1024;
constexpr int64_t kResidentLanes = 152 * 2048;

// Calls f(sub) for the subsets of rho (c = |rho| set bits) with t elements of
// colex ranks lo .. lo + cnt - 1: the first by colex unranking (binom = C(p, i)),
// the rest by Gosper's successor on the t-of-c index mask; each index mask is
// spread onto rho's bits.
template <class Fn>
__device__ __forceinline__ void for_subsets_range(int rho, int c, int t, int lo, int cnt,
                                                  const int (*binom)[kMaxK + 1], Fn&& f) {
  if (cnt <= 0) return;
  unsigned u = 0;
  for (int i = t, p = c - 1, rank = lo; i >= 1; --i) {
    while (binom[p][i] > rank) --p;
    u |= 1u << p;
    rank -= binom[p][i];
    --p;
  }
  for (int j = 0;;) {
    int sub = 0;
    for (unsigned uu = u, r = (unsigned)rho; uu; uu >>= 1) {
      const unsigned low = r & (0u - r);
      if (uu & 1u) sub |= (int)low;
      r ^= low;
    }
    f(sub);
    if (++j == cnt) return;
    const unsigned l = u & (0u - u), v = u + l;  // t >= 1 here: C(c, 0) = 1 subset
    u = v + (((v ^ u) / l) >> 2);
  }
}

// The Theorem 1 sum over position sets rho = [k] \ A of the size classes in
// `rc`: team i of class c takes the rho of colex rank i among the c-element
// sets; its lanes split each enumeration below into contiguous colex ranges
// and add their partial sums in a fixed butterfly, and the first lane forms
// the rho's term. For the sets A, B of one multiset alpha (Per(S_{A,B}) = prod_v alpha_v!, 0 for
// different multisets), rho_A and rho_B have equal sub-Hafnians, so
//   q_n = sum_rho w(rho) sum_{ja, jb} F(k, k - |rho|, ja, jb) / f_n G(rho, ja) conj(G(rho, jb)),
//   G(rho, j) = sum_{sigma subset of rho, |sigma| = j} Haf(W_sigma) Haf(W_{rho \ sigma}),
//   w(rho) = prod_v alpha_v! C(m_v, alpha_v),  alpha_v = m_v - |rho cap (positions of mode v)|
// (m_v the multiplicity of mode v in the prefix; w = 1 without repeated
// modes, the Proposition). Only the sizes ja with some jb in range are
// enumerated, and by their complements when those are smaller; G(rho, j) =
// G(rho, |rho| - j) (the same products), so each such pair is formed once.
//   H: Haf(W_T) by position mask T (0 for odd |T|); for prefix b, T without
//      position k-1 reads Hlo + ((lo_off + b) / lo_div) * slo, T with it
//      Hhi + b * shi, at T minus that position.
//   modes: the k modes of prefix b at modes + b * k (repeated modes give w).
// With seg < kMargThreads (one block per prefix suffices, gridDim.x == 1),
// a block holds kMargThreads / seg prefixes, seg threads each, and each
// segment's fixed tree gives q_out[b]. Otherwise prefix b = blockIdx.y spans
// gridDim.x blocks: each writes the sum of its threads (fixed tree) to
// part[b * gridDim.x + blockIdx.x], and the last block of prefix b to finish
// (counted in counters[b], which starts at 0 and is left at 0) writes
// q_out[b], the block sums added in a fixed order (a single block writes it
// directly).
__global__ void __launch_bounds__(kMargThreads, 5) marginal_terms_kernel(int k, int n, RhoClasses rc,
                                                                     const double2* __restrict__ Hlo,
                                                                     int64_t slo, int64_t lo_off, int lo_div,
                                                                     const double2* __restrict__ Hhi,
                                                                     int64_t shi, const double* __restrict__ F,
                                                                     const int* __restrict__ modes,
                                                                     double* __restrict__ part,
                                                                     unsigned* __restrict__ counters,
                                                                     double* __restrict__ q_out, int batch,
                                                                     int seg) {
  constexpr int kSlots = kMargThreads / 32;      // prefixes per block at most (segments of 32 threads)
  __shared__ double red[kMargThreads];
  __shared__ int s_mask[kSlots][kMaxK], s_mult[kSlots][kMaxK];
  __shared__ int s_nrep[kSlots];
  __shared__ int s_binom[kMaxK + 1][kMaxK + 1];  // C(p, i)
  __shared__ double2 s_team[kMargThreads / 32];   // per warp: its share of a team's sum
  // seg < kMargThreads: the block holds kMargThreads / seg prefixes, seg threads each
  // (gridDim.x == 1); else one prefix per blockIdx.y over gridDim.x blocks
  const int slot = threadIdx.x / seg, lt = threadIdx.x % seg;
  const int b = blockIdx.y * (kMargThreads / seg) + slot;
  const bool live = b < batch;
  load_binom(s_binom, k);
  const int K2 = k / 2 + 1;
  if (lt == 0 && live) {
    // position masks of the repeated modes only (a mode seen once has weight 1 either way)
    const int* xb = modes + (int64_t)b * k;
    int r = 0;
    unsigned seen = 0;
    for (int i = 0; i < k; ++i) {
      if (seen >> i & 1u) continue;
      int mask = 1 << i;
      for (int j = i + 1; j < k; ++j)
        if (xb[j] == xb[i]) mask |= 1 << j;
      seen |= (unsigned)mask;
      if (mask != (1 << i)) {
        s_mask[slot][r] = mask;
        s_mult[slot][r] = __popc(mask);
        ++r;
      }
    }
    s_nrep[slot] = r;
  }
  __syncthreads();
  const double2* lo = Hlo + ((lo_off + b) / lo_div) * slo;
  const double2* hi = Hhi + b * shi;
  const int half = k > 0 ? 1 << (k - 1) : 0;
  auto haf = [&](int T) { return (T & half) ? hi[T ^ half] : lo[T]; };
  const int64_t idx = (int64_t)blockIdx.x * kMargThreads + lt;
  double acc = 0.0;
  if (live && idx < rc.total()) {  // whole warps: every class spans a multiple of 32 threads
    int cls = 0;
    while (idx >= rc.start[cls + 1]) ++cls;
    const int c = rc.c[cls], T = rc.team[cls];
    const int64_t local = idx - rc.start[cls];
    const int64_t team = local / T;
    const int member = (int)(local % T);
    const bool real = team < rc.count[cls];  // the rest pad the class to whole warps
    // colex unranking: rank = sum_i C(p_i, i) over the positions p_1 < .. < p_c
    // (over the first k-1 positions when rc.part selects by position k-1)
    int rho = 0;
    if (real) {
      const int bits = rc.part ? k - 1 : k, csub = rc.part == 1 ? c - 1 : c;
      for (int i = csub, p = bits - 1, rank = (int)team; i >= 1; --i) {
        while (s_binom[p][i] > rank) --p;
        rho |= 1 << p;
        rank -= s_binom[p][i];
        --p;
      }
      if (rc.part == 1) rho |= 1 << (k - 1);
    }
    const unsigned need = rc.need[k - c] & ((2u << (c >> 1)) - 1);
    const int mu = k - c;
    double2 G[kMaxK / 2 + 1];
    for (int a = 0; a < K2; ++a) G[a] = make_double2(0.0, 0.0);
    for (int a = 0; 2 * a <= c; ++a) {
      if (!(need >> a & 1)) continue;  // the same for the whole warp (block, if T > 32)
      const int a2 = (c >> 1) - a;     // G(rho, 2a) = G(rho, c - 2a)
      if (a2 < a && (need >> a2 & 1)) {
        G[a] = G[a2];
        continue;
      }
      const int s = 2 * a;
      const bool direct = s <= c - s;  // enumerate sigma, or its complement in rho
      const int t = direct ? s : c - s;
      const int N = s_binom[c][t];
      const int lo = (int)((int64_t)N * member / T), hi = (int)((int64_t)N * (member + 1) / T);
      double gx = 0.0, gy = 0.0;
      if (real)
        for_subsets_range(rho, c, t, lo, hi - lo, s_binom, [&](int sub) {
          const int sg = direct ? sub : rho ^ sub;
          const double2 h1 = haf(sg), h2 = haf(rho ^ sg);
          gx = fma(h1.x, h2.x, fma(-h1.y, h2.y, gx));
          gy = fma(h1.x, h2.y, fma(h1.y, h2.x, gy));
        });
      for (int off = min(T, 32) >> 1; off > 0; off >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, off);
        gy += __shfl_xor_sync(0xffffffffu, gy, off);
      }
      if (T > 32) {  // the team's warps: their sums in warp order (every thread of the block is here)
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) s_team[w] = make_double2(gx, gy);
        __syncthreads();
        if (member == 0)
          for (int v = w + 1; v < w + T / 32; ++v) {
            gx += s_team[v].x;
            gy += s_team[v].y;
          }
        __syncthreads();
      }
      G[a] = make_double2(gx, gy);
    }
    if (real && member == 0) {
      // F is symmetric in (ja, jb): the diagonal once, each pair a < e twice
      double t = 0.0;
      for (int a = 0; 2 * a <= c; ++a) {
        if (!(need >> a & 1)) continue;
        for (int e = a; 2 * e <= c; ++e) {
          if (!(need >> e & 1)) continue;
          const double f = F[(a * K2 + e) * (k + 1) + mu];
          if (f != 0.0) t = fma(e == a ? f : 2.0 * f, G[a].x * G[e].x + G[a].y * G[e].y, t);
        }
      }
      int64_t w = 1;  // at most 20!, exact
      for (int v = 0; v < s_nrep[slot]; ++v) {
        const int mv = s_mult[slot][v], al = mv - __popc(rho & s_mask[slot][v]);
        for (int i = 2; i <= al; ++i) w *= i;
        w *= s_binom[mv][al];
      }
      acc = (double)w * t;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = seg / 2; s2 > 0; s2 >>= 1) {  // a fixed tree per segment
    if (lt < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (gridDim.x == 1) {  // the prefix's whole sum is this segment's
    if (lt == 0 && live) q_out[b] = red[threadIdx.x];
    return;
  }
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    part[(int64_t)b * gridDim.x + blockIdx.x] = red[0];
    __threadfence();  // the block sum before the count
    s_last = atomicAdd(&counters[b], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    // the prefix's last block: q_out[b] = the block sums in block order
    // (lane-strided, then a fixed butterfly), and the counter back to 0
    __threadfence();
    double sum = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) sum += __ldcg(part + (int64_t)b * gridDim.x + i);
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (threadIdx.x == 0) {
      q_out[b] = sum;
      counters[b] = 0;
    }
  }
}

// H_W[b][T] = Haf(B_{x_T}) / t^{|T|/2} for the sets with a Hafnian in the
// list (slot >= 0), 0 for the rest (odd |T|, and sizes that no term reads).
__global__ void rescale_kernel(const double* __restrict__ hafB, const int* __restrict__ slot, int count,
                               int k, SizeScale scale, double2* __restrict__ H, int batch) {
  const int64_t total = (int64_t)batch << k;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int T = (int)(q & ((1 << k) - 1));
    const int c = __popc(T);
    double2 v = make_double2(0.0, 0.0);
    const int j = slot[q];
    if (j >= 0) {
      const double sc = scale.s[c];
      v.x = hafB[2 * j] * sc;
      v.y = hafB[2 * j + 1] * sc;
    }
    H[q] = v;
  }
}

// Exponential-space variant (Appendix D) for the chain sampler: each sample's
// sampled prefix keeps its sub-Hafnians Haf(B_T) in a cache (index = position
// mask over the prefix x_1..x_{k-1}). A set T that holds the new photon
// (position k-1, mode l) needs no Hafnian of its own: expanding along that
// photon's row,
//   Haf(B_T) = sum_{i in T'} B(l, x_i) Haf(B_{T' \ i}),   T' = T minus position k-1,
// where every T' \ i is an even subset of the prefix, so its Hafnian is in the
// cache. The terms are added in increasing position order.
__device__ __forceinline__ double2 chain_expand(const double2* __restrict__ cache, const double2* __restrict__ Brow,
                                                const int* __restrict__ xs, int Tp) {
  double2 acc = make_double2(0.0, 0.0);
  for (int rest = Tp; rest; rest &= rest - 1) {
    const int i = __ffs(rest) - 1;
    const double2 b = Brow[xs[i]], h = cache[Tp ^ (1 << i)];
    acc.x = fma(b.x, h.x, fma(-b.y, h.y, acc.x));
    acc.y = fma(b.x, h.y, fma(b.y, h.x, acc.y));
  }
  return acc;
}

// The subsets of `bits` positions with the sizes t[i] (C(bits, t[i]) each,
// numbered from start[i]): the table entries that some term reads.
struct SubsetClasses {
  int bits = 0, ncls = 0;
  int t[kMaxK + 1];
  int64_t start[kMaxK + 2];
  __host__ __device__ int64_t total() const { return start[ncls]; }
};

// Entry r of the classes: its size class, then colex unranking of its rank
// (rank = sum_i C(p_i, i) over the positions p_1 < .. < p_t).
__device__ __forceinline__ int subset_of(const SubsetClasses& sc, int64_t r, const int (*binom)[kMaxK + 1]) {
  int cls = 0;
  while (r >= sc.start[cls + 1]) ++cls;
  int rank = (int)(r - sc.start[cls]), mask = 0;
  for (int i = sc.t[cls], p = sc.bits - 1; i >= 1; --i) {
    while (binom[p][i] > rank) --p;
    mask |= 1 << p;
    rank -= binom[p][i];
    --p;
  }
  return mask;
}

// The Pascal table into a block's shared memory.
__device__ __forceinline__ void fill_binom(int (*binom)[kMaxK + 1], int rows) {
  load_binom(binom, rows);
  __syncthreads();
}

// Step k's table, in one launch. When `samples` > 0 (the first pass of a
// step): Hp[s][T] = Haf(W_T) = Haf(B_T) t^{-|T|/2} for the sets T of sample s's
// prefix (k-1 positions) in the classes `pre` (the sizes some term reads; the
// others are not written), the half of the table that every candidate
// shares, and each sample's k modes for the sum over the sets without
// position k-1 (its prefix, then -1: a mode of its own) into pmodes[s * k ..].
// For candidates g0 .. g0 + cnt - 1 (candidate g: sample g / m, mode g % m):
// Hn[b][T'] = Haf(W) of T' plus the new photon (the expansion above), for the
// T' of the classes `nw` (odd T' whose set with the new photon has a size some
// term reads; the others are not written), and the candidate's k modes (its
// sample's prefix, then its own mode) into modes[b * k ..].
//   cache: caches of cstride entries; x: kMaxK sampled modes per sample.
__global__ void chain_table_kernel(const double2* __restrict__ cache, int64_t cstride, const double2* __restrict__ B,
                                   const int* __restrict__ x, int k, SubsetClasses pre, SubsetClasses nw,
                                   SizeScale scale, int samples, int64_t g0, int cnt, int m, double2* __restrict__ Hp,
                                   int* __restrict__ pmodes, double2* __restrict__ Hn, int* __restrict__ modes) {
  __shared__ int s_binom[kMaxK + 1][kMaxK + 1];
  fill_binom(s_binom, k);
  const int half = 1 << (k - 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t q = first; q < (int64_t)samples * k; q += stride) {
    const int64_t smp = q / k;
    const int i = (int)(q - smp * k);
    pmodes[q] = i < k - 1 ? x[smp * kMaxK + i] : -1;
  }
  const int64_t Ep = pre.total();
  for (int64_t q = first; q < (int64_t)samples * Ep; q += stride) {
    const int64_t smp = q / Ep;
    const int T = subset_of(pre, q - smp * Ep, s_binom);
    const double2 h = cache[smp * cstride + T];
    const double sc = scale.s[__popc(T)];
    Hp[smp * half + T] = make_double2(h.x * sc, h.y * sc);
  }
  for (int64_t q = first; q < (int64_t)cnt * k; q += stride) {
    const int64_t b = q / k, g = g0 + b, smp = g / m;
    const int i = (int)(q - b * k);
    modes[q] = i < k - 1 ? x[smp * kMaxK + i] : (int)(g - smp * m);
  }
  const int64_t E = nw.total();
  for (int64_t q = first; q < (int64_t)cnt * E; q += stride) {
    const int64_t b = q / E, g = g0 + b, smp = g / m;
    const int l = (int)(g - smp * m);
    const int T = subset_of(nw, q - b * E, s_binom);
    const double2 h = chain_expand(cache + smp * cstride, B + (int64_t)l * m, x + smp * kMaxK, T);
    const double sc = scale.s[__popc(T) + 1];
    Hn[b * half + T] = make_double2(h.x * sc, h.y * sc);
  }
}

// Every cache starts as Haf of the empty matrix, 1.
__global__ void chain_init_kernel(double2* __restrict__ cache, int64_t cstride, int samples) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < samples; s += gridDim.x * blockDim.x)
    cache[s * cstride] = make_double2(1.0, 0.0);
}

// Step k's draw for sample blockIdx.y, then (k < n) its cache update; every
// block of the sample draws (the same inputs give the same mode) and updates
// its share of the cache. The draw, by warp 0: the weights
// w_l = max(q_l + f_l s0, 0), l = 0..m-1 (with the per-sample sum s0 over the
// sets without the new photon, f_l = 1 + the multiplicity of l in the prefix;
// without it, w_l = max(q_l, 0)), their running sums in mode order (each lane
// a contiguous run of modes, the runs joined by a fixed warp scan), and x_k =
// the first l of positive weight whose running sum exceeds u_k times the total
// (m - 1 if there is none); block 0 writes it. The update:
// cache[T' | 2^(k-1)] = Haf(B) of T' plus x_k for every T' over the first k-1
// positions (the expansion above; 0 for even |T'|).
//   u: n uniforms per sample; x: kMaxK sampled modes per sample.
__global__ void chain_pick_kernel(const double* __restrict__ q, const double* __restrict__ s0,
                                  const double* __restrict__ u, int n, int k, int m, int* __restrict__ x,
                                  double2* __restrict__ cache, int64_t cstride, const double2* __restrict__ B) {
  __shared__ int s_pick;
  const int smp = blockIdx.y;
  const int* xs = x + (int64_t)smp * kMaxK;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double* qs = q + (int64_t)smp * m;
    const double sv = s0 ? s0[smp] : 0.0;
    auto weight = [&](int l) {
      if (!s0) return fmax(qs[l], 0.0);
      int mult = 1;  // 1 + the multiplicity of l in the prefix
      for (int i = 0; i < k - 1; ++i) mult += xs[i] == l;
      return fmax(fma((double)mult, sv, qs[l]), 0.0);
    };
    const int per = (m + 31) / 32, lo = min(m, lane * per), hi = min(m, lo + per);
    double part = 0.0;
    for (int l = lo; l < hi; ++l) part += weight(l);
    double inc = part;  // inclusive scan over the lanes, fixed order
    for (int off = 1; off < 32; off <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += v;
    }
    const double tot = __shfl_sync(0xffffffffu, inc, 31);
    double run = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) run = 0.0;
    const double target = u[(int64_t)smp * n + k - 1] * tot;
    int found = m;
    for (int l = lo; l < hi; ++l) {
      const double w = weight(l);
      run += w;
      if (w > 0.0 && run > target) {
        found = l;
        break;
      }
    }
    const unsigned ball = __ballot_sync(0xffffffffu, found < m);
    const int first = __shfl_sync(0xffffffffu, found, ball ? __ffs(ball) - 1 : 0);
    if (lane == 0) s_pick = ball ? first : m - 1;
  }
  __syncthreads();
  const int pick = s_pick;
  if (blockIdx.x == 0 && threadIdx.x == 0) x[(int64_t)smp * kMaxK + k - 1] = pick;
  if (k == n) return;
  const int half = 1 << (k - 1);
  double2* c = cache + (int64_t)smp * cstride;
  const double2* Brow = B + (int64_t)pick * m;
  for (int Tp = blockIdx.x * blockDim.x + threadIdx.x; Tp < half; Tp += gridDim.x * blockDim.x)
    c[half + Tp] = (__popc(Tp) & 1) ? chain_expand(c, Brow, xs, Tp) : make_double2(0.0, 0.0);
}

// Subsets that one prefix's sum enumerates, per size class of rho (0 where
// the class has no term in range).
int64_t rho_work(int k, int n, int c) {
  auto binom = [](int a, int b) -> int64_t {
    if (b < 0 || b > a) return 0;
    int64_t v = 1;
    for (int i = 1; i <= b; ++i) v = v * (a - b + i) / i;
    return v;
  };
  int64_t work = 0;
  for (int ja = 0; ja <= c; ja += 2) {
    bool any = false;
    for (int jb = 0; jb <= c && !any; jb += 2) any = theorem_range(k, n, k - c, ja, jb);
    const int a = ja / 2, a2 = c / 2 - a;  // G(rho, ja) = G(rho, c - ja), formed once
    bool twin = false;
    for (int jb = 0; jb <= c && !twin && a2 < a; jb += 2) twin = theorem_range(k, n, k - c, 2 * a2, jb);
    if (any && !twin) work += binom(c, std::min(ja, c - ja));
  }
  return work;
}

int64_t rho_count(int k, int c, int part) {
  auto binom = [](int a, int b) -> int64_t {
    if (b < 0 || b > a) return 0;
    int64_t v = 1;
    for (int i = 1; i <= b; ++i) v = v * (a - b + i) / i;
    return v;
  };
  return part == 0 ? binom(k, c) : part == 1 ? binom(k - 1, c - 1) : binom(k - 1, c);
}

// Subsets one launch enumerates per prefix.
int64_t prefix_work(int k, int n, int part) {
  int64_t w = 0;
  for (int c = 0; c <= k; c += 2) w += rho_count(k, c, part) * rho_work(k, n, c);
  return w;
}

// The classes for a launch over `batch` prefixes (batch 0: the widest teams,
// an upper bound on the threads of any batch).
RhoClasses rho_classes(int k, int n, int part, int64_t batch) {
  int64_t largest = 0;
  for (int c = 0; c <= k; c += 2)
    if (rho_count(k, c, part)) largest = std::max(largest, rho_work(k, n, c));
  const int64_t cap = largest >= kLargeSetWork ? kTeamWorkMaxLarge : kTeamWorkMax;
  const int64_t per_lane =
      std::min<int64_t>(cap, std::max<int64_t>(kTeamWorkMin, batch * prefix_work(k, n, part) / kResidentLanes));
  RhoClasses rc;
  rc.part = part;
  rc.start[0] = 0;
  for (int mu = 0; mu <= kMaxK; ++mu) {
    unsigned need = 0;
    for (int a = 0; mu <= k && a <= k / 2; ++a)
      for (int e = 0; e <= k / 2; ++e)
        if (theorem_range(k, n, mu, 2 * a, 2 * e)) need |= 1u << a;
    rc.need[mu] = need;
  }
  // the largest sets first: their teams run longest, so they start first and
  // the short ones fill in behind them
  for (int c = k & ~1; c >= 0; c -= 2) {
    const int64_t work = rho_work(k, n, c), count = rho_count(k, c, part);
    if (!work || !count) continue;
    int T = 1;
    while (T < kMargThreads && (int64_t)T * per_lane < work) T *= 2;
    const int i = rc.ncls++;
    const int64_t align = T > 32 ? kMargThreads : 32;  // teams of several warps own whole blocks
    rc.start[i] = (rc.start[i] + align - 1) / align * align;
    rc.c[i] = c;
    rc.team[i] = T;
    rc.count[i] = count;
    rc.start[i + 1] = rc.start[i] + (count * T + align - 1) / align * align;
  }
  return rc;
}

int marginal_blocks(int k, int n, int part, int64_t batch) {
  return (int)std::max<int64_t>(1, (rho_classes(k, n, part, batch).total() + kMargThreads - 1) / kMargThreads);
}

// At least marginal_blocks for any batch: the widest teams (batch 0), plus
// the block alignment that narrower teams may add ahead of each class.
int marginal_blocks_bound(int k, int n, int part) { return marginal_blocks(k, n, part, 0) + 2 * (kMaxK / 2 + 1); }

// The sum for `batch` prefixes: q_out[b] for each (part: batch * blocks
// doubles; counters: batch zeros, left at zero).
cudaError_t launch_marginals(int k, int n, const double2* Hlo, int64_t slo, int64_t lo_off, int lo_div,
                             const double2* Hhi, int64_t shi, const double* F, const int* modes, int batch,
                             double* part, unsigned* counters, double* q_out, cudaStream_t st, int sel = 0) {
  const RhoClasses rc = rho_classes(k, n, sel, batch);
  const int nblk = (int)std::max<int64_t>(1, (rc.total() + kMargThreads - 1) / kMargThreads);
  // a prefix whose sets need at most half a block shares the block with others
  int seg = kMargThreads;
  while (nblk == 1 && seg > 32 && rc.total() <= seg / 2) seg /= 2;
  const int per = kMargThreads / seg;
  marginal_terms_kernel<<<dim3(nblk, (batch + per - 1) / per), kMargThreads, 0, st>>>(
      k, n, rc, Hlo, slo, lo_off, lo_div, Hhi, shi, F, modes, part, counters, q_out, batch, seg);
  return cudaGetLastError();
}

// Bit s set if some term of the Theorem 1 sum at prefix length k reads a
// sub-Hafnian of s photons (a sigma of a size in range, or its complement in rho).
unsigned needed_sizes(int k, int n) {
  unsigned sizes = 0;
  for (int c = 0; c <= k; c += 2)
    for (int ja = 0; ja <= c; ja += 2)
      for (int jb = 0; jb <= c; jb += 2)
        if (theorem_range(k, n, k - c, ja, jb)) sizes |= (1u << ja) | (1u << (c - ja));
  return sizes;
}

// The subsets of `bits` positions of size s - shift for the sizes s marked in
// `sizes` (bit s: s photons).
SubsetClasses subset_classes(int bits, unsigned sizes, int shift) {
  SubsetClasses sc;
  sc.bits = bits;
  sc.start[0] = 0;
  for (int s = 0; s <= kMaxK; ++s) {
    const int t = s - shift;
    if (!(sizes >> s & 1u) || t < 0 || t > bits) continue;
    int64_t cnt = 1;
    for (int i = 1; i <= t; ++i) cnt = cnt * (bits - t + i) / i;
    sc.t[sc.ncls] = t;
    sc.start[sc.ncls + 1] = sc.start[sc.ncls] + cnt;
    ++sc.ncls;
  }
  return sc;
}

size_t marginal_part_bytes(int k, int n, int batch) {
  return sizeof(double) * (size_t)marginal_blocks_bound(k, n, 0) * batch;
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
  std::vector<int> idx, nv_list, slot((size_t)batch * nsub, 0);
  std::vector<int64_t> offs;
  const unsigned sizes = needed_sizes(kk, n);  // the sub-Hafnian sizes that some term reads
  for (int b = 0; b < batch; ++b) {
    const int* xb = hx.data() + (size_t)b * kk;
    for (int T = 0; T < nsub; ++T) {
      slot[(size_t)b * nsub + T] = -1;
      if (!(sizes >> __builtin_popcount(T) & 1u)) continue;
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
  }
  if (idx.empty()) idx.push_back(0);
  const int nh = (int)nv_list.size();
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t hafB_b = al(16 * (size_t)nh), H_b = al(16 * ((size_t)batch << kk)), slot_b = al(4 * slot.size());
  const size_t F_b = al(8 * (size_t)fcoef_stride(kk)), x_b = al(4 * hx.size()), q_b = al(8 * (size_t)batch);
  const size_t part_b = al(marginal_part_bytes(kk, n, batch)), cnt_b = al(4 * (size_t)std::min(batch, 65535));
  void* tmp = nullptr;
  cudaError_t e = scratch_alloc(&tmp, hafB_b + H_b + slot_b + F_b + x_b + q_b + part_b + cnt_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "marginal scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double* d_hafB = (double*)t;
  double2* d_H = (double2*)(t + hafB_b);
  int* d_slot = (int*)(t + hafB_b + H_b);
  double* d_F = (double*)(t + hafB_b + H_b + slot_b);
  int* d_x = (int*)(t + hafB_b + H_b + slot_b + F_b);
  double* d_q = (double*)(t + hafB_b + H_b + slot_b + F_b + x_b);
  double* d_part = (double*)(t + hafB_b + H_b + slot_b + F_b + x_b + q_b);
  unsigned* d_count = (unsigned*)(t + hafB_b + H_b + slot_b + F_b + x_b + q_b + part_b);
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
        (e = cudaMemcpyAsync(d_x, hx.data(), 4 * hx.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_count, 0, cnt_b, st)) != cudaSuccess) {
      ret = cuda_fail(e, "marginal upload");
      break;
    }
    rescale_kernel<<<std::min(4096, (int)((((int64_t)batch << kk) + 255) / 256)), 256, 0, st>>>(
        d_hafB, d_slot, nh, kk, size_scale(k->t_uniform), d_H, batch);
    fcoef_kernel<<<dim3((int)((fcoef_stride(kk) + 255) / 256), 1), 256, 0, st>>>(kk, n, k->m, 0, d_F);
    double* qd = q_dev ? q_out : d_q;
    const int nblk = marginal_blocks_bound(kk, n, 0);
    for (int b0 = 0; b0 < batch && e == cudaSuccess; b0 += 65535)  // the grid's y extent
      e = launch_marginals(kk, n, d_H + ((int64_t)b0 << kk), (int64_t)1 << kk, 0, 1,
                           d_H + ((int64_t)b0 << kk) + (kk > 0 ? (int64_t)1 << (kk - 1) : 0), (int64_t)1 << kk, d_F,
                           d_x + (int64_t)b0 * kk, std::min(65535, batch - b0), d_part + (int64_t)b0 * nblk,
                           d_count, qd + b0, st);
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

// Algorithm 1 for `samples` independent samples at once: x_k of each drawn
// from its m conditional weights q_n(x_1..x_{k-1}, l), l = 0..m-1, with its
// own uniform number (inverse CDF in mode order). The exponential-space
// variant of Appendix D: each sample's prefix sub-Hafnians stay on the device
// across steps, and those of the sets that hold the new photon come from them
// by the row expansion of chain_table_kernel (at most k-1 products each, no
// Hafnian evaluation). A step covers every sample's candidates in the same
// launches, in chunks of at most 2^26 new table entries, and chain_pick_kernel
// draws every sample's mode on the device, so the steps run without a host
// synchronisation; the modes come back once per group of samples. Groups
// keep their caches within 2^28 entries (4 GB).
extern "C" int gbs_sample_chain_batch(const gbs_kernel* k, int n, int samples, const double* uniforms, void* stream,
                                      int* x_out) {
  clear_error();
  if (!k || (n > 0 && samples > 0 && (!uniforms || !x_out))) return fail(GBS_EINVAL, "null argument");
  if (samples < 0) return fail(GBS_EINVAL, "samples = %d is negative", samples);
  if (n < 0 || n > kMaxK || (n & 1)) return fail(GBS_ERANGE, "n = %d must be even and <= %d", n, kMaxK);
  if (n == 0 || samples == 0) return GBS_OK;
  if (!k->r_uniform) return fail(GBS_EINVAL, "marginals need identical squeezing on every mode");
  if (!(k->t_uniform > 0.0)) return fail(GBS_EINVAL, "marginals need r > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = k->m;
  const int group = std::min({samples, std::max(1, (1 << 28) >> n), 65535});
  // candidates per pass: at most 2^26 new table entries (1 GB), and the grid's y extent
  auto chunk_of = [&](int kk) {
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)group * m, 65535, (int64_t)1 << (27 - kk)}));
  };
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int64_t cstride = (int64_t)1 << n;
  size_t Hn_n = 0, part_n = 0, modes_n = 0;
  for (int kk = 1; kk <= n; ++kk) {
    Hn_n = std::max(Hn_n, (size_t)chunk_of(kk) << (kk - 1));
    part_n = std::max({part_n, (size_t)marginal_blocks_bound(kk, n, 0) * chunk_of(kk),
                       (size_t)marginal_blocks_bound(kk, n, 1) * chunk_of(kk),
                       (size_t)marginal_blocks_bound(kk, n, 2) * group});
    modes_n = std::max(modes_n, (size_t)chunk_of(kk) * kk);
  }
  const int64_t fstride = fcoef_stride(n);  // one F table per prefix length 1..n
  const size_t cache_b = al(16 * (size_t)(group * cstride)), x_b = al(4 * (size_t)group * kMaxK);
  const size_t Hp_b = al(16 * ((size_t)group << (n - 1))), Hn_b = al(16 * Hn_n), F_b = al(8 * (size_t)(n * fstride));
  const size_t md_b = al(4 * modes_n), q_b = al(8 * (size_t)group * (m + 1)), part_b = al(8 * part_n);
  const size_t pm_b = al(4 * (size_t)group * n), u_b = al(8 * (size_t)group * n);
  size_t cnt_n = (size_t)group;
  for (int kk = 1; kk <= n; ++kk) cnt_n = std::max(cnt_n, (size_t)chunk_of(kk));
  const size_t cnt_b = al(4 * cnt_n);
  void* tmp = nullptr;
  cudaError_t e =
      scratch_alloc(&tmp, cache_b + x_b + Hp_b + Hn_b + F_b + md_b + q_b + part_b + pm_b + u_b + cnt_b, st);
  if (e != cudaSuccess) return fail(GBS_ENOMEM, "chain scratch: %s", cudaGetErrorString(e));
  unsigned char* t = (unsigned char*)tmp;
  double2* d_cache = (double2*)t;
  int* d_x = (int*)(t += cache_b);
  double2* d_Hp = (double2*)(t += x_b);
  double2* d_Hn = (double2*)(t += Hp_b);
  double* d_F = (double*)(t += Hn_b);
  int* d_modes = (int*)(t += F_b);
  double* d_q = (double*)(t += md_b);
  double* d_part = (double*)(t += q_b);
  int* d_pmodes = (int*)(t += part_b);
  double* d_u = (double*)(t += pm_b);
  unsigned* d_count = (unsigned*)(t += u_b);  // per prefix: blocks of the terms kernel done (left at 0)
  double* d_s0 = d_q + (size_t)group * m;  // per sample: the sum over the sets without the new photon
  const double2* B = (const double2*)k->B;
  const SizeScale scale = size_scale(k->t_uniform);
  std::vector<int> hx((size_t)group * kMaxK);
  int ret = GBS_OK;
  fcoef_kernel<<<dim3((int)((fstride + 255) / 256), n), 256, 0, st>>>(1, n, m, fstride, d_F);
  if ((e = cudaMemsetAsync(d_count, 0, 4 * cnt_n, st)) != cudaSuccess) ret = cuda_fail(e, "chain counters");
  for (int s0 = 0; s0 < samples && ret == GBS_OK; s0 += group) {
    const int S = std::min(group, samples - s0);
    chain_init_kernel<<<(S + 255) / 256, 256, 0, st>>>(d_cache, cstride, S);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_u, uniforms + (size_t)s0 * n, 8 * (size_t)S * n, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess) {
      ret = cuda_fail(e, "chain setup");
      break;
    }
    for (int kk = 1; kk <= n && ret == GBS_OK; ++kk) {
      const int half = 1 << (kk - 1);
      const int chunk = chunk_of(kk);
      const unsigned sizes = needed_sizes(kk, n);
      const SubsetClasses pre = subset_classes(kk - 1, sizes, 0), nw = subset_classes(kk - 1, sizes, 1);
      const int64_t items = (int64_t)S * m;
      // On steps with much work, the sets without the new photon get one sum
      // per sample (the candidates differ there only by the factor 1 + the
      // multiplicity of their mode); on light steps the extra launch would
      // cost more than the work it saves.
      const bool split = items * prefix_work(kk, n, 0) >= ((int64_t)1 << 24);
      e = cudaSuccess;
      for (int64_t g0 = 0; g0 < items && e == cudaSuccess; g0 += chunk) {
        const int cnt = (int)std::min<int64_t>(chunk, items - g0);
        const int Sp = g0 == 0 ? S : 0;  // the first pass also writes the prefix half
        const int64_t work = std::max({(int64_t)cnt * kk, cnt * nw.total(), (int64_t)Sp * kk, Sp * pre.total()});
        chain_table_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(4096, (work + 255) / 256)), 256, 0, st>>>(
            d_cache, cstride, B, d_x, kk, pre, nw, scale, Sp, g0, cnt, m, d_Hp, d_pmodes, d_Hn, d_modes);
        e = cudaGetLastError();
        if (e == cudaSuccess && split && g0 == 0)
          e = launch_marginals(kk, n, d_Hp, half, 0, 1, d_Hp, 0, d_F + (kk - 1) * fstride, d_pmodes, S, d_part,
                               d_count, d_s0, st, 2);
        if (e == cudaSuccess)
          e = launch_marginals(kk, n, d_Hp, half, g0, m, d_Hn, half, d_F + (kk - 1) * fstride, d_modes, cnt, d_part,
                               d_count, d_q + g0, st, split ? 1 : 0);
      }
      if (e != cudaSuccess) {
        ret = cuda_fail(e, "chain kernels");
        break;
      }
      // the draws, then the chosen modes' new sub-Hafnians (sets that hold
      // position kk-1) into the caches
      const int nb = kk < n ? (int)std::max<int64_t>(1, std::min<int64_t>(64, (half + 1023) / 1024)) : 1;
      chain_pick_kernel<<<dim3(nb, S), 256, 0, st>>>(d_q, split ? d_s0 : nullptr, d_u, n, kk, m, d_x, d_cache, cstride,
                                                      B);
      if ((e = cudaGetLastError()) != cudaSuccess) {
        ret = cuda_fail(e, "chain draw");
        break;
      }
    }
    if (ret != GBS_OK) break;
    if ((e = cudaMemcpyAsync(hx.data(), d_x, 4 * (size_t)S * kMaxK, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      ret = cuda_fail(e, "chain samples");
      break;
    }
    for (int s = 0; s < S; ++s)
      for (int i = 0; i < n; ++i) x_out[(size_t)(s0 + s) * n + i] = hx[(size_t)s * kMaxK + i];
  }
  scratch_free(tmp, st);
  return ret;
}

// One sample: the batch of one.
extern "C" int gbs_sample_chain(const gbs_kernel* k, int n, const double* uniforms, void* stream, int* x_out) {
  return gbs_sample_chain_batch(k, n, 1, uniforms, stream, x_out);
}

namespace {

// Step 1 of Sec. 3: n from P_n truncated at n_max (renormalised) by the inverse
// CDF with the uniform u.
int pick_photon_number(const std::vector<double>& Pn, int n_max, double tot, double u) {
  const double target = u * tot;
  double run = 0.0;
  for (int v = 0; v <= n_max; v += 2) {
    run += std::max(Pn[v], 0.0);
    if (run > target) return v;
  }
  return n_max & ~1;
}

// P_n for n = 0..n_max and the total of its even entries (GBS_EINVAL if 0).
int truncated_pn(const gbs_kernel* k, int n_max, void* stream, std::vector<double>& Pn, double& tot) {
  Pn.assign((size_t)n_max + 1, 0.0);
  const int rc = gbs_photon_number_dist(k, n_max, stream, Pn.data());
  if (rc) return rc;
  tot = 0.0;
  for (int v = 0; v <= n_max; v += 2) tot += std::max(Pn[v], 0.0);
  if (!(tot > 0.0)) return fail(GBS_EINVAL, "P_n vanishes for every n <= n_max");
  return GBS_OK;
}

}  // namespace

// Steps 1-3 of Sec. 3: n from P_n (truncated at n_max, renormalised) by the
// inverse CDF with uniforms[0], then the chain rule for the n photons.
extern "C" int gbs_sample(const gbs_kernel* k, int n_max, const double* uniforms, void* stream, int* n_out,
                          int* x_out) {
  clear_error();
  if (!k || !uniforms || !n_out || (n_max > 0 && !x_out)) return fail(GBS_EINVAL, "null argument");
  if (n_max < 0 || n_max > kMaxK) return fail(GBS_ERANGE, "n_max = %d outside [0, %d]", n_max, kMaxK);
  if (!k->r_uniform) return fail(GBS_EINVAL, "sampling needs identical squeezing on every mode");
  std::vector<double> Pn;
  double tot = 0.0;
  int rc = truncated_pn(k, n_max, stream, Pn, tot);
  if (rc) return rc;
  const int n = pick_photon_number(Pn, n_max, tot, uniforms[0]);
  *n_out = n;
  if (n == 0) return GBS_OK;
  return gbs_sample_chain(k, n, uniforms + 1, stream, x_out);
}

// gbs_sample for `samples` samples at once: each draws its n, then the samples
// of each n run as one gbs_sample_chain_batch.
extern "C" int gbs_sample_batch(const gbs_kernel* k, int n_max, int samples, const double* uniforms, void* stream,
                                int* n_out, int* x_out) {
  clear_error();
  if (!k || (samples > 0 && (!uniforms || !n_out || (n_max > 0 && !x_out)))) return fail(GBS_EINVAL, "null argument");
  if (samples < 0) return fail(GBS_EINVAL, "samples = %d is negative", samples);
  if (n_max < 0 || n_max > kMaxK) return fail(GBS_ERANGE, "n_max = %d outside [0, %d]", n_max, kMaxK);
  if (!k->r_uniform) return fail(GBS_EINVAL, "sampling needs identical squeezing on every mode");
  if (samples == 0) return GBS_OK;
  std::vector<double> Pn;
  double tot = 0.0;
  int rc = truncated_pn(k, n_max, stream, Pn, tot);
  if (rc) return rc;
  const size_t row = (size_t)n_max + 1;
  std::vector<std::vector<int>> by_n((size_t)n_max + 1);
  for (int s = 0; s < samples; ++s) {
    const int n = pick_photon_number(Pn, n_max, tot, uniforms[s * row]);
    n_out[s] = n;
    by_n[n].push_back(s);
    for (int i = 0; i < n_max; ++i) x_out[(size_t)s * n_max + i] = -1;
  }
  for (int n = 2; n <= n_max; n += 2) {
    const std::vector<int>& idx = by_n[n];
    if (idx.empty()) continue;
    std::vector<double> u(idx.size() * n);
    std::vector<int> x(idx.size() * n);
    for (size_t j = 0; j < idx.size(); ++j)
      for (int i = 0; i < n; ++i) u[j * n + i] = uniforms[idx[j] * row + 1 + i];
    if ((rc = gbs_sample_chain_batch(k, n, (int)idx.size(), u.data(), stream, x.data())) != GBS_OK) return rc;
    for (size_t j = 0; j < idx.size(); ++j)
      for (int i = 0; i < n; ++i) x_out[(size_t)idx[j] * n_max + i] = x[j * n + i];
  }
  return GBS_OK;
}
