// Subset-sum Hafnian kernels (FP64 and mixed FP32 paths) and the per-pattern
// finalisation.
//
// Method (Sec. 2.3 cites it for the O(n^3 2^{n/2}) cost; Bjorklund, Gupt,
// Quesada): for an n x n symmetric A, n = 2h, pairs {2i, 2i+1},
//     Haf(A) = sum_{S subset of [h]} (-1)^{h-|S|} f(X A_S),
//     f(M)   = [x^h] exp( sum_{k=1..h} tr(M^k) x^k / (2k) ),
// where A_S keeps the rows/columns of the pairs in S and X swaps the two
// members of every pair. Per subset (order N = 2|S|) the kernel
//   1. gathers A_S into shared memory (packed upper triangle, zero diagonal),
//   2. forms the power traces tr((X A_S)^k), k = 1..h, through the symmetric
//      matrices R_k = A_S (X A_S)^{k-1}:  (X A_S)^k = X R_k,
//      R_{a+b} = R_a X R_b  (symmetric, so only the upper triangle is
//      computed), tr(X R_k) = 2 sum_t R_k[2t][2t+1] and
//      tr(X R_a X R_b) = sum_{i,j} R_a[i][j] R_b[i^1][j^1];
//      a fixed schedule per h picks the fewest such products that cover
//      k = 1..h (at most five for h <= 15),
//   3. expands e = exp(sum_k tr_k x^k / (2k)): e_k = (1/(2k)) sum_j tr_j e_{k-j},
//      f = e_h,
//   4. adds (-1)^{h-|S|} f to a compensated (double-double or float-float)
//      accumulator.
// Power traces by products keep the per-term rounding error near the unit
// roundoff; a similarity reduction (Hessenberg form and a characteristic
// polynomial recurrence) was measured to lose about an order of magnitude per
// term, which the cancellation of the signed sum (up to ~1e7 at n = 30)
// turns into errors above 1e-10.
//
// GB300 mapping. FP64 issue costs the same per warp instruction whatever the
// active mask, so all 32 lanes must do useful FP64 work: a warp works on
// subsets of one order N only (uniform control flow), split into G = 32/L lane
// groups, each group owning one subset's matrices in shared memory and
// spreading the output entries of each product (and the terms of each trace)
// evenly over its L lanes. Integer work (unranking, packed-triangle
// addressing) runs on other pipes beside the FP64 pipe. Work items are taken
// from a global queue by persistent warps; each item writes one partial sum,
// and partials are added per pattern in a fixed order, so results do not
// depend on scheduling.
#include <math.h>

#include <atomic>

#include "gbs_internal.cuh"

namespace gbs {
namespace {

template <typename T> struct V2t;
template <> struct V2t<double> { typedef double2 type; };
template <> struct V2t<float> { typedef float2 type; };
template <typename T> using C2 = typename V2t<T>::type;

template <typename T> __device__ __forceinline__ C2<T> mk(T x, T y) {
  C2<T> r;
  r.x = x;
  r.y = y;
  return r;
}
// acc + a*b (4 fused multiply-adds)
template <typename T> __device__ __forceinline__ C2<T> cfma(C2<T> a, C2<T> b, C2<T> acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc - a*b
template <typename T> __device__ __forceinline__ C2<T> cfms(C2<T> a, C2<T> b, C2<T> acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  C2<T> r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

// Compensated accumulation (Knuth two-sum, Dekker fast two-sum).
template <typename T> struct Comp { T hi, lo; };
template <typename T> __device__ __forceinline__ void comp_add(Comp<T>& a, T v) {
  const T s = a.hi + v;
  const T bb = s - a.hi;
  const T e = (a.hi - (s - bb)) + (v - bb);
  const T lo = a.lo + e;
  const T h2 = s + lo;
  a.lo = lo - (h2 - s);
  a.hi = h2;
}
__device__ __forceinline__ void dd_add(double& ahi, double& alo, double bhi, double blo) {
  double s = ahi + bhi;
  double bb = s - ahi;
  double e = (ahi - (s - bb)) + (bhi - bb);
  double t = alo + blo;
  double tb = t - alo;
  double f = (alo - (t - tb)) + (blo - tb);
  e += t;
  double h = s + e;
  e = e - (h - s);
  e += f;
  double h2 = h + e;
  alo = e - (h2 - h);
  ahi = h2;
}

struct Tables {
  int binom[kMaxH + 1][kMaxH + 1];  // C(a, b), a, b <= 16
  double inv2k[kMaxH + 1];          // 1 / (2k)
};

// Power-trace schedule per h: the fewest products R_{a+b} = R_a X R_b whose
// index set F (with R_1 = A_S) satisfies F + F >= {1..h}, each trace k taken
// as tr(X R_k) when k is in F, else tr(X R_a X R_b) with a + b = k (a = b
// where R_{k/2} is kept: that square trace needs about half the terms), and
// each R kept in a buffer that is reused once its traces are taken. Among the
// schedules with the fewest products, the rows for h = 7, 8, 11, 12, 15, 16
// (found by an exhaustive search) hold the fewest matrices at once (3, 3, 3,
// 3, 4, 4) and have the cheapest traces. Products per h = 1..16:
// 0 0 1 1 2 2 3 3 3 3 4 4 4 4 5 5.
enum { kEnd = -1, kProd = 0, kTr1 = 1, kTr2 = 2 };
struct SchedOp {
  signed char kind;  // kProd: buf[k] = buf[a] X buf[b]; kTr1: p_k = tr(X buf[a]); kTr2: p_k = tr(X buf[a] X buf[b])
  signed char k, a, b;
};
constexpr int kMaxOps = 24;
__constant__ SchedOp c_sched[kMaxH + 1][kMaxOps] = {
    {{kEnd, 0, 0, 0}},  // h = 0
    {{kTr1, 1, 0, 0}, {kEnd, 0, 0, 0}},  // h = 1
    {{kTr1, 1, 0, 0}, {kTr2, 2, 0, 0}, {kEnd, 0, 0, 0}},  // h = 2
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 3, 1, 0}, {kEnd, 0, 0, 0}},  // h = 3
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 3, 1, 0}, {kTr2, 4, 1, 1}, {kEnd, 0, 0, 0}},  // h = 4
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 4, 1, 1}, {kTr2, 5, 2, 1}, {kEnd, 0, 0, 0}},  // h = 5
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 4, 1, 1}, {kTr2, 5, 2, 1}, {kTr2, 6, 2, 2}, {kEnd, 0, 0, 0}},  // h = 6
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 4, 1, 1}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 6, 2, 2}, {kProd, 0, 2, 1}, {kTr1, 5, 0, 0}, {kTr2, 7, 0, 1}, {kEnd, 0, 0, 0}},  // h = 7
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 5, 2, 1}, {kTr2, 6, 2, 2}, {kProd, 1, 2, 0}, {kTr1, 4, 1, 0}, {kTr2, 7, 1, 2}, {kTr2, 8, 1, 1}, {kEnd, 0, 0, 0}},  // h = 8
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 0}, {kProd, 3, 2, 2}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 4, 1, 1}, {kTr2, 5, 2, 1}, {kTr1, 6, 3, 0}, {kTr2, 7, 3, 0}, {kTr2, 8, 3, 1}, {kTr2, 9, 3, 2}, {kEnd, 0, 0, 0}},  // h = 9
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 1}, {kProd, 3, 2, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 3, 1, 0}, {kTr1, 4, 2, 0}, {kTr1, 5, 3, 0}, {kTr2, 6, 2, 1}, {kTr2, 7, 3, 1}, {kTr2, 8, 2, 2}, {kTr2, 9, 3, 2}, {kTr2, 10, 3, 3}, {kEnd, 0, 0, 0}},  // h = 10
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 4, 1, 1}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kProd, 0, 2, 1}, {kTr1, 5, 0, 0}, {kTr2, 7, 0, 1}, {kTr2, 8, 0, 2}, {kTr2, 10, 0, 0}, {kProd, 1, 2, 2}, {kTr1, 6, 1, 0}, {kTr2, 9, 1, 2}, {kTr2, 11, 1, 0}, {kEnd, 0, 0, 0}},  // h = 11
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 4, 1, 1}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kProd, 0, 2, 1}, {kTr1, 5, 0, 0}, {kTr2, 7, 0, 1}, {kTr2, 8, 0, 2}, {kTr2, 10, 0, 0}, {kProd, 1, 2, 2}, {kTr1, 6, 1, 0}, {kTr2, 9, 1, 2}, {kTr2, 11, 1, 0}, {kTr2, 12, 1, 1}, {kEnd, 0, 0, 0}},  // h = 12
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 1}, {kProd, 3, 2, 1}, {kProd, 4, 3, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 3, 1, 0}, {kTr1, 4, 2, 0}, {kTr2, 5, 2, 0}, {kTr1, 6, 3, 0}, {kTr1, 7, 4, 0}, {kTr2, 8, 2, 2}, {kTr2, 9, 4, 1}, {kTr2, 10, 3, 2}, {kTr2, 11, 4, 2}, {kTr2, 12, 3, 3}, {kTr2, 13, 4, 3}, {kEnd, 0, 0, 0}},  // h = 13
    {{kProd, 1, 0, 0}, {kProd, 2, 1, 1}, {kProd, 3, 2, 1}, {kProd, 4, 3, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 3, 1, 0}, {kTr1, 4, 2, 0}, {kTr2, 5, 2, 0}, {kTr1, 6, 3, 0}, {kTr1, 7, 4, 0}, {kTr2, 8, 2, 2}, {kTr2, 9, 4, 1}, {kTr2, 10, 3, 2}, {kTr2, 11, 4, 2}, {kTr2, 12, 3, 3}, {kTr2, 13, 4, 3}, {kTr2, 14, 4, 4}, {kEnd, 0, 0, 0}},  // h = 14
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 4, 1, 1}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 6, 2, 2}, {kProd, 3, 2, 1}, {kTr1, 5, 3, 0}, {kTr2, 10, 3, 3}, {kProd, 0, 3, 1}, {kTr1, 7, 0, 0}, {kTr2, 9, 0, 1}, {kTr2, 12, 0, 3}, {kTr2, 14, 0, 0}, {kProd, 1, 3, 2}, {kTr1, 8, 1, 0}, {kTr2, 11, 1, 2}, {kTr2, 13, 1, 3}, {kTr2, 15, 1, 0}, {kEnd, 0, 0, 0}},  // h = 15
    {{kProd, 1, 0, 0}, {kTr1, 1, 0, 0}, {kTr1, 2, 1, 0}, {kTr2, 4, 1, 1}, {kProd, 2, 1, 0}, {kTr1, 3, 2, 0}, {kTr2, 6, 2, 2}, {kProd, 3, 2, 1}, {kTr1, 5, 3, 0}, {kTr2, 10, 3, 3}, {kProd, 0, 3, 1}, {kTr1, 7, 0, 0}, {kTr2, 9, 0, 1}, {kTr2, 12, 0, 3}, {kTr2, 14, 0, 0}, {kProd, 1, 3, 2}, {kTr1, 8, 1, 0}, {kTr2, 11, 1, 2}, {kTr2, 13, 1, 3}, {kTr2, 15, 1, 0}, {kTr2, 16, 1, 1}, {kEnd, 0, 0, 0}},  // h = 16
};

// Asynchronous 8-byte copy global -> shared (cp.async, bypassing registers);
// zero = true writes zeros and reads nothing. Completed copies are visible to
// the issuing thread after cp_async_wait_all, to the rest of the warp after a
// __syncwarp that follows it.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool zero) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(zero ? 0 : 8) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Position of entry (r, c) of a symmetric N x N matrix stored as its packed
// upper triangle, rows in order: row r holds columns r..N-1.
__device__ __forceinline__ int tri_off(int r, int N) { return r * N - ((r * (r - 1)) >> 1); }
__device__ __forceinline__ int tri_pos(int r, int c, int N) {
  const int lo = min(r, c), hi = max(r, c);
  return tri_off(lo, N) + hi - lo;
}
// Advance the packed-upper coordinate (i, j) by `step` entries.
__device__ __forceinline__ void tri_advance(int& i, int& j, int step, int N) {
  j += step;
  while (j >= N && i < N) {
    const int over = j - N;
    ++i;
    j = i + over;
  }
}

// Sum over the L lanes of a group (groups are aligned blocks of L lanes).
template <typename T>
__device__ __forceinline__ C2<T> group_sum(C2<T> v, int L) {
  for (int off = L >> 1; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Sums over the L >= 2 lanes of a group of two values at once: at the first
// level (offset L/2) each lane sends its partner the value the partner keeps,
// so the lower half of the group carries a's partial sums and the upper half
// b's; the remaining levels sum each within its half. Lane 0 of the group ends
// with the total of a, lane L/2 with the total of b: one addition per level
// for both values instead of one per level for each.
template <typename T>
__device__ __forceinline__ C2<T> group_sum2(C2<T> a, C2<T> b, int l, int L) {
  const int half = L >> 1;
  const bool up = (l & half) != 0;
  const C2<T> send = up ? a : b;
  C2<T> keep = up ? b : a;
  keep.x += __shfl_xor_sync(0xffffffffu, send.x, half);
  keep.y += __shfl_xor_sync(0xffffffffu, send.y, half);
  for (int off = half >> 1; off > 0; off >>= 1) {
    keep.x += __shfl_xor_sync(0xffffffffu, keep.x, off);
    keep.y += __shfl_xor_sync(0xffffffffu, keep.y, off);
  }
  return keep;
}

// dst = Ra X Rb (upper triangle), X swapping 2t <-> 2t+1. Each lane takes
// two output entries at a time (e and e + L) so that four independent FMA
// chains are in flight.
template <typename T>
__device__ __forceinline__ void sym_prod(C2<T>* __restrict__ dst, const C2<T>* __restrict__ Ra,
                                         const C2<T>* __restrict__ Rb, int N, int P, int l, int L) {
  int i1 = 0, j1 = l;
  tri_advance(i1, j1, 0, N);
  for (int e = l; e < P; e += 2 * L) {
    if (e - l + L >= P) {
      // no lane has a second entry in this (last) pass: one chain only; the
      // condition is the same for every lane of the warp
      C2<T> acc = mk<T>(T(0), T(0));
      const int o1 = tri_off(i1, N);
      for (int k = 0; k < N; ++k) {
        const int ok = tri_off(k, N);
        const C2<T> a1 = (k >= i1) ? Ra[o1 + k - i1] : Ra[ok + i1 - k];
        acc = cfma<T>(a1, Rb[tri_pos(k ^ 1, j1, N)], acc);
      }
      dst[e] = acc;
      break;
    }
    int i2 = i1, j2 = j1;
    tri_advance(i2, j2, L, N);
    const bool two = (e + L < P);
    if (!two) {  // keep the second entry's loads in range; its result is dropped
      i2 = i1;
      j2 = j1;
    }
    C2<T> acc1 = mk<T>(T(0), T(0)), acc2 = mk<T>(T(0), T(0));
    const int o1 = tri_off(i1, N), o2 = tri_off(i2, N);
    for (int k = 0; k < N; ++k) {
      const int ok = tri_off(k, N);
      const C2<T> a1 = (k >= i1) ? Ra[o1 + k - i1] : Ra[ok + i1 - k];
      const C2<T> a2 = (k >= i2) ? Ra[o2 + k - i2] : Ra[ok + i2 - k];
      const int r = k ^ 1;
      const C2<T> b1 = Rb[tri_pos(r, j1, N)];
      const C2<T> b2 = Rb[tri_pos(r, j2, N)];
      acc1 = cfma<T>(a1, b1, acc1);
      acc2 = cfma<T>(a2, b2, acc2);
    }
    dst[e] = acc1;
    if (two) dst[e + L] = acc2;
    tri_advance(i1, j1, 2 * L, N);
  }
}

// tr(X Ra) = 2 sum_t Ra[2t][2t+1] (partial over this lane's pairs).
template <typename T>
__device__ __forceinline__ C2<T> tr1_part(const C2<T>* __restrict__ Ra, int N, int l, int L) {
  C2<T> acc = mk<T>(T(0), T(0));
  for (int t = l; 2 * t < N; t += L) {
    const C2<T> v = Ra[tri_off(2 * t, N) + 1];
    acc.x += v.x;
    acc.y += v.y;
  }
  acc.x *= T(2);
  acc.y *= T(2);
  return acc;
}

// tr(X Ra X Rb) = sum_{i,j} Ra[i][j] Rb[i^1][j^1] over the packed upper
// triangle, off-diagonal entries counted twice (partial over this lane).
template <typename T>
__device__ __forceinline__ C2<T> tr2_part(const C2<T>* __restrict__ Ra, const C2<T>* __restrict__ Rb,
                                          int N, int P, int l, int L) {
  C2<T> acc = mk<T>(T(0), T(0)), dg = mk<T>(T(0), T(0));
  int i = 0, j = l;
  tri_advance(i, j, 0, N);
  for (int e = l; e < P; e += L) {
    const C2<T> a = Ra[e];
    const C2<T> b = Rb[tri_pos(i ^ 1, j ^ 1, N)];
    const bool diag = (i == j);
    C2<T> cur = diag ? dg : acc;  // selects, not a divergent branch
    cur = cfma<T>(a, b, cur);
    dg = diag ? cur : dg;
    acc = diag ? acc : cur;
    tri_advance(i, j, L, N);
  }
  acc.x = fma(T(2), acc.x, dg.x);
  acc.y = fma(T(2), acc.y, dg.y);
  return acc;
}

// tr(X Ra X Ra): the term Ra[i][j] Ra[i^1][j^1] is unchanged by transposing
// (i, j) -> (j, i) and by swapping both indices within their pairs
// (i, j) -> (i^1, j^1), so one entry per orbit is enough: row 2t (columns
// j >= 2t) against row 2t+1,
//   T = 2 sum_t sum_{j >= 2t} c_j Ra[2t][j] Ra[2t+1][j^1],
// c_j = 1 for j in {2t, 2t+1} (orbits of two) and 2 otherwise (orbits of four):
// N(N+2)/4 terms instead of N(N+1)/2. The even rows are walked in packed order
// (row 2t holds N - 2t entries).
template <typename T>
__device__ __forceinline__ C2<T> tr2sq_part(const C2<T>* __restrict__ Ra, int N, int l, int L) {
  const int E = (N * N) / 4 + N / 2;
  C2<T> acc = mk<T>(T(0), T(0)), dg = mk<T>(T(0), T(0));
  int t = 0, j = l;
  while (j >= N && 2 * t < N) {
    const int over = j - N;
    ++t;
    j = 2 * t + over;
  }
  for (int e = l; e < E; e += L) {
    const int o = tri_off(2 * t, N), ow = o + (N - 2 * t);  // rows 2t and 2t+1
    const C2<T> a = Ra[o + j - 2 * t];
    const C2<T> b = (j == 2 * t + 1) ? a : Ra[ow + (j ^ 1) - 2 * t - 1];
    const bool w2 = j >= 2 * t + 2;
    C2<T> cur = w2 ? acc : dg;  // selects, not a divergent branch
    cur = cfma<T>(a, b, cur);
    acc = w2 ? cur : acc;
    dg = w2 ? dg : cur;
    j += L;
    while (j >= N && 2 * t < N) {
      const int over = j - N;
      ++t;
      j = 2 * t + over;
    }
  }
  acc.x = T(2) * fma(T(2), acc.x, dg.x);
  acc.y = T(2) * fma(T(2), acc.y, dg.y);
  return acc;
}

// R_2 = A_S X A_S (upper triangle) from the matrix's pair sums: entry (i, j)
// is low[S](I_i, I_j) + high[S](I_i, I_j), I_i = 2 pairs[i/2] + (i mod 2) the
// position of subset row i in the matrix and klo, khi the slots of S's low and
// high pairs. Since (A_S X A_S)(i, j) = sum_k A_S(i, k) A_S(k^1, j) and the k
// of S come in whole pairs, this is the product's sum grouped by pair: one
// complex addition per entry instead of 2s complex multiply-adds. pairs[]
// increases, so I_i <= I_j whenever i <= j. The loads of four entries are
// issued before their sums (the pair sums stream from L2 or memory).
__device__ __forceinline__ void pair_sum(double2* __restrict__ dst, const double2* __restrict__ q,
                                         const int* __restrict__ pairs, int N, int P, int W, int n,
                                         int klo, int khi, int l, int L) {
  int i = 0, j = l;
  tri_advance(i, j, 0, N);
  for (int e0 = l; e0 < P; e0 += 4 * L) {
    double2 a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e0 + u * L < P) {
        const int Ii = 2 * pairs[i >> 1] + (i & 1), Ij = 2 * pairs[j >> 1] + (j & 1);
        const double2* qe = q + (int64_t)(tri_off(Ii, n) + Ij - Ii) * W;
        a[u] = __ldg(qe + klo);
        b[u] = __ldg(qe + khi);
        tri_advance(i, j, L, N);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (e0 + u * L < P) dst[e0 + u * L] = make_double2(a[u].x + b[u].x, a[u].y + b[u].y);
  }
}

// ---- FP32 path: full N x N tiles (row stride N), rows read as float4 pairs.
// C[i][j] = sum_k Ra[i][k] Rb[k^1][j] = sum_t Ra[i][2t] Rb[j][2t+1] + Ra[i][2t+1] Rb[j][2t]
// (Rb symmetric), computed for i <= j and stored to both (i, j) and (j, i).
__device__ __forceinline__ float2 pair_dot(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                           int half, float2 acc) {
  for (int t = 0; t < half; ++t) {
    const float4 a = ra[t], b = rb[t];
    // (a.x + i a.y)(b.z + i b.w) + (a.z + i a.w)(b.x + i b.y)
    acc.x = fmaf(a.x, b.z, acc.x);
    acc.x = fmaf(-a.y, b.w, acc.x);
    acc.y = fmaf(a.x, b.w, acc.y);
    acc.y = fmaf(a.y, b.z, acc.y);
    acc.x = fmaf(a.z, b.x, acc.x);
    acc.x = fmaf(-a.w, b.y, acc.x);
    acc.y = fmaf(a.z, b.y, acc.y);
    acc.y = fmaf(a.w, b.x, acc.y);
  }
  return acc;
}

// C = Ra X Rb in 2 x 2 register blocks: block (r, c), r <= c, of the
// (N/2) x (N/2) grid of 2 x 2 blocks holds rows 2r, 2r+1 and columns 2c, 2c+1;
// per chunk t the lane loads four float4 (two rows of each operand) for 32
// FMAs. (One output per row pair would take two 16-byte loads per 8 FMAs,
// which shared-memory bandwidth, not the FP32 pipe, would bound.) Each output
// adds its t terms in increasing order; a diagonal block stores its
// (2r+1, 2r) entry from (2r, 2r+1), which keeps C exactly symmetric.
__device__ __forceinline__ void sym_prod_full(float2* __restrict__ dst, const float2* __restrict__ Ra,
                                              const float2* __restrict__ Rb, int N, int l, int L) {
  const int half = N >> 1, E = half * (half + 1) / 2;
  int r = 0, c = l;
  tri_advance(r, c, 0, half);
  for (int e = l; e < E; e += L) {
    const float4* a0 = reinterpret_cast<const float4*>(Ra + 2 * r * N);
    const float4* a1 = reinterpret_cast<const float4*>(Ra + (2 * r + 1) * N);
    const float4* b0 = reinterpret_cast<const float4*>(Rb + 2 * c * N);
    const float4* b1 = reinterpret_cast<const float4*>(Rb + (2 * c + 1) * N);
    float2 c00 = make_float2(0.f, 0.f), c01 = c00, c10 = c00, c11 = c00;
    for (int t = 0; t < half; ++t) {
      const float4 x0 = a0[t], x1 = a1[t], y0 = b0[t], y1 = b1[t];
      c00 = pair_dot(&x0, &y0, 1, c00);
      c01 = pair_dot(&x0, &y1, 1, c01);
      c10 = pair_dot(&x1, &y0, 1, c10);
      c11 = pair_dot(&x1, &y1, 1, c11);
    }
    const int i0 = 2 * r, j0 = 2 * c;
    dst[i0 * N + j0] = c00;
    dst[j0 * N + i0] = c00;
    dst[i0 * N + j0 + 1] = c01;
    dst[(j0 + 1) * N + i0] = c01;
    dst[(i0 + 1) * N + j0 + 1] = c11;
    dst[(j0 + 1) * N + i0 + 1] = c11;
    if (r != c) {
      dst[(i0 + 1) * N + j0] = c10;
      dst[j0 * N + i0 + 1] = c10;
    }
    tri_advance(r, c, L, half);
  }
}

// tr(X Ra) = 2 sum_t Ra[2t][2t+1] (partial over this lane's pairs).
__device__ __forceinline__ float2 tr1_full(const float2* __restrict__ Ra, int N, int l, int L) {
  float2 acc = make_float2(0.f, 0.f);
  for (int t = l; 2 * t < N; t += L) {
    const float2 v = Ra[2 * t * N + 2 * t + 1];
    acc.x += v.x;
    acc.y += v.y;
  }
  acc.x *= 2.f;
  acc.y *= 2.f;
  return acc;
}

// tr(X Ra X Rb) = sum_{p,u} B(p, u), B(p, u) = sum_{i in pair p} (Ra[i][2u]
// Rb[i^1][2u+1] + Ra[i][2u+1] Rb[i^1][2u]) the block of row pair p and column
// pair u. Both matrices are symmetric, so B(p, u) = B(u, p) and
// T = sum_p B(p, p) + 2 sum_{p < u} B(p, u): the upper triangle p <= u of the
// s x s block grid, s = N/2, walked like a packed triangle (partial over this
// lane's blocks). Half the products of the plain sum over all rows.
__device__ __forceinline__ float2 tr2_full(const float2* __restrict__ Ra, const float2* __restrict__ Rb,
                                           int N, int l, int L) {
  const int s = N >> 1, E = s * (s + 1) / 2;
  float2 acc = make_float2(0.f, 0.f), dg = make_float2(0.f, 0.f);
  int p = 0, u = l;
  tri_advance(p, u, 0, s);
  for (int e = l; e < E; e += L) {
    const float4* a0 = reinterpret_cast<const float4*>(Ra + 2 * p * N) + u;
    const float4* a1 = reinterpret_cast<const float4*>(Ra + (2 * p + 1) * N) + u;
    const float4* b0 = reinterpret_cast<const float4*>(Rb + (2 * p + 1) * N) + u;
    const float4* b1 = reinterpret_cast<const float4*>(Rb + 2 * p * N) + u;
    const bool off = u > p;
    float2 cur = off ? acc : dg;
    cur = pair_dot(a0, b0, 1, cur);
    cur = pair_dot(a1, b1, 1, cur);
    acc = off ? cur : acc;
    dg = off ? dg : cur;
    tri_advance(p, u, L, s);
  }
  acc.x = fmaf(2.f, acc.x, dg.x);
  acc.y = fmaf(2.f, acc.y, dg.y);
  return acc;
}

// tr(X Ra X Ra): within the block grid, B(p, u) further splits into two equal
// halves (the pair swap maps row 2p's terms onto row 2p+1's), so
// T = 2 (sum_p D(p, p) + 2 sum_{p < u} D(p, u)) with D(p, u) the row-2p half
// alone: a quarter of the products of the plain sum.
__device__ __forceinline__ float2 tr2sq_full(const float2* __restrict__ Ra, int N, int l, int L) {
  const int s = N >> 1, E = s * (s + 1) / 2;
  float2 acc = make_float2(0.f, 0.f), dg = make_float2(0.f, 0.f);
  int p = 0, u = l;
  tri_advance(p, u, 0, s);
  for (int e = l; e < E; e += L) {
    const float4* a0 = reinterpret_cast<const float4*>(Ra + 2 * p * N) + u;
    const float4* b0 = reinterpret_cast<const float4*>(Ra + (2 * p + 1) * N) + u;
    const bool off = u > p;
    float2 cur = off ? acc : dg;
    cur = pair_dot(a0, b0, 1, cur);
    acc = off ? cur : acc;
    dg = off ? dg : cur;
    tri_advance(p, u, L, s);
  }
  acc.x = 2.f * fmaf(2.f, acc.x, dg.x);
  acc.y = 2.f * fmaf(2.f, acc.y, dg.y);
  return acc;
}

template <typename T>
// Launch bounds: the double instance names its largest block (12 warps), which
// lets it keep up to 170 registers a thread; the float instance is held to 128
// (it runs faster with a small spill than with 150 registers and no spill).
__global__ void __launch_bounds__(sizeof(T) == 8 ? kMaxWarpsPerBlock * 32 : 512, 1)
    haf_subsets_kernel(const HafLaunch P) {
  typedef C2<T> C;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Tables tab;
  if (threadIdx.x == 0) {
    for (int a = 0; a <= kMaxH; ++a)
      for (int b = 0; b <= kMaxH; ++b)
        tab.binom[a][b] = (b == 0) ? 1 : (a == 0 ? 0 : tab.binom[a - 1][b - 1] + tab.binom[a - 1][b]);
    for (int k = 0; k <= kMaxH; ++k) {
      tab.inv2k[k] = (k == 0) ? 0.0 : 1.0 / (2.0 * k);
    }
  }
  __syncthreads();

  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int cb = (int)sizeof(C);
  const int n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;
  unsigned char* wbase = smem + (size_t)warp * P.warp_bytes;
  int* xs = reinterpret_cast<int*>(wbase);
  // staging: the power traces of up to `slots` finished subsets, their signs and orders
  C* stP = reinterpret_cast<C*>(wbase + kWarpHeaderBytes);
  const int sts = stage_stride(P.stage_h);  // entries between two subsets' slots
  const int slots = stage_slots(P.stage_h);  // subsets staged at most
  int* stF = reinterpret_cast<int*>(stP + slots * sts);
  unsigned char* gbase = wbase + kWarpHeaderBytes + stage_bytes(P.stage_h, cb);
  const double2* src2 = reinterpret_cast<const double2*>(P.src);

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(P.counter, 1);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    const WorkItem w = P.items[it];
    if (P.skip != nullptr && P.skip[w.pat] != 0) {
      // the repeated-row sum computes this matrix: leave a zero partial
      if (lane == 0) {
        Partial pr;
        pr.re_hi = pr.re_lo = pr.im_hi = pr.im_lo = pr.kappa = 0.0;
        pr.pad[0] = pr.pad[1] = pr.pad[2] = 0.0;
        P.parts[w.part] = pr;
      }
      __syncwarp();
      continue;
    }
    const PatDesc d = P.pats[w.pat];
    const int n = d.n, h = n >> 1;
    // sizes s_first..s_last: one size (a rank range of it), or every subset of
    // every size of the matrix (s_last > s), staged and reduced together
    const int s_first = w.s, s_last = (w.s_last > w.s) ? w.s_last : w.s;
    const bool whole = s_last > s_first;
    {
      // the item must name sizes and ranks that exist for this matrix: a
      // malformed one flags the matrix (status, NaN partial) and is skipped
      bool ok = s_first >= 1 && s_last <= h && h <= kMaxH && w.count >= 1 && w.rank0 >= 0;
      if (ok && !whole) {
        const int64_t last = (int64_t)w.rank0 + (int64_t)(w.count - 1) * (w.stride > 1 ? w.stride : 1);
        ok = last < (int64_t)tab.binom[h][s_first];
      }
      if (!ok) {
        if (lane == 0) {
          if (P.status) P.status[w.pat] = 1;
          Partial pr;
          pr.re_hi = pr.im_hi = __longlong_as_double(0x7ff8000000000000ll);
          pr.re_lo = pr.im_lo = pr.kappa = 0.0;
          pr.pad[0] = pr.pad[1] = pr.pad[2] = 0.0;
          P.parts[w.part] = pr;
        }
        __syncwarp();
        continue;
      }
    }

    if (lane < n) {
      int pos = default_pos(lane, h);
      if (P.perm != nullptr) {
        const int po = P.perm_off[w.pat];
        if (po >= 0) pos = P.perm[po + lane];
      }
      int v = (d.idx_off >= 0) ? P.idx[d.idx_off + pos] : pos;
      if (P.m_bound > 0 && (v < 0 || v >= P.m_bound)) {
        P.status[w.pat] = 1;
        v = 0;
      }
      xs[lane] = v;
    }
    __syncwarp();

    const double2* ptp = nullptr;
    if (sizeof(T) == 8 && P.pt != nullptr) {
      const int64_t po = P.pt_off[w.pat];
      if (po >= 0) ptp = reinterpret_cast<const double2*>(P.pt) + po;
    }
    int staged = 0;  // subsets whose traces wait in the staging area
    int lanes_used = 1;  // the most subsets one flush of this item held (lanes with terms)
    const double2* srcp = src2 + d.src_off;
    const float2* src32p = P.src32 ? reinterpret_cast<const float2*>(P.src32) + d.src_off : nullptr;

    // the signed sum of the subset terms in double-double (both paths)
    Comp<double> acc_re = {0.0, 0.0}, acc_im = {0.0, 0.0};
    double kap = 0.0;

    // the exponential series e_k = (1/(2k)) sum_j tr_j e_{k-j}, f = e_h, in
    // FP64 for both paths (one staged subset per lane), and the signed
    // compensated accumulation
    // (pq: this lane's subset's traces in FP64)
    auto series = [&](double2* pq, double2* dk) {
        const int sv = stF[lane];
        const int Nl = sv < 0 ? -sv : sv;  // traces taken directly (the subset's order N when < h)
        // the loops run exact trip counts (not unrolled to the largest
        // order): terms past h or N would be issued predicated off and still
        // hold the FP64 pipe, whose warp instructions occupy it for many
        // cycles on this part
        if (Nl > 0 && Nl < h) {
          // an order-N subset has traces 1..N only: det(I - xM) = sum_i d_i x^i
          // has degree N, so by Newton's identities d_k = -(1/k) sum_{i<=k}
          // d_{k-i} p_i (d_0 = 1) and, for k > N, p_k = -sum_{i<=N} d_i p_{k-i}
#pragma unroll 1
          for (int k = 1; k <= Nl; ++k) {
            double2 a = pq[k - 1];
#pragma unroll 1
            for (int i = 1; i < k; ++i) a = cfma<double>(dk[i], pq[k - i - 1], a);
            const double c = -2.0 * tab.inv2k[k];
            dk[k] = mk<double>(a.x * c, a.y * c);
          }
#pragma unroll 1
          for (int k = Nl + 1; k <= h; ++k) {
            double2 a = mk<double>(0.0, 0.0);
#pragma unroll 1
            for (int i = 1; i <= Nl; ++i) a = cfma<double>(dk[i], pq[k - i - 1], a);
            pq[k - 1] = mk<double>(-a.x, -a.y);
          }
        }
        // e_k = (1/(2k)) (p_k e_0 + sum_{j<k} p_j e_{k-j}), e_0 = 1; f = e_h
        double2* e = dk;  // the d_k are no longer needed
        double2 f = mk<double>(1.0, 0.0);
#pragma unroll 1
        for (int k = 1; k <= h; ++k) {
          double2 a = pq[k - 1];
#pragma unroll 1
          for (int j = 1; j < k; ++j) a = cfma<double>(pq[j - 1], e[k - j], a);
          const double c = tab.inv2k[k];
          f = mk<double>(a.x * c, a.y * c);
          if (k < h) e[k] = f;
        }
        const int sg = sv;
        if (sg != 0) {
          comp_add<double>(acc_re, sg > 0 ? f.x : -f.x);
          comp_add<double>(acc_im, sg > 0 ? f.y : -f.y);
          kap += fabs(f.x) + fabs(f.y);
        }
    };
    // The FP32 path converts its staged traces into the lane groups' region
    // when no copy is in flight there (region_free) and the region holds
    // every slot in double, else into a per-lane array.
    const int region = P.warp_bytes - kWarpHeaderBytes - stage_bytes(P.stage_h, cb);
    const bool conv_fits = (sizeof(T) == 4) && region >= slots * sts * 16;
    const bool conv2_fits = (sizeof(T) == 4) && region >= 2 * slots * sts * 16;
    auto flush = [&](bool region_free) {
      if (lane < staged) {
        double2 dk[kMaxH];  // d_1..d_N, then e_1..e_{h-1}
        if constexpr (sizeof(T) == 8) {
          series(stP + lane * sts, dk);
        } else {
          const C* ps = stP + lane * sts;
          if (region_free && conv_fits) {
            double2* q = reinterpret_cast<double2*>(gbase) + lane * sts;
#pragma unroll 1
            for (int k = 0; k < h; ++k) q[k] = make_double2((double)ps[k].x, (double)ps[k].y);
            if (conv2_fits)  // the coefficients beside them
              series(q, reinterpret_cast<double2*>(gbase) + (slots + lane) * sts);
            else
              series(q, dk);
          } else {
            double2 pconv[kMaxH];
#pragma unroll 1
            for (int k = 0; k < h; ++k) pconv[k] = make_double2((double)ps[k].x, (double)ps[k].y);
            series(pconv, dk);
          }
        }
      }
      lanes_used = max(lanes_used, staged);
      staged = 0;
      __syncwarp();
    };

   for (int s = s_first; s <= s_last; ++s) {
    const int N = 2 * s;
    const int NP = (sizeof(T) == 8) ? N * (N + 1) / 2 : N * N;  // entries per matrix
    // traces taken directly: FP64 1..min(N, h) (those past N follow from
    // Newton's identities in the series step, which saves products on the
    // FP64 pipe); FP32 1..h (extra FP32 products are cheaper than the FP64
    // extension)
    const int hs = sched_row(N, h, cb);
    const int L = lanes_for(N, h, P.warp_bytes, P.stage_h, cb);
    const int G = 32 / L;
    const int g = lane / L, l = lane - g * L;
    // FP32 path on the float copy of B, where the spare tile fits: the next
    // round's A_S is copied into it (cp.async) while this round's products
    // run, and the two tiles take turns as R_1
    const bool pf = (sizeof(T) == 4) && src32p != nullptr && spare_tile(N, h, P.warp_bytes, P.stage_h, cb);
    C* buf = reinterpret_cast<C*>(gbase + (size_t)g * group_bytes(N, h, cb, pf));
    const int nb = sched_nbuf(hs);  // matrices of the schedule row
    int* rowidx = reinterpret_cast<int*>(buf + (nb + (pf ? 1 : 0)) * NP);
    int* pairs = rowidx + N;  // FP64: the subset's pair numbers, increasing
    const int count = whole ? tab.binom[h][s] : w.count;
    const int rank0 = whole ? 0 : w.rank0;
    const int stride = (!whole && w.stride > 1) ? w.stride : 1;
    const int rounds = (count + G - 1) / G;

    // Group g takes the subsets numbered g * rounds .. g * rounds + rounds - 1
    // of the item (those below count), one per round. A subset's pair mask
    // comes from its colex rank, rank = sum_i C(c_i, i) over its pairs
    // c_1 < ... < c_s (every lane of the group walks it); with stride 1 the
    // next round's mask is the next larger one with s bits (consecutive colex
    // ranks), which costs a few integer operations instead of the walk.
    auto mask_of = [&](int js) -> unsigned {
      unsigned msk = 0;
      int r = rank0 + (js < count ? js : 0) * stride;
      int c = h - 1;
      for (int i = s; i >= 1; --i) {
        while (tab.binom[c][i] > r) --c;
        r -= tab.binom[c][i];
        msk |= 1u << c;
        --c;
      }
      return msk;
    };
    unsigned gmask = 0;  // the mask of the group's latest subset
    // mask of round rdx's subset (rounds in order) and its rows: position t
    // of the subset is its t-th pair in increasing order
    auto unrank = [&](int rdx) -> unsigned {
      const int js = g * rounds + rdx;
      if (rdx == 0 || stride != 1) {
        gmask = mask_of(js);
      } else if (js < count) {
        const unsigned u = gmask & (0u - gmask), v = gmask + u;
        gmask = v + (((v ^ gmask) >> 2) >> (__ffs(u) - 1));
      }  // (past count the group idles on its last subset)
      unsigned m = gmask;
      for (int t = 0; t < s; ++t) {
        const int c = __ffs(m) - 1;
        m &= m - 1;
        if ((t & (L - 1)) == l) {
          rowidx[2 * t] = xs[2 * c];
          rowidx[2 * t + 1] = xs[2 * c + 1];
          if (sizeof(T) == 8) pairs[t] = c;
        }
      }
      return gmask;
    };

    for (int rd = 0; rd < rounds; ++rd) {
      if (staged + G > slots) flush(!(pf && rd > 0));  // only when the group count changed between sizes
      const bool active = g * rounds + rd < count;
      const int cur = (pf && (rd & 1)) ? nb : 0;  // the tile holding this round's R_1
      unsigned smask = 0;
      if (pf && rd > 0) {
        cp_async_wait_all();  // this round's A_S, copied during the last round
        __syncwarp();
      } else {
        smask = unrank(rd);
        __syncwarp();
        // -- R_1 = A_S (packed upper triangle). Its diagonal is set to zero: no
        //    perfect matching uses V(i, i), and a zero diagonal lowers the
        //    cancellation of the signed sum (collision entries B(x_i, x_i) with
        //    i != j are off the diagonal of B_x and are kept).
        if (sizeof(T) == 8) {
          int i = 0, j = l;
          tri_advance(i, j, 0, N);
          for (int e = l; e < NP; e += L) {
            const double2 v = (i == j) ? make_double2(0.0, 0.0)
                                       : __ldg(srcp + (int64_t)rowidx[i] * d.ld + rowidx[j]);
            buf[e] = mk<T>((T)v.x, (T)v.y);
            tri_advance(i, j, L, N);
          }
        } else if (src32p) {
          for (int e = l; e < NP; e += L) {
            const int i = e / N, j = e - i * N;
            const float2 v = (i == j) ? make_float2(0.f, 0.f)
                                      : __ldg(src32p + (int64_t)rowidx[i] * d.ld + rowidx[j]);
            buf[e] = mk<T>((T)v.x, (T)v.y);
          }
        } else {
          for (int e = l; e < NP; e += L) {
            const int i = e / N, j = e - i * N;
            const double2 v = (i == j) ? make_double2(0.0, 0.0)
                                       : __ldg(srcp + (int64_t)rowidx[i] * d.ld + rowidx[j]);
            buf[e] = mk<T>((T)v.x, (T)v.y);
          }
        }
        __syncwarp();
      }
      if (pf && rd + 1 < rounds) {
        // the next round's rows (this round's A_S is in place), then its A_S
        // into the other tile, in flight during the products below
        unrank(rd + 1);
        __syncwarp();
        C* nxt = buf + (cur == 0 ? nb : 0) * NP;
        for (int e = l; e < NP; e += L) {
          const int i = e / N, j = e - i * N;
          cp_async8(nxt + e, src32p + (int64_t)rowidx[i] * d.ld + rowidx[j], i == j);
        }
        cp_async_commit();
      }
      // schedule matrix b lives in tile b, except R_1's (b = 0): tile cur
      auto bp = [&](int b) -> C* { return buf + (b == 0 ? cur : b) * NP; };
      // -- power traces tr((X A_S)^k), k = 1..hs, by the schedule for hs; the
      //    lanes' partial traces are summed over the group two traces at a
      //    time (one waits in registers for the next)
      C pend_v = mk<T>(T(0), T(0));
      int pend_k = 0;  // 0: none waiting
      C* const strow = stP + (staged + g) * sts;
      for (int o = 0; o < kMaxOps; ++o) {
        const SchedOp op = c_sched[hs][o];
        if (op.kind == kEnd) break;
        if (op.kind == kProd) {
          if constexpr (sizeof(T) == 8) {
            if (ptp != nullptr && op.k == 1 && op.a == 0 && op.b == 0) {
              const int hl = pair_split_lo(h);
              pair_sum(bp(1), ptp, pairs, N, NP, pair_sums_width(h), n, (int)(smask & ((1u << hl) - 1)),
                       (1 << hl) + (int)(smask >> hl), l, L);
            }
            else
              sym_prod<T>(bp(op.k), bp(op.a), bp(op.b), N, NP, l, L);
          } else
            sym_prod_full(bp(op.k), bp(op.a), bp(op.b), N, l, L);
        } else {
          C part;
          if constexpr (sizeof(T) == 8)
            part = (op.kind == kTr1)  ? tr1_part<T>(bp(op.a), N, l, L)
                   : (op.a == op.b) ? tr2sq_part<T>(bp(op.a), N, l, L)
                                    : tr2_part<T>(bp(op.a), bp(op.b), N, NP, l, L);
          else
            part = (op.kind == kTr1)  ? tr1_full(bp(op.a), N, l, L)
                   : (op.a == op.b) ? tr2sq_full(bp(op.a), N, l, L)
                                    : tr2_full(bp(op.a), bp(op.b), N, l, L);
          if (L == 1) {
            strow[op.k - 1] = part;
          } else if (pend_k == 0) {
            pend_v = part;
            pend_k = op.k;
          } else {
            const C t = group_sum2<T>(pend_v, part, l, L);
            if (l == 0) strow[pend_k - 1] = t;
            if (l == (L >> 1)) strow[op.k - 1] = t;
            pend_k = 0;
          }
        }
        __syncwarp();
      }
      if (pend_k != 0) {  // uniform over the warp
        const C t = group_sum<T>(pend_v, L);
        if (l == 0) strow[pend_k - 1] = t;
      }
      // sign (-1)^{h-s} times the number of traces taken directly (< h: the
      // series step extends them; 0: no subset in this slot)
      if (l == 0) stF[staged + g] = active ? (((h - s) & 1) ? -hs : hs) : 0;
      staged += G;
      __syncwarp();
      // -- once the staging slots are full, or the item ends
      if (staged == slots || (rd == rounds - 1 && s == s_last)) flush(!(pf && rd + 1 < rounds));
    }
   }

    // warp reduction of the group accumulators (fixed butterfly: deterministic)
    // in double-double, over the levels that reach the lanes holding terms
    // (lanes past lanes_used hold exact zeros all item long; an item of one
    // round of few large subsets then skips most of the FP64 additions)
    double rh = acc_re.hi, rl = acc_re.lo, ih = acc_im.hi, il = acc_im.lo, kp = kap;
    int span = 1;
    while (span < lanes_used) span <<= 1;
    for (int off = span >> 1; off > 0; off >>= 1) {
      const double orh = __shfl_xor_sync(FULL, rh, off), orl = __shfl_xor_sync(FULL, rl, off);
      const double oih = __shfl_xor_sync(FULL, ih, off), oil = __shfl_xor_sync(FULL, il, off);
      kp += __shfl_xor_sync(FULL, kp, off);
      dd_add(rh, rl, orh, orl);
      dd_add(ih, il, oih, oil);
    }
    if (lane == 0) {
      Partial pr;
      pr.re_hi = rh;
      pr.re_lo = rl;
      pr.im_hi = ih;
      pr.im_lo = il;
      pr.kappa = kp;
      pr.pad[0] = pr.pad[1] = pr.pad[2] = 0.0;
      P.parts[w.part] = pr;
    }
    __syncwarp();
  }
}

// Warp sum of parts[begin, end): lane j adds j, j+32, ... in that order (four
// loads issued ahead of their additions), the lanes meet in a fixed
// butterfly; lane 0 ends with the total (deterministic for a given range).
__device__ __forceinline__ void sum_partials(const Partial* __restrict__ parts, int begin, int end,
                                             int lane, double& rh, double& rl, double& ih, double& il,
                                             double& K) {
  const unsigned FULL = 0xffffffffu;
  const int count = end - begin;
  if (count <= 32) {
    // one partial per lane and only the butterfly levels that reach them: lane
    // 0 gets the same sum as the full butterfly, whose other levels would add
    // exact zeros (a single partial is taken as it is)
    if (lane < count) {
      const Partial pr = parts[begin + lane];
      rh = pr.re_hi;
      rl = pr.re_lo;
      ih = pr.im_hi;
      il = pr.im_lo;
      K = pr.kappa;
    }
    int span = 1;
    while (span < count) span <<= 1;
    for (int off = span >> 1; off > 0; off >>= 1) {
      const double orh = __shfl_xor_sync(FULL, rh, off), orl = __shfl_xor_sync(FULL, rl, off);
      const double oih = __shfl_xor_sync(FULL, ih, off), oil = __shfl_xor_sync(FULL, il, off);
      K += __shfl_xor_sync(FULL, K, off);
      dd_add(rh, rl, orh, orl);
      dd_add(ih, il, oih, oil);
    }
    return;
  }
  int q = begin + lane;
  for (; q + 96 < end; q += 128) {
    Partial pr[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) pr[u] = parts[q + 32 * u];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      dd_add(rh, rl, pr[u].re_hi, pr[u].re_lo);
      dd_add(ih, il, pr[u].im_hi, pr[u].im_lo);
      K += pr[u].kappa;
    }
  }
  for (; q < end; q += 32) {
    const Partial pr = parts[q];
    dd_add(rh, rl, pr.re_hi, pr.re_lo);
    dd_add(ih, il, pr.im_hi, pr.im_lo);
    K += pr.kappa;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double orh = __shfl_xor_sync(FULL, rh, off), orl = __shfl_xor_sync(FULL, rl, off);
    const double oih = __shfl_xor_sync(FULL, ih, off), oil = __shfl_xor_sync(FULL, il, off);
    K += __shfl_xor_sync(FULL, K, off);
    dd_add(rh, rl, orh, orl);
    dd_add(ih, il, oih, oil);
  }
}

// First stage of the two-stage finalisation (matrices with many items): one
// warp per chunk of up to kChunkItems consecutive item partials of a matrix.
// A lone warp's FP64 additions are slow on this part, so the long per-matrix
// sums are spread over many warps; the chunking is fixed by the item counts,
// which keeps the result deterministic.
__global__ void chunk_sum_kernel(const ChunkLaunch C) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int g = blockIdx.x * wpb + (threadIdx.x >> 5); g < C.n_chunks; g += gridDim.x * wpb) {
    const int b = C.chunk_pat[g];
    const PatDesc d = C.pats[b];
    const int begin = d.item_begin + (g - C.chunk_off[b]) * kChunkItems;
    const int end = min(begin + kChunkItems, d.item_end);
    double rh = 0, rl = 0, ih = 0, il = 0, K = 0;
    sum_partials(C.parts, begin, end, lane, rh, rl, ih, il, K);
    if (lane == 0) {
      Partial pr;
      pr.re_hi = rh;
      pr.re_lo = rl;
      pr.im_hi = ih;
      pr.im_lo = il;
      pr.kappa = K;
      pr.pad[0] = pr.pad[1] = pr.pad[2] = 0.0;
      C.out[g] = pr;
    }
  }
}

// One warp per pattern adds its item partials (or, after chunk_sum_kernel,
// the chunk sums) and forms prod_j s_j! (each lane counts the earlier
// occurrences of its index among the other lanes' indices; the c-th
// occurrence of a mode contributes a factor c). The sums go to shared memory and warp 0 finishes the block's
// patterns one per lane (hypot, log, exp): that scalar tail costs one warp
// instruction per block instead of one per pattern.
constexpr int kFinWarps = 16;  // most warps in a finalisation block
__global__ void __launch_bounds__(kFinWarps * 32) finalize_kernel(const FinalizeLaunch F) {
  __shared__ double sv[6][kFinWarps];  // re hi/lo, im hi/lo, sum |f|, prod s_j!
  __shared__ int sbad[kFinWarps];     // status flag of the pattern
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const bool want_p = F.p_out || F.logp_out || F.err_out;
  const int batch = F.batch_dev ? *F.batch_dev : F.batch;
  // pattern of warp w in round `base`: base + w * gridDim.x + blockIdx.x, so
  // that consecutive patterns (alike in their partial counts, which the batch
  // order groups) fall into different blocks and SMs: the FP64 additions of
  // patterns with many partials then spread over the device
  const int nb = gridDim.x;
  for (int base = 0; base < batch; base += nb * wpb) {
    const int b = base + warp * nb + blockIdx.x;
    if (b < batch) {  // uniform over the warp
      const int pb = F.sel ? F.sel[b] : b;
      const PatDesc d = F.pats[pb];
      const int n = d.n;
      // loads that do not depend on the partial sums go first
      const int xi = (want_p && d.idx_off >= 0 && lane < n) ? F.idx[d.idx_off + lane] : -1 - lane;
      const int bad = (lane == 0 && F.status != nullptr) ? F.status[pb] : 0;
      double rh = 0, rl = 0, ih = 0, il = 0, K = 0;
      if (!(n & 1) && n > 0) {
        const int rep = F.rep_half ? F.rep_half[pb] : 0;
        if (rep > 0) {
          const int end = F.rep_end[pb];
          sum_partials(F.rep_parts, end - (rep + kRepTermsPerItem - 1) / kRepTermsPerItem, end, lane, rh, rl,
                       ih, il, K);
        } else if (F.chunk_parts)
          sum_partials(F.chunk_parts, F.chunk_off[pb], F.chunk_off[pb + 1], lane, rh, rl, ih, il, K);
        else
          sum_partials(F.parts, d.item_begin, d.item_end, lane, rh, rl, ih, il, K);
      } else if (n == 0) {
        rh = 1.0;  // the empty matrix has one (empty) perfect matching
        K = 1.0;
      }
      // odd n: no perfect matching, Haf = 0 (Sec. 3.1: P_n = 0 for odd n)
      double fac = 1.0;
      if (want_p && d.idx_off >= 0) {  // uniform over the warp
        // one load per lane; the earlier occurrences come by shuffles
        int c = 1;
#pragma unroll
        for (int q = 0; q < 31; ++q) {
          const int v = __shfl_sync(FULL, xi, q);
          c += (q < lane && v == xi) ? 1 : 0;
        }
        if (lane < n) fac = (double)c;
      }
      for (int off = 16; off > 0; off >>= 1) fac *= __shfl_xor_sync(FULL, fac, off);
      if (lane == 0) {
        sv[0][warp] = rh;
        sv[1][warp] = rl;
        sv[2][warp] = ih;
        sv[3][warp] = il;
        sv[4][warp] = K;
        sv[5][warp] = fac;
        sbad[warp] = bad;
      }
    }
    __syncthreads();
    if (warp == 0 && lane < wpb && base + lane * nb + blockIdx.x < batch) {
      const int bo = base + lane * nb + blockIdx.x;
      const int pb = F.sel ? F.sel[bo] : bo;
      const int n = F.pats[pb].n;
      const bool bad = sbad[lane] != 0;
      const double hr = sv[0][lane] + sv[1][lane], hi = sv[2][lane] + sv[3][lane];
      const double K = sv[4][lane];
      // |Haf| by a plain square root unless the squares could leave the
      // normal range (hypot's scaling costs FP64 instructions on this part)
      const double ar = fabs(hr), ai = fabs(hi);
      const double big = fmax(ar, ai);
      const double mod = (big < 0x1p500 && big > 0x1p-500) ? sqrt(hr * hr + hi * hi) : hypot(hr, hi);
      const double kappa = (mod > 0.0) ? K / mod : (K > 0.0 ? INFINITY : 0.0);
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      if (F.haf_out) {
        F.haf_out[2 * bo] = bad ? nan : hr;
        F.haf_out[2 * bo + 1] = bad ? nan : hi;
      }
      if (F.kappa_out) F.kappa_out[bo] = bad ? nan : kappa;
      if (want_p) {
        // p = q exp(-L), q = |Haf|^2 / prod_j s_j!, and log p = log q - L,
        // with the normaliser exp(-L) precomputed; where q or exp(-L) leaves
        // the normal range, p = exp(log p) with log p = 2 log|Haf| -
        // log prod s_j! - L
        const double L = F.log_norm ? F.log_norm[0] : 0.0;
        const double eL = F.log_norm ? F.log_norm[1] : 1.0;
        const double q = (mod / sv[5][lane]) * mod;
        const bool qn = q >= 0x1p-1022 && q <= 0x1p1023;
        const bool direct = qn && eL >= 0x1p-1022;
        double logp = -INFINITY;
        if (mod > 0.0 && (F.logp_out || !direct))
          logp = qn ? log(q) - L : 2.0 * log(mod) - log(sv[5][lane]) - L;
        if (F.p_out) F.p_out[bo] = bad ? nan : ((mod > 0.0) ? (direct ? q * eL : exp(logp)) : 0.0);
        if (F.logp_out) F.logp_out[bo] = bad ? nan : logp;
        if (F.err_out) F.err_out[bo] = bad ? nan : err_estimate(F.precision, n, kappa);
      }
    }
    __syncthreads();
  }
}

// Pair sums, one block per chunk of kPairChunk packed entries of a matrix (a
// lone matrix spreads over several SMs). The block stages the zero-diagonal
// matrix in shared memory, then the pair terms Q_p(e) = A(i, 2p) A(2p+1, j) +
// A(i, 2p+1) A(2p, j) of its entries e = (i, j), and from those each entry's W
// subset sums (low pairs by mask, then high pairs by mask), each added in
// increasing pair order and written with the slots innermost (coalesced).
constexpr int kPairChunk = 32;
__global__ void __launch_bounds__(256) pair_terms_kernel(const HafLaunch P) {
  __shared__ double2 A[kMaxN * kMaxN];
  __shared__ double2 Q[kPairChunk * kMaxH];  // entries x pairs, pairs innermost
  __shared__ int rows[kMaxN];
  __shared__ int tri[kMaxN + 1];
  const double2* src2 = reinterpret_cast<const double2*>(P.src);
  double2* pt2 = reinterpret_cast<double2*>(P.pt);
  // a serving step with no new request reads its count here (0: nothing to do)
  if (P.n_items_dev != nullptr && *P.n_items_dev == 0) return;
  const int nmax = 2 * P.stage_h;
  const int cpm = (nmax * (nmax + 1) / 2 + kPairChunk - 1) / kPairChunk;  // chunks per matrix
  const int64_t n_chunks = (int64_t)P.batch * cpm;
  for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const int b = (int)(c / cpm), e0 = (int)(c - (int64_t)b * cpm) * kPairChunk;
    const int64_t po = P.pt_off[b];
    const PatDesc d = P.pats[b];
    const int n = d.n, h = n >> 1, NPn = n * (n + 1) / 2;
    // uniform over the block; a matrix beyond the launch's order, or one that
    // the repeated-row sum computes, is not read
    if (po < 0 || pair_terms_elems(n) == 0 || n > nmax || e0 >= NPn) continue;
    if (P.skip != nullptr && P.skip[b] != 0) continue;
    const int ne = min(kPairChunk, NPn - e0);
    if (threadIdx.x < n) {
      int pos = default_pos(threadIdx.x, h);
      if (P.perm != nullptr && P.perm_off[b] >= 0) pos = P.perm[P.perm_off[b] + threadIdx.x];
      int v = (d.idx_off >= 0) ? P.idx[d.idx_off + pos] : pos;
      if (P.m_bound > 0 && (v < 0 || v >= P.m_bound)) v = 0;  // flagged by the subset kernel
      rows[threadIdx.x] = v;
    }
    if (threadIdx.x <= n) tri[threadIdx.x] = threadIdx.x * n - ((threadIdx.x * (threadIdx.x - 1)) >> 1);
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      A[e] = (i == j) ? make_double2(0.0, 0.0) : __ldg(src2 + d.src_off + (int64_t)rows[i] * d.ld + rows[j]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ne * h; t += blockDim.x) {
      const int el = t / h, p = t - el * h, e = e0 + el;
      int i = 0;
      while (tri[i + 1] <= e) ++i;
      const int j = i + (e - tri[i]);
      double2 q = make_double2(0.0, 0.0);
      q = cfma<double>(A[i * n + 2 * p], A[(2 * p + 1) * n + j], q);
      q = cfma<double>(A[i * n + 2 * p + 1], A[2 * p * n + j], q);
      Q[t] = q;
    }
    __syncthreads();
    const int hl = pair_split_lo(h), W = pair_sums_width(h);
    double2* out = pt2 + po + (int64_t)e0 * W;
    for (int t = threadIdx.x; t < ne * W; t += blockDim.x) {
      const int el = t / W, k = t - el * W;
      const bool lo = k < (1 << hl);
      unsigned m = lo ? (unsigned)k : (unsigned)(k - (1 << hl));
      const double2* qe = Q + el * h + (lo ? 0 : hl);
      double2 acc = make_double2(0.0, 0.0);
      if (m) {
        acc = qe[__ffs(m) - 1];
        m &= m - 1;
        while (m) {
          const double2 v = qe[__ffs(m) - 1];
          acc.x += v.x;
          acc.y += v.y;
          m &= m - 1;
        }
      }
      out[t] = acc;
    }
    __syncthreads();
  }
}

// C(a, b) for a, b <= kMaxH (the probe's weights C(h, s) / K)
__constant__ int c_binom[kMaxH + 1][kMaxH + 1] = {
    {1},
    {1, 1},
    {1, 2, 1},
    {1, 3, 3, 1},
    {1, 4, 6, 4, 1},
    {1, 5, 10, 10, 5, 1},
    {1, 6, 15, 20, 15, 6, 1},
    {1, 7, 21, 35, 35, 21, 7, 1},
    {1, 8, 28, 56, 70, 56, 28, 8, 1},
    {1, 9, 36, 84, 126, 126, 84, 36, 9, 1},
    {1, 10, 45, 120, 210, 252, 210, 120, 45, 10, 1},
    {1, 11, 55, 165, 330, 462, 462, 330, 165, 55, 11, 1},
    {1, 12, 66, 220, 495, 792, 924, 792, 495, 220, 66, 12, 1},
    {1, 13, 78, 286, 715, 1287, 1716, 1716, 1287, 715, 286, 78, 13, 1},
    {1, 14, 91, 364, 1001, 2002, 3003, 3432, 3003, 2002, 1001, 364, 91, 14, 1},
    {1, 15, 105, 455, 1365, 3003, 5005, 6435, 6435, 5005, 3003, 1365, 455, 105, 15, 1},
    {1, 16, 120, 560, 1820, 4368, 8008, 11440, 12870, 11440, 8008, 4368, 1820, 560, 120, 16, 1}};

// 1/K for the probe's sample counts K = 1..kMaxProbeSample - 1
__constant__ double c_recip[kMaxProbeSample] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,
    1.0 / 8,    1.0 / 9,    1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15,
    1.0 / 16,   1.0 / 17,   1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23,
    1.0 / 24,   1.0 / 25,   1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31};

// One warp per probed matrix, lane c < n_cand for candidate ordering c: the
// candidate's sum of |f| over the whole subset sum is estimated from its
// sampled items (the K sampled subsets of size s stand for all C(h, s), so
// each item's kappa counts C(h, s) / K times), and the candidate with the
// smallest estimate (the lowest c on a tie) becomes the matrix's ordering.
__global__ void pairing_select_kernel(const PairingSelect S) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= S.n_sel) return;  // uniform over the warp
  double est = INFINITY;
  if (lane < S.n_cand) {
    const int q = k * S.n_cand + lane;
    const PatDesc d = S.probe_pats[q];
    est = 0.0;
    const int h = min(max(d.n >> 1, 0), kMaxH);
#pragma unroll 4
    for (int it = d.item_begin; it < d.item_end; ++it) {
      const WorkItem w = S.probe_items[it];
      const double kp = S.probe_parts[it].kappa;
      const int sz = min(max(w.s, 0), h);
      const int K = min(max(w.aux, 1), kMaxProbeSample - 1);
      est = fma((double)c_binom[h][sz] * c_recip[K], kp, est);
    }
    if (!(est == est)) est = INFINITY;  // a NaN estimate never wins
  }
  int c = lane;
  for (int off = 16; off > 0; off >>= 1) {
    const double oe = __shfl_xor_sync(FULL, est, off);
    const int oc = __shfl_xor_sync(FULL, c, off);
    if (oe < est || (oe == est && oc < c)) {
      est = oe;
      c = oc;
    }
  }
  if (lane == 0) S.main_perm_off[S.sel_pat[k]] = S.probe_perm_off[k * S.n_cand + (c < S.n_cand ? c : 0)];
}

// ---- repeated-row route (Kan's moment identity; see RepLaunch) ----------

struct RepWarp {
  double2 B[kRepMaxDistinct * kRepMaxDistinct];  // B_v, row stride kRepMaxDistinct
  double x[kRepMaxDistinct][32];                  // x_j of each lane's current term (column = lane)
  int c[kRepMaxDistinct];                         // multiplicities c_j
  int mode[kRepMaxDistinct];                      // distinct modes v_j
};

// Warp sum of compensated accumulators (fixed butterfly, double-double) into
// one item partial.
__device__ __forceinline__ void store_warp_partial(Comp<double> re, Comp<double> im, double kap, int lane,
                                                   Partial* out) {
  const unsigned FULL = 0xffffffffu;
  double rh = re.hi, rl = re.lo, ih = im.hi, il = im.lo;
  for (int off = 16; off > 0; off >>= 1) {
    const double orh = __shfl_xor_sync(FULL, rh, off), orl = __shfl_xor_sync(FULL, rl, off);
    const double oih = __shfl_xor_sync(FULL, ih, off), oil = __shfl_xor_sync(FULL, il, off);
    kap += __shfl_xor_sync(FULL, kap, off);
    dd_add(rh, rl, orh, orl);
    dd_add(ih, il, oih, oil);
  }
  if (lane == 0) {
    Partial pr;
    pr.re_hi = rh;
    pr.re_lo = rl;
    pr.im_hi = ih;
    pr.im_lo = il;
    pr.kappa = kap;
    pr.pad[0] = pr.pad[1] = pr.pad[2] = 0.0;
    *out = pr;
  }
}

// Terms t0 + q, q = lane, lane + 32, ... < count, for D distinct modes: digits
// nu_j of t (mixed radix c_j + 1, j = 0 fastest), x_j = c_j - 2 nu_j (kept in
// the lane's own column of W.x), the weight prod (-1)^nu_j C(c_j, nu_j),
// Q = x^T B_v x / 2 evaluated as sum_j x_j (B_jj x_j / 2 + sum_{k>j} B_jk x_k)
// (x integer, so every product with x is one rounding), Q^h by squaring, and
// the term times 2 / (2^n h!) (1 / (2^n h!) for the middle term
// t = (T - 1) / 2, which is its own mirror).
__device__ __forceinline__ void rep_terms(RepWarp& W, const int (*binom)[kMaxN + 1], int D, int h, int t0,
                                          int count, int T, double scale, int lane, Comp<double>& re,
                                          Comp<double>& im, double& kap) {
  for (int q = lane; q < count; q += 32) {
    const int t = t0 + q;
    int rem = t;
    double w = 1.0;
    for (int j = 0; j < D; ++j) {
      const int cj = W.c[j];
      const int nu = rem % (cj + 1);
      rem /= (cj + 1);
      W.x[j][lane] = (double)(cj - 2 * nu);
      const double bw = (double)binom[cj][nu];
      w *= (nu & 1) ? -bw : bw;
    }
    double qr = 0.0, qi = 0.0;
    for (int j = 0; j < D; ++j) {
      const double xj = W.x[j][lane];
      const double2 bjj = W.B[j * kRepMaxDistinct + j];
      const double hx = 0.5 * xj;
      double sr = bjj.x * hx, si = bjj.y * hx;
      for (int k = j + 1; k < D; ++k) {
        const double2 b = W.B[j * kRepMaxDistinct + k];
        const double xk = W.x[k][lane];
        sr = fma(b.x, xk, sr);
        si = fma(b.y, xk, si);
      }
      qr = fma(xj, sr, qr);
      qi = fma(xj, si, qi);
    }
    double pr = 1.0, pi = 0.0, br = qr, bi = qi;
    for (int e = h; e > 0; e >>= 1) {
      if (e & 1) {
        const double tr = fma(pr, br, -pi * bi);
        pi = fma(pr, bi, pi * br);
        pr = tr;
      }
      if (e > 1) {
        const double tr = fma(br, br, -bi * bi);
        bi = 2.0 * br * bi;
        br = tr;
      }
    }
    const double f = w * ((2 * t + 1 == T) ? scale : 2.0 * scale);
    const double vr = f * pr, vi = f * pi;
    comp_add<double>(re, vr);
    comp_add<double>(im, vi);
    kap += fabs(vr) + fabs(vi);
  }
}

// Persistent warps over repeated-row work items. Per item: the matrix's index
// list (lane i holds x_i), its distinct modes and multiplicities by
// __match_any_sync (order of first occurrence), B_v gathered into the warp's
// shared slot, then the item's terms.
__global__ void __launch_bounds__(128) haf_repeated_kernel(const RepLaunch R) {
  __shared__ RepWarp ws[4];
  __shared__ int binom[kMaxN + 1][kMaxN + 1];
  // the grid covers the reservation; with no item (no bunched pattern) every
  // block leaves before building its table (uniform over the block)
  const int n_items = min(*R.n_items_dev, R.n_items);
  if (n_items <= 0) return;
  if (threadIdx.x <= kMaxN) {  // row a = threadIdx.x: C(a, b) = C(a, b-1) (a-b+1) / b
    const int a = threadIdx.x;
    long long c = 1;
    for (int b = 0; b <= kMaxN; ++b) {
      binom[a][b] = (b <= a) ? (int)c : 0;
      if (b < a) c = c * (a - b) / (b + 1);
    }
  }
  __syncthreads();
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  RepWarp& W = ws[threadIdx.x >> 5];
  const double2* src2 = reinterpret_cast<const double2*>(R.B);
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(R.counter, 1);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    WorkItem w;
    // route choice on the device: the pattern whose partial range holds
    // slot it (the smallest b with rep_end[b] > it), and its chunk
    int lo = 0, hi = R.batch - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (R.rep_end[mid] > it) hi = mid;
      else lo = mid + 1;
    }
    const int half = R.rep_half[lo];
    const int chunks = (half + kRepTermsPerItem - 1) / kRepTermsPerItem;
    const int c = it - (R.rep_end[lo] - chunks);
    w.pat = lo;
    w.s = 0;
    w.rank0 = c * kRepTermsPerItem;
    w.count = min(kRepTermsPerItem, half - w.rank0);
    w.part = it;
    w.stride = 1;
    w.s_last = 0;
    w.aux = 0;
    if (half <= 0 || c < 0 || c >= chunks) {  // never for a consistent plan
      if (lane == 0) R.status[lo] = 1;
      const Comp<double> z = {0.0, 0.0};
      store_warp_partial(z, z, 0.0, lane, R.parts + it);
      __syncwarp();
      continue;
    }
    const PatDesc d = R.pats[w.pat];
    const int n = d.n, h = n >> 1;
    int v = -1 - lane;  // lanes past n: values no index takes
    bool bad = false;
    if (lane < n) {
      v = (d.idx_off >= 0) ? R.idx[d.idx_off + lane] : lane;
      if (R.m_bound > 0 && (v < 0 || v >= R.m_bound)) bad = true;
    }
    const unsigned same = __match_any_sync(FULL, v);
    const bool leader = (lane < n) && ((__ffs(same) - 1) == lane);
    const unsigned leaders = __ballot_sync(FULL, leader);
    const int D = __popc(leaders);
    if (__any_sync(FULL, bad) || D > kRepMaxDistinct) {
      // an out-of-range index (NaN output) or a matrix this route was not
      // planned for: flag it, leave a zero partial, read nothing
      if (lane == 0) R.status[w.pat] = 1;
      const Comp<double> z = {0.0, 0.0};
      store_warp_partial(z, z, 0.0, lane, R.parts + w.part);
      __syncwarp();
      continue;
    }
    if (leader) {
      const int j = __popc(leaders & ((1u << lane) - 1u));
      W.mode[j] = v;
      W.c[j] = __popc(same);
    }
    __syncwarp();
    for (int e = lane; e < D * D; e += 32) {
      const int j = e / D, k = e - j * D;
      W.B[j * kRepMaxDistinct + k] = __ldg(src2 + d.src_off + (int64_t)W.mode[j] * d.ld + W.mode[k]);
    }
    __syncwarp();
    int T = 1;
    for (int j = 0; j < D; ++j) T *= W.c[j] + 1;
    double hf = 1.0;
    for (int i = 2; i <= h; ++i) hf *= (double)i;  // exact: h! < 2^53 for h <= 16
    const double scale = ldexp(1.0 / hf, -n);
    Comp<double> re = {0.0, 0.0}, im = {0.0, 0.0};
    double kap = 0.0;
    rep_terms(W, binom, D, h, w.rank0, w.count, T, scale, lane, re, im, kap);
    store_warp_partial(re, im, kap, lane, R.parts + w.part);
    __syncwarp();
  }
}

// Route choice on the device (see RoutePlan): one warp per pattern decides
// between the subset sum and the repeated-row sum by the cost rule, then the
// last block to finish assigns each repeated-row pattern its partial range in
// pattern order (a block-wide prefix sum over tiles of the batch).
__global__ void __launch_bounds__(256) route_plan_kernel(const RoutePlan R) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + warp; b < R.batch; b += gridDim.x * wpb) {
    const PatDesc d = R.pats[b];
    const int n = d.n;
    int half = 0;
    if (n >= 4 && !(n & 1) && n <= kMaxN) {  // uniform over the warp
      int v = -1 - lane;  // lanes past n: values no index takes
      bool bad = false;
      if (lane < n) {
        v = R.idx[d.idx_off + lane];
        if (R.m_bound > 0 && (v < 0 || v >= R.m_bound)) bad = true;
      }
      const unsigned same = __match_any_sync(FULL, v);
      const bool leader = lane < n && (__ffs(same) - 1) == lane;
      const int D = __popc(__ballot_sync(FULL, leader));
      if (!__any_sync(FULL, bad) && D < n && D <= R.d_max[n]) {
        // T = prod_j (c_j + 1) over the distinct modes; partial products
        // above 2^31 are capped there (exact below, and the rule needs only
        // T <= 2^30)
        double t = leader ? (double)(__popc(same) + 1) : 1.0;
        for (int off = 16; off > 0; off >>= 1) t = fmin(t * __shfl_xor_sync(FULL, t, off), 0x1p31);
        if (t <= 0x1p30) {
          const int T = (int)t;
          const int hh = (T + 1) / 2;
          const double rep_cost = (double)hh * (double)(D * D + 3 * D + 60);
          if (4.0 * rep_cost < R.subset_cost[n]) half = hh;
        }
      }
    }
    if (lane == 0) {
      R.rep_half[b] = half;
      if (half > 0) atomicAdd(R.n_chosen, 1);
    }
  }
  __shared__ int s_last, s_total;
  __shared__ long long s_warp[8], s_base;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(R.blocks_done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (__ldcg(R.n_chosen) == 0) {  // every pattern keeps the subset sum: no ranges to assign
    if (threadIdx.x == 0) *R.rep_total = 0;
    return;
  }
  if (threadIdx.x == 0) {
    s_base = 0;
    s_total = 0;
  }
  __syncthreads();
  for (int b0 = 0; b0 < R.batch; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const int half = (b < R.batch) ? __ldcg(R.rep_half + b) : 0;
    const long long c = (half + kRepTermsPerItem - 1) / kRepTermsPerItem;
    long long x = c;  // inclusive prefix within the warp
    for (int off = 1; off < 32; off <<= 1) {
      const long long y = __shfl_up_sync(FULL, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    long long wbase = s_base;
    for (int q = 0; q < warp; ++q) wbase += s_warp[q];
    const long long incl = wbase + x;
    if (b < R.batch) {
      if (incl <= R.cap) {
        R.rep_end[b] = (int)incl;
        if (c > 0) atomicMax(&s_total, (int)incl);
      } else {  // past the capacity: the subset sum instead
        R.rep_end[b] = R.cap;
        if (half > 0) R.rep_half[b] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_base = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *R.rep_total = s_total;
}

}  // namespace

cudaError_t launch_route_plan(const RoutePlan& R, cudaStream_t st) {
  if (R.batch <= 0) return cudaSuccess;
  int blocks = (R.batch + 7) / 8;
  if (blocks > 1024) blocks = 1024;
  route_plan_kernel<<<blocks, 256, 0, st>>>(R);
  return cudaGetLastError();
}

cudaError_t launch_haf_repeated(const RepLaunch& R, cudaStream_t st) {
  // the item count is on the device; n_items is its upper bound (the grid)
  if (R.n_items <= 0) return cudaSuccess;
  if (R.n_items_dev == nullptr || R.rep_half == nullptr || R.rep_end == nullptr) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (R.n_items + 3) / 4;
  const int cap = (sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  haf_repeated_kernel<<<blocks, 128, 0, st>>>(R);
  return cudaGetLastError();
}

cudaError_t launch_pairing_select(const PairingSelect& S, cudaStream_t st) {
  if (S.n_sel <= 0 || S.n_cand > 32) return S.n_sel <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  pairing_select_kernel<<<(S.n_sel + 3) / 4, 128, 0, st>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_pair_terms(const HafLaunch& L, cudaStream_t st) {
  if (L.pt == nullptr || L.batch <= 0) return cudaSuccess;
  if (2 * L.stage_h > kMaxN) return cudaErrorInvalidValue;
  pair_terms_kernel<<<pair_terms_grid(L), 256, 0, st>>>(L);
  return cudaGetLastError();
}

// Raise the kernel's dynamic shared-memory limit to the device maximum once
// (per device and precision); it is never lowered, so every launch shape, and
// any CUDA graph instantiated with one, stays valid.
static cudaError_t ensure_smem_limit(int precision) {
  static std::atomic<int> done[2][64];  // zero-initialised (static storage)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int p = precision == GBS_FP64 ? 0 : 1;
  if (done[p][dev].load(std::memory_order_acquire)) return cudaSuccess;
  const void* fn = p == 0 ? (const void*)haf_subsets_kernel<double> : (const void*)haf_subsets_kernel<float>;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  done[p][dev].store(1, std::memory_order_release);
  return cudaSuccess;
}

cudaError_t launch_haf_subsets(const HafLaunch& L, int precision, int blocks, int warps_per_block,
                               cudaStream_t st) {
  if (warps_per_block < 1 || warps_per_block > kMaxWarpsPerBlock) return cudaErrorInvalidValue;
  const size_t smem = (size_t)warps_per_block * L.warp_bytes;
  cudaError_t e = ensure_smem_limit(precision);
  if (e != cudaSuccess) return e;
  if (precision == GBS_FP64)
    haf_subsets_kernel<double><<<blocks, warps_per_block * 32, smem, st>>>(L);
  else
    haf_subsets_kernel<float><<<blocks, warps_per_block * 32, smem, st>>>(L);
  return cudaGetLastError();
}

int max_blocks_per_sm(int precision, int warps_per_block, int smem_bytes) {
  int nb = 0;
  if (ensure_smem_limit(precision) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const void* fn = precision == GBS_FP64 ? (const void*)haf_subsets_kernel<double>
                                         : (const void*)haf_subsets_kernel<float>;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, warps_per_block * 32, smem_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

const void* pair_terms_kernel_fn() { return (const void*)pair_terms_kernel; }

int pair_terms_grid(const HafLaunch& L) {
  const int nmax = 2 * L.stage_h;
  const int64_t chunks = (int64_t)L.batch * ((nmax * (nmax + 1) / 2 + kPairChunk - 1) / kPairChunk);
  return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, 16384));
}

const void* haf_kernel_fn(int precision) {
  return precision == GBS_FP64 ? (const void*)haf_subsets_kernel<double>
                               : (const void*)haf_subsets_kernel<float>;
}

const void* finalize_kernel_fn() { return (const void*)finalize_kernel; }

cudaError_t prepare_haf_kernel(int precision, int smem_bytes) {
  (void)smem_bytes;
  return ensure_smem_limit(precision);
}

cudaError_t launch_chunk_sums(const ChunkLaunch& C, cudaStream_t st) {
  if (C.n_chunks <= 0) return cudaSuccess;
  int blocks = (C.n_chunks + 3) / 4;
  if (blocks > 8192) blocks = 8192;
  chunk_sum_kernel<<<blocks, 128, 0, st>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeLaunch& F, cudaStream_t st) {
  if (F.batch <= 0) return cudaSuccess;
  const int threads = kFinWarps * 32;  // one warp per pattern
  int blocks = (F.batch + kFinWarps - 1) / kFinWarps;
  if (blocks > 8192) blocks = 8192;
  finalize_kernel<<<blocks, threads, 0, st>>>(F);
  return cudaGetLastError();
}

}  // namespace gbs
