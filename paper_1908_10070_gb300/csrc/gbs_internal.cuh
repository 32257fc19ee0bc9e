// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbs.h"

namespace gbs {

// One matrix of a batch: the n x n matrix whose (i, j) entry is
// src[src_off + row(i) * ld + row(j)], row(i) = idx[idx_off + i] (or i when
// idx_off < 0). For probabilities src is B and the rows are the pattern's mode
// list x, which is the gather B_x(i, j) = B(x_i, x_j) of Sec. 3.2.
struct PatDesc {
  int64_t src_off;  // complex-element offset of the source matrix
  int64_t idx_off;  // offset of the index list, or -1 for the identity
  int ld;           // leading dimension of the source
  int n;            // order (photon number)
  int item_begin;   // this matrix's work items are parts[item_begin, item_end)
  int item_end;
};

// `count` colex ranks rank0, rank0 + stride, ... among the C(h, s) subsets
// with s pairs of one matrix (stride 1: a consecutive run; larger strides make
// the systematic samples of the pairing probe); or, when s_last > s, every
// subset of every size s..s_last of the matrix (rank0, count and stride unused).
// The subset kernel checks 1 <= s, s_last <= h and that the last rank is below
// C(h, s) before it uses an item, and flags the matrix otherwise.
struct WorkItem {
  int pat;
  int s;
  int rank0;
  int count;
  int part;    // slot of this item's partial sum
  int stride;
  int s_last;  // 0 (or <= s): a single size
  int aux;     // probe items: the number K of subsets sampled of size s
};

// Partial sum of one work item: sum (-1)^{h-|S|} f(X A_S) as a double-double
// complex number, plus sum |f|_1 for the cancellation ratio.
struct Partial {
  double re_hi, re_lo, im_hi, im_lo, kappa, pad[3];
};

constexpr int kMaxN = GBS_MAX_N;
constexpr int kMaxH = kMaxN / 2;
// Most warps in a block of the subset kernel (one block per SM); the kernel's
// launch bounds allow 65536 / (32 * kMaxWarpsPerBlock) = 170 registers a thread.
constexpr int kMaxWarpsPerBlock = 12;
constexpr int kWarpHeaderBytes = 128;  // per-warp index-list buffer (32 ints)

// Estimated relative error of a Hafnian of order n with cancellation ratio
// kappa = sum_S |f_S|_1 / |Haf|: c u kappa, u the unit roundoff of the
// per-subset arithmetic. FP64: c = n. Mixed path (FP32 traces): c = min(n, 4),
// fitted on the oracle: the largest observed error / (2^-24 kappa) is 1.9 (at
// n = 4) over the n = 16, mixed-n (8..24), n = 28/30 and tiny workloads and
// random matrices n = 2..32, and falls with n (below 0.1 from n = 24).
__host__ __device__ inline double err_estimate(int precision, int n, double kappa) {
  if (precision == GBS_FP64) return (double)(n > 0 ? n : 1) * 0x1p-53 * kappa;
  return (double)(n < 1 ? 1 : (n > 4 ? 4 : n)) * 0x1p-24 * kappa;
}

// Default order of a matrix of order n = 2h in the subset sum: position p reads
// source position p/2 (p even) or p/2 + h (p odd), so pair t joins source
// positions t and t + h. A sorted index list with repeated modes then puts two
// copies of one mode into a pair only when that mode holds more than half of
// the photons; pairing copies (adjacent positions (2t, 2t+1) of a sorted list)
// made the signed sum cancel up to ~1e4 times more in measurements.
__host__ __device__ inline int default_pos(int p, int h) { return (p >> 1) + ((p & 1) ? h : 0); }

// The row of the power-trace schedule (see haf_subsets.cu) that subsets of
// order N of a matrix of order 2h run: FP64 takes traces 1..min(N, h) by
// products (those past N follow from Newton's identities), FP32 all of 1..h.
__host__ __device__ inline int sched_row(int N, int h, int cbytes) { return (cbytes == 16 && N < h) ? N : h; }

// Matrix buffers schedule row hs holds at once (its largest buffer index plus
// one; 3 bits per row, rows 0..16: 1 1 1 2 2 3 3 3 3 4 4 3 3 5 5 4 4).
__host__ __device__ inline int sched_nbuf(int hs) { return (int)((0x496b7236da449ull >> (3 * hs)) & 7u); }

// Shared-memory bytes of one lane group's region for subsets of order N (and
// half photon number h) with complex elements of `cbytes` bytes: the
// matrices its schedule row holds at once (FP64: packed upper triangles of
// N(N+1)/2 entries; FP32: full N x N tiles, whose rows the products read as
// float4 pairs), with `spare` one more tile (FP32: the next subset's A_S is
// copied into it while the current one's products run), N row indices and,
// for FP64, the N/2 pair numbers of the subset.
__host__ __device__ inline int group_bytes(int N, int h, int cbytes, bool spare = false) {
  const int P = (cbytes == 16) ? N * (N + 1) / 2 : N * N;
  const int mats = sched_nbuf(sched_row(N, h, cbytes)) + (spare ? 1 : 0);
  const int bytes = mats * P * cbytes + N * 4 + (cbytes == 16 ? N * 2 : 0);
  return (bytes + 15) & ~15;
}

// Pair sums of a matrix of order n = 2h. With the pair terms
// Q_p(i, j) = A(i, 2p) A(2p+1, j) + A(i, 2p+1) A(2p, j), the pairs split into
// a low part (p < hl, hl = ceil(h/2)) and a high part (p >= hl). For every
// entry (i, j), i <= j, of the packed upper triangle the matrix keeps W values:
// the sum of Q_p over each subset of the low pairs (slot = its bit mask), then
// over each subset of the high pairs (slot 2^hl + mask >> hl). For a subset S
// of pairs, A_S X A_S (i, j) = low[S] + high[S]: one complex addition per
// entry (used for h >= 3).
__host__ __device__ inline int pair_split_lo(int h) { return (h + 1) >> 1; }
__host__ __device__ inline int pair_sums_width(int h) { return (1 << ((h + 1) >> 1)) + (1 << (h >> 1)); }
// Complex elements of one matrix's pair sums (0 where they are not used).
__host__ __device__ inline int64_t pair_terms_elems(int n) {
  const int h = n / 2;
  return (n >= 6 && !(n & 1)) ? (int64_t)(n * (n + 1) / 2) * pair_sums_width(h) : 0;
}

// Per-warp staging of finished subsets' power traces (32 slots of stage_h
// complex values of the path's own type, plus 32 sign flags); the exponential
// series then runs in FP64 with one subset per lane, the FP32 path's traces
// converted there, all 32 lanes at once (a conversion to double runs on the
// FP64 pipe, whose warp instructions cost the same with one active lane).
// Slots are stage_stride(stage_h) entries apart, an odd number, so that the
// lanes reading entry k of their own slots touch different bank groups (at an
// even stride such as 8 entries they all hit the same few banks).
// Matrices of order 2 stage_h >= 2 kStageHalfFrom stage 16 subsets at a time
// instead of 32: their lane groups are large (one or two per warp for the
// orders that dominate) and the shared memory saved holds more warps per SM,
// while the series of their small subsets runs on half the lanes.
constexpr int kStageHalfFrom = 13;
__host__ __device__ inline int stage_slots(int stage_h) { return stage_h >= kStageHalfFrom ? 16 : 32; }
__host__ __device__ inline int stage_stride(int stage_h) { return stage_h | 1; }
__host__ __device__ inline int stage_bytes(int stage_h, int cbytes) {
  const int slots = stage_slots(stage_h);
  return (slots * stage_stride(stage_h) * cbytes + slots * 4 + 15) & ~15;
}

// Lane-group size L (a power of two) for subsets of order N of a matrix of
// order 2h: the smallest L whose 32/L groups fit the warp's bytes left after
// the header and the staging area, and no more groups than staging slots; 0
// if none does.
__host__ __device__ inline int lanes_for(int N, int h, int warp_bytes, int stage_h, int cbytes) {
  const int avail = warp_bytes - kWarpHeaderBytes - stage_bytes(stage_h, cbytes);
  const int gb = group_bytes(N, h, cbytes);
  for (int L = 32 / stage_slots(stage_h); L <= 32; L <<= 1)
    if ((32 / L) * gb <= avail) return L;
  return 0;
}

// FP32 lane groups take the spare tile where the warp's shared memory holds
// it for all 32/L groups at the size lanes_for chose without it (the group
// count, which the host plans with, never changes).
__host__ __device__ inline bool spare_tile(int N, int h, int warp_bytes, int stage_h, int cbytes) {
  if (cbytes != 8) return false;
  const int L = lanes_for(N, h, warp_bytes, stage_h, cbytes);
  if (L == 0) return false;
  const int avail = warp_bytes - kWarpHeaderBytes - stage_bytes(stage_h, cbytes);
  return (32 / L) * group_bytes(N, h, cbytes, true) <= avail;
}

struct HafLaunch {
  const double* src;       // interleaved complex source matrices
  const float* src32;      // the same rounded to float (FP32 path; may be null)
  const int* idx;          // index lists (may be null when every idx_off < 0)
  const PatDesc* pats;
  const WorkItem* items;   // in schedule order (device or mapped host memory)
  int n_items;
  const int* n_items_dev;  // if non-null, the item count is read here (device memory)
  int m_bound;             // index lists must be < m_bound (0 = no check)
  int* counter;            // work-queue head, zero before launch
  int* status;             // per-pattern flag, set to 1 on an out-of-range index
  Partial* parts;
  int warp_bytes;          // dynamic shared memory per warp
  int stage_h;             // power traces staged per subset (>= the batch's largest n/2)
  // May be null: a reordering of each matrix's rows and columns. Position i of
  // matrix b reads source position perm[perm_off[b] + i] (perm_off < 0 or a
  // null perm: default_pos). The Hafnian does not depend on the order; the
  // pairing of positions (2t, 2t+1) that the subset sum uses does, and with it
  // the cancellation of the signed sum.
  const int* perm;
  const int* perm_off;
  // FP64 only, may be null: per-matrix pair sums (layout of pair_terms_elems)
  // at pt + pt_off[pattern]; pt_off < 0 means that matrix forms A_S X A_S by
  // the product instead
  double* pt;
  const int64_t* pt_off;
  int batch;               // matrices in pats (read by the pair-term kernel)
  // May be null: per matrix, nonzero when the route choice on the device sent
  // it to the repeated-row sum; its subset items then leave a zero partial and
  // the pair-term kernel skips it.
  const int* skip;
};

// Two-stage finalisation: chunk g (of matrix chunk_pat[g]) sums up to
// kChunkItems consecutive item partials of that matrix; matrix b's chunks are
// [chunk_off[b], chunk_off[b + 1]).
constexpr int kChunkItems = 128;
struct ChunkLaunch {
  const PatDesc* pats;
  const Partial* parts;
  const int* chunk_pat;
  const int* chunk_off;
  int n_chunks;
  Partial* out;
};

struct FinalizeLaunch {
  const int* sel;          // if non-null, entry b finalises pattern sel[b] (outputs at b)
  // If non-null (route choice on the device): a pattern with rep_half > 0 sums
  // its ceil(rep_half / kRepTermsPerItem) repeated-row partials, which end at
  // rep_parts[rep_end[pattern]], instead of its subset items.
  const int* rep_half;
  const int* rep_end;
  const Partial* rep_parts;
  const int* batch_dev;    // if non-null, the number of entries is read here (device memory)
  const Partial* chunk_parts;  // if non-null, sum these chunk sums (chunk_off ranges) instead
  const int* chunk_off;
  const PatDesc* pats;
  const Partial* parts;
  const int* idx;
  const int* status;
  int batch;
  int precision;
  const double* log_norm;  // device [L = sum_i log cosh r_i, exp(-L)], or null (Hafnians only)
  double* p_out;
  double* logp_out;
  double* haf_out;
  double* err_out;         // relative error estimate (probabilities)
  double* kappa_out;       // kappa (Hafnians)
};

// Choice of each large matrix's ordering from a probe launch: probe matrix
// k * n_cand + c is matrix sel_pat[k] in candidate ordering c, its items
// (part slot = item index) a systematic sample of K subsets of each sampled
// size s; each probe item carries K (< kMaxProbeSample) in aux.
constexpr int kMaxProbeSample = 32;
struct PairingSelect {
  const PatDesc* probe_pats;
  const WorkItem* probe_items;
  const Partial* probe_parts;
  const int* probe_perm_off;  // ordering of each probe matrix (offset into perm)
  const int* sel_pat;
  int n_sel;
  int n_cand;
  int* main_perm_off;         // written: the chosen ordering of each probed matrix
};

// Repeated-row route (index-list matrices with collisions, FP64): with
// distinct modes v_1..v_d of multiplicities c_j (sum c_j = n, h = n/2),
//   Haf(B_x) = (1 / (2^n h!)) sum_{0 <= nu_j <= c_j}
//              prod_j (-1)^nu_j C(c_j, nu_j) (x^T B_v x / 2)^h,  x_j = c_j - 2 nu_j,
// B_v the d x d submatrix of B on the distinct modes (the moment-extraction
// identity of Kan, 2008). Terms are numbered in mixed radix (digit j = nu_j,
// radix c_j + 1); term t and T - 1 - t (nu and c - nu) are equal, so only
// t < ceil(T / 2) is summed, T = prod (c_j + 1). A work item is a run of
// kRepTermsPerItem term numbers of one matrix (the last one shorter).
constexpr int kRepMaxDistinct = 16;
constexpr int kRepTermsPerItem = 1024;
struct RepLaunch {
  const double* B;         // interleaved complex, m x m, row stride ld (the PatDesc's)
  const int* idx;
  const PatDesc* pats;
  int n_items;             // grid coverage (the reservation); *n_items_dev items run
  int m_bound;             // index lists must be < m_bound (0 = no check)
  int* counter;            // work-queue head, zero before launch
  int* status;             // per-pattern flag, set to 1 on an out-of-range index
  Partial* parts;
  // Item v of the *n_items_dev items (written by route_plan_kernel) is term
  // chunk v - (rep_end[b] - chunks_b) of the pattern b whose partial range
  // [rep_end[b] - chunks_b, rep_end[b]) holds v, chunks_b =
  // ceil(rep_half[b] / kRepTermsPerItem); its partial goes to parts[v].
  const int* rep_half = nullptr;
  const int* rep_end = nullptr;
  const int* n_items_dev = nullptr;
  int batch = 0;
};

// Route choice on the device, for FP64 probabilities (index lists from the
// host are copied to the device first, so one rule serves both). One warp per
// pattern finds its distinct modes and multiplicities and applies the cost
// rule: the repeated-row sum when the
// pattern has a repeated mode, at most d_max[n] distinct modes, T <= 2^30 and
// 4 ceil(T / 2) (d^2 + 3d + 60) < subset_cost[n]. The last block to finish
// then assigns partial ranges in pattern order: a pattern keeps the route
// only while the running total of chunks stays within cap (later ones fall
// back to the subset sum), so the choice is the same for the same batch.
struct RoutePlan {
  const int* idx;
  const PatDesc* pats;
  int batch;
  int m_bound;             // index lists must be < m_bound (0 = no check)
  int cap;                 // repeated-row partial slots available
  double subset_cost[kMaxN + 1];
  int d_max[kMaxN + 1];
  int* rep_half;           // out, per pattern: terms summed (ceil(T / 2)), 0 = subset sum
  int* rep_end;            // out, per pattern: end of its partial range (non-decreasing)
  int* rep_total;          // out: partial slots used (the repeated-row item count)
  unsigned* blocks_done;   // zero before launch
  int* n_chosen;           // zero before launch: patterns given the repeated-row sum
};

// Defined in haf_subsets.cu
cudaError_t launch_haf_repeated(const RepLaunch& R, cudaStream_t st);
cudaError_t launch_route_plan(const RoutePlan& R, cudaStream_t st);
cudaError_t launch_haf_subsets(const HafLaunch& L, int precision, int blocks, int warps_per_block,
                               cudaStream_t st);
cudaError_t launch_finalize(const FinalizeLaunch& F, cudaStream_t st);
cudaError_t launch_chunk_sums(const ChunkLaunch& C, cudaStream_t st);
cudaError_t launch_pairing_select(const PairingSelect& S, cudaStream_t st);
// Fill L.pt for every matrix whose pt_off is >= 0 (one block per matrix).
cudaError_t launch_pair_terms(const HafLaunch& L, cudaStream_t st);
int max_blocks_per_sm(int precision, int warps_per_block, int smem_bytes);
// Kernel entry points, for CUDA graph kernel nodes (the serving loop).
const void* haf_kernel_fn(int precision);
// The pair-term kernel (argument: HafLaunch, 256 threads a block) and the grid
// launch_pair_terms gives it; with n_items_dev set it returns at once when
// that count is 0 (serving steps without a new request).
const void* pair_terms_kernel_fn();
int pair_terms_grid(const HafLaunch& L);
const void* finalize_kernel_fn();
cudaError_t prepare_haf_kernel(int precision, int smem_bytes);

// Defined in build_b.cu
cudaError_t launch_build_B(const double* U, const double* r, int m, double* B, double* log_norm,
                           double* t_scratch, cudaStream_t st);
// dst[i] = (float)src[i], i < count
cudaError_t launch_to_float(const double* src, float* dst, int64_t count, cudaStream_t st);

}  // namespace gbs
