// Kernel matrix B = U diag(tanh r) U^T and log normaliser L = sum_i log cosh r_i.
//
// Sec. 2.3 defines W = U U^T for identical squeezing and puts tanh^n(r) /
// cosh^m(r) in front of |Haf(W_s)|^2 (Eq. ProOri). With per-mode squeezing the
// same Gaussian-state formula reads |Haf(B_s)|^2 / prod_i cosh r_i with
// B = U diag(tanh r_i) U^T, which reduces to Eq. ProOri when all r_i are equal
// (Haf is homogeneous of degree n/2).
//
// B is complex symmetric, so only tiles on or above the diagonal are computed
// and each is written to both (i, j) and (j, i). The product is summed in
// double-double and rounded once (FP64 bound, about ten times the plain
// product's work); it runs once per interferometer.
#include <math.h>

#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int TB = 16;

// t_i = tanh r_i and L = sum_i log cosh r_i; one block, fixed-order reduction.
__global__ void tanh_lognorm_kernel(const double* __restrict__ r, int m, double* __restrict__ t,
                                    double* __restrict__ log_norm) {
  __shared__ double part[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ri = r[i];
    t[i] = tanh(ri);
    const double a = fabs(ri);
    acc += a + log1p(exp(-2.0 * a)) - 0.69314718055994530942;  // log cosh r
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    log_norm[0] = part[0];
    log_norm[1] = exp(-part[0]);  // the normaliser itself, 1 / prod cosh r_i
  }
}

// Error-free transformations (Knuth's two-sum; the FMA-based exact product).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = fma(a, b, -p);
}

// acc (hi, lo) += (ah + al) * v: the product of a double-double and a double,
// its leading part exact (two_prod) and the rest added to the low word.
__device__ __forceinline__ void dot2_add(double& hi, double& lo, double ah, double al, double v) {
  double p, e, s, f;
  two_prod(ah, v, p, e);
  two_sum(hi, p, s, f);
  hi = s;
  lo += f + fma(al, v, e);
}

// One 16x16 tile of B per block: B[i][j] = sum_k U[i][k] t_k U[j][k], summed in
// double-double (the compensated dot product of Ogita, Rump and Oishi, with
// U[i][k] t_k kept exact as a double-double), then rounded once: every entry
// is within about an ulp of the exact sum of the given U and t, however small
// it is beside its m terms (a plain FP64 sum of m = 144 terms left small entries
// relative errors near 1e-14, which the Hafnian's cancellation amplifies).
__global__ void build_B_kernel(const double2* __restrict__ U, const double* __restrict__ t, int m,
                               double2* __restrict__ B) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;  // upper triangle of tiles; mirrored on store
  __shared__ double4 Ui[TB][TB + 1];  // U[i][k] t_k: re hi, re lo, im hi, im lo
  __shared__ double2 Uj[TB][TB + 1];
  const int ty = threadIdx.y, tx = threadIdx.x;
  const int i = bi * TB + ty, j = bj * TB + tx;
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (int k0 = 0; k0 < m; k0 += TB) {
    const int kk = k0 + tx;
    const int ri = bi * TB + ty, rj = bj * TB + ty;
    double4 a = make_double4(0.0, 0.0, 0.0, 0.0);
    double2 b = make_double2(0.0, 0.0);
    if (ri < m && kk < m) {
      const double2 u = U[(int64_t)ri * m + kk];
      const double tk = t[kk];
      two_prod(u.x, tk, a.x, a.y);
      two_prod(u.y, tk, a.z, a.w);
    }
    if (rj < m && kk < m) b = U[(int64_t)rj * m + kk];
    Ui[ty][tx] = a;
    Uj[ty][tx] = b;
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < TB; ++q) {
      const double4 u = Ui[ty][q];
      const double2 v = Uj[tx][q];
      dot2_add(rh, rl, u.x, u.y, v.x);    // + re(a) re(v)
      dot2_add(rh, rl, -u.z, -u.w, v.y);  // - im(a) im(v)
      dot2_add(ih, il, u.x, u.y, v.y);    // + re(a) im(v)
      dot2_add(ih, il, u.z, u.w, v.x);    // + im(a) re(v)
    }
    __syncthreads();
  }
  // In a diagonal tile only the thread with i <= j stores the pair, so B is
  // exactly symmetric and every entry has one writer.
  if (i < m && j < m && (bi < bj || ty <= tx)) {
    const double2 acc = make_double2(rh + rl, ih + il);
    B[(int64_t)i * m + j] = acc;
    B[(int64_t)j * m + i] = acc;
  }
}

__global__ void to_float_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_to_float(const double* src, float* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  to_float_kernel<<<(int)blocks, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_build_B(const double* U, const double* r, int m, double* B, double* log_norm,
                           double* t_scratch, cudaStream_t st) {
  tanh_lognorm_kernel<<<1, 256, 0, st>>>(r, m, t_scratch, log_norm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (m + TB - 1) / TB;
  dim3 grid(nt, nt), block(TB, TB);
  build_B_kernel<<<grid, block, 0, st>>>(reinterpret_cast<const double2*>(U), t_scratch, m,
                                         reinterpret_cast<double2*>(B));
  return cudaGetLastError();
}

}  // namespace gbs
