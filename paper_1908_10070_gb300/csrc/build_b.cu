// Kernel matrix B = U diag(tanh r) U^T and log normaliser L = sum_i log cosh r_i.
//
// Sec. 2.3 defines W = U U^T for identical squeezing and puts tanh^n(r) /
// cosh^m(r) in front of |Haf(W_s)|^2 (Eq. ProOri). With per-mode squeezing the
// same Gaussian-state formula reads |Haf(B_s)|^2 / prod_i cosh r_i with
// B = U diag(tanh r_i) U^T, which reduces to Eq. ProOri when all r_i are equal
// (Haf is homogeneous of degree n/2).
//
// B is complex symmetric, so only tiles on or above the diagonal are computed
// and each is written to both (i, j) and (j, i). The product is FP64 (DFMA
// bound); it runs once per interferometer.
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
  if (threadIdx.x == 0) *log_norm = part[0];
}

// One 16x16 tile of B per block: B[i][j] = sum_k U[i][k] t_k U[j][k].
__global__ void build_B_kernel(const double2* __restrict__ U, const double* __restrict__ t, int m,
                               double2* __restrict__ B) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;  // upper triangle of tiles; mirrored on store
  __shared__ double2 Ui[TB][TB + 1];
  __shared__ double2 Uj[TB][TB + 1];
  const int ty = threadIdx.y, tx = threadIdx.x;
  const int i = bi * TB + ty, j = bj * TB + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < m; k0 += TB) {
    const int kk = k0 + tx;
    const int ri = bi * TB + ty, rj = bj * TB + ty;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    if (ri < m && kk < m) {
      a = U[(int64_t)ri * m + kk];
      const double tk = t[kk];
      a.x *= tk;
      a.y *= tk;
    }
    if (rj < m && kk < m) b = U[(int64_t)rj * m + kk];
    Ui[ty][tx] = a;
    Uj[ty][tx] = b;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TB; ++q) {
      const double2 u = Ui[ty][q], v = Uj[tx][q];
      acc.x = fma(u.x, v.x, acc.x);
      acc.x = fma(-u.y, v.y, acc.x);
      acc.y = fma(u.x, v.y, acc.y);
      acc.y = fma(u.y, v.x, acc.y);
    }
    __syncthreads();
  }
  // In a diagonal tile only the thread with i <= j stores the pair, so B is
  // exactly symmetric and every entry has one writer.
  if (i < m && j < m && (bi < bj || ty <= tx)) {
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
