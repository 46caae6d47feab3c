// Iterative refinement of a solve (not in the paper): the factorization's solution x of
// C x = y is corrected by x += C^-1 r with the FP64 residual r = y - C~ x, where C~ is the
// HODLR matrix itself (dense leaves recomputed from the points, U V^T off-diagonal blocks;
// levels.cu launch_matvec). This removes the rounding error of the factor (double-float
// leaves in the mixed form) up to the accuracy of the FP64 product.
#include <cuda_runtime.h>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kResBlocks = 256;
constexpr int kResThreads = 256;

// r = y - ax (written over ax); per-block partial sums of r^2 and y^2.
__global__ void __launch_bounds__(kResThreads)
k_residual(const double* __restrict__ y, double* __restrict__ ax, int64_t n,
           double* __restrict__ part) {
  __shared__ double s1[kResThreads], s2[kResThreads];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kResThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kResThreads) {
    double yi = y[i];
    double r = yi - ax[i];
    ax[i] = r;
    a += r * r;
    b += yi * yi;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = kResThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1[0];
    part[kResBlocks + blockIdx.x] = s2[0];
  }
}

// ratio = ||r|| / ||y|| (0 for y = 0), partials summed in block order.
__global__ void k_residual_finish(const double* __restrict__ part, double* ratio) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < kResBlocks; ++i) a += part[i];
  for (int i = 0; i < kResBlocks; ++i) b += part[kResBlocks + i];
  ratio[0] = b > 0.0 ? sqrt(a / b) : 0.0;
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

}  // namespace

// work buffer: C~ x / r (n), partial sums (2 kResBlocks), ratio
int64_t refine_work_elems(int64_t n) { return n + 2 * kResBlocks + 8; }

// ax (n doubles) holds C~ x on entry and r on exit; *ratio = ||r|| / ||y||.
cudaError_t launch_residual(Ctx& c, const double* y_sorted, double* ax, double* part, double* ratio) {
  k_residual<<<kResBlocks, kResThreads, 0, c.stream>>>(y_sorted, ax, c.n, part);
  k_residual_finish<<<1, 32, 0, c.stream>>>(part, ratio);
  c.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_axpy(Ctx& c, double* x, const double* d) {
  k_axpy<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(x, d, c.n);
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
