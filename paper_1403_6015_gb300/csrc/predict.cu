// GP prediction with the HODLR factorization (the conditional distribution behind the
// likelihood of Sec. 1, the standard GP regression formulas): at each test point x*, the
// posterior mean k_*^T C^-1 y and the latent posterior variance k(x*, x*) - k_*^T C^-1 k_*,
// where k_* = (k(x_i, x*))_i. The solves reuse the stored factorization; the
// cross-covariances are evaluated in FP64 from the sorted training points.
#include <cuda_runtime.h>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kPT = 256;       // threads per block
constexpr int kPSlices = 64;   // slices of the training points per test point

__device__ __forceinline__ double cross_r(const Pts& pts, int64_t i, const double* xt, int64_t j) {
  double a = pts.x[i] - xt[j * pts.d];
  if (pts.d == 1) return fabs(a);
  double b = pts.x[pts.n + i] - xt[j * pts.d + 1];
  if (pts.d == 2) return sqrt(a * a + b * b);
  double s = a * a + b * b;
  for (int c = 2; c < pts.d; ++c) {
    double e = pts.x[c * pts.n + i] - xt[j * pts.d + c];
    s += e * e;
  }
  return sqrt(s);
}

// partial[b * kPSlices + s] = sum over the training points of slice s of k(x_i, x*_{j0+b})
// times w_i, w the b-th column of W (wstep = 1) or its first column (wstep = 0); the block's
// threads stride over the slice and are reduced in a fixed order.
__global__ void __launch_bounds__(kPT) k_cross_dot(Pts pts, const double* __restrict__ xt,
                                                   int64_t j0, int kind, const double* hyp,
                                                   const double* __restrict__ W, int64_t ldw,
                                                   int wstep, double* __restrict__ partial) {
  __shared__ double red[kPT];
  const Cov cov = cov_from(kind, hyp);
  int b = blockIdx.x, s = blockIdx.y;
  int64_t j = j0 + b;
  int64_t per = (pts.n + kPSlices - 1) / kPSlices;
  int64_t i0 = s * per, i1 = i0 + per < pts.n ? i0 + per : pts.n;
  const double* w = W + (wstep ? (int64_t)b * ldw : 0);
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kPT) acc += cov_r(cov, cross_r(pts, i, xt, j)) * w[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kPT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)b * kPSlices + s] = red[0];
}

// Y[:, b] = k_* of test point j0 + b, in tree order (n x nc, column stride n).
__global__ void k_cross_fill(Pts pts, const double* __restrict__ xt, int64_t j0, int nc, int kind,
                             const double* hyp, double* __restrict__ Y) {
  const Cov cov = cov_from(kind, hyp);
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pts.n) return;
  for (int b = 0; b < nc; ++b) Y[(int64_t)b * pts.n + i] = cov_r(cov, cross_r(pts, i, xt, j0 + b));
}

// out[j0 + b] = sum_s partial[b * kPSlices + s] (mode 0), or k(0) minus that sum (mode 1).
__global__ void k_cross_finish(const double* __restrict__ partial, int nc, int64_t j0, int kind,
                               const double* hyp, int mode, double* __restrict__ out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nc) return;
  double t = 0.0;
  for (int s = 0; s < kPSlices; ++s) t += partial[(int64_t)b * kPSlices + s];
  out[j0 + b] = mode == 0 ? t : cov_r(cov_from(kind, hyp), 0.0) - t;
}

}  // namespace

int64_t predict_partial_elems(int64_t m) { return m * kPSlices; }

// out[j0 + b], b < nc: k_*(x*_{j0+b})^T w_b (mode 0) or k(0) minus it (mode 1), with w_b the
// b-th column of W (wstep 1) or W's first column for every b (wstep 0).
cudaError_t launch_cross_dot(Ctx& c, const double* xt, int64_t j0, int nc, const double* W,
                             int64_t ldw, int wstep, double* partial, int mode, double* out) {
  dim3 g((unsigned)nc, kPSlices);
  k_cross_dot<<<g, kPT, 0, c.stream>>>(Pts{c.xs, c.n, c.d}, xt, j0, c.kind, c.hyp, W, ldw, wstep, partial);
  k_cross_finish<<<(nc + 127) / 128, 128, 0, c.stream>>>(partial, nc, j0, c.kind, c.hyp, mode, out);
  c.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_cross_fill(Ctx& c, const double* xt, int64_t j0, int nc) {
  k_cross_fill<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(Pts{c.xs, c.n, c.d}, xt, j0, nc,
                                                                    c.kind, c.hyp, c.Y);
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
