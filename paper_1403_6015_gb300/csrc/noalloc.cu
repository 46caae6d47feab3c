// hodlr_loglik_small_noalloc: the Gaussian log-likelihood of a problem that fits one leaf
// block (n <= 128 points), computed without any device allocation.
//
// Who needs it: code that must not call cudaMalloc or cudaFree (or a caching allocator
// such as torch's) on the path that evaluates the likelihood, for example an inner
// sampling loop running under a fixed memory budget, a host thread that shares the device
// with a stream-ordered allocator it must not disturb, or a caller that records the work
// into a CUDA graph and wants no allocation nodes in it. The regular entry points allocate
// their buffers in hodlr_build; this one uses a fixed array in device global memory that
// the library defines once per loaded module.
//
// The scratch: a file-scope __device__ array of kNoAllocBytes (136,384 bytes). Every GPU
// that loads the library holds one copy until the process exits. Host code cannot use the
// array's name as a device address; the first call on a device (with that device current)
// asks the runtime for the address with cudaGetSymbolAddress and keeps it for calls made
// while a stream capture is under way. That first call should therefore come before any
// stream capture. Calls outside a capture look the address up again, so that a device
// reset (which reloads the module and can move the array) never leaves a stale address
// in use; a capture begun after a reset must again follow one uncaptured call.
// Covariances: the four of Table 1 (exponential, squared-exponential, Matern-3/2,
// Matern-5/2) only; the radial kinds return HODLR_EINVAL.
// All calls on a device share the array: calls whose work overlaps on the GPU (different
// streams, no ordering between them) race and give wrong results. Each call first clears
// the words that must start at zero.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace {

constexpr int kNoAllocMaxN = hodlr::kMaxLeaf;  // largest n accepted (one leaf block)

// Scratch layout, in doubles.
constexpr int kOffX = 0;                                       // sorted-free coordinates, d x 128 (SoA)
constexpr int kOffY = kOffX + 3 * kNoAllocMaxN;                // y, kept for y^T C^-1 y
constexpr int kOffSol = kOffY + kNoAllocMaxN;                  // y, overwritten by C^-1 y
constexpr int kOffL = kOffSol + kNoAllocMaxN;                  // Cholesky factor, 128 x 128
constexpr int kOffLd = kOffL + kNoAllocMaxN * kNoAllocMaxN;    // log det
constexpr int kOffInt = kOffLd + 8;                            // int32 words: nodes[2], flags
constexpr int kOffHyp = kOffInt + 8;                           // hyperparameter slot
constexpr int kNoAllocDoubles = kOffHyp + 8;
constexpr size_t kNoAllocBytes = sizeof(double) * kNoAllocDoubles;
static_assert(kNoAllocBytes == 136384, "the documented scratch size");

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device. Looked up on every call made
// outside a stream capture (so that it follows a device reset); under capture the address
// kept from the last uncaptured call on this device is used.
cudaError_t scratch_address(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // treat as capturing: use the kept address
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone || !g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Clear the flag word, write the one-leaf tree, copy x (row-major n x d) to structure of
// arrays and y to both vectors.
__global__ void k_noalloc_prep(double* s, const double* __restrict__ x, const double* __restrict__ y,
                               int n, int d, int kind, double ell, double amp, double sigma2) {
  int32_t* iw = reinterpret_cast<int32_t*>(s + kOffInt);
  if (threadIdx.x == 0) {
    iw[0] = 0;  // node begin
    iw[1] = n;  // node size
    iw[2] = 0;  // flags
    double* hyp = s + kOffHyp;
    hyp[hodlr::kHypInvEll] = 1.0 / ell;
    hyp[hodlr::kHypAmp] = amp;
    hyp[hodlr::kHypSigma2] = sigma2;
    hyp[hodlr::kHypScale] = hodlr::cov_scale(kind, ell);
    hyp[hodlr::kHypAlpha] = 1.0;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int c = 0; c < d; ++c) s[kOffX + c * n + i] = x[i * d + c];
    s[kOffY + i] = y[i];
    s[kOffSol + i] = y[i];
  }
}

// log-likelihood = -y^T C^-1 y / 2 - log det C / 2 - n log(2 pi) / 2 (NaN if C was not
// positive definite), summed in a fixed order.
__global__ void k_noalloc_finish(const double* s, int n, double* out) {
  __shared__ double red[128];
  double q = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) q += s[kOffY + i] * s[kOffSol + i];
  red[threadIdx.x] = q;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int32_t* iw = reinterpret_cast<const int32_t*>(s + kOffInt);
    double ll = -0.5 * red[0] - 0.5 * s[kOffLd] - 0.5 * (double)n * log(2.0 * 3.14159265358979323846);
    out[0] = iw[2] ? nan("") : ll;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" hodlr_status hodlr_loglik_small_noalloc(const double* x, int64_t n, int d,
                                                   hodlr_kernel kernel, const double* theta,
                                                   double sigma2, const double* y, double* out,
                                                   void* stream) {
  if (n < 1 || n > kNoAllocMaxN || d < 1 || d > 3 || (int)kernel < 0 || (int)kernel > 3 ||
      !theta || !(theta[0] > 0) || !(theta[1] > 0) || !std::isfinite(theta[0]) ||
      !std::isfinite(theta[1]) || !(sigma2 >= 0) || !std::isfinite(sigma2) || !x || !y || !out)
    return HODLR_EINVAL;
  if (!on_device(x) || !on_device(y) || !on_device(out)) return HODLR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* s = nullptr;
  if (scratch_address(st, &s) != cudaSuccess) {
    cudaGetLastError();
    return HODLR_ECUDA;
  }
  int32_t* iw = reinterpret_cast<int32_t*>(s + kOffInt);
  k_noalloc_prep<<<1, 128, 0, st>>>(s, x, y, (int)n, d, (int)kernel, theta[0], theta[1], sigma2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = hodlr::launch_leaf_single(s + kOffX, (int)n, d, (int)kernel, s + kOffHyp, iw,
                                  s + kOffSol, s + kOffL, s + kOffLd, iw + 2, st);
  if (e == cudaSuccess) {
    k_noalloc_finish<<<1, 128, 0, st>>>(s, (int)n, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HODLR_ECUDA;
  }
  return HODLR_OK;
}
