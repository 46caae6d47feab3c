// Learned rank predictor: block features and a small multilayer perceptron trained on the
// GPU by hand-written forward, backward and Adam kernels (FP32).
//
// The paper's compression is adaptive (Sec. 3.1: ranks "fluctuate" with the accuracy and
// the block); a rank predicted before compression lets the factorization be sized up front
// (hodlr_presize), so an evaluation runs without host round trips and can be captured as a
// graph, with adaptive ACA as the fallback when a block needs more than its predicted rank.
//
// Features of the off-diagonal block of node id (children L, R; bounding boxes of their
// points): log(diam_L / ell), log(diam_R / ell), log(|c_L - c_R| / ell), log2(m_L + m_R)/20,
// -log10(eps)/12, one-hot covariance (4), d - 1, log(max diam / |c_L - c_R|), 0.
// Network: 12 -> 64 -> 64 -> 1 with tanh hidden units, regressing log(1 + rank).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kF = 12;   // features
constexpr int kH = 64;   // hidden width
constexpr int kNParams = kF * kH + kH + kH * kH + kH + kH + 1;
constexpr int kOffW1 = 0, kOffB1 = kF * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
constexpr int kSampPerBlock = 64;  // samples per block in the gradient reduction

// Bounding boxes of every node (level order): box[id][0..d) = min, [d..2d) = max.
__global__ void k_node_boxes(const double* __restrict__ xs, int64_t n, int d,
                             const int32_t* __restrict__ nb, const int32_t* __restrict__ ns,
                             int nnodes, double* __restrict__ box) {
  int id = blockIdx.x;
  if (id >= nnodes) return;
  int b = nb[id], m = ns[id];
  __shared__ double red[2][256];
  for (int c = 0; c < d; ++c) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double v = xs[c * n + b + i];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    red[0][threadIdx.x] = lo;
    red[1][threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        red[0][threadIdx.x] = fmin(red[0][threadIdx.x], red[0][threadIdx.x + o]);
        red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      box[(int64_t)id * 2 * d + c] = red[0][0];
      box[(int64_t)id * 2 * d + d + c] = red[1][0];
    }
    __syncthreads();
  }
}

__global__ void k_block_features(const double* __restrict__ box, int d,
                                 const int32_t* __restrict__ ns, int nint, int kind,
                                 double inv_ell, double eps, float* __restrict__ X, int64_t ld) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nint) return;
  int L = 2 * id + 1, R = 2 * id + 2;
  double dl = 0, dr = 0, dc = 0;
  for (int c = 0; c < d; ++c) {
    double l0 = box[(int64_t)L * 2 * d + c], l1 = box[(int64_t)L * 2 * d + d + c];
    double r0 = box[(int64_t)R * 2 * d + c], r1 = box[(int64_t)R * 2 * d + d + c];
    dl += (l1 - l0) * (l1 - l0);
    dr += (r1 - r0) * (r1 - r0);
    double cc = 0.5 * (l0 + l1) - 0.5 * (r0 + r1);
    dc += cc * cc;
  }
  dl = sqrt(dl);
  dr = sqrt(dr);
  dc = sqrt(dc);
  float* f = X + (int64_t)id * ld;
  f[0] = (float)log(fmax(dl * inv_ell, 1e-30));
  f[1] = (float)log(fmax(dr * inv_ell, 1e-30));
  f[2] = (float)log(fmax(dc * inv_ell, 1e-30));
  f[3] = (float)(log2((double)(ns[L] + ns[R])) / 20.0);
  f[4] = (float)(-log10(eps) / 12.0);
  for (int k = 0; k < 4; ++k) f[5 + k] = kind == k ? 1.0f : 0.0f;
  f[9] = (float)(d - 1);
  f[10] = (float)log(fmax(fmax(dl, dr) / fmax(dc, 1e-300), 1e-30));
  f[11] = 0.0f;
}

// Forward pass, one thread per sample; weights staged in shared memory. Optionally keeps
// the hidden activations (for the backward pass).
__global__ void k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                              int64_t N, float* __restrict__ Y, float* __restrict__ H1,
                              float* __restrict__ H2) {
  __shared__ float w[kNParams];
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) w[i] = P[i];
  __syncthreads();
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= N) return;
  float x[kF];
#pragma unroll
  for (int i = 0; i < kF; ++i) x[i] = X[s * kF + i];
  float h1[kH];
#pragma unroll 4
  for (int k = 0; k < kH; ++k) {
    float a = w[kOffB1 + k];
#pragma unroll
    for (int i = 0; i < kF; ++i) a += x[i] * w[kOffW1 + i * kH + k];
    h1[k] = tanhf(a);
    if (H1) H1[s * kH + k] = h1[k];
  }
  float y = w[kOffB3];
  for (int o = 0; o < kH; ++o) {
    float a = w[kOffB2 + o];
#pragma unroll 8
    for (int k = 0; k < kH; ++k) a += h1[k] * w[kOffW2 + k * kH + o];
    float h2 = tanhf(a);
    if (H2) H2[s * kH + o] = h2;
    y += h2 * w[kOffW3 + o];
  }
  Y[s] = y;
}

// Backward pass of the mean squared error (1/N) sum (y - t)^2: block b handles samples
// [b S, (b + 1) S) and writes its partial gradient (all parameters) to G + b * kNParams;
// sums are over the block's samples in order (deterministic).
__global__ void k_mlp_backward(const float* __restrict__ P, const float* __restrict__ X,
                               const float* __restrict__ T, const float* __restrict__ Y,
                               const float* __restrict__ H1, const float* __restrict__ H2,
                               int64_t N, float* __restrict__ G) {
  __shared__ float d1[kSampPerBlock][kH + 1];
  __shared__ float d2[kSampPerBlock][kH + 1];
  __shared__ float dy[kSampPerBlock];
  int64_t s0 = (int64_t)blockIdx.x * kSampPerBlock;
  int ns = (int)(N - s0 < kSampPerBlock ? N - s0 : kSampPerBlock);
  float invN = 1.0f / (float)N;
  // per-sample deltas: thread t handles sample t (blockDim >= kSampPerBlock)
  int t = threadIdx.x;
  if (t < ns) {
    int64_t s = s0 + t;
    float g = 2.0f * (Y[s] - T[s]) * invN;
    dy[t] = g;
    for (int o = 0; o < kH; ++o) {
      float h2 = H2[s * kH + o];
      d2[t][o] = g * P[kOffW3 + o] * (1.0f - h2 * h2);
    }
    for (int k = 0; k < kH; ++k) {
      float a = 0.0f;
      for (int o = 0; o < kH; ++o) a += P[kOffW2 + k * kH + o] * d2[t][o];
      float h1 = H1[s * kH + k];
      d1[t][k] = a * (1.0f - h1 * h1);
    }
  }
  __syncthreads();
  float* g = G + (int64_t)blockIdx.x * kNParams;
  for (int e = threadIdx.x; e < kNParams; e += blockDim.x) {
    float acc = 0.0f;
    if (e < kOffB1) {  // W1[i][k]
      int i = e / kH, k = e - i * kH;
      for (int q = 0; q < ns; ++q) acc += X[(s0 + q) * kF + i] * d1[q][k];
    } else if (e < kOffW2) {
      int k = e - kOffB1;
      for (int q = 0; q < ns; ++q) acc += d1[q][k];
    } else if (e < kOffB2) {  // W2[k][o]
      int k = (e - kOffW2) / kH, o = (e - kOffW2) - k * kH;
      for (int q = 0; q < ns; ++q) acc += H1[(s0 + q) * kH + k] * d2[q][o];
    } else if (e < kOffW3) {
      int o = e - kOffB2;
      for (int q = 0; q < ns; ++q) acc += d2[q][o];
    } else if (e < kOffB3) {
      int o = e - kOffW3;
      for (int q = 0; q < ns; ++q) acc += dy[q] * H2[(s0 + q) * kH + o];
    } else {
      for (int q = 0; q < ns; ++q) acc += dy[q];
    }
    g[e] = acc;
  }
}

// Sum the per-block partial gradients in block order.
__global__ void k_sum_grads(const float* __restrict__ G, int nblk, float* __restrict__ grad) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParams) return;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += G[(int64_t)b * kNParams + e];
  grad[e] = s;
}

// Adam (Kingma and Ba, 2015) with bias correction.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParams) return;
  float g = grad[e];
  float mm = b1 * m[e] + (1.0f - b1) * g;
  float vv = b2 * v[e] + (1.0f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  P[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t N,
                      float* __restrict__ out) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    float e = Y[i] - T[i];
    s += e * e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (float)N;
}

}  // namespace

struct Mlp {
  float* P = nullptr;     // parameters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* scratch = nullptr;  // H1, H2, Y, G
  int64_t scratch_n = 0;
  int64_t t = 0;             // Adam step
  cudaStream_t stream = nullptr;
  std::string last_error;
};


}  // namespace hodlr

using hodlr::Mlp;

namespace {

cudaError_t mlp_scratch(Mlp* m, int64_t N) {
  int64_t nblk = (N + hodlr::kSampPerBlock - 1) / hodlr::kSampPerBlock;
  int64_t need = N * (2 * hodlr::kH + 1) + nblk * hodlr::kNParams;
  if (need <= m->scratch_n) return cudaSuccess;
  if (m->scratch) cudaFree(m->scratch);
  m->scratch = nullptr;
  m->scratch_n = 0;
  cudaError_t e = cudaMalloc(&m->scratch, sizeof(float) * need);
  if (e == cudaSuccess) m->scratch_n = need;
  return e;
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int hodlr_mlp_num_params(void) { return hodlr::kNParams; }
int hodlr_mlp_num_features(void) { return hodlr::kF; }

hodlr_status hodlr_mlp_create(uint64_t seed, void* stream, hodlr_mlp** out) {
  if (!out) return HODLR_EINVAL;
  *out = nullptr;
  Mlp* m = new (std::nothrow) Mlp;
  if (!m) return HODLR_ENOMEM;
  m->stream = (cudaStream_t)stream;
  if (cudaMalloc(&m->P, sizeof(float) * hodlr::kNParams) != cudaSuccess ||
      cudaMalloc(&m->grad, sizeof(float) * hodlr::kNParams) != cudaSuccess ||
      cudaMalloc(&m->m, sizeof(float) * hodlr::kNParams) != cudaSuccess ||
      cudaMalloc(&m->v, sizeof(float) * hodlr::kNParams) != cudaSuccess) {
    cudaGetLastError();
    hodlr_mlp_destroy(reinterpret_cast<hodlr_mlp*>(m));
    return HODLR_ENOMEM;
  }
  // Glorot-uniform weights from a splitmix64 stream, zero biases
  std::vector<float> p(hodlr::kNParams, 0.0f);
  uint64_t st = seed;
  auto next = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int fan_in, int fan_out) {
    double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < fan_in * fan_out; ++i) p[off + i] = (float)((2.0 * next() - 1.0) * a);
  };
  fill(hodlr::kOffW1, hodlr::kF, hodlr::kH);
  fill(hodlr::kOffW2, hodlr::kH, hodlr::kH);
  fill(hodlr::kOffW3, hodlr::kH, 1);
  cudaMemcpy(m->P, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice);
  cudaMemset(m->m, 0, sizeof(float) * hodlr::kNParams);
  cudaMemset(m->v, 0, sizeof(float) * hodlr::kNParams);
  *out = reinterpret_cast<hodlr_mlp*>(m);
  return HODLR_OK;
}

void hodlr_mlp_destroy(hodlr_mlp* mp) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m) return;
  cudaFree(m->P);
  cudaFree(m->grad);
  cudaFree(m->m);
  cudaFree(m->v);
  if (m->scratch) cudaFree(m->scratch);
  delete m;
}

hodlr_status hodlr_mlp_params(hodlr_mlp* mp, float* params, int set) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || !params) return HODLR_EINVAL;
  cudaMemcpyKind k = dev_ptr(params) ? cudaMemcpyDeviceToDevice
                                     : (set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  cudaError_t e = set ? cudaMemcpyAsync(m->P, params, sizeof(float) * hodlr::kNParams, k, m->stream)
                      : cudaMemcpyAsync(params, m->P, sizeof(float) * hodlr::kNParams, k, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (set && e == cudaSuccess) {
    m->t = 0;
    cudaMemsetAsync(m->m, 0, sizeof(float) * hodlr::kNParams, m->stream);
    cudaMemsetAsync(m->v, 0, sizeof(float) * hodlr::kNParams, m->stream);
  }
  return e == cudaSuccess ? HODLR_OK : HODLR_ECUDA;
}

hodlr_status hodlr_mlp_forward(hodlr_mlp* mp, const float* X, int64_t N, float* Y) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || N < 1 || !dev_ptr(X) || !dev_ptr(Y)) return HODLR_EINVAL;
  hodlr::k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, m->stream>>>(m->P, X, N, Y, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? HODLR_OK : HODLR_ECUDA;
}

hodlr_status hodlr_mlp_gradient(hodlr_mlp* mp, const float* X, const float* T, int64_t N,
                                float* grad, float* loss) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || N < 1 || !dev_ptr(X) || !dev_ptr(T)) return HODLR_EINVAL;
  if (mlp_scratch(m, N) != cudaSuccess) {
    cudaGetLastError();
    return HODLR_ENOMEM;
  }
  float* H1 = m->scratch;
  float* H2 = H1 + N * hodlr::kH;
  float* Y = H2 + N * hodlr::kH;
  float* G = Y + N;
  int nblk = (int)((N + hodlr::kSampPerBlock - 1) / hodlr::kSampPerBlock);
  hodlr::k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, m->stream>>>(m->P, X, N, Y, H1, H2);
  hodlr::k_mlp_backward<<<nblk, 128, 0, m->stream>>>(m->P, X, T, Y, H1, H2, N, G);
  hodlr::k_sum_grads<<<(hodlr::kNParams + 255) / 256, 256, 0, m->stream>>>(G, nblk, m->grad);
  if (cudaGetLastError() != cudaSuccess) return HODLR_ECUDA;
  if (loss) {
    // the loss into the first slot of G (free after the gradient sum), then out
    hodlr::k_mse<<<1, 256, 0, m->stream>>>(Y, T, N, G);
    cudaError_t e = dev_ptr(loss) ? cudaMemcpyAsync(loss, G, sizeof(float), cudaMemcpyDeviceToDevice, m->stream)
                                  : cudaMemcpyAsync(loss, G, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return HODLR_ECUDA;
  }
  if (grad) {
    cudaError_t e = dev_ptr(grad) ? cudaMemcpyAsync(grad, m->grad, sizeof(float) * hodlr::kNParams, cudaMemcpyDeviceToDevice, m->stream)
                                  : cudaMemcpyAsync(grad, m->grad, sizeof(float) * hodlr::kNParams, cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return HODLR_ECUDA;
  }
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return HODLR_ECUDA;
  return HODLR_OK;
}

hodlr_status hodlr_mlp_train(hodlr_mlp* mp, const float* X, const float* T, int64_t N,
                             int steps, float lr, float* loss) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || N < 1 || steps < 0 || !dev_ptr(X) || !dev_ptr(T)) return HODLR_EINVAL;
  if (mlp_scratch(m, N) != cudaSuccess) {
    cudaGetLastError();
    return HODLR_ENOMEM;
  }
  float* H1 = m->scratch;
  float* H2 = H1 + N * hodlr::kH;
  float* Y = H2 + N * hodlr::kH;
  float* G = Y + N;
  int nblk = (int)((N + hodlr::kSampPerBlock - 1) / hodlr::kSampPerBlock);
  const float b1 = 0.9f, b2 = 0.999f;
  for (int s = 0; s < steps; ++s) {
    ++m->t;
    float c1 = 1.0f - std::pow(b1, (float)m->t), c2 = 1.0f - std::pow(b2, (float)m->t);
    hodlr::k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, m->stream>>>(m->P, X, N, Y, H1, H2);
    hodlr::k_mlp_backward<<<nblk, 128, 0, m->stream>>>(m->P, X, T, Y, H1, H2, N, G);
    hodlr::k_sum_grads<<<(hodlr::kNParams + 255) / 256, 256, 0, m->stream>>>(G, nblk, m->grad);
    hodlr::k_adam<<<(hodlr::kNParams + 255) / 256, 256, 0, m->stream>>>(m->P, m->grad, m->m, m->v, lr, b1, b2, 1e-8f, c1, c2);
  }
  if (cudaGetLastError() != cudaSuccess) return HODLR_ECUDA;
  if (loss) {
    hodlr::k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, m->stream>>>(m->P, X, N, Y, nullptr, nullptr);
    hodlr::k_mse<<<1, 256, 0, m->stream>>>(Y, T, N, G);
    cudaMemcpyAsync(loss, G, sizeof(float), dev_ptr(loss) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream);
  }
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? HODLR_OK : HODLR_ECUDA;
}

// Checkpoint: "HODLRMLP" magic, uint32 version, uint32 parameter count, FP32 parameters.
hodlr_status hodlr_mlp_save(hodlr_mlp* mp, const char* path) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || !path) return HODLR_EINVAL;
  std::vector<float> p(hodlr::kNParams);
  if (hodlr_mlp_params(mp, p.data(), 0) != HODLR_OK) return HODLR_ECUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) return HODLR_EINVAL;
  uint32_t hdr[2] = {1u, (uint32_t)hodlr::kNParams};
  bool ok = std::fwrite("HODLRMLP", 1, 8, f) == 8 && std::fwrite(hdr, 4, 2, f) == 2 &&
            std::fwrite(p.data(), 4, p.size(), f) == p.size();
  std::fclose(f);
  return ok ? HODLR_OK : HODLR_EINVAL;
}

hodlr_status hodlr_mlp_load(hodlr_mlp* mp, const char* path) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  if (!m || !path) return HODLR_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return HODLR_EINVAL;
  char magic[8];
  uint32_t hdr[2];
  std::vector<float> p(hodlr::kNParams);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "HODLRMLP", 8) == 0 &&
            std::fread(hdr, 4, 2, f) == 2 && hdr[0] == 1u && hdr[1] == (uint32_t)hodlr::kNParams &&
            std::fread(p.data(), 4, p.size(), f) == p.size();
  std::fclose(f);
  if (!ok) return HODLR_EINVAL;
  return hodlr_mlp_params(mp, p.data(), 1);
}

}  // extern "C"

namespace hodlr {

cudaError_t launch_block_features(Ctx& c, double ell, float* X, int64_t ld) {
  int K = c.kappa;
  int nint = (1 << K) - 1;
  if (nint == 0) return cudaSuccess;
  int nnodes = (2 << K) - 1;
  if (!c.boxes) {
    HODLR_CUDA_TRY(cudaMalloc(&c.boxes, sizeof(double) * 2 * c.d * (size_t)nnodes));
    k_node_boxes<<<nnodes, 256, 0, c.stream>>>(c.xs, c.n, c.d, c.nodes,
                                               c.nodes + ((int64_t)2 << K), nnodes, c.boxes);
    ++c.launches;
  }
  k_block_features<<<(nint + 127) / 128, 128, 0, c.stream>>>(c.boxes, c.d,
                                                             c.nodes + ((int64_t)2 << K), nint,
                                                             c.kind, 1.0 / ell, c.eps, X, ld);
  ++c.launches;
  return cudaGetLastError();
}


cudaError_t launch_mlp_forward(Ctx& c, hodlr_mlp* mp, const float* X, int64_t N, float* Y) {
  Mlp* m = reinterpret_cast<Mlp*>(mp);
  k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, c.stream>>>(m->P, X, N, Y, nullptr, nullptr);
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
