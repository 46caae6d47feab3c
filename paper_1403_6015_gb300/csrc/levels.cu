// Level-by-level factorization and solve (Sec. 3.2): for j = kappa-1 down to 0, every node
// of level j forms M = [I, V^T Vt; U^T Ut, I] (I + W L in the Sherman-Morrison-Woodbury
// formula with L = blockdiag(Ut, Vt), W = [0 V^T; U^T 0]), LU-factors it (log det by
// Sylvester's theorem, Sec. 4), and applies (I + L W)^-1 = I - L M^-1 W to every coarser
// ancestor's U/V rows and to the right-hand sides on its rows:
//   Z = M^-1 [V^T P_R; U^T P_L],  P_L -= Ut Z_top,  P_R -= Vt Z_bot.
//
// Work is expressed over leaf row tiles so all levels have the same parallelism:
//   per-leaf partials  Phi_j[leaf]^T Q[leaf]       (written by the previous sweep step)
//   k_segsum           fixed-order sums over each node half
//   k_node             M, LU, log det, Z per node (M in shared memory, ranks <= 64; larger
//                      ranks: the blocked node step of levels_big.cu)
//   k_sweep            update of level u on each leaf fused with the partials of level u-1
#include <cuda_runtime.h>

#include <cmath>

#include "hodlr_internal.cuh"
#include "ff.cuh"
#include "node_solve.cuh"

namespace hodlr {
namespace {

constexpr int kSweepThreads = 256;
constexpr int kSegChunk = 64;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out[g * stride + e] = sum_{t < h} in[(g h + t) * stride + e], e < E, fixed order.
__global__ void k_segsum(const double* __restrict__ in, int64_t stride, int E, int h,
                         double* __restrict__ out) {
  int g = blockIdx.x;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const double* p = in + (int64_t)g * h * stride + e;
    double s = 0.0;
    for (int t = 0; t < h; ++t) s += p[(int64_t)t * stride];
    out[(int64_t)g * stride + e] = s;
  }
}

cudaError_t segsum(const double* in, int64_t stride, int E, int64_t nleaf, int h, double* tmp,
                   double* out, cudaStream_t s, int64_t* launches) {
  int64_t groups = nleaf / h;
  if (E == 0) return cudaSuccess;
  int thr = E < 128 ? 64 : 128;
  *launches += h <= kSegChunk ? 1 : 2;
  if (h <= kSegChunk) {
    k_segsum<<<(unsigned)groups, thr, 0, s>>>(in, stride, E, h, out);
  } else {
    k_segsum<<<(unsigned)(nleaf / kSegChunk), thr, 0, s>>>(in, stride, E, kSegChunk, tmp);
    k_segsum<<<(unsigned)groups, thr, 0, s>>>(tmp, stride, E, h / kSegChunk, out);
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(128) k_node(NodeArgs a, bool factor) {
  extern __shared__ double M[];  // m2 x m2 row-major
  __shared__ int piv[2 * kSmemRank];
  __shared__ double lds;
  __shared__ int sgn;
  node_solve(a, blockIdx.x, factor, M, piv, &lds, &sgn);
}

// Node step of every node of level na.j: M in shared memory up to rank kSmemRank (one CTA
// per node), else in global memory, factored and solved blocked over many CTAs.
cudaError_t launch_node(Ctx& c, const NodeArgs& na, bool factor_mode) {
  int r = na.r;
  if (r > kSmemRank) return launch_node_blocked(c, na, factor_mode);
  size_t smem = sizeof(double) * 4 * r * r;
  if (smem > kSmemOptIn)
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_node, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_node<<<1u << na.j, 128, smem, c.stream>>>(na, factor_mode);
  ++c.launches;
  return cudaGetLastError();
}

struct SweepArgs {
  const int32_t* nb;
  const int32_t* ns;
  int leaf0, kappa, u;
  double* pan;
  const double* phi;
  double* Y;
  int cP;        // panel columns updated (c_u in factor mode, 0 in solve mode)
  int nrhs;
  int cu, ru;    // level u: own columns in pan (Ut/Vt), rank
  int cl, rl;    // level u-1: columns in phi, rank (rl = 0: no partial)
  const double* Z;
  int64_t z_stride;
  double* part;
  int64_t part_stride;
  int64_t n;
};

// Level-u update of one leaf's rows, fused with the level-(u-1) partial products.
// kStage: the leaf's rows of Ut/Vt (level u) and Phi (level u-1) are staged in shared
// memory (p x (ru + rl) elements); otherwise (large ranks) they are read from the panels.
// T = ff (mixed form): the panels and Z's panel columns are double-float pairs and their
// arithmetic runs in double-float on the FP32 pipe; the right-hand-side columns (and Z's
// right-hand-side columns) stay FP64, reading the panels through conversions.
template <class T> struct Elem;
template <> struct Elem<double> {
  static __device__ __forceinline__ double to_double(double v) { return v; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double from_rhs(double v) { return v; }
  static __device__ __forceinline__ double to_rhs(double v) { return v; }
  static __device__ __forceinline__ double fms(double c, double a, double b) { return c - a * b; }
  static __device__ __forceinline__ double fma(double c, double a, double b) { return c + a * b; }
  static __device__ __forceinline__ double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
};
template <> struct Elem<ff> {
  static __device__ __forceinline__ double to_double(ff v) { return ff_to_double(v); }
  static __device__ __forceinline__ ff zero() { return ff{0.0f, 0.0f}; }
  static __device__ __forceinline__ ff from_rhs(double v) { return ff_from_double(v); }
  static __device__ __forceinline__ double to_rhs(ff v) { return ff_to_double(v); }
  static __device__ __forceinline__ ff fms(ff c, ff a, ff b) { return ff_fms(c, a, b); }
  static __device__ __forceinline__ ff fma(ff c, ff a, ff b) { return ff_fma(c, a, b); }
  static __device__ __forceinline__ ff wsum(ff v) {
    for (int o = 16; o > 0; o >>= 1)
      v = ff_add(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
  }
};

template <bool kStage, class T>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(SweepArgs a) {
  using E = Elem<T>;
  extern __shared__ double smd[];
  T* sm = reinterpret_cast<T*>(smd);
  T* pan = reinterpret_cast<T*>(a.pan);
  const T* phi = reinterpret_cast<const T*>(a.phi);
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // element (i, c): staged at [i * r + c], in the panels at column c, row b + i
  const T* tl = kStage ? sm : pan + (int64_t)a.cu * a.n + b;
  const T* ph = kStage ? sm + kMaxLeaf * a.ru : phi + (int64_t)a.cl * a.n + b;
  const int64_t tl_i = kStage ? a.ru : 1, tl_c = kStage ? 1 : a.n;
  const int64_t ph_i = kStage ? a.rl : 1, ph_c = kStage ? 1 : a.n;
  if (kStage) {
    for (int e = tid; e < p * a.ru; e += kSweepThreads) {
      int i = e % p, c = e / p;
      sm[i * a.ru + c] = pan[(int64_t)(a.cu + c) * a.n + b + i];
    }
    for (int e = tid; e < p * a.rl; e += kSweepThreads) {
      int i = e % p, c = e / p;
      sm[kMaxLeaf * a.ru + i * a.rl + c] = phi[(int64_t)(a.cl + c) * a.n + b + i];
    }
    __syncthreads();
  }
  int sh = a.kappa - a.u;
  int side = (leaf >> (sh - 1)) & 1;
  int wz = a.cP + a.nrhs;
  const T* Zs = reinterpret_cast<const T*>(a.Z) + (int64_t)(leaf >> sh) * a.z_stride + (int64_t)side * a.ru * wz;
  double* out = a.part + (int64_t)leaf * a.part_stride;
  for (int q = w; q < wz; q += kSweepThreads / 32) {
    if (q < a.cP) {
      T* colp = pan + (int64_t)q * a.n + b;
      T x[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        x[m] = i < p ? colp[i] : E::zero();
      }
      for (int c = 0; c < a.ru; ++c) {
        T z = Zs[c * wz + q];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          if (i < p) x[m] = E::fms(x[m], tl[i * tl_i + c * tl_c], z);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) colp[i] = x[m];
      }
      for (int c = 0; c < a.rl; ++c) {
        T s = E::zero();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          if (i < p) s = E::fma(s, ph[i * ph_i + c * ph_c], x[m]);
        }
        s = E::wsum(s);
        if (lane == 0) out[c * wz + q] = E::to_rhs(s);
      }
    } else {
      // a right-hand side: FP64 throughout
      double* coly = a.Y + (int64_t)(q - a.cP) * a.n + b;
      const double* Zd = reinterpret_cast<const double*>(Zs);
      double x[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        x[m] = i < p ? coly[i] : 0.0;
      }
      for (int c = 0; c < a.ru; ++c) {
        double z = Zd[c * wz + q];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          if (i < p) x[m] -= E::to_double(tl[i * tl_i + c * tl_c]) * z;
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) coly[i] = x[m];
      }
      for (int c = 0; c < a.rl; ++c) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          if (i < p) s += E::to_double(ph[i * ph_i + c * ph_c]) * x[m];
        }
        s = Elem<double>::wsum(s);
        if (lane == 0) out[c * wz + q] = s;
      }
    }
  }
}

// Deterministic sum of a (fixed-size grid of per-block partials, then one block).
__global__ void k_sum_blocks(const double* __restrict__ v, const double* __restrict__ v2,
                             int64_t m, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    s += v2 ? v[i] * v2[i] : v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

constexpr int kRedBlocks = 256;

// One warp: lane l sums the partials l, l + 32, ... in index order, then a fixed xor
// butterfly combines the 32 lane sums (each pair added the same way on both lanes), so the
// result is the same on every lane and on every run.
__global__ void k_finish(const double* __restrict__ pl, const double* __restrict__ pn,
                         const double* __restrict__ pq, double* scal, int64_t n, int mode) {
  // mode 0: logdet only; mode 1: logdet and quadratic form -> log-likelihood
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  int l = threadIdx.x;
  double a = 0.0, b = 0.0, q = 0.0;
#pragma unroll
  for (int i = l; i < kRedBlocks; i += 32) {
    a += pl[i];
    b += pn[i];
    if (mode == 1) q += pq[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if (l != 0) return;
  scal[0] = a + b;
  if (mode == 1) {
    scal[1] = q;
    scal[2] = -0.5 * q - 0.5 * scal[0] - 0.5 * (double)n * log(2.0 * 3.14159265358979323846);
  }
}

__global__ void k_gather(const double* __restrict__ y, int64_t ld, int nrhs,
                         const int32_t* __restrict__ perm, int64_t n, double* __restrict__ Y,
                         double* __restrict__ ysort) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  for (int c = 0; c < nrhs; ++c) {
    double v = y[c * ld + p];
    Y[c * n + i] = v;
    if (c == 0 && ysort) ysort[i] = v;
  }
}

__global__ void k_scatter(const double* __restrict__ Y, int nrhs, const int32_t* __restrict__ perm,
                          int64_t n, double* __restrict__ x, int64_t ld) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  for (int c = 0; c < nrhs; ++c) x[c * ld + p] = Y[c * n + i];
}

// ---- HODLR operator product (dense leaves + U V^T blocks) ------------------------------
struct MvArgs {
  Pts pts;
  int kind;
  const double* hyp;
  const int32_t* nb;
  const int32_t* ns;
  int leaf0, kappa, R;
  const double* phi;
  const int* coff;   // device copy not needed: passed by value below
  const double* xin;
  double* yout;
  double* part;      // leaf x R partials (Phi^T x)
  const double* half;  // per level half sums, level j at half + hoff[j]
  int64_t n;
  int phiff;           // 1: Phi holds double-float pairs (mixed form)
};

__device__ __forceinline__ double phi_at(const MvArgs& a, int64_t k) {
  return a.phiff ? ff_to_double(reinterpret_cast<const ff*>(a.phi)[k]) : a.phi[k];
}

struct LevelTab {
  int coff[33];
  int rl[32];
  int64_t hoff[32];
};

__global__ void k_mv_partials(MvArgs a, LevelTab t) {
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = w; c < a.R; c += blockDim.x / 32) {
    double s = 0.0;
    for (int i = lane; i < p; i += 32) s += phi_at(a, (int64_t)c * a.n + b + i) * a.xin[b + i];
    s = wsum(s);
    if (lane == 0) a.part[(int64_t)leaf * a.R + c] = s;
  }
}

__global__ void k_mv_apply(MvArgs a, LevelTab t) {
  const Cov cov = cov_from(a.kind, a.hyp);
  const double sigma2 = a.hyp[kHypSigma2];
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    double s = 0.0;
    for (int jj = 0; jj < p; ++jj) {
      double r = dist(a.pts, b + i, b + jj);
      double c = cov_r(cov, r);
      if (jj == i) c += sigma2;
      s += c * a.xin[b + jj];
    }
    for (int l = 0; l < a.kappa; ++l) {
      int sh = a.kappa - l;
      int k = leaf >> sh;
      int side = (leaf >> (sh - 1)) & 1;
      const double* hs = a.half + t.hoff[l] + (int64_t)(2 * k + (1 - side)) * t.rl[l];
      for (int c = 0; c < t.rl[l]; ++c) s += phi_at(a, (int64_t)(t.coff[l] + c) * a.n + b + i) * hs[c];
    }
    a.yout[b + i] = s;
  }
}

}  // namespace

cudaError_t launch_gather_rhs(Ctx& c, const double* y, int64_t ld, int nrhs) {
  unsigned g = (unsigned)((c.n + 255) / 256);
  k_gather<<<g, 256, 0, c.stream>>>(y, ld, nrhs, c.perm, c.n, c.Y, c.ysort);
  ++c.launches;
  return cudaGetLastError();
}

cudaError_t launch_scatter_rhs(Ctx& c, double* x, int64_t ld, int nrhs) {
  unsigned g = (unsigned)((c.n + 255) / 256);
  k_scatter<<<g, 256, 0, c.stream>>>(c.Y, nrhs, c.perm, c.n, x, ld);
  ++c.launches;
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sweep(const SweepArgs& sa, unsigned grid, size_t smem, cudaStream_t st) {
  if (smem <= 200 * 1024) {
    if (smem > kSmemOptIn)
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_sweep<true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sweep<true, T><<<grid, kSweepThreads, smem, st>>>(sa);
  } else {
    k_sweep<false, T><<<grid, kSweepThreads, 0, st>>>(sa);
  }
  return cudaGetLastError();
}

// Sweep of all internal levels after the leaf stage has written the level-(kappa-1)
// partials. factor_mode: build and factor M per node (panel columns included); otherwise
// reuse the stored LU factors and carry only the right-hand sides.
// Levels whose sweep step is in product form (gemm_step) hand the next level its half sums
// directly (stride r_j w_j); the others go through per-leaf partials and segmented sums.
cudaError_t launch_levels(Ctx& c, int nrhs, bool factor_mode) {
  int K = c.kappa;
  int64_t nleaf = (int64_t)1 << K;
  for (int j = K - 1; j >= 0; --j) {
    int r = c.h_rl[j];
    int cj = c.h_coff[j];
    int cP = factor_mode ? cj + r : 0;  // panel columns in the level-j partials
    int w = cP + nrhs;
    int h = 1 << (K - j - 1);
    const bool direct = j + 1 < K && gemm_step(c, j + 1);
    if (!direct)
      HODLR_CUDA_TRY(segsum(c.part, c.part_stride, r * w, nleaf, h, c.part2, c.half, c.stream, &c.launches));
    NodeArgs na;
    na.half = c.half;
    na.stride = direct ? (int64_t)r * w : c.part_stride;
    na.j = j;
    na.r = r;
    na.w = w;
    na.cj = factor_mode ? cj : -1;
    na.wz = (factor_mode ? cj : 0) + nrhs;
    na.Mlu = c.Mlu + c.h_mlu_off[j];
    na.Mpiv = c.Mpiv + c.h_piv_off[j];
    na.node_logdet = c.node_logdet;
    na.Z = c.Z;
    na.z_stride = (int64_t)2 * r * na.wz;
    na.flags = c.dflags;
    na.zff = c.precision == 1;
    na.signed_det = c.indefinite;
    if (r > 0) {
      HODLR_CUDA_TRY(launch_node(c, na, factor_mode));
    } else if (factor_mode) {
      HODLR_CUDA_TRY(cudaMemsetAsync(c.node_logdet + ((1 << j) - 1), 0, sizeof(double) << j, c.stream));
    }
    if (r == 0) {
      // nothing to apply at this level; the level-(j-1) partials must still be formed
      // from unchanged rows: run the sweep with rank 0 (pure reduction).
    }
    SweepArgs sa;
    sa.nb = c.nodes;
    sa.ns = c.nodes + ((int64_t)2 << K);
    sa.leaf0 = (int)(nleaf - 1);
    sa.kappa = K;
    sa.u = j;
    sa.pan = c.pan;
    sa.phi = c.phi;
    sa.Y = c.Y;
    sa.cP = factor_mode ? cj : 0;
    sa.nrhs = nrhs;
    sa.cu = cj;
    sa.ru = r;
    sa.cl = j > 0 ? c.h_coff[j - 1] : 0;
    sa.rl = j > 0 ? c.h_rl[j - 1] : 0;
    sa.Z = c.Z;
    sa.z_stride = (int64_t)2 * r * (sa.cP + nrhs);
    sa.part = c.part;
    sa.part_stride = c.part_stride;
    sa.n = c.n;
    if (sa.cP + nrhs == 0) continue;  // nothing left to update (root level, no right-hand side)
    if (gemm_step(c, j)) {
      HODLR_CUDA_TRY(launch_sweep_gemm(c, j, nrhs, factor_mode));
      continue;
    }
    size_t smem = sizeof(double) * kMaxLeaf * (sa.ru + sa.rl);
    if (c.precision == 1)
      HODLR_CUDA_TRY(launch_sweep<ff>(sa, (unsigned)nleaf, smem, c.stream));
    else
      HODLR_CUDA_TRY(launch_sweep<double>(sa, (unsigned)nleaf, smem, c.stream));
    ++c.launches;
    HODLR_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Node step of the finest internal level for the fused sweep: its half-nodes are single
// leaves, so the leaf stage's partials are the half sums. Z goes to buffer (kappa-1) & 1.
cudaError_t launch_level_first(Ctx& c, int nrhs, bool factor_mode) {
  int j = c.kappa - 1;
  int r = c.h_rl[j], cj = c.h_coff[j];
  int w = (factor_mode ? cj + r : 0) + nrhs;
  NodeArgs na;
  na.half = c.part;
  na.stride = c.part_stride;
  na.j = j;
  na.r = r;
  na.w = w;
  na.cj = factor_mode ? cj : -1;
  na.wz = (factor_mode ? cj : 0) + nrhs;
  na.Mlu = c.Mlu + c.h_mlu_off[j];
  na.Mpiv = c.Mpiv + c.h_piv_off[j];
  na.node_logdet = c.node_logdet;
  na.Z = c.Z + (j & 1) * c.z_elems;
  na.z_stride = (int64_t)2 * r * na.wz;
  na.flags = c.dflags;
  na.zff = c.precision == 1;
  na.signed_det = c.indefinite;
  if (r == 0) {
    if (factor_mode)
      HODLR_CUDA_TRY(cudaMemsetAsync(c.node_logdet + ((1 << j) - 1), 0, sizeof(double) << j, c.stream));
    return cudaSuccess;
  }
  return launch_node(c, na, factor_mode);
}

// Device hyperparameter slot from host values (stream-ordered, capturable).
__global__ void k_set_hyp(double* hyp, int kind, double ell, double amp, double sigma2,
                          double alpha) {
  hyp[kHypInvEll] = 1.0 / ell;
  hyp[kHypAmp] = amp;
  hyp[kHypSigma2] = sigma2;
  hyp[kHypScale] = cov_scale(kind, ell);
  hyp[kHypAlpha] = alpha;
  set_hyp_ff(hyp);
}

// The same from setting idx[0] of device arrays theta (ell, a pairs) and sigma2.
__global__ void k_load_setting(double* hyp, int kind, const double* theta, const double* sigma2,
                               const int32_t* idx) {
  int b = idx[0];
  double ell = theta[2 * b], amp = theta[2 * b + 1];
  hyp[kHypInvEll] = 1.0 / ell;
  hyp[kHypAmp] = amp;
  hyp[kHypSigma2] = sigma2[b];
  hyp[kHypScale] = cov_scale(kind, ell);
  set_hyp_ff(hyp);
}

cudaError_t launch_set_hyp(Ctx& c, double ell, double amp, double sigma2) {
  k_set_hyp<<<1, 1, 0, c.stream>>>(c.hyp, c.kind, ell, amp, sigma2, c.alpha);
  ++c.launches;
  return cudaGetLastError();
}

cudaError_t launch_load_setting(Ctx& c, const double* theta, const double* sigma2,
                                const int32_t* idx) {
  k_load_setting<<<1, 1, 0, c.stream>>>(c.hyp, c.kind, theta, sigma2, idx);
  ++c.launches;
  return cudaGetLastError();
}

cudaError_t launch_logdet_sum(Ctx& c) {
  int64_t nleaf = (int64_t)1 << c.kappa;
  double* tmp = c.part2;  // scratch: 3 x kRedBlocks
  k_sum_blocks<<<kRedBlocks, 256, 0, c.stream>>>(c.leaf_logdet, nullptr, nleaf, tmp);
  k_sum_blocks<<<kRedBlocks, 256, 0, c.stream>>>(c.node_logdet, nullptr, nleaf - 1, tmp + kRedBlocks);
  k_finish<<<1, 32, 0, c.stream>>>(tmp, tmp + kRedBlocks, nullptr, c.scal, c.n, 0);
  c.launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_quad_loglik(Ctx& c) {
  int64_t nleaf = (int64_t)1 << c.kappa;
  double* tmp = c.part2;
  k_sum_blocks<<<kRedBlocks, 256, 0, c.stream>>>(c.leaf_logdet, nullptr, nleaf, tmp);
  k_sum_blocks<<<kRedBlocks, 256, 0, c.stream>>>(c.node_logdet, nullptr, nleaf - 1, tmp + kRedBlocks);
  k_sum_blocks<<<kRedBlocks, 256, 0, c.stream>>>(c.ysort, c.Y, c.n, tmp + 2 * kRedBlocks);
  k_finish<<<1, 32, 0, c.stream>>>(tmp, tmp + kRedBlocks, tmp + 2 * kRedBlocks, c.scal, c.n, 1);
  c.launches += 4;
  return cudaGetLastError();
}

cudaError_t launch_matvec(Ctx& c, const double* xin, double* yout) {
  int K = c.kappa;
  int64_t nleaf = (int64_t)1 << K;
  MvArgs a;
  a.pts = Pts{c.xs, c.n, c.d};
  a.kind = c.kind;
  a.hyp = c.hyp;
  a.nb = c.nodes;
  a.ns = c.nodes + ((int64_t)2 << K);
  a.leaf0 = (int)(nleaf - 1);
  a.kappa = K;
  a.R = c.R;
  a.phi = c.phi;
  a.coff = nullptr;
  a.xin = xin;
  a.yout = yout;
  a.part = c.part;
  a.n = c.n;
  a.phiff = c.precision == 1;
  LevelTab t;
  int64_t off = 0;
  for (int j = 0; j < 32; ++j) {
    t.rl[j] = j < K ? c.h_rl[j] : 0;
    t.hoff[j] = off;
    if (j < K) off += ((int64_t)2 << j) * c.h_rl[j];
  }
  for (int j = 0; j < 33; ++j) t.coff[j] = j <= K ? c.h_coff[j] : 0;
  double* half = c.half;
  a.half = half;
  if (K > 0 && c.R > 0) {
    k_mv_partials<<<(unsigned)nleaf, 128, 0, c.stream>>>(a, t);
    ++c.launches;
    HODLR_CUDA_TRY(cudaGetLastError());
    for (int j = 0; j < K; ++j) {
      if (c.h_rl[j] == 0) continue;
      // half sums of level j: groups of 2^(K-j-1) leaves; the level's columns start at coff_j
      HODLR_CUDA_TRY(segsum(c.part + c.h_coff[j], c.R, c.h_rl[j], nleaf, 1 << (K - j - 1),
                            c.part2, c.Z, c.stream, &c.launches));
      // compact rows of width rl_j into half + hoff_j
      HODLR_CUDA_TRY(cudaMemcpy2DAsync(half + t.hoff[j], sizeof(double) * c.h_rl[j], c.Z,
                                       sizeof(double) * c.R, sizeof(double) * c.h_rl[j],
                                       (size_t)2 << j, cudaMemcpyDeviceToDevice, c.stream));
    }
  }
  k_mv_apply<<<(unsigned)nleaf, 128, 0, c.stream>>>(a, t);
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
