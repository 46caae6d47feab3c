// Level sweep with one launch per level (Sec. 3.2, the level-by-level factorization and the
// SMW solve), for the usual case of small partial products.
//
// k_level(u) updates every leaf's rows with the level-u SMW correction,
//   P_L -= Ut Z_top, P_R -= Vt Z_bot     (Z of level u, computed by the previous launch),
// forms the level-(u-1) partial products Phi_{u-1}^T P of its leaves, and then, in the
// same launch, finishes level u-1: the last block to finish a half-node sums that half's
// partials in leaf order (fixed order: results are deterministic), and the last half of a
// node runs the node step (M, LU, log det, Z of level u-1; node_solve.cuh). Blocks only
// count arrivals with atomics; no block ever waits for another.
#include <cuda_runtime.h>

#include "ff.cuh"
#include "hodlr_internal.cuh"
#include "node_solve.cuh"

namespace hodlr {
namespace {

// Tile shapes of the fused sweep: leaves per block (kTileG); the threads per block of
// shapes 0..6 are 256, 128, 256, 512, 64, 64 and 128 (the launch switch below).
constexpr int kSweepTiles = 7;
constexpr int kTileG[kSweepTiles] = {4, 2, 8, 8, 2, 1, 1};

struct FusedArgs {
  const int32_t* nb;
  const int32_t* ns;
  int leaf0, kappa, u;
  double* pan;
  const double* phi;
  double* Y;
  int cP, nrhs;       // updated columns: panel [0, cP), right-hand sides [0, nrhs)
  int cu, ru;         // level u: Ut/Vt columns in pan, rank
  const double* Zu;   // level-u Z, 2 ru wz per node
  int cl, rl;         // level u-1: Phi columns, rank (no reduction if rl == 0 or u == 0)
  double* part;
  int64_t part_stride;
  int32_t* cnt;       // arrival counters: half-nodes [0, 2^u), then nodes [2^u, 2^u + 2^(u-1))
  NodeArgs na;        // node step of level u-1
  int factor;
  int64_t n;
};

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Mixed form, a right-hand-side column: FP64 arithmetic (the solution keeps FP64
// accuracy), the double-float panel values converted as they are read; Z's right-hand-side
// columns are FP64.
__device__ __forceinline__ void leaf_column_rhs(const FusedArgs& a, int leaf, int b, int p, int q,
                                                int wz, int sh, int zs, int lane) {
  const ff* panf = reinterpret_cast<const ff*>(a.pan);
  const ff* phif = reinterpret_cast<const ff*>(a.phi);
  double* col = a.Y + (int64_t)(q - a.cP) * a.n + b;
  double x[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = m * 32 + lane;
    x[m] = i < p ? col[i] : 0.0;
  }
  if (a.ru > 0) {
    int side = (leaf >> (sh - 1)) & 1;
    const double* Zs = a.Zu + (int64_t)(leaf >> sh) * zs + (int64_t)side * a.ru * wz;
    for (int c = 0; c < a.ru; ++c) {
      double z = Zs[c * wz + q];
      const ff* tl = panf + (int64_t)(a.cu + c) * a.n + b;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) x[m] -= ff_to_double(tl[i]) * z;
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int i = m * 32 + lane;
      if (i < p) col[i] = x[m];
    }
  }
  if (a.u > 0 && a.rl > 0) {
    double* out = a.part + (int64_t)leaf * a.part_stride;
    for (int c = 0; c < a.rl; ++c) {
      const ff* ph = phif + (int64_t)(a.cl + c) * a.n + b;
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) s += ff_to_double(ph[i]) * x[m];
      }
      s = wsum(s);
      if (lane == 0) out[c * wz + q] = s;
    }
  }
}

// Read-only loads: the level's own Ut/Vt columns, Phi and the level's Z are not written by
// this launch (it writes the coarser levels' columns, the right-hand sides and the other Z
// buffer), so they may take the non-coherent path and be scheduled ahead of the stores.
__device__ __forceinline__ ff ldg_ff(const ff* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return ff{v.x, v.y};
}

// Finish two partial sums of one warp at once (a reduce-scatter): after exchanging across
// lane ^ 16, lanes 0..15 carry s0 and lanes 16..31 carry s1, and four more xor steps leave
// the totals in lanes 0 and 16. Fixed order: deterministic.
__device__ __forceinline__ double wsum2(double s0, double s1, int lane) {
  const bool hi = (lane & 16) != 0;
  double mine = hi ? s1 : s0, other = hi ? s0 : s1;
  mine += __shfl_xor_sync(0xffffffffu, other, 16);
  for (int o = 8; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  return mine;
}

// FP64 form, two columns q and q1 of [panel | right-hand sides] of one leaf.
__device__ __forceinline__ void leaf_pair_f64(const FusedArgs& a, int leaf, int b, int p, int q,
                                              bool two, int wz, int sh, int zs, int lane) {
  const int q1 = two ? q + 1 : q;
  double* c0p = q < a.cP ? a.pan + (int64_t)q * a.n + b : a.Y + (int64_t)(q - a.cP) * a.n + b;
  double* c1p = q1 < a.cP ? a.pan + (int64_t)q1 * a.n + b : a.Y + (int64_t)(q1 - a.cP) * a.n + b;
  double x0[4], x1[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = m * 32 + lane;
    x0[m] = i < p ? c0p[i] : 0.0;
    x1[m] = (two && i < p) ? c1p[i] : 0.0;
  }
  if (a.ru > 0) {
    int side = (leaf >> (sh - 1)) & 1;
    const double* Zs = a.Zu + (int64_t)(leaf >> sh) * zs + (int64_t)side * a.ru * wz;
    for (int c = 0; c < a.ru; ++c) {
      double z0 = __ldg(Zs + c * wz + q), z1 = __ldg(Zs + c * wz + q1);
      const double* tl = a.pan + (int64_t)(a.cu + c) * a.n + b;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) {
          double t = __ldg(tl + i);
          x0[m] -= t * z0;
          x1[m] -= t * z1;
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int i = m * 32 + lane;
      if (i < p) {
        c0p[i] = x0[m];
        if (two) c1p[i] = x1[m];
      }
    }
  }
  if (a.u > 0 && a.rl > 0) {
    double* out = a.part + (int64_t)leaf * a.part_stride;
    for (int c = 0; c < a.rl; ++c) {
      const double* ph = a.phi + (int64_t)(a.cl + c) * a.n + b;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) {
          double h = __ldg(ph + i);
          s0 += h * x0[m];
          s1 += h * x1[m];
        }
      }
      double t = wsum2(s0, s1, lane);
      if (lane == 0) out[c * wz + q] = t;
      if (two && lane == 16) out[c * wz + q1] = t;
    }
  }
}

// Mixed form, a panel column: the panels and Z's panel columns are double-float pairs; the
// update and the partial products run on the FP32 pipe.
__device__ __forceinline__ void leaf_column_ff(const FusedArgs& a, int leaf, int b, int p, int q,
                                               int wz, int sh, int zs, int lane) {
  if (q >= a.cP) {
    leaf_column_rhs(a, leaf, b, p, q, wz, sh, zs, lane);
    return;
  }
  ff* panf = reinterpret_cast<ff*>(a.pan);
  const ff* phif = reinterpret_cast<const ff*>(a.phi);
  ff x[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = m * 32 + lane;
    x[m] = i < p ? panf[(int64_t)q * a.n + b + i] : ff{0.0f, 0.0f};
  }
  if (a.ru > 0) {
    int side = (leaf >> (sh - 1)) & 1;
    const ff* Zs = reinterpret_cast<const ff*>(a.Zu) + (int64_t)(leaf >> sh) * zs + (int64_t)side * a.ru * wz;
    for (int c = 0; c < a.ru; ++c) {
      ff z = ldg_ff(Zs + c * wz + q);
      const ff* tl = panf + (int64_t)(a.cu + c) * a.n + b;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) x[m] = ff_fms(x[m], ldg_ff(tl + i), z);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int i = m * 32 + lane;
      if (i < p) panf[(int64_t)q * a.n + b + i] = x[m];
    }
  }
  if (a.u > 0 && a.rl > 0) {
    double* out = a.part + (int64_t)leaf * a.part_stride;
    for (int c = 0; c < a.rl; ++c) {
      const ff* ph = phif + (int64_t)(a.cl + c) * a.n + b;
      ff s = {0.0f, 0.0f};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) s = ff_fma(s, ldg_ff(ph + i), x[m]);
      }
      for (int o = 16; o > 0; o >>= 1)
        s = ff_add(s, ff{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)});
      if (lane == 0) out[c * wz + q] = ff_to_double(s);
    }
  }
}

// G leaves per block, T threads (the tile shape, chosen per problem by the autotuner).
template <bool kFF, int G, int T>
__global__ void __launch_bounds__(T) k_level(FusedArgs a) {
  extern __shared__ double M[];  // node step, (2 rl)^2
  __shared__ int piv[2 * kSmemRank];
  __shared__ double lds;
  __shared__ int sgn;
  __shared__ int flag;
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int nleaf = 1 << a.kappa;
  int leaf_base = blockIdx.x * G;
  int nl = nleaf - leaf_base < G ? nleaf - leaf_base : G;
  int wz = a.cP + a.nrhs;
  int sh = a.kappa - a.u;  // leaves per level-u half-node = 2^(sh - 1); per node = 2^sh
  int zs = 2 * a.ru * wz;
  // tasks. FP64 form: pairs of columns of one leaf (the level's columns read once for two,
  // one reduce-scatter for both partial sums). Mixed form: one column of one leaf per
  // task, twice as many warps in flight for the longer double-float chains (measured
  // faster than pairs there).
  const int npair = kFF ? 0 : (wz + 1) >> 1;
  const int ntask = kFF ? wz : npair;
  for (int t = w; t < nl * ntask; t += T / 32) {
    int g = t / ntask, k = t - g * ntask;
    int leaf = leaf_base + g;
    int id = a.leaf0 + leaf;
    int b = a.nb[id], p = a.ns[id];
    if (kFF) {
      leaf_column_ff(a, leaf, b, p, k, wz, sh, zs, lane);
    } else {
      int q = 2 * k;
      leaf_pair_f64(a, leaf, b, p, q, q + 1 < wz, wz, sh, zs, lane);
    }
  }
  if (a.u == 0 || a.rl == 0) return;
  // finish level l = u - 1: half-nodes of 2^sh' leaves with sh' = kappa - l - 1 = sh
  int hl = 1 << sh;            // leaves per level-l half-node
  int E = a.rl * wz;
  // Where a half-node spans several blocks, each block first sums its own leaves'
  // partials (fixed order) into its first leaf's slot, so the last block of the half sums
  // one value per block instead of one per leaf.
  const bool pre = hl >= 2 * G;  // then this block's G leaves lie inside one half-node
  __syncthreads();
  if (pre) {
    double* p0 = a.part + (int64_t)leaf_base * a.part_stride;
    for (int e = tid; e < E; e += T) {
      double s = p0[e];
      for (int t = 1; t < nl; ++t) s += p0[(int64_t)t * a.part_stride + e];
      p0[e] = s;
    }
  }
  const int step = pre ? G : 1;   // leaf stride between the slots to sum
  const int nsl = hl / step;       // slots per half-node
  __threadfence();
  __syncthreads();
  int h0 = leaf_base >> sh, h1 = (leaf_base + nl - 1) >> sh;
  for (int h = h0; h <= h1; ++h) {
    int lo = h * hl > leaf_base ? h * hl : leaf_base;
    int hi = (h + 1) * hl < leaf_base + nl ? (h + 1) * hl : leaf_base + nl;
    __syncthreads();  // every thread has read the previous flag
    if (tid == 0) {
      int old = atomicAdd(&a.cnt[h], hi - lo);
      flag = old + (hi - lo) == hl;
    }
    __syncthreads();
    if (!flag) continue;  // uniform across the block
    __threadfence();
    double* hs = const_cast<double*>(a.na.half) + (int64_t)h * a.na.stride;
    const double* pbase = a.part + (int64_t)h * hl * a.part_stride;
    const int64_t sst = (int64_t)step * a.part_stride;
    if (nsl >= 32) {
      // one warp per entry: lanes stride over the half's slots, then a fixed xor tree
      for (int e = w; e < E; e += T / 32) {
        double s = 0.0;
        for (int t = lane; t < nsl; t += 32) s += __ldcg(pbase + (int64_t)t * sst + e);
        s = wsum(s);
        if (lane == 0) hs[e] = s;
      }
    } else {
      for (int e = tid; e < E; e += T) {
        double s = 0.0;
        for (int t = 0; t < nsl; ++t) s += __ldcg(pbase + (int64_t)t * sst + e);
        hs[e] = s;
      }
    }
    __threadfence();
    __syncthreads();
    int node = h >> 1;
    if (tid == 0) {
      a.cnt[h] = 0;
      int old = atomicAdd(&a.cnt[(1 << a.u) + node], 1);
      flag = old == 1;
    }
    __syncthreads();
    if (!flag) continue;
    __threadfence();
    node_solve(a.na, node, a.factor != 0, M, piv, &lds, &sgn);
    if (tid == 0) a.cnt[(1 << a.u) + node] = 0;
  }
}

template <bool kFF, int G, int T>
cudaError_t launch_level(const FusedArgs& fa, unsigned grid, size_t smem, cudaStream_t s) {
  if (smem > kSmemOptIn)
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_level<kFF, G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_level<kFF, G, T><<<grid, T, smem, s>>>(fa);
  return cudaGetLastError();
}

}  // namespace

// Sweep of levels kappa-1 .. 0 when the leaf stage has written the level-(kappa-1)
// partials: the level-(kappa-1) node step by the segmented path, then one k_level launch
// per level. Z alternates between two buffers so a launch never overwrites the Z it reads.
cudaError_t launch_levels_fused(Ctx& c, int nrhs, bool factor_mode) {
  int K = c.kappa;
  if (K == 0) return cudaSuccess;
  int64_t nleaf = (int64_t)1 << K;
  HODLR_CUDA_TRY(cudaMemsetAsync(c.cnt, 0, sizeof(int32_t) * (size_t)(nleaf + nleaf / 2 + 2), c.stream));
  HODLR_CUDA_TRY(launch_level_first(c, nrhs, factor_mode));  // node step of level kappa-1
  for (int u = K - 1; u >= 0; --u) {
    int ru = c.h_rl[u], cu = c.h_coff[u];
    int cP = factor_mode ? cu : 0;
    int wz = cP + nrhs;
    int l = u - 1;
    FusedArgs fa;
    fa.nb = c.nodes;
    fa.ns = c.nodes + ((int64_t)2 << K);
    fa.leaf0 = (int)(nleaf - 1);
    fa.kappa = K;
    fa.u = u;
    fa.pan = c.pan;
    fa.phi = c.phi;
    fa.Y = c.Y;
    fa.cP = cP;
    fa.nrhs = nrhs;
    fa.cu = cu;
    fa.ru = ru;
    fa.Zu = c.Z + (u & 1) * c.z_elems;
    fa.cl = l >= 0 ? c.h_coff[l] : 0;
    fa.rl = l >= 0 ? c.h_rl[l] : 0;
    fa.part = c.part;
    fa.part_stride = c.part_stride;
    fa.cnt = c.cnt;
    fa.factor = factor_mode;
    fa.n = c.n;
    if (l >= 0) {
      NodeArgs& na = fa.na;
      na.half = c.half;
      na.stride = c.part_stride;
      na.j = l;
      na.r = fa.rl;
      na.w = wz;
      na.cj = factor_mode ? fa.cl : -1;
      na.wz = (factor_mode ? fa.cl : 0) + nrhs;
      na.Mlu = c.Mlu + c.h_mlu_off[l];
      na.Mpiv = c.Mpiv + c.h_piv_off[l];
      na.node_logdet = c.node_logdet;
      na.Z = c.Z + (l & 1) * c.z_elems;
      na.z_stride = (int64_t)2 * fa.rl * na.wz;
      na.flags = c.dflags;
      na.zff = c.precision == 1;
      na.signed_det = c.indefinite;
      if (factor_mode && fa.rl == 0)
        HODLR_CUDA_TRY(cudaMemsetAsync(c.node_logdet + ((1 << l) - 1), 0, sizeof(double) << l, c.stream));
    }
    if (wz == 0 && (l < 0 || fa.rl == 0)) continue;
    size_t smem = sizeof(double) * 4 * fa.rl * fa.rl;
    const int tile = c.sweep_tile >= 0 && c.sweep_tile < kSweepTiles ? c.sweep_tile : 0;
    unsigned grid = (unsigned)((nleaf + kTileG[tile] - 1) / kTileG[tile]);
    switch (tile * 2 + (c.precision == 1 ? 1 : 0)) {
      case 0: HODLR_CUDA_TRY((launch_level<false, 4, 256>(fa, grid, smem, c.stream))); break;
      case 1: HODLR_CUDA_TRY((launch_level<true, 4, 256>(fa, grid, smem, c.stream))); break;
      case 2: HODLR_CUDA_TRY((launch_level<false, 2, 128>(fa, grid, smem, c.stream))); break;
      case 3: HODLR_CUDA_TRY((launch_level<true, 2, 128>(fa, grid, smem, c.stream))); break;
      case 4: HODLR_CUDA_TRY((launch_level<false, 8, 256>(fa, grid, smem, c.stream))); break;
      case 5: HODLR_CUDA_TRY((launch_level<true, 8, 256>(fa, grid, smem, c.stream))); break;
      case 6: HODLR_CUDA_TRY((launch_level<false, 8, 512>(fa, grid, smem, c.stream))); break;
      case 7: HODLR_CUDA_TRY((launch_level<true, 8, 512>(fa, grid, smem, c.stream))); break;
      case 8: HODLR_CUDA_TRY((launch_level<false, 2, 64>(fa, grid, smem, c.stream))); break;
      case 9: HODLR_CUDA_TRY((launch_level<true, 2, 64>(fa, grid, smem, c.stream))); break;
      case 10: HODLR_CUDA_TRY((launch_level<false, 1, 64>(fa, grid, smem, c.stream))); break;
      case 11: HODLR_CUDA_TRY((launch_level<true, 1, 64>(fa, grid, smem, c.stream))); break;
      case 12: HODLR_CUDA_TRY((launch_level<false, 1, 128>(fa, grid, smem, c.stream))); break;
      default: HODLR_CUDA_TRY((launch_level<true, 1, 128>(fa, grid, smem, c.stream)));
    }
    ++c.launches;
    HODLR_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace hodlr
