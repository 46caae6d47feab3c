// Level-batched adaptive cross approximation (Sec. 3.1: partial-pivoted LU of each
// off-diagonal block, O(r m) work per block, with the Frobenius-norm estimate as the
// sub-sampled error check). Every internal node of every level advances together, one
// cross step per four launches:
//   A  residual row    R(i,:) = B(i,:) - sum_l u_l(i) v_l        (tile of columns per CTA)
//   B  pivot column    j = argmax |R(i,:)| (lowest index on ties), delta = R(i,j)
//   C  residual column u = B(:,j) - sum_l u_l v_l(j), v = R(i,:) / delta, tile dots
//   D  norm update     |S_k|^2 += 2 sum_l (u_l.u)(v_l.v) + |u|^2 |v|^2; stop (dropping the
//                      term) when |u||v| <= eps |S_k|; next row = argmax over unused rows
// The block B = K[I_left, I_right] of node id lives in one column of the level's raw panel:
// rows of the left child hold u, rows of the right child hold v. All reductions use fixed
// orders, so results are deterministic. The cross starts at the first row; a zero pivot
// moves to the unused row nearest the right child's first point (rows far from the
// interface of a fast-decaying kernel can be exactly zero).
// In the mixed form the block entries are evaluated
// in double-float (ff.cuh) from the FP64 distances and the columns are stored and updated
// as double-float pairs (8 bytes, like a double), so the per-element work runs on the FP32
// pipe; the norm and dot-product partial sums that drive the stopping test are taken in
// FP32 per thread and combined in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kAcaThreads = 256;
constexpr int kPer = kAcaTile / kAcaThreads;  // elements per thread
// Shared memory of the tiled kernels does not grow with the rank: the cross's earlier
// vectors at the pivot (u_l(i), v_l(j)), the used rows and the per-warp dot products pass
// through fixed-size chunks, each sum keeping its order.
constexpr int kRankChunk = 1024;  // u_l(i) or v_l(j) values per chunk
constexpr int kUsedChunk = 1024;  // used rows per chunk
constexpr int kDotChunk = 64;     // dot products u_l.u, v_l.v per chunk

struct AcaArgs {
  Pts pts;
  int kind;
  const double* hyp;   // device hyperparameter slot
  double eps;
  const int32_t* nb;   // node begin
  const int32_t* ns;   // node size
  const int32_t* item_node;
  const int32_t* item_start;
  const int32_t* node_item0;
  const int32_t* node_item1;
  double* raw;
  int64_t raw_off[32];
  int32_t *rank, *row, *col, *done, *ok, *zero, *phase, *nused, *used;
  int used_stride;
  double *delta, *s2, *part;
  int part_stride;
  int max_rank;
  const ff* tab;       // 2^(j/64) as double-floats (mixed form)
  const ff* xrel;      // mixed form: per level, coordinates relative to each node's split
                       // point (kappa x d x n double-floats)
  int32_t* active;
  int nint;
  int pre[32];         // presized rank of each level (0: adaptive)
  const int32_t* node_witem0;  // per node: first wide item (-1: none), one past the last
  const int32_t* node_witem1;
  const int32_t* wide_nodes;   // the nodes with wide items
};

// Entry k(x_i, x_j) of an off-diagonal block: FP64, or (mixed form) double-float
// evaluation of the covariance from the FP64 distance. kGen = false: the kernels
// specialised for points in one or two dimensions and the four covariances of Table 1
// (the common case, whose code stays free of the general paths); true: any d and kind.
template <bool kFF, bool kGen>
__device__ __forceinline__ double block_entry(const AcaArgs& a, const Cov& cov, int i, int j,
                                              const ff* tab, const CovFF& cf) {
  double r = kGen ? dist(a.pts, i, j) : dist12(a.pts, i, j);
  if (!kFF) return kGen ? cov_r(cov, r) : cov_r_table1(cov, r);
  ff v = kGen ? cov_ff(cf, ff_from_double(r), tab) : cov_ff_table1(cf, ff_from_double(r), tab);
  return ff_to_double(v);
}

// The same entry as a double-float (mixed form), for i in the left and j in the right
// child of a level-lev node. The distance comes from the coordinates relative to the
// node's split point (the first point of its right child): in 1-D the left child's are
// <= 0 and the right child's >= 0, so r = x_j - x_i is a same-sign double-float sum whose
// error is relative to r itself, also for the closest pairs across the split; no FP64.
template <bool kGen>
__device__ __forceinline__ ff block_entry_ff(const AcaArgs& a, int lev, int i, int j,
                                            const ff* tab, const CovFF& cf) {
  const int64_t n = a.pts.n;
  const ff* xr = a.xrel + (int64_t)lev * a.pts.d * n;
  ff r;
  if (a.pts.d == 1) {
    r = ff_sub(xr[j], xr[i]);
    if (r.hi < 0.0f) r = ff_neg(r);
  } else {
    ff u = ff_sub(xr[j], xr[i]), v = ff_sub(xr[n + j], xr[n + i]);
    ff s = ff_add(ff_mul(u, u), ff_mul(v, v));
    if (kGen)
      for (int c = 2; c < a.pts.d; ++c) {
        ff w = ff_sub(xr[c * n + j], xr[c * n + i]);
        s = ff_add(s, ff_mul(w, w));
      }
    r = ff_sqrt(s);
  }
  return kGen ? cov_ff(cf, r, tab) : cov_ff_table1(cf, r, tab);
}

__device__ __forceinline__ int level_of(int id) { return 31 - __clz(id + 1); }

// Node id's cross runs on its 32-row wide items once its rank has reached kWideRank (the
// rank changes only at the end of a step, so every kernel of a step agrees), before that on
// its 1024-row tiles.
__device__ __forceinline__ bool wide_now(const AcaArgs& a, int id) {
  return a.node_witem0[id] >= 0 && a.rank[id] >= kWideRank;
}

// Squared distance of point i to point s, accumulated coordinate by coordinate without
// fused multiply-adds (the same operations, in the same order, as the oracle's restart
// rule, so both pick the same rows).
__device__ __forceinline__ double split_d2(const Pts& p, int64_t i, int64_t s) {
  double d2 = 0.0;
  for (int c = 0; c < p.d; ++c) {
    double t = __dsub_rn(p.x[c * p.n + i], p.x[c * p.n + s]);
    d2 = __dadd_rn(d2, __dmul_rn(t, t));
  }
  return d2;
}

// Rank cap of a block: min(m_left, m_right, max_rank), and in presized mode the level's
// rank + 1 (one extra cross step shows whether the block converged within its rank).
__device__ __forceinline__ int rmax_of(const AcaArgs& a, int id) {
  int ml = a.ns[2 * id + 1], mr = a.ns[2 * id + 2];
  int m = ml < mr ? ml : mr;
  m = m < a.max_rank ? m : a.max_rank;
  int pre = a.pre[level_of(id)];
  if (pre > 0 && pre + 1 < m) m = pre + 1;
  return m;
}

// Argmax of |v| with the lowest index on ties (idx < 0 means empty).
__device__ __forceinline__ void amax_merge(double& bv, int& bi, double v, int i) {
  if (i < 0) return;
  double av = fabs(v), ab = fabs(bv);
  if (bi < 0 || av > ab || (av == ab && i < bi)) {
    bv = v;
    bi = i;
  }
}

__device__ __forceinline__ void warp_amax(double& bv, int& bi) {
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    amax_merge(bv, bi, ov, oi);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Argmax on float magnitudes (mixed form: the high word of each double-float).
__device__ __forceinline__ void amax_merge_f(float& bv, int& bi, float v, int i) {
  if (i < 0) return;
  float av = fabsf(v), ab = fabsf(bv);
  if (bi < 0 || av > ab || (av == ab && i < bi)) {
    bv = v;
    bi = i;
  }
}

__device__ __forceinline__ void warp_amax_f(float& bv, int& bi) {
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    amax_merge_f(bv, bi, ov, oi);
  }
}

__global__ void k_aca_init(AcaArgs a) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.nint) return;
  a.rank[id] = 0;
  a.row[id] = 0;
  a.col[id] = 0;
  a.done[id] = rmax_of(a, id) <= 0;
  a.ok[id] = 0;
  a.zero[id] = 0;
  a.phase[id] = 0;
  a.nused[id] = 0;
  a.s2[id] = 0.0;
  a.delta[id] = 0.0;
}

// A: residual row of the current pivot row, stored unnormalised in column k of the V rows.
template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kAcaThreads) k_aca_row(AcaArgs a) {
  int item = blockIdx.x;
  int id = a.item_node[item];
  if (a.done[id] || wide_now(a, id)) return;
  __shared__ double dsm[kRankChunk];  // u_l(i) for a chunk of l
  __shared__ ff tab[64];
  __shared__ double wv[kAcaThreads / 32];
  __shared__ int wi[kAcaThreads / 32];
  const Cov cov = cov_from(a.kind, a.hyp);
  CovFF cf{};
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kAcaThreads) tab[q] = a.tab[q];
    cf = load_cov_ff(a.kind, a.hyp);
  }
  int k = a.rank[id], i = a.row[id];
  int bl = a.nb[2 * id + 1], br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  int64_t n = a.pts.n;
  double* raw = a.raw + a.raw_off[level_of(id)];
  int start = a.item_start[item];
  int w = threadIdx.x >> 5;
  int bi = -1;
  if (kFF) __syncthreads();  // tab
  if (!kFF) {
    double* uik = dsm;
    double v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int b = start + q * kAcaThreads + threadIdx.x;
      v[q] = b < mr ? block_entry<false, kGen>(a, cov, bl + i, br + b, tab, cf) : 0.0;
    }
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kAcaThreads) uik[l - l0] = raw[l * n + bl + i];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int b = start + q * kAcaThreads + threadIdx.x;
        if (b < mr)
          for (int l = l0; l < l1; ++l) v[q] -= uik[l - l0] * raw[l * n + br + b];
      }
    }
    double bv = 0.0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int b = start + q * kAcaThreads + threadIdx.x;
      if (b < mr) {
        raw[(int64_t)k * n + br + b] = v[q];
        amax_merge(bv, bi, v[q], b);
      }
    }
    warp_amax(bv, bi);
    if ((threadIdx.x & 31) == 0) {
      wv[w] = bv;
      wi[w] = bi;
    }
  } else {
    ff* rawf = reinterpret_cast<ff*>(raw);
    ff* uik = reinterpret_cast<ff*>(dsm);
    ff v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int b = start + q * kAcaThreads + threadIdx.x;
      v[q] = b < mr ? block_entry_ff<kGen>(a, level_of(id), bl + i, br + b, tab, cf) : ff{0.0f, 0.0f};
    }
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kAcaThreads) uik[l - l0] = rawf[l * n + bl + i];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int b = start + q * kAcaThreads + threadIdx.x;
        if (b < mr)
          for (int l = l0; l < l1; ++l) v[q] = ff_fms(v[q], uik[l - l0], rawf[l * n + br + b]);
      }
    }
    float bv = 0.0f;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int b = start + q * kAcaThreads + threadIdx.x;
      if (b < mr) {
        rawf[(int64_t)k * n + br + b] = v[q];
        amax_merge_f(bv, bi, v[q].hi, b);
      }
    }
    warp_amax_f(bv, bi);
    if ((threadIdx.x & 31) == 0) {
      wv[w] = bv;
      wi[w] = bi;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double fv = 0.0;
    int fi = -1;
    for (int q = 0; q < kAcaThreads / 32; ++q) amax_merge(fv, fi, wv[q], wi[q]);
    // the mixed form chose by the high word; the pivot value is the full double-float
    if (kFF && fi >= 0) fv = ff_to_double(reinterpret_cast<const ff*>(raw)[(int64_t)k * n + br + fi]);
    a.part[(int64_t)item * a.part_stride + 0] = fv;
    a.part[(int64_t)item * a.part_stride + 1] = (double)fi;
  }
}

// B: one warp per node picks the pivot column (or handles an all-zero residual row).
__global__ void k_aca_pivot_row(AcaArgs a) {
  int id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (id >= a.nint || a.done[id]) return;
  const bool wd = wide_now(a, id);
  int i0 = wd ? a.node_witem0[id] : a.node_item0[id], i1 = wd ? a.node_witem1[id] : a.node_item1[id];
  double bv = 0.0;
  int bi = -1;
  for (int it = i0 + lane; it < i1; it += 32) {
    const double* p = a.part + (int64_t)it * a.part_stride;
    amax_merge(bv, bi, p[0], (int)p[1]);
  }
  warp_amax(bv, bi);
  int i = a.row[id];
  int* used = a.used + (int64_t)id * a.used_stride;
  int nu = a.nused[id];
  if (lane == 0) {
    used[nu] = i;
    a.nused[id] = nu + 1;
  }
  ++nu;
  if (bi >= 0 && bv != 0.0) {
    if (lane == 0) {
      a.col[id] = bi;
      a.delta[id] = bv;
      a.phase[id] = 1;
    }
    return;
  }
  // zero pivot: move to the unused row nearest the split (whole warp; lowest index on ties)
  int rmax = rmax_of(a, id);
  if (a.zero[id] + 1 > rmax) {
    if (lane == 0) {
      a.phase[id] = 0;
      a.zero[id] += 1;
      a.done[id] = 1;
      a.ok[id] = 1;
    }
    return;
  }
  __syncwarp();
  int bl = a.nb[2 * id + 1], ml = a.ns[2 * id + 1], br = a.nb[2 * id + 2];
  double bd = 0.0;
  int nx = -1;
  for (int r = lane; r < ml; r += 32) {
    bool u = false;
    for (int q = 0; q < nu; ++q) u |= used[q] == r;
    if (u) continue;
    double d2 = split_d2(a.pts, bl + r, br);
    if (nx < 0 || d2 < bd) {
      bd = d2;
      nx = r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double od = __shfl_xor_sync(0xffffffffu, bd, o);
    int on = __shfl_xor_sync(0xffffffffu, nx, o);
    if (on >= 0 && (nx < 0 || od < bd || (od == bd && on < nx))) {
      bd = od;
      nx = on;
    }
  }
  if (lane != 0) return;
  a.phase[id] = 0;
  a.zero[id] += 1;
  if (nx < 0) {
    a.done[id] = 1;
    a.ok[id] = 1;
    return;
  }
  a.row[id] = nx;
}

// C: residual column u (stored in column k of the U rows), normalised row v, and this tile's
// contributions to |u|^2, |v|^2, u_l.u, v_l.v and argmax over unused rows of |u|.
template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kAcaThreads) k_aca_col(AcaArgs a) {
  int item = blockIdx.x;
  int id = a.item_node[item];
  if (a.done[id] || !a.phase[id] || wide_now(a, id)) return;
  constexpr int kW = kAcaThreads / 32;
  __shared__ double vjk_s[kRankChunk];           // v_l(j) for a chunk of l
  __shared__ int used_s[kUsedChunk];             // a chunk of the used rows
  __shared__ double red[2 * kDotChunk * kW];     // per-warp u_l.u, then v_l.v, of a chunk
  __shared__ double rn[2 * kW];                  // per-warp |u|^2, |v|^2
  __shared__ ff tab[64];
  CovFF cf{};
  const Cov cov = cov_from(a.kind, a.hyp);
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kAcaThreads) tab[q] = a.tab[q];
    cf = load_cov_ff(a.kind, a.hyp);
  }
  __shared__ double wv[kAcaThreads / 32];
  __shared__ int wi[kAcaThreads / 32];
  int k = a.rank[id], j = a.col[id];
  double delta = a.delta[id];
  int bl = a.nb[2 * id + 1], ml = a.ns[2 * id + 1];
  int br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  int nu = a.nused[id];
  int64_t n = a.pts.n;
  double* raw = a.raw + a.raw_off[level_of(id)];
  int start = a.item_start[item];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // which of this thread's rows are used (pivot rows of earlier steps)
  bool isu[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) isu[q] = false;
  for (int s0 = 0; s0 < nu; s0 += kUsedChunk) {
    const int s1 = min(nu - s0, kUsedChunk);
    __syncthreads();
    for (int q = threadIdx.x; q < s1; q += kAcaThreads) used_s[q] = a.used[(int64_t)id * a.used_stride + s0 + q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = start + q * kAcaThreads + threadIdx.x;
      if (t < ml)
        for (int s = 0; s < s1; ++s) isu[q] |= used_s[s] == t;
    }
  }
  if (kFF) __syncthreads();  // tab
  int bi = -1;
  if (!kFF) {
    const double inv = 1.0 / delta;
    double uu[kPer], vv[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = start + q * kAcaThreads + threadIdx.x;
      uu[q] = t < ml ? block_entry<false, kGen>(a, cov, bl + t, br + j, tab, cf) : 0.0;
    }
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kAcaThreads) vjk_s[l - l0] = raw[l * n + br + j];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int t = start + q * kAcaThreads + threadIdx.x;
        if (t < ml)
          for (int l = l0; l < l1; ++l) uu[q] -= raw[l * n + bl + t] * vjk_s[l - l0];
      }
    }
    double nu2 = 0.0, nv2 = 0.0, bv = 0.0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = start + q * kAcaThreads + threadIdx.x;
      vv[q] = 0.0;
      if (t < ml) {
        const double u = uu[q];
        raw[(int64_t)k * n + bl + t] = u;
        nu2 += u * u;
        if (!isu[q]) amax_merge(bv, bi, u, t);
      }
      if (t < mr) {
        double v = raw[(int64_t)k * n + br + t] * inv;
        raw[(int64_t)k * n + br + t] = v;
        vv[q] = v;
        nv2 += v * v;
      }
    }
    nu2 = warp_sum(nu2);
    nv2 = warp_sum(nv2);
    warp_amax(bv, bi);
    if (lane == 0) {
      rn[w] = nu2;
      rn[kW + w] = nv2;
      wv[w] = bv;
      wi[w] = bi;
    }
    for (int l0 = 0; l0 < k; l0 += kDotChunk) {
      const int l1 = min(k, l0 + kDotChunk);
      for (int l = l0; l < l1; ++l) {
        double du = 0.0, dv = 0.0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          int t = start + q * kAcaThreads + threadIdx.x;
          if (t < ml) du += raw[l * n + bl + t] * uu[q];
          if (t < mr) dv += raw[l * n + br + t] * vv[q];
        }
        du = warp_sum(du);
        dv = warp_sum(dv);
        if (lane == 0) {
          red[(l - l0) * kW + w] = du;
          red[(kDotChunk + l - l0) * kW + w] = dv;
        }
      }
      __syncthreads();
      double* out = a.part + (int64_t)item * a.part_stride;
      for (int e = threadIdx.x; e < 2 * kDotChunk; e += kAcaThreads) {
        const int l = e < kDotChunk ? l0 + e : l0 + e - kDotChunk;
        if (l >= l1) continue;
        double s = 0.0;
        for (int q = 0; q < kW; ++q) s += red[e * kW + q];
        out[(e < kDotChunk ? 4 : 4 + a.max_rank) + l] = s;
      }
      __syncthreads();
    }
  } else {
    ff* rawf = reinterpret_cast<ff*>(raw);
    ff* vjk = reinterpret_cast<ff*>(vjk_s);
    __shared__ ff inv_s;  // 1 / delta, converted by one thread (FP64 pipe)
    if (threadIdx.x == 0) inv_s = ff_rcp(ff_from_double(delta));
    ff u[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = start + q * kAcaThreads + threadIdx.x;
      u[q] = t < ml ? block_entry_ff<kGen>(a, level_of(id), bl + t, br + j, tab, cf) : ff{0.0f, 0.0f};
    }
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kAcaThreads) vjk[l - l0] = rawf[l * n + br + j];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int t = start + q * kAcaThreads + threadIdx.x;
        if (t < ml)
          for (int l = l0; l < l1; ++l) u[q] = ff_fms(u[q], rawf[l * n + bl + t], vjk[l - l0]);
      }
    }
    __syncthreads();  // inv_s
    const ff inv = inv_s;
    float uu[kPer], vv[kPer];  // high words, for the dot products of the stopping test
    float nu2 = 0.0f, nv2 = 0.0f, bv = 0.0f;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = start + q * kAcaThreads + threadIdx.x;
      uu[q] = 0.0f;
      vv[q] = 0.0f;
      if (t < ml) {
        rawf[(int64_t)k * n + bl + t] = u[q];
        uu[q] = u[q].hi;
        nu2 += u[q].hi * u[q].hi;
        if (!isu[q]) amax_merge_f(bv, bi, u[q].hi, t);
      }
      if (t < mr) {
        ff v = ff_mul(rawf[(int64_t)k * n + br + t], inv);
        rawf[(int64_t)k * n + br + t] = v;
        vv[q] = v.hi;
        nv2 += v.hi * v.hi;
      }
    }
    double nu2d = warp_sum((double)nu2), nv2d = warp_sum((double)nv2);
    warp_amax_f(bv, bi);
    if (lane == 0) {
      rn[w] = nu2d;
      rn[kW + w] = nv2d;
      wv[w] = bv;
      wi[w] = bi;
    }
    for (int l0 = 0; l0 < k; l0 += kDotChunk) {
      const int l1 = min(k, l0 + kDotChunk);
      for (int l = l0; l < l1; ++l) {
        float du = 0.0f, dv = 0.0f;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          int t = start + q * kAcaThreads + threadIdx.x;
          if (t < ml) du += rawf[l * n + bl + t].hi * uu[q];
          if (t < mr) dv += rawf[l * n + br + t].hi * vv[q];
        }
        du = warp_sum_f(du);
        dv = warp_sum_f(dv);
        if (lane == 0) {
          red[(l - l0) * kW + w] = du;
          red[(kDotChunk + l - l0) * kW + w] = dv;
        }
      }
      __syncthreads();
      double* out = a.part + (int64_t)item * a.part_stride;
      for (int e = threadIdx.x; e < 2 * kDotChunk; e += kAcaThreads) {
        const int l = e < kDotChunk ? l0 + e : l0 + e - kDotChunk;
        if (l >= l1) continue;
        double s = 0.0;
        for (int q = 0; q < kW; ++q) s += red[e * kW + q];
        out[(e < kDotChunk ? 4 : 4 + a.max_rank) + l] = s;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // layout: [0] argmax value, [1] argmax index, [2] |u|^2, [3] |v|^2, [4..] u_l.u, v_l.v
  if (threadIdx.x == 0) {
    double* out = a.part + (int64_t)item * a.part_stride;
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < kW; ++q) {
      s0 += rn[q];
      s1 += rn[kW + q];
    }
    out[2] = s0;
    out[3] = s1;
    double fv = 0.0;
    int fi = -1;
    for (int q = 0; q < kAcaThreads / 32; ++q) amax_merge(fv, fi, wv[q], wi[q]);
    out[0] = fv;
    out[1] = (double)fi;
  }
}

// A and C for small nodes (both children <= kSmallNode points, one work item each): one warp
// per node, eight nodes per block, warp-level reductions only; the same per-item outputs
// as the tiled kernels (argmax, |u|^2, |v|^2, u_l.u, v_l.v).
constexpr int kSmallPer = kSmallNode / 32;  // elements per lane

template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kAcaThreads) k_aca_row_small(AcaArgs a, int item0, int nitem) {
  __shared__ ff tab[64];
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kAcaThreads) tab[q] = a.tab[q];
    __syncthreads();
  }
  int lane = threadIdx.x & 31;
  int item = item0 + blockIdx.x * (kAcaThreads / 32) + (threadIdx.x >> 5);
  if (item >= item0 + nitem) return;
  int id = a.item_node[item];
  if (a.done[id]) return;
  const Cov cov = cov_from(a.kind, a.hyp);
  int k = a.rank[id], i = a.row[id];
  int bl = a.nb[2 * id + 1], br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  int64_t n = a.pts.n;
  int lev = level_of(id);
  double* raw = a.raw + a.raw_off[lev];
  int bi = -1;
  double fv = 0.0;
  if (!kFF) {
    double bv = 0.0;
#pragma unroll
    for (int q = 0; q < kSmallPer; ++q) {
      int b = q * 32 + lane;
      if (b < mr) {
        double v = block_entry<false, kGen>(a, cov, bl + i, br + b, tab, CovFF{});
        for (int l = 0; l < k; ++l) v -= raw[l * n + bl + i] * raw[l * n + br + b];
        raw[(int64_t)k * n + br + b] = v;
        amax_merge(bv, bi, v, b);
      }
    }
    warp_amax(bv, bi);
    fv = bv;
  } else {
    const CovFF cf = load_cov_ff(a.kind, a.hyp);
    ff* rawf = reinterpret_cast<ff*>(raw);
    float bv = 0.0f;
#pragma unroll
    for (int q = 0; q < kSmallPer; ++q) {
      int b = q * 32 + lane;
      if (b < mr) {
        ff v = block_entry_ff<kGen>(a, lev, bl + i, br + b, tab, cf);
        for (int l = 0; l < k; ++l) v = ff_fms(v, rawf[l * n + bl + i], rawf[l * n + br + b]);
        rawf[(int64_t)k * n + br + b] = v;
        amax_merge_f(bv, bi, v.hi, b);
      }
    }
    warp_amax_f(bv, bi);
    if (bi >= 0) fv = ff_to_double(rawf[(int64_t)k * n + br + bi]);  // full pivot value
  }
  if (lane == 0) {
    a.part[(int64_t)item * a.part_stride + 0] = fv;
    a.part[(int64_t)item * a.part_stride + 1] = (double)bi;
  }
}

template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kAcaThreads) k_aca_col_small(AcaArgs a, int item0, int nitem) {
  __shared__ ff tab[64];
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kAcaThreads) tab[q] = a.tab[q];
    __syncthreads();
  }
  int lane = threadIdx.x & 31;
  int item = item0 + blockIdx.x * (kAcaThreads / 32) + (threadIdx.x >> 5);
  if (item >= item0 + nitem) return;
  int id = a.item_node[item];
  if (a.done[id] || !a.phase[id]) return;
  const Cov cov = cov_from(a.kind, a.hyp);
  int k = a.rank[id], j = a.col[id];
  double delta = a.delta[id];
  int bl = a.nb[2 * id + 1], ml = a.ns[2 * id + 1];
  int br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  int nu = a.nused[id];
  const int* used = a.used + (int64_t)id * a.used_stride;
  int64_t n = a.pts.n;
  int lev = level_of(id);
  double* raw = a.raw + a.raw_off[lev];
  double* out = a.part + (int64_t)item * a.part_stride;
  int bi = -1;
  if (!kFF) {
    const double inv = 1.0 / delta;
    double uu[kSmallPer], vv[kSmallPer];
    double nu2 = 0.0, nv2 = 0.0, bv = 0.0;
#pragma unroll
    for (int q = 0; q < kSmallPer; ++q) {
      int t = q * 32 + lane;
      uu[q] = 0.0;
      vv[q] = 0.0;
      if (t < ml) {
        double u = block_entry<false, kGen>(a, cov, bl + t, br + j, tab, CovFF{});
        for (int l = 0; l < k; ++l) u -= raw[l * n + bl + t] * raw[l * n + br + j];
        raw[(int64_t)k * n + bl + t] = u;
        uu[q] = u;
        nu2 += u * u;
        bool isu = false;
        for (int s2 = 0; s2 < nu; ++s2) isu |= used[s2] == t;
        if (!isu) amax_merge(bv, bi, u, t);
      }
      if (t < mr) {
        double v = raw[(int64_t)k * n + br + t] * inv;
        raw[(int64_t)k * n + br + t] = v;
        vv[q] = v;
        nv2 += v * v;
      }
    }
    nu2 = warp_sum(nu2);
    nv2 = warp_sum(nv2);
    warp_amax(bv, bi);
    for (int l = 0; l < k; ++l) {
      double du = 0.0, dv = 0.0;
#pragma unroll
      for (int q = 0; q < kSmallPer; ++q) {
        int t = q * 32 + lane;
        if (t < ml) du += raw[l * n + bl + t] * uu[q];
        if (t < mr) dv += raw[l * n + br + t] * vv[q];
      }
      du = warp_sum(du);
      dv = warp_sum(dv);
      if (lane == 0) {
        out[4 + l] = du;
        out[4 + a.max_rank + l] = dv;
      }
    }
    if (lane == 0) {
      out[0] = bv;
      out[1] = (double)bi;
      out[2] = nu2;
      out[3] = nv2;
    }
  } else {
    const CovFF cf = load_cov_ff(a.kind, a.hyp);
    ff* rawf = reinterpret_cast<ff*>(raw);
    const ff inv = ff_rcp(ff_from_double(delta));
    float uu[kSmallPer], vv[kSmallPer];
    float nu2 = 0.0f, nv2 = 0.0f, bv = 0.0f;
#pragma unroll
    for (int q = 0; q < kSmallPer; ++q) {
      int t = q * 32 + lane;
      uu[q] = 0.0f;
      vv[q] = 0.0f;
      if (t < ml) {
        ff u = block_entry_ff<kGen>(a, lev, bl + t, br + j, tab, cf);
        for (int l = 0; l < k; ++l) u = ff_fms(u, rawf[l * n + bl + t], rawf[l * n + br + j]);
        rawf[(int64_t)k * n + bl + t] = u;
        uu[q] = u.hi;
        nu2 += u.hi * u.hi;
        bool isu = false;
        for (int s2 = 0; s2 < nu; ++s2) isu |= used[s2] == t;
        if (!isu) amax_merge_f(bv, bi, u.hi, t);
      }
      if (t < mr) {
        ff v = ff_mul(rawf[(int64_t)k * n + br + t], inv);
        rawf[(int64_t)k * n + br + t] = v;
        vv[q] = v.hi;
        nv2 += v.hi * v.hi;
      }
    }
    double nu2d = warp_sum((double)nu2), nv2d = warp_sum((double)nv2);
    warp_amax_f(bv, bi);
    for (int l = 0; l < k; ++l) {
      float du = 0.0f, dv = 0.0f;
#pragma unroll
      for (int q = 0; q < kSmallPer; ++q) {
        int t = q * 32 + lane;
        if (t < ml) du += rawf[l * n + bl + t].hi * uu[q];
        if (t < mr) dv += rawf[l * n + br + t].hi * vv[q];
      }
      du = warp_sum_f(du);
      dv = warp_sum_f(dv);
      if (lane == 0) {
        out[4 + l] = du;
        out[4 + a.max_rank + l] = dv;
      }
    }
    if (lane == 0) {
      out[0] = bv;
      out[1] = (double)bi;
      out[2] = nu2d;
      out[3] = nv2d;
    }
  }
}

// Norm update and stopping decision of node id after its step k (one thread): |S_k|^2 +=
// 2 cross + |u|^2 |v|^2; stop when |u||v| <= eps |S_k| (the term dropped), when no unused
// row is left, or at the rank cap; else the next pivot row is bi.
__device__ void col_decide(const AcaArgs& a, int id, int k, int bi, double nu2, double nv2,
                           double cross) {
  double s2 = a.s2[id] + 2.0 * cross + nu2 * nv2;
  a.s2[id] = s2;
  if (sqrt(nu2 * nv2) <= a.eps * sqrt(s2)) {
    a.done[id] = 1;
    a.ok[id] = 1;
    return;
  }
  int r = k + 1;
  a.rank[id] = r;
  if (bi < 0) {
    a.done[id] = 1;
    a.ok[id] = 1;
    return;
  }
  a.row[id] = bi;
  int rmax = rmax_of(a, id);
  if (r >= rmax) {
    int ml = a.ns[2 * id + 1], mr = a.ns[2 * id + 2];
    a.done[id] = 1;
    a.ok[id] = rmax == (ml < mr ? ml : mr);
    return;
  }
  atomicAdd(a.active, 1);
}


// D: one warp per node combines the tiles, updates the norm estimate and decides (wide
// nodes: k_aca_pivot_col_wide).
__global__ void k_aca_pivot_col(AcaArgs a) {
  int id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (id >= a.nint || a.done[id] || wide_now(a, id)) return;
  if (!a.phase[id]) {
    if (lane == 0) atomicAdd(a.active, 1);
    return;
  }
  int k = a.rank[id];
  int i0 = a.node_item0[id], i1 = a.node_item1[id];
  double bv = 0.0, nu2 = 0.0, nv2 = 0.0;
  int bi = -1;
  for (int it = i0 + lane; it < i1; it += 32) {
    const double* p = a.part + (int64_t)it * a.part_stride;
    amax_merge(bv, bi, p[0], (int)p[1]);
    nu2 += p[2];
    nv2 += p[3];
  }
  warp_amax(bv, bi);
  nu2 = warp_sum(nu2);
  nv2 = warp_sum(nv2);
  // sum_l (u_l.u)(v_l.v), in whichever of two fixed orders costs fewer dependent adds: many
  // tiles and a small rank (the top levels of a large problem): lanes over tiles and one warp
  // sum per l; else lane l mod 32 takes l and sums the tiles in item order
  double cross = 0.0;
  const int items = i1 - i0;
  if (k * ((items + 31) / 32 + 5) <= ((k + 31) / 32) * items) {
    for (int l = 0; l < k; ++l) {
      double du = 0.0, dv = 0.0;
      for (int it = i0 + lane; it < i1; it += 32) {
        const double* p = a.part + (int64_t)it * a.part_stride;
        du += p[4 + l];
        dv += p[4 + a.max_rank + l];
      }
      du = warp_sum(du);
      dv = warp_sum(dv);
      cross += du * dv;
    }
  } else {
    for (int l = lane; l < k; l += 32) {
      double du = 0.0, dv = 0.0;
      for (int it = i0; it < i1; ++it) {
        const double* p = a.part + (int64_t)it * a.part_stride;
        du += p[4 + l];
        dv += p[4 + a.max_rank + l];
      }
      cross += du * dv;
    }
    cross = warp_sum(cross);
  }
  if (lane == 0) col_decide(a, id, k, bi, nu2, nv2, cross);
}

// ---- wide nodes: rank cap above kWideRank ----------------------------------------------
// Work items of kWideTile rows, so that a block of a top-level node spreads over many CTAs.
// The sum over the cross's earlier vectors is split over the warps (warp w takes l = w,
// w + 8, ...; the warps' partial sums are added in warp order); the dot products u_l.u and
// v_l.v of a tile run with threads over l and the tile's rows in order. The FP64 form
// computes in FP64; the mixed form as its 1024-row kernels do: residuals in double-float
// on the FP32 pipe, dot products and norms from the high words in FP32.
static_assert(kWideTile == 32, "one row of a wide item per lane");
constexpr int kCrossL = 128;  // l values per CTA of the wide cross term
constexpr int kWideThreads = 512;  // CTA of the wide row and column kernels (16 warps)

// A for a wide item: residual row entries b = start + lane of the right child.
template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kWideThreads) k_aca_row_wide(AcaArgs a, int item0) {
  constexpr int kW = kWideThreads / 32;
  const int item = item0 + blockIdx.x;
  const int id = a.item_node[item];
  if (a.done[id] || a.rank[id] < kWideRank) return;
  __shared__ double uik[kRankChunk];
  __shared__ double red[kW][kWideTile];
  __shared__ ff tab[64];
  const Cov cov = cov_from(a.kind, a.hyp);
  CovFF cf{};
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kWideThreads) tab[q] = a.tab[q];
    cf = load_cov_ff(a.kind, a.hyp);
  }
  const int k = a.rank[id], i = a.row[id];
  const int bl = a.nb[2 * id + 1], br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  const int64_t n = a.pts.n;
  double* raw = a.raw + a.raw_off[level_of(id)];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = a.item_start[item] + lane;
  if constexpr (kFF) {
    // mixed form: double-float sums on the FP32 pipe, the argmax on the high words (as in
    // k_aca_row<true>); the pivot value is the stored double-float
    const ff* rawf = reinterpret_cast<const ff*>(raw);
    ff* uf = reinterpret_cast<ff*>(uik);
    ff* rf = reinterpret_cast<ff*>(&red[0][0]);
    ff acc = {0.0f, 0.0f};
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kWideThreads) uf[l - l0] = rawf[l * n + bl + i];
      __syncthreads();
      if (b < mr)
        for (int l = l0 + w; l < l1; l += kW) acc = ff_fma(acc, uf[l - l0], rawf[l * n + br + b]);
    }
    rf[w * kWideTile + lane] = acc;
    __syncthreads();
    if (w != 0) return;
    float bv = 0.0f;
    int bi = -1;
    if (b < mr) {
      ff sum = rf[lane];
      for (int q = 1; q < kW; ++q) sum = ff_add(sum, rf[q * kWideTile + lane]);
      const ff v = ff_sub(block_entry_ff<kGen>(a, level_of(id), bl + i, br + b, tab, cf), sum);
      reinterpret_cast<ff*>(raw)[(int64_t)k * n + br + b] = v;
      amax_merge_f(bv, bi, v.hi, b);
    }
    warp_amax_f(bv, bi);
    __syncwarp();  // the winning lane's store is visible to lane 0
    if (lane == 0) {
      a.part[(int64_t)item * a.part_stride + 0] = bi >= 0 ? ff_to_double(rawf[(int64_t)k * n + br + bi]) : 0.0;
      a.part[(int64_t)item * a.part_stride + 1] = (double)bi;
    }
  } else {
    double acc = 0.0;
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kWideThreads) uik[l - l0] = raw[l * n + bl + i];
      __syncthreads();
      if (b < mr)
        for (int l = l0 + w; l < l1; l += kW) acc += uik[l - l0] * raw[l * n + br + b];
    }
    red[w][lane] = acc;
    __syncthreads();
    if (w != 0) return;
    double bv = 0.0;
    int bi = -1;
    if (b < mr) {
      double s = 0.0;
      for (int q = 0; q < kW; ++q) s += red[q][lane];
      const double v = block_entry<false, kGen>(a, cov, bl + i, br + b, tab, cf) - s;
      raw[(int64_t)k * n + br + b] = v;
      amax_merge(bv, bi, v, b);
    }
    warp_amax(bv, bi);
    if (lane == 0) {
      a.part[(int64_t)item * a.part_stride + 0] = bv;
      a.part[(int64_t)item * a.part_stride + 1] = (double)bi;
    }
  }
}

// C for a wide item: rows t = start + lane of u (left child) and of v (right child), their
// norms and unused-row argmax, then the tile's u_l.u and v_l.v for every l < k.
template <bool kFF, bool kGen>
__global__ void __launch_bounds__(kWideThreads) k_aca_col_wide(AcaArgs a, int item0) {
  constexpr int kW = kWideThreads / 32;
  const int item = item0 + blockIdx.x;
  const int id = a.item_node[item];
  if (a.done[id] || !a.phase[id] || a.rank[id] < kWideRank) return;
  __shared__ double vjk[kRankChunk];
  __shared__ int used_s[kUsedChunk];
  __shared__ double red[kW][kWideTile];
  __shared__ double us[kWideTile], vs[kWideTile];
  __shared__ int isu_s[kWideTile];
  __shared__ ff tab[64];
  const Cov cov = cov_from(a.kind, a.hyp);
  CovFF cf{};
  if (kFF) {
    for (int q = threadIdx.x; q < 64; q += kWideThreads) tab[q] = a.tab[q];
    cf = load_cov_ff(a.kind, a.hyp);
  }
  const int k = a.rank[id], j = a.col[id];
  const double delta = a.delta[id];
  const int bl = a.nb[2 * id + 1], ml = a.ns[2 * id + 1];
  const int br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  const int nu = a.nused[id];
  const int64_t n = a.pts.n;
  double* raw = a.raw + a.raw_off[level_of(id)];
  const int start = a.item_start[item];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = start + lane;
  if (threadIdx.x < kWideTile) isu_s[threadIdx.x] = 0;
  for (int s0 = 0; s0 < nu; s0 += kUsedChunk) {
    const int s1 = min(nu - s0, kUsedChunk);
    __syncthreads();
    for (int q = threadIdx.x; q < s1; q += kWideThreads) used_s[q] = a.used[(int64_t)id * a.used_stride + s0 + q];
    __syncthreads();
    bool f = false;
    for (int q = w; q < s1; q += kW) f |= used_s[q] == t;
    if (f) isu_s[lane] = 1;
  }
  if constexpr (kFF) {
    // mixed form: the residual column in double-float on the FP32 pipe, the norms and the
    // dot products from the high words in FP32 (combined in FP64 by the norm update), the
    // argmax on the high words: as in k_aca_col<true>
    const ff* rawf = reinterpret_cast<const ff*>(raw);
    ff* vf = reinterpret_cast<ff*>(vjk);
    ff* rf = reinterpret_cast<ff*>(&red[0][0]);
    __shared__ ff inv_s;  // 1 / delta, converted by one thread (FP64 pipe)
    __shared__ float ush[kWideTile], vsh[kWideTile];
    if (threadIdx.x == 0) inv_s = ff_rcp(ff_from_double(delta));
    ff acc = {0.0f, 0.0f};
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kWideThreads) vf[l - l0] = rawf[l * n + br + j];
      __syncthreads();
      if (t < ml)
        for (int l = l0 + w; l < l1; l += kW) acc = ff_fma(acc, rawf[l * n + bl + t], vf[l - l0]);
    }
    rf[w * kWideTile + lane] = acc;
    __syncthreads();
    double* out = a.part + (int64_t)item * a.part_stride;
    if (w == 0) {
      float uh = 0.0f, vh = 0.0f, bv = 0.0f;
      int bi = -1;
      if (t < ml) {
        ff sum = rf[lane];
        for (int q = 1; q < kW; ++q) sum = ff_add(sum, rf[q * kWideTile + lane]);
        const ff u = ff_sub(block_entry_ff<kGen>(a, level_of(id), bl + t, br + j, tab, cf), sum);
        reinterpret_cast<ff*>(raw)[(int64_t)k * n + bl + t] = u;
        uh = u.hi;
        if (!isu_s[lane]) amax_merge_f(bv, bi, u.hi, t);
      }
      if (t < mr) {
        const int64_t e = (int64_t)k * n + br + t;
        const ff v = ff_mul(rawf[e], inv_s);
        reinterpret_cast<ff*>(raw)[e] = v;
        vh = v.hi;
      }
      ush[lane] = uh;
      vsh[lane] = vh;
      const double nu2 = warp_sum((double)(uh * uh)), nv2 = warp_sum((double)(vh * vh));
      warp_amax_f(bv, bi);
      if (lane == 0) {
        out[0] = bv;
        out[1] = (double)bi;
        out[2] = nu2;
        out[3] = nv2;
      }
    }
    // u_l.u and v_l.v from the high words: the tile's columns staged as FP32 (coalesced
    // 32-row loads), thread l summing its column in row order
    extern __shared__ double tile[];
    float* tf = reinterpret_cast<float*>(tile);
    constexpr int kLd = kWideTile + 1;
    const int tu = min(kWideTile, ml - start), tv = min(kWideTile, mr - start);
    for (int lb = 0; lb < k; lb += kWideThreads) {
      const int nl = min(kWideThreads, k - lb);
      const int l = lb + threadIdx.x;
      __syncthreads();
      for (int ll = w; ll < nl; ll += kW)
        tf[ll * kLd + lane] = lane < tu ? rawf[(int64_t)(lb + ll) * n + bl + start + lane].hi : 0.0f;
      __syncthreads();
      float du = 0.0f;
      if (threadIdx.x < nl)
        for (int q = 0; q < tu; ++q) du += tf[threadIdx.x * kLd + q] * ush[q];
      __syncthreads();
      for (int ll = w; ll < nl; ll += kW)
        tf[ll * kLd + lane] = lane < tv ? rawf[(int64_t)(lb + ll) * n + br + start + lane].hi : 0.0f;
      __syncthreads();
      if (threadIdx.x < nl) {
        float dv = 0.0f;
        for (int q = 0; q < tv; ++q) dv += tf[threadIdx.x * kLd + q] * vsh[q];
        out[4 + l] = du;
        out[4 + a.max_rank + l] = dv;
      }
    }
  } else {
    double acc = 0.0;
    for (int l0 = 0; l0 < k; l0 += kRankChunk) {
      const int l1 = min(k, l0 + kRankChunk);
      __syncthreads();
      for (int l = l0 + threadIdx.x; l < l1; l += kWideThreads) vjk[l - l0] = raw[l * n + br + j];
      __syncthreads();
      if (t < ml)
        for (int l = l0 + w; l < l1; l += kW) acc += raw[l * n + bl + t] * vjk[l - l0];
    }
    red[w][lane] = acc;
    __syncthreads();
    double* out = a.part + (int64_t)item * a.part_stride;
    if (w == 0) {
      double u = 0.0, v = 0.0, bv = 0.0;
      int bi = -1;
      if (t < ml) {
        double s = 0.0;
        for (int q = 0; q < kW; ++q) s += red[q][lane];
        u = block_entry<false, kGen>(a, cov, bl + t, br + j, tab, cf) - s;
        raw[(int64_t)k * n + bl + t] = u;
        if (!isu_s[lane]) amax_merge(bv, bi, u, t);
      }
      if (t < mr) {
        const int64_t e = (int64_t)k * n + br + t;
        v = raw[e] * (1.0 / delta);
        raw[e] = v;
      }
      us[lane] = u;
      vs[lane] = v;
      const double nu2 = warp_sum(u * u), nv2 = warp_sum(v * v);
      warp_amax(bv, bi);
      if (lane == 0) {
        out[0] = bv;
        out[1] = (double)bi;
        out[2] = nu2;
        out[3] = nv2;
      }
    }
    // u_l.u and v_l.v over this tile's rows: kWideThreads values of l at a time, their columns
    // staged through shared memory (each warp loads whole 32-row columns, coalesced), then
    // thread l sums its column in row order
    extern __shared__ double tile[];  // kWideThreads x (kWideTile + 1)
    constexpr int kLd = kWideTile + 1;
    const int tu = min(kWideTile, ml - start), tv = min(kWideTile, mr - start);
    for (int lb = 0; lb < k; lb += kWideThreads) {
      const int nl = min(kWideThreads, k - lb);
      const int l = lb + threadIdx.x;
      __syncthreads();
      for (int ll = w; ll < nl; ll += kW)
        tile[ll * kLd + lane] = lane < tu ? raw[(int64_t)(lb + ll) * n + bl + start + lane] : 0.0;
      __syncthreads();
      double du = 0.0;
      if (threadIdx.x < nl)
        for (int q = 0; q < tu; ++q) du += tile[threadIdx.x * kLd + q] * us[q];
      __syncthreads();
      for (int ll = w; ll < nl; ll += kW)
        tile[ll * kLd + lane] = lane < tv ? raw[(int64_t)(lb + ll) * n + br + start + lane] : 0.0;
      __syncthreads();
      if (threadIdx.x < nl) {
        double dv = 0.0;
        for (int q = 0; q < tv; ++q) dv += tile[threadIdx.x * kLd + q] * vs[q];
        out[4 + l] = du;
        out[4 + a.max_rank + l] = dv;
      }
    }
  }
}

// Cross term of a wide node, spread over CTAs: CTA (c, node) takes l in [c kCrossL,
// (c + 1) kCrossL), each thread one l summing the tiles in item order, and folds
// (u_l.u)(v_l.v) over its l's (warp sums, then the warps in order) into cross_part.
__global__ void __launch_bounds__(kCrossL) k_aca_cross_wide(AcaArgs a, double* cross_part, int nchunk) {
  const int id = a.wide_nodes[blockIdx.y];
  if (a.done[id] || !a.phase[id] || a.rank[id] < kWideRank) return;
  const int k = a.rank[id];
  const int l = blockIdx.x * kCrossL + threadIdx.x;
  if (blockIdx.x * kCrossL >= k) return;
  const int i0 = a.node_witem0[id], i1 = a.node_witem1[id];
  double c = 0.0;
  if (l < k) {
    double du = 0.0, dv = 0.0;
    for (int it = i0; it < i1; ++it) {
      const double* p = a.part + (int64_t)it * a.part_stride;
      du += p[4 + l];
      dv += p[4 + a.max_rank + l];
    }
    c = du * dv;
  }
  __shared__ double red[kCrossL / 32];
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kCrossL / 32; ++q) s += red[q];
    cross_part[(int64_t)blockIdx.y * nchunk + blockIdx.x] = s;
  }
}

// D for a wide node: one warp; the argmax and norms as in k_aca_pivot_col, the cross term
// from k_aca_cross_wide's chunks in order.
__global__ void __launch_bounds__(32) k_aca_pivot_col_wide(AcaArgs a, const double* cross_part, int nchunk) {
  const int id = a.wide_nodes[blockIdx.x];
  if (a.done[id] || a.rank[id] < kWideRank) return;  // k_aca_pivot_col's node
  const int lane = threadIdx.x;
  if (!a.phase[id]) {
    if (lane == 0) atomicAdd(a.active, 1);
    return;
  }
  const int k = a.rank[id];
  const int i0 = a.node_witem0[id], i1 = a.node_witem1[id];
  double bv = 0.0, nu2 = 0.0, nv2 = 0.0;
  int bi = -1;
  for (int it = i0 + lane; it < i1; it += 32) {
    const double* p = a.part + (int64_t)it * a.part_stride;
    amax_merge(bv, bi, p[0], (int)p[1]);
    nu2 += p[2];
    nv2 += p[3];
  }
  warp_amax(bv, bi);
  nu2 = warp_sum(nu2);
  nv2 = warp_sum(nv2);
  if (lane != 0) return;
  double c = 0.0;
  for (int q = 0; q * kCrossL < k; ++q) c += cross_part[(int64_t)blockIdx.x * nchunk + q];
  col_decide(a, id, k, bi, nu2, nv2, c);
}

// Presized mode: flag every block that did not converge within its level's rank.
__global__ void k_aca_check(AcaArgs a, int32_t* flags) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.nint) return;
  int pre = a.pre[level_of(id)];
  int ml = a.ns[2 * id + 1], mr = a.ns[2 * id + 2];
  bool full = a.rank[id] >= (ml < mr ? ml : mr);  // the whole block: exact
  if (!a.done[id] || (!a.ok[id] && !full) || a.rank[id] > pre) atomicOr(flags, kFlagRankCap);
}

// Compact panels: level j's columns [coff_j, coff_j + r_j) of phi take the node's first
// rank columns of the raw panel and zeros beyond (zero columns leave every product of the
// factorization unchanged). The working panel is written by the leaf stage, which reads
// its columns from phi.
struct PackArgs {
  const double* raw;
  int64_t raw_off[32];
  int coff[33];
  int rl[32];
  const int32_t* nb;
  const int32_t* rank;
  double* phi;
  int64_t n;
};

__global__ void k_pack(PackArgs p) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= p.n) return;
  int id = 0;
  for (int l = 0; l < j; ++l) id = i < p.nb[2 * id + 2] ? 2 * id + 1 : 2 * id + 2;
  int r = p.rank[id];
  // 64-bit moves: the same code serves FP64 values and double-float pairs (all-zero bits
  // are 0 in both)
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p.raw + p.raw_off[j]);
  unsigned long long* phi = reinterpret_cast<unsigned long long*>(p.phi);
  for (int c = 0; c < p.rl[j]; ++c) {
    unsigned long long v = c < r ? src[c * p.n + i] : 0ull;
    phi[(int64_t)(p.coff[j] + c) * p.n + i] = v;
  }
}

}  // namespace

// Launch K<kFF, kGen> for the context's form (double-float or FP64) and case (gen: any d
// and kind; else the kernels specialised for d <= 2 and Table 1's covariances).
#define ACA_LAUNCH_T(K, grid, threads, smem, ...)                                    \
  do {                                                                               \
    if (c.precision == 1) {                                                          \
      if (gen)                                                                       \
        K<true, true><<<grid, threads, smem, c.stream>>>(__VA_ARGS__);               \
      else                                                                           \
        K<true, false><<<grid, threads, smem, c.stream>>>(__VA_ARGS__);              \
    } else {                                                                         \
      if (gen)                                                                       \
        K<false, true><<<grid, threads, smem, c.stream>>>(__VA_ARGS__);              \
      else                                                                           \
        K<false, false><<<grid, threads, smem, c.stream>>>(__VA_ARGS__);             \
    }                                                                                \
  } while (0)
#define ACA_LAUNCH(K, grid, smem, ...) ACA_LAUNCH_T(K, grid, kAcaThreads, smem, __VA_ARGS__)

cudaError_t launch_aca(Ctx& c, int* steps_out) {
  int nint = (1 << c.kappa) - 1;
  *steps_out = 0;
  if (nint == 0) return cudaSuccess;
  AcaArgs a;
  int maxpre = 0;
  for (int j = 0; j < 32; ++j) {
    a.pre[j] = (c.presized && j < c.kappa) ? std::max(c.h_rl[j], 1) : 0;
    maxpre = std::max(maxpre, a.pre[j]);
  }
  a.pts = Pts{c.xs, c.n, c.d};
  a.kind = c.kind;
  a.hyp = c.hyp;
  a.eps = c.eps;
  a.nb = c.nodes;
  a.ns = c.nodes + ((int64_t)2 << c.kappa);
  a.item_node = c.item_node;
  a.item_start = c.item_start;
  a.node_item0 = c.node_item0;
  a.node_item1 = c.node_item1;
  a.raw = c.raw;
  for (int j = 0; j < 32; ++j) a.raw_off[j] = j < c.kappa ? c.h_raw_off[j] : 0;
  a.rank = c.st_rank; a.row = c.st_row; a.col = c.st_col; a.done = c.st_done; a.ok = c.st_ok;
  a.zero = c.st_zero; a.phase = c.st_phase; a.nused = c.st_nused; a.used = c.st_used;
  a.used_stride = 2 * c.max_rank + 2;
  a.delta = c.st_delta; a.s2 = c.st_s2; a.part = c.aca_part;
  a.part_stride = 4 + 2 * c.max_rank;
  a.max_rank = c.max_rank;
  a.tab = reinterpret_cast<const ff*>(c.exp_tab);
  a.xrel = reinterpret_cast<const ff*>(c.xrel);
  a.active = c.active;
  a.nint = nint;
  a.node_witem0 = c.node_witem0;
  a.node_witem1 = c.node_witem1;
  a.wide_nodes = c.wide_nodes;
  k_aca_init<<<(nint + 255) / 256, 256, 0, c.stream>>>(a);
  ++c.launches;
  int wblocks = (nint * 32 + 255) / 256;
  const int64_t nbig = c.n_big_items, nwide = c.n_wide_items;
  const int nchunk = (c.max_rank + kCrossL - 1) / kCrossL;  // cross-term chunks per wide node
  const int64_t nsmall = c.n_items - nbig - nwide, small0 = nbig + nwide;
  const unsigned sgrid = (unsigned)((nsmall + kAcaThreads / 32 - 1) / (kAcaThreads / 32));
  const size_t smem_row = 0, smem_col = 0;  // static, independent of the rank
  // the wide column kernel's dot-product tile: kWideThreads columns of kWideTile + 1 doubles
  const size_t smem_wide = sizeof(double) * kWideThreads * (kWideTile + 1);
  if (nwide > 0) {
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_aca_col_wide<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wide));
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_aca_col_wide<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wide));
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_aca_col_wide<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wide));
    HODLR_CUDA_TRY(cudaFuncSetAttribute(k_aca_col_wide<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wide));
  }
  // adaptive: until no block is active (host check per step); presized: a fixed number of
  // steps (rank + 1 per block, one spare for a zero pivot) and a device-side check
  int max_steps = c.presized ? maxpre + 2 : 2 * c.max_rank + 4;
  // the specialised kernels cover points in one or two dimensions and Table 1's kernels
  const bool gen = c.d > 2 || c.kind > HODLR_K_MATERN52;
  for (int s = 0; s < max_steps; ++s) {
    if (!c.presized) HODLR_CUDA_TRY(cudaMemsetAsync(c.active, 0, sizeof(int32_t), c.stream));
    if (nbig > 0) {
      ACA_LAUNCH(k_aca_row, (unsigned)nbig, smem_row, a);
      ++c.launches;
    }
    const bool wide_step = nwide > 0 && s >= kWideRank;  // a rank grows by one per step at most
    if (wide_step) {
      ACA_LAUNCH_T(k_aca_row_wide, (unsigned)nwide, kWideThreads, 0, a, (int)nbig);
      ++c.launches;
    }
    if (nsmall > 0) {
      ACA_LAUNCH(k_aca_row_small, sgrid, 0, a, (int)small0, (int)nsmall);
      ++c.launches;
    }
    k_aca_pivot_row<<<wblocks, 256, 0, c.stream>>>(a);
    if (nbig > 0) {
      ACA_LAUNCH(k_aca_col, (unsigned)nbig, smem_col, a);
      ++c.launches;
    }
    if (wide_step) {
      ACA_LAUNCH_T(k_aca_col_wide, (unsigned)nwide, kWideThreads, smem_wide, a, (int)nbig);
      ++c.launches;
    }
    if (nsmall > 0) {
      ACA_LAUNCH(k_aca_col_small, sgrid, 0, a, (int)small0, (int)nsmall);
      ++c.launches;
    }
    k_aca_pivot_col<<<wblocks, 256, 0, c.stream>>>(a);
    if (wide_step) {
      k_aca_cross_wide<<<dim3((unsigned)nchunk, (unsigned)c.n_wide_nodes), kCrossL, 0, c.stream>>>(a, c.wide_cross, nchunk);
      k_aca_pivot_col_wide<<<(unsigned)c.n_wide_nodes, 32, 0, c.stream>>>(a, c.wide_cross, nchunk);
      c.launches += 2;
    }
    c.launches += 2;
    HODLR_CUDA_TRY(cudaGetLastError());
    *steps_out = s + 1;
    if (c.presized) continue;
    // the host looks at the active count after every step of the first 128, then after
    // every eighth (steps past the end change nothing: finished blocks skip every kernel)
    if (s >= 128 && (s & 7) != 7 && s + 1 < max_steps) continue;
    HODLR_CUDA_TRY(cudaMemcpyAsync(c.h_active, c.active, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    HODLR_CUDA_TRY(cudaStreamSynchronize(c.stream));
    ++c.syncs;
    if (*c.h_active == 0) break;
  }
  if (c.presized) {
    k_aca_check<<<(nint + 255) / 256, 256, 0, c.stream>>>(a, c.dflags);
    ++c.launches;
  }
  return cudaGetLastError();
}

namespace {
__global__ void k_exp_table(ff* tab) { ff_exp_table(tab, threadIdx.x, blockDim.x); }

// xrel[(j d + c) n + i] = x_c(i) - x_c(s), s the first point of the right child of i's
// level-j node, as a double-float (the one FP64 subtraction per point and level).
__global__ void k_xrel(const double* __restrict__ xs, int64_t n, int d, const int32_t* nb,
                       ff* __restrict__ xrel) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n) return;
  int id = 0;
  for (int l = 0; l < j; ++l) id = i < nb[2 * id + 2] ? 2 * id + 1 : 2 * id + 2;
  int64_t s = nb[2 * id + 2];
  for (int c = 0; c < d; ++c)
    xrel[((int64_t)j * d + c) * n + i] = ff_from_double(xs[c * n + i] - xs[c * n + s]);
}

}  // namespace

// Relative coordinates for the mixed form's ACA (once per context: they do not depend on
// the hyperparameters).
cudaError_t launch_xrel(Ctx& c) {
  if (c.kappa == 0) return cudaSuccess;
  dim3 g((unsigned)((c.n + 255) / 256), (unsigned)c.kappa);
  k_xrel<<<g, 256, 0, c.stream>>>(c.xs, c.n, c.d, c.nodes, reinterpret_cast<ff*>(c.xrel));
  ++c.launches;
  return cudaGetLastError();
}

// 2^(j/64), j < 64, as double-floats for the double-float exp (once per context).
cudaError_t launch_exp_table(Ctx& c) {
  k_exp_table<<<1, 64, 0, c.stream>>>(reinterpret_cast<ff*>(c.exp_tab));
  ++c.launches;
  return cudaGetLastError();
}

cudaError_t launch_pack(Ctx& c) {
  if (c.kappa == 0 || c.R == 0) return cudaSuccess;
  PackArgs p;
  p.raw = c.raw;
  for (int j = 0; j < 32; ++j) {
    p.raw_off[j] = j < c.kappa ? c.h_raw_off[j] : 0;
    p.rl[j] = j < c.kappa ? c.h_rl[j] : 0;
  }
  for (int j = 0; j < 33; ++j) p.coff[j] = j <= c.kappa ? c.h_coff[j] : 0;
  p.nb = c.nodes;
  p.rank = c.rank_dev;
  p.phi = c.phi;
  p.n = c.n;
  dim3 g((unsigned)((c.n + 255) / 256), (unsigned)c.kappa);
  k_pack<<<g, 256, 0, c.stream>>>(p);
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
