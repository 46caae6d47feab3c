// Leaf stage in double-float arithmetic (the mixed-precision form of the factorization).
//
// Same work as k_leaf (Sec. 3.2: factor K_kappa out of C, applying each leaf inverse to the
// ancestors' U/V rows and to the right-hand sides; Sec. 4: leaf determinants), but every
// operation on the leaf block runs in double-float (ff.cuh) on the FP32 pipe: the block is
// built from the points with a double-float exp, factored as L D L^T, and applied to the
// panel columns. Values enter and leave HBM as FP64; the log of each pivot is taken in
// FP64. Unit roundoff ~2^-48 instead of 2^-53, at several times the FP64 throughput of
// GB300. If leafC is given, the assembled block of C is also stored (FP64) for the
// iterative-refinement residual.
#include <cuda_runtime.h>

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kLD = kMaxLeaf + 1;

struct LeafFFArgs {
  const double* x;
  int64_t n;
  int d;
  int kind;
  double cr;     // factor applied to r before f: 1/ell (exp, SE), sqrt3/ell, sqrt5/ell
  double amp, sigma2;
  const int32_t* nb;
  const int32_t* ns;
  int leaf0, kappa;
  double* pan;
  int cP;
  double* Y;
  int nrhs;
  const double* phi;
  int coff, rl;
  double* part;
  int64_t part_stride;
  double* leafL;
  double* leafC;
  double* leaf_logdet;
  int32_t* flags;
};

__device__ __forceinline__ ff cov_ff(int kind, ff r, ff cr, ff amp, const ff* tab) {
  ff s = ff_mul(r, cr);
  const ff one = {1.0f, 0.0f};
  switch (kind) {
    case HODLR_K_EXP:
      return ff_mul(amp, ff_exp(ff_neg(s), tab));
    case HODLR_K_SE:
      return ff_mul(amp, ff_exp(ff_mulf(ff_mul(s, s), -0.5f), tab));
    case HODLR_K_MATERN32:
      return ff_mul(amp, ff_mul(ff_add(one, s), ff_exp(ff_neg(s), tab)));
    default: {
      const ff third = {0.3333333432674408f, -9.934107481068821e-09f};
      ff poly = ff_add(ff_add(one, s), ff_mul(ff_mul(s, s), third));
      return ff_mul(amp, ff_mul(poly, ff_exp(ff_neg(s), tab)));
    }
  }
}

__device__ __forceinline__ ff shfl_ff(ff v, int src) {
  return ff{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ __forceinline__ ff wsum_ff(ff v) {
  for (int o = 16; o > 0; o >>= 1) {
    ff t = ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, t);
  }
  return v;
}

// L D L^T x = b for NC columns held by a warp (element i of column c in lane i % 32,
// slot i / 32); L unit lower below the diagonal of A, dinv = 1 / D.
template <int NC>
__device__ __forceinline__ void warp_ldl_solve_ff(const ff* __restrict__ A,
                                                  const ff* __restrict__ dinv, int p, int lane,
                                                  ff (&x)[NC][4]) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    for (int kk = 0; kk < 32; ++kk) {
      int k = s * 32 + kk;
      if (k >= p) break;
      ff wk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) wk[c] = shfl_ff(x[c][s], kk);
#pragma unroll
      for (int m = s; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i > k && i < p) {
          ff lik = A[i * kLD + k];
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c][m] = ff_fms(x[c][m], lik, wk[c]);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = m * 32 + lane;
    ff di = i < p ? dinv[i] : ff{0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c][m] = ff_mul(x[c][m], di);
  }
#pragma unroll
  for (int s = 3; s >= 0; --s) {
    for (int kk = 31; kk >= 0; --kk) {
      int k = s * 32 + kk;
      if (k >= p) continue;
      ff xk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) xk[c] = shfl_ff(x[c][s], kk);
#pragma unroll
      for (int m = 0; m <= s; ++m) {
        int i = m * 32 + lane;
        if (i < k) {
          ff lki = A[k * kLD + i];
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c][m] = ff_fms(x[c][m], lki, xk[c]);
        }
      }
    }
  }
}

template <int kT>
__global__ void __launch_bounds__(kT) k_leaf_ff(LeafFFArgs a) {
  extern __shared__ ff A[];  // [kMaxLeaf][kLD]
  __shared__ ff xl[2 * kMaxLeaf];
  __shared__ ff dinv[kMaxLeaf];
  __shared__ ff T0[kMaxLeaf], T1[kMaxLeaf];
  __shared__ ff tab[64];
  __shared__ double red[kT / 32];
  __shared__ ff piv_inv[2], piv_t;
  __shared__ int bad;
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) bad = 0;
  if (tid < 64) tab[tid] = ff_from_double(exp2((double)tid / 64.0));
  // coordinates relative to the leaf's first point: the FP64 subtraction keeps the small
  // offsets (and so the distances) to full relative precision in double-float
  for (int i = tid; i < p; i += kT) {
    xl[i] = ff_from_double(a.x[b + i] - a.x[b]);
    if (a.d == 2) xl[kMaxLeaf + i] = ff_from_double(a.x[a.n + b + i] - a.x[a.n + b]);
  }
  __syncthreads();
  const ff cr = ff_from_double(a.cr), amp = ff_from_double(a.amp), s2 = ff_from_double(a.sigma2);
  // lower triangle of the leaf block of C
  for (int e = tid; e < p * p; e += kT) {
    int i = e / p, j = e - i * p;
    if (j > i) continue;
    ff r;
    if (a.d == 1) {
      r = ff_sub(xl[i], xl[j]);
      if (r.hi < 0.0f) r = ff_neg(r);
    } else {
      ff u = ff_sub(xl[i], xl[j]), v = ff_sub(xl[kMaxLeaf + i], xl[kMaxLeaf + j]);
      ff q = ff_add(ff_mul(u, u), ff_mul(v, v));
      // sqrt in double-float: float sqrt refined by one Newton step
      float h = sqrtf(q.hi);
      if (h > 0.0f) {
        ff hh = ff_mul(ff{h, 0.0f}, ff{h, 0.0f});
        ff res = ff_sub(q, hh);
        r = ff_make(h, res.hi / (2.0f * h));
      } else {
        r = ff{0.0f, 0.0f};
      }
    }
    ff c = cov_ff(a.kind, r, cr, amp, tab);
    if (i == j) c = ff_add(c, s2);
    A[i * kLD + j] = c;
  }
  __syncthreads();
  if (a.leafC) {
    double* Cout = a.leafC + (int64_t)leaf * kMaxLeaf * kMaxLeaf;
    for (int e = tid; e < p * p; e += kT) {
      int i = e / p, j = e - i * p;
      Cout[i * kMaxLeaf + j] = ff_to_double(j <= i ? A[i * kLD + j] : A[j * kLD + i]);
    }
  }
  // L D L^T, two pivots per step (as in the FP64 leaf kernel)
  for (int k = 0; k < p; k += 2) {
    bool two = k + 1 < p;
    if (tid == 0) {
      ff dk = A[k * kLD + k];
      if (!(dk.hi > 0.0f)) {
        bad = 1;
        dk = ff{1.0f, 0.0f};
      }
      A[k * kLD + k] = dk;
      ff ik = ff_rcp(dk);
      piv_inv[0] = ik;
      if (two) {
        ff t = A[(k + 1) * kLD + k];
        ff l = ff_mul(t, ik);
        A[(k + 1) * kLD + k] = l;
        ff d1 = ff_fms(A[(k + 1) * kLD + k + 1], l, t);
        if (!(d1.hi > 0.0f)) {
          bad = 1;
          d1 = ff{1.0f, 0.0f};
        }
        A[(k + 1) * kLD + k + 1] = d1;
        piv_inv[1] = ff_rcp(d1);
        piv_t = t;
      }
    }
    __syncthreads();
    ff i0v = piv_inv[0];
    for (int i = k + 2 + tid; i < p; i += kT) {
      ff t = A[i * kLD + k];
      ff l = ff_mul(t, i0v);
      A[i * kLD + k] = l;
      T0[i] = t;
      if (two) {
        ff u = ff_fms(A[i * kLD + k + 1], l, piv_t);
        A[i * kLD + k + 1] = ff_mul(u, piv_inv[1]);
        T1[i] = u;
      }
    }
    __syncthreads();
    if (two) {
      for (int j = k + 2 + w; j < p; j += kT / 32) {
        ff t0 = T0[j], t1 = T1[j];
        for (int i = j + lane; i < p; i += 32) {
          ff v = A[i * kLD + j];
          v = ff_fms(v, A[i * kLD + k], t0);
          v = ff_fms(v, A[i * kLD + k + 1], t1);
          A[i * kLD + j] = v;
        }
      }
    }
    __syncthreads();
  }
  double* Lout = a.leafL + (int64_t)leaf * kMaxLeaf * kMaxLeaf;
  for (int e = tid; e < p * p; e += kT) {
    int i = e / p, j = e - i * p;
    if (j <= i) Lout[i * kMaxLeaf + j] = ff_to_double(A[i * kLD + j]);
  }
  double sl = 0.0;
  for (int i = tid; i < p; i += kT) sl += log(ff_to_double(A[i * kLD + i]));
  for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
  if (lane == 0) red[w] = sl;
  for (int i = tid; i < p; i += kT) dinv[i] = ff_rcp(A[i * kLD + i]);
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < kT / 32; ++q) t += red[q];
    a.leaf_logdet[leaf] = t;
    if (bad) atomicOr(a.flags, kFlagNotSpd);
  }
  int ncol = a.cP + a.nrhs;
  constexpr int NC = 2;
  for (int c0 = w * NC; c0 < ncol; c0 += NC * (kT / 32)) {
    double* col[NC];
    ff x[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      int cc = c0 + c < ncol ? c0 + c : c0;
      col[c] = cc < a.cP ? a.pan + (int64_t)cc * a.n + b : a.Y + (int64_t)(cc - a.cP) * a.n + b;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        x[c][m] = i < p ? ff_from_double(col[c][i]) : ff{0.0f, 0.0f};
      }
    }
    warp_ldl_solve_ff<NC>(A, dinv, p, lane, x);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c0 + c >= ncol) break;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) col[c][i] = ff_to_double(x[c][m]);
      }
    }
    if (a.kappa > 0) {
      double* out = a.part + (int64_t)leaf * a.part_stride;
      for (int r = 0; r < a.rl; ++r) {
        const double* ph = a.phi + (int64_t)(a.coff + r) * a.n + b;
        ff phv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          phv[m] = i < p ? ff_from_double(ph[i]) : ff{0.0f, 0.0f};
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (c0 + c >= ncol) break;
          ff s = {0.0f, 0.0f};
#pragma unroll
          for (int m = 0; m < 4; ++m) s = ff_fma(s, phv[m], x[c][m]);
          s = wsum_ff(s);
          if (lane == 0) out[r * ncol + c0 + c] = ff_to_double(s);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_leaf_factor_ff(Ctx& c, int nrhs, double* leafC) {
  LeafFFArgs a;
  a.x = c.xs;
  a.n = c.n;
  a.d = c.d;
  a.kind = c.kind;
  a.cr = (c.kind == HODLR_K_MATERN32 ? 1.7320508075688772 : c.kind == HODLR_K_MATERN52 ? 2.23606797749979 : 1.0) / c.ell;
  a.amp = c.amp;
  a.sigma2 = c.sigma2;
  a.nb = c.nodes;
  a.ns = c.nodes + ((int64_t)2 << c.kappa);
  a.leaf0 = (1 << c.kappa) - 1;
  a.kappa = c.kappa;
  a.pan = c.pan;
  a.cP = c.R;
  a.Y = c.Y;
  a.nrhs = nrhs;
  a.phi = c.phi;
  a.coff = c.kappa > 0 ? c.h_coff[c.kappa - 1] : 0;
  a.rl = c.kappa > 0 ? c.h_rl[c.kappa - 1] : 0;
  a.part = c.part;
  a.part_stride = c.part_stride;
  a.leafL = c.leafL;
  a.leafC = leafC;
  a.leaf_logdet = c.leaf_logdet;
  a.flags = c.dflags;
  size_t smem = sizeof(ff) * kMaxLeaf * kLD;
  unsigned grid = 1u << c.kappa;
  switch (c.leaf_threads) {
    case 1024:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf_ff<1024><<<grid, 1024, smem, c.stream>>>(a);
      break;
    case 256:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf_ff<256><<<grid, 256, smem, c.stream>>>(a);
      break;
    default:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf_ff<512><<<grid, 512, smem, c.stream>>>(a);
  }
  ++c.launches;
  return cudaGetLastError();
}

}  // namespace hodlr
