// Leaf stage of the factorization (Sec. 3.2: factoring K_kappa, the block diagonal of dense
// leaf blocks, out of C applies each leaf inverse to the rows of every ancestor's U/V that
// lie in the leaf; Sec. 4: the leaf determinants enter log det C).
//
// One CTA per leaf, 256 threads, the leaf block in shared memory (row-major, stride 129):
//   factor mode: build C[I_leaf, I_leaf] from the sorted points (sigma^2 on the diagonal),
//                factor it in place as L D L^T (the square-root-free Cholesky form, L unit
//                lower, two pivots per step), store it, log det = sum log D_ii;
//                for an indefinite C (multiquadric, biharmonic) instead P A = L D U~ (LU
//                with partial pivoting, U = D U~ with U~ unit upper), the row order P
//                stored beside it, log |det| = sum log |D_ii| and the sign from the row
//                swaps and the signs of D_ii;
//   solve mode:  load the stored factor.
// Then every panel column (the ancestors' U/V rows in factor mode, and the right-hand sides)
// is solved by one warp, two columns at a time (L D L^T: one column per 16-lane half, lanes
// own rows l + 16 m; LU: both columns in all lanes, rows lane + 32 m; unit triangular
// factors make every step one shuffle and FMAs), and the warp also forms the
// level-(kappa-1) partial products Phi_{kappa-1}^T x of the leaf's rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kLD = kMaxLeaf + 1;

struct LeafArgs {
  Pts pts;
  int kind;
  const double* hyp;  // device hyperparameter slot
  const int32_t* nb;
  const int32_t* ns;
  int leaf0;          // node id of leaf 0
  int kappa;
  double* pan;        // n x R working panel (factor mode: cP = R columns processed)
  int cP;             // panel columns to solve
  double* Y;          // n x nrhs right-hand sides (sorted order)
  int nrhs;
  const double* phi;  // originals, for the partial of level kappa-1
  int coff;           // column offset of level kappa-1 in phi
  int rl;             // r_{kappa-1}
  double* part;       // partial products, leaf-major
  int64_t part_stride;
  double* leafL;
  double* leaf_logdet;
  int32_t* leaf_perm;  // LU row order, kMaxLeaf per leaf (lu only)
  int lu;              // 1: LU with partial pivoting (indefinite C), 0: L D L^T
  int32_t* flags;
  int64_t n;
};

// Row of the lower-triangle element with linear index e (row-major, diagonal included).
__device__ __forceinline__ int tri_row(int e) {
  int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > e) --i;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  return i;
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Solve L D V x = b for NC columns held by a warp: element i of column c in lane i % 32,
// slot i / 32 of x[c]. L is unit lower (below the diagonal of A), dinv holds 1 / D_ii and
// V is unit upper: L^T (kUpper = false, read from below the diagonal) or the scaled LU
// factor U~ (kUpper = true, above the diagonal).
template <int NC, bool kUpper>
__device__ __forceinline__ void warp_ldl_solve(const double* __restrict__ A,
                                               const double* __restrict__ dinv, int p, int lane,
                                               double (&x)[NC][4]) {
  // forward: L w = b
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    for (int kk = 0; kk < 32; ++kk) {
      int k = s * 32 + kk;
      if (k >= p) break;
      double wk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) wk[c] = __shfl_sync(0xffffffffu, x[c][s], kk);
#pragma unroll
      for (int m = s; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i > k && i < p) {
          double lik = A[i * kLD + k];
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c][m] -= lik * wk[c];
        }
      }
    }
  }
  // v = D^-1 w
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = m * 32 + lane;
    double di = i < p ? dinv[i] : 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c][m] *= di;
  }
  // backward: V x = v
#pragma unroll
  for (int s = 3; s >= 0; --s) {
    for (int kk = 31; kk >= 0; --kk) {
      int k = s * 32 + kk;
      if (k >= p) continue;
      double xk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) xk[c] = __shfl_sync(0xffffffffu, x[c][s], kk);
#pragma unroll
      for (int m = 0; m <= s; ++m) {
        int i = m * 32 + lane;
        if (i < k) {
          double lki = kUpper ? A[i * kLD + k] : A[k * kLD + i];
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c][m] -= lki * xk[c];
        }
      }
    }
  }
}

// The same solve with L^T (L D L^T factor) for two columns per warp, one per 16-lane half:
// lane l = lane % 16 of half h holds rows 16 j + l (j = 0..7) of column h in x[j]. Every
// 16-row diagonal chunk leaves at most 15 of a half's lanes idle per step (instead of 31
// of 32), and one shuffle serves one column instead of two.
__device__ __forceinline__ void half_ldl_solve(const double* __restrict__ A,
                                               const double* __restrict__ dinv, int p, int lane,
                                               double (&x)[8]) {
  const int l = lane & 15, base = lane & 16;
  // forward: L w = b
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    for (int kk = 0; kk < 16; ++kk) {
      int k = s * 16 + kk;
      if (k >= p) break;
      double wk = __shfl_sync(0xffffffffu, x[s], base + kk);
#pragma unroll
      for (int m = s; m < 8; ++m) {
        int i = m * 16 + l;
        if (i > k && i < p) x[m] -= A[i * kLD + k] * wk;
      }
    }
  }
  // v = D^-1 w
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    int i = m * 16 + l;
    x[m] *= i < p ? dinv[i] : 0.0;
  }
  // backward: L^T x = v
#pragma unroll
  for (int s = 7; s >= 0; --s) {
    for (int kk = 15; kk >= 0; --kk) {
      int k = s * 16 + kk;
      if (k >= p) continue;
      double xk = __shfl_sync(0xffffffffu, x[s], base + kk);
#pragma unroll
      for (int m = 0; m <= s; ++m) {
        int i = m * 16 + l;
        if (i < k) x[m] -= A[k * kLD + i] * xk;
      }
    }
  }
}

// In-place LU with partial pivoting of the p x p block in A (stride kLD), right-looking:
// at step k warp 0 picks the row of largest |A_ik|, i >= k (lowest index on ties), the
// rows are swapped, and every warp updates its rows of the trailing block with its own
// multiplier. On exit L (unit lower) is below the diagonal, D = diag(U) on it and
// U~ = D^-1 U above it; perm[i] = original row now at position i; *nswap = row swaps;
// *bad = 1 if a pivot was exactly zero (it is replaced by 1 to keep going).
template <int kThreads>
__device__ void lu_factor(double* A, int p, int* perm, int* prow, int* nswap, int* bad) {
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < p; i += kThreads) perm[i] = i;
  if (tid == 0) *nswap = 0;
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    if (w == 0) {
      double bv = -1.0;
      int bi = k;
      for (int i = k + lane; i < p; i += 32) {
        double v = fabs(A[i * kLD + k]);
        if (v > bv) {  // rows are visited in increasing order: ties keep the lower one
          bv = v;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        *prow = bi;
        if (bi != k) {
          int t = perm[k];
          perm[k] = perm[bi];
          perm[bi] = t;
          ++*nswap;
        }
      }
    }
    __syncthreads();
    int pr = *prow;
    if (pr != k)
      for (int j = tid; j < p; j += kThreads) {
        double t = A[k * kLD + j];
        A[k * kLD + j] = A[pr * kLD + j];
        A[pr * kLD + j] = t;
      }
    __syncthreads();
    double akk = A[k * kLD + k];
    if (akk == 0.0) {
      akk = 1.0;
      if (tid == 0) {
        *bad = 1;
        A[k * kLD + k] = 1.0;
      }
    }
    const double inv = 1.0 / akk;
    for (int i = k + 1 + w; i < p; i += kThreads / 32) {
      double l = A[i * kLD + k] * inv;
      __syncwarp();
      for (int j = k + 1 + lane; j < p; j += 32) A[i * kLD + j] -= l * A[k * kLD + j];
      if (lane == 0) A[i * kLD + k] = l;
    }
    __syncthreads();
  }
  // U~ = D^-1 U: scale each row above the diagonal by 1 / D_ii
  for (int i = w; i < p; i += kThreads / 32) {
    double inv = 1.0 / A[i * kLD + i];
    for (int j = i + 1 + lane; j < p; j += 32) A[i * kLD + j] *= inv;
  }
  __syncthreads();
}

template <bool kFactor, int kLeafThreads>
__device__ __forceinline__ void leaf_body(const LeafArgs& a, int leaf) {
  extern __shared__ double A[];  // [kMaxLeaf][kLD]
  __shared__ double xl[3 * kMaxLeaf];
  __shared__ double dinv[kMaxLeaf];
  __shared__ double T0[kMaxLeaf], T1[kMaxLeaf];
  __shared__ double red[kLeafThreads / 32];
  __shared__ double piv_inv[2], piv_t;
  __shared__ int bad;
  __shared__ int perm[kMaxLeaf];
  __shared__ int prow, nswap;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double* Lout = a.leafL + (int64_t)leaf * kMaxLeaf * kMaxLeaf;
  if (kFactor) {
    const Cov cov = cov_from(a.kind, a.hyp);
    const double sigma2 = a.hyp[kHypSigma2];
    if (tid == 0) bad = 0;
    for (int i = tid; i < p; i += kLeafThreads) {
      for (int c = 0; c < a.pts.d && c < 3; ++c) xl[c * kMaxLeaf + i] = a.pts.x[c * a.pts.n + b + i];
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += kLeafThreads) {
      int i = e / p, j = e - i * p;
      if (j > i && !a.lu) continue;
      double r;
      if (a.pts.d == 1) {
        r = fabs(xl[i] - xl[j]);
      } else {
        double u = xl[i] - xl[j], v = xl[kMaxLeaf + i] - xl[kMaxLeaf + j];
        if (a.pts.d == 2) {
          r = sqrt(u * u + v * v);
        } else if (a.pts.d == 3) {
          double w = xl[2 * kMaxLeaf + i] - xl[2 * kMaxLeaf + j];
          r = sqrt(u * u + v * v + w * w);
        } else {
          r = dist(a.pts, b + i, b + j);  // d > 3: coordinates from global memory
        }
      }
      double c = cov_r(cov, r);
      if (i == j) c += sigma2;
      A[i * kLD + j] = c;
    }
    __syncthreads();
    if (a.lu) {
      lu_factor<kLeafThreads>(A, p, perm, &prow, &nswap, &bad);
      int32_t* pout = a.leaf_perm + (int64_t)leaf * kMaxLeaf;
      for (int e = tid; e < p * p; e += kLeafThreads) {
        int i = e / p, j = e - i * p;
        Lout[i * kMaxLeaf + j] = A[i * kLD + j];
      }
      for (int i = tid; i < p; i += kLeafThreads) pout[i] = perm[i];
      // log |det| = sum log |D_ii|; sign = (-1)^(row swaps) times the signs of D_ii
      double s = 0.0;
      int neg = 0;
      for (int i = tid; i < p; i += kLeafThreads) {
        double dii = A[i * kLD + i];
        s += log(fabs(dii));
        neg += dii < 0.0;
      }
      s = wsum(s);
      neg = __reduce_add_sync(0xffffffffu, neg);
      if (lane == 0) {
        red[w] = s;
        T0[w] = (double)neg;
      }
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        int ng = nswap;
        for (int q = 0; q < kLeafThreads / 32; ++q) {
          t += red[q];
          ng += (int)T0[q];
        }
        a.leaf_logdet[leaf] = t;
        if (bad) atomicOr(a.flags, kFlagNotSpd);
        if (ng & 1) atomicXor(a.flags, kFlagNegDet);
      }
    } else {
    // L D L^T, right-looking, pivots k and k+1 per step: on exit A[i][j] (j < i) = L_ij and
    // A[k][k] = D_kk. The trailing update uses the unscaled columns kept in T0, T1:
    // A_ij -= L_ik (L_jk D_kk) + L_i,k+1 (L_j,k+1 D_k+1,k+1).
    for (int k = 0; k < p; k += 2) {
      bool two = k + 1 < p;
      if (tid == 0) {
        double dk = A[k * kLD + k];
        if (!(dk > 0.0)) {
          bad = 1;
          dk = 1.0;
        }
        A[k * kLD + k] = dk;
        double ik = 1.0 / dk;
        piv_inv[0] = ik;
        if (two) {
          double t = A[(k + 1) * kLD + k];
          double l = t * ik;
          A[(k + 1) * kLD + k] = l;
          double d1 = A[(k + 1) * kLD + k + 1] - l * t;
          if (!(d1 > 0.0)) {
            bad = 1;
            d1 = 1.0;
          }
          A[(k + 1) * kLD + k + 1] = d1;
          piv_inv[1] = 1.0 / d1;
          piv_t = t;
        }
      }
      __syncthreads();
      double i0v = piv_inv[0];
      for (int i = k + 2 + tid; i < p; i += kLeafThreads) {
        double t = A[i * kLD + k];
        double l = t * i0v;
        A[i * kLD + k] = l;
        T0[i] = t;
        if (two) {
          double u = A[i * kLD + k + 1] - l * piv_t;
          A[i * kLD + k + 1] = u * piv_inv[1];
          T1[i] = u;
        }
      }
      __syncthreads();
      if (two) {
        // the trailing lower triangle (rows and columns >= k + 2) flattened over all
        // threads, element e at row tri_row(e): no idle lanes but in the last pass
        const int m = p - k - 2;
        for (int e = tid; e < m * (m + 1) / 2; e += kLeafThreads) {
          int ii = tri_row(e), jj = e - ii * (ii + 1) / 2;
          int i = k + 2 + ii, j = k + 2 + jj;
          double v = A[i * kLD + j];
          v -= A[i * kLD + k] * T0[j];
          v -= A[i * kLD + k + 1] * T1[j];
          A[i * kLD + j] = v;
        }
      }
      __syncthreads();
    }
    // store the factor (L below the diagonal, D on it; row-major, stride kMaxLeaf)
    for (int e = tid; e < p * p; e += kLeafThreads) {
      int i = e / p, j = e - i * p;
      if (j <= i) Lout[i * kMaxLeaf + j] = A[i * kLD + j];
    }
    // log det = sum log D_ii, fixed order
    double s = 0.0;
    for (int i = tid; i < p; i += kLeafThreads) s += log(A[i * kLD + i]);
    s = wsum(s);
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < kLeafThreads / 32; ++q) t += red[q];
      a.leaf_logdet[leaf] = t;
      if (bad) atomicOr(a.flags, kFlagNotSpd);
    }
    }  // L D L^T
  } else {
    for (int e = tid; e < p * p; e += kLeafThreads) {
      int i = e / p, j = e - i * p;
      if (j <= i || a.lu) A[i * kLD + j] = Lout[i * kMaxLeaf + j];
    }
    if (a.lu)
      for (int i = tid; i < p; i += kLeafThreads) perm[i] = a.leaf_perm[(int64_t)leaf * kMaxLeaf + i];
    __syncthreads();
  }
  for (int i = tid; i < p; i += kLeafThreads) dinv[i] = 1.0 / A[i * kLD + i];
  __syncthreads();
  // columns: panel [0, cP) then right-hand sides [0, nrhs), two per warp at a time
  int ncol = a.cP + a.nrhs;
  int wtot = ncol;  // partial row width
  constexpr int NC = 2;
  if (!a.lu) {
    // L D L^T: two columns per warp in the half-warp layout (half_ldl_solve)
    const int l = lane & 15;
    for (int c0 = w * 2; c0 < ncol; c0 += 2 * (kLeafThreads / 32)) {
      const int c = c0 + (lane >> 4);
      const bool valid = c < ncol;
      const int cc = valid ? c : c0;  // a missing second column repeats the first
      double* col = cc < a.cP ? a.pan + (int64_t)cc * a.n + b : a.Y + (int64_t)(cc - a.cP) * a.n + b;
      const double* src = cc < a.cP ? a.phi + (int64_t)cc * a.n + b : col;
      double x[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        int i = m * 16 + l;
        x[m] = i < p ? src[i] : 0.0;
      }
      half_ldl_solve(A, dinv, p, lane, x);
      if (valid) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          int i = m * 16 + l;
          if (i < p) col[i] = x[m];
        }
      }
      if (a.kappa > 0) {
        double* out = a.part + (int64_t)leaf * a.part_stride;
        for (int r = 0; r < a.rl; ++r) {
          const double* ph = a.phi + (int64_t)(a.coff + r) * a.n + b;
          double sum = 0.0;
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            int i = m * 16 + l;
            if (i < p) sum += ph[i] * x[m];
          }
          for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (l == 0 && valid) out[r * wtot + c] = sum;
        }
      }
    }
    return;
  }
  for (int c0 = w * NC; c0 < ncol; c0 += NC * (kLeafThreads / 32)) {
    double* col[NC];
    double x[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      int cc = c0 + c < ncol ? c0 + c : c0;  // a missing second column repeats the first
      // panel columns are read from Phi (the packed U/V) and written, solved, to the panel
      col[c] = cc < a.cP ? a.pan + (int64_t)cc * a.n + b : a.Y + (int64_t)(cc - a.cP) * a.n + b;
      const double* src = cc < a.cP ? a.phi + (int64_t)cc * a.n + b : col[c];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        x[c][m] = i < p ? src[a.lu ? perm[i] : i] : 0.0;  // LU: rows in pivot order
      }
    }
    warp_ldl_solve<NC, true>(A, dinv, p, lane, x);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c0 + c >= ncol) break;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int i = m * 32 + lane;
        if (i < p) col[c][i] = x[c][m];
      }
    }
    if (a.kappa > 0) {
      double* out = a.part + (int64_t)leaf * a.part_stride;
      for (int r = 0; r < a.rl; ++r) {
        const double* ph = a.phi + (int64_t)(a.coff + r) * a.n + b;
        double phv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          int i = m * 32 + lane;
          phv[m] = i < p ? ph[i] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (c0 + c >= ncol) break;
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < 4; ++m) s += phv[m] * x[c][m];
          s = wsum(s);
          if (lane == 0) out[r * wtot + c0 + c] = s;
        }
      }
    }
  }
}

template <bool kFactor, int kLeafThreads>
__global__ void __launch_bounds__(kLeafThreads) k_leaf(LeafArgs a) {
  leaf_body<kFactor, kLeafThreads>(a, blockIdx.x);
}

// Persistent factor launch over the leaves of many problems (batched evaluation): every
// CTA takes work items (problem, leaf) from a device counter until all are done; item t
// belongs to the problem whose first item, first[problem], is the largest <= t.
template <int kLeafThreads>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_multi(const LeafArgs* __restrict__ args,
                                                            const int32_t* __restrict__ first,
                                                            int nprob, int32_t* counter) {
  __shared__ int item_s;
  const int total = first[nprob];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= total) break;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    leaf_body<true, kLeafThreads>(args[lo], item - first[lo]);
    __syncthreads();
  }
}

LeafArgs make_args(Ctx& c, int nrhs, bool factor) {
  LeafArgs a;
  a.pts = Pts{c.xs, c.n, c.d};
  a.kind = c.kind;
  a.hyp = c.hyp;
  a.nb = c.nodes;
  a.ns = c.nodes + ((int64_t)2 << c.kappa);
  a.leaf0 = (1 << c.kappa) - 1;
  a.kappa = c.kappa;
  a.pan = c.pan;
  a.cP = factor ? c.R : 0;
  a.Y = c.Y;
  a.nrhs = nrhs;
  a.phi = c.phi;
  a.coff = c.kappa > 0 ? c.h_coff[c.kappa - 1] : 0;
  a.rl = c.kappa > 0 ? c.h_rl[c.kappa - 1] : 0;
  a.part = c.part;
  a.part_stride = c.part_stride;
  a.leafL = c.leafL;
  a.leaf_logdet = c.leaf_logdet;
  a.leaf_perm = c.leaf_perm;
  a.lu = c.indefinite ? 1 : 0;
  a.flags = c.dflags;
  a.n = c.n;
  return a;
}

}  // namespace

template <bool kFactor>
cudaError_t launch_leaf(const LeafArgs& a, unsigned grid, int threads, cudaStream_t s) {
  size_t smem = sizeof(double) * kMaxLeaf * kLD;
  switch (threads) {
    case 1024:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf<kFactor, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf<kFactor, 1024><<<grid, 1024, smem, s>>>(a);
      break;
    case 512:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf<kFactor, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf<kFactor, 512><<<grid, 512, smem, s>>>(a);
      break;
    default:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf<kFactor, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf<kFactor, 256><<<grid, 256, smem, s>>>(a);
  }
  return cudaGetLastError();
}

size_t leaf_args_bytes() { return sizeof(LeafArgs); }

void leaf_args_fill(Ctx& c, int nrhs, void* out) {
  LeafArgs a = make_args(c, nrhs, true);
  memcpy(out, &a, sizeof(a));
}

cudaError_t launch_leaf_factor_multi(const void* args, const int32_t* first, int nprob, int total,
                                     int32_t* counter, int sms, cudaStream_t s) {
  size_t smem = sizeof(double) * kMaxLeaf * kLD;
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_multi<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned grid = (unsigned)std::min(total, sms);
  if (grid == 0) return cudaSuccess;
  k_leaf_multi<512><<<grid, 512, smem, s>>>(static_cast<const LeafArgs*>(args), first, nprob, counter);
  return cudaGetLastError();
}

cudaError_t launch_leaf_factor(Ctx& c, int nrhs) {
  LeafArgs a = make_args(c, nrhs, true);
  ++c.launches;
  return launch_leaf<true>(a, 1u << c.kappa, c.leaf_threads64, c.stream);
}

cudaError_t launch_leaf_solve(Ctx& c, int nrhs) {
  LeafArgs a = make_args(c, nrhs, false);
  ++c.launches;
  return launch_leaf<false>(a, 1u << c.kappa, c.leaf_threads64, c.stream);
}

}  // namespace hodlr

namespace hodlr {

// The leaf kernel on caller-provided device buffers, for a problem that is a single leaf
// (kappa = 0): nodes[0] = 0 (begin), nodes[1] = n (size); Y holds the right-hand side and
// receives C^-1 y; L receives the Cholesky factor; logdet receives log det C.
cudaError_t launch_leaf_single(const double* xs_soa, int n, int d, int kind, const double* hyp,
                               const int32_t* nodes, double* Y, double* L, double* logdet,
                               int32_t* flags, cudaStream_t s) {
  LeafArgs a;
  a.pts = Pts{xs_soa, n, d};
  a.kind = kind;
  a.hyp = hyp;
  a.nb = nodes;
  a.ns = nodes + 1;
  a.leaf0 = 0;
  a.kappa = 0;
  a.pan = nullptr;
  a.cP = 0;
  a.Y = Y;
  a.nrhs = 1;
  a.phi = nullptr;
  a.coff = 0;
  a.rl = 0;
  a.part = nullptr;
  a.part_stride = 0;
  a.leafL = L;
  a.leaf_logdet = logdet;
  a.leaf_perm = nullptr;
  a.lu = 0;
  a.flags = flags;
  a.n = n;
  return launch_leaf<true>(a, 1, 256, s);
}

}  // namespace hodlr
