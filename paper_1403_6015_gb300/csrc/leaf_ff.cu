// Leaf stage in double-float arithmetic (the mixed-precision form of the factorization).
//
// Same work as k_leaf (Sec. 3.2: factor K_kappa out of C, applying each leaf inverse to the
// ancestors' U/V rows and to the right-hand sides; Sec. 4: leaf determinants), but every
// operation on the leaf block runs in double-float (ff.cuh) on the FP32 pipe. The panels
// (Phi and the U/V columns) enter and leave HBM as double-float pairs, the right-hand sides
// as FP64; the stored factor is kept as double-float pairs; the log of each pivot is taken
// in FP64. Unit roundoff ~2^-48 instead of 2^-53.
//
// Blocked for the FP32 pipe (one CTA per leaf, all of it in shared memory, two CTAs per
// SM so that one leaf's barriers overlap the other's work):
//   - only the lower triangle is kept, packed by rows (element (i, j), j <= i, at
//     i (i + 1) / 2 + j); the unscaled panel columns of the factorization and the solve
//     chunk share one buffer, which also holds the coordinates while the block is built;
//   - the block is padded to P = 32 ceil(p / 32) with the identity, which changes neither
//     the factor of the leading p x p block, the solutions, nor the log det;
//   - L D L^T by 32-column panels: inside a panel, two columns per step (three barriers
//     per pair; the next pair's first pivot is computed by the thread that updates it);
//     below it, the trailing matrix is updated in 2 x 2 register tiles (32-term dots);
//   - the panel columns and right-hand sides are solved in chunks of 32 columns held in
//     shared memory: 32 x 32 diagonal blocks by one warp per column, the rest as dense
//     updates with one thread per output element;
//   - the dot products (trailing update, solve updates, partial products) accumulate in
//     compensated form (ffacc: the error of each sum kept apart and added once at the end).
#include <cuda_runtime.h>

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kTri = kMaxLeaf * (kMaxLeaf + 1) / 2;  // packed lower triangle
constexpr int kBS = 33;            // row stride of the 32-column buffer
constexpr int kCW = 32;            // columns per solve chunk

// Offset of row i in the packed lower triangle.
__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

struct LeafFFArgs {
  const double* x;
  int64_t n;
  int d;
  int kind;
  const double* hyp;  // device hyperparameter slot (cr, amplitude, sigma^2)
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
  ff* leafL;          // stored factor: L below the diagonal, D on it (double-float pairs)
  const ff* tab;      // 2^(j/64) as double-floats
  double* leaf_logdet;
  int32_t* flags;
};

__device__ __forceinline__ ff shfl_ff(ff v, int src) {
  return ff{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ __forceinline__ ff xor_ff(ff v, int m) {
  return ff{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// Row of the lower-triangle element with linear index e (row-major, diagonal included).
__device__ __forceinline__ int tri_row(int e) {
  int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > e) --i;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  return i;
}

template <int kT, bool kFactor>
__global__ void __launch_bounds__(kT, 1024 / kT) k_leaf_ff(LeafFFArgs a) {
  extern __shared__ ff sm[];
  ff* A = sm;                          // packed lower triangle, kTri
  ff* Up = A + kTri;                   // [kMaxLeaf][kBS] unscaled panel columns (factor)
  ff* B = Up;                          // [kMaxLeaf][kBS] solve chunk (after the factor)
  ff* xl = Up;                         // d x kMaxLeaf coordinates (block build only)
  __shared__ ff dinv[kMaxLeaf];
  __shared__ ff tab[64];
  __shared__ ff pinv[2];
  __shared__ double red[kT / 32];
  __shared__ int bad;
  constexpr int NW = kT / 32;
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int P = (p + 31) & ~31, NB = P / 32;
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  ff* Lst = a.leafL + (int64_t)leaf * kMaxLeaf * kMaxLeaf;
  if (kFactor) {
    if (tid == 0) bad = 0;
    for (int q = tid; q < 64; q += kT) tab[q] = a.tab[q];
    // coordinates relative to the leaf's first point (keeps small offsets exact)
    for (int i = tid; i < p; i += kT) {
      for (int c = 0; c < a.d && c < 3; ++c)
        xl[c * kMaxLeaf + i] = ff_from_double(a.x[c * a.n + b + i] - a.x[c * a.n + b]);
    }
    __syncthreads();
    const CovFF cf = make_cov_ff(a.kind, a.hyp[kHypScale], a.hyp[kHypAmp], a.hyp[kHypAlpha]);
    const ff s2 = ff_from_double(a.hyp[kHypSigma2]);
    // lower triangle of the padded block
    for (int e = tid; e < P * (P + 1) / 2; e += kT) {
      int i = tri_row(e), j = e - i * (i + 1) / 2;
      ff c;
      if (i < p) {
        ff r;
        if (a.d == 1) {
          r = ff_sub(xl[i], xl[j]);
          if (r.hi < 0.0f) r = ff_neg(r);
        } else if (a.d <= 3) {
          ff u = ff_sub(xl[i], xl[j]), v = ff_sub(xl[kMaxLeaf + i], xl[kMaxLeaf + j]);
          ff s = ff_add(ff_mul(u, u), ff_mul(v, v));
          if (a.d == 3) {
            ff w = ff_sub(xl[2 * kMaxLeaf + i], xl[2 * kMaxLeaf + j]);
            s = ff_add(s, ff_mul(w, w));
          }
          r = ff_sqrt(s);
        } else {
          r = ff_from_double(dist(Pts{a.x, a.n, a.d}, b + i, b + j));  // d > 3: FP64 distance
        }
        c = cov_ff(cf, r, tab);
        if (i == j) c = ff_add(c, s2);
      } else {
        c = ff{i == j ? 1.0f : 0.0f, 0.0f};
      }
      A[e] = c;  // e = tri(i) + j
    }
    __syncthreads();
    // blocked L D L^T
    for (int J = 0; J < NB; ++J) {
      int c0 = 32 * J;
      if (tid == 0) {
        ff dk = A[tri(c0) + c0];
        if (!(dk.hi > 0.0f)) {
          bad = 1;
          dk = ff{1.0f, 0.0f};
          A[tri(c0) + c0] = dk;
        }
        pinv[0] = ff_rcp(dk);
      }
      __syncthreads();
      // panel, two columns (col, col + 1) per step: pinv[0] holds 1 / D_col on entry
      for (int c = 0; c < 32; c += 2) {
        int col = c0 + c;
        // the second pivot of the pair: D_{col+1} = A_{col+1,col+1} - L_{col+1,col} A_{col+1,col}
        if (tid == 0) {
          ff t = A[tri(col + 1) + col];
          ff l = ff_mul(t, pinv[0]);
          A[tri(col + 1) + col] = l;
          Up[(col + 1) * kBS + c] = t;
          ff d1 = ff_fms(A[tri(col + 1) + col + 1], l, t);
          if (!(d1.hi > 0.0f)) {
            bad = 1;
            d1 = ff{1.0f, 0.0f};
          }
          A[tri(col + 1) + col + 1] = d1;
          pinv[1] = ff_rcp(d1);
        }
        __syncthreads();
        // rows below the pair: scale both columns, keep the unscaled values
        ff iv0 = pinv[0], iv1 = pinv[1], t10 = Up[(col + 1) * kBS + c];
        for (int i = col + 2 + tid; i < P; i += kT) {
          ff t = A[tri(i) + col];
          ff l = ff_mul(t, iv0);
          A[tri(i) + col] = l;
          Up[i * kBS + c] = t;
          ff u = ff_fms(A[tri(i) + col + 1], l, t10);
          A[tri(i) + col + 1] = ff_mul(u, iv1);
          Up[i * kBS + c + 1] = u;
        }
        __syncthreads();
        // update the remaining panel columns cc in [c + 2, 32) on rows >= c0 + cc; warps
        // take columns, lanes take rows; the next pair's first pivot by its updater
        for (int cc = c + 2 + w; cc < 32; cc += NW) {
          int jc = c0 + cc;
          ff uj0 = Up[jc * kBS + c], uj1 = Up[jc * kBS + c + 1];
          for (int i = jc + lane; i < P; i += 32) {
            ffacc acc = ffacc_init(A[tri(i) + jc]);
            ffacc_fms(acc, A[tri(i) + col], uj0);
            ffacc_fms(acc, A[tri(i) + col + 1], uj1);
            ff v = ffacc_get(acc);
            if (i == jc && cc == c + 2) {
              if (!(v.hi > 0.0f)) {
                bad = 1;
                v = ff{1.0f, 0.0f};
              }
              pinv[0] = ff_rcp(v);
            }
            A[tri(i) + jc] = v;
          }
        }
        __syncthreads();
      }
      // trailing update of rows/columns [c0 + 32, P): A_ij -= sum_c L_ic U_jc, 2 x 2 tiles
      int r0 = c0 + 32;
      int M = (P - r0) / 2;
      for (int e = tid; e < M * (M + 1) / 2; e += kT) {
        int ti = tri_row(e), tj = e - ti * (ti + 1) / 2;
        int i0 = r0 + 2 * ti, j0 = r0 + 2 * tj;
        // two compensated accumulators per entry (the first starts from A_ij)
        const ff z = {0.0f, 0.0f};
        ffacc s00a = ffacc_init(A[tri(i0) + j0]), s10a = ffacc_init(A[tri(i0 + 1) + j0]);
        ffacc s11a = ffacc_init(A[tri(i0 + 1) + j0 + 1]);
        ffacc s01a = ffacc_init(ti != tj ? A[tri(i0) + j0 + 1] : z);  // above the diagonal if ti == tj
        ffacc s00b = ffacc_init(z), s01b = ffacc_init(z), s10b = ffacc_init(z), s11b = ffacc_init(z);
#pragma unroll 4
        for (int c = 0; c < 32; c += 2) {
          ff l0 = A[tri(i0) + c0 + c], l1 = A[tri(i0 + 1) + c0 + c];
          ff u0 = Up[j0 * kBS + c], u1 = Up[(j0 + 1) * kBS + c];
          ffacc_fms(s00a, l0, u0);
          ffacc_fms(s01a, l0, u1);
          ffacc_fms(s10a, l1, u0);
          ffacc_fms(s11a, l1, u1);
          ff m0 = A[tri(i0) + c0 + c + 1], m1 = A[tri(i0 + 1) + c0 + c + 1];
          ff v0 = Up[j0 * kBS + c + 1], v1 = Up[(j0 + 1) * kBS + c + 1];
          ffacc_fms(s00b, m0, v0);
          ffacc_fms(s01b, m0, v1);
          ffacc_fms(s10b, m1, v0);
          ffacc_fms(s11b, m1, v1);
        }
        A[tri(i0) + j0] = ffacc_get2(s00a, s00b);
        A[tri(i0 + 1) + j0] = ffacc_get2(s10a, s10b);
        A[tri(i0 + 1) + j0 + 1] = ffacc_get2(s11a, s11b);
        if (ti != tj) A[tri(i0) + j0 + 1] = ffacc_get2(s01a, s01b);
      }
      __syncthreads();
    }
    // store the factor (leading p x p lower triangle)
    for (int e = tid; e < p * (p + 1) / 2; e += kT) {
      int i = tri_row(e), j = e - i * (i + 1) / 2;
      Lst[i * kMaxLeaf + j] = A[tri(i) + j];
    }
  } else {
    for (int e = tid; e < P * (P + 1) / 2; e += kT) {
      int i = tri_row(e), j = e - i * (i + 1) / 2;
      A[tri(i) + j] = i < p ? Lst[i * kMaxLeaf + j] : ff{i == j ? 1.0f : 0.0f, 0.0f};
    }
    __syncthreads();
  }
  // log det = sum log D_ii (FP64), 1 / D
  double sl = 0.0;
  for (int i = tid; i < p; i += kT) {
    ff di = A[tri(i) + i];
    if (kFactor) sl += log(ff_to_double(di));
    dinv[i] = ff_rcp(di);
  }
  for (int i = p + tid; i < P; i += kT) dinv[i] = ff{1.0f, 0.0f};
  if (kFactor) {
    for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
    if (lane == 0) red[w] = sl;
  }
  __syncthreads();
  if (kFactor && tid == 0) {
    double t = 0.0;
    for (int q = 0; q < NW; ++q) t += red[q];
    a.leaf_logdet[leaf] = t;
    if (bad) atomicOr(a.flags, kFlagNotSpd);
  }
  // solves, 32 columns at a time: panel [0, cP) then right-hand sides [0, nrhs)
  int ncol = a.cP + a.nrhs;
  for (int q0 = 0; q0 < ncol; q0 += kCW) {
    int cw = ncol - q0 < kCW ? ncol - q0 : kCW;
    const ff* panf = reinterpret_cast<const ff*>(a.phi);  // panel columns read from Phi
    for (int e = tid; e < P * cw; e += kT) {
      int c = e / P, i = e - c * P;
      int q = q0 + c;
      ff v = {0.0f, 0.0f};
      if (i < p)
        v = q < a.cP ? panf[(int64_t)q * a.n + b + i] : ff_from_double(a.Y[(int64_t)(q - a.cP) * a.n + b + i]);
      B[i * kBS + c] = v;
    }
    __syncthreads();
    // forward: L w = b
    for (int J = 0; J < NB; ++J) {
      int c0 = 32 * J;
      for (int c = w; c < cw; c += NW) {
        ff xv = B[(c0 + lane) * kBS + c];
        for (int k = 0; k < 32; ++k) {
          ff xk = shfl_ff(xv, k);
          if (lane > k) xv = ff_fms(xv, A[tri(c0 + lane) + c0 + k], xk);
        }
        B[(c0 + lane) * kBS + c] = xv;
      }
      __syncthreads();
      int r0 = c0 + 32;
      for (int e = tid; e < (P - r0) * cw; e += kT) {
        int i = r0 + e / cw, c = e - (e / cw) * cw;
        ffacc sa = ffacc_init(B[i * kBS + c]), sb = ffacc_init(ff{0.0f, 0.0f});
#pragma unroll 4
        for (int k = 0; k < 32; k += 2) {
          ffacc_fms(sa, A[tri(i) + c0 + k], B[(c0 + k) * kBS + c]);
          ffacc_fms(sb, A[tri(i) + c0 + k + 1], B[(c0 + k + 1) * kBS + c]);
        }
        B[i * kBS + c] = ffacc_get2(sa, sb);
      }
      __syncthreads();
    }
    // v = D^-1 w
    for (int e = tid; e < P * cw; e += kT) {
      int i = e / cw, c = e - i * cw;
      B[i * kBS + c] = ff_mul(B[i * kBS + c], dinv[i]);
    }
    __syncthreads();
    // backward: L^T x = v
    for (int J = NB - 1; J >= 0; --J) {
      int c0 = 32 * J;
      for (int c = w; c < cw; c += NW) {
        ff xv = B[(c0 + lane) * kBS + c];
        for (int k = 31; k >= 0; --k) {
          ff xk = shfl_ff(xv, k);
          if (lane < k) xv = ff_fms(xv, A[tri(c0 + k) + c0 + lane], xk);
        }
        B[(c0 + lane) * kBS + c] = xv;
      }
      __syncthreads();
      for (int e = tid; e < c0 * cw; e += kT) {
        int i = e / cw, c = e - i * cw;
        ffacc sa = ffacc_init(B[i * kBS + c]), sb = ffacc_init(ff{0.0f, 0.0f});
#pragma unroll 4
        for (int k = 0; k < 32; k += 2) {
          ffacc_fms(sa, A[tri(c0 + k) + i], B[(c0 + k) * kBS + c]);
          ffacc_fms(sb, A[tri(c0 + k + 1) + i], B[(c0 + k + 1) * kBS + c]);
        }
        B[i * kBS + c] = ffacc_get2(sa, sb);
      }
      __syncthreads();
    }
    // write back (FP64) and the level-(kappa-1) partial products, one warp per (r, column)
    for (int e = tid; e < p * cw; e += kT) {
      int c = e / p, i = e - c * p;
      int q = q0 + c;
      if (q < a.cP)
        reinterpret_cast<ff*>(a.pan)[(int64_t)q * a.n + b + i] = B[i * kBS + c];
      else
        a.Y[(int64_t)(q - a.cP) * a.n + b + i] = ff_to_double(B[i * kBS + c]);
    }
    if (a.kappa > 0) {
      double* out = a.part + (int64_t)leaf * a.part_stride;
      for (int t = w; t < a.rl * cw; t += NW) {
        int r = t / cw, c = t - r * cw;
        const ff* ph = reinterpret_cast<const ff*>(a.phi) + (int64_t)(a.coff + r) * a.n + b;
        ffacc acc = ffacc_init(ff{0.0f, 0.0f});
        for (int i = lane; i < p; i += 32) ffacc_fma(acc, ph[i], B[i * kBS + c]);
        ff s = ffacc_get(acc);
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, xor_ff(s, o));
        if (lane == 0) out[r * ncol + q0 + c] = ff_to_double(s);
      }
    }
    __syncthreads();
  }
}

LeafFFArgs make_ff_args(Ctx& c, int nrhs, bool factor) {
  LeafFFArgs a;
  a.x = c.xs;
  a.n = c.n;
  a.d = c.d;
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
  a.leafL = reinterpret_cast<ff*>(c.leafL);
  a.tab = reinterpret_cast<const ff*>(c.exp_tab);
  a.leaf_logdet = c.leaf_logdet;
  a.flags = c.dflags;
  return a;
}

template <bool kFactor>
cudaError_t launch_ff(const LeafFFArgs& a, unsigned grid, int threads, cudaStream_t s) {
  size_t smem = sizeof(ff) * (kTri + kMaxLeaf * kBS);
  switch (threads) {
    case 512:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff<512, kFactor>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf_ff<512, kFactor><<<grid, 512, smem, s>>>(a);
      break;
    default:
      HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff<1024, kFactor>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_leaf_ff<1024, kFactor><<<grid, 1024, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_factor_ff(Ctx& c, int nrhs) {
  ++c.launches;
  return launch_ff<true>(make_ff_args(c, nrhs, true), 1u << c.kappa, c.leaf_threads, c.stream);
}

cudaError_t launch_leaf_solve_ff(Ctx& c, int nrhs) {
  ++c.launches;
  return launch_ff<false>(make_ff_args(c, nrhs, false), 1u << c.kappa, c.leaf_threads, c.stream);
}

}  // namespace hodlr
