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
//     shared memory: 32 x 32 diagonal blocks by one warp per two columns (diag_fwd2,
//     diag_bwd2), the rest as dense updates with one thread per output element;
//   - the dot products (trailing update, solve updates, partial products) accumulate in
//     compensated form (ffacc: the error of each sum kept apart and added once at the end).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ff.cuh"
#include "hodlr_internal.cuh"
#include "tc.cuh"

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

// Unit lower 32 x 32 diagonal-block solves for two columns per warp: half h (lane / 16) of
// the warp holds column h of the pair, lane l = lane % 16 its rows l (top) and 16 + l
// (bottom). Forward (L w = b): a 16-step chain over the top rows whose every step also
// applies the new value to the 16 bottom rows (the dense 16 x 16 block, no idle lanes),
// then a 16-step chain over the bottom rows. Backward (L^T x = v) mirrors it. Each row
// receives its terms in the same order as a 32-step chain, so the results are the same,
// with half the critical path and a quarter fewer double-float operations.
template <class LF>
__device__ __forceinline__ void diag_fwd2(ff& top, ff& bot, int lane, LF L) {
  const int l = lane & 15, base = lane & 16;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    ff xk = shfl_ff(top, base + k);
    if (l > k) top = ff_fms(top, L(l, k), xk);
    bot = ff_fms(bot, L(16 + l, k), xk);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    ff xk = shfl_ff(bot, base + k);
    if (l > k) bot = ff_fms(bot, L(16 + l, 16 + k), xk);
  }
}

template <class LF>
__device__ __forceinline__ void diag_bwd2(ff& top, ff& bot, int lane, LF L) {
  const int l = lane & 15, base = lane & 16;
#pragma unroll
  for (int k = 15; k >= 0; --k) {
    ff xk = shfl_ff(bot, base + k);
    if (l < k) bot = ff_fms(bot, L(16 + k, 16 + l), xk);
    top = ff_fms(top, L(16 + k, l), xk);
  }
#pragma unroll
  for (int k = 15; k >= 0; --k) {
    ff xk = shfl_ff(top, base + k);
    if (l < k) top = ff_fms(top, L(k, l), xk);
  }
}

template <int kT, bool kFactor>
__device__ __forceinline__ void leaf_ff_body(const LeafFFArgs& a, int leaf) {
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
      for (int c2 = w; 2 * c2 < cw; c2 += NW) {
        const int c = 2 * c2 + (lane >> 4), l = lane & 15;  // c <= 31 < kBS: in bounds
        ff top = B[(c0 + l) * kBS + c], bot = B[(c0 + 16 + l) * kBS + c];
        diag_fwd2(top, bot, lane, [&](int i, int k) { return A[tri(c0 + i) + c0 + k]; });
        if (c < cw) {
          B[(c0 + l) * kBS + c] = top;
          B[(c0 + 16 + l) * kBS + c] = bot;
        }
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
      for (int c2 = w; 2 * c2 < cw; c2 += NW) {
        const int c = 2 * c2 + (lane >> 4), l = lane & 15;
        ff top = B[(c0 + l) * kBS + c], bot = B[(c0 + 16 + l) * kBS + c];
        diag_bwd2(top, bot, lane, [&](int i, int k) { return A[tri(c0 + i) + c0 + k]; });
        if (c < cw) {
          B[(c0 + l) * kBS + c] = top;
          B[(c0 + 16 + l) * kBS + c] = bot;
        }
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

template <int kT, bool kFactor>
__global__ void __launch_bounds__(kT, 1024 / kT) k_leaf_ff(LeafFFArgs a) {
  leaf_ff_body<kT, kFactor>(a, blockIdx.x);
}

// Persistent factor launch over the leaves of many problems (batched evaluation): every
// CTA takes work items (problem, leaf) from a device counter until all are done; item t
// belongs to the problem whose first item, first[problem], is the largest <= t.
template <int kT>
__global__ void __launch_bounds__(kT, 1024 / kT) k_leaf_ff_multi(const LeafFFArgs* __restrict__ args,
                                                                const int32_t* __restrict__ first,
                                                                int nprob, int32_t* counter) {
  __shared__ int item_s;
  const int total = first[nprob];
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();  // every thread has read the item before thread 0 takes the next
    if (item >= total) break;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    leaf_ff_body<kT, true>(args[lo], item - first[lo]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// The same leaf stage with its GEMM-shaped updates on the tensor cores (tcgen05, tc.cuh).
//
// What runs where (one CTA of 512 threads per leaf, two CTAs per SM, 256 columns of tensor
// memory each):
//   - the block build, the 32-column panels of L D L^T and the 32 x 32 diagonal-block
//     solves: double-float on the FP32 pipe, as in k_leaf_ff;
//   - the trailing update after each panel, A22 -= L21 D L21^T = G G^T with
//     G = L21 D^(1/2) (D > 0 for an SPD block), and the off-diagonal block updates of the
//     forward and backward solves, X_below -= L_IJ X_J and X_above -= L_JI^T X_J: exact
//     products of bf16 slices on the tensor cores (seven slices per operand, six FP32
//     accumulators per output in tensor memory), subtracted from the double-float target
//     in one compensated sum: double-float accuracy, as the compensated dot products of
//     k_leaf_ff.
// Shared memory (109,056 bytes dynamic):
//   R1 (43,008 B)  the left-operand slices: 7 slices of up to 96 rows x K = 32 (G in the
//                  factor phase, blocks of L in the solves); the M = 128 MMA also reads
//                  32 rows past the 96th of each slice (the next slice, or the start of R0
//                  after the last one), whose outputs are never read;
//   R0 (66,048 B)  factor phase: the packed lower triangle A (double-float); solve phase:
//                  the 32-column chunk X [128][33], the slices of X_J (7 x 2,048 B) and
//                  the diagonal block L_JJ [32][33].
// In the solve phase the blocks of L come back from the stored factor (global memory,
// written by this CTA just before and still in L2), which frees R0 for the chunk.
constexpr int kTcRows = 96;                                  // left-operand rows (<= P - 32)
constexpr uint32_t kTcSliceA = tc::slice_bytes(kTcRows);     // 6,144 B per slice
constexpr uint32_t kTcSliceX = tc::slice_bytes(32);          // 2,048 B per slice
constexpr size_t kTcR1 = tc::kSlices * kTcSliceA;            // 43,008 B
constexpr size_t kTcR0 = sizeof(ff) * kTri;                  // 66,048 B
constexpr size_t kTcSmem = kTcR1 + kTcR0;                    // 109,056 B
constexpr size_t kTcXBytes = sizeof(ff) * kMaxLeaf * kBS;    // 33,792 B
constexpr int kTcCols = 256;                                 // tensor-memory columns per CTA
constexpr int kTcPolls = 50000;                              // mbarrier polls (<= 1 s) before giving up
static_assert(kTcXBytes + tc::kSlices * kTcSliceX + sizeof(ff) * 32 * kBS <= kTcR0,
              "solve-phase buffers must fit in R0");
static_assert(32 * tc::kAcc <= kTcCols, "accumulators of one 32-column tile");
static_assert(kTcR1 + 512 <= kTcSmem, "the MMA's reads past R1 stay in shared memory");

// D_a (+)= sum over s + t = L with acc_of(L) = a of A_s B_t^T, K = 32 (two K = 16 steps),
// into tensor-memory columns tm + 32 a, for every level L < kSlices. A: M = 128 rows from
// a_base (slices a_stride bytes apart, core matrices along K a_lbo apart); B: N = 32 rows
// from b_base. One thread issues; descriptors differ only in their address field.
__device__ __forceinline__ void tc_levels(uint32_t tm, uint32_t a_base, uint32_t a_stride,
                                          uint32_t a_lbo, uint32_t b_base, uint32_t b_stride,
                                          uint32_t b_lbo) {
  constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
  const uint64_t a0 = tc::sdesc(a_base, a_lbo, 128), b0 = tc::sdesc(b_base, b_lbo, 128);
#pragma unroll 1
  for (int L = 0; L < tc::kSlices; ++L) {
    const uint32_t d = tm + 32 * tc::acc_of(L);
    const bool first = L < tc::kAcc;  // the first level of its accumulator
#pragma unroll 1
    for (int s = 0; s <= L; ++s) {
      int t = L - s;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint64_t ad = a0 + ((s * a_stride + 2 * h * a_lbo) >> 4);
        uint64_t bd = b0 + ((t * b_stride + 2 * h * b_lbo) >> 4);
        tc::mma_bf16(d, ad, bd, idesc, !(first && s == 0 && h == 0));
      }
    }
  }
}

// Read the kAcc accumulators of this warp's 32 rows (tensor-memory lanes 32 (w % 4) ..)
// and 8 columns (8 (w / 4) ..) and pass each output's accumulators (exact FP32 values still
// to be scaled by 2^(e_row + e_col)) to f(row, col, d). Rows outside [lo, hi) are
// skipped; a warp none of whose rows is in range skips the loads as a whole.
template <class F>
__device__ __forceinline__ void tc_drain(uint32_t tm, int w, int lane, int lo, int hi, F&& f) {
  int lq = w & 3, cg = w >> 2;
  if (32 * lq >= hi || 32 * lq + 32 <= lo) return;
  int i = 32 * lq + lane;
  uint32_t base = tm + ((uint32_t)(32 * lq) << 16) + 8 * cg;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float d[tc::kAcc][4];
#pragma unroll
    for (int q = 0; q < tc::kAcc; ++q) tc::tmem_ld4(base + 32 * q + 4 * half, d[q]);
    if (i >= lo && i < hi) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        float lv[tc::kAcc];
#pragma unroll
        for (int q = 0; q < tc::kAcc; ++q) lv[q] = d[q][jj];
        f(i, 8 * cg + 4 * half + jj, lv);
      }
    }
  }
}

// Slice one operand row: this thread holds 8 consecutive values (k = 8 q .. 8 q + 7) of
// row r, the four lanes lane, lane ^ 8, lane ^ 16, lane ^ 24 the whole row. The row's
// bound exponent e (|v| < 2^e) is reduced over them; slice s of v 2^-e goes to
// base + s * stride + slice_off(R, r, 8 q) when store is set. Returns e.
__device__ __forceinline__ int tc_slice_row(ff* v, int q, unsigned char* base, uint32_t stride,
                                            int R, int r, bool store) {
  float mx = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) mx = fmaxf(mx, fabsf(v[k].hi));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
  int e = tc::bound_exp(mx);
  if (store) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = tc::ff_ldexp(v[k], -e);
    uint4 out[tc::kSlices];
    tc::cut8(v, out);
    uint32_t off = tc::slice_off(R, r, 8 * q);
#pragma unroll
    for (int s = 0; s < tc::kSlices; ++s)
      *reinterpret_cast<uint4*>(base + s * stride + off) = out[s];
  }
  return e;
}

__global__ void __launch_bounds__(512, 2) k_leaf_tc(LeafFFArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int kT = 512, NW = kT / 32;
  unsigned char* R1 = smraw;                                     // left-operand slices
  unsigned char* R0 = smraw + kTcR1;
  ff* A = reinterpret_cast<ff*>(R0);                             // factor phase
  ff* xl = reinterpret_cast<ff*>(R1);                            // coordinates (block build)
  ff* X = reinterpret_cast<ff*>(R0);                             // solve phase [128][kBS]
  unsigned char* Xs = R0 + kTcXBytes;                            // slices of X_J
  ff* LJJ = reinterpret_cast<ff*>(Xs + tc::kSlices * kTcSliceX);  // [32][kBS]
  __shared__ ff dinv[kMaxLeaf];
  __shared__ ff tab[64];
  __shared__ ff pinv[2];
  __shared__ ff upc[32][2];   // unscaled values of the current column pair, panel rows
  __shared__ ff sqd[32];      // D^(1/2) of the current panel
  __shared__ int exA[kMaxLeaf];
  __shared__ int exB[32];
  __shared__ double red[NW];
  __shared__ int bad, tc_fail;
  __shared__ uint32_t fail_parity;
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  int leaf = blockIdx.x;
  int id = a.leaf0 + leaf;
  int b = a.nb[id], p = a.ns[id];
  int P = (p + 31) & ~31, NB = P / 32;
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  ff* Lst = a.leafL + (int64_t)leaf * kMaxLeaf * kMaxLeaf;
  const ff zero = {0.0f, 0.0f};
  uint32_t phase = 0;

  if (tid == 0) {
    bad = 0;
    tc_fail = 0;
    tc::mbar_init(&bar, 1);
  }
  if (w == 0) tc::tmem_alloc(&tslot, kTcCols);
  for (int q = tid; q < 64; q += kT) tab[q] = a.tab[q];
  for (int i = tid; i < p; i += kT) {
    for (int c = 0; c < a.d && c < 3; ++c)
      xl[c * kMaxLeaf + i] = ff_from_double(a.x[c * a.n + b + i] - a.x[c * a.n + b]);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = tslot;
  const uint32_t aR1 = tc::smem_addr(R1), aXs = tc::smem_addr(Xs);
  // one MMA round: issue, wait (bounded), then every thread may drain
  auto mma_round = [&](uint32_t b_base, uint32_t b_stride, uint32_t b_lbo) {
    if (tid == 0 && !tc_fail) {
      tc_levels(tm, aR1, kTcSliceA, kTcRows * 16, b_base, b_stride, b_lbo);
      tc::mma_commit(&bar);
    }
    if (!tc_fail && !tc::mbar_wait(&bar, phase, kTcPolls)) {
      fail_parity = phase;  // the round still in flight
      tc_fail = 1;
    }
    phase ^= 1;
    tc::fence_after_sync();
  };
  auto round_sync = [&]() {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };

  {
    const CovFF cf = make_cov_ff(a.kind, a.hyp[kHypScale], a.hyp[kHypAmp], a.hyp[kHypAlpha]);
    const ff s2 = ff_from_double(a.hyp[kHypSigma2]);
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
            ff t = ff_sub(xl[2 * kMaxLeaf + i], xl[2 * kMaxLeaf + j]);
            s = ff_add(s, ff_mul(t, t));
          }
          r = ff_sqrt(s);
        } else {
          r = ff_from_double(dist(Pts{a.x, a.n, a.d}, b + i, b + j));
        }
        c = cov_ff(cf, r, tab);
        if (i == j) c = ff_add(c, s2);
      } else {
        c = ff{i == j ? 1.0f : 0.0f, 0.0f};
      }
      A[e] = c;
    }
  }
  __syncthreads();
  // blocked L D L^T: panels on the FP32 pipe, trailing updates on the tensor cores
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
    for (int c = 0; c < 32; c += 2) {
      int col = c0 + c;
      if (tid == 0) {
        ff t = A[tri(col + 1) + col];
        ff l = ff_mul(t, pinv[0]);
        A[tri(col + 1) + col] = l;
        upc[c + 1][0] = t;
        ff d1 = ff_fms(A[tri(col + 1) + col + 1], l, t);
        if (!(d1.hi > 0.0f)) {
          bad = 1;
          d1 = ff{1.0f, 0.0f};
        }
        A[tri(col + 1) + col + 1] = d1;
        pinv[1] = ff_rcp(d1);
      }
      __syncthreads();
      ff iv0 = pinv[0], iv1 = pinv[1], t10 = upc[c + 1][0];
      for (int i = col + 2 + tid; i < P; i += kT) {
        ff t = A[tri(i) + col];
        ff l = ff_mul(t, iv0);
        A[tri(i) + col] = l;
        ff u = ff_fms(A[tri(i) + col + 1], l, t10);
        A[tri(i) + col + 1] = ff_mul(u, iv1);
        if (i < c0 + 32) {
          upc[i - c0][0] = t;
          upc[i - c0][1] = u;
        }
      }
      __syncthreads();
      for (int cc = c + 2 + w; cc < 32; cc += NW) {
        int jc = c0 + cc;
        ff uj0 = upc[cc][0], uj1 = upc[cc][1];
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
    int r0 = c0 + 32;
    if (r0 < P) {
      int m = P - r0;
      if (tid < 32) sqd[tid] = ff_sqrt(A[tri(c0 + tid) + c0 + tid]);
      __syncthreads();
      if (8 * w < m) {  // G = L21 D^(1/2), rows 8 w + (lane % 8), k = 8 (lane / 8) .. + 7
        int r = 8 * w + (lane & 7), q = lane >> 3;
        ff v[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          v[kk] = r < m ? ff_mul(A[tri(r0 + r) + c0 + 8 * q + kk], sqd[8 * q + kk]) : zero;
        int e = tc_slice_row(v, q, R1, kTcSliceA, kTcRows, r, true);
        if (q == 0) exA[r] = e;
      }
      tc::fence_async_smem();
      round_sync();
      for (int nt = 0; nt < m / 32; ++nt) {
        mma_round(aR1 + 4 * nt * 128, kTcSliceA, kTcRows * 16);
        tc_drain(tm, w, lane, 32 * nt, m, [&](int i, int j, const float* d) {
          int jg = 32 * nt + j;
          if (jg <= i) {
            ff* dst = &A[tri(r0 + i) + r0 + jg];
            *dst = tc::sub_acc(*dst, d, exA[i] + exA[jg]);
          }
        });
        round_sync();
      }
    }
  }
  // store the factor (leading p x p lower triangle), log det, 1 / D
  for (int e = tid; e < p * (p + 1) / 2; e += kT) {
    int i = tri_row(e), j = e - i * (i + 1) / 2;
    Lst[i * kMaxLeaf + j] = A[tri(i) + j];
  }
  double sl = 0.0;
  for (int i = tid; i < p; i += kT) {
    ff di = A[tri(i) + i];
    sl += log(ff_to_double(di));
    dinv[i] = ff_rcp(di);
  }
  for (int i = p + tid; i < P; i += kT) dinv[i] = ff{1.0f, 0.0f};
  for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
  if (lane == 0) red[w] = sl;
  __syncthreads();  // A is not read after this point (R0 becomes the solve chunk)
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < NW; ++q) t += red[q];
    a.leaf_logdet[leaf] = t;
    if (bad) atomicOr(a.flags, kFlagNotSpd);
  }
  // solves, 32 columns at a time: panel [0, cP) then right-hand sides [0, nrhs)
  int ncol = a.cP + a.nrhs;
  const ff* panf = reinterpret_cast<const ff*>(a.phi);
  for (int q0 = 0; q0 < ncol; q0 += kCW) {
    int cw = ncol - q0 < kCW ? ncol - q0 : kCW;
    for (int e = tid; e < P * kCW; e += kT) {
      int c = e / P, i = e - c * P;
      int q = q0 + c;
      ff v = zero;
      if (i < p && c < cw)
        v = q < a.cP ? panf[(int64_t)q * a.n + b + i] : ff_from_double(a.Y[(int64_t)(q - a.cP) * a.n + b + i]);
      X[i * kBS + c] = v;
    }
    // forward: L w = b
    for (int J = 0; J < NB; ++J) {
      int c0 = 32 * J, r0 = c0 + 32, m = P - r0;
      for (int e = tid; e < 32 * 32; e += kT) {
        int i = e >> 5, k = e & 31;
        LJJ[i * kBS + k] = (k < i && c0 + i < p) ? Lst[(c0 + i) * kMaxLeaf + c0 + k] : zero;
      }
      __syncthreads();
      for (int c2 = w; 2 * c2 < cw; c2 += NW) {
        const int c = 2 * c2 + (lane >> 4), l = lane & 15;
        ff top = X[(c0 + l) * kBS + c], bot = X[(c0 + 16 + l) * kBS + c];
        diag_fwd2(top, bot, lane, [&](int i, int k) { return LJJ[i * kBS + k]; });
        if (c < cw) {
          X[(c0 + l) * kBS + c] = top;
          X[(c0 + 16 + l) * kBS + c] = bot;
        }
      }
      __syncthreads();
      if (m > 0) {
        if (w < 4) {  // X_J: operand row = chunk column c, k = row c0 + k
          int c = 8 * w + (lane & 7), q = lane >> 3;
          ff v[8];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) v[kk] = c < cw ? X[(c0 + 8 * q + kk) * kBS + c] : zero;
          int e = tc_slice_row(v, q, Xs, kTcSliceX, 32, c, true);
          if (q == 0) exB[c] = e;
        } else if (8 * (w - 4) < m) {  // L rows r0 + r below the block, columns c0 + k
          int r = 8 * (w - 4) + (lane & 7), q = lane >> 3;
          int gi = r0 + r;
          ff v[8];
          if (r < m && gi < p) {
            const float4* src = reinterpret_cast<const float4*>(Lst + gi * kMaxLeaf + c0 + 8 * q);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float4 t = src[u];
              v[2 * u] = ff{t.x, t.y};
              v[2 * u + 1] = ff{t.z, t.w};
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) v[kk] = zero;
          }
          int e = tc_slice_row(v, q, R1, kTcSliceA, kTcRows, r, true);
          if (q == 0) exA[r] = e;
        }
        tc::fence_async_smem();
        round_sync();
        mma_round(aXs, kTcSliceX, 32 * 16);
        tc_drain(tm, w, lane, 0, m, [&](int i, int j, const float* d) {
          if (j < cw) {
            ff* dst = &X[(r0 + i) * kBS + j];
            *dst = tc::sub_acc(*dst, d, exA[i] + exB[j]);
          }
        });
        round_sync();
      }
    }
    // v = D^-1 w
    for (int e = tid; e < P * cw; e += kT) {
      int i = e / cw, c = e - i * cw;
      X[i * kBS + c] = ff_mul(X[i * kBS + c], dinv[i]);
    }
    __syncthreads();
    // backward: L^T x = v
    for (int J = NB - 1; J >= 0; --J) {
      int c0 = 32 * J;
      for (int e = tid; e < 32 * 32; e += kT) {
        int i = e >> 5, k = e & 31;
        LJJ[i * kBS + k] = (k < i && c0 + i < p) ? Lst[(c0 + i) * kMaxLeaf + c0 + k] : zero;
      }
      __syncthreads();
      for (int c2 = w; 2 * c2 < cw; c2 += NW) {
        const int c = 2 * c2 + (lane >> 4), l = lane & 15;
        ff top = X[(c0 + l) * kBS + c], bot = X[(c0 + 16 + l) * kBS + c];
        diag_bwd2(top, bot, lane, [&](int i, int k) { return LJJ[i * kBS + k]; });
        if (c < cw) {
          X[(c0 + l) * kBS + c] = top;
          X[(c0 + 16 + l) * kBS + c] = bot;
        }
      }
      __syncthreads();
      if (c0 > 0) {
        if (w < 4) {
          int c = 8 * w + (lane & 7), q = lane >> 3;
          ff v[8];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) v[kk] = c < cw ? X[(c0 + 8 * q + kk) * kBS + c] : zero;
          int e = tc_slice_row(v, q, Xs, kTcSliceX, 32, c, true);
          if (q == 0) exB[c] = e;
        } else if (8 * (w - 4) < c0) {  // operand row i = column i < c0 of L, k = row c0 + k
          int r = 8 * (w - 4) + (lane & 7), q = lane >> 3;
          ff v[8];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            int gk = c0 + 8 * q + kk;
            v[kk] = (r < c0 && gk < p) ? Lst[gk * kMaxLeaf + r] : zero;
          }
          int e = tc_slice_row(v, q, R1, kTcSliceA, kTcRows, r, true);
          if (q == 0) exA[r] = e;
        }
        tc::fence_async_smem();
        round_sync();
        mma_round(aXs, kTcSliceX, 32 * 16);
        tc_drain(tm, w, lane, 0, c0, [&](int i, int j, const float* d) {
          if (j < cw) {
            ff* dst = &X[i * kBS + j];
            *dst = tc::sub_acc(*dst, d, exA[i] + exB[j]);
          }
        });
        round_sync();
      }
    }
    // write back (FP64) and the level-(kappa-1) partial products, one warp per (r, column)
    for (int e = tid; e < p * cw; e += kT) {
      int c = e / p, i = e - c * p;
      int q = q0 + c;
      if (q < a.cP)
        reinterpret_cast<ff*>(a.pan)[(int64_t)q * a.n + b + i] = X[i * kBS + c];
      else
        a.Y[(int64_t)(q - a.cP) * a.n + b + i] = ff_to_double(X[i * kBS + c]);
    }
    if (a.kappa > 0) {
      double* out = a.part + (int64_t)leaf * a.part_stride;
      for (int t = w; t < a.rl * cw; t += NW) {
        int r = t / cw, c = t - r * cw;
        const ff* ph = panf + (int64_t)(a.coff + r) * a.n + b;
        ffacc acc = ffacc_init(zero);
        for (int i = lane; i < p; i += 32) ffacc_fma(acc, ph[i], X[i * kBS + c]);
        ff s = ffacc_get(acc);
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, xor_ff(s, o));
        if (lane == 0) out[r * ncol + q0 + c] = ff_to_double(s);
      }
    }
    __syncthreads();
  }
  // release the tensor memory; after a wait that gave up, wait once more (bounded) for the
  // MMAs still in flight before freeing what they write
  round_sync();
  if (tc_fail) {
    tc::mbar_wait(&bar, fail_parity, kTcPolls);
    if (tid == 0) atomicOr(a.flags, kFlagTimeout);
  }
  if (w == 0) tc::tmem_dealloc(tm, kTcCols);
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

cudaError_t launch_tc(const LeafFFArgs& a, unsigned grid, cudaStream_t s) {
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  k_leaf_tc<<<grid, 512, kTcSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t leaf_args_bytes_ff() { return sizeof(LeafFFArgs); }

void leaf_args_fill_ff(Ctx& c, int nrhs, void* out) {
  LeafFFArgs a = make_ff_args(c, nrhs, true);
  memcpy(out, &a, sizeof(a));
}

cudaError_t launch_leaf_factor_multi_ff(const void* args, const int32_t* first, int nprob,
                                        int total, int32_t* counter, int sms, cudaStream_t s) {
  size_t smem = sizeof(ff) * (kTri + kMaxLeaf * kBS);
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_leaf_ff_multi<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned grid = (unsigned)std::min(total, 2 * sms);
  if (grid == 0) return cudaSuccess;
  k_leaf_ff_multi<512><<<grid, 512, smem, s>>>(static_cast<const LeafFFArgs*>(args), first, nprob, counter);
  return cudaGetLastError();
}

cudaError_t launch_leaf_factor_ff(Ctx& c, int nrhs) {
  ++c.launches;
  if (c.leaf_tc) return launch_tc(make_ff_args(c, nrhs, true), 1u << c.kappa, c.stream);
  return launch_ff<true>(make_ff_args(c, nrhs, true), 1u << c.kappa, c.leaf_threads, c.stream);
}

cudaError_t launch_leaf_solve_ff(Ctx& c, int nrhs) {
  ++c.launches;
  return launch_ff<false>(make_ff_args(c, nrhs, false), 1u << c.kappa, c.leaf_threads, c.stream);
}

}  // namespace hodlr
