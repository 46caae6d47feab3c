// Levels with large ranks (Sec. 3.2 when the off-diagonal blocks need ranks in the hundreds
// or thousands, as in the three-dimensional and d-dimensional Gaussian tables of Sec. 5,
// where the top blocks are nearly of full rank). The operations are those of levels.cu and
// node_solve.cuh, written as blocked dense linear algebra spread over the whole GPU:
//   node step  M = [I, V^T Vt; U^T Ut, I] (2r x 2r per node, row-major in global memory),
//              LU with partial pivoting by panels of kNB columns:
//                k_lu_panel  the panel's columns; the rows are split over several CTAs
//                            that meet at a grid barrier once per column (cooperative
//                            launch, bounded waits)
//                k_lu_rows   the panel's row swaps on every other column, and the block
//                            row U12 = L11^-1 A12
//                k_gemm      the trailing update A22 -= L21 U12
//              log|det M| and its sign from U's diagonal and the pivots (Sylvester's
//              theorem, Sec. 4), then Z = M^-1 [V^T P_R; U^T P_L] by blocked forward and
//              back substitution (k_z_fill applies the pivots, k_z_diag solves a diagonal
//              block, k_gemm updates the rows below or above it).
//   sweep      the level-u update P -= Ut Z (k_gemm, one product per half of a level-u
//              node: its rows share one block of Z), then the half-node sums Phi_{u-1}^T P
//              of the next level as one product per half-node (k_gemm over the half-node's
//              rows), in place of per-leaf partials and their segmented sums.
// All arithmetic is FP64, also in the mixed form (its double-float panels are converted on
// load and store), and every sum runs in a fixed order: results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "ff.cuh"
#include "hodlr_internal.cuh"
#include "node_solve.cuh"

namespace hodlr {
namespace {

// ---- batched FP64 product C (-)= A B --------------------------------------------------
constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

enum GemmMode : int {
  kUniform = 0,   // problem t at fixed offsets t * a_bs, t * b_bs, t * c_bs
  kNodeRows = 1,  // problem t = node id0 + t: rows nb[id0 + t] .. + ns[id0 + t] of A and C;
                  // B = the Z block of its ancestor (t >> sh) and side ((t >> (sh - 1)) & 1)
  kHalfRows = 2   // problem t = half-node t: the sum runs over its rows nb[id0 + t] ..
};

// Element (i, k) of A at a[i * ai + k * ak], (k, j) of B at b[k * bk + j * bj], (i, j) of C
// at c[i * ci + j * cj], after the problem's offset.
struct GemmArgs {
  const void* a;
  const void* b;
  void* c;
  int64_t ai, ak, bk, bj, ci, cj;
  int m, n, k;              // kNodeRows: m is the problem's node size; kHalfRows: k likewise
  int mode;
  int64_t a_bs, b_bs, c_bs;
  const int32_t* nb;
  const int32_t* ns;
  int id0;
  int sh;                   // kNodeRows: problems per Z block's node = 2^sh
  int64_t z_stride, z_side; // kNodeRows: Z of node (t >> sh), side ((t >> (sh-1)) & 1)
  int ksplit;               // kHalfRows: blockIdx.z = t ksplit + s, split s summing rows
  int kchunk;               // [s kchunk, (s + 1) kchunk) of the half-node into its own C
};

__device__ __forceinline__ double ldv(const double* p, int64_t i) { return p[i]; }
__device__ __forceinline__ double ldv(const ff* p, int64_t i) { return ff_to_double(p[i]); }
__device__ __forceinline__ void stv(double* p, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ void stv(ff* p, int64_t i, double v) { p[i] = ff_from_double(v); }

// 64 x 64 tile of one problem per CTA (blockIdx.z = problem), 4 x 4 outputs per thread,
// K in chunks of 16 staged in shared memory. Each output sums its K products in index order
// and is then subtracted from C (kSub) or stored.
template <class TA, class TB, class TC, bool kSub>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g) {
  int t = blockIdx.z;
  int m = g.m, K = g.k;
  int64_t oa = (int64_t)t * g.a_bs, ob = (int64_t)t * g.b_bs, oc = (int64_t)t * g.c_bs;
  if (g.mode == kNodeRows) {
    const int id = g.id0 + t;
    const int b = g.nb[id];
    m = g.ns[id];
    oa = b;
    oc = b;
    ob = (int64_t)(t >> g.sh) * g.z_stride + (int64_t)((t >> (g.sh - 1)) & 1) * g.z_side;
  } else if (g.mode == kHalfRows) {
    const int sp = t % g.ksplit;  // C = problem slot t ksplit + sp (its own partial sum)
    t /= g.ksplit;
    const int id = g.id0 + t;
    const int b = g.nb[id] + sp * g.kchunk;
    K = min(g.kchunk, g.ns[id] - sp * g.kchunk);
    oa = b;
    ob = b;
    oc = (int64_t)blockIdx.z * g.c_bs;
  }
  const int i0 = blockIdx.y * kBM, j0 = blockIdx.x * kBN;
  if (i0 >= m || j0 >= g.n) return;
  const TA* A = static_cast<const TA*>(g.a) + oa;
  const TB* B = static_cast<const TB*>(g.b) + ob;
  TC* C = static_cast<TC*>(g.c) + oc;
  __shared__ double As[kBK][kBM];
  __shared__ double Bs[kBK][kBN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;
  const bool a_kfast = g.ak == 1, b_kfast = g.bk == 1;
  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int e = threadIdx.x; e < kBM * kBK; e += kGemmThreads) {
      int ii, kk;
      if (a_kfast) {
        ii = e / kBK;
        kk = e - ii * kBK;
      } else {
        kk = e / kBM;
        ii = e - kk * kBM;
      }
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < m && gk < K) ? ldv(A, gi * g.ai + gk * g.ak) : 0.0;
    }
    for (int e = threadIdx.x; e < kBK * kBN; e += kGemmThreads) {
      int jj, kk;
      if (b_kfast) {
        jj = e / kBK;
        kk = e - jj * kBK;
      } else {
        kk = e / kBN;
        jj = e - kk * kBN;
      }
      const int gj = j0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < g.n && gk < K) ? ldv(B, gk * g.bk + gj * g.bj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= m) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + tx + 16 * q;
      if (gj >= g.n) continue;
      const int64_t idx = gi * g.ci + gj * g.cj;
      stv(C, idx, kSub ? ldv(C, idx) - acc[r][q] : acc[r][q]);
    }
  }
}

template <class TA, class TB, class TC, bool kSub>
cudaError_t gemm(const GemmArgs& g, int mmax, int batches, cudaStream_t s) {
  if (g.n <= 0 || mmax <= 0 || batches <= 0) return cudaSuccess;
  if (batches > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((g.n + kBN - 1) / kBN), (unsigned)((mmax + kBM - 1) / kBM), (unsigned)batches);
  k_gemm<TA, TB, TC, kSub><<<grid, kGemmThreads, 0, s>>>(g);
  return cudaGetLastError();
}

GemmArgs gemm_uniform(const void* a, int64_t ai, int64_t ak, int64_t a_bs, const void* b,
                      int64_t bk, int64_t bj, int64_t b_bs, void* c, int64_t ci, int64_t cj,
                      int64_t c_bs, int m, int n, int k) {
  GemmArgs g{};
  g.a = a; g.ai = ai; g.ak = ak; g.a_bs = a_bs;
  g.b = b; g.bk = bk; g.bj = bj; g.b_bs = b_bs;
  g.c = c; g.ci = ci; g.cj = cj; g.c_bs = c_bs;
  g.m = m; g.n = n; g.k = k;
  g.mode = kUniform;
  return g;
}

// ---- node matrix ----------------------------------------------------------------------
// M of node t (row-major, m2 = 2r): identity blocks on the diagonal, V^T Vt top right and
// U^T Ut bottom left, from the half-node sums (left half at 2t, right half at 2t + 1, each
// r x w row-major, the node's own panel columns starting at column cj).
__global__ void k_m_build(NodeArgs a, int64_t m_bs) {
  const int t = blockIdx.y;
  const int r = a.r, m2 = 2 * r;
  const double* L = a.half + (int64_t)(2 * t) * a.stride;
  const double* Rt = a.half + (int64_t)(2 * t + 1) * a.stride;
  double* M = a.Mlu + (int64_t)t * m_bs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m2 * m2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / m2), col = (int)(e - (int64_t)row * m2);
    double v;
    if ((row < r) == (col < r)) v = row == col ? 1.0 : 0.0;
    else if (row < r) v = __ldcg(Rt + (int64_t)row * a.w + a.cj + (col - r));  // V^T Vt
    else v = __ldcg(L + (int64_t)(row - r) * a.w + a.cj + col);                 // U^T Ut
    M[e] = v;
  }
}


// ---- LU panel: rows over several CTAs, one grid barrier per column --------------------
constexpr int kNB = 32;             // panel width (columns per panel)
constexpr int kPanelThreads = 256;  // one thread per row of the CTA's share
constexpr int kPanelRows = 256;     // largest share of rows per CTA
constexpr int kSlot = kNB + 2;      // published candidate: |value|, row, the row's kNB entries
constexpr long long kBarrierNs = 2000000000LL;  // a grid barrier gives up after 2 s

struct PanelArgs {
  double* M;            // the level's node matrices, m_bs doubles apart
  int64_t m_bs;
  int32_t* piv;         // the level's pivots, m2 per node
  double* logdet;       // per node: log|det M| (the level's entries of node_logdet)
  int32_t* sign;        // per node: sign of det M so far
  uint32_t* bar;        // per node: arrival counter of the grid barrier
  uint32_t bar_base;    // the counters' value when this panel starts
  double* slots;        // per launched node: 2 (parity) x (G + 1) x kSlot doubles
  int32_t* flags;
  int m2, c0, nb, G, rpc, node0;
  int G_wait;           // CTAs the barrier waits for: G (more only to test the timeout path)
  int last, signed_det;
};

__device__ __forceinline__ long long gtime() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Every CTA of the node arrives, then waits until all G have arrived at this step (the
// counter reaches base + (step + 1) G). Returns false if the wait gave up (the flag is set).
__device__ bool grid_barrier(uint32_t* ctr, uint32_t target, int32_t* flags, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const long long t0 = gtime();
    int ok = 1;
    while (ld_acquire(ctr) < target) {
      if (gtime() - t0 > kBarrierNs) {
        ok = 0;
        atomicOr(flags, kFlagTimeout);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

// Larger |value| wins; equal values: the lower row (the serial search's first maximum).
__device__ __forceinline__ void piv_merge(double& bv, int& bi, double v, int i) {
  if (i < 0) return;
  if (bi < 0 || v > bv || (v == bv && i < bi)) {
    bv = v;
    bi = i;
  }
}

// Panel columns [c0, c0 + nb) of node node0 + blockIdx.y, rows [c0, m2): CTA g holds rows
// [c0 + g rpc, c0 + (g + 1) rpc) in shared memory. Per column c: each CTA publishes its
// largest |entry| (its row with it) and, if it holds row c, row c; after the barrier every
// CTA picks the same pivot p from the G candidates, the holders of rows c and p exchange
// them, and each CTA eliminates its rows below c. The pivot search, the swap (whole panel
// rows), the multipliers and the updates are those of the unblocked LU, column by column.
__global__ void __launch_bounds__(kPanelThreads) k_lu_panel(PanelArgs a) {
  extern __shared__ double S[];  // rpc x (kNB + 1)
  __shared__ double urow[kNB], crow[kNB];
  __shared__ double wv[kPanelThreads / 32];
  __shared__ int wi[kPanelThreads / 32];
  __shared__ int sbi, sp, swg, ok_s;
  const int y = blockIdx.y, g = blockIdx.x, node = a.node0 + y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int m2 = a.m2, c0 = a.c0, nb = a.nb, G = a.G;
  const int r_lo = c0 + g * a.rpc;
  const int nrow = max(0, min(a.rpc, m2 - r_lo));
  constexpr int kLd = kNB + 1;
  int32_t* pivn = a.piv + (int64_t)node * a.m2;
  if (__ldcg(a.flags) & kFlagTimeout) {  // an earlier barrier gave up: no more waits; the
    if (g == 0)                          // pivots stay valid row indices for the kernels after
      for (int t = threadIdx.x; t < a.nb; t += kPanelThreads) pivn[a.c0 + t] = a.c0 + t;
    return;
  }
  double* M = a.M + (int64_t)node * a.m_bs;
  uint32_t* ctr = a.bar + node;
  for (int e = tid; e < nrow * nb; e += kPanelThreads) {
    const int i = e / nb, t = e - i * nb;
    S[i * kLd + t] = M[(int64_t)(r_lo + i) * m2 + c0 + t];
  }
  double lds = 0.0;
  int sgn = 1;
  if (g == 0 && tid == 0 && c0 > 0) {
    lds = a.logdet[node];
    sgn = a.sign[node];
  }
  __syncthreads();
  for (int t = 0; t < nb; ++t) {
    const int c = c0 + t;
    double* sl = a.slots + (int64_t)((y * 2 + (t & 1)) * (G + 1)) * kSlot;
    // this CTA's candidate
    double bv = -1.0;
    int bi = -1;
    if (tid < nrow && r_lo + tid >= c) piv_merge(bv, bi, fabs(S[tid * kLd + t]), r_lo + tid);
    if (bv != bv) bi = -1;  // NaN never wins (the serial search keeps the diagonal)
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      piv_merge(bv, bi, ov, oi);
    }
    if (lane == 0) {
      wv[w] = bv;
      wi[w] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double fv = -1.0;
      int fi = -1;
      for (int q = 0; q < kPanelThreads / 32; ++q) piv_merge(fv, fi, wv[q], wi[q]);
      sbi = fi;
      sl[(int64_t)g * kSlot] = fv;
      sl[(int64_t)g * kSlot + 1] = (double)fi;
    }
    __syncthreads();
    if (tid < nb) {
      if (sbi >= 0) sl[(int64_t)g * kSlot + 2 + tid] = S[(sbi - r_lo) * kLd + tid];
      if (c >= r_lo && c < r_lo + nrow) sl[(int64_t)G * kSlot + 2 + tid] = S[(c - r_lo) * kLd + tid];
    }
    if (!grid_barrier(ctr, a.bar_base + (uint32_t)(t + 1) * a.G_wait, a.flags, &ok_s)) {
      if (g == 0)
        for (int q = t + tid; q < nb; q += kPanelThreads) pivn[c0 + q] = c0 + q;
      return;
    }
    // the pivot, the same in every CTA
    if (w == 0) {
      double fv = -1.0;
      int fi = -1, fg = -1;
      for (int q = lane; q < G; q += 32) {
        const double v = __ldcg(sl + (int64_t)q * kSlot);
        const int i = (int)__ldcg(sl + (int64_t)q * kSlot + 1);
        if (i >= 0 && (fi < 0 || v > fv || (v == fv && i < fi))) {
          fv = v;
          fi = i;
          fg = q;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, fv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, fi, o);
        const int og = __shfl_xor_sync(0xffffffffu, fg, o);
        if (oi >= 0 && (fi < 0 || ov > fv || (ov == fv && oi < fi))) {
          fv = ov;
          fi = oi;
          fg = og;
        }
      }
      if (lane == 0) {
        sp = fi < 0 ? c : fi;  // every candidate NaN: keep the diagonal
        swg = fi < 0 ? G : fg;
      }
    }
    __syncthreads();
    const int p = sp;
    if (tid < nb) {
      urow[tid] = __ldcg(sl + (int64_t)swg * kSlot + 2 + tid);
      crow[tid] = __ldcg(sl + (int64_t)G * kSlot + 2 + tid);
    }
    __syncthreads();
    if (p != c && tid < nb) {
      if (c >= r_lo && c < r_lo + nrow) S[(c - r_lo) * kLd + tid] = urow[tid];
      if (p >= r_lo && p < r_lo + nrow) S[(p - r_lo) * kLd + tid] = crow[tid];
    }
    const double d = urow[t];
    if (g == 0 && tid == 0) {
      pivn[c] = p;
      if (p != c) sgn = -sgn;
      if (d == 0.0) sgn = 0;
      else {
        if (d < 0) sgn = -sgn;
        lds += log(fabs(d));
      }
    }
    __syncthreads();
    if (tid < nrow && r_lo + tid > c) {
      double* row = S + tid * kLd;
      const double l = d != 0.0 ? row[t] / d : 0.0;
      row[t] = l;
      if (l != 0.0)  // subtracting 0 * x leaves the row unchanged
        for (int j = t + 1; j < nb; ++j) row[j] -= l * urow[j];
    }
  }
  __syncthreads();
  for (int e = tid; e < nrow * nb; e += kPanelThreads) {
    const int i = e / nb, t = e - i * nb;
    M[(int64_t)(r_lo + i) * m2 + c0 + t] = S[i * kLd + t];
  }
  if (g == 0 && tid == 0) {
    a.logdet[node] = lds;
    a.sign[node] = sgn;
    if (a.last) {
      NodeArgs na{};
      na.flags = a.flags;
      na.signed_det = a.signed_det;
      record_sign(na, sgn);
    }
  }
}

// The panel's row swaps on every column outside it (in pivot order), then, for the
// columns right of it, U12 = L11^-1 A12 (L11 unit lower, the panel's top nb x nb block):
// one thread per column.
__global__ void __launch_bounds__(128) k_lu_rows(double* Mall, int64_t m_bs, const int32_t* pivall,
                                                 int m2, int c0, int nb) {
  __shared__ double L[kNB][kNB + 1];
  __shared__ int pv[kNB];
  const int node = blockIdx.y;
  double* M = Mall + (int64_t)node * m_bs;
  const int32_t* piv = pivall + (int64_t)node * m2;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    L[i][j] = M[(int64_t)(c0 + i) * m2 + c0 + j];
  }
  for (int e = threadIdx.x; e < nb; e += blockDim.x) {
    const int p = piv[c0 + e];
    pv[e] = (unsigned)p < (unsigned)m2 ? p : c0 + e;  // a pivot outside M: keep the row
  }
  __syncthreads();
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c0) col += nb;  // skip the panel's own columns
  if (col >= m2) return;
  for (int t = 0; t < nb; ++t) {
    const int p = pv[t];
    if (p != c0 + t) {
      double* x = M + (int64_t)(c0 + t) * m2 + col;
      double* z = M + (int64_t)p * m2 + col;
      const double v = *x;
      *x = *z;
      *z = v;
    }
  }
  if (col < c0) return;
  double x[kNB];
#pragma unroll
  for (int t = 0; t < kNB; ++t) {
    if (t < nb) {
      double s = M[(int64_t)(c0 + t) * m2 + col];
#pragma unroll
      for (int q = 0; q < t; ++q) s -= L[t][q] * x[q];
      x[t] = s;
    }
  }
#pragma unroll
  for (int t = 0; t < kNB; ++t)
    if (t < nb) M[(int64_t)(c0 + t) * m2 + col] = x[t];
}


// ---- Z = M^-1 [V^T P_R; U^T P_L] ------------------------------------------------------
// Row order of P M after the sequential swaps of the pivots: perm[i] = the row of M (and of
// the right-hand side) that ends at position i. One CTA per node, the swaps in shared memory.
__global__ void k_z_perm(const int32_t* __restrict__ pivall, int m2, int32_t* __restrict__ permall) {
  extern __shared__ int pm[];
  const int node = blockIdx.x;
  const int32_t* piv = pivall + (int64_t)node * m2;
  for (int i = threadIdx.x; i < m2; i += blockDim.x) pm[i] = i;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < m2; ++c) {
      int p = piv[c];
      if ((unsigned)p >= (unsigned)m2) p = c;  // a pivot outside M: keep the row
      const int v = pm[c];
      pm[c] = pm[p];
      pm[p] = v;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < m2; i += blockDim.x) permall[(int64_t)node * m2 + i] = pm[i];
}

// Z row i, column q = right-hand side row perm[i]: V^T P_R (rows < r) over U^T P_L, P's
// column zcol(q) of the half-node sums.
__global__ void k_z_fill(NodeArgs a, const int32_t* __restrict__ permall) {
  const int node = blockIdx.y;
  const int r = a.r, m2 = 2 * r, wz = a.wz;
  const double* L = a.half + (int64_t)(2 * node) * a.stride;
  const double* Rt = a.half + (int64_t)(2 * node + 1) * a.stride;
  const int32_t* perm = permall + (int64_t)node * m2;
  double* Zn = a.Z + (int64_t)node * a.z_stride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m2 * wz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / wz), q = (int)(e - (int64_t)i * wz);
    const int row = perm[i], pc = zcol(a, q);
    Zn[e] = row < r ? __ldcg(Rt + (int64_t)row * a.w + pc) : __ldcg(L + (int64_t)(row - r) * a.w + pc);
  }
}

// Diagonal block [b0, b0 + nb) of the substitution, one thread per column of Z:
// forward (L unit lower) or backward (U, divided by its diagonal).
template <bool kFwd>
__global__ void __launch_bounds__(128) k_z_diag(const double* __restrict__ Mall, int64_t m_bs,
                                                double* Zall, int64_t z_stride, int m2, int wz,
                                                int b0, int nb) {
  __shared__ double D[kNB][kNB + 1];
  const int node = blockIdx.y;
  const double* M = Mall + (int64_t)node * m_bs;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    D[i][j] = M[(int64_t)(b0 + i) * m2 + b0 + j];
  }
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= wz) return;
  double* Z = Zall + (int64_t)node * z_stride + (int64_t)b0 * wz + q;
  double x[kNB];
#pragma unroll
  for (int t = 0; t < kNB; ++t) x[t] = t < nb ? Z[(int64_t)t * wz] : 0.0;
  if (kFwd) {
#pragma unroll
    for (int t = 1; t < kNB; ++t) {
      if (t < nb) {
        double s = x[t];
#pragma unroll
        for (int c = 0; c < t; ++c) s -= D[t][c] * x[c];
        x[t] = s;
      }
    }
  } else {
#pragma unroll
    for (int t = kNB - 1; t >= 0; --t) {
      if (t < nb) {
        double s = x[t];
#pragma unroll
        for (int c = t + 1; c < kNB; ++c)
          if (c < nb) s -= D[t][c] * x[c];
        x[t] = s / D[t][t];
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kNB; ++t)
    if (t < nb) Z[(int64_t)t * wz] = x[t];
}

// Mixed form: Z's panel columns (q < cj) become double-float pairs in place.
__global__ void k_z_toff(double* Zall, int64_t z_stride, int m2, int wz, int cj) {
  const int node = blockIdx.y;
  double* Z = Zall + (int64_t)node * z_stride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m2 * cj;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cj), q = (int)(e - (int64_t)i * cj);
    double* z = Z + (int64_t)i * wz + q;
    reinterpret_cast<ff*>(z)[0] = ff_from_double(*z);
  }
}

// half[t][e] = sum over s < S of part[(t S + s)][e], e < E, in split order.
__global__ void k_split_sum(const double* __restrict__ part, int S, int64_t E, double* __restrict__ half) {
  const int t = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double* p = part + (int64_t)t * S * E + e;
    double v = 0.0;
    for (int q = 0; q < S; ++q) v += p[(int64_t)q * E];
    half[(int64_t)t * E + e] = v;
  }
}

unsigned grid_for(int64_t elems, int per_block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((elems + per_block - 1) / per_block, 4096));
}

}  // namespace

// Shared-memory attributes and the co-resident CTA count of the cooperative panel launch
// (once per context with a large-rank level).
cudaError_t big_setup(Ctx& c) {
  if (c.coop_cap > 0) return cudaSuccess;
  const int smem = (int)(sizeof(double) * kPanelRows * (kNB + 1));
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_z_perm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(int) * 2 * kMaxRank)));
  int occ = 0;
  HODLR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lu_panel, kPanelThreads, smem));
  c.coop_cap = std::max(1, occ) * c.sms;
  // HODLR_TEST_COOP_CAP=k: at most k co-resident CTAs per panel launch, so that a test can
  // run a level's nodes over several launches (a smaller cap only splits launches)
  if (const char* ev = getenv("HODLR_TEST_COOP_CAP")) c.coop_cap = std::max(1, std::min(c.coop_cap, atoi(ev)));
  return cudaSuccess;
}

// Published panel candidates per launch: 2 parities x (G + 1) slots for each of its cnt
// nodes, cnt <= max(1, coop_cap / G), so at most 4 max(coop_cap, G) slots; G is at most
// the CTAs of a 2 kMaxRank-row panel.
int64_t big_slot_elems(int coop_cap) {
  const int g_max = (2 * kMaxRank + kPanelRows - 1) / kPanelRows;
  return (int64_t)4 * std::max(coop_cap, g_max) * kSlot;
}

// Splits of the half-node sums of level u - 1 (sweep step u, product form): enough that the
// products fill the GPU twice (tiles of the rl x w outputs of the 2^u half-nodes times the
// splits), each split at least 2048 rows, at most 64.
int half_sum_splits(const Ctx& c, int u, int w) {
  if (u < 1) return 1;
  const int rl = c.h_rl[u - 1];
  const int64_t tiles = (int64_t)((rl + kBM - 1) / kBM) * ((w + kBN - 1) / kBN) << u;
  int mh = 0;
  for (int t = 0; t < (1 << u); ++t) mh = std::max(mh, c.h_nodes[((size_t)2 << c.kappa) + (1 << u) - 1 + t]);
  const int64_t want = (2 * (int64_t)c.sms + tiles - 1) / std::max<int64_t>(tiles, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)mh / 2048, 64}));
}

// Node step of level na.j with the blocked LU (factor mode) and the blocked substitution.
cudaError_t launch_node_blocked(Ctx& c, const NodeArgs& na, bool factor) {
  const int nodes = 1 << na.j, r = na.r, m2 = 2 * r;
  const int64_t m_bs = (int64_t)m2 * m2;
  HODLR_CUDA_TRY(big_setup(c));
  int32_t* sign = c.big_i32;
  uint32_t* bar = reinterpret_cast<uint32_t*>(c.big_i32 + c.big_nodes);
  if (factor) {
    // HODLR_TEST_BARRIER_EXTRA=k: each barrier waits for k CTAs that are never launched, so
    // that a test can check the bounded wait and the ETIMEOUT status (0 in normal use)
    const char* ev = getenv("HODLR_TEST_BARRIER_EXTRA");
    const int barrier_extra = ev ? std::max(0, atoi(ev)) : 0;
    k_m_build<<<dim3(grid_for(m_bs, 256), nodes), 256, 0, c.stream>>>(na, m_bs);
    ++c.launches;
    HODLR_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(uint32_t) * nodes, c.stream));
    uint32_t base = 0;
    for (int c0 = 0; c0 < m2; c0 += kNB) {
      const int nb = std::min(kNB, m2 - c0);
      const int rows = m2 - c0;
      const int G = (rows + kPanelRows - 1) / kPanelRows;
      const int rpc = (rows + G - 1) / G;
      const size_t smem = sizeof(double) * rpc * (kNB + 1);
      const int per = std::max(1, c.coop_cap / G);
      for (int k0 = 0; k0 < nodes; k0 += per) {
        const int cnt = std::min(per, nodes - k0);
        PanelArgs pa;
        pa.M = na.Mlu;
        pa.m_bs = m_bs;
        pa.piv = na.Mpiv;
        pa.logdet = na.node_logdet + ((1 << na.j) - 1);
        pa.sign = sign;
        pa.bar = bar;
        pa.bar_base = base;
        pa.slots = c.big_slots;
        pa.flags = na.flags;
        pa.m2 = m2;
        pa.c0 = c0;
        pa.nb = nb;
        pa.G = G;
        pa.G_wait = G + barrier_extra;
        pa.rpc = rpc;
        pa.node0 = k0;
        pa.last = c0 + nb == m2;
        pa.signed_det = na.signed_det;
        void* args[] = {&pa};
        HODLR_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_lu_panel, dim3(G, cnt),
                                                   dim3(kPanelThreads), args, smem, c.stream));
        ++c.launches;
      }
      base += (uint32_t)(nb * (G + barrier_extra));
      if (m2 > nb) {
        k_lu_rows<<<dim3((unsigned)((m2 - nb + 127) / 128), nodes), 128, 0, c.stream>>>(
            na.Mlu, m_bs, na.Mpiv, m2, c0, nb);
        ++c.launches;
      }
      const int rest = m2 - c0 - nb;
      if (rest > 0) {
        double* M = na.Mlu;
        GemmArgs g = gemm_uniform(M + (int64_t)(c0 + nb) * m2 + c0, m2, 1, m_bs,
                                  M + (int64_t)c0 * m2 + c0 + nb, m2, 1, m_bs,
                                  M + (int64_t)(c0 + nb) * m2 + c0 + nb, m2, 1, m_bs, rest, rest, nb);
        HODLR_CUDA_TRY((gemm<double, double, double, true>(g, rest, nodes, c.stream)));
        ++c.launches;
      }
    }
  }
  const int wz = na.wz;
  if (wz <= 0) return cudaGetLastError();
  int32_t* perm = c.big_perm;
  k_z_perm<<<nodes, 256, sizeof(int) * m2, c.stream>>>(na.Mpiv, m2, perm);
  k_z_fill<<<dim3(grid_for((int64_t)m2 * wz, 256), nodes), 256, 0, c.stream>>>(na, perm);
  c.launches += 2;
  const unsigned gq = (unsigned)((wz + 127) / 128);
  double* Z = na.Z;
  const int64_t zs = na.z_stride;
  for (int b0 = 0; b0 < m2; b0 += kNB) {
    const int nb = std::min(kNB, m2 - b0), b1 = b0 + nb;
    k_z_diag<true><<<dim3(gq, nodes), 128, 0, c.stream>>>(na.Mlu, m_bs, Z, zs, m2, wz, b0, nb);
    ++c.launches;
    if (b1 < m2) {
      GemmArgs g = gemm_uniform(na.Mlu + (int64_t)b1 * m2 + b0, m2, 1, m_bs, Z + (int64_t)b0 * wz,
                                wz, 1, zs, Z + (int64_t)b1 * wz, wz, 1, zs, m2 - b1, wz, nb);
      HODLR_CUDA_TRY((gemm<double, double, double, true>(g, m2 - b1, nodes, c.stream)));
      ++c.launches;
    }
  }
  for (int b0 = ((m2 - 1) / kNB) * kNB; b0 >= 0; b0 -= kNB) {
    const int nb = std::min(kNB, m2 - b0);
    k_z_diag<false><<<dim3(gq, nodes), 128, 0, c.stream>>>(na.Mlu, m_bs, Z, zs, m2, wz, b0, nb);
    ++c.launches;
    if (b0 > 0) {
      GemmArgs g = gemm_uniform(na.Mlu + b0, m2, 1, m_bs, Z + (int64_t)b0 * wz, wz, 1, zs, Z, wz,
                                1, zs, b0, wz, nb);
      HODLR_CUDA_TRY((gemm<double, double, double, true>(g, b0, nodes, c.stream)));
      ++c.launches;
    }
  }
  if (na.zff && na.cj > 0) {
    k_z_toff<<<dim3(grid_for((int64_t)m2 * na.cj, 256), nodes), 256, 0, c.stream>>>(Z, zs, m2, wz, na.cj);
    ++c.launches;
  }
  return cudaGetLastError();
}

static int ns_host(const Ctx& c, int id) { return c.h_nodes[((size_t)2 << c.kappa) + id]; }

// Sweep step of level u in product form: the rows of each half of a level-u node
// P -= Ut Z_side (panel columns [0, cP) and the right-hand sides), then, for u > 0, the
// half-node sums of level u - 1,
// half + t hs with rows c < r_{u-1} and columns q < cP + nrhs (hs = r_{u-1} (cP + nrhs)).
template <class T>
static cudaError_t sweep_gemm_t(Ctx& c, int u, int nrhs, bool factor_mode) {
  const int K = c.kappa;
  const int64_t n = c.n;
  const int ru = c.h_rl[u], cu = c.h_coff[u];
  const int cP = factor_mode ? cu : 0, wz = cP + nrhs;
  const int rl = u > 0 ? c.h_rl[u - 1] : 0, cl = u > 0 ? c.h_coff[u - 1] : 0;
  T* pan = reinterpret_cast<T*>(c.pan);
  const T* phi = reinterpret_cast<const T*>(c.phi);
  const int32_t* nb = c.nodes;
  const int32_t* ns = c.nodes + ((int64_t)2 << K);
  if (ru > 0 && wz > 0) {
    // the halves of the level-u nodes are the level-(u + 1) nodes, 2^(u+1) of them
    const int halves = 2 << u, id0 = halves - 1;
    int mh = 0;
    for (int t = 0; t < halves; ++t) mh = std::max(mh, c.h_nodes[((size_t)2 << K) + id0 + t]);
    GemmArgs g{};
    g.mode = kNodeRows;
    g.a = pan + (int64_t)cu * n;
    g.ai = 1;
    g.ak = n;
    g.bk = wz;
    g.bj = 1;
    g.ci = 1;
    g.cj = n;
    g.k = ru;
    g.nb = nb;
    g.ns = ns;
    g.id0 = id0;
    g.sh = 1;
    g.z_stride = (int64_t)2 * ru * wz;
    g.z_side = (int64_t)ru * wz;
    if (cP > 0) {
      g.b = reinterpret_cast<const T*>(c.Z);
      g.c = pan;
      g.n = cP;
      HODLR_CUDA_TRY((gemm<T, T, T, true>(g, mh, halves, c.stream)));
      ++c.launches;
    }
    if (nrhs > 0) {
      g.b = c.Z + cP;
      g.c = c.Y;
      g.n = nrhs;
      HODLR_CUDA_TRY((gemm<T, double, double, true>(g, mh, halves, c.stream)));
      ++c.launches;
    }
  }
  if (u > 0 && rl > 0 && wz > 0) {
    GemmArgs h{};
    h.mode = kHalfRows;
    h.a = phi + (int64_t)cl * n;
    h.ai = n;
    h.ak = 1;
    h.bk = 1;
    h.bj = n;
    h.ci = wz;
    h.cj = 1;
    h.c_bs = (int64_t)rl * wz;
    h.m = rl;
    h.nb = nb;
    h.ns = ns;
    h.id0 = (1 << u) - 1;
    // split-K when the 2^u half-nodes' outputs are too few tiles for the GPU: each split's
    // sum into its own slot of the split buffer, then the splits added in order
    const int S = half_sum_splits(c, u, wz);
    int mh = 0;
    for (int t = 0; t < (1 << u); ++t) mh = std::max(mh, ns_host(c, h.id0 + t));
    h.ksplit = S;
    h.kchunk = (mh + S - 1) / S;
    double* dst = S > 1 ? c.split_buf : c.half;
    if (cP > 0) {
      h.b = pan;
      h.c = dst;
      h.n = cP;
      HODLR_CUDA_TRY((gemm<T, T, double, false>(h, rl, S << u, c.stream)));
      ++c.launches;
    }
    if (nrhs > 0) {
      h.b = c.Y;
      h.c = dst + cP;
      h.n = nrhs;
      HODLR_CUDA_TRY((gemm<T, double, double, false>(h, rl, S << u, c.stream)));
      ++c.launches;
    }
    if (S > 1) {
      const int64_t E = (int64_t)rl * wz;
      k_split_sum<<<dim3(grid_for(E, 256), 1u << u), 256, 0, c.stream>>>(c.split_buf, S, E, c.half);
      ++c.launches;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_gemm(Ctx& c, int u, int nrhs, bool factor_mode) {
  return c.precision == 1 ? sweep_gemm_t<ff>(c, u, nrhs, factor_mode)
                          : sweep_gemm_t<double>(c, u, nrhs, factor_mode);
}

}  // namespace hodlr
