// Analytic compression by Chebyshev interpolation (Sec. 3.1: for a smooth kernel the block
// A = k(x_i, y_j) is approximated as E A~ P, A~ the kernel sampled at Chebyshev nodes of
// the two clusters and E, P interpolation matrices, by the barycentric formula of Berrut and
// Trefethen). Points in one dimension; an alternative to the adaptive cross approximation
// that fills the same per-level panels and ranks.
//
//   k_cheb_node    one CTA per internal node (all levels at once): nodes on each child's
//                  interval [first point, last point]; for q = 8, 16, 32, 64 the kernel
//                  at the q x q node pairs and its 2-D Chebyshev coefficients (two shared
//                  memory products with a cosine table); the first q whose last quarter of
//                  coefficients is at most eps times the largest is kept; then a cross with
//                  full pivoting on A~ down to a residual of eps ||A~||_F gives the rank r
//                  and the q x r factors of A~ = A~_u A~_v^T, turned into Chebyshev
//                  coefficients (c = T A~_u, the same transform). A block that interpolation
//                  cannot represent within its caps (no q passes, or the cross reaches
//                  min(m_L, m_R)) is stored exactly when m = min(m_L, m_R) <= max_rank
//                  (rank m: identity on the smaller side, the block's entries on the
//                  other; q = -1 marks it), else its rank is 0 and ok = 0.
//   k_cheb_expand  one CTA per (leaf, level): the leaf's rows of the level's U (left child)
//                  or V (right child): the interpolating polynomial evaluated in the
//                  Chebyshev basis, T_k(u) by the three-term recurrence at u = the point
//                  mapped to [-1, 1], times the coefficients. This is the polynomial the
//                  barycentric form gives (Lagrange basis at the same nodes), with no
//                  division per point and node.
#include <cuda_runtime.h>

#include "ff.cuh"
#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kChebQ = 64;  // most nodes per cluster
constexpr int kChebThreads = 256;
constexpr int kW = kChebThreads / 32;
constexpr double kPi = 3.141592653589793;

struct ChebArgs {
  const double* xs;  // sorted 1-D points
  int64_t n;
  const int32_t* nb;
  const int32_t* ns;
  int kind;
  const double* hyp;
  double eps;
  int max_rank;
  int kappa;
  int32_t* rank;   // per internal node
  int32_t* ok;     // 1 if converged below the caps
  int32_t* qn;     // nodes per cluster chosen, 0 if none up to kChebQ, -1: stored exactly
  double* coef;    // per node: Chebyshev coefficients of A~_u then of A~_v, each
                   // kChebQ x kChebQ, column l at l * kChebQ
  double* raw;
  int64_t raw_off[32];
  int ff_out;      // 1: store the panels as double-float pairs (mixed form)
};

// Chebyshev point k of the first kind (of q) on [lo, hi].
__device__ __forceinline__ double cheb_point(double lo, double hi, int q, int k) {
  double th = (2.0 * k + 1.0) * kPi / (2.0 * q);
  return 0.5 * (lo + hi) + 0.5 * (hi - lo) * cos(th);
}

// Block-wide max of v (all threads get it).
__device__ double block_max(double v, double* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = red[0];
  for (int q = 1; q < kW; ++q) m = fmax(m, red[q]);
  return m;
}

// Block-wide sum of v in a fixed order (all threads get it).
__device__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int q = 0; q < kW; ++q) m += red[q];
  return m;
}

__global__ void __launch_bounds__(kChebThreads) k_cheb_node(ChebArgs a) {
  extern __shared__ double sm[];  // A (q x q, then A~_u), W (q x q residual), V (A~_v)
  double* A = sm;
  double* W = sm + kChebQ * kChebQ;
  double* V = sm + 2 * kChebQ * kChebQ;
  __shared__ double s[kChebQ], t[kChebQ], ctab[4 * kChebQ], us[kChebQ], vs[kChebQ];
  __shared__ double red[kW], redb[kW];
  __shared__ int redi[kW];
  const int id = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int bl = a.nb[2 * id + 1], ml = a.ns[2 * id + 1];
  const int br = a.nb[2 * id + 2], mr = a.ns[2 * id + 2];
  if (ml == 0 || mr == 0) {  // an empty block (leaf size 1 can leave a child empty): exact
    if (tid == 0) {
      a.qn[id] = 0;
      a.rank[id] = 0;
      a.ok[id] = 1;
    }
    return;
  }
  const double a1 = a.xs[bl], b1 = a.xs[bl + ml - 1], a2 = a.xs[br], b2 = a.xs[br + mr - 1];
  const Cov cov = cov_from(a.kind, a.hyp);
  int q = 0;
  for (int qq = 8; qq <= kChebQ; qq *= 2) {
    for (int k = tid; k < qq; k += kChebThreads) {
      s[k] = cheb_point(a1, b1, qq, k);
      t[k] = cheb_point(a2, b2, qq, k);
    }
    for (int m = tid; m < 4 * qq; m += kChebThreads) ctab[m] = cos(m * kPi / (2.0 * qq));
    __syncthreads();
    for (int e = tid; e < qq * qq; e += kChebThreads) {
      int i = e / qq, j = e - i * qq;
      A[e] = cov_r(cov, fabs(s[i] - t[j]));
    }
    __syncthreads();
    // W = T A, T_ja = (2/q) cos(j (2a + 1) pi / (2q)), row 0 halved
    for (int e = tid; e < qq * qq; e += kChebThreads) {
      int jj = e / qq, b = e - jj * qq;
      double acc = 0.0;
      for (int aa = 0; aa < qq; ++aa) acc += ctab[(jj * (2 * aa + 1)) % (4 * qq)] * A[aa * qq + b];
      W[e] = acc * (jj == 0 ? 1.0 : 2.0) / qq;
    }
    __syncthreads();
    // coefficients C = W T^T: the largest, and the largest in the last quarter
    double cmax = 0.0, tail = 0.0;
    for (int e = tid; e < qq * qq; e += kChebThreads) {
      int jj = e / qq, kk = e - jj * qq;
      double acc = 0.0;
      for (int b = 0; b < qq; ++b) acc += W[jj * qq + b] * ctab[(kk * (2 * b + 1)) % (4 * qq)];
      double c = fabs(acc * (kk == 0 ? 1.0 : 2.0) / qq);
      cmax = fmax(cmax, c);
      if (jj >= qq - qq / 4 || kk >= qq - qq / 4) tail = fmax(tail, c);
    }
    cmax = block_max(cmax, red);
    tail = block_max(tail, redb);
    if (tail <= a.eps * cmax) {
      q = qq;
      break;
    }
  }
  const int mmin = ml < mr ? ml : mr;
  if (q == 0) {
    if (tid == 0) {
      bool exact = mmin <= a.max_rank;
      a.qn[id] = exact ? -1 : 0;
      a.rank[id] = exact ? mmin : 0;
      a.ok[id] = exact ? 1 : 0;
    }
    return;
  }
  // cross with full pivoting on A (residual in W)
  int rmax = ml < mr ? ml : mr;
  rmax = rmax < a.max_rank ? rmax : a.max_rank;
  rmax = rmax < q ? rmax : q;
  double n0 = 0.0;
  for (int e = tid; e < q * q; e += kChebThreads) {
    W[e] = A[e];
    n0 += A[e] * A[e];
  }
  n0 = block_sum(n0, red);  // (its barriers also end the reads of A: it now holds A~_u)
  double* cu = a.coef + (int64_t)id * 2 * kChebQ * kChebQ;
  double* cv = cu + kChebQ * kChebQ;
  int r = 0, okv = 1;
  for (;;) {
    double res = 0.0, bv = -1.0;
    int bi = 0;
    for (int e = tid; e < q * q; e += kChebThreads) {
      double v = W[e];
      res += v * v;
      if (fabs(v) > bv) {  // increasing e per thread: ties keep the lower index
        bv = fabs(v);
        bi = e;
      }
    }
    res = block_sum(res, red);
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    __syncthreads();
    if (lane == 0) {
      redb[w] = bv;
      redi[w] = bi;
    }
    __syncthreads();
    bv = redb[0];
    bi = redi[0];
    for (int k = 1; k < kW; ++k)
      if (redb[k] > bv || (redb[k] == bv && redi[k] < bi)) {
        bv = redb[k];
        bi = redi[k];
      }
    if (res <= a.eps * a.eps * n0 || bv == 0.0) break;
    if (r == rmax) {
      okv = 0;
      break;
    }
    const int pi = bi / q, pj = bi - pi * q;
    const double piv = W[pi * q + pj];
    for (int k = tid; k < q; k += kChebThreads) {
      double u = W[k * q + pj], v = W[pi * q + k] / piv;
      us[k] = u;
      vs[k] = v;
      A[r * kChebQ + k] = u;
      V[r * kChebQ + k] = v;
    }
    __syncthreads();
    for (int e = tid; e < q * q; e += kChebThreads) {
      int i = e / q, j = e - i * q;
      W[e] -= us[i] * vs[j];
    }
    __syncthreads();
    ++r;
  }
  const bool exact = !okv && mmin <= a.max_rank;
  if (tid == 0) {
    a.qn[id] = exact ? -1 : q;
    a.rank[id] = exact ? mmin : r;
    a.ok[id] = exact ? 1 : okv;
  }
  if (exact) return;
  // Chebyshev coefficients of each factor column: c_kl = (2/q) sum_a cos(k th_a) F_al,
  // row 0 halved (ctab still holds the cosines of the accepted q)
  for (int e = tid; e < 2 * r * q; e += kChebThreads) {
    int side = e / (r * q), f = e - side * r * q;
    int l = f / q, k = f - l * q;
    const double* F = side ? V : A;
    double acc = 0.0;
    for (int aa = 0; aa < q; ++aa) acc += ctab[(k * (2 * aa + 1)) % (4 * q)] * F[l * kChebQ + aa];
    (side ? cv : cu)[l * kChebQ + k] = acc * (k == 0 ? 1.0 : 2.0) / q;
  }
}

// kFF (mixed form): the recurrence and the sums in double-float on the FP32 pipe (the
// panels are stored as double-floats anyway); otherwise FP64.
template <bool kFF>
__global__ void __launch_bounds__(kMaxLeaf) k_cheb_expand(ChebArgs a) {
  extern __shared__ double sm[];  // coefficients (q x r, column l at l * kChebQ), T (128 x 65)
  double* cf = sm;
  double* L = sm + kChebQ * kChebQ;
  constexpr int kLS = kChebQ + 1;
  const int leaf = blockIdx.x, j = blockIdx.y, tid = threadIdx.x;
  const int K = a.kappa;
  const int anc = (leaf >> (K - j)) + (1 << j) - 1;                 // node at level j
  const int cid = (leaf >> (K - j - 1)) + (1 << (j + 1)) - 1;       // its child over the leaf
  const bool left = cid == 2 * anc + 1;
  const int q = a.qn[anc], r = a.rank[anc];
  if (r == 0) return;
  const int cb = a.nb[cid], cm = a.ns[cid];
  const int lid = (1 << K) - 1 + leaf;
  const int b = a.nb[lid], p = a.ns[lid];
  double* raw = a.raw + a.raw_off[j];
  if (q < 0) {  // stored exactly: identity on the smaller child, the block on the other
    if (tid >= p) return;
    const int bl = a.nb[2 * anc + 1], ml = a.ns[2 * anc + 1];
    const int br = a.nb[2 * anc + 2], mr = a.ns[2 * anc + 2];
    const Cov cov = cov_from(a.kind, a.hyp);
    const int row = b + tid, rel = row - cb;
    const bool ident = left ? ml <= mr : mr < ml;
    for (int l = 0; l < r; ++l) {
      double v;
      if (ident)
        v = rel == l ? 1.0 : 0.0;
      else
        v = cov_r(cov, fabs(a.xs[row] - a.xs[left ? br + l : bl + l]));
      int64_t o = (int64_t)l * a.n + row;
      if (a.ff_out)
        reinterpret_cast<ff*>(raw)[o] = ff_from_double(v);
      else
        raw[o] = v;
    }
    return;
  }
  const double lo = a.xs[cb], hi = a.xs[cb + cm - 1];
  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  const double inv_half = half > 0.0 ? 1.0 / half : 0.0;  // a zero-length interval: u = 0
  const double* src = a.coef + (int64_t)anc * 2 * kChebQ * kChebQ + (left ? 0 : kChebQ * kChebQ);
  for (int e = tid; e < r * kChebQ; e += kMaxLeaf) {
    int l = e / kChebQ, k = e - l * kChebQ;
    if (k < q) {
      if (kFF)
        reinterpret_cast<ff*>(cf)[e] = ff_from_double(src[e]);
      else
        cf[e] = src[e];
    }
  }
  __syncthreads();
  if (tid >= p) return;
  double u = (a.xs[b + tid] - mid) * inv_half;
  u = fmin(1.0, fmax(-1.0, u));
  if (kFF) {
    const ff* cff = reinterpret_cast<const ff*>(cf);
    ff* Lf = reinterpret_cast<ff*>(L) + tid * kLS;  // T_k(u), k < q
    const ff uf = ff_from_double(u), u2 = ff{2.0f * uf.hi, 2.0f * uf.lo};
    ff t0 = {1.0f, 0.0f}, t1 = uf;
    Lf[0] = t0;
    if (q > 1) Lf[1] = uf;
    for (int k = 2; k < q; ++k) {
      ff t2 = ff_neg(ff_fms(t0, u2, t1));  // 2 u T_{k-1} - T_{k-2}
      Lf[k] = t2;
      t0 = t1;
      t1 = t2;
    }
    ff* rawf = reinterpret_cast<ff*>(raw);
    for (int l = 0; l < r; ++l) {
      ff acc = {0.0f, 0.0f};
      for (int k = 0; k < q; ++k) acc = ff_fma(acc, Lf[k], cff[l * kChebQ + k]);
      rawf[(int64_t)l * a.n + b + tid] = acc;
    }
    return;
  }
  double* Li = L + tid * kLS;  // T_k(u), k < q
  double t0 = 1.0, t1 = u;
  Li[0] = 1.0;
  if (q > 1) Li[1] = u;
  for (int k = 2; k < q; ++k) {
    double t2 = 2.0 * u * t1 - t0;
    Li[k] = t2;
    t0 = t1;
    t1 = t2;
  }
  for (int l = 0; l < r; ++l) {
    double acc = 0.0;
    for (int k = 0; k < q; ++k) acc += Li[k] * cf[l * kChebQ + k];
    raw[(int64_t)l * a.n + b + tid] = acc;
  }
}

}  // namespace

size_t cheb_coef_elems(int nint) { return (size_t)nint * 2 * kChebQ * kChebQ; }

// Chebyshev compression of every off-diagonal block: ranks into c.st_rank, convergence into
// c.st_ok, the panels into c.raw (the same layout the cross approximation fills).
cudaError_t launch_cheb(Ctx& c) {
  int nint = (1 << c.kappa) - 1;
  if (nint == 0) return cudaSuccess;
  ChebArgs a;
  a.xs = c.xs;
  a.n = c.n;
  a.nb = c.nodes;
  a.ns = c.nodes + ((int64_t)2 << c.kappa);
  a.kind = c.kind;
  a.hyp = c.hyp;
  a.eps = c.eps;
  a.max_rank = c.max_rank;
  a.kappa = c.kappa;
  a.rank = c.st_rank;
  a.ok = c.st_ok;
  a.qn = c.cheb_q;
  a.coef = c.cheb_coef;
  a.raw = c.raw;
  for (int j = 0; j < 32; ++j) a.raw_off[j] = j < c.kappa ? c.h_raw_off[j] : 0;
  a.ff_out = c.precision == 1;
  const size_t smem_node = sizeof(double) * 3 * kChebQ * kChebQ;
  const size_t smem_exp = sizeof(double) * (kChebQ * kChebQ + kMaxLeaf * (kChebQ + 1));
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_cheb_node, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_node));
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_cheb_expand<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_exp));
  HODLR_CUDA_TRY(cudaFuncSetAttribute(k_cheb_expand<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_exp));
  k_cheb_node<<<nint, kChebThreads, smem_node, c.stream>>>(a);
  if (a.ff_out)
    k_cheb_expand<true><<<dim3(1u << c.kappa, c.kappa), kMaxLeaf, smem_exp, c.stream>>>(a);
  else
    k_cheb_expand<false><<<dim3(1u << c.kappa, c.kappa), kMaxLeaf, smem_exp, c.stream>>>(a);
  c.launches += 2;
  return cudaGetLastError();
}

}  // namespace hodlr
