// Internal declarations of the GB300 HODLR library: the problem context, the covariance
// functions evaluated on the device, and the host-side launch wrappers of every kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hodlr.h"
#include "ff.cuh"

namespace hodlr {

constexpr int kMaxLeaf = 128;      // leaf blocks live in shared memory
constexpr int kMaxDim = 64;        // largest point dimension d
// Dynamic shared memory above which a launch opts in with
// cudaFuncAttributeMaxDynamicSharedMemorySize: without it static plus dynamic must stay
// within 48 KB, and the kernels' static arrays take up to about 1 KB.
constexpr size_t kSmemOptIn = 40 * 1024;
constexpr int kMaxRank = 8192;     // hard cap on a block's rank (opts.max_rank)
constexpr int kDefaultMaxRank = 64;  // default opts.max_rank
constexpr int kSmemRank = 64;      // ranks up to this use the shared-memory node step
                                   // (2r x 2r in smem) and the fused level sweep
constexpr int kBlockRank = 128;    // ranks from this up: the sweep in product form
                                   // (levels_big.cu; node steps above kSmemRank are blocked)
constexpr int kAcaTile = 1024;     // columns (rows) of one ACA work item
constexpr int kSmallNode = 256;    // nodes whose children both fit: one warp per node
constexpr int kWideRank = 256;     // nodes whose rank cap min(m_left, m_right, max_rank)
constexpr int kWideTile = 32;      // exceeds this also get ACA work items of 32 rows (one
                                   // per lane), used once their rank reaches kWideRank

// ---------------------------------------------------------------------------------------
// Covariance functions (Table 1 with length scale ell and amplitude a; Matern nu = 3/2 and
// 5/2 in closed form). r is the Euclidean distance between the two points.
// ---------------------------------------------------------------------------------------
struct Cov {
  int kind;
  double inv_ell;
  double amp;
  double alpha;  // rational quadratic exponent
};

__host__ __device__ inline bool kind_indefinite(int kind) {
  return kind == HODLR_K_MQ || kind == HODLR_K_BIHARMONIC;
}

// The radial functions of Sec. 5, t = r / ell. Kept out of line so that their pow and log
// do not raise the register count of every kernel that evaluates the common covariances.
static __device__ __noinline__ double cov_r_radial(int kind, double t, double amp, double alpha) {
  switch (kind) {
    case HODLR_K_RQ: return amp * pow(1.0 + t * t, -alpha);
    case HODLR_K_IMQ: return amp / sqrt(1.0 + t * t);
    case HODLR_K_MQ: return amp * sqrt(1.0 + t * t);
    case HODLR_K_BIHARMONIC: return t > 0.0 ? amp * t * t * log(t) : 0.0;  // 0: the limit
    default: return nan("");
  }
}

// exp(x) in FP64 by the table-driven method of P. T. P. Tang (ACM Trans. Math. Software 15,
// 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128, so exp(x) = 2^m 2^(j/64) exp(r);
// ln2/64 is split in two (its first part with 32 significant bits, so n times it is exact
// for |n| < 2^21), exp(r) - 1 is its Taylor polynomial to degree 6 (the next term is below
// 3e-20 relative), the 64 values 2^(j/64) are rounded to the nearest double, and 2^m is
// added to the exponent field. About ten FP64 operations, against about 25 for the
// general-purpose exp (GB300 runs FP64 at 1/64 of the FP32 rate). Results within about
// one unit in the last place of the exact value.
static __device__ double kExp2J[64] = {
    1.0, 1.0108892860517005, 1.0218971486541166, 1.0330248790212284,
    1.0442737824274138, 1.0556451783605572, 1.0671404006768237, 1.0787607977571199,
    1.0905077326652577, 1.102382583307841, 1.1143867425958924, 1.1265216186082418,
    1.1387886347566916, 1.1511892299529827, 1.1637248587775775, 1.1763969916502812,
    1.189207115002721, 1.202156731452703, 1.215247359980469, 1.22848053610687,
    1.241857812073484, 1.255380757024691, 1.2690509571917332, 1.2828700160787783,
    1.2968395546510096, 1.3109612115247644, 1.3252366431597413, 1.339667524053303,
    1.3542555469368927, 1.3690024229745905, 1.383909881963832, 1.3989796725383112,
    1.4142135623730951, 1.42961333839197, 1.4451808069770467, 1.460917794180647,
    1.4768261459394993, 1.4929077282912648, 1.5091644275934228, 1.5255981507445384,
    1.5422108254079407, 1.559004400237837, 1.5759808451078865, 1.593142151342267,
    1.6104903319492543, 1.6280274218573478, 1.645755478153965, 1.6636765803267364,
    1.681792830507429, 1.7001063537185235, 1.718619298122478, 1.7373338352737062,
    1.7562521603732995, 1.7753764925265212, 1.7947090750031072, 1.8142521755003989,
    1.8340080864093424, 1.8539791250833855, 1.8741676341103, 1.8945759815869656,
    1.9152065613971474, 1.9360617934922943, 1.9571441241754002, 1.978456026387951};

__device__ __forceinline__ double exp_tang(double x) {
  if (!(x > -745.2)) return x != x ? x : 0.0;  // NaN stays NaN; below: underflow to 0
  if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);  // overflow
  const double n = rint(x * 92.33248261689366);   // x 64 / ln2
  double r = fma(-n, 0.01083042469326756, x);     // first part of ln2/64
  r = fma(-n, 2.9815858269852933e-12, r);         // second part
  const int ni = (int)n;
  const int j = ni & 63, m = ni >> 6;             // n = 64 m + j (floor division)
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(r, q, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);              // exp(r) - 1
  const double t = __ldg(&kExp2J[j]);
  const double y = fma(t, p, t);                  // 2^(j/64) exp(r), in [0.99, 2.02]
  if (m < -1020) return scalbn(y, m);             // subnormal results
  return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
}

// The four covariances of Table 1 (exponential, squared-exponential, Matern-3/2,
// Matern-5/2) alone: what kernels specialised for the common case evaluate.
__device__ __forceinline__ double cov_r_table1(const Cov& c, double r) {
  switch (c.kind) {
    case HODLR_K_EXP:
      return c.amp * exp_tang(-r * c.inv_ell);
    case HODLR_K_SE: {
      double t = r * c.inv_ell;
      return c.amp * exp_tang(-0.5 * t * t);
    }
    case HODLR_K_MATERN32: {
      double s = 1.7320508075688772 * r * c.inv_ell;  // sqrt(3) r / ell
      return c.amp * (1.0 + s) * exp_tang(-s);
    }
    default: {  // Matern-5/2
      double s = 2.23606797749979 * r * c.inv_ell;  // sqrt(5) r / ell
      return c.amp * (1.0 + s + s * s * (1.0 / 3.0)) * exp_tang(-s);
    }
  }
}

// Any covariance kind.
__device__ __forceinline__ double cov_r(const Cov& c, double r) {
  if (c.kind <= HODLR_K_MATERN52) return cov_r_table1(c, r);
  return cov_r_radial(c.kind, r * c.inv_ell, c.amp, c.alpha);
}

// Hyperparameters in device memory, so that kernels (and captured graphs) read the current
// setting: hyp[0] = 1/ell, hyp[1] = amplitude a, hyp[2] = sigma^2, hyp[3] = covariance
// scale cr (1/ell, 1/ell, sqrt3/ell, sqrt5/ell for exp, SE, Matern-3/2, Matern-5/2; 1/ell
// for the radial functions), hyp[4] = the rational quadratic's exponent alpha.
enum {
  kHypInvEll = 0, kHypAmp = 1, kHypSigma2 = 2, kHypScale = 3, kHypAlpha = 4,
  kHypCrFF = 5, kHypAmpFF = 6, kHypAlphaFF = 7, kHypLen = 8
};

__device__ __forceinline__ Cov cov_from(int kind, const double* __restrict__ hyp) {
  return Cov{kind, hyp[kHypInvEll], hyp[kHypAmp], hyp[kHypAlpha]};
}

// Slots kHypCrFF.. hold the double-float kernels' covariance parameters (the factor applied
// to r, the amplitude, the rational quadratic's exponent) as double-float pairs. They are
// converted once, by the kernel that writes the slots, instead of by every thread that
// reads them: FP64-to-float conversions run on the FP64 pipe, 1/64 of the FP32 rate.
__device__ __forceinline__ void set_hyp_ff(double* hyp) {
  ff* h = reinterpret_cast<ff*>(hyp);
  h[kHypCrFF] = ff_from_double(hyp[kHypScale]);
  h[kHypAmpFF] = ff_from_double(hyp[kHypAmp]);
  h[kHypAlphaFF] = ff_from_double(hyp[kHypAlpha]);
}

__device__ __forceinline__ CovFF load_cov_ff(int kind, const double* __restrict__ hyp) {
  const ff* h = reinterpret_cast<const ff*>(hyp);
  return CovFF{kind, h[kHypCrFF], h[kHypAmpFF], h[kHypAlphaFF]};
}

// Sorted points in structure-of-arrays form: coordinate c of sorted point i is x[c * n + i].
struct Pts {
  const double* x;
  int64_t n;
  int d;
};

// Distance for points in one or two dimensions only (kernels specialised for that case).
__device__ __forceinline__ double dist12(const Pts& p, int i, int j) {
  if (p.d == 1) return fabs(p.x[i] - p.x[j]);
  double a = p.x[i] - p.x[j];
  double b = p.x[p.n + i] - p.x[p.n + j];
  return sqrt(a * a + b * b);
}

__device__ __forceinline__ double dist(const Pts& p, int i, int j) {
  if (p.d == 1) return fabs(p.x[i] - p.x[j]);
  double a = p.x[i] - p.x[j];
  double b = p.x[p.n + i] - p.x[p.n + j];
  if (p.d == 2) return sqrt(a * a + b * b);
  double e = p.x[2 * p.n + i] - p.x[2 * p.n + j];
  double s = a * a + b * b + e * e;
  for (int c = 3; c < p.d; ++c) {
    double t = p.x[c * p.n + i] - p.x[c * p.n + j];
    s += t * t;
  }
  return sqrt(s);
}


// Device error word bits (ctx->dflags).
// kFlagNegDet: parity of the negative block determinants of an indefinite C (the sign of
// det C), toggled by each one.
enum : int { kFlagNotSpd = 1, kFlagRankCap = 2, kFlagTimeout = 4, kFlagNegDet = 8 };  // rank cap: also presize

// ---------------------------------------------------------------------------------------
// Context: everything one problem owns on the device. Layouts (n rows, column stride n):
//   xs       d x n sorted coordinates (SoA)
//   perm     n int32: sorted row i is the caller's point perm[i]
//   nodes    2^(kappa+1) int32: begin row of node id (level order, root = 0) and nodes[last]=n
//   raw      per level j: n x rcap_j ACA columns (U rows in left children, V in right)
//   phi      n x R   original U/V of every level, level j at columns [coff_j, coff_j + r_j)
//   pan      n x R   working copy; after factor it holds Ut/Vt (finer inverses applied)
//   Y        n x max_nrhs right-hand sides in sorted order (overwritten by C^-1 y)
//   leafL    2^kappa x 128 x 128 L D L^T factors of the leaf blocks (row-major, lower;
//            FP64, or double-float pairs in the mixed form)
// ---------------------------------------------------------------------------------------
struct Ctx {
  // problem
  int64_t n = 0;
  int d = 1;
  int kind = 0;
  double ell = 1, amp = 1, sigma2 = 0, eps = 1e-12;
  double alpha = 1;               // rational quadratic exponent
  bool indefinite = false;        // multiquadric / biharmonic: LU leaves, signed log |det|
  int det_sign = 1;               // sign of det C after the last factorization
  int32_t* leaf_perm = nullptr;   // LU row orders, kMaxLeaf per leaf (indefinite only)
  int compression = 0;            // 0: cross approximation, 1: Chebyshev interpolation
  int32_t* cheb_q = nullptr;      // Chebyshev nodes per cluster of each internal node
  double* cheb_coef = nullptr;    // Chebyshev: factors of the sampled blocks
  int leaf = 128, kappa = 0, max_rank = kDefaultMaxRank, max_nrhs = 16;
  int precision = 0;              // 0: FP64, 1: double-float leaf stage (mixed)
  int leaf_threads = 512;         // CTA size of the double-float leaf kernel (two CTAs per SM)
  bool leaf_tc = false;           // mixed form: leaf updates on the tensor cores (k_leaf_tc)
  // batched evaluation with this context as its first lane: the persistent leaf launch's
  // argument blocks and leaf offsets (device), grown as needed
  void* batch_args = nullptr;
  int32_t* batch_first = nullptr;  // offsets, then one counter per form
  int64_t batch_cap = 0;           // bytes of batch_args
  int64_t batch_first_cap = 0;     // ints of batch_first
  int leaf_threads64 = 512;       // CTA size of the FP64 leaf kernel (measured best)
  bool no_fused = false;          // force the segmented level sweep
  int sweep_tile = 0;             // tile shape of the fused sweep (leaves, threads per block)
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 152;

  // tree (host mirror + device)
  std::vector<int32_t> h_nodes;   // begin rows, 2^(kappa+1) entries (+1 sentinel)
  int32_t* nodes = nullptr;
  double* xs = nullptr;
  int32_t* perm = nullptr;
  int max_leaf_size = 0;

  // ACA work decomposition (host-built, device copies)
  int64_t n_items = 0;
  int32_t* item_node = nullptr;   // internal node id of each work item
  int32_t* item_start = nullptr;  // first row/column of the item's tile
  int32_t* node_item0 = nullptr;  // first item of each internal node (nint + 1 entries)
  int32_t* node_item1 = nullptr;  // one past its last item
  int64_t n_big_items = 0;        // items [0, n_big_items): tiles of kAcaTile rows; then
  int64_t n_wide_items = 0;       // n_wide_items tiles of kWideTile rows; the rest: small nodes
  int32_t* wide_nodes = nullptr;  // ids of the nodes with wide items
  int32_t* node_witem0 = nullptr; // per node: its first wide item (-1: none), then one past
  int32_t* node_witem1 = nullptr; // its last
  double* wide_cross = nullptr;   // their cross-term chunks, ceil(max_rank / 128) each
  int n_wide_nodes = 0;
  std::vector<int64_t> h_raw_off; // offset (in doubles) of level j's raw panel
  std::vector<int> h_rcap;        // raw columns of level j
  double* raw = nullptr;
  int64_t raw_elems = 0;

  // ACA state, one entry per internal node
  int32_t* st_rank = nullptr;
  int32_t* st_row = nullptr;
  int32_t* st_col = nullptr;
  int32_t* st_done = nullptr;
  int32_t* st_ok = nullptr;
  int32_t* st_zero = nullptr;
  int32_t* st_phase = nullptr;
  int32_t* st_nused = nullptr;
  int32_t* st_used = nullptr;     // nint x (2 max_rank + 2)
  double* st_delta = nullptr;
  double* st_s2 = nullptr;
  double* aca_part = nullptr;     // n_items x (4 + 2 max_rank)
  int32_t* active = nullptr;      // device counter
  int32_t* h_active = nullptr;    // pinned host mirror

  // compact factor panels
  std::vector<int32_t> h_rank;    // per internal node
  std::vector<int> h_rl;          // per-level padded rank r_j
  std::vector<int> h_coff;        // column offset of level j (kappa + 1 entries)
  int R = 0;
  int64_t R_cap = 0;
  double* phi = nullptr;
  double* pan = nullptr;
  int32_t* rank_dev = nullptr;

  // factorization
  double* Y = nullptr;            // n x max_nrhs
  double* ysort = nullptr;        // copy of the first rhs (sorted) for the quadratic form
  double* leafL = nullptr;
  double* leaf_logdet = nullptr;  // 2^kappa
  double* node_logdet = nullptr;  // 2^kappa - 1
  double* Mlu = nullptr;          // level j at h_mlu_off[j]: (2 r_j)^2 per node
  int32_t* Mpiv = nullptr;        // level j at h_piv_off[j]: 2 r_j per node
  std::vector<int64_t> h_mlu_off, h_piv_off;
  int64_t mlu_cap = 0, piv_cap = 0;
  double* part = nullptr;         // leaf partial products, 2^kappa x part_stride
  int64_t part_stride = 0;
  double* part2 = nullptr;        // first-stage segment sums
  double* half = nullptr;         // per half-node sums (2^(j+1) x part_stride)
  double* Z = nullptr;            // two buffers of z_elems: Z of levels with even / odd index
  int64_t z_elems = 0;
  int32_t* cnt = nullptr;         // arrival counters of the fused level sweep
  // large-rank levels (levels_big.cu): per node sign and barrier counter (big_nodes each),
  // the panel kernel's published candidates, the substitution's row orders
  int32_t* big_i32 = nullptr;
  int64_t big_nodes = 0;
  double* big_slots = nullptr;
  int32_t* big_perm = nullptr;
  int64_t big_perm_cap = 0;
  int coop_cap = 0;               // co-resident CTAs of the cooperative panel launch
  double* split_buf = nullptr;    // split-K partial half-node sums of the product-form sweep
  int64_t split_cap = 0;
  int64_t fused_work = 0;         // largest per-block reduction of the fused sweep (values)
  int64_t half_elems = 0;
  double* scal = nullptr;         // [0] logdet, [1] quad, [2] loglik
  double* hyp = nullptr;          // device hyperparameter slot (kHyp* layout)
  int32_t* dflags = nullptr;
  double* tmpvec = nullptr;       // n x max_nrhs staging for host/device copies
  double* exp_tab = nullptr;      // 64 double-float pairs, 2^(j/64) (mixed form)
  double* xrel = nullptr;         // mixed form: kappa x d x n double-float pairs, each
                                  // point's coordinates relative to its level-j split point
  // iterative refinement (refine.cu): sorted right-hand sides and work vectors
  double refine_tol = 1e-10;
  int refine_maxit = 0;
  double* ry = nullptr;           // n x max_nrhs sorted right-hand sides (refine_maxit > 0)
  double* rw = nullptr;           // C~ x, then r and its correction (n), partials, ratio
  int refine_corr = 0;            // corrections taken by the last solve (all columns)
  double refine_res = 0.0;        // largest final ||y - C~ x|| / ||y|| of the last solve

  bool compressed = false;
  bool factored = false;
  int nrhs_fused = 0;
  bool rank_capped = false;
  bool presized = false;          // fixed per-level ranks, no host synchronisation
  // hyperparameter sweep: one captured evaluation replayed per setting
  int32_t* sweep_idx = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_valid = false;
  const void *g_theta = nullptr, *g_sigma2 = nullptr, *g_y = nullptr, *g_out = nullptr,
             *g_status = nullptr;
  int64_t graph_launches = 0, launches_captured = 0;
  // learned rank predictor
  double* boxes = nullptr;        // bounding box of every node's points
  float* feat = nullptr;          // block features (nint x 12) and predictions (nint)

  cudaEvent_t ev[8] = {};
  float phase_ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t launches = 0;   // kernels launched by this context
  int64_t syncs = 0;      // host synchronisations
  bool solve_timed = false;
  std::string last_error;
};

// Sweep step of level u (update of level u, half-node sums of level u - 1) in product form,
// when either level's rank is large. Level j's half sums then come straight from step j + 1,
// without per-leaf partials. The FP64 form always takes it there: its batched FP64 products
// run near the FP64 peak, while the per-leaf kernel spends about 8 FP64 instructions per
// dot product. The mixed form's per-leaf kernel works in double-float on the FP32 pipe and
// is faster at moderate ranks (2-D, n = 2^20, ranks up to 225: 1.52 against 2.01 s per
// evaluation) but far slower at ranks in the thousands (factor of the d = 4, n = 5000
// Gaussian row: 2.30 against 0.54 s), where it also loops over thousands of coarser panel
// columns per leaf. So it takes the product form from rank 512 or 1024 panel columns, or
// where its per-leaf partials would need more than 8 GB.
constexpr int kMixedProductRank = 512;
constexpr int kMixedProductCols = 1024;
inline bool gemm_step(const Ctx& c, int u) {
  const std::vector<int>& rl = c.h_rl;
  if (!(rl[u] >= kBlockRank || (u >= 1 && rl[u - 1] >= kBlockRank))) return false;
  if (c.precision == 0) return true;
  if (rl[u] >= kMixedProductRank || (u >= 1 && rl[u - 1] >= kMixedProductRank)) return true;
  if (c.h_coff[u] >= kMixedProductCols) return true;
  if (u < 1) return false;
  const double bytes = 8.0 * (double)((int64_t)1 << c.kappa) * rl[u - 1] * (c.h_coff[u] + c.max_nrhs);
  return bytes > 8e9;
}

// Launch wrappers (each .cu file defines its own); all are stream-ordered on ctx.stream.
cudaError_t launch_sort_1d(Ctx& c, const double* x_dev_rowmajor);
cudaError_t launch_sort_kd(Ctx& c, const double* x_dev_rowmajor);
cudaError_t launch_aca(Ctx& c, int* steps_out);
cudaError_t launch_cheb(Ctx& c);
size_t cheb_coef_elems(int nint);
cudaError_t launch_pack(Ctx& c);
cudaError_t launch_exp_table(Ctx& c);
cudaError_t launch_xrel(Ctx& c);
cudaError_t launch_gather_rhs(Ctx& c, const double* y, int64_t ld, int nrhs);
cudaError_t launch_scatter_rhs(Ctx& c, double* x, int64_t ld, int nrhs);
cudaError_t launch_leaf_factor(Ctx& c, int nrhs);
cudaError_t launch_leaf_factor_ff(Ctx& c, int nrhs);
// Batched evaluation: one persistent factor launch over the leaves of many contexts of one
// form. args: device array of nprob argument blocks (leaf_args_fill / leaf_args_fill_ff,
// leaf_args_bytes / leaf_args_bytes_ff each), first: device array of nprob + 1 leaf
// offsets (first[nprob] = total), counter: device int, zero before the launch.
size_t leaf_args_bytes();
size_t leaf_args_bytes_ff();
void leaf_args_fill(Ctx& c, int nrhs, void* out);
void leaf_args_fill_ff(Ctx& c, int nrhs, void* out);
cudaError_t launch_leaf_factor_multi(const void* args, const int32_t* first, int nprob, int total,
                                     int32_t* counter, int sms, cudaStream_t s);
cudaError_t launch_leaf_factor_multi_ff(const void* args, const int32_t* first, int nprob,
                                        int total, int32_t* counter, int sms, cudaStream_t s);
cudaError_t launch_leaf_solve_ff(Ctx& c, int nrhs);
cudaError_t launch_leaf_solve(Ctx& c, int nrhs);
cudaError_t launch_levels(Ctx& c, int nrhs, bool factor_mode);
cudaError_t launch_level_first(Ctx& c, int nrhs, bool factor_mode);
cudaError_t launch_levels_fused(Ctx& c, int nrhs, bool factor_mode);
struct NodeArgs;
cudaError_t big_setup(Ctx& c);
int64_t big_slot_elems(int coop_cap);
cudaError_t launch_node_blocked(Ctx& c, const NodeArgs& na, bool factor);
cudaError_t launch_sweep_gemm(Ctx& c, int u, int nrhs, bool factor_mode);
int half_sum_splits(const Ctx& c, int u, int w);
cudaError_t launch_logdet_sum(Ctx& c);
cudaError_t launch_quad_loglik(Ctx& c);
cudaError_t launch_matvec(Ctx& c, const double* xin_sorted, double* yout_sorted);
int64_t refine_work_elems(int64_t n);
int64_t predict_partial_elems(int64_t m);
cudaError_t launch_cross_dot(Ctx& c, const double* xt, int64_t j0, int nc, const double* W,
                             int64_t ldw, int wstep, double* partial, int mode, double* out);
cudaError_t launch_cross_fill(Ctx& c, const double* xt, int64_t j0, int nc);
cudaError_t launch_residual(Ctx& c, const double* y_sorted, double* ax, double* part, double* ratio);
cudaError_t launch_axpy(Ctx& c, double* x, const double* d);
cudaError_t launch_set_hyp(Ctx& c, double ell, double amp, double sigma2);
cudaError_t launch_block_features(Ctx& c, double ell, float* X, int64_t ld);
cudaError_t launch_mlp_forward(Ctx& c, hodlr_mlp* m, const float* X, int64_t N, float* Y);
cudaError_t launch_load_setting(Ctx& c, const double* theta, const double* sigma2,
                                const int32_t* idx);
cudaError_t launch_leaf_single(const double* xs_soa, int n, int d, int kind, const double* hyp,
                               const int32_t* nodes, double* Y, double* L, double* logdet,
                               int32_t* flags, cudaStream_t s);

}  // namespace hodlr

#define HODLR_CUDA_TRY(expr)                  \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return _e;         \
  } while (0)
