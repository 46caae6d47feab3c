/*
 * hodlr.h — C ABI of the GB300 (sm_103a) HODLR Gaussian-process solver.
 *
 * The library factors the covariance matrix C = sigma^2 I + K, K_ij = k(x_i, x_j), of a
 * Gaussian process into the hierarchical product C = K_kappa K_{kappa-1} ... K_1 K_0 of
 * Ambikasaran et al., "Fast Direct Methods for Gaussian Processes" (arXiv:1403.6015),
 * Sec. 3.2: K_kappa is block diagonal with the dense leaf blocks of C, and every other
 * factor is block diagonal with blocks I + [Ut 0; 0 Vt][0 V^T; U^T 0] (low-rank updates of
 * the identity). From it the library computes C^-1 y (Sherman-Morrison-Woodbury on each
 * factor, Sec. 3.2), log det C (Sylvester's determinant theorem on each factor, Sec. 4)
 * and the Gaussian log-likelihood (Sec. 1, Eq. 1).
 *
 * Conventions shared by every entry point:
 *   - Pointers to arrays may be host or device (CUDA) pointers; the library asks the CUDA
 *     runtime which one it was given. Host arrays are copied in and out inside the call,
 *     and a call that writes a host array returns only after the result is there. Device
 *     arrays are read and written in stream order on opts.stream and the call may return
 *     before the GPU is done.
 *   - Vectors and matrices are FP64. Matrices of right-hand sides and solutions are
 *     column-major, n rows, nrhs columns, leading dimension ld >= n.
 *   - y and x are in the caller's point order; the tree permutation is internal.
 *   - The context owns every buffer it allocates; the caller owns every pointer it passes.
 *   - Errors are return codes; nothing is thrown across the ABI. hodlr_last_error() gives
 *     a one-line description of the last failure on that context.
 *   - Sizes: 1 <= n < 2^31, 1 <= leaf <= 128, 1 <= d <= 64.
 */
#ifndef HODLR_GB300_H
#define HODLR_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hodlr_ctx hodlr_ctx; /* opaque; owns all device memory of one problem */
typedef struct hodlr_mlp hodlr_mlp; /* opaque; the learned rank predictor */

typedef enum {
  HODLR_OK = 0,
  HODLR_EINVAL = 1,   /* argument out of range or non-finite input */
  HODLR_ENOMEM = 2,   /* device allocation failed */
  HODLR_ENOTSPD = 3,  /* a leaf pivot or a factor determinant was not positive */
  HODLR_ERANK = 4,    /* compression hit opts.max_rank before reaching eps */
  HODLR_ETIMEOUT = 5, /* a bounded device wait gave up */
  HODLR_ESTATE = 6,   /* call out of order (e.g. solve before factor) */
  HODLR_ECUDA = 7     /* a CUDA runtime call failed */
} hodlr_status;

/* Covariance functions k(r) = a f(r / ell), theta = {ell, a} (Table 1 with a length scale
 * ell and amplitude a; Matern nu = 3/2 and 5/2 in closed form; nu = 1/2 is HODLR_K_EXP),
 * and the radial functions of Sec. 5 with t = r / ell. The multiquadric and biharmonic
 * give indefinite matrices: they factor with LU leaves and a signed log |det|
 * (hodlr_logdet_signed), need precision 0, and have no log-likelihood (EINVAL). */
typedef enum {
  HODLR_K_EXP = 0,      /* a exp(-r/ell)                              (Ornstein-Uhlenbeck) */
  HODLR_K_SE = 1,       /* a exp(-r^2/(2 ell^2))                      (Gaussian)           */
  HODLR_K_MATERN32 = 2, /* a (1 + sqrt3 r/ell) exp(-sqrt3 r/ell)                           */
  HODLR_K_MATERN52 = 3, /* a (1 + sqrt5 r/ell + 5r^2/(3ell^2)) exp(-sqrt5 r/ell)           */
  HODLR_K_RQ = 4,       /* a (1 + t^2)^-alpha, alpha = opts.rq_alpha   (rational quadratic)*/
  HODLR_K_IMQ = 5,      /* a / sqrt(1 + t^2)                     (inverse multiquadric)    */
  HODLR_K_MQ = 6,       /* a sqrt(1 + t^2)             (multiquadric; indefinite C)        */
  HODLR_K_BIHARMONIC = 7 /* a t^2 log t, 0 at t = 0    (thin-plate spline; indefinite C)   */
} hodlr_kernel;

typedef struct {
  int precision;       /* 0: FP64 throughout; 1: mixed: the leaf stage (block build,       */
                       /*    L D L^T, panel solves) in double-float arithmetic on the FP32 */
                       /*    pipe (~2^-48 unit roundoff), everything else FP64; it keeps  */
                       /*    per-level relative coordinates, kappa x d x n x 8 bytes     */
  int rank_mode;       /* 0: adaptive ACA ranks                                            */
  int max_rank;        /* cap on the ACA rank of one off-diagonal block (1..8192), default */
                       /*    64. Levels whose rank exceeds 64 factor their node matrices  */
                       /*    in global memory and use the unfused level sweep; from rank  */
                       /*    128 the node step is a blocked LU over many CTAs (a          */
                       /*    cooperative launch per panel) and the sweep a set of batched */
                       /*    FP64 products. Memory grows with max_rank (ACA columns        */
                       /*    n x min(max_rank, m/2) per level) and with the ranks reached  */
                       /*    (node matrices 2^j (2 r_j)^2 per level, half-node sums        */
                       /*    2^(j+1) r_j (R + max_nrhs), R the sum of the level ranks)      */
  int max_nrhs;        /* right-hand sides carried through a fused factor, default 16     */
  double refine_tol;   /* iterative refinement (not in the paper): stop when              */
                       /*    ||y - C~ x||_2 <= refine_tol ||y||_2, C~ the FP64 HODLR       */
                       /*    matrix (hodlr_matvec); default 1e-10, > 0 when refine_maxit>0 */
  int refine_maxit;    /* most correction solves per right-hand side after every solve   */
                       /*    (hodlr_factor_solve, hodlr_solve, hodlr_loglik and the sweep   */
                       /*    and batched forms); each is one matvec + one solve with the   */
                       /*    stored factor. 0 = off (default). The sweep and batched forms */
                       /*    and solves under stream capture take exactly refine_maxit     */
                       /*    corrections (no host check of the residual).                  */
  void* stream;        /* cudaStream_t for all device work; NULL = legacy default stream  */
  double rq_alpha;     /* exponent alpha > 0 of HODLR_K_RQ, default 1                      */
  int compression;     /* 0: adaptive cross approximation (default); 1: Chebyshev          */
                       /*    interpolation (Sec. 3.1's analytic A ~ E A~ P, barycentric    */
                       /*    form): q = 8..64 nodes per cluster, the first q whose last    */
                       /*    quarter of 2-D Chebyshev coefficients is below eps, then A~   */
                       /*    recompressed to rank by a fully pivoted cross. d = 1 only; no  */
                       /*    presize. A block needing more than 64 nodes (a kernel that is */
                       /*    not smooth where the clusters meet, or ell much shorter than  */
                       /*    the clusters) gets rank 0 and the build returns ERANK.         */
} hodlr_opts;

/* Fill *o with the defaults listed above. */
void hodlr_default_opts(hodlr_opts* o);

/* Point ordering and compression (paper: the "Assembly" column of Sec. 5).
 *   x      n points, row-major n x d (host or device). Copied; not kept.
 *   kernel covariance function; theta = {ell, a} (host pointer, 2 doubles), ell > 0, a > 0.
 *   sigma2 noise variance on the diagonal (>= 0).
 *   leaf   largest leaf block; the tree has kappa = ceil(log2(n / leaf)) levels (Sec. 3.2,
 *          pseudo-code figure, read so that no leaf exceeds `leaf` points).
 *   eps    ACA tolerance relative to each block's Frobenius norm (Sec. 3.1), > 0.
 *   o      options (NULL = defaults).
 * Sorts the points (Sec. 3: split by point count, one dimension at a time), then compresses
 * every off-diagonal block K[I_left, I_right] ~ U V^T by partial-pivoted adaptive cross
 * approximation. Synchronises opts.stream once (to size the rank pool).
 * Errors: EINVAL, ENOMEM, ERANK (rank cap reached; *out is still returned and usable),
 * ECUDA. On EINVAL/ENOMEM/ECUDA *out is NULL. */
hodlr_status hodlr_build(const double* x, int64_t n, int d, hodlr_kernel kernel,
                         const double* theta, double sigma2, int leaf, double eps,
                         const hodlr_opts* o, hodlr_ctx** out);

/* Recompress for new hyperparameters on the same points (the ordering is reused), as in a
 * hyperparameter sweep (Sec. 2.5). theta as in hodlr_build. Drops any factorization.
 * Errors: EINVAL, ENOMEM, ERANK, ECUDA. */
hodlr_status hodlr_rebuild(hodlr_ctx* ctx, const double* theta, double sigma2);

/* Factorization C = K_kappa ... K_0 (Sec. 3.2 and its pseudo-code figure): Cholesky of the
 * dense leaf blocks, their inverses applied to the ancestors' U/V rows, then level by level
 * from the finest internal level to the root the 2r x 2r matrices [I, V^T Vt; U^T Ut, I],
 * their LU factors and log dets. Synchronises once to check pivots.
 * Errors: ESTATE (already factored), ENOTSPD, ECUDA. */
hodlr_status hodlr_factor(hodlr_ctx* ctx);

/* Factor as above with nrhs right-hand sides y (n x nrhs, column stride ld) carried through
 * the same sweep, so that on return x = C^-1 y (the solve fused into the factorization).
 * nrhs <= opts.max_nrhs. Errors: EINVAL, ESTATE, ENOTSPD, ECUDA. */
hodlr_status hodlr_factor_solve(hodlr_ctx* ctx, const double* y, double* x, int nrhs,
                                int64_t ld);

/* x = C^-1 y with the stored factors: C^-1 = K_0^-1 K_1^-1 ... K_kappa^-1 (Sec. 3.2), each
 * inverse by the Sherman-Morrison-Woodbury formula. y and x may alias.
 * Errors: ESTATE (not factored), EINVAL, ECUDA. */
hodlr_status hodlr_solve(hodlr_ctx* ctx, const double* y, double* x, int nrhs, int64_t ld);

/* log det C = sum of the leaf log dets and of log det(I + W L) over all nodes (Sec. 4,
 * Sylvester's theorem and the product of block determinants), summed in a fixed order.
 * logdet is a host or device pointer to one double; for the indefinite kernels it receives
 * log |det C|. Errors: ESTATE, ENOTSPD, ECUDA. */
hodlr_status hodlr_logdet(hodlr_ctx* ctx, double* logdet);

/* log |det C| and its sign (+1 or -1; the product of the signs of the leaf and node
 * determinants, Sec. 4). For the positive definite kernels the sign is +1 and logabsdet
 * equals hodlr_logdet. logabsdet: host or device pointer; sign: host pointer.
 * Errors: ESTATE (not factored), EINVAL, ECUDA. */
hodlr_status hodlr_logdet_signed(hodlr_ctx* ctx, double* logabsdet, int* sign);

/* Gaussian log-likelihood of y (length n): -y^T C^-1 y / 2 - log det C / 2 - n log(2 pi) / 2
 * (Sec. 1, Eq. 1, with the normalising constant). If the context is not yet factored the
 * solve is fused into the factorization. out: host or device pointer to one double.
 * Errors: ENOTSPD, EINVAL (an indefinite kernel: C is not a covariance), ECUDA. */
hodlr_status hodlr_loglik(hodlr_ctx* ctx, const double* y, double* out);

/* Presized compression (no host synchronisation): fix the padded rank of every level,
 * level_ranks[j] for j = 0 .. kappa-1 (host array, 0 <= rank < opts.max_rank), e.g. from
 * a learned predictor or an earlier adaptive build (hodlr_ranks). Buffers are sized here;
 * later rebuilds run rank + 2 cross steps per level without reading anything back, and
 * factorizations skip their pivot check. A block whose ACA needs more than its level's
 * rank, or does not converge, sets bit 2 of the device flags (its result is then not
 * trustworthy: re-run that setting in adaptive mode); a non-positive pivot sets bit 1.
 * level_ranks = NULL returns to adaptive mode. Not for the indefinite kernels (EINVAL).
 * Errors: EINVAL, ENOMEM, ECUDA. */
hodlr_status hodlr_presize(hodlr_ctx* ctx, const int32_t* level_ranks, int nlevels);

/* Device flags accumulated since the last read (bit 1: a leaf pivot or node determinant
 * was not positive, or for an indefinite kernel was zero; bit 2: a presized rank was
 * exceeded or a block did not converge; bit 8: odd number of negative block determinants
 * of an indefinite kernel, i.e. det C < 0), into
 * *flags (host); clears them. Synchronises opts.stream. */
hodlr_status hodlr_status_flags(hodlr_ctx* ctx, int32_t* flags);

/* Log-likelihoods of nset hyperparameter settings on the same points and right-hand side
 * (a hyperparameter sweep, Sec. 2.5): for each setting b, recompression with
 * theta[2b], theta[2b+1] (ell, a) and sigma2[b], fused factorization and solve, log det
 * and log-likelihood -> out[b], and the device flags of that evaluation -> status[b]
 * (0 = valid; status may be NULL). All arrays are device pointers; y has n entries.
 * Requires presized mode and a non-default opts.stream. The first call captures one
 * evaluation as a CUDA graph (after one direct evaluation) and replays it for every other
 * setting; later calls with the same pointers replay it directly. Stream-ordered: the call
 * returns before the results are ready. Errors: ESTATE (not presized), EINVAL, ECUDA. */
hodlr_status hodlr_loglik_sweep(hodlr_ctx* ctx, int64_t nset, const double* theta,
                                const double* sigma2, const double* y, double* out,
                                int32_t* status);

/* One lane of a batched run: a presized context on a non-default stream, and the
 * settings it evaluates: b = first, first + stride, ..., count of them, each reading
 * theta[2b], theta[2b+1] (ell, a), sigma2[b], writing out[b] and status[b] (status may be
 * NULL). y is the context's right-hand side (its n entries). All arrays device pointers. */
typedef struct {
  hodlr_ctx* ctx;
  const double* theta;
  const double* sigma2;
  const double* y;
  double* out;
  int32_t* status;
  int64_t first, stride, count;
} hodlr_batch_lane;

/* Batched evaluation (many settings of one problem, or many independent problems of uneven
 * size): every lane evaluates its settings in rounds; one round of all lanes is captured as
 * a single CUDA graph and replayed for the remaining rounds. A round forks from `stream`
 * (cudaStream_t, not a lane's) into the lanes' streams for their compressions and
 * right-hand sides, joins into one persistent leaf-stage launch per form (FP64, mixed) in
 * which every CTA takes (lane, leaf) work items from a device counter until the leaves of
 * all lanes are factored and solved (Sec. 3.2's leaf factor K_kappa), and forks again for
 * each lane's level sweep, log det and log-likelihood before joining. The first round
 * runs directly (it sets kernel attributes). Lanes must use distinct contexts; lanes whose
 * contexts share a stream run one after another on it. No lane's stream may be `stream`
 * itself. The leaf work list lives in the first lane's context. Stream-ordered on `stream`.
 * Errors (message in the offending lane's hodlr_last_error): EINVAL, ENOMEM, ECUDA. */
hodlr_status hodlr_loglik_batched(const hodlr_batch_lane* lanes, int nlanes, void* stream);

/* ---- Learned rank predictor (not in the paper; sizes presized mode from features) ------
 * A multilayer perceptron 12 -> 64 -> 64 -> 1 (tanh hidden units, FP32) maps the features
 * of an off-diagonal block to log(1 + rank). Parameters: W1 (12 x 64, row-major by input),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1). Trained on the GPU (Adam, mean squared
 * error) on (features, rank) pairs that the FP64 compressor emits. */
int hodlr_mlp_num_params(void);   /* 5057 */
int hodlr_mlp_num_features(void); /* 12 */

/* Create with Glorot-uniform weights drawn from splitmix64(seed), zero biases; stream is a
 * cudaStream_t (NULL = default). */
hodlr_status hodlr_mlp_create(uint64_t seed, void* stream, hodlr_mlp** out);
void hodlr_mlp_destroy(hodlr_mlp* m);

/* Copy the parameters out (set = 0) or in (set = 1; resets the Adam state); params is a
 * host or device array of hodlr_mlp_num_params() floats. Synchronises. */
hodlr_status hodlr_mlp_params(hodlr_mlp* m, float* params, int set);

/* Y[i] = network(X[i, 0..12)), X device N x 12 row-major, Y device N. Stream-ordered. */
hodlr_status hodlr_mlp_forward(hodlr_mlp* m, const float* X, int64_t N, float* Y);

/* Gradient of the mean squared error (1/N) sum (Y - T)^2 with respect to the parameters
 * (grad: host or device, num_params floats; may be NULL), and the loss (host or device
 * float; may be NULL). X, T device. Synchronises. */
hodlr_status hodlr_mlp_gradient(hodlr_mlp* m, const float* X, const float* T, int64_t N,
                                float* grad, float* loss);

/* steps full-batch Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on (X, T); the final
 * loss into *loss (host or device; may be NULL). Synchronises. */
hodlr_status hodlr_mlp_train(hodlr_mlp* m, const float* X, const float* T, int64_t N,
                             int steps, float lr, float* loss);

/* Checkpoint file: "HODLRMLP", uint32 version 1, uint32 parameter count, FP32 parameters. */
hodlr_status hodlr_mlp_save(hodlr_mlp* m, const char* path);
hodlr_status hodlr_mlp_load(hodlr_mlp* m, const char* path);

/* Features of the 2^kappa - 1 off-diagonal blocks (level order) for length scale ell, into
 * the device array X (row stride ld >= 12): log(diam_L/ell), log(diam_R/ell),
 * log(|c_L - c_R|/ell), log2(m_L + m_R)/20, -log10(eps)/12, one-hot covariance (4), d - 1,
 * log(max diam / |c_L - c_R|), 0 (diam, c: bounding-box diagonal and centre of a child's
 * points). */
hodlr_status hodlr_block_features(hodlr_ctx* ctx, double ell, float* X, int64_t ld);

/* Predicted padded rank of every level for length scale ell: the largest predicted block
 * rank of the level plus margin, capped at max_rank - 1, into the host array level_ranks
 * (kappa entries), ready for hodlr_presize. Synchronises. */
hodlr_status hodlr_predict_ranks(hodlr_ctx* ctx, hodlr_mlp* mlp, double ell, int margin,
                                 int32_t* level_ranks);

/* Ranks of the 2^kappa - 1 off-diagonal blocks in level order (root first), into a host
 * array of capacity cap, as found by the last adaptive compression. Returns the number of
 * blocks via *count. Errors: EINVAL. */
hodlr_status hodlr_ranks(hodlr_ctx* ctx, int32_t* ranks, int64_t cap, int64_t* count);

/* Number of tree levels kappa, and the point permutation (sorted row i holds point
 * perm[i]) into a host array of n int64. Either output may be NULL. */
hodlr_status hodlr_tree(hodlr_ctx* ctx, int* kappa, int64_t* perm);

/* C~ x with the compressed operator (dense leaves + U V^T blocks), x and y of length n. */
hodlr_status hodlr_matvec(hodlr_ctx* ctx, const double* x, double* y);

/* Device time in milliseconds (CUDA events on opts.stream) of the last calls, into a host
 * array of 6 floats: out[0] ordering, out[1] compression, out[2] factorization (all of
 * it), out[3] last standalone solve, out[4] the leaf kernel of the last factorization,
 * out[5] the level sweep and log det of the last factorization. */
hodlr_status hodlr_phase_ms(hodlr_ctx* ctx, float* out6);

/* Counters since hodlr_build, into a host array of 2 int64: out[0] CUDA kernels this
 * context launched, out[1] host synchronisations it performed. */
hodlr_status hodlr_counters(hodlr_ctx* ctx, int64_t* out2);

/* Launch configuration of a context (not in the paper; nothing here changes what is
 * computed, only how the work maps onto the GPU).
 *   leaf_threads  CTA size of this context's leaf kernel: FP64 form 256, 512 or 1024;
 *                 mixed form 512 (two leaves per SM) or 1024 (one).
 *   sweep_mode    0: one launch per level when every level's reductions fit a block and
 *                 no rank exceeds 64, else the segmented sweep; 1: always segmented.
 *   leaf_kernel   mixed form only: 0 = every leaf operation in double-float on the FP32
 *                 pipe; 1 = the trailing updates of the leaf factorization and the
 *                 off-diagonal block updates of its solves as exact bf16-slice products
 *                 on the tensor cores (512 threads, two leaves per SM; leaf_threads is
 *                 then ignored). Must be 0 in the FP64 form.
 *   sweep_tile    tile shape of the one-launch-per-level sweep (sweep_mode 0): leaves and
 *                 threads per block, 0: 4 x 256, 1: 2 x 128, 2: 8 x 256, 3: 8 x 512,
 *                 4: 2 x 64, 5: 1 x 64, 6: 1 x 128. */
typedef struct {
  int leaf_threads;
  int sweep_mode;
  int leaf_kernel;
  int sweep_tile;
} hodlr_tuning;

/* Read or set the launch configuration. Errors: EINVAL (a value outside the lists). */
hodlr_status hodlr_get_tuning(hodlr_ctx* ctx, hodlr_tuning* out);
hodlr_status hodlr_set_tuning(hodlr_ctx* ctx, const hodlr_tuning* t);

/* Autotuner: time every candidate configuration (leaf CTA sizes and, in the mixed form,
 * the tensor-core leaf kernel, each with the segmented sweep and with every tile shape of
 * the one-launch-per-level sweep) on this
 * context's own problem (one fused factorization with the right-hand side y, n doubles,
 * host or device), each reps times after one untimed run, with CUDA events on
 * opts.stream; keep the fastest (lowest median) and write it to *best (may be NULL) and
 * its median milliseconds to *best_ms (may be NULL). The context must be compressed; it
 * is left compressed and unfactored. Results do not depend on the configuration beyond
 * the order of a few fixed-order sums (last bits). Errors: EINVAL, ESTATE, ENOTSPD, ECUDA. */
hodlr_status hodlr_autotune(hodlr_ctx* ctx, const double* y, int reps, hodlr_tuning* best,
                            float* best_ms);

/* GP prediction with the factorization (the conditional distribution behind the
 * likelihood of Sec. 1; the standard GP regression formulas): at each test point x*,
 * mean = k_*^T C^-1 y and the latent variance var = k(x*, x*) - k_*^T C^-1 k_*, with
 * k_* = (k(x_i, x*))_i over the training points. The solves use the stored factorization
 * (without refinement); the cross-covariances are evaluated in FP64.
 *   xtest  m test points, row-major m x d (host or device)
 *   y      the n training targets in the order of hodlr_build's x (host or device)
 *   mean   m doubles out (host or device); var m doubles out, or NULL for the mean only
 * Requires a factored context (hodlr_factor, hodlr_factor_solve or hodlr_loglik); the
 * factorization is not changed. Synchronises the stream before returning.
 * Errors: EINVAL, ESTATE (not factored, or under stream capture), ENOMEM, ECUDA. */
hodlr_status hodlr_predict(hodlr_ctx* ctx, const double* xtest, int64_t m, const double* y,
                           double* mean, double* var);

/* Iterative refinement of the last solve (opts.refine_maxit > 0; not in the paper): the
 * corrections it took over all right-hand sides, and the largest final relative residual
 * ||y - C~ x|| / ||y|| it measured (0 when refinement is off or ran without host checks).
 * Either output may be NULL. Errors: EINVAL. */
hodlr_status hodlr_refine_info(hodlr_ctx* ctx, int32_t* corrections, double* residual);

/* Log-likelihood of a problem small enough to be one leaf block, with no device
 * allocation. The paper has no counterpart: this entry exists for callers that must not
 * allocate device memory while they evaluate, such as sampling loops under a fixed memory
 * budget or code recorded into a CUDA graph that should hold no allocation nodes.
 *   x      device pointer, n points row-major n x d (d in {1, 2, 3}); y device pointer (n);
 *   out    device pointer to one double: -y^T C^-1 y/2 - log det C/2 - n log(2 pi)/2, or
 *          NaN if C is not positive definite;
 *   stream cudaStream_t (NULL = legacy default stream); the call is stream-ordered and
 *          does not synchronise.
 *   kernel the four covariances of Table 1 only (HODLR_K_EXP, HODLR_K_SE,
 *          HODLR_K_MATERN32, HODLR_K_MATERN52); any other kind returns HODLR_EINVAL.
 * Limits: 1 <= n <= 128; larger n returns HODLR_EINVAL, as do host pointers.
 * Scratch: a fixed 136,384-byte array in device global memory that every GPU loading the
 * library holds until exit. The first call on a device looks up its address (with that
 * device current), so make that first call before any stream capture; calls outside a
 * capture look it up again, so the address stays valid across a device reset, but a
 * capture begun after a reset must again follow one uncaptured call. All calls on a
 * device share the array: calls that overlap on the GPU race. */
hodlr_status hodlr_loglik_small_noalloc(const double* x, int64_t n, int d, hodlr_kernel kernel,
                                        const double* theta, double sigma2, const double* y,
                                        double* out, void* stream);

const char* hodlr_last_error(const hodlr_ctx* ctx);
const char* hodlr_status_string(hodlr_status s);

/* Frees all device memory of the context. NULL is ignored. */
void hodlr_destroy(hodlr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HODLR_GB300_H */
