/*
 * ORACLE — test infrastructure only. A plain, slow, FP64 CPU statement of what the GPU
 * path computes, written from the paper (Ambikasaran, Foreman-Mackey, Greengard, Hogg,
 * O'Neil, "Fast Direct Methods for Gaussian Processes", arXiv:1403.6015). Only the tests,
 * the smoke check and the bench's CPU-baseline leg may load it. It shares no code,
 * header, table or constant with the CUDA library: it includes libc and libm only.
 *
 * Contents (each function cites the passage it follows):
 *   - covariance functions (Table 1; Sec. 5, entries C_ij = s_i delta_ij + k(r_i, r_j))
 *   - O1: dense Cholesky solve and log det of C = sigma^2 I + K (the plain definition, Sec. 1)
 *   - exact sampled rows of C v (residual checks at any n)
 *   - Ornstein-Uhlenbeck closed form (tridiagonal inverse; textbook, not in the paper)
 *   - Kalman filter for half-integer Matern (state-space form cited in Sec. 2.3)
 *   - O2: the HODLR method, step by step: point ordering (Sec. 3), adaptive cross
 *     approximation with partial pivoting (Sec. 3.1), factorization K = K_kappa...K_0
 *     (Sec. 3.2, Eq. for the HODLR factorization and the pseudo-code figure), solve by
 *     Sherman-Morrison-Woodbury per factor (Sec. 3.2), determinant by Sylvester's
 *     theorem (Sec. 4), plus the HODLR matrix-vector product.
 *
 * Parity status: every function here is pinned by a test in tests/test_oracle_*.py
 * against a closed form, a library routine of a different algorithm, brute force or an
 * identity. None is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_EXP = 0, ORC_SE = 1, ORC_M32 = 2, ORC_M52 = 3, ORC_RQ = 4, ORC_IMQ = 5, ORC_MQ = 6,
       ORC_BH = 7 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOTSPD = 3, ORC_ERANK = 4, ORC_ESTATE = 6 };
/* Largest point dimension accepted (the high-dimension experiments of Sec. 5 go to 64). */
#define ORC_MAX_D 64

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads used by the parallel loops that follow (t < 1: all host cores). Timing only;
 * every result is independent of the thread count. */
void oracle_set_num_threads(int t) {
#ifdef _OPENMP
  omp_set_num_threads(t >= 1 ? t : omp_get_num_procs());
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------------------
 * Covariance functions. k(r) = a f(r / ell), r the Euclidean distance (Table 1 with a
 * length scale ell and amplitude a; Matern nu = 3/2 and 5/2 in their closed forms), and
 * the radial functions of Sec. 5 with the distance in units of ell: rational quadratic
 * (1 + r^2)^-alpha (Table 1), inverse multiquadric 1/sqrt(1 + r^2), multiquadric
 * sqrt(1 + r^2) (the form of Sec. 5's text; its table caption prints sqrt(1 + r)), and
 * biharmonic r^2 log r (0 at r = 0, its limit). The last two give indefinite matrices.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int kind;
  double ell, amp, alpha; /* alpha: the rational quadratic's exponent */
} orc_cov;

/* theta = {ell, a} (and alpha third for the rational quadratic). */
static orc_cov orc_cov_make(int kind, const double* theta) {
  orc_cov k;
  k.kind = kind;
  k.ell = theta[0];
  k.amp = theta[1];
  k.alpha = kind == ORC_RQ ? theta[2] : 1.0;
  return k;
}

static int orc_indefinite(int kind) { return kind == ORC_MQ || kind == ORC_BH; }

/* r is the distance, r2 its square (both passed so neither is recomputed from the other). */
static double orc_kernel(const orc_cov* k, double r, double r2) {
  double ell = k->ell, amp = k->amp;
  switch (k->kind) {
    case ORC_EXP: return amp * exp(-r / ell);
    case ORC_SE: return amp * exp(-0.5 * r2 / (ell * ell));
    case ORC_M32: {
      double s = sqrt(3.0) * r / ell;
      return amp * (1.0 + s) * exp(-s);
    }
    case ORC_M52: {
      double s = sqrt(5.0) * r / ell;
      return amp * (1.0 + s + s * s / 3.0) * exp(-s);
    }
    case ORC_RQ: return amp * pow(1.0 + r2 / (ell * ell), -k->alpha);
    case ORC_IMQ: return amp / sqrt(1.0 + r2 / (ell * ell));
    case ORC_MQ: return amp * sqrt(1.0 + r2 / (ell * ell));
    case ORC_BH: {
      if (!(r > 0.0)) return 0.0;
      double t = r / ell;
      return amp * t * t * log(t);
    }
  }
  return NAN;
}

/* k(x_i, x_j): in 1-D r = |x_i - x_j|, otherwise r = sqrt(sum of squared differences). */
static double orc_kij(const double* x, int d, const orc_cov* k, int64_t i, int64_t j) {
  if (d == 1) {
    double r = fabs(x[i] - x[j]);
    return orc_kernel(k, r, r * r);
  }
  double s = 0.0;
  for (int c = 0; c < d; ++c) {
    double t = x[i * d + c] - x[j * d + c];
    s += t * t;
  }
  return orc_kernel(k, sqrt(s), s);
}

/* Entry of C = sigma^2 I + K (Sec. 5, C_ij = sigma^2 delta_ij + k(r_i, r_j)). */
static double orc_entry(const double* x, int d, const orc_cov* k, double sigma2, int64_t i,
                        int64_t j) {
  double v = orc_kij(x, d, k, i, j);
  return i == j ? v + sigma2 : v;
}

void oracle_kernel_values(int kind, const double* r, int64_t m, const double* theta, double* out) {
  orc_cov k = orc_cov_make(kind, theta);
  for (int64_t i = 0; i < m; ++i) out[i] = orc_kernel(&k, r[i], r[i] * r[i]);
}

/* ------------------------------------------------------------------------------------
 * O1: dense Cholesky C = L L^T, x = L^-T L^-1 y, log det C = 2 sum log L_jj.
 * Column-by-column (left-looking) so each entry is one dot product of two rows of L.
 * ---------------------------------------------------------------------------------- */
static double dot4(const double* a, const double* b, int64_t m) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int64_t k = 0;
  for (; k + 4 <= m; k += 4) {
    s0 += a[k] * b[k];
    s1 += a[k + 1] * b[k + 1];
    s2 += a[k + 2] * b[k + 2];
    s3 += a[k + 3] * b[k + 3];
  }
  for (; k < m; ++k) s0 += a[k] * b[k];
  return (s0 + s1) + (s2 + s3);
}

int oracle_dense_solve(const double* x, int64_t n, int d, int kind, const double* theta,
                       double sigma2, const double* y, int nrhs, int64_t ldy, double* xout,
                       int64_t ldx, double* logdet) {
  if (n < 1 || d < 1) return ORC_EINVAL;
  orc_cov k = orc_cov_make(kind, theta);
  double* L = (double*)malloc(sizeof(double) * n * n);
  if (!L) return ORC_ENOMEM;
  /* lower triangle of C, row-major */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j <= i; ++j) L[i * n + j] = orc_entry(x, d, &k, sigma2, i, j);
  int bad = 0;
  for (int64_t j = 0; j < n && !bad; ++j) {
    double djj = L[j * n + j] - dot4(L + j * n, L + j * n, j);
    if (!(djj > 0.0)) { bad = 1; break; }
    double ljj = sqrt(djj);
    L[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i)
      L[i * n + j] = (L[i * n + j] - dot4(L + i * n, L + j * n, j)) / ljj;
  }
  if (bad) { free(L); return ORC_ENOTSPD; }
  double ld = 0.0;
  for (int64_t j = 0; j < n; ++j) ld += log(L[j * n + j]);
  *logdet = 2.0 * ld;
  double* z = (double*)malloc(sizeof(double) * n);
  for (int c = 0; c < nrhs; ++c) {
    const double* b = y + (int64_t)c * ldy;
    for (int64_t i = 0; i < n; ++i) z[i] = (b[i] - dot4(L + i * n, z, i)) / L[i * n + i];
    double* xo = xout + (int64_t)c * ldx;
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = z[i];
      for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * xo[k];
      xo[i] = s / L[i * n + i];
    }
  }
  free(z);
  free(L);
  return ORC_OK;
}

/* Exact rows of C v: out[t] = sum_j C[rows[t], j] v[j], Neumaier-compensated. */
void oracle_dense_matvec_rows(const double* x, int64_t n, int d, int kind, const double* theta,
                              double sigma2, const double* v, const int64_t* rows, int64_t nrows,
                              double* out) {
  orc_cov k = orc_cov_make(kind, theta);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nrows; ++t) {
    int64_t i = rows[t];
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double term = orc_entry(x, d, &k, sigma2, i, j) * v[j];
      double u = s + term;
      if (fabs(s) >= fabs(term)) c += (s - u) + term; else c += (term - u) + s;
      s = u;
    }
    out[t] = s + c;
  }
}

/* ------------------------------------------------------------------------------------
 * Ornstein-Uhlenbeck closed form (exponential kernel in 1-D; a textbook Markov identity
 * used as an independent check). Sorted points, rho_i = exp(-(x_{i+1}-x_i)/ell),
 * q_i = 1 - rho_i^2 = -expm1(-2 d_i / ell). R = K / a has the tridiagonal inverse
 *   T_11 = 1/q_1, T_nn = 1/q_{n-1}, T_ii = 1/q_{i-1} + 1/q_i - 1, T_{i,i+1} = -rho_i/q_i,
 * log det R = sum log q_i, C = a R (I + (sigma^2/a) T), C^-1 y = (I + (sigma^2/a) T)^-1 T y / a.
 * ---------------------------------------------------------------------------------- */
int oracle_ou_closed_form(const double* xs, int64_t n, double ell, double amp, double sigma2,
                          const double* ys, int nrhs, int64_t ldy, double* xout, int64_t ldx,
                          double* logdet) {
  if (n < 1) return ORC_EINVAL;
  if (n == 1) {
    *logdet = log(amp + sigma2);
    for (int c = 0; c < nrhs; ++c) xout[(int64_t)c * ldx] = ys[(int64_t)c * ldy] / (amp + sigma2);
    return ORC_OK;
  }
  double* rho = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  double* diag = (double*)malloc(sizeof(double) * n);
  double* off = (double*)malloc(sizeof(double) * n);
  double* dd = (double*)malloc(sizeof(double) * n);
  double* ll = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double ldr = 0.0;
  for (int64_t i = 0; i + 1 < n; ++i) {
    double di = xs[i + 1] - xs[i];
    rho[i] = exp(-di / ell);
    q[i] = -expm1(-2.0 * di / ell);
    if (!(q[i] > 0.0)) { ldr = NAN; }
    ldr += log(q[i]);
  }
  /* T entries */
  for (int64_t i = 0; i < n; ++i) {
    double t = 0.0;
    if (i == 0) t = 1.0 / q[0];
    else if (i == n - 1) t = 1.0 / q[n - 2];
    else t = 1.0 / q[i - 1] + 1.0 / q[i] - 1.0;
    diag[i] = t;
    if (i + 1 < n) off[i] = -rho[i] / q[i];
  }
  /* B = I + s T, s = sigma^2 / a; LDL^T of the tridiagonal B */
  double s = sigma2 / amp;
  double ldb = 0.0;
  dd[0] = 1.0 + s * diag[0];
  for (int64_t i = 0; i + 1 < n; ++i) {
    double b_off = s * off[i];
    ll[i] = b_off / dd[i];
    dd[i + 1] = 1.0 + s * diag[i + 1] - ll[i] * b_off;
  }
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(dd[i] > 0.0)) bad = 1;
    ldb += log(dd[i]);
  }
  *logdet = (double)n * log(amp) + ldr + ldb;
  for (int c = 0; c < nrhs; ++c) {
    const double* yc = ys + (int64_t)c * ldy;
    double* xc = xout + (int64_t)c * ldx;
    /* w = T y */
    for (int64_t i = 0; i < n; ++i) {
      double t = diag[i] * yc[i];
      if (i > 0) t += off[i - 1] * yc[i - 1];
      if (i + 1 < n) t += off[i] * yc[i + 1];
      w[i] = t / amp;
    }
    /* solve L D L^T x = w */
    for (int64_t i = 1; i < n; ++i) w[i] -= ll[i - 1] * w[i - 1];
    for (int64_t i = 0; i < n; ++i) w[i] /= dd[i];
    for (int64_t i = n - 2; i >= 0; --i) w[i] -= ll[i] * w[i + 1];
    memcpy(xc, w, sizeof(double) * n);
  }
  free(rho); free(q); free(diag); free(off); free(dd); free(ll); free(w);
  return bad ? ORC_ENOTSPD : ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Kalman filter for Matern nu = 1/2, 3/2, 5/2 (the state-space family cited in Sec. 2.3;
 * textbook, not in the paper). State s = (f, f', ...), ds = F s dt + noise, with
 * lambda = sqrt(2 nu)/ell and characteristic polynomial (s + lambda)^q. F = -lambda I + N,
 * N nilpotent, so expm(F D) = exp(-lambda D)(I + N D + N^2 D^2 / 2) exactly. P_inf is the
 * stationary covariance of (f, f', f''), Q = P_inf - A P_inf A^T. Returns log det C and
 * y^T C^-1 y from the innovations: sum log S_k and sum v_k^2 / S_k.
 * ---------------------------------------------------------------------------------- */
int oracle_matern_kalman(const double* xs, int64_t n, int nu2, double ell, double amp,
                         double sigma2, const double* ys, double* logdet, double* quad) {
  int q = (nu2 + 1) / 2; /* state dimension: 1, 2, 3 */
  if (n < 1 || (nu2 != 1 && nu2 != 3 && nu2 != 5)) return ORC_EINVAL;
  double lam = sqrt((double)nu2) / ell;
  double F[3][3] = {{0}}, Pinf[3][3] = {{0}};
  if (q == 1) {
    F[0][0] = -lam;
    Pinf[0][0] = amp;
  } else if (q == 2) {
    F[0][1] = 1.0; F[1][0] = -lam * lam; F[1][1] = -2.0 * lam;
    Pinf[0][0] = amp; Pinf[1][1] = amp * lam * lam;
  } else {
    F[0][1] = 1.0; F[1][2] = 1.0;
    F[2][0] = -lam * lam * lam; F[2][1] = -3.0 * lam * lam; F[2][2] = -3.0 * lam;
    Pinf[0][0] = amp; Pinf[1][1] = amp * lam * lam / 3.0; Pinf[2][2] = amp * lam * lam * lam * lam;
    Pinf[0][2] = Pinf[2][0] = -amp * lam * lam / 3.0;
  }
  double Nm[3][3], N2[3][3];
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) Nm[i][j] = F[i][j] + (i == j ? lam : 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double t = 0;
      for (int k = 0; k < q; ++k) t += Nm[i][k] * Nm[k][j];
      N2[i][j] = t;
    }
  double m[3] = {0, 0, 0}, P[3][3];
  memcpy(P, Pinf, sizeof(P));
  double ld = 0.0, qd = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0) {
      double D = xs[k] - xs[k - 1];
      double e = exp(-lam * D);
      double A[3][3], T[3][3], Pn[3][3], Qm[3][3], mn[3];
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j)
          A[i][j] = e * ((i == j ? 1.0 : 0.0) + Nm[i][j] * D + 0.5 * N2[i][j] * D * D);
      /* Q = Pinf - A Pinf A^T */
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          double t = 0;
          for (int l = 0; l < q; ++l) t += A[i][l] * Pinf[l][j];
          T[i][j] = t;
        }
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          double t = 0;
          for (int l = 0; l < q; ++l) t += T[i][l] * A[j][l];
          Qm[i][j] = Pinf[i][j] - t;
        }
      /* P = A P A^T + Q, m = A m */
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          double t = 0;
          for (int l = 0; l < q; ++l) t += A[i][l] * P[l][j];
          T[i][j] = t;
        }
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          double t = 0;
          for (int l = 0; l < q; ++l) t += T[i][l] * A[j][l];
          Pn[i][j] = t + Qm[i][j];
        }
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) P[i][j] = 0.5 * (Pn[i][j] + Pn[j][i]);
      for (int i = 0; i < q; ++i) {
        double t = 0;
        for (int l = 0; l < q; ++l) t += A[i][l] * m[l];
        mn[i] = t;
      }
      for (int i = 0; i < q; ++i) m[i] = mn[i];
    }
    double S = P[0][0] + sigma2;
    double v = ys[k] - m[0];
    if (!(S > 0.0)) return ORC_ENOTSPD;
    ld += log(S);
    qd += v * v / S;
    double Kg[3];
    for (int i = 0; i < q; ++i) Kg[i] = P[i][0] / S;
    for (int i = 0; i < q; ++i) m[i] += Kg[i] * v;
    double Pn[3][3];
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) Pn[i][j] = P[i][j] - Kg[i] * S * Kg[j];
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) P[i][j] = 0.5 * (Pn[i][j] + Pn[j][i]);
  }
  *logdet = ld;
  *quad = qd;
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Small dense LU with partial pivoting (row-major, in place). Used for the leaf blocks
 * and the 2r x 2r node matrices. Returns log|det|, writes the sign to *sign, returns
 * -INFINITY for an exactly singular matrix.
 * ---------------------------------------------------------------------------------- */
static double orc_lu(double* A, int m, int* piv, int* sign) {
  int sg = 1;
  double ld = 0.0;
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(A[k * m + k]);
    for (int i = k + 1; i < m; ++i)
      if (fabs(A[i * m + k]) > best) { best = fabs(A[i * m + k]); p = i; }
    piv[k] = p;
    if (p != k) {
      sg = -sg;
      for (int j = 0; j < m; ++j) {
        double t = A[k * m + j];
        A[k * m + j] = A[p * m + j];
        A[p * m + j] = t;
      }
    }
    double akk = A[k * m + k];
    if (akk == 0.0) { *sign = 0; return -INFINITY; }
    if (akk < 0) sg = -sg;
    ld += log(fabs(akk));
    for (int i = k + 1; i < m; ++i) {
      double l = A[i * m + k] / akk;
      A[i * m + k] = l;
      for (int j = k + 1; j < m; ++j) A[i * m + j] -= l * A[k * m + j];
    }
  }
  *sign = sg;
  return ld;
}

/* Solve A z = b in place with the factors of orc_lu; b has stride `inc`. */
static void orc_lu_solve(const double* A, int m, const int* piv, double* b, int64_t inc) {
  for (int k = 0; k < m; ++k)
    if (piv[k] != k) {
      double t = b[k * inc];
      b[k * inc] = b[piv[k] * inc];
      b[piv[k] * inc] = t;
    }
  for (int i = 1; i < m; ++i) {
    double s = b[i * inc];
    for (int k = 0; k < i; ++k) s -= A[i * m + k] * b[k * inc];
    b[i * inc] = s;
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i * inc];
    for (int k = i + 1; k < m; ++k) s -= A[i * m + k] * b[k * inc];
    b[i * inc] = s / A[i * m + i];
  }
}

/* Test hooks for the Sylvester and Sherman-Morrison-Woodbury identities (Sec. 4, Sec. 3.2). */
double oracle_lu_logdet(const double* A, int m, int* sign) {
  double* W = (double*)malloc(sizeof(double) * m * m);
  int* piv = (int*)malloc(sizeof(int) * (m > 0 ? m : 1));
  memcpy(W, A, sizeof(double) * m * m);
  double ld = orc_lu(W, m, piv, sign);
  free(W);
  free(piv);
  return ld;
}

void oracle_lu_solve_dense(const double* A, int m, const double* b, double* x) {
  double* W = (double*)malloc(sizeof(double) * m * m);
  int* piv = (int*)malloc(sizeof(int) * (m > 0 ? m : 1));
  int sg;
  memcpy(W, A, sizeof(double) * m * m);
  orc_lu(W, m, piv, &sg);
  memcpy(x, b, sizeof(double) * m);
  orc_lu_solve(W, m, piv, x, 1);
  free(W);
  free(piv);
}

/* O1 for any C, positive definite or not: the dense matrix, LU with partial pivoting,
 * x = C^-1 y, log |det C| and its sign. Limited to n < 46341 (m^2 in int). */
int oracle_dense_lu_solve(const double* x, int64_t n, int d, int kind, const double* theta,
                          double sigma2, const double* y, int nrhs, int64_t ldy, double* xout,
                          int64_t ldx, double* logabsdet, int* sign) {
  if (n < 1 || d < 1 || n > 46340) return ORC_EINVAL;
  orc_cov k = orc_cov_make(kind, theta);
  int m = (int)n;
  double* A = (double*)malloc(sizeof(double) * n * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  if (!A || !piv) { free(A); free(piv); return ORC_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) A[i * n + j] = orc_entry(x, d, &k, sigma2, i, j);
  int sg = 1;
  double ld = orc_lu(A, m, piv, &sg);
  *logabsdet = ld;
  *sign = sg;
  if (sg == 0) { free(A); free(piv); return ORC_ENOTSPD; }
  for (int c = 0; c < nrhs; ++c) {
    double* xo = xout + (int64_t)c * ldx;
    memcpy(xo, y + (int64_t)c * ldy, sizeof(double) * n);
    orc_lu_solve(A, m, piv, xo, 1);
  }
  free(A);
  free(piv);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * O2: the HODLR method.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  int d, kind, leaf, max_rank, kappa;
  orc_cov cov;
  double sigma2, eps;
  int logdet_sign; /* sign of det C (indefinite kernels; +1 otherwise) */
  double* xs;      /* sorted points, n x d row-major */
  int64_t* perm;   /* sorted row i is original point perm[i] */
  int64_t* nb;     /* node begin, node id (j, k) -> (1 << j) - 1 + k */
  int64_t* ns;     /* node size */
  int* rank;       /* internal nodes */
  int* aca_ok;     /* 1 if the node converged to eps below the rank cap */
  double** U;      /* left factor, m_left x r, column-major */
  double** V;      /* right factor, m_right x r, column-major */
  double** Ut;     /* transformed copies (inverse of the finer factors applied) */
  double** Vt;
  double** leafLU; /* row-major LU of each leaf block */
  int** leafpiv;
  double* leaflogdet;
  double** Mlu;    /* LU of each node's 2r x 2r matrix */
  int** Mpiv;
  double* nodelogdet;
  double logdet;
  int factored;
} orc_hodlr;

/* Sort (key, original index) pairs: ties broken by the original index. */
typedef struct { double key; int64_t idx; } orc_pair;
static int orc_pair_cmp(const void* a, const void* b) {
  const orc_pair* p = (const orc_pair*)a;
  const orc_pair* q = (const orc_pair*)b;
  if (p->key < q->key) return -1;
  if (p->key > q->key) return 1;
  return (p->idx > q->idx) - (p->idx < q->idx);
}

int oracle_kappa(int64_t n, int leaf) {
  /* Number of levels: smallest kappa with n <= leaf * 2^kappa, so every leaf has at most
   * `leaf` points (reading of kappa = floor(log2 n / p_max) in the pseudo-code figure,
   * whose floor would allow leaves of up to 2 p_max points). */
  int k = 0;
  while ((int64_t)leaf << k < n) ++k;
  return k;
}

/* Point ordering (Sec. 3): recursive median split by point count, one dimension at a
 * time (dimension = depth mod d), left child = first floor(m/2) points. In 1-D this is a
 * plain sort. perm must hold 0..n-1 on entry; it is reordered in place. */
static void orc_kd_order(const double* x, int d, int64_t* perm, int64_t begin, int64_t size,
                         int depth, int kappa, orc_pair* scratch) {
  int dim = depth % d;
  for (int64_t t = 0; t < size; ++t) {
    scratch[t].key = x[perm[begin + t] * d + dim];
    scratch[t].idx = perm[begin + t];
  }
  qsort(scratch, (size_t)size, sizeof(orc_pair), orc_pair_cmp);
  for (int64_t t = 0; t < size; ++t) perm[begin + t] = scratch[t].idx;
  if (d == 1 || depth + 1 >= kappa) return;
  int64_t ml = size / 2;
  orc_kd_order(x, d, perm, begin, ml, depth + 1, kappa, scratch);
  orc_kd_order(x, d, perm, begin + ml, size - ml, depth + 1, kappa, scratch);
}

void oracle_tree_order(const double* x, int64_t n, int d, int leaf, int64_t* perm) {
  int kappa = oracle_kappa(n, leaf);
  orc_pair* scratch = (orc_pair*)malloc(sizeof(orc_pair) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  orc_kd_order(x, d, perm, 0, n, 0, kappa > 0 ? kappa : 1, scratch);
  free(scratch);
}

/* Adaptive cross approximation with partial pivoting of the block
 * B(a, b) = k(xs[bl + a], xs[br + b]), a < ml, b < mr (Sec. 3.1; the paper defers the
 * listing to its reference, so this follows the standard partial-pivoted ACA):
 *   residual row R(i,:) = B(i,:) - sum_l u_l(i) v_l^T; pivot column j = argmax |R(i,:)|;
 *   v = R(i,:) / R(i,j); u = residual column R(:,j); next row = argmax over unused rows of
 *   |u|. Frobenius norm of S_k = sum u_l v_l^T kept incrementally; stop (without keeping
 *   the term) when |u_k| |v_k| <= eps |S_k|_F. Returns the rank; *ok = 0 if the cap was
 *   reached before the tolerance. Ties in argmax take the lowest index.
 * Start row and zero pivots (reading; the paper does not fix them): the cross starts at
 *   the first row; a zero pivot marks the row used and moves to the unused row nearest the
 *   right child's first point (squared Euclidean distance, lowest index on ties). Rows far
 *   from the interface of a fast-decaying kernel can be exactly zero in floating point;
 *   moving on to the next rows by index would reach only more of them and end the cross
 *   with rank 0 on a block that has entries of order one near the interface. */
static double orc_d2_split(const orc_hodlr* H, int64_t a, int64_t s) {
  double d2 = 0.0;
  for (int c = 0; c < H->d; ++c) {
    double t = H->xs[a * H->d + c] - H->xs[s * H->d + c];
    d2 += t * t;
  }
  return d2;
}

static int64_t orc_nearest_unused(const orc_hodlr* H, int64_t bl, int64_t ml, int64_t br,
                                  const char* used) {
  int64_t best = -1;
  double bd = 0.0;
  for (int64_t a = 0; a < ml; ++a) {
    if (used && used[a]) continue;
    double d2 = orc_d2_split(H, bl + a, br);
    if (best < 0 || d2 < bd) {
      best = a;
      bd = d2;
    }
  }
  return best;
}

static int orc_aca(const orc_hodlr* H, int64_t bl, int64_t ml, int64_t br, int64_t mr,
                   double** Uo, double** Vo, int* ok) {
  int64_t cap64 = ml < mr ? ml : mr;
  int rmax = (int)(cap64 < H->max_rank ? cap64 : H->max_rank);
  double* U = (double*)malloc(sizeof(double) * ml * (rmax > 0 ? rmax : 1));
  double* V = (double*)malloc(sizeof(double) * mr * (rmax > 0 ? rmax : 1));
  double* row = (double*)malloc(sizeof(double) * mr);
  double* col = (double*)malloc(sizeof(double) * ml);
  char* used = (char*)calloc((size_t)ml, 1);
  int k = 0;
  int64_t i = 0;
  double s2 = 0.0;
  int zero_tries = 0;
  *ok = 0;
  while (k < rmax) {
    for (int64_t b = 0; b < mr; ++b) {
      double v = orc_kij(H->xs, H->d, &H->cov, bl + i, br + b);
      for (int l = 0; l < k; ++l) v -= U[l * ml + i] * V[l * mr + b];
      row[b] = v;
    }
    int64_t j = 0;
    for (int64_t b = 1; b < mr; ++b)
      if (fabs(row[b]) > fabs(row[j])) j = b;
    double delta = row[j];
    used[i] = 1;
    if (delta == 0.0) {
      if (++zero_tries > rmax) { *ok = 1; break; }
      int64_t nx = orc_nearest_unused(H, bl, ml, br, used);
      if (nx < 0) { *ok = 1; break; }
      i = nx;
      continue;
    }
    for (int64_t b = 0; b < mr; ++b) row[b] /= delta;
    for (int64_t a = 0; a < ml; ++a) {
      double u = orc_kij(H->xs, H->d, &H->cov, bl + a, br + j);
      for (int l = 0; l < k; ++l) u -= U[l * ml + a] * V[l * mr + j];
      col[a] = u;
    }
    double nu2 = 0.0, nv2 = 0.0, cross = 0.0;
    for (int64_t a = 0; a < ml; ++a) nu2 += col[a] * col[a];
    for (int64_t b = 0; b < mr; ++b) nv2 += row[b] * row[b];
    for (int l = 0; l < k; ++l) {
      double du = 0.0, dv = 0.0;
      for (int64_t a = 0; a < ml; ++a) du += U[l * ml + a] * col[a];
      for (int64_t b = 0; b < mr; ++b) dv += V[l * mr + b] * row[b];
      cross += du * dv;
    }
    s2 += 2.0 * cross + nu2 * nv2;
    if (sqrt(nu2 * nv2) <= H->eps * sqrt(s2)) { *ok = 1; break; }
    memcpy(U + (int64_t)k * ml, col, sizeof(double) * ml);
    memcpy(V + (int64_t)k * mr, row, sizeof(double) * mr);
    ++k;
    int64_t nx = -1;
    for (int64_t a = 0; a < ml; ++a)
      if (!used[a] && (nx < 0 || fabs(col[a]) > fabs(col[nx]))) nx = a;
    if (nx < 0) { *ok = 1; break; }
    i = nx;
  }
  if (k == rmax && rmax == cap64) *ok = 1; /* full rank of the block is exact */
  free(row); free(col); free(used);
  *Uo = U;
  *Vo = V;
  return k;
}

static int64_t orc_nid(int j, int64_t k) { return ((int64_t)1 << j) - 1 + k; }

/* Analytic compression by Chebyshev interpolation (Sec. 3.1: A ~ E A~ P, A~ the kernel
 * sampled at Chebyshev nodes of the two clusters, E and P interpolation matrices; the
 * barycentric formula of Berrut and Trefethen 2004). 1-D only. Reading of the paper's
 * "spectral analysis of the interpolating Chebyshev polynomial", which it does not spell
 * out:
 *   - nodes: q Chebyshev points of the first kind on each child's interval [first point,
 *     last point], s_a = mid + half cos((2a + 1) pi / (2q));
 *   - q from 8, 16, 32, 64: the first q for which the 2-D Chebyshev coefficients of the
 *     interpolant, C = T A~ T^T with T_ja = (2/q) cos(j (2a + 1) pi / (2q)) (row j = 0
 *     halved), have their last quarter (max(j, k) >= 3q/4) at most eps times the largest
 *     coefficient; no q up to 64 passing is a failure (*ok = 0);
 *   - rank: A~ is recompressed by a cross with full pivoting (the largest residual entry,
 *     lowest row-major index on ties) until the residual's Frobenius norm is at most eps
 *     times A~'s, capped at min(m_left, m_right, max_rank) (*ok = 0 at the cap);
 *   - U = E A~_u and V = P A~_v, E_ia = L_a(x_i) the Lagrange basis of the left nodes at
 *     the left points (barycentric weights (-1)^a sin((2a + 1) pi / (2q))), P likewise;
 *   - a block that interpolation cannot represent within its caps (no q up to 64 passes,
 *     or the cross reaches min(m_left, m_right)) is stored exactly when
 *     m = min(m_left, m_right) <= max_rank: rank m, the identity on the smaller side and
 *     the block's entries on the other (a small block has rank at most m, while its
 *     interpolant can need more terms); otherwise *ok = 0.
 * Returns the rank; U (m_left x r) and V (m_right x r) column-major. */
#define ORC_CHEB_QMAX 64

static void orc_cheb_nodes(double a, double b, int q, double* s, double* w) {
  for (int k = 0; k < q; ++k) {
    double th = (2.0 * k + 1.0) * M_PI / (2.0 * q);
    s[k] = 0.5 * (a + b) + 0.5 * (b - a) * cos(th);
    w[k] = ((k & 1) ? -1.0 : 1.0) * sin(th);
  }
}

/* Lagrange basis of the nodes s (weights w) at x: L[a] = (w_a / (x - s_a)) / sum_b (w_b /
 * (x - s_b)); at a node (x == s_a, also every node of a zero-length interval) L = e_a. */
static void orc_bary(double x, const double* s, const double* w, int q, double* L) {
  for (int a = 0; a < q; ++a)
    if (x == s[a]) {
      for (int b = 0; b < q; ++b) L[b] = b == a ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int a = 0; a < q; ++a) {
    L[a] = w[a] / (x - s[a]);
    den += L[a];
  }
  for (int a = 0; a < q; ++a) L[a] /= den;
}

static int orc_cheb(const orc_hodlr* H, int64_t bl, int64_t ml, int64_t br, int64_t mr,
                    double** Uo, double** Vo, int* ok) {
  const int Q = ORC_CHEB_QMAX;
  double s[ORC_CHEB_QMAX], ws[ORC_CHEB_QMAX], t[ORC_CHEB_QMAX], wt[ORC_CHEB_QMAX];
  double* A = (double*)malloc(sizeof(double) * Q * Q);
  double* W = (double*)malloc(sizeof(double) * Q * Q);
  const double* x = H->xs; /* 1-D: sorted, so each child's interval is [first, last] */
  if (ml == 0 || mr == 0) { /* an empty block: exact at rank 0 */
    free(A); free(W);
    *Uo = (double*)malloc(sizeof(double));
    *Vo = (double*)malloc(sizeof(double));
    *ok = 1;
    return 0;
  }
  double a1 = x[bl], b1 = x[bl + ml - 1], a2 = x[br], b2 = x[br + mr - 1];
  int q = 0;
  *ok = 0;
  for (int qq = 8; qq <= Q; qq *= 2) {
    orc_cheb_nodes(a1, b1, qq, s, ws);
    orc_cheb_nodes(a2, b2, qq, t, wt);
    for (int i = 0; i < qq; ++i)
      for (int j = 0; j < qq; ++j) {
        double r = fabs(s[i] - t[j]);
        A[i * qq + j] = orc_kernel(&H->cov, r, r * r);
      }
    /* C = T A T^T */
    for (int jj = 0; jj < qq; ++jj)
      for (int b = 0; b < qq; ++b) {
        double acc = 0.0;
        for (int a = 0; a < qq; ++a)
          acc += cos(jj * (2.0 * a + 1.0) * M_PI / (2.0 * qq)) * A[a * qq + b];
        W[jj * qq + b] = acc * (jj == 0 ? 1.0 : 2.0) / qq;
      }
    double cmax = 0.0, tail = 0.0;
    for (int jj = 0; jj < qq; ++jj)
      for (int kk = 0; kk < qq; ++kk) {
        double acc = 0.0;
        for (int b = 0; b < qq; ++b)
          acc += W[jj * qq + b] * cos(kk * (2.0 * b + 1.0) * M_PI / (2.0 * qq));
        double c = fabs(acc * (kk == 0 ? 1.0 : 2.0) / qq);
        if (c > cmax) cmax = c;
        if ((jj >= qq - qq / 4 || kk >= qq - qq / 4) && c > tail) tail = c;
      }
    if (tail <= H->eps * cmax) {
      q = qq;
      break;
    }
  }
  int64_t cap64 = ml < mr ? ml : mr;
  int rmax = (int)(cap64 < H->max_rank ? cap64 : H->max_rank);
  double* Ua = (double*)malloc(sizeof(double) * Q * (rmax > 0 ? rmax : 1));
  double* Va = (double*)malloc(sizeof(double) * Q * (rmax > 0 ? rmax : 1));
  int r = 0;
  if (q > 0) {
    /* cross with full pivoting on A (q x q), residual in W */
    double n0 = 0.0;
    for (int e = 0; e < q * q; ++e) {
      W[e] = A[e];
      n0 += A[e] * A[e];
    }
    *ok = 1;
    for (;;) {
      double res = 0.0, best = -1.0;
      int pi = 0, pj = 0;
      for (int e = 0; e < q * q; ++e) {
        res += W[e] * W[e];
        if (fabs(W[e]) > best) {
          best = fabs(W[e]);
          pi = e / q;
          pj = e % q;
        }
      }
      if (res <= H->eps * H->eps * n0 || best == 0.0) break;
      if (r == rmax) {
        *ok = 0;
        break;
      }
      double piv = W[pi * q + pj];
      for (int a = 0; a < q; ++a) {
        Ua[r * Q + a] = W[a * q + pj];
        Va[r * Q + a] = W[pi * q + a] / piv;
      }
      for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) W[a * q + b] -= Ua[r * Q + a] * Va[r * Q + b];
      ++r;
    }
  }
  double* U = (double*)malloc(sizeof(double) * ml * (r > 0 ? r : 1));
  double* V = (double*)malloc(sizeof(double) * mr * (r > 0 ? r : 1));
  double L[ORC_CHEB_QMAX];
  for (int64_t i = 0; i < ml && r > 0; ++i) {
    orc_bary(x[bl + i], s, ws, q, L);
    for (int l = 0; l < r; ++l) {
      double acc = 0.0;
      for (int a = 0; a < q; ++a) acc += L[a] * Ua[l * Q + a];
      U[l * ml + i] = acc;
    }
  }
  for (int64_t j = 0; j < mr && r > 0; ++j) {
    orc_bary(x[br + j], t, wt, q, L);
    for (int l = 0; l < r; ++l) {
      double acc = 0.0;
      for (int b = 0; b < q; ++b) acc += L[b] * Va[l * Q + b];
      V[l * mr + j] = acc;
    }
  }
  free(A); free(W); free(Ua); free(Va);
  int64_t mmin = ml < mr ? ml : mr;
  if (!*ok && mmin <= H->max_rank) { /* exact storage */
    free(U);
    free(V);
    int m = (int)mmin;
    U = (double*)malloc(sizeof(double) * ml * m);
    V = (double*)malloc(sizeof(double) * mr * m);
    for (int l = 0; l < m; ++l) {
      for (int64_t i = 0; i < ml; ++i)
        U[l * ml + i] = ml <= mr ? (i == l ? 1.0 : 0.0) : orc_kij(x, 1, &H->cov, bl + i, br + l);
      for (int64_t j = 0; j < mr; ++j)
        V[l * mr + j] = ml <= mr ? orc_kij(x, 1, &H->cov, bl + l, br + j) : (j == l ? 1.0 : 0.0);
    }
    *ok = 1;
    r = m;
  }
  *Uo = U;
  *Vo = V;
  return r;
}

/* compression: 0 = adaptive cross approximation, 1 = Chebyshev interpolation (1-D). */
void* oracle_hodlr_build(const double* x, int64_t n, int d, int kind, const double* theta,
                         double sigma2, int leaf, double eps, int max_rank, int compression,
                         int* status) {
  if (n < 1 || d < 1 || d > ORC_MAX_D || leaf < 1 || !(eps > 0) || sigma2 < 0 || max_rank < 1 ||
      kind < 0 || kind > ORC_BH || (kind == ORC_RQ && !(theta[2] > 0)) ||
      compression < 0 || compression > 1 || (compression == 1 && d != 1)) {
    *status = ORC_EINVAL;
    return NULL;
  }
  orc_hodlr* H = (orc_hodlr*)calloc(1, sizeof(orc_hodlr));
  H->n = n; H->d = d; H->kind = kind; H->leaf = leaf; H->max_rank = max_rank;
  H->cov = orc_cov_make(kind, theta); H->sigma2 = sigma2; H->eps = eps;
  H->kappa = oracle_kappa(n, leaf);
  int kap = H->kappa;
  H->perm = (int64_t*)malloc(sizeof(int64_t) * n);
  oracle_tree_order(x, n, d, leaf, H->perm);
  H->xs = (double*)malloc(sizeof(double) * n * d);
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < d; ++c) H->xs[i * d + c] = x[H->perm[i] * d + c];
  int64_t nnodes = ((int64_t)2 << kap) - 1;
  H->nb = (int64_t*)malloc(sizeof(int64_t) * nnodes);
  H->ns = (int64_t*)malloc(sizeof(int64_t) * nnodes);
  H->nb[0] = 0;
  H->ns[0] = n;
  for (int j = 0; j < kap; ++j)
    for (int64_t k = 0; k < ((int64_t)1 << j); ++k) {
      int64_t id = orc_nid(j, k), m = H->ns[id], ml = m / 2;
      H->nb[orc_nid(j + 1, 2 * k)] = H->nb[id];
      H->ns[orc_nid(j + 1, 2 * k)] = ml;
      H->nb[orc_nid(j + 1, 2 * k + 1)] = H->nb[id] + ml;
      H->ns[orc_nid(j + 1, 2 * k + 1)] = m - ml;
    }
  int64_t nint = ((int64_t)1 << kap) - 1;
  H->rank = (int*)calloc((size_t)(nint > 0 ? nint : 1), sizeof(int));
  H->aca_ok = (int*)calloc((size_t)(nint > 0 ? nint : 1), sizeof(int));
  H->U = (double**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double*));
  H->V = (double**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double*));
  /* Compression of every off-diagonal block to precision eps (pseudo-code figure). */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t id = 0; id < nint; ++id) {
    int64_t l = 2 * id + 1, r = 2 * id + 2;
    H->rank[id] = (compression == 1 ? orc_cheb : orc_aca)(H, H->nb[l], H->ns[l], H->nb[r],
                                                         H->ns[r], &H->U[id], &H->V[id],
                          &H->aca_ok[id]);
  }
  int st = ORC_OK;
  for (int64_t id = 0; id < nint; ++id)
    if (!H->aca_ok[id]) st = ORC_ERANK;
  *status = st;
  return H;
}

int oracle_hodlr_kappa(void* h) { return ((orc_hodlr*)h)->kappa; }

int64_t oracle_hodlr_ranks(void* h, int* out, int64_t cap) {
  orc_hodlr* H = (orc_hodlr*)h;
  int64_t nint = ((int64_t)1 << H->kappa) - 1;
  for (int64_t i = 0; i < nint && i < cap; ++i) out[i] = H->rank[i];
  return nint;
}

void oracle_hodlr_perm(void* h, int64_t* out) {
  orc_hodlr* H = (orc_hodlr*)h;
  memcpy(out, H->perm, sizeof(int64_t) * H->n);
}

/* Factor copies of U, V for node id (row slice `off`, `rows` rows): the slice of the
 * ancestor's left (Ut) or right (Vt) transformed factor that covers those rows. */
static double* orc_anc_slice(orc_hodlr* H, int ja, int64_t ka, int64_t begin, int64_t* ld,
                             int* r) {
  int64_t id = orc_nid(ja, ka);
  int64_t lc = 2 * id + 1, rc = 2 * id + 2;
  *r = H->rank[id];
  if (begin < H->nb[rc]) {
    *ld = H->ns[lc];
    return H->Ut[id] + (begin - H->nb[lc]);
  }
  *ld = H->ns[rc];
  return H->Vt[id] + (begin - H->nb[rc]);
}

/* Apply the SMW inverse of node (j, k)'s factor I + [Ut 0; 0 Vt][0 V^T; U^T 0] to a block
 * P of `nc` columns (column stride ld) covering the node's rows (Sec. 3.2):
 *   Z = M^-1 [V^T P_R; U^T P_L], P_L -= Ut Z_top, P_R -= Vt Z_bot. */
static void orc_node_apply(orc_hodlr* H, int64_t id, double* P, int64_t ld, int nc) {
  int r = H->rank[id];
  if (r == 0 || nc == 0) return;
  int64_t ml = H->ns[2 * id + 1], mr = H->ns[2 * id + 2];
  double* z = (double*)malloc(sizeof(double) * 2 * r);
  for (int c = 0; c < nc; ++c) {
    double* pl = P + (int64_t)c * ld;
    double* pr = pl + ml;
    for (int a = 0; a < r; ++a) {
      double s = 0.0;
      for (int64_t t = 0; t < mr; ++t) s += H->V[id][(int64_t)a * mr + t] * pr[t];
      z[a] = s;
      s = 0.0;
      for (int64_t t = 0; t < ml; ++t) s += H->U[id][(int64_t)a * ml + t] * pl[t];
      z[r + a] = s;
    }
    orc_lu_solve(H->Mlu[id], 2 * r, H->Mpiv[id], z, 1);
    for (int a = 0; a < r; ++a) {
      const double* ut = H->Ut[id] + (int64_t)a * ml;
      const double* vt = H->Vt[id] + (int64_t)a * mr;
      for (int64_t t = 0; t < ml; ++t) pl[t] -= ut[t] * z[a];
      for (int64_t t = 0; t < mr; ++t) pr[t] -= vt[t] * z[r + a];
    }
  }
  free(z);
}

/* Leaf solve: apply the leaf LU inverse to `nc` columns of length s (stride ld). */
static void orc_leaf_apply(orc_hodlr* H, int64_t k, double* P, int64_t ld, int nc) {
  int s = (int)H->ns[orc_nid(H->kappa, k)];
  for (int c = 0; c < nc; ++c) orc_lu_solve(H->leafLU[k], s, H->leafpiv[k], P + (int64_t)c * ld, 1);
}

/* Factorization K = K_kappa K_{kappa-1} ... K_0 (Sec. 3.2 and its pseudo-code figure):
 * K_kappa holds the dense leaf blocks; factoring it out applies each leaf inverse to the
 * rows of every ancestor's U/V copy lying in that leaf; then, from the finest internal
 * level to the root, each node's 2r x 2r matrix M = [I, V^T Vt; U^T Ut, I] is LU-factored
 * and its SMW inverse is applied to every coarser ancestor's copy on the node's rows.
 * If y != NULL (sorted order, column-major, nrhs columns, stride n) the same inverses are
 * applied to it, so on return it holds C^-1 y. log det C = sum of leaf and node log dets
 * (Sec. 4: Sylvester's theorem gives det(I + L W) = det(I + W L) = det M). For a positive
 * definite C every factor has a positive determinant and a non-positive one is an error;
 * for the indefinite kernels (multiquadric, biharmonic) the factors' signs multiply into
 * the sign of det C and only a zero determinant is an error. */
static int orc_factor_impl(orc_hodlr* H, double* y, int nrhs) {
  int kap = H->kappa;
  int64_t nint = ((int64_t)1 << kap) - 1, nleaf = (int64_t)1 << kap;
  H->Ut = (double**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double*));
  H->Vt = (double**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double*));
  for (int64_t id = 0; id < nint; ++id) {
    int64_t ml = H->ns[2 * id + 1], mr = H->ns[2 * id + 2];
    int r = H->rank[id];
    H->Ut[id] = (double*)malloc(sizeof(double) * (ml * r > 0 ? ml * r : 1));
    H->Vt[id] = (double*)malloc(sizeof(double) * (mr * r > 0 ? mr * r : 1));
    memcpy(H->Ut[id], H->U[id], sizeof(double) * ml * r);
    memcpy(H->Vt[id], H->V[id], sizeof(double) * mr * r);
  }
  H->leafLU = (double**)calloc((size_t)nleaf, sizeof(double*));
  H->leafpiv = (int**)calloc((size_t)nleaf, sizeof(int*));
  H->leaflogdet = (double*)calloc((size_t)nleaf, sizeof(double));
  H->Mlu = (double**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double*));
  H->Mpiv = (int**)calloc((size_t)(nint > 0 ? nint : 1), sizeof(int*));
  H->nodelogdet = (double*)calloc((size_t)(nint > 0 ? nint : 1), sizeof(double));
  int bad = 0, nneg = 0;
  const int indef = orc_indefinite(H->kind);
  /* Leaves: LU of the dense diagonal blocks of C, then K_kappa^-1 on the ancestors' rows. */
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad) reduction(+ : nneg)
  for (int64_t k = 0; k < nleaf; ++k) {
    int64_t id = orc_nid(kap, k), b = H->nb[id];
    int s = (int)H->ns[id];
    double* A = (double*)malloc(sizeof(double) * (s > 0 ? s * s : 1));
    for (int a = 0; a < s; ++a)
      for (int c = 0; c < s; ++c)
        A[a * s + c] = orc_entry(H->xs, H->d, &H->cov, H->sigma2, b + a, b + c);
    int* piv = (int*)malloc(sizeof(int) * (s > 0 ? s : 1));
    int sg = 1;
    double ld = s > 0 ? orc_lu(A, s, piv, &sg) : 0.0;
    if (sg == 0 || (sg < 0 && !indef)) bad = 1;
    if (sg < 0) nneg += 1;
    H->leafLU[k] = A;
    H->leafpiv[k] = piv;
    H->leaflogdet[k] = ld;
    for (int j = 0; j < kap; ++j) {
      int64_t ldp;
      int r;
      double* P = orc_anc_slice(H, j, k >> (kap - j), b, &ldp, &r);
      orc_leaf_apply(H, k, P, ldp, r);
    }
    if (y) orc_leaf_apply(H, k, y + b, H->n, nrhs);
  }
  /* Levels, finest internal level first. */
  for (int j = kap - 1; j >= 0 && !bad; --j) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad) reduction(+ : nneg)
    for (int64_t k = 0; k < ((int64_t)1 << j); ++k) {
      int64_t id = orc_nid(j, k);
      int r = H->rank[id];
      int64_t ml = H->ns[2 * id + 1], mr = H->ns[2 * id + 2];
      int m2 = 2 * r;
      double* M = (double*)malloc(sizeof(double) * (m2 > 0 ? m2 * m2 : 1));
      int* piv = (int*)malloc(sizeof(int) * (m2 > 0 ? m2 : 1));
      for (int a = 0; a < m2 * m2; ++a) M[a] = 0.0;
      for (int a = 0; a < m2; ++a) M[a * m2 + a] = 1.0;
      for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) {
          double sx = 0.0, sy = 0.0;
          for (int64_t t = 0; t < mr; ++t) sx += H->V[id][(int64_t)a * mr + t] * H->Vt[id][(int64_t)c * mr + t];
          for (int64_t t = 0; t < ml; ++t) sy += H->U[id][(int64_t)a * ml + t] * H->Ut[id][(int64_t)c * ml + t];
          M[a * m2 + (r + c)] = sx;
          M[(r + a) * m2 + c] = sy;
        }
      int sg = 1;
      double ld = m2 > 0 ? orc_lu(M, m2, piv, &sg) : 0.0;
      if (sg == 0 || (sg < 0 && !indef)) bad = 1;
      if (sg < 0) nneg += 1;
      H->Mlu[id] = M;
      H->Mpiv[id] = piv;
      H->nodelogdet[id] = ld;
      for (int ja = 0; ja < j; ++ja) {
        int64_t ldp;
        int ra;
        double* P = orc_anc_slice(H, ja, k >> (j - ja), H->nb[id], &ldp, &ra);
        orc_node_apply(H, id, P, ldp, ra);
      }
      if (y) orc_node_apply(H, id, y + H->nb[id], H->n, nrhs);
    }
  }
  if (bad) return ORC_ENOTSPD;
  /* log det: sequential sums, in a fixed order, of the leaf terms and of the node terms. */
  double sl = 0.0, sn = 0.0;
  for (int64_t k = 0; k < nleaf; ++k) sl += H->leaflogdet[k];
  for (int64_t id = 0; id < nint; ++id) sn += H->nodelogdet[id];
  H->logdet = sl + sn;
  H->logdet_sign = (nneg & 1) ? -1 : 1;
  H->factored = 1;
  return ORC_OK;
}

/* Gather y (original order, column stride ldy) into sorted order, column stride n. */
static double* orc_gather(orc_hodlr* H, const double* y, int nrhs, int64_t ldy) {
  double* w = (double*)malloc(sizeof(double) * H->n * (nrhs > 0 ? nrhs : 1));
  for (int c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < H->n; ++i) w[(int64_t)c * H->n + i] = y[(int64_t)c * ldy + H->perm[i]];
  return w;
}

static void orc_scatter(orc_hodlr* H, const double* w, int nrhs, double* x, int64_t ldx) {
  for (int c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < H->n; ++i) x[(int64_t)c * ldx + H->perm[i]] = w[(int64_t)c * H->n + i];
}

int oracle_hodlr_factor(void* h) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (H->factored) return ORC_ESTATE;
  return orc_factor_impl(H, NULL, 0);
}

/* Solve C x = y with the stored factors: C^-1 = K_0^-1 K_1^-1 ... K_kappa^-1 (Sec. 3.2),
 * so the leaf inverses come first and the root's SMW inverse last. */
int oracle_hodlr_solve(void* h, const double* y, double* x, int nrhs, int64_t ld) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (!H->factored) return ORC_ESTATE;
  int kap = H->kappa;
  double* w = orc_gather(H, y, nrhs, ld);
  int64_t nleaf = (int64_t)1 << kap;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nleaf; ++k) orc_leaf_apply(H, k, w + H->nb[orc_nid(kap, k)], H->n, nrhs);
  for (int j = kap - 1; j >= 0; --j) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < ((int64_t)1 << j); ++k) {
      int64_t id = orc_nid(j, k);
      orc_node_apply(H, id, w + H->nb[id], H->n, nrhs);
    }
  }
  orc_scatter(H, w, nrhs, x, ld);
  free(w);
  return ORC_OK;
}

/* Factor with the right-hand side carried through the sweep (same inverses, same order). */
int oracle_hodlr_factor_solve(void* h, const double* y, double* x, int nrhs, int64_t ld) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (H->factored) return ORC_ESTATE;
  double* w = orc_gather(H, y, nrhs, ld);
  int st = orc_factor_impl(H, w, nrhs);
  if (st == ORC_OK) orc_scatter(H, w, nrhs, x, ld);
  free(w);
  return st;
}

/* log |det C| (log det C for a positive definite C). */
int oracle_hodlr_logdet(void* h, double* out) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (!H->factored) return ORC_ESTATE;
  *out = H->logdet;
  return ORC_OK;
}

/* Sign of det C: the product of the leaf and node determinants' signs. */
int oracle_hodlr_logdet_sign(void* h, int* out) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (!H->factored) return ORC_ESTATE;
  *out = H->logdet_sign;
  return ORC_OK;
}

void oracle_hodlr_level_logdets(void* h, double* leaf_out, double* node_out) {
  orc_hodlr* H = (orc_hodlr*)h;
  int64_t nleaf = (int64_t)1 << H->kappa, nint = nleaf - 1;
  if (leaf_out) memcpy(leaf_out, H->leaflogdet, sizeof(double) * nleaf);
  if (node_out && nint > 0) memcpy(node_out, H->nodelogdet, sizeof(double) * nint);
}

/* Gaussian log-likelihood (Sec. 1, Eq. 1, with the normalising constant written out):
 * -1/2 y^T C^-1 y - 1/2 log det C - n/2 log(2 pi). */
int oracle_hodlr_loglik(void* h, const double* y, double* out) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (orc_indefinite(H->kind)) return ORC_EINVAL; /* not a covariance: no Gaussian density */
  double* x = (double*)malloc(sizeof(double) * H->n);
  int st = H->factored ? oracle_hodlr_solve(h, y, x, 1, H->n)
                       : oracle_hodlr_factor_solve(h, y, x, 1, H->n);
  if (st != ORC_OK) { free(x); return st; }
  double q = 0.0;
  for (int64_t i = 0; i < H->n; ++i) q += y[i] * x[i];
  *out = -0.5 * q - 0.5 * H->logdet - 0.5 * (double)H->n * log(2.0 * M_PI);
  free(x);
  return ORC_OK;
}

/* HODLR operator product out = C~ v (original order): dense leaves plus, for each node,
 * out_L += U (V^T v_R), out_R += V (U^T v_L) (the block structure of Sec. 3). */
void oracle_hodlr_matvec(void* h, const double* v, double* out) {
  orc_hodlr* H = (orc_hodlr*)h;
  int kap = H->kappa;
  int64_t n = H->n;
  double* w = orc_gather(H, v, 1, n);
  double* o = (double*)calloc((size_t)n, sizeof(double));
  int64_t nleaf = (int64_t)1 << kap;
  for (int64_t k = 0; k < nleaf; ++k) {
    int64_t id = orc_nid(kap, k), b = H->nb[id], s = H->ns[id];
    for (int64_t a = 0; a < s; ++a) {
      double t = 0.0;
      for (int64_t c = 0; c < s; ++c)
        t += orc_entry(H->xs, H->d, &H->cov, H->sigma2, b + a, b + c) * w[b + c];
      o[b + a] += t;
    }
  }
  for (int64_t id = 0; id < nleaf - 1; ++id) {
    int64_t bl = H->nb[2 * id + 1], ml = H->ns[2 * id + 1];
    int64_t br = H->nb[2 * id + 2], mr = H->ns[2 * id + 2];
    for (int a = 0; a < H->rank[id]; ++a) {
      const double* u = H->U[id] + (int64_t)a * ml;
      const double* vv = H->V[id] + (int64_t)a * mr;
      double sv = 0.0, su = 0.0;
      for (int64_t t = 0; t < mr; ++t) sv += vv[t] * w[br + t];
      for (int64_t t = 0; t < ml; ++t) su += u[t] * w[bl + t];
      for (int64_t t = 0; t < ml; ++t) o[bl + t] += u[t] * sv;
      for (int64_t t = 0; t < mr; ++t) o[br + t] += vv[t] * su;
    }
  }
  orc_scatter(H, o, 1, out, n);
  free(w);
  free(o);
}

/* Copy node id's factors (U: ml x r, V: mr x r, column-major) for tests. */
int oracle_hodlr_node_factors(void* h, int64_t id, double* U, double* V) {
  orc_hodlr* H = (orc_hodlr*)h;
  int64_t ml = H->ns[2 * id + 1], mr = H->ns[2 * id + 2];
  int r = H->rank[id];
  if (U) memcpy(U, H->U[id], sizeof(double) * ml * r);
  if (V) memcpy(V, H->V[id], sizeof(double) * mr * r);
  return r;
}

void oracle_hodlr_node_range(void* h, int64_t id, int64_t* begin, int64_t* size) {
  orc_hodlr* H = (orc_hodlr*)h;
  *begin = H->nb[id];
  *size = H->ns[id];
}

void oracle_hodlr_destroy(void* h) {
  orc_hodlr* H = (orc_hodlr*)h;
  if (!H) return;
  int64_t nint = ((int64_t)1 << H->kappa) - 1, nleaf = (int64_t)1 << H->kappa;
  for (int64_t id = 0; id < nint; ++id) {
    free(H->U[id]); free(H->V[id]);
    if (H->Ut) free(H->Ut[id]);
    if (H->Vt) free(H->Vt[id]);
    if (H->Mlu) free(H->Mlu[id]);
    if (H->Mpiv) free(H->Mpiv[id]);
  }
  if (H->leafLU)
    for (int64_t k = 0; k < nleaf; ++k) { free(H->leafLU[k]); free(H->leafpiv[k]); }
  free(H->U); free(H->V); free(H->Ut); free(H->Vt); free(H->Mlu); free(H->Mpiv);
  free(H->leafLU); free(H->leafpiv); free(H->leaflogdet); free(H->nodelogdet);
  free(H->rank); free(H->aca_ok); free(H->xs); free(H->perm); free(H->nb); free(H->ns);
  free(H);
}
