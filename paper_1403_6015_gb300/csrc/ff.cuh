// Double-float ("ff") arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits (unit roundoff ~2^-48).
// On GB300 the FP32 pipe issues ~64x the operations of the FP64 pipe, so the dense leaf
// work runs faster in ff than in native double while keeping ~1e-14 relative accuracy.
//
// Building blocks are the classic error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum, and the FMA-based exact product (TwoProd). The double-word operations follow
// the algorithms analysed by Joldes, Muller and Popescu ("Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic", ACM TOMS 2017): products
// (DWTimesDW with FMA) and the "sloppy" sum, whose error is bounded by a small multiple of
// u^2 (|a| + |b|), the form that backward-stable factorizations rely on.
#pragma once

#include <cuda_runtime.h>

namespace hodlr {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  fast_two_sum(h, l, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_from_double(double d) {
  ff r;
  r.hi = __double2float_rn(d);
  r.lo = __double2float_rn(d - (double)r.hi);
  return r;
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

// a + b, sloppy double-word sum
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * b, double-word product with FMA
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// c - a * b in one pass (exact leading product, sloppy sum)
__device__ __forceinline__ ff ff_fms(ff c, ff a, ff b) {
  float p = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  two_sum(c.hi, -p, s, e);
  e += c.lo - pe;
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// c + a * b
__device__ __forceinline__ ff ff_fma(ff c, ff a, ff b) { return ff_fms(c, ff_neg(a), b); }

// Compensated dot-product accumulator (the "Dot2" scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005, with double-word operands):
// a float running sum s and a float sum e of the errors. Each product enters as its exact
// leading part (TwoProd) plus the cross terms, the running sum by TwoSum with its error
// moved to e, and the pair is renormalised once, when read. 12 instructions per term
// against 15 for ff_fms, with an error of order n^2 u^2 sum |x_i y_i| for n terms
// (u = 2^-24), the same order as n renormalised sloppy sums for the short (<= 32-term)
// dot products it is used for.
struct ffacc {
  float s, e;
};

__device__ __forceinline__ ffacc ffacc_init(ff c) { return ffacc{c.hi, c.lo}; }

// acc -= x * y
__device__ __forceinline__ void ffacc_fms(ffacc& a, ff x, ff y) {
  float p = x.hi * y.hi;
  float pe = fmaf(x.hi, y.hi, -p);
  pe = fmaf(x.hi, y.lo, pe);
  pe = fmaf(x.lo, y.hi, pe);
  float s, t;
  two_sum(a.s, -p, s, t);
  a.s = s;
  a.e += t - pe;
}

// acc += x * y
__device__ __forceinline__ void ffacc_fma(ffacc& a, ff x, ff y) { ffacc_fms(a, ff_neg(x), y); }

__device__ __forceinline__ ff ffacc_get(ffacc a) { return ff_make(a.s, a.e); }

// the sum of two accumulators, renormalised
__device__ __forceinline__ ff ffacc_get2(ffacc a, ffacc b) {
  float s, t;
  two_sum(a.s, b.s, s, t);
  return ff_make(s, t + (a.e + b.e));
}

// a * f for a float f
__device__ __forceinline__ ff ff_mulf(ff a, float f) {
  float p = a.hi * f;
  float e = fmaf(a.hi, f, -p);
  e = fmaf(a.lo, f, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// 1 / a: float reciprocal refined by one Newton step in double-word arithmetic
__device__ __forceinline__ ff ff_rcp(ff a) {
  float x = 1.0f / a.hi;
  // residual 1 - a x, computed to double-word accuracy
  ff ax = ff_mulf(a, x);
  ff res = ff_sub(ff{1.0f, 0.0f}, ax);
  // x + x * res
  float corr = x * res.hi;
  return ff_make(x, corr);
}

// sqrt(q) for q >= 0: the float root h refined by one Newton step, h + (q - h^2) / (2h).
__device__ __forceinline__ ff ff_sqrt(ff q) {
  float h = sqrtf(q.hi);
  if (!(h > 0.0f)) return ff{0.0f, 0.0f};
  ff res = ff_sub(q, ff_mul(ff{h, 0.0f}, ff{h, 0.0f}));
  return ff_make(h, res.hi / (2.0f * h));
}

// exp(x) for a double-float x <= ~0 (covariances use exp of minus a distance). Reduction
// x = n ln2/64 + r, |r| <= ln2/128 (Cody-Waite: ln2/64 = L1 + L2 with L1 holding 11
// significant bits so n L1 is exact for |n| < 2^13, L2 a double-float), then
// exp(x) = 2^(n div 64) 2^((n mod 64)/64) exp(r), exp(r) by its Taylor series to degree 6
// in double-word arithmetic (remainder below 3e-20). tab64[j] = 2^(j/64) as double-floats.
// Arguments below -87 return 0 (the covariances they model are below 2^-125).
__device__ __forceinline__ ff ff_exp(ff x, const ff* __restrict__ tab64) {
  if (x.hi < -87.0f) return ff{0.0f, 0.0f};
  const float kInvL = 92.33248f;             // 64 / ln2
  const float kL1 = 0.010833740234375f;      // 11-bit head of ln2/64
  const ff kL2 = {-3.3155381515825866e-06f, 2.572804640231345e-14f};  // ln2/64 - kL1
  float nf = rintf(x.hi * kInvL);
  int n = (int)nf;
  ff r = ff_add(x, ff{-nf * kL1, 0.0f});
  r = ff_fms(r, ff{nf, 0.0f}, kL2);
  // 1/k! as double-floats, k = 0..6
  const ff c2 = {0.5f, 0.0f};
  const ff c3 = {0.1666666716337204f, -4.967053879312289e-09f};
  const ff c4 = {0.0416666679084301f, -1.2417634698280722e-09f};
  const ff c5 = {0.008333333767950535f, -4.34617203337595e-10f};
  const ff c6 = {0.0013888889225199819f, -3.3631094437103215e-11f};
  ff q = ff_fma(c5, c6, r);
  q = ff_fma(c4, q, r);
  q = ff_fma(c3, q, r);
  q = ff_fma(c2, q, r);
  q = ff_fma(ff{1.0f, 0.0f}, q, r);
  q = ff_fma(ff{1.0f, 0.0f}, q, r);
  int j = n & 63;
  int k = (n - j) / 64;
  ff t = ff_mul(q, tab64[j]);
  float sc = ldexpf(1.0f, k);
  return ff{t.hi * sc, t.lo * sc};
}

// log(x) for a double-float x >= 1 (the argument 1 + t^2 of the rational quadratic): the
// float logarithm y0 of x.hi, refined by one Newton step on exp: e = x exp(-y0) - 1 and
// log x = y0 + log1p(e) = y0 + e - e^2/2 + O(e^3), |e| below ~1e-6 (the float log's error),
// so the truncation is below 1e-18 and the result is good to about 2^-48 absolute.
__device__ __forceinline__ ff ff_log(ff x, const ff* __restrict__ tab64) {
  float y0 = logf(x.hi);
  ff e = ff_sub(ff_mul(x, ff_exp(ff{-y0, 0.0f}, tab64)), ff{1.0f, 0.0f});
  ff corr = ff_sub(e, ff_mulf(ff_mul(e, e), 0.5f));
  return ff_add(ff{y0, 0.0f}, corr);
}

// A covariance's parameters as double-floats: kind, cr (the factor applied to r), the
// amplitude a and the rational quadratic's exponent alpha.
struct CovFF {
  int kind;
  ff cr, amp, alpha;
};

__device__ __forceinline__ CovFF make_cov_ff(int kind, double cr, double amp, double alpha) {
  return CovFF{kind, ff_from_double(cr), ff_from_double(amp), ff_from_double(alpha)};
}

// Covariance k(r) = a f(cr r) in double-float (Table 1 with a length scale: exponential,
// squared-exponential, Matern-3/2, Matern-5/2; cr = 1/ell, 1/ell, sqrt3/ell, sqrt5/ell; and
// the positive definite radial functions of Sec. 5, rational quadratic (1 + t^2)^-alpha and
// inverse multiquadric 1/sqrt(1 + t^2), t = r/ell). The indefinite multiquadric and
// biharmonic have no double-float form (the mixed form's L D L^T leaves need a positive
// definite C): NaN.
// Rational quadratic (kind 4) and inverse multiquadric (kind 5) of s = t, out of line (see
// cov_ff).
static __device__ __noinline__ ff cov_ff_radial(const CovFF& k, ff s, const ff* tab) {
  const ff one = {1.0f, 0.0f};
  ff q = ff_add(one, ff_mul(s, s));
  if (k.kind == 4) return ff_mul(k.amp, ff_exp(ff_neg(ff_mul(k.alpha, ff_log(q, tab))), tab));
  if (k.kind == 5) return ff_mul(k.amp, ff_rcp(ff_sqrt(q)));
  return ff{nanf(""), 0.0f};
}

// The four covariances of Table 1 alone (kernels specialised for the common case).
__device__ __forceinline__ ff cov_ff_table1(const CovFF& k, ff r, const ff* tab) {
  ff s = ff_mul(r, k.cr);
  const ff one = {1.0f, 0.0f};
  switch (k.kind) {
    case 0:  // exponential
      return ff_mul(k.amp, ff_exp(ff_neg(s), tab));
    case 1:  // squared-exponential
      return ff_mul(k.amp, ff_exp(ff_mulf(ff_mul(s, s), -0.5f), tab));
    case 2:  // Matern-3/2
      return ff_mul(k.amp, ff_mul(ff_add(one, s), ff_exp(ff_neg(s), tab)));
    default: {  // Matern-5/2
      const ff third = {0.3333333432674408f, -9.934107481068821e-09f};
      ff poly = ff_add(ff_add(one, s), ff_mul(ff_mul(s, s), third));
      return ff_mul(k.amp, ff_mul(poly, ff_exp(ff_neg(s), tab)));
    }
  }
}

// Any kind with a double-float form (rational quadratic exp(-alpha log(1 + t^2)) and
// inverse multiquadric out of line).
__device__ __forceinline__ ff cov_ff(const CovFF& k, ff r, const ff* tab) {
  if (k.kind <= 3) return cov_ff_table1(k, r, tab);
  return cov_ff_radial(k, ff_mul(r, k.cr), tab);
}

// 2^(j/64), j = 0..63, as double-floats (from the FP64 exp2), for ff_exp.
__device__ __forceinline__ void ff_exp_table(ff* tab, int tid, int nthreads) {
  for (int j = tid; j < 64; j += nthreads) tab[j] = ff_from_double(exp2((double)j / 64.0));
}

// Factor applied to r for each covariance: 1/ell, 1/ell, sqrt3/ell, sqrt5/ell.
__host__ __device__ inline double cov_scale(int kind, double ell) {
  return (kind == 2 ? 1.7320508075688772 : kind == 3 ? 2.23606797749979 : 1.0) / ell;
}

}  // namespace hodlr
