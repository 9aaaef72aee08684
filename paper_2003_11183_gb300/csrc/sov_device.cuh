// Device functions of the float32 integrand and of the Student-t scale, shared
// by the single-problem integrand (prob.cu) and the batched persistent kernel (batch.cu).
#pragma once
#include "common.cuh"

namespace tlrmvn {

// ---- Student-t scale (Algorithm 7): chi_nu^-1(w0)/sqrt(nu) ------------------------
// Regularised incomplete gamma P(a,x) and Q(a,x) = 1 - P: power series below
// x = a + 1, Legendre continued fraction (modified Lentz) above.
__device__ inline void gamma_pq(double a, double x, double& P, double& Q) {
  if (!(x > 0.0)) {
    P = 0.0;
    Q = 1.0;
    return;
  }
  double lpref = a * log(x) - x - lgamma(a);
  if (x < a + 1.0) {
    double ap = a, term = 1.0 / a, sum = term;
    for (int it = 0; it < 2000; it++) {
      ap += 1.0;
      term *= x / ap;
      sum += term;
      if (fabs(term) <= fabs(sum) * 1.2e-16) break;
    }
    P = sum * exp(lpref);
    Q = 1.0 - P;
  } else {
    const double tiny = 1e-300;
    double bq = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / bq, h = d;
    for (int i = 1; i < 2000; i++) {
      double an = -i * (i - a);
      bq += 2.0;
      d = an * d + bq;
      if (fabs(d) < tiny) d = tiny;
      c = bq + an / c;
      if (fabs(c) < tiny) c = tiny;
      d = 1.0 / d;
      double del = d * c;
      h *= del;
      if (fabs(del - 1.0) <= 4.5e-16) break;  // a few ulp: exact equality may never occur
    }
    Q = exp(lpref) * h;
    P = 1.0 - Q;
  }
}

// x with P(a, x) = p (q = 1 - p exactly): Wilson-Hilferty start, Halley steps.
__device__ inline double gamma_p_inv(double a, double p, double q) {
  double z = ndtri2(p, q, log(p));
  double t = 1.0 / (9.0 * a);
  double base = 1.0 - t + z * sqrt(t);
  double x = a * base * base * base;
  if (!(x > 0.0)) x = exp((log(p) + lgamma(a + 1.0)) / a);
  const double lga = lgamma(a);
  for (int it = 0; it < 100; it++) {
    double P, Q;
    gamma_pq(a, x, P, Q);
    double f = (p < 0.5) ? (P - p) : (q - Q);
    double f1 = exp((a - 1.0) * log(x) - x - lga);
    if (!(f1 > 0.0)) break;
    double dx = f / f1;
    double h2 = (a - 1.0) / x - 1.0;
    double corr = 0.5 * dx * h2;
    double step = (fabs(corr) < 0.5) ? dx / (1.0 - corr) : dx;
    double xn = x - step;
    if (!(xn > 0.0)) xn = 0.5 * x;
    // Halley converges cubically: once a step is below 1e-12 x the next iterate
    // is exact to rounding, so stop there instead of chasing the last ulp
    const bool done = fabs(xn - x) <= 1e-12 * x;
    x = xn;
    if (done) break;
  }
  return x;
}

// ---- float32 integrand helpers ------------------------------------------------------
// Lattice value as floats for the float32 integrands: the cell midpoint of the
// point's top 32 bits, (h + 1/2) / 2^32 with h = x >> 32, through the tent map
// when periodised, |2 (h + 1/2) / 2^32 - 1| = (2a + 1) / 2^32 with a = d ^ (d >> 31)
// and d = h - 2^31 as a signed 32-bit integer (|2d + 1| = 2a + 1).  Integer
// arithmetic and two 32-bit conversions only (the float path issues no float64
// instruction).  It differs from the exact value of the 53-bit definition
// (lattice_w) by at most 2^-32 (2^-33 without the tent map): within half a
// float32 ulp for w >= 2^-8, and a relative 2^-32 / w below that.
__device__ __forceinline__ void lattice_wf(uint64_t x, int periodize, float& w, float& wc) {
  const uint32_t h = (uint32_t)(x >> 32);
  if (periodize) {
    const int32_t d = (int32_t)(h ^ 0x80000000u);
    const uint32_t a = (uint32_t)(d ^ (d >> 31));  // in [0, 2^31)
    w = fmaf((float)a, 4.656612873077393e-10f, 2.3283064365386963e-10f);                   // (2a + 1) / 2^32
    wc = fmaf((float)(0x7FFFFFFFu - a), 4.656612873077393e-10f, 2.3283064365386963e-10f);  // 1 - w
  } else {
    w = fmaf((float)h, 2.3283064365386963e-10f, 1.1641532182693481e-10f);                  // (h + 1/2) / 2^32
    wc = fmaf((float)(0xFFFFFFFFu - h), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  }
}

// eq. (2) for one variable in float32.  The one-sided case (at = -inf), which is
// the whole integrand for upper-limit problems, has a branch-free fast path for
// bt >= -12 (Phi(bt) > 1.7e-33): one complementary error function of |bt|, one
// log, and the library's float quantile (ndtri_f32); samples of one
// warp take the same instructions whatever the sign of their limit.  log Phi(bt)
// near 1 uses Goldberg's form of log1p (D. Goldberg, What every computer
// scientist should know about floating-point arithmetic, 1991, Theorem 4):
// log1p(-c) = log(s) * (-c) / (s - 1) with s = fl(1 - c).  Quantiles whose
// probability is below 1e-30 take the log of that probability from logs of its
// factors, and limits below -12 go through the log-domain code.
__device__ __forceinline__ void sov_step_f32(float at, float bt, float w, float wc, float& ld, float& y) {
  const float rs2 = (float)TLR_RSQRT2;
  if (at == -INFINITY && bt != INFINITY) {
    if (bt >= -12.0f) {
      const float h = 0.5f * erfcf(fabsf(bt) * rs2);  // Phi(-|bt|)
      const bool neg = bt < 0.0f;
      const float ph = neg ? h : 1.0f - h;  // Phi(bt)
      const float pc = neg ? 1.0f - h : h;  // 1 - Phi(bt)
      const float s1 = 1.0f - pc;
      const float lg = logf(neg ? ph : s1);
      ld = neg ? lg : ((s1 == 1.0f) ? -pc : lg * (-pc / (s1 - 1.0f)));
      const float u = w * ph, uc = pc + wc * ph;  // u + uc = 1
      const bool lower = u <= uc;
      const float pp = lower ? u : uc;
      float lpp = 0.0f;
      if (pp < 1e-30f) lpp = logf(w) + ld;  // (u underflows: its log from the logs of its factors)
      const float z = ndtri_f32(pp, lpp);
      y = lower ? z : -z;
      return;
    }
    const float t = -bt * rs2;
    const float le = logf(0.5f * erfcxf(t)) - t * t;  // log Phi(bt)
    const float lu = logf(w) + le;                      // log u, u = w Phi(bt) < 1/2
    y = ndtri_lower(expf(lu), lu);
    ld = le;
    return;
  }
  sov_step<float>(at, bt, w, wc, ld, y);
}

// Phi(-x) for x >= 0 in float32 (relative error about 1e-7 on [0, 12]; beyond
// 12 the value is below 2e-33 and only needs to be small): phi(x) R(x), with R
// the Mills ratio fitted as a degree-10 polynomial in t = 3 / (3 + x)
// (coefficients from csrc/fit_mills.py), and exp(-x^2/2) taken from
// x = xh + xl, xh the leading 12 significant bits of x, so that xh^2 is exact:
// exp(-xh^2/2) exp(-xl (x + xh)/2).  Cheaper than 0.5 erfcf(x / sqrt 2).
__device__ __forceinline__ float phi_neg_f32(float x) {
  const float xh = __int_as_float(__float_as_int(x) & 0xFFFFF000);
  const float xl = x - xh;
  const float e1 = expf(-0.5f * (xh * xh));
  const float e2 = __expf(-0.5f * (xl * (x + xh)));
  const float t = __fdividef(3.0f, 3.0f + fminf(x, 12.5f));
  float r = 2.330137213e-04f;
  r = fmaf(r, t, -7.265756279e-02f);
  r = fmaf(r, t, 3.999014199e-01f);
  r = fmaf(r, t, -8.397881985e-01f);
  r = fmaf(r, t, 7.416802049e-01f);
  r = fmaf(r, t, -2.781317532e-01f);
  r = fmaf(r, t, 3.698102236e-01f);
  r = fmaf(r, t, 2.605797350e-01f);
  r = fmaf(r, t, 3.388197124e-01f);
  r = fmaf(r, t, 3.328486085e-01f);
  r = fmaf(r, t, 1.874211193e-05f);
  return (e1 * e2) * (0.3989422804014327f * r);
}

// The same step for a caller that keeps the sample's probability as a running
// product: returns y, a factor f to multiply into the product and a log la to
// add to a separate sum (the step's probability is f exp(la)).  The one-sided
// fast path returns f = Phi(bt), except when 1 - Phi(bt) = c < 2^-12, where
// fl(1 - c) would lose c's digits and the step returns la = log1p(-c) taken as
// -c - c^2/2 (the next term is below 2^-24 c); the deep tail and two-sided
// intervals return their log.  No log is evaluated on the fast path.
// sov_step_f32_upper is the one-sided (at = -inf) case on its own.
__device__ __forceinline__ void sov_step_f32_upper(float bt, float w, float wc, float& f, float& la, float& y) {
  if (bt != INFINITY && bt >= -12.0f) {
    const float h = phi_neg_f32(fabsf(bt));  // Phi(-|bt|)
    const bool neg = bt < 0.0f;
    const float ph = neg ? h : 1.0f - h;  // Phi(bt)
    const float pc = neg ? 1.0f - h : h;  // 1 - Phi(bt)
    const bool near1 = !neg && pc < 0x1p-12f;
    f = near1 ? 1.0f : ph;
    la = near1 ? -pc * fmaf(0.5f, pc, 1.0f) : 0.0f;
    const float u = w * ph, uc = pc + wc * ph;  // u + uc = 1
    const bool lower = u <= uc;
    const float pp = lower ? u : uc;
    float lpp = 0.0f;
    if (pp < 1e-30f) lpp = logf(w) + logf(ph);  // (u underflows; here ph < 1/2, so log Phi(bt) = log ph)
    const float z = ndtri_f32(pp, lpp);
    y = lower ? z : -z;
    return;
  }
  float ld;
  sov_step_f32(-INFINITY, bt, w, wc, ld, y);
  f = 1.0f;
  la = ld;
}
__device__ __forceinline__ void sov_step_f32_prod(float at, float bt, float w, float wc, float& f, float& la,
                                                  float& y) {
  if (at == -INFINITY) {
    sov_step_f32_upper(bt, w, wc, f, la, y);
    return;
  }
  float ld;
  sov_step_f32(at, bt, w, wc, ld, y);
  f = 1.0f;
  la = ld;
}

}  // namespace tlrmvn
