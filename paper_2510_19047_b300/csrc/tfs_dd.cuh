// Double-double ("dd") arithmetic in FP64: a value is hi + lo with |lo| <= ulp(hi)/2,
// ~106 significant bits. Error-free transformations after Knuth (two-sum) and Dekker
// (two-product, here with an FMA). Used where FP64 alone is not enough for the FP64
// path: the chirp constants t_c, P5, P3 and the absolute GW phase Phi(t'), which
// reaches ~1e7 rad over two years, so that one FP64 rounding of a constant (~1e-16
// relative) would already move the phase by ~1e-9 rad.
//
// Written for host and device (the device build uses the round-to-nearest intrinsics,
// which the compiler does not contract into FMAs or reorder).
#pragma once

#include <math.h>

#ifndef TFS_HD
#define TFS_HD __host__ __device__ __forceinline__
#endif

namespace tfs {

struct dd {
  double hi, lo;
};

TFS_HD double dd_add_rn(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
TFS_HD double dd_sub_rn(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
TFS_HD double dd_mul_rn(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}

// a + b exactly, for |a| >= |b| (or a = 0)
TFS_HD dd dd_quick_two_sum(double a, double b) {
  const double s = dd_add_rn(a, b);
  return dd{s, dd_sub_rn(b, dd_sub_rn(s, a))};
}
// a + b exactly
TFS_HD dd dd_two_sum(double a, double b) {
  const double s = dd_add_rn(a, b);
  const double bb = dd_sub_rn(s, a);
  return dd{s, dd_add_rn(dd_sub_rn(a, dd_sub_rn(s, bb)), dd_sub_rn(b, bb))};
}
// a * b exactly
TFS_HD dd dd_two_prod(double a, double b) {
  const double p = dd_mul_rn(a, b);
  return dd{p, fma(a, b, -p)};
}

TFS_HD dd dd_from(double a) { return dd{a, 0.0}; }
TFS_HD dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }

TFS_HD dd dd_add(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  const dd t = dd_two_sum(x.lo, y.lo);
  s = dd_quick_two_sum(s.hi, dd_add_rn(s.lo, t.hi));
  return dd_quick_two_sum(s.hi, dd_add_rn(s.lo, t.lo));
}
TFS_HD dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
TFS_HD dd dd_add_d(dd x, double b) {
  const dd s = dd_two_sum(x.hi, b);
  return dd_quick_two_sum(s.hi, dd_add_rn(s.lo, x.lo));
}
TFS_HD dd dd_mul(dd x, dd y) {
  const dd p = dd_two_prod(x.hi, y.hi);
  const double e = fma(x.hi, y.lo, fma(x.lo, y.hi, p.lo));
  return dd_quick_two_sum(p.hi, e);
}
TFS_HD dd dd_mul_d(dd x, double b) {
  const dd p = dd_two_prod(x.hi, b);
  return dd_quick_two_sum(p.hi, fma(x.lo, b, p.lo));
}
TFS_HD dd dd_sqr(dd x) { return dd_mul(x, x); }
// x / y: three quotient digits (long division by y.hi, remainders in dd)
TFS_HD dd dd_div(dd x, dd y) {
  const double q1 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q1));
  const double q2 = r.hi / y.hi;
  r = dd_sub(r, dd_mul_d(y, q2));
  const double q3 = r.hi / y.hi;
  return dd_add_d(dd_quick_two_sum(q1, q2), q3);
}
// x - floor(x) in [0, 1), to the dd value's absolute precision
TFS_HD double dd_frac(dd x) {
  double r = dd_add_rn(dd_sub_rn(x.hi, floor(x.hi)), x.lo);  // hi - floor(hi) is exact
  r = dd_sub_rn(r, floor(r));
  return r < 1.0 ? r : 0.0;
}

// Constants, rounded to dd from 50-digit values.
constexpr dd kPiDD = {3.141592653589793, 1.2246467991473532e-16};
constexpr dd k8PiDD = {25.132741228718345, 9.797174393178826e-16};
constexpr dd k16Pi5DD = {10.053096491487338, 3.91886975727153e-16};       // 16 pi / 5
constexpr dd kInv2PiDD = {0.15915494309189535, -9.839338337591243e-18};   // 1 / (2 pi)
constexpr dd kGMsunDD = {4.925490947e-06, 1.7186622153220198e-23};       // 4.925490947e-6 s
constexpr dd kCf0DD = {0.27641369047619047, 1.057355261547768e-17};       // 743 / 2688
constexpr dd kCp0DD = {0.46068948412698413, -8.8112938462314e-19};        // 3715 / 8064
constexpr dd kCp1DD = {0.5729166666666666, 3.700743415417188e-17};        // 55 / 96

// Chirp constants of a template in dd: t_c, P5, P3 of
//   Phi(t') = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)),  u = 1 - t'/t_c,
// from (M_c [M_sun], eta, f0 [Hz]). Newtonian (pn_order 0):
//   t_c = (5/256) (pi f0)^(-8/3) Mc^(-5/3), P5 = (16 pi/5) f0 t_c, P3 = 0;
// 1PN TaylorT3 (pn_order 1): M = Mc eta^(-3/5), x^3 (1 + cf x^2) = 8 pi M f0 with
//   cf = 743/2688 + 11 eta/32, then t_c = 5 M x^(-8)/eta, P5 = 2 x^(-5)/eta,
//   P3 = 2 cp x^(-3)/eta, cp = 3715/8064 + 55 eta/96.
// Each fractional power starts from its FP64 value and takes one Newton step whose
// residual is formed in dd, which squares the FP64 value's ~1e-16 relative error.
struct ChirpDD {
  dd tc, P5, P3;
  double F0, C2;  // f_src = F0 y^3 (1 + C2 y^2) (FP64)
};

TFS_HD ChirpDD chirp_dd(double Mc_sun, double eta, double f0, int pn_order) {
  ChirpDD r;
  const dd Mc = dd_mul_d(kGMsunDD, Mc_sun);
  if (pn_order == 0) {
    // w = z^(-1/3), z = (pi f0)^8 Mc^5: t_c = (5/256) w
    const dd a = dd_mul_d(kPiDD, f0);
    const dd a2 = dd_sqr(a), a4 = dd_sqr(a2), a8 = dd_sqr(a4);
    const dd b2 = dd_sqr(Mc), b4 = dd_sqr(b2), b5 = dd_mul(b4, Mc);
    const dd z = dd_mul(a8, b5);
    const double w0 = 1.0 / cbrt(z.hi);
    const dd w03 = dd_mul_d(dd_two_prod(w0, w0), w0);
    const dd res = dd_add_d(dd_neg(dd_mul(w03, z)), 1.0);  // 1 - w0^3 z
    const dd w = dd_quick_two_sum(w0, w0 * (res.hi + res.lo) * (1.0 / 3.0));
    r.tc = dd_mul_d(w, 5.0 / 256.0);  // exact scaling
    r.P5 = dd_mul(dd_mul_d(k16Pi5DD, f0), r.tc);
    r.P3 = dd_from(0.0);
    r.F0 = f0;
    r.C2 = 0.0;
    return r;
  }
  // s = eta^(-3/5): s^5 eta^3 = 1
  const double s0 = pow(eta, -0.6);
  const dd s02 = dd_two_prod(s0, s0);
  const dd s05 = dd_mul_d(dd_sqr(s02), s0);
  const dd e3 = dd_mul_d(dd_two_prod(eta, eta), eta);
  const dd res_s = dd_add_d(dd_neg(dd_mul(s05, e3)), 1.0);
  const dd s = dd_quick_two_sum(s0, s0 * (res_s.hi + res_s.lo) * 0.2);
  const dd M = dd_mul(Mc, s);
  const dd cf = dd_add(kCf0DD, dd_two_prod(11.0 / 32.0, eta));
  const dd cp = dd_add(kCp0DD, dd_mul_d(kCp1DD, eta));
  const dd yv = dd_mul_d(dd_mul(k8PiDD, M), f0);
  // x^3 + cf x^5 = yv: Newton in FP64, then one step with the residual in dd
  double x0 = cbrt(yv.hi);
  for (int it = 0; it < 50; ++it) {
    const double x2 = x0 * x0;
    const double dx = (x0 * x2 * (1.0 + cf.hi * x2) - yv.hi) / (x2 * (3.0 + 5.0 * cf.hi * x2));
    x0 -= dx;
    if (fabs(dx) < 1e-9 * x0) break;  // quadratic: the remaining error is ~1e-18 x0
  }
  {
    const dd x2 = dd_two_prod(x0, x0);
    const dd x3 = dd_mul_d(x2, x0);
    const dd x5 = dd_mul(x3, x2);
    const dd g = dd_sub(dd_add(x3, dd_mul(cf, x5)), yv);
    const double gp = x2.hi * (3.0 + 5.0 * cf.hi * x2.hi);
    const dd x = dd_quick_two_sum(x0, -(g.hi + g.lo) / gp);
    const dd xx2 = dd_sqr(x), xx3 = dd_mul(xx2, x), xx4 = dd_sqr(xx2);
    const dd xx5 = dd_mul(xx4, x), xx8 = dd_sqr(xx4);
    // t_c = 5 M / (eta x^8), P5 = 2 x^3 / (eta x^8), P3 = 2 cp x^5 / (eta x^8): one
    // reciprocal
    const dd rinv = dd_div(dd_from(1.0), dd_mul_d(xx8, eta));
    r.tc = dd_mul(dd_mul_d(M, 5.0), rinv);
    r.P5 = dd_mul_d(dd_mul(xx3, rinv), 2.0);
    r.P3 = dd_mul(dd_mul_d(cp, 2.0), dd_mul(xx5, rinv));
    // C2 = cf x^2; F0 = x^3 / (8 pi M) = f0 / (1 + C2) since x^3 (1 + cf x^2) = 8 pi M f0
    const dd c2 = dd_mul(cf, xx2);
    r.C2 = c2.hi + c2.lo;
    r.F0 = f0 / (1.0 + r.C2);
  }
  return r;
}

// Phi(t') / 2 pi in cycles, as dd, at barycentre time t' = t + d0 (t and d0 exact
// doubles), without phi0: (P5 (1 - u^(5/8)) + P3 (1 - u^(3/8))) / 2 pi. u = (t_c - t')/t_c
// is formed in dd; y = u^(-1/8) takes one Newton step (u y^8 = 1) from its FP64 value;
// u^(5/8) = u y^3 and u^(3/8) = u y^5.
TFS_HD dd chirp_cycles_dd(dd tc, dd P5, dd P3, double t, double d0) {
  const dd T = dd_add_d(dd_add_d(tc, -t), -d0);
  const dd u = dd_div(T, tc);
  const double y0 = pow(u.hi, -0.125);
  const dd y02 = dd_two_prod(y0, y0);
  const dd y08 = dd_sqr(dd_sqr(y02));
  const dd res = dd_add_d(dd_neg(dd_mul(u, y08)), 1.0);  // 1 - u y0^8
  const dd y = dd_quick_two_sum(y0, y0 * (res.hi + res.lo) * 0.125);
  const dd y2 = dd_sqr(y);
  const dd u58 = dd_mul(u, dd_mul(y2, y));
  const dd u38 = dd_mul(u58, y2);
  const dd ph = dd_add(dd_mul(P5, dd_add_d(dd_neg(u58), 1.0)), dd_mul(P3, dd_add_d(dd_neg(u38), 1.0)));
  return dd_mul(ph, kInv2PiDD);
}

}  // namespace tfs
