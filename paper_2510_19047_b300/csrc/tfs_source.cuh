// Source model of a template (its per-template constants), written once over the
// scalar type R: R = double for values, R = D1 (value and one directional derivative,
// forward mode) for the derivatives of the constants with respect to theta that the
// gradient kernel contracts its adjoints with.
//
// Chirp (Sec. "Time-frequency waveform representation" expands the GW phase about
// the tranche start; the chirp model itself is the reading stated in the header):
//   Newtonian: t_c = tau0 = (5/256) (pi f0)^(-8/3) Mc^(-5/3),
//              f = f0 u^(-3/8), Phi = phi0 + (16 pi/5) f0 tau0 (1 - u^(5/8)), u = 1 - t'/t_c
//   1PN TaylorT3 in x = Theta^(-1/8), Theta = eta (t_c - t')/(5 M), M = Mc eta^(-3/5):
//              f = x^3 (1 + (743/2688 + 11 eta/32) x^2) / (8 pi M)
//              Phi = phi_c - (2/eta) (Theta^(5/8) + (3715/8064 + 55 eta/96) Theta^(3/8))
//   Both as f = F0 y^3 (1 + C2 y^2), y = u^(-1/8), Phi = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)).
// Response (Eq. tdi2 in the long-wavelength limit): T_alpha = D_alpha : (A+ e+) - i D_alpha : (Ax ex),
// with the barycentre delay t' = t + n.r(t)/c; the constants here are A+ e+, Ax ex and
// the delay's amplitudes (R/c) cos(beta) (cos lambda, sin lambda).
#pragma once

#include <math.h>

#include "tfs_internal.cuh"

namespace tfs {

struct D1 {
  double v, d;
};
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator-(D1 a) { return {-a.v, -a.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ D1 operator+(D1 a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ D1 operator+(double b, D1 a) { return {a.v + b, a.d}; }
__device__ __forceinline__ D1 operator-(D1 a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ D1 operator-(double b, D1 a) { return {b - a.v, -a.d}; }
__device__ __forceinline__ D1 operator*(D1 a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ D1 operator*(double b, D1 a) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ D1 operator/(D1 a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ D1 operator/(double a, D1 b) {
  const double q = a / b.v;
  return {q, -q * b.d / b.v};
}

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(D1 x) { return x.v; }
__device__ __forceinline__ D1 mk(double v, double d) { return {v, d}; }

__device__ __forceinline__ double r_pow(double x, double p) { return pow(x, p); }
__device__ __forceinline__ D1 r_pow(D1 x, double p) {
  const double y = pow(x.v, p);
  return {y, p * y / x.v * x.d};
}
__device__ __forceinline__ void r_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void r_sincos(D1 x, D1* s, D1* c) {
  double sv, cv;
  sincos(x.v, &sv, &cv);
  *s = {sv, cv * x.d};
  *c = {cv, -sv * x.d};
}
__device__ __forceinline__ double r_cos(double x) { return cos(x); }
__device__ __forceinline__ D1 r_cos(D1 x) { return {cos(x.v), -sin(x.v) * x.d}; }

template <class R>
struct SrcT {
  R tc, F0, C2, P5, P3, phi0, dop_c, dop_s;
  R pp[6], px[6];  // A+ e+ and Ax ex packed (xx, yy, zz, 2xy, 2xz, 2yz)
  R nz;            // sin(beta)
};

// The chirp constants (t_c, F0, C2, P5, P3) from (Mc, eta, f0).
template <class R>
__device__ void source_chirp(const R th[8], int pn_order, SrcT<R>& s) {
  const R Mc = th[0] * kGMsunS;
  const R eta = th[1];
  const R f0 = th[2];
  if (pn_order == 0) {
    const R tau0 = (5.0 / 256.0) * r_pow(kPi * f0, -8.0 / 3.0) * r_pow(Mc, -5.0 / 3.0);
    s.tc = tau0;
    s.F0 = f0;
    s.C2 = f0 * 0.0;
    s.P5 = (16.0 * kPi / 5.0) * f0 * tau0;
    s.P3 = f0 * 0.0;
  } else {
    const R M = Mc * r_pow(eta, -0.6);
    const R cf = 743.0 / 2688.0 + (11.0 / 32.0) * eta;
    const R cp = 3715.0 / 8064.0 + (55.0 / 96.0) * eta;
    const R yv = 8.0 * kPi * M * f0;
    // x^3 (1 + cf x^2) = yv: Newton on the value, then two steps in R so that the
    // derivative follows the implicit function theorem
    double x = cbrt(val(yv));
    for (int it = 0; it < 50; ++it) {
      const double x2 = x * x;
      const double dx = (x * x2 * (1.0 + val(cf) * x2) - val(yv)) / (x2 * (3.0 + 5.0 * val(cf) * x2));
      x -= dx;
      if (fabs(dx) < 1e-16 * x) break;
    }
    R xr = yv * 0.0 + x;
    for (int it = 0; it < 2; ++it) {
      const R x2 = xr * xr;
      xr = xr - (xr * x2 * (1.0 + cf * x2) - yv) / (x2 * (3.0 + 5.0 * cf * x2));
    }
    const R x2 = xr * xr, x4 = x2 * x2;
    const R Theta0 = 1.0 / (x4 * x4);
    s.tc = 5.0 * M * Theta0 / eta;
    s.F0 = xr * x2 / (8.0 * kPi * M);
    s.C2 = cf * x2;
    s.P5 = (2.0 / eta) * r_pow(Theta0, 0.625);
    s.P3 = (2.0 / eta) * cp * r_pow(Theta0, 0.375);
  }
}

// The angle-dependent constants (phi0, polarisation tensors, barycentre delay, sky
// direction) from (phi0, lambda, beta, psi, iota).
template <class R>
__device__ void source_geometry(const R th[8], SrcT<R>& s) {
  s.phi0 = th[3];
  R sl, cl, sb, cb, sps, cps;
  r_sincos(th[4], &sl, &cl);
  r_sincos(th[5], &sb, &cb);
  r_sincos(th[6], &sps, &cps);
  const R zero = th[0] * 0.0;
  const R p0[3] = {sl, -cl, zero}, q0[3] = {sb * cl, sb * sl, -cb};
  R p[3], q[3];
  for (int k = 0; k < 3; ++k) {
    p[k] = cps * p0[k] + sps * q0[k];
    q[k] = (-sps) * p0[k] + cps * q0[k];
  }
  const R ci = r_cos(th[7]);
  const R Ap = 0.5 * (1.0 + ci * ci), Ax = ci;
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k) {
    const double two = k < 3 ? 1.0 : 2.0;  // off-diagonal terms appear twice in D:e
    s.pp[k] = two * Ap * (p[ia[k]] * p[ib[k]] - q[ia[k]] * q[ib[k]]);
    s.px[k] = two * Ax * (p[ia[k]] * q[ib[k]] + q[ia[k]] * p[ib[k]]);
  }
  s.dop_c = kAuS * cb * cl;
  s.dop_s = kAuS * cb * sl;
  s.nz = sb;
}

// Template constants from theta = (Mc, eta, f0, phi0, lambda, beta, psi, iota).
template <class R>
__device__ SrcT<R> source_of(const R th[8], int pn_order) {
  SrcT<R> s;
  source_chirp<R>(th, pn_order, s);
  source_geometry<R>(th, s);
  return s;
}

}  // namespace tfs
