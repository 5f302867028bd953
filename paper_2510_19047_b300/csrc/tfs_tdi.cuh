// TDI-1.5 transfer of the A and E channels for one tranche (Eq. tdi2 with the full
// response; the paper builds its TDI variables from single-link observables of a
// rigidly rotating, constant-arm constellation and evaluates the transfer at the
// tranche's central frequency f_nm).
//
// Constellation: guiding centre on a 1 AU circle at orbital phase a (cos a, sin a
// given); the spacecraft sit at L/sqrt3 from it at angles sigma_i = -a + 2 pi i/3 in
// the plane spanned by e1 = (sqrt3/2 cos a, sqrt3/2 sin a, 1/2) and
// e2 = (-sin a, cos a, 0) (the same triangle as the long-wavelength tensors).
// For the complex polarisation tensor P = A+ e+ - i Ax ex, packed as pp = A+ e+ and
// px = Ax ex (xx, yy, zz, 2xy, 2xz, 2yz), and propagation direction k = -n:
//   link s -> r, unit vector n_sr = (p_r - p_s)/L:
//     G_sr = i pi f L sinc(pi f L (1 - k.n_sr)) exp(-i pi f (L + k.(p_s + p_r))) n_sr.P.n_sr
//   z = exp(-2 pi i f L);  X = (1 - z^2) [(G_10 + z G_01) - (G_20 + z G_02)],
//   Y = (1 - z^2) [(G_21 + z G_12) - (G_01 + z G_10)],
//   Z = (1 - z^2) [(G_02 + z G_20) - (G_12 + z G_21)],
//   A = (Z - X)/sqrt2,  E = (X - 2Y + Z)/sqrt6.
// The guiding centre's barycentre delay is not here: it is in the template phase
// (t' = t + n.r/c). In the long-wavelength limit X -> -16 pi^2 f^2 L^2 D_X : P.
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

template <class T>
struct TdiMath;

template <>
struct TdiMath<double> {
  // e^{2 pi i c}
  __device__ static void cis_cycles(double c, double& s, double& co) { sincospi(2.0 * c, &s, &co); }
  // sin(pi x) / (pi x)
  __device__ static double sinc_pi(double x) {
    const double px = kPi * x;
    return fabs(px) < 1e-6 ? 1.0 - px * px / 6.0 : sinpi(x) / px;
  }
};

template <>
struct TdiMath<float> {
  __device__ static void cis_cycles(float c, float& s, float& co) {
    const float r = c - rint_small(c);  // |c| is a few cycles at most
    __sincosf(6.283185307f * r, &s, &co);
  }
  __device__ static float sinc_pi(float x) {
    const float px = 3.141592654f * x;
    if (fabsf(px) < 1e-3f) return 1.0f - px * px * (1.0f / 6.0f);
    const float r = x - 2.0f * rint_small(0.5f * x);  // sin(pi x) = sin(pi r), |r| <= 1
    return __sinf(3.141592654f * r) * rcp_approx(px);
  }
};

template <class T>
struct Cplx {
  T re, im;
};
template <class T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) { return {a.re - b.re, a.im - b.im}; }

// T_A, T_E at GW frequency f [Hz], orbital phase (ca, sa), source direction n.
template <class T>
__device__ __forceinline__ void tdi_transfer(T f, T ca, T sa, T nx, T ny, T nz, const T pp[6],
                                             const T px[6], Cplx<T>& TA, Cplx<T>& TE) {
  using M = TdiMath<T>;
  const T L = T(kArmS);
  const T h3 = T(0.8660254037844386);  // sqrt3 / 2
  const T rad = T(kArmS / 1.7320508075688772);
  const T e1[3] = {h3 * ca, h3 * sa, T(0.5)};
  const T e2[3] = {-sa, ca, T(0)};
  // cos and sin of sigma_i = -a + 2 pi i / 3
  const T cs[3] = {ca, T(-0.5) * ca + h3 * sa, T(-0.5) * ca - h3 * sa};
  const T sn[3] = {-sa, T(0.5) * sa + h3 * ca, T(0.5) * sa - h3 * ca};
  T p[3][3], kp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) p[i][k] = rad * (cs[i] * e1[k] + sn[i] * e2[k]);
    kp[i] = -(nx * p[i][0] + ny * p[i][1] + nz * p[i][2]);  // k . p_i
  }
  // n.P.n of the arm (i, j)
  auto nPn = [&](int i, int j) {
    const T iL = T(1) / L;
    const T a0 = (p[j][0] - p[i][0]) * iL, a1 = (p[j][1] - p[i][1]) * iL, a2 = (p[j][2] - p[i][2]) * iL;
    const T q[6] = {a0 * a0, a1 * a1, a2 * a2, a0 * a1, a0 * a2, a1 * a2};
    T ep = T(0), ex = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ep += q[k] * pp[k];
      ex += q[k] * px[k];
    }
    return Cplx<T>{ep, -ex};
  };
  const Cplx<T> q01 = nPn(0, 1), q02 = nPn(0, 2), q12 = nPn(1, 2);
  const T fL = f * L;
  auto link = [&](int sd, int rc, Cplx<T> q) {
    const T kn = (kp[rc] - kp[sd]) / L;
    const T amp = T(kPi) * fL * M::sinc_pi(fL * (T(1) - kn));
    T s, c;
    M::cis_cycles(T(-0.5) * f * (L + kp[sd] + kp[rc]), s, c);
    // i amp q e^{i ph}
    const Cplx<T> iq = {-amp * q.im, amp * q.re};
    return cmul(Cplx<T>{c, s}, iq);
  };
  const Cplx<T> G01 = link(0, 1, q01), G10 = link(1, 0, q01);
  const Cplx<T> G02 = link(0, 2, q02), G20 = link(2, 0, q02);
  const Cplx<T> G12 = link(1, 2, q12), G21 = link(2, 1, q12);
  T zs, zc;
  M::cis_cycles(-fL, zs, zc);
  const Cplx<T> z = {zc, zs};
  const Cplx<T> z2 = cmul(z, z);
  const Cplx<T> w = {T(1) - z2.re, -z2.im};
  const Cplx<T> X = cmul(w, csub(cadd(G10, cmul(z, G01)), cadd(G20, cmul(z, G02))));
  const Cplx<T> Y = cmul(w, csub(cadd(G21, cmul(z, G12)), cadd(G01, cmul(z, G10))));
  const Cplx<T> Z = cmul(w, csub(cadd(G02, cmul(z, G20)), cadd(G12, cmul(z, G21))));
  const T r2 = T(0.7071067811865476), r6 = T(0.4082482904638631);
  TA = {(Z.re - X.re) * r2, (Z.im - X.im) * r2};
  TE = {(X.re - T(2) * Y.re + Z.re) * r6, (X.im - T(2) * Y.im + Z.im) * r6};
}

// Out-of-line entry: keeps the transfer's registers out of the calling kernel's
// allocation (its long-wavelength path stays as it is). out = (Re T_A, Im T_A, Re T_E,
// Im T_E).
template <class T>
__device__ __noinline__ void tdi_transfer_call(T f, T ca, T sa, T nx, T ny, T nz, const T* pp,
                                               const T* px, T* out) {
  T p6[6], x6[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    p6[k] = pp[k];
    x6[k] = px[k];
  }
  Cplx<T> TA, TE;
  tdi_transfer<T>(f, ca, sa, nx, ny, nz, p6, x6, TA, TE);
  out[0] = TA.re;
  out[1] = TA.im;
  out[2] = TE.re;
  out[3] = TE.im;
}

}  // namespace tfs
