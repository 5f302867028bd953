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
  // pi a sinc(pi a u) = sin(pi a u) / u
  __device__ static double pi_a_sinc(double a, double u) {
    const double x = a * u, px = kPi * x;
    return fabs(px) < 1e-6 ? kPi * a * (1.0 - px * px / 6.0) : sinpi(x) / u;
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
  // pi a sinc(pi a u) = sin(pi a u) / u (the series below |pi a u| = 1e-3)
  __device__ static float pi_a_sinc(float a, float u) {
    const float x = a * u;
    if (fabsf(x) < 1e-3f / 3.141592654f) {
      const float px = 3.141592654f * x;
      return 3.141592654f * a * (1.0f - px * px * (1.0f / 6.0f));
    }
    const float r = x - 2.0f * rint_small(0.5f * x);
    return __sinf(3.141592654f * r) * rcp_approx(u);
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

// The constellation's geometry at orbital phase (ca, sa) = (cos a, sin a): spacecraft
// positions p_i relative to the guiding centre [s] and the products of the unit vectors
// of arms 01, 02, 12 (xx, yy, zz, xy, xz, yz). It depends on the time only, so the
// mixed kernels read it from a per-tranche table (tfs_setup.cu) instead of forming it
// for every template.
template <class T>
struct TdiGeom {
  T p[3][3];
  T q[3][6];
};
template <class T>
__device__ __forceinline__ TdiGeom<T> tdi_geom(T ca, T sa) {
  TdiGeom<T> G;
  const T h3 = T(0.8660254037844386);  // sqrt3 / 2
  const T rad = T(kArmS / 1.7320508075688772);
  const T e1[3] = {h3 * ca, h3 * sa, T(0.5)};
  const T e2[3] = {-sa, ca, T(0)};
  // cos and sin of sigma_i = -a + 2 pi i / 3
  const T cs[3] = {ca, T(-0.5) * ca + h3 * sa, T(-0.5) * ca - h3 * sa};
  const T sn[3] = {-sa, T(0.5) * sa + h3 * ca, T(0.5) * sa - h3 * ca};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) G.p[i][k] = rad * (cs[i] * e1[k] + sn[i] * e2[k]);
  const int arm_i[3] = {0, 0, 1}, arm_j[3] = {1, 2, 2};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T iL = T(1) / T(kArmS);
    const int i = arm_i[r], j = arm_j[r];
    const T a0 = (G.p[j][0] - G.p[i][0]) * iL, a1 = (G.p[j][1] - G.p[i][1]) * iL,
            a2 = (G.p[j][2] - G.p[i][2]) * iL;
    G.q[r][0] = a0 * a0;
    G.q[r][1] = a1 * a1;
    G.q[r][2] = a2 * a2;
    G.q[r][3] = a0 * a1;
    G.q[r][4] = a0 * a2;
    G.q[r][5] = a1 * a2;
  }
  return G;
}

// A geometry as a table entry of 7 float4: p[0][0..2], p[1][0..2], p[2][0..2], then
// q[0][0..5], q[1][0..5], q[2][0..5], one float of padding.
constexpr int kTdiGeomF4 = 7;
__device__ __forceinline__ void tdi_geom_store(float4* g, const TdiGeom<double>& G) {
  float v[4 * kTdiGeomF4];
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = (float)G.p[i / 3][i % 3];
#pragma unroll
  for (int i = 0; i < 18; ++i) v[9 + i] = (float)G.q[i / 6][i % 6];
  v[27] = 0.0f;
#pragma unroll
  for (int i = 0; i < kTdiGeomF4; ++i) g[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ TdiGeom<float> tdi_geom_load(const float4* __restrict__ g) {
  float v[4 * kTdiGeomF4];
#pragma unroll
  for (int i = 0; i < kTdiGeomF4; ++i) {
    const float4 x = __ldg(g + i);
    v[4 * i] = x.x;
    v[4 * i + 1] = x.y;
    v[4 * i + 2] = x.z;
    v[4 * i + 3] = x.w;
  }
  TdiGeom<float> G;
#pragma unroll
  for (int i = 0; i < 9; ++i) G.p[i / 3][i % 3] = v[i];
#pragma unroll
  for (int i = 0; i < 18; ++i) G.q[i / 6][i % 6] = v[9 + i];
  return G;
}

// The A and E transfer factors from a precomputed geometry (see tdi_transfer).
template <class T>
__device__ __forceinline__ void tdi_transfer_geom(T f, const TdiGeom<T>& G, T nx, T ny, T nz,
                                                  const T pp[6], const T px[6], Cplx<T>& TA,
                                                  Cplx<T>& TE) {
  using M = TdiMath<T>;
  const T L = T(kArmS);
  const T iL = T(1.0 / kArmS);  // a product, not a division per arm
  T kp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) kp[i] = -(nx * G.p[i][0] + ny * G.p[i][1] + nz * G.p[i][2]);  // k . p_i
  // n.P.n of arm r
  auto nPn = [&](int r) {
    T ep = T(0), ex = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ep += G.q[r][k] * pp[k];
      ex += G.q[r][k] * px[k];
    }
    return Cplx<T>{ep, -ex};
  };
  const Cplx<T> q01 = nPn(0), q02 = nPn(1), q12 = nPn(2);
  const T fL = f * L;
  // both directions of an arm share the phase factor (k.(p_s + p_r) is symmetric) and
  // differ in the sinc argument (1 - k.n versus 1 + k.n): G_ij = a_ij e, G_ji = a_ji e
  // with e = i q e^{i ph} and a = pi f L sinc(pi f L (1 -+ k.n))
  auto arm = [&](int i, int j, Cplx<T> q, Cplx<T>& e, T& aij, T& aji) {
    const T kn = (kp[j] - kp[i]) * iL;  // k . n_ij
    T s, c;
    M::cis_cycles(T(-0.5) * f * (L + kp[i] + kp[j]), s, c);
    e = cmul(Cplx<T>{c, s}, Cplx<T>{-q.im, q.re});
    aij = M::pi_a_sinc(fL, T(1) - kn);
    aji = M::pi_a_sinc(fL, T(1) + kn);
  };
  Cplx<T> e01, e02, e12;
  T a01, a10, a02, a20, a12, a21;
  arm(0, 1, q01, e01, a01, a10);
  arm(0, 2, q02, e02, a02, a20);
  arm(1, 2, q12, e12, a12, a21);
  T zs, zc;
  M::cis_cycles(-fL, zs, zc);
  const Cplx<T> z = {zc, zs};
  // z G_ij = a_ij (z e): one rotation per arm
  const Cplx<T> y01 = cmul(z, e01), y02 = cmul(z, e02), y12 = cmul(z, e12);
  // X, Y, Z without their common factor w = 1 - z^2:
  //   X = G10 + z G01 - G20 - z G02, Y = G21 + z G12 - G01 - z G10,
  //   Z = G02 + z G20 - G12 - z G21
  auto comb = [](T c1, Cplx<T> v1, T c2, Cplx<T> v2, T c3, Cplx<T> v3, T c4, Cplx<T> v4) {
    return Cplx<T>{c1 * v1.re + c2 * v2.re - c3 * v3.re - c4 * v4.re,
                   c1 * v1.im + c2 * v2.im - c3 * v3.im - c4 * v4.im};
  };
  const Cplx<T> X = comb(a10, e01, a01, y01, a20, e02, a02, y02);
  const Cplx<T> Y = comb(a21, e12, a12, y12, a01, e01, a10, y01);
  const Cplx<T> Z = comb(a02, e02, a20, y02, a12, e12, a21, y12);
  // A = w (Z - X) / sqrt2, E = w (X - 2Y + Z) / sqrt6
  const Cplx<T> z2 = cmul(z, z);
  const T r2 = T(0.7071067811865476), r6 = T(0.4082482904638631);
  const Cplx<T> w2 = {(T(1) - z2.re) * r2, -z2.im * r2}, w6 = {(T(1) - z2.re) * r6, -z2.im * r6};
  TA = cmul(w2, csub(Z, X));
  TE = cmul(w6, Cplx<T>{X.re - T(2) * Y.re + Z.re, X.im - T(2) * Y.im + Z.im});
}

// T_A, T_E at GW frequency f [Hz], orbital phase (ca, sa), source direction n.
template <class T>
__device__ __forceinline__ void tdi_transfer(T f, T ca, T sa, T nx, T ny, T nz, const T pp[6],
                                             const T px[6], Cplx<T>& TA, Cplx<T>& TE) {
  tdi_transfer_geom<T>(f, tdi_geom<T>(ca, sa), nx, ny, nz, pp, px, TA, TE);
}

// ---------------------------------------------------------------------------------
// Per-arm form for the gradient: T_c = sum_arm C[c][arm] (q_arm . (pp - i px)), with
// q_arm the products (n0 n0, n1 n1, n2 n2, n0 n1, n0 n2, n1 n2) of the arm's unit vector
// (geometry only) and C the arm's complex coefficient in channel c (A, E), which
// carries the dependence on f and on the source direction. Written over T so that a
// forward-mode dual type gives dC/d(f, n).
// ---------------------------------------------------------------------------------
template <class T>
struct TdiArms {
  Cplx<T> C[2][3];  // arms (0,1), (0,2), (1,2)
};

template <class T, class G>
__device__ __forceinline__ void tdi_arms(T f, G ca, G sa, T nx, T ny, T nz, TdiArms<T>& out,
                                         G q[3][6]) {
  using M = TdiMath<T>;
  const G L = G(kArmS);
  const G iL = G(1.0 / kArmS);
  const G h3 = G(0.8660254037844386);
  const G rad = G(kArmS / 1.7320508075688772);
  const G e1[3] = {h3 * ca, h3 * sa, G(0.5)};
  const G e2[3] = {-sa, ca, G(0)};
  const G cs[3] = {ca, G(-0.5) * ca + h3 * sa, G(-0.5) * ca - h3 * sa};
  const G sn[3] = {-sa, G(0.5) * sa + h3 * ca, G(0.5) * sa - h3 * ca};
  G p[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) p[i][k] = rad * (cs[i] * e1[k] + sn[i] * e2[k]);
  T kp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) kp[i] = -(nx * p[i][0] + ny * p[i][1] + nz * p[i][2]);
  const int ai[3] = {0, 0, 1}, aj[3] = {1, 2, 2};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const G a0 = (p[aj[r]][0] - p[ai[r]][0]) * iL, a1 = (p[aj[r]][1] - p[ai[r]][1]) * iL,
            a2 = (p[aj[r]][2] - p[ai[r]][2]) * iL;
    q[r][0] = a0 * a0;
    q[r][1] = a1 * a1;
    q[r][2] = a2 * a2;
    q[r][3] = a0 * a1;
    q[r][4] = a0 * a2;
    q[r][5] = a1 * a2;
  }
  const T fL = f * L;
  // link coefficient c_sr = i pi f L sinc(pi f L (1 - k.n_sr)) e^{-i pi f (L + k.(p_s + p_r))};
  // both directions of an arm share the phase factor
  auto lc = [&](int i, int j, Cplx<T>& cij, Cplx<T>& cji) {
    const T kn = (kp[j] - kp[i]) * iL;
    T s, c;
    M::cis_cycles(T(-0.5) * f * (L + kp[i] + kp[j]), s, c);
    const T pfl = T(kPi) * fL;
    const T aij = pfl * M::sinc_pi(fL * (T(1) - kn)), aji = pfl * M::sinc_pi(fL * (T(1) + kn));
    cij = {T(0) - aij * s, aij * c};
    cji = {T(0) - aji * s, aji * c};
  };
  Cplx<T> c01, c10, c02, c20, c12, c21;
  lc(0, 1, c01, c10);
  lc(0, 2, c02, c20);
  lc(1, 2, c12, c21);
  T zs, zc;
  M::cis_cycles(-fL, zs, zc);
  const Cplx<T> z = {zc, zs};
  const Cplx<T> z2 = cmul(z, z);
  const Cplx<T> w = {T(1) - z2.re, T(0) - z2.im};
  // arm coefficients of X, Y, Z
  const Cplx<T> x01 = cmul(w, cadd(c10, cmul(z, c01)));
  const Cplx<T> x02 = cmul(w, cadd(c20, cmul(z, c02)));
  const Cplx<T> y12 = cmul(w, cadd(c21, cmul(z, c12)));
  const Cplx<T> y01 = cmul(w, cadd(c01, cmul(z, c10)));
  const Cplx<T> z02 = cmul(w, cadd(c02, cmul(z, c20)));
  const Cplx<T> z12 = cmul(w, cadd(c12, cmul(z, c21)));
  // X = x01 P01 - x02 P02; Y = y12 P12 - y01 P01; Z = z02 P02 - z12 P12
  const T r2 = T(0.7071067811865476), r6 = T(0.4082482904638631);
  // A = (Z - X)/sqrt2
  out.C[0][0] = {T(0) - x01.re * r2, T(0) - x01.im * r2};
  out.C[0][1] = {(z02.re + x02.re) * r2, (z02.im + x02.im) * r2};
  out.C[0][2] = {T(0) - z12.re * r2, T(0) - z12.im * r2};
  // E = (X - 2Y + Z)/sqrt6
  out.C[1][0] = {(x01.re + T(2) * y01.re) * r6, (x01.im + T(2) * y01.im) * r6};
  out.C[1][1] = {(z02.re - x02.re) * r6, (z02.im - x02.im) * r6};
  out.C[1][2] = {(T(0) - T(2) * y12.re - z12.re) * r6, (T(0) - T(2) * y12.im - z12.im) * r6};
}

}  // namespace tfs
