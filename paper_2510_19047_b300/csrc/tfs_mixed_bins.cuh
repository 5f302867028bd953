// Pixel loads and per-bin sums of the warp-per-template kernels (tfs_eval_mixed.cu,
// tfs_eval_harm.cu): FP16/BF16/FP32 pixel elements holding both channels, the paper's
// Fresnel auxiliary functions in FP32, and the phase-cancelled W'' of a general bin.
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Pixel loads: one element per (bin, tranche) holds both channels of u and w,
// ur = (Re u_A, Re u_E), ui = (Im u_A, Im u_E), w = (w_A, w_E): one 128-bit load for
// FP16/BF16 u (w is stored in FP32 in the same 16 bytes), two for FP32. raw() loads,
// cvt() widens u to FP32 at the point of use (the prefetched element stays packed).
template <int PIX>
struct PixLoad;
template <>
struct PixLoad<TFS_PIX_F32> {
  struct __align__(16) P {
    float4 u, w;
  };
  __device__ static P raw(const P* p) { return P{__ldg(&p->u), __ldg(&p->w)}; }
  __device__ static void cvt(const P& v, float2& ur, float2& ui, float2& w) {
    ur = make_float2(v.u.x, v.u.y);
    ui = make_float2(v.u.z, v.u.w);
    w = make_float2(v.w.x, v.w.y);
  }
};
template <>
struct PixLoad<TFS_PIX_F16> {
  using P = uint4;
  __device__ static float2 cv(unsigned int x) {
    __half2 h = *reinterpret_cast<__half2*>(&x);
    return __half22float2(h);
  }
  __device__ static P raw(const P* p) { return __ldg(p); }
  __device__ static void cvt(const P& v, float2& ur, float2& ui, float2& w) {
    ur = cv(v.x);
    ui = cv(v.y);
    w = make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
  }
};
template <>
struct PixLoad<TFS_PIX_BF16> {
  using P = uint4;
  __device__ static float2 cv(unsigned int x) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&x);
    return __bfloat1622float2(h);
  }
  __device__ static P raw(const P* p) { return __ldg(p); }
  __device__ static void cvt(const P& v, float2& ur, float2& ui, float2& w) {
    ur = cv(v.x);
    ui = cv(v.y);
    w = make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
  }
};

// u and w both 16-bit (the precision-study pixel types): (Re u, Im u, w) as half2 /
// bfloat162 pairs of the two channels, the last word unused.
template <>
struct PixLoad<TFS_PIX_F16_ALL> {
  using P = uint4;
  __device__ static P raw(const P* p) { return __ldg(p); }
  __device__ static void cvt(const P& v, float2& ur, float2& ui, float2& w) {
    ur = PixLoad<TFS_PIX_F16>::cv(v.x);
    ui = PixLoad<TFS_PIX_F16>::cv(v.y);
    w = PixLoad<TFS_PIX_F16>::cv(v.z);
  }
};
template <>
struct PixLoad<TFS_PIX_BF16_ALL> {
  using P = uint4;
  __device__ static P raw(const P* p) { return __ldg(p); }
  __device__ static void cvt(const P& v, float2& ur, float2& ui, float2& w) {
    ur = PixLoad<TFS_PIX_BF16>::cv(v.x);
    ui = PixLoad<TFS_PIX_BF16>::cv(v.y);
    w = PixLoad<TFS_PIX_BF16>::cv(v.z);
  }
};

// Number of general-form bins on each side of f_nm in an unrolled window (a type, so that
// the window's loops unroll at compile time).
template <int G>
struct GeneralBins {
  static constexpr int value = G;
};

// x rounded to FP16 and back: a template value held at FP16 precision (precision studies).
__device__ __forceinline__ float round_f16(float x) { return __half2float(__float2half_rn(x)); }

// The paper's auxiliary Fresnel functions f, g in FP32 with approximate division,
// branch-free: the rational forms for a <= 6 and the printed asymptotic form
// f = 1/(pi a), g = 0 beyond (Sec. "Time-frequency waveform representation").
__device__ __forceinline__ void fg_sel(float a, float& f, float& g) {
  const bool big = a > 6.0f;
  const float num = big ? 1.0f : fmaf(0.926f, a, 1.0f);
  const float den = big ? (float)kPi * a : fmaf(a, fmaf(3.104f, a, 1.792f), 2.0f);
  f = num * rcp_approx(den);
  const float e = fmaf(a, fmaf(a, fmaf(6.670f, a, 3.492f), 4.142f), 2.0f);
  g = big ? 0.0f : rcp_approx(e);
}

// General bin: W''_k = sigma pi W_k with W_k = s1 G(|v1|) - s2 G(|v2|) e^{i Psi}
// + [s1 != s2] (1+i) e^{-i pi v1^2 / 2}, G = g + i f, v = sigma x.
__device__ __forceinline__ void w_general(float x1, float x2, float sig, float spi, float cpsi,
                                          float spsi, bool sweep, float& wr, float& wi) {
  const float v1 = sig * x1, v2 = sig * x2;
  float f1, g1, f2, g2;
  fg_sel(fabsf(v1), f1, g1);
  fg_sel(fabsf(v2), f2, g2);
  const float s1 = v1 < 0.f ? -spi : spi, s2 = v2 < 0.f ? -spi : spi;
  wr = s1 * g1 - s2 * (g2 * cpsi - f2 * spsi);
  wi = s1 * f1 - s2 * (g2 * spsi + f2 * cpsi);
  if (sweep && v1 < 0.f && v2 >= 0.f) {  // f_k inside this tranche's sweep
    // e^{-i pi v1^2/2}: the argument (in units of pi) reduced to [-1, 1] on the FMA pipe,
    // then the hardware sine/cosine (~5e-7 absolute there; |v1| <= sigma eps is small)
    const float h = 0.5f * v1 * v1;
    float sp, cp;
    __sincosf(3.141592654f * (h - 2.0f * rint_small(0.5f * h)), &sp, &cp);
    wr = fmaf(spi, cp + sp, wr);
    wi = fmaf(spi, cp - sp, wi);
  }
}

// Per-tranche bin sums, channels A and E paired: with real weights q = 1/x the
// asymptotic bins need only U1 = sum u q1 and U2 = sum u q2, since
// sum conj(u) W'' = i conj(U1) - i e^{i Psi} conj(U2) for W'' = i q1 - i e^{i Psi} q2.
// A general bin with complex W'' adds i u conj(W'') to U1, which the same formula maps
// back to conj(u) W''. nn = sum w |W''|^2.
struct BinAcc {
  float2 u1r, u1i, u2r, u2i, nn;
};

template <bool R16 = false>
__device__ __forceinline__ void acc_asym(BinAcc& s, float2 ur, float2 ui, float2 w, float2 x,
                                         float m2c) {
  // x = (x1, x2); m2c = -2 cos(Psi); R16: the real weights q held at FP16 precision
  float q1 = rcp_approx(x.x), q2 = rcp_approx(x.y);
  if (R16) {
    q1 = round_f16(q1);
    q2 = round_f16(q2);
  }
  const float2 Q1 = make_float2(q1, q1), Q2 = make_float2(q2, q2);
  s.u1r = __ffma2_rn(ur, Q1, s.u1r);
  s.u1i = __ffma2_rn(ui, Q1, s.u1i);
  s.u2r = __ffma2_rn(ur, Q2, s.u2r);
  s.u2i = __ffma2_rn(ui, Q2, s.u2i);
  const float ww = fmaf(q1, fmaf(m2c, q2, q1), q2 * q2);  // |W''|^2 = q1^2 + q2^2 - 2 cos(Psi) q1 q2
  s.nn = __ffma2_rn(w, make_float2(ww, ww), s.nn);
}

__device__ __forceinline__ void acc_general(BinAcc& s, float2 ur, float2 ui, float2 w, float wr,
                                            float wi) {
  const float2 WR = make_float2(wr, wr), WI = make_float2(wi, wi);
  s.u1r = __ffma2_rn(ur, WI, __ffma2_rn(ui, make_float2(-wr, -wr), s.u1r));
  s.u1i = __ffma2_rn(ur, WR, __ffma2_rn(ui, WI, s.u1i));
  const float ww = fmaf(wr, wr, wi * wi);
  s.nn = __ffma2_rn(w, make_float2(ww, ww), s.nn);
}

}  // namespace

}  // namespace tfs
