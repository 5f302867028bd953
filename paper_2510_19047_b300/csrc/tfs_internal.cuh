// Internal declarations of libtfs: data layouts, per-template constants, double-float
// arithmetic and the Fresnel auxiliary functions shared by the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tfs.h"

namespace tfs {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kGMsunS = 4.925490947e-6;  // G M_sun / c^3 [s]
constexpr double kAuS = 499.004784;         // 1 AU / c [s]
constexpr double kYearS = 31557600.0;       // Julian year [s]
constexpr double kOmega = 2.0 * kPi / kYearS;
constexpr double kArmS = 2.5e9 / 299792458.0;  // constellation arm length / c [s]
constexpr int kNF = 21;      // N_F bins per tranche
constexpr int kNFHalf = 10;  // window k_c - 10 .. k_c + 10
constexpr int kMixedPitch = 8192;  // m-pitch of the mixed pixel plane for N_t <= 8192
constexpr int kMaxLevels = 4;

// Grid geometry.
struct GridDesc {
  int n_chan, n_tranche, n_bins;
  double dT, df, t0;
};

// Segment levels of one call. seg_len[l] = N_t / N_seg[l]; anchor = lcm of the
// segment lengths (every segment of every level lies inside one anchor block);
// fine = gcd of the segment lengths (every segment is a union of fine segments).
struct Levels {
  int n;
  int seg_len[kMaxLevels];
  int anchor_len;
  int fine_len;
  int n_fine;
};

// Per-tranche geometry (FP64): start time, orbital phase and the long-wavelength
// detector tensors of A and E in packed form (xx, yy, zz, 2xy, 2xz, 2yz).
struct TrancheD {
  double t, ca, sa;
  double DA[6], DE[6];
  double pad;
};
// Same for the mixed path: double-float time and orbital cos/sin, FP32 tensors with
// the two channels' components paired, D[q] = (DA[q], DE[q]), so that both channels'
// antenna patterns are formed with packed f32x2 FMAs.
struct __align__(16) TrancheF {
  float t_hi, t_lo, ca_hi, ca_lo;
  float sa_hi, sa_lo, pad0, pad1;
  float2 D[6];
};

// Per-template constants, computed once in FP64 by the set-up kernel.
struct __align__(16) TplConst {
  double tc;          // coalescence time at the barycentre [s]
  double F0, C2;      // f(t') = F0 y^3 (1 + C2 y^2), y = (1 - t'/t_c)^(-1/8)
  double P5, P3;      // Phi(t') = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)), u = 1 - t'/t_c
  double phi0;
  double dop_c, dop_s;  // (R/c) cos(beta) cos(lambda), (R/c) cos(beta) sin(lambda)
  double pp[6], px[6];  // A+ e+ and Ax ex, packed (xx, yy, zz, 2xy, 2xz, 2yz)
  int m_lo, m_hi;       // tranche range that can be active: [m_lo, m_hi)
  uint32_t key;         // sort key (longer tracks first, then start frequency)
  int kc_lo;            // window centre bin at m_lo
  double nz;            // sin(beta): z component of the direction to the source
  double tc_lo, P5_lo, P3_lo;  // t_c, P5, P3 as double-doubles (tc + tc_lo, ...): the
                               // FP64 path's absolute phase needs them beyond FP64
};

// The same constants split for the mixed path's double-float / FP32 arithmetic
// (hi + lo pairs), so that kernel needs no FP64 instruction.
struct __align__(16) TplMix {
  float tcinv_hi, tcinv_lo;  // 1 / t_c
  float F0_hi, F0_lo;
  float P5_hi, P5_lo;        // P5 / 2 pi (cycles)
  float P3_hi, P3_lo;        // P3 / 2 pi
  float K_hi, K_lo;          // frac(phi0 / 2 pi + P5 / 2 pi + P3 / 2 pi): Phi = K - P5 u^5/8 - P3 u^3/8
  float dopc, dops;          // barycentre delay coefficients (FP32: |delay| <= 500 s)
  float C2_hi, C2_lo;        // f_src = F0 y^3 (1 + C2 y^2); C2 y^2 moves f_nm / df by
                             // up to ~1e4 bins, so C2 is kept to double-float precision
  float fd_k, C2x5;          // fdot_src = fd_k y^11 (3 + C2x5 y^2), fd_k = F0 / (8 t_c), C2x5 = 5 C2
  float pp[6], px[6];
  float nx, ny, nz, pad;     // direction to the source (TDI response)
  int m_lo, m_hi;
};

// ---------------------------------------------------------------------------------
// Paper's Fresnel auxiliary functions: C + iS = sgn(z) [(1+i)/2 - (g + i f) e^{i pi z^2/2}]
// with f, g rational for |z| <= 6 and f = 1/(pi z), g = 0 for |z| > 6 (the printed
// asymptotic form), evaluated at a = |z|.
// ---------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void fresnel_fg(T a, T& f, T& g) {
  if (a > T(6)) {
    f = T(1) / (T(kPi) * a);
    g = T(0);
  } else {
    f = (T(1) + T(0.926) * a) / (T(2) + a * (T(1.792) + T(3.104) * a));
    g = T(1) / (T(2) + a * (T(4.142) + a * (T(3.492) + T(6.670) * a)));
  }
}

// ---------------------------------------------------------------------------------
// Double-float ("df") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, giving
// ~48 significant bits from FP32 operations. Error-free transformations after Knuth
// (two-sum) and Dekker (two-product, here with an FMA). The intrinsics keep the
// compiler from contracting or reassociating the exact steps.
// ---------------------------------------------------------------------------------
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_make(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  df r;
  r.hi = __fadd_rn(a, b);
  r.lo = __fsub_rn(b, __fsub_rn(r.hi, a));
  return r;
}
__device__ __forceinline__ df two_sum(float a, float b) {
  df r;
  r.hi = __fadd_rn(a, b);
  float bb = __fsub_rn(r.hi, a);
  r.lo = __fadd_rn(__fsub_rn(a, __fsub_rn(r.hi, bb)), __fsub_rn(b, bb));
  return r;
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_add_f(df x, float b) {
  df s = two_sum(x.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ df df_mul(df x, df y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df x, float b) {
  float p = __fmul_rn(x.hi, b);
  float e = __fmaf_rn(x.hi, b, -p);
  e = __fmaf_rn(x.lo, b, e);
  return quick_two_sum(p, e);
}
// Products without the final renormalisation: (p, e) with p = fl(x.hi y.hi) and e the
// rest, |e| <~ 2^-22 |p|. Such a pair keeps ~46 bits and is a valid operand of the df
// operations above; it is used where the result only feeds further df arithmetic
// (a comparison or rounding of the value needs the normalised form).
__device__ __forceinline__ df df_mul_u(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df{p, e};
}
__device__ __forceinline__ df df_sqr_u(df x) {
  const float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(2.0f * x.hi, x.lo, e);
  return df{p, e};
}
// Sums without the final renormalisation (operands as in df_add / quick_add_f / one_minus).
__device__ __forceinline__ df df_add_u(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ df df_sub_u(df x, df y) { return df_add_u(x, df{-y.hi, -y.lo}); }
__device__ __forceinline__ df quick_add_f_u(df x, float b) {
  const df s = quick_two_sum(x.hi, b);
  return df{s.hi, __fadd_rn(s.lo, x.lo)};
}
// 1 + x for |x.hi| <= 1
__device__ __forceinline__ df one_plus_u(df x) {
  const df s = quick_two_sum(1.0f, x.hi);
  return df{s.hi, __fadd_rn(s.lo, x.lo)};
}
__device__ __forceinline__ df one_minus_u(df x) {
  const df s = quick_two_sum(1.0f, -x.hi);
  return df{s.hi, __fsub_rn(s.lo, x.lo)};
}
__device__ __forceinline__ df df_sqr(df x) {
  float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(2.0f * x.hi, x.lo, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ float df_to_f(df x) { return __fadd_rn(x.hi, x.lo); }
// x + b for |x.hi| >= |b| (or x.hi = 0): one quick two-sum in place of a two-sum
__device__ __forceinline__ df quick_add_f(df x, float b) {
  df s = quick_two_sum(x.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
// 1 - x for 0 <= x.hi <= 1 (for larger x the sign of the result is still right)
__device__ __forceinline__ df one_minus(df x) {
  df s = quick_two_sum(1.0f, -x.hi);
  return quick_two_sum(s.hi, __fsub_rn(s.lo, x.lo));
}

// ---------------------------------------------------------------------------------
// Single-instruction FP32 helpers shared by the mixed and gradient kernels.
// ---------------------------------------------------------------------------------
// Rounding to an integer on the FMA pipe (the conversion units are slow on this part):
// exact round-half-even for |x| < 2^22, and the integer value of such a float.
__device__ __forceinline__ float rint_small(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}
__device__ __forceinline__ int int_small(float x) {
  return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;
}

// Non-coherent 16-byte load kept in place (volatile: not hoisted out of the tranche
// loop, so its result does not occupy registers across it).
__device__ __forceinline__ float4 ldg_nc4(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// x^(-1/8) to ~2^-21 relative from the hardware base-2 logarithm and exponential
// (x > 0); the seed of a Newton step.
__device__ __forceinline__ float pow_m18(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.125f * l));
  return r;
}

// x^(2/3) the same way (x near 1: ~1e-7 relative, as a cube root squared).
__device__ __forceinline__ float pow_2_3(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((2.0f / 3.0f) * l));
  return r;
}

__device__ __forceinline__ df two_prod(float a, float b) {
  df r;
  r.hi = __fmul_rn(a, b);
  r.lo = __fmaf_rn(a, b, -r.hi);
  return r;
}

// The hardware reciprocal and reciprocal square root (one MUFU instruction each, ~1 ulp;
// subnormal inputs flush to zero, which the callers never pass).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Host/device status word written by checked kernels.
enum DeviceErr : int { kDevOk = 0, kDevBadIndex = 1 };

}  // namespace tfs
