// Set-up kernels of libtfs: per-tranche geometry, packing of the weighted data
// u = d~ / S and weights w = 1/S into each evaluation path's layout, and the
// per-template constants (FP64, once per template per call).
#include <math.h>

#include <algorithm>

#include "tfs_dd.cuh"
#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_source.cuh"
#include "tfs_tdi.cuh"

namespace tfs {

// Long-wavelength detector tensors of A and E at detector time t (FP64), packed
// (xx, yy, zz, xy, xz, yz). The constellation's guiding centre moves on a circular
// 1 AU orbit, r = (cos a, sin a, 0), a = 2 pi t / yr; the constellation plane is
// inclined by 60 degrees (normal -r/2 + (sqrt3/2) z) and the spacecraft sit at
// angles -a + 2 pi i / 3 in that plane. X = (l01 l01 - l02 l02)/2 and cyclic,
// A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6.
__device__ void lw_tensors(double t, double DA[6], double DE[6], double* ca_out,
                           double* sa_out) {
  const double tt = fmod(t, kYearS);
  double sa, ca;
  sincospi(2.0 * tt / kYearS, &sa, &ca);
  *ca_out = ca;
  *sa_out = sa;
  const double h3 = 0.5 * sqrt(3.0);
  const double e1[3] = {h3 * ca, h3 * sa, 0.5};
  const double e2[3] = {-sa, ca, 0.0};
  double q[3][3];
  for (int i = 0; i < 3; ++i) {
    double s, c;
    sincos(-2.0 * kPi * tt / kYearS + 2.0 * kPi * i / 3.0, &s, &c);
    for (int k = 0; k < 3; ++k) q[i][k] = c * e1[k] + s * e2[k];
  }
  double D[3][6];
  for (int c = 0; c < 3; ++c) {
    double l1[3], l2[3], n1 = 0, n2 = 0;
    const int i1 = (c + 1) % 3, i2 = (c + 2) % 3;
    for (int k = 0; k < 3; ++k) {
      l1[k] = q[i1][k] - q[c][k];
      l2[k] = q[i2][k] - q[c][k];
      n1 += l1[k] * l1[k];
      n2 += l2[k] * l2[k];
    }
    n1 = rsqrt(n1);
    n2 = rsqrt(n2);
    for (int k = 0; k < 3; ++k) {
      l1[k] *= n1;
      l2[k] *= n2;
    }
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int p = 0; p < 6; ++p) D[c][p] = 0.5 * (l1[ia[p]] * l1[ib[p]] - l2[ia[p]] * l2[ib[p]]);
  }
  for (int p = 0; p < 6; ++p) {
    DA[p] = (D[2][p] - D[0][p]) * (1.0 / sqrt(2.0));
    DE[p] = (D[0][p] - 2.0 * D[1][p] + D[2][p]) * (1.0 / sqrt(6.0));
  }
}

__global__ void k_tranche_table(GridDesc g, TrancheD* td, TrancheF* tf, float4* tdi) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.n_tranche) return;
  const double t = g.t0 + (double)m * g.dT;
  TrancheD d;
  d.t = t;
  lw_tensors(t, d.DA, d.DE, &d.ca, &d.sa);
  d.pad = 0.0;
  td[m] = d;
  TrancheF f;
  f.t_hi = (float)t;
  f.t_lo = (float)(t - (double)f.t_hi);
  f.ca_hi = (float)d.ca;
  f.ca_lo = (float)(d.ca - (double)f.ca_hi);
  f.sa_hi = (float)d.sa;
  f.sa_lo = (float)(d.sa - (double)f.sa_hi);
  f.pad0 = f.pad1 = 0.0f;
  for (int p = 0; p < 6; ++p) {
    f.D[p] = make_float2((float)d.DA[p], (float)d.DE[p]);
  }
  tf[m] = f;
  tdi_geom_store(tdi + (int64_t)m * kTdiGeomF4, tdi_geom<double>(d.ca, d.sa));
}

// Largest |Re u|, |Im u| and w over the grid, and a count of invalid weights
// (negative, NaN or infinite) or non-finite data under a positive weight.
__global__ void k_absmax(int64_t n, const double* d_re, const double* d_im, const double* w,
                         unsigned long long* umax, unsigned long long* wmax, int* bad) {
  double lu = 0.0, lw = 0.0;
  int lbad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    if (!(wi >= 0.0) || isinf(wi)) {
      ++lbad;
      continue;
    }
    if (wi == 0.0) continue;
    const double ur = d_re[i] * wi, ui = d_im[i] * wi;
    if (!isfinite(ur) || !isfinite(ui)) {
      ++lbad;
      continue;
    }
    lu = fmax(lu, fmax(fabs(ur), fabs(ui)));
    lw = fmax(lw, wi);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lu = fmax(lu, __shfl_down_sync(0xffffffffu, lu, o));
    lw = fmax(lw, __shfl_down_sync(0xffffffffu, lw, o));
    lbad += __shfl_down_sync(0xffffffffu, lbad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(umax, (unsigned long long)__double_as_longlong(lu));
    atomicMax(wmax, (unsigned long long)__double_as_longlong(lw));
    if (lbad) atomicAdd(bad, lbad);
  }
}

// [c][m][k] layouts of the FP64 path (unscaled) and of the plain FP32 path (scaled by
// su, sw so that FP32 sums cannot overflow for any physical units of d and S).
__global__ void k_pack_ref(int64_t n, const double* d_re, const double* d_im, const double* w,
                           double su, double sw, double2* u64, double* w64, float2* u32,
                           float* w32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    double ur = 0.0, ui = 0.0;
    if (wi > 0.0) {
      ur = d_re[i] * wi;
      ui = d_im[i] * wi;
    }
    u64[i] = make_double2(ur, ui);
    w64[i] = wi > 0.0 ? wi : 0.0;
    u32[i] = make_float2((float)(ur * su), (float)(ui * su));
    w32[i] = (float)((wi > 0.0 ? wi : 0.0) * sw);
  }
}

// Mixed-path layout: one frequency-major plane P[k][m], m padded to `pitch`, so that
// the 32 lanes of a warp, which handle 32 consecutive tranches of one template, read
// consecutive elements. Each element holds both channels of u and w,
// (Re u_A, Re u_E, Im u_A, Im u_E, w_A, w_E): one 16-byte element for FP16/BF16 u (four
// halves) with w in FP32 (two floats, which need no widening in the kernel), 32 bytes
// for FP32; one packed f32x2 operation updates both channels' sums.
__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_b2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <int PIX>
__global__ void k_pack_mixed(GridDesc g, int pitch, const double* d_re, const double* d_im,
                             const double* w, double su, double sw, void* out) {
  const int64_t npix = (int64_t)g.n_bins * pitch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / pitch), m = (int)(i % pitch);
    float v[2][3] = {{0, 0, 0}, {0, 0, 0}};
    if (m < g.n_tranche) {
      for (int c = 0; c < g.n_chan; ++c) {
        const int64_t s = ((int64_t)c * g.n_tranche + m) * g.n_bins + k;
        const double wi = w[s];
        if (wi > 0.0) {
          v[c][0] = (float)(d_re[s] * wi * su);
          v[c][1] = (float)(d_im[s] * wi * su);
          v[c][2] = (float)(wi * sw);
        }
      }
    }
    if (PIX == TFS_PIX_F32) {
      float4* o = (float4*)out + 2 * i;
      o[0] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
      o[1] = make_float4(v[0][2], v[1][2], 0.f, 0.f);
    } else if (PIX == TFS_PIX_F16) {
      ((uint4*)out)[i] = make_uint4(pack_h2(v[0][0], v[1][0]), pack_h2(v[0][1], v[1][1]),
                                    __float_as_uint(v[0][2]), __float_as_uint(v[1][2]));
    } else if (PIX == TFS_PIX_F16_ALL) {
      ((uint4*)out)[i] = make_uint4(pack_h2(v[0][0], v[1][0]), pack_h2(v[0][1], v[1][1]),
                                    pack_h2(v[0][2], v[1][2]), 0u);
    } else if (PIX == TFS_PIX_BF16_ALL) {
      ((uint4*)out)[i] = make_uint4(pack_b2(v[0][0], v[1][0]), pack_b2(v[0][1], v[1][1]),
                                    pack_b2(v[0][2], v[1][2]), 0u);
    } else {
      ((uint4*)out)[i] = make_uint4(pack_b2(v[0][0], v[1][0]), pack_b2(v[0][1], v[1][1]),
                                    __float_as_uint(v[0][2]), __float_as_uint(v[1][2]));
    }
  }
}

// ---------------------------------------------------------------------------------
// Per-template constants.
// ---------------------------------------------------------------------------------

// Barycentre time t' at which the source-frame frequency equals f_target:
// F0 (y^3 + C2 y^5) = f_target with y = (1 - t'/t_c)^(-1/8), by Newton's method.
__device__ double time_at_frequency(double tc, double F0, double C2, double f_target) {
  double y = cbrt(f_target / F0);
  for (int it = 0; it < 30; ++it) {
    const double y2 = y * y;
    const double g = F0 * y * y2 * (1.0 + C2 * y2) - f_target;
    const double gp = F0 * y2 * (3.0 + 5.0 * C2 * y2);
    const double dy = g / gp;
    y -= dy;
    // quadratic convergence: after a step below 1e-9 y the error is ~1e-18 y
    if (fabs(dy) < 1e-9 * y) break;
  }
  const double y2 = y * y, y4 = y2 * y2;
  return tc * (1.0 - 1.0 / (y4 * y4));
}

__device__ __forceinline__ void split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// The template's constant phase K = (phi0 + P5 + P3) / 2 pi in cycles (dd).
__device__ __forceinline__ dd const_cycles(const TplConst& c) {
  const dd B = dd_add_d(dd_add(dd{c.P5, c.P5_lo}, dd{c.P3, c.P3_lo}), c.phi0);
  return dd_mul(B, kInv2PiDD);
}

__device__ TplMix mix_of(const TplConst& c) {
  TplMix t;
  split(1.0 / c.tc, t.tcinv_hi, t.tcinv_lo);
  split(c.F0, t.F0_hi, t.F0_lo);
  const dd P5c = dd_mul(dd{c.P5, c.P5_lo}, kInv2PiDD), P3c = dd_mul(dd{c.P3, c.P3_lo}, kInv2PiDD);
  split(P5c.hi, t.P5_hi, t.P5_lo);
  split(P3c.hi, t.P3_hi, t.P3_lo);
  // Phi/2pi = phi0/2pi + P5 (1 - u^5/8) + P3 (1 - u^3/8) = K - P5 u^5/8 - P3 u^3/8; the
  // integer part of K is irrelevant
  split(dd_frac(const_cycles(c)), t.K_hi, t.K_lo);
  t.dopc = (float)c.dop_c;
  t.dops = (float)c.dop_s;
  split(c.C2, t.C2_hi, t.C2_lo);
  t.fd_k = (float)(c.F0 / (8.0 * c.tc));
  t.C2x5 = (float)(5.0 * c.C2);
  for (int k = 0; k < 6; ++k) {
    t.pp[k] = (float)c.pp[k];
    t.px[k] = (float)c.px[k];
  }
  t.nx = (float)(c.dop_c / kAuS);
  t.ny = (float)(c.dop_s / kAuS);
  t.nz = (float)c.nz;
  t.pad = 0.0f;
  t.m_lo = c.m_lo;
  t.m_hi = c.m_hi;
  return t;
}

__global__ void k_setup(const double* __restrict__ theta, int64_t n, int pn_order,
                        GridDesc g, double nu_min, double nu_max, TplConst* __restrict__ out,
                        TplMix* __restrict__ mix) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double th[8];
  for (int p = 0; p < 8; ++p) th[p] = theta[(int64_t)p * n + i];
  TplConst c;
  const double Mc = th[0] * kGMsunS, eta = th[1], f0 = th[2];
  const bool ok = isfinite(th[0]) && isfinite(eta) && isfinite(f0) && isfinite(th[3]) &&
                  isfinite(th[4]) && isfinite(th[5]) && isfinite(th[6]) && isfinite(th[7]) &&
                  Mc > 0.0 && f0 > 0.0 && (pn_order == 0 || (eta > 0.0 && eta <= 0.25));
  if (!ok) {
    c = TplConst{};
    c.tc = 1.0;
    c.F0 = 1.0;
    c.key = 0xffffffffu;
    out[i] = c;
    if (mix) mix[i] = mix_of(c);
    return;
  }
  SrcT<double> src;
  source_geometry<double>(th, src);  // the chirp constants come from chirp_dd below
  // t_c, P5, P3 to double-double precision (their FP64 roundings would move a two-year
  // phase by ~1e-9 rad); the FP64 values are the dd values' leading parts
  const ChirpDD cd = chirp_dd(th[0], eta, f0, pn_order);
  c.tc = cd.tc.hi;
  c.tc_lo = cd.tc.lo;
  c.F0 = cd.F0;
  c.C2 = cd.C2;
  c.P5 = cd.P5.hi;
  c.P5_lo = cd.P5.lo;
  c.P3 = cd.P3.hi;
  c.P3_lo = cd.P3.lo;
  c.phi0 = src.phi0;
  for (int k = 0; k < 6; ++k) {
    c.pp[k] = src.pp[k];
    c.px[k] = src.px[k];
  }
  c.dop_c = src.dop_c;
  c.dop_s = src.dop_s;
  c.nz = src.nz;
  // Tranches that can be active: the window k_c +- 10 must lie in [1, N_bins - 1],
  // i.e. 10 df < nu f_nm <= (N_bins - 11) df for some harmonic nu in [nu_min, nu_max]
  // (nu = 1 for the dominant mode alone), and t' < t_c. The Doppler factor moves f by
  // at most 1.1e-4 relative and t' by at most 1 AU/c; a margin covers both.
  const double dop_f = 1.5e-4, dop_t = kAuS + 1.0;
  const double f_lo = 10.0 * g.df / (1.0 + dop_f) / nu_max;
  const double f_hi = (g.n_bins - 11) * g.df / (1.0 - dop_f) / nu_min;
  const double tp_lo = time_at_frequency(c.tc, c.F0, c.C2, f_lo);
  const double tp_hi = fmin(time_at_frequency(c.tc, c.F0, c.C2, f_hi), c.tc);
  const double T_end = g.t0 + g.n_tranche * g.dT;
  double m_lo = floor((tp_lo - dop_t - g.t0) / g.dT);
  double m_hi = floor((tp_hi + dop_t - g.t0) / g.dT) + 1.0;
  m_lo = fmax(0.0, fmin(m_lo, (double)g.n_tranche));
  m_hi = fmax(m_lo, fmin(m_hi, (double)g.n_tranche));
  if (tp_hi + dop_t < g.t0 || tp_lo - dop_t > T_end) m_hi = m_lo;
  c.m_lo = (int)m_lo;
  c.m_hi = (int)m_hi;
  // sort key: longer ranges first (in 32-tranche blocks), then by start frequency
  const int blocks = (c.m_hi - c.m_lo + 31) >> 5;
  const double tp0 = g.t0 + c.m_lo * g.dT;
  double f_start = c.F0;
  if (tp0 < c.tc) {
    const double u = 1.0 - tp0 / c.tc;
    const double y = 1.0 / sqrt(sqrt(sqrt(u))), y2 = y * y;  // u^(-1/8): a sort key only
    f_start = c.F0 * y * y2 * (1.0 + c.C2 * y2);
  }
  const int kc_lo = (int)fmin(65535.0, fmax(0.0, ceil(f_start / g.df)));
  c.kc_lo = kc_lo;
  c.key = ((uint32_t)(0xffff - min(blocks, 0xffff)) << 16) | (uint32_t)kc_lo;
  out[i] = c;
  if (mix) mix[i] = mix_of(c);
}

// Checked mode: every template's tranche range must lie inside the grid.
__global__ void k_check_tpl(const TplConst* __restrict__ tpl, int64_t n, int n_tranche, int* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const TplConst c = tpl[i];
  if (c.m_lo < 0 || c.m_hi < c.m_lo || c.m_hi > n_tranche) atomicOr(err, kDevBadIndex);
}

// ---------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------
cudaError_t launch_tranche_table(const GridDesc& g, TrancheD* td, TrancheF* tf, float4* tdi,
                                 cudaStream_t s) {
  k_tranche_table<<<(g.n_tranche + 127) / 128, 128, 0, s>>>(g, td, tf, tdi);
  return cudaGetLastError();
}

cudaError_t launch_absmax(int64_t n, const double* d_re, const double* d_im, const double* w,
                          unsigned long long* umax, unsigned long long* wmax, int* bad,
                          int n_sm, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 8);
  k_absmax<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(n, d_re, d_im, w, umax, wmax, bad);
  return cudaGetLastError();
}

cudaError_t launch_pack_ref(int64_t n, const double* d_re, const double* d_im, const double* w,
                            double su, double sw, double2* u64, double* w64, float2* u32,
                            float* w32, int n_sm, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 16);
  k_pack_ref<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(n, d_re, d_im, w, su, sw, u64, w64, u32,
                                                     w32);
  return cudaGetLastError();
}

cudaError_t launch_pack_mixed(int pix, const GridDesc& g, int pitch, const double* d_re,
                              const double* d_im, const double* w, double su, double sw, void* P,
                              int n_sm, cudaStream_t s) {
  const int64_t npix = (int64_t)g.n_bins * pitch;
  const int blocks = (int)std::min<int64_t>((npix + 255) / 256, (int64_t)n_sm * 16);
  switch (pix) {
    case TFS_PIX_F32:
      k_pack_mixed<TFS_PIX_F32><<<blocks, 256, 0, s>>>(g, pitch, d_re, d_im, w, su, sw, P);
      break;
    case TFS_PIX_F16:
      k_pack_mixed<TFS_PIX_F16><<<blocks, 256, 0, s>>>(g, pitch, d_re, d_im, w, su, sw, P);
      break;
    case TFS_PIX_F16_ALL:
      k_pack_mixed<TFS_PIX_F16_ALL><<<blocks, 256, 0, s>>>(g, pitch, d_re, d_im, w, su, sw, P);
      break;
    case TFS_PIX_BF16_ALL:
      k_pack_mixed<TFS_PIX_BF16_ALL><<<blocks, 256, 0, s>>>(g, pitch, d_re, d_im, w, su, sw, P);
      break;
    default:
      k_pack_mixed<TFS_PIX_BF16><<<blocks, 256, 0, s>>>(g, pitch, d_re, d_im, w, su, sw, P);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_check_tpl(const TplConst* tpl, int64_t n, int n_tranche, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_tpl<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tpl, n, n_tranche, err);
  return cudaGetLastError();
}

// Constant phase of each harmonic of each template: with Phi / 2 pi = K - S,
// K = (phi0 + P5 + P3) / 2 pi and S = (P5 u^(5/8) + P3 u^(3/8)) / 2 pi, harmonic h has
// phase nu_h K - nu_h S cycles; K[i][h] = frac(nu_h K), formed in double-double.
__global__ void k_harm_phase(const TplConst* __restrict__ tpl, int64_t n, HarmSet h,
                             float2* __restrict__ K) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * h.n) return;
  const int64_t i = t / h.n;
  const int q = (int)(t - i * h.n);
  const TplConst c = tpl[i];
  const df v = df_make(dd_frac(dd_mul_d(const_cycles(c), h.nu[q])));
  K[t] = make_float2(v.hi, v.lo);
}

cudaError_t launch_harm_phase(const TplConst* tpl, int64_t n, const HarmSet& h, float2* K,
                              cudaStream_t s) {
  if (n <= 0 || h.n <= 0) return cudaSuccess;
  const int64_t work = n * h.n;
  k_harm_phase<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(tpl, n, h, K);
  return cudaGetLastError();
}

cudaError_t launch_setup(const double* theta, int64_t n, int pn_order, const GridDesc& g,
                         TplConst* out, TplMix* mix, cudaStream_t s, double nu_min,
                         double nu_max) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(theta, n, pn_order, g, nu_min, nu_max, out,
                                                        mix);
  return cudaGetLastError();
}

}  // namespace tfs
