// Gradient-ascent update of candidate templates (refinement of candidates by
// d Upsilon / d theta).
#include <math.h>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_source.cuh"
#include "tfs_tdi.cuh"

namespace tfs {

// theta[p][i] += step[p] grad[p][i]; phi_0 and lambda wrap to [0, 2 pi), psi to
// [0, pi); the other parameters are clamped to [lo[p], hi[p]].
__global__ void k_ascent(double* __restrict__ theta, const double* __restrict__ grad, int64_t n,
                         AscentParams p) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < 8; ++q) {
    double x = theta[(int64_t)q * n + i] + p.step[q] * grad[(int64_t)q * n + i];
    if (q == 3 || q == 4) {
      x = x - 2.0 * kPi * floor(x / (2.0 * kPi));
    } else if (q == 6) {
      x = x - kPi * floor(x / kPi);
    } else {
      x = fmin(fmax(x, p.lo[q]), p.hi[q]);
    }
    theta[(int64_t)q * n + i] = x;
  }
}

cudaError_t launch_ascent(double* theta, const double* grad, int64_t n, const AscentParams& p,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_ascent<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, grad, n, p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Adjoint gradient of Upsilon_{N_seg} (Eq. Upsilon-seg):
//   dUpsilon = sum_n Re(lambda_n dZ_n) + mu_n dN_n,
//   lambda_n = 2 s conj(Z_n) / N_n,  mu_n = -s |Z_n|^2 / N_n^2,  Upsilon = s sum |Z_n|^2/N_n
// (s folds the constant 4 delta f and the storage scales of u and w). One warp per
// template, one lane per tranche; the warps of a persistent launch take templates from a
// longest-first queue. Pass A forms Z_n, N_n in shared memory; pass B
// recomputes the track (it is never stored), the per-bin sums of the Fresnel-kernel
// derivatives with respect to v_1, v_2 and Psi, and turns them into the tranche's
// sensitivities to (f, fdot, phi, A, T_alpha). A reverse-mode step through the track
// (double-float values as in the mixed kernel, FP32 derivatives) gives the tranche's
// share of the adjoints of the 20 template constants (t_c, F0, C2, P5, P3, phi0, the
// delay amplitudes, A+ e+, Ax ex); the warp sums them per 32-tranche block and
// accumulates in FP64, and at the end contracts them with the constants' derivatives
// with respect to theta (FP64 forward mode, one direction per parameter, once per
// template). Pixels come from an FP32 frequency-major plane (coalesced across lanes).
// Bins with |v_1|, |v_2| > 6 take the paper's asymptotic Fresnel form in both passes, so
// their sums reduce to sums of u and w with real weights (powers of 1/v), folded into
// the complex sums once per tranche; only the warp's union of the other bins takes the
// full form.
// The window position and the Fresnel branch are held fixed: the almost-everywhere
// derivative.
// ---------------------------------------------------------------------------------
namespace {

constexpr unsigned kFullG = 0xffffffffu;
constexpr int kGradWarps = 4;
constexpr int kSrcFields = 21;  // tc F0 C2 P5 P3 phi0 dop_c dop_s pp[6] px[6] n_z
static_assert(kSrcFields + 3 <= 32, "one lane per field and per phase share");
#ifndef TFS_GRAD_UNROLL
#define TFS_GRAD_UNROLL 3
#endif
constexpr int kGradUnroll = TFS_GRAD_UNROLL;  // asymptotic-bin loop unroll (load batching)
#ifndef TFS_GRAD_DEPTH
#define TFS_GRAD_DEPTH 3
#endif
constexpr int kGradDepth = TFS_GRAD_DEPTH;  // pixel-load lead of pass A's unrolled window, in bins
// number of general-form bins on each side of f_nm in an unrolled window (a type, so that
// the window unrolls at compile time)
template <int G>
struct GradBins {
  static constexpr int value = G;
};

// The paper's auxiliary Fresnel functions and their derivatives at a = |v| (the
// hardware reciprocal in place of IEEE division: ~1 ulp).
__device__ __forceinline__ void fg_deriv(float a, float& f, float& g, float& fp, float& gp) {
  if (a > 6.0f) {
    const float ra = rcp_approx(a);
    f = (float)(1.0 / kPi) * ra;
    g = 0.0f;
    fp = -f * ra;
    gp = 0.0f;
  } else {
    const float N = fmaf(0.926f, a, 1.0f);
    const float D = fmaf(a, fmaf(3.104f, a, 1.792f), 2.0f);
    const float rD = rcp_approx(D);
    f = N * rD;
    fp = (0.926f * D - N * fmaf(6.208f, a, 1.792f)) * rD * rD;
    const float E = fmaf(a, fmaf(a, fmaf(6.670f, a, 3.492f), 4.142f), 2.0f);
    g = rcp_approx(E);
    gp = -fmaf(a, fmaf(20.01f, a, 6.984f), 4.142f) * g * g;
  }
}

// Warp sums of K <= 32 per-lane values, lane k receiving the sum of v[k] (0 for
// k >= K): at each of the five steps a lane keeps half of its partial sums, sends the
// other half to its partner and adds what it receives (31 shuffles instead of 5 K).
template <int K>
__device__ __forceinline__ float transpose_sum(const float (&v)[K], int lane) {
  float w[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float a = i < K ? v[i] : 0.0f, b = i + 16 < K ? v[i + 16] : 0.0f;
    const bool up = lane & 16;
    w[i] = (up ? b : a) + __shfl_xor_sync(0xffffffffu, up ? a : b, 16);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < o; ++i)
      w[i] = (up ? w[i + o] : w[i]) + __shfl_xor_sync(0xffffffffu, up ? w[i] : w[i + o], o);
  }
  return w[0];
}

// (float)j for 0 <= j < 2^22 on the FMA pipe (2^23 + j is exact in FP32)
__device__ __forceinline__ float small_int_f(int j) {
  return __fsub_rn(__int_as_float(0x4B000000 + j), 8388608.0f);
}

struct BinW {
  float wr, wi;    // W
  float a1r, a1i;  // dW/dv1
  float a2r, a2i;  // dW/dv2
  float a3r, a3i;  // dW/dPsi
};

template <bool DERIV>
__device__ __forceinline__ BinW bin_w(float v1, float v2, float cps, float sps) {
  BinW b;
  float f1, g1, fp1, gp1, f2, g2, fp2, gp2;
  fg_deriv(fabsf(v1), f1, g1, fp1, gp1);
  fg_deriv(fabsf(v2), f2, g2, fp2, gp2);
  const float s1 = v1 < 0.f ? -1.f : 1.f, s2 = v2 < 0.f ? -1.f : 1.f;
  const float G2r = g2 * cps - f2 * sps, G2i = g2 * sps + f2 * cps;  // G(|v2|) e^{i Psi}
  b.wr = s1 * g1 - s2 * G2r;
  b.wi = s1 * f1 - s2 * G2i;
  float cp = 1.f, sp = 0.f;
  const bool sweep = s1 != s2;
  if (sweep) {
    // argument in units of pi reduced to [-1, 1], then the hardware sine/cosine
    const float h = 0.5f * v1 * v1;
    __sincosf(3.141592654f * (h - 2.0f * rint_small(0.5f * h)), &sp, &cp);
    b.wr += cp + sp;  // (1+i) e^{-i pi v1^2/2}
    b.wi += cp - sp;
  }
  if (DERIV) {
    b.a1r = gp1;
    b.a1i = fp1;
    if (sweep) {
      const float k = (float)kPi * v1;  // d/dv1 of (1+i) e^{-i pi v1^2/2}
      b.a1r += k * (cp - sp);
      b.a1i -= k * (cp + sp);
    }
    b.a2r = -(gp2 * cps - fp2 * sps);
    b.a2i = -(gp2 * sps + fp2 * cps);
    b.a3r = s2 * G2i;  // -i s2 G2 e^{i Psi}
    b.a3i = -s2 * G2r;
  }
  return b;
}

// FP32 forward-mode dual in four directions (f, n_x, n_y, n_z): the TDI-1.5 arm
// coefficients and their derivatives in one evaluation.
struct DF4 {
  float v, d[4];
  __device__ DF4() {}
  __device__ DF4(double x) : v((float)x) { d[0] = d[1] = d[2] = d[3] = 0.0f; }
  __device__ DF4(float x, int dir) : v(x) {
    for (int k = 0; k < 4; ++k) d[k] = k == dir ? 1.0f : 0.0f;
  }
};
__device__ __forceinline__ DF4 operator+(DF4 a, DF4 b) {
  DF4 r;
  r.v = a.v + b.v;
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ DF4 operator-(DF4 a, DF4 b) {
  DF4 r;
  r.v = a.v - b.v;
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ DF4 operator-(DF4 a) {
  DF4 r;
  r.v = -a.v;
  for (int k = 0; k < 4; ++k) r.d[k] = -a.d[k];
  return r;
}
__device__ __forceinline__ DF4 operator*(DF4 a, DF4 b) {
  DF4 r;
  r.v = a.v * b.v;
  for (int k = 0; k < 4; ++k) r.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
__device__ __forceinline__ DF4 operator*(DF4 a, float b) {
  DF4 r;
  r.v = a.v * b;
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b;
  return r;
}
__device__ __forceinline__ DF4 operator/(DF4 a, float b) { return a * (1.0f / b); }
__device__ __forceinline__ DF4 operator+(float b, DF4 a) {
  a.v += b;
  return a;
}

// Window-relative bins jp = j - 10 that need the general Fresnel form (|v| <= 6 for v1
// or v2, or the sweep [v1, v2] holding 0), joined over the warp: the other bins take
// the asymptotic form W = (i/pi)(1/v1 - e^{i Psi}/v2), whose sums reduce to sums of
// u and w with real weights. Every lane of the warp must call this.
__device__ __forceinline__ void general_range(bool ok, float aa, float eps, float sig, int& JLO,
                                              int& JHI) {
  int jlo = 100, jhi = -100;
  if (ok) {
    const float r6 = 6.0f * rcp_approx(sig);
    jlo = (int)ceilf(aa - r6 - 0.01f);
    jhi = (int)floorf(aa + eps + r6 + 0.01f);
  }
  JLO = __reduce_min_sync(0xffffffffu, jlo);
  JHI = __reduce_max_sync(0xffffffffu, jhi);
}

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

}  // namespace

template <>
struct TdiMath<DF4> {
  __device__ static void cis_cycles(DF4 c, DF4& s, DF4& co) {
    float sv, cv;
    TdiMath<float>::cis_cycles(c.v, sv, cv);
    const float w = 6.283185307f;
    s.v = sv;
    co.v = cv;
    for (int k = 0; k < 4; ++k) {
      s.d[k] = w * cv * c.d[k];
      co.d[k] = -w * sv * c.d[k];
    }
  }
  // sin(pi x)/(pi x) and its derivative (cos(pi x) - sinc)/x (-> -pi^2 x/3 at x -> 0)
  __device__ static DF4 sinc_pi(DF4 x) {
    const float px = 3.141592654f * x.v;
    float v, dv;
    if (fabsf(px) < 1e-3f) {
      v = 1.0f - px * px * (1.0f / 6.0f);
      dv = -3.141592654f * px * (1.0f / 3.0f);
    } else {
      float s, c;
      const float r = x.v - 2.0f * rint_small(0.5f * x.v);
      __sincosf(3.141592654f * r, &s, &c);
      const float ipx = rcp_approx(px);  // 1/x = pi/(pi x)
      v = s * ipx;
      dv = (c - v) * (3.141592654f * ipx);
    }
    DF4 o;
    o.v = v;
    for (int k = 0; k < 4; ++k) o.d[k] = dv * x.d[k];
    return o;
  }
};

namespace {

struct GradArgs {
  GridDesc g;
  MixConst mc;
  int response;
  int pitch;            // m-pitch of the pixel plane
  const TrancheF* tabF;
  const float4* P;      // FP32 pixel plane [k][pitch] x {u (urA, urE, uiA, uiE), w (wA, wE, 0, 0)}
  const uint8_t* mask;
  const double* theta;  // [8][n]
  const TplConst* tpl;  // set-up constants (FP64; ranges)
  const TplMix* tplm;   // the same split into double-float / FP32
  int pn_order;
  int64_t n_tpl;
  int seg_len, n_seg;
  double scale;         // Upsilon = scale * sum |Z|^2 / N
  float twopidT, pidT2;  // 2 pi dT and pi dT^2 (FP32, formed on the host)
  double* out_stat;
  double* out_grad;     // [8][n]
  unsigned* counter;    // work tickets of the persistent launches: [0] pass A, [1] pass B
  const int32_t* perm;  // queue order (longest templates first), or null for 0..n-1
  int parts;            // work items per template: contiguous groups of its segments
  int parts_a;          // work items per template of pass A (it holds more warps)
  double* part_out;     // [max(parts, parts_a)][9][n] partial sums: field 0 (Upsilon) from
                        // pass A when parts_a > 1, fields 1-8 from pass B when parts > 1
  const double* dsrc;   // [n][8][kSrcFields]: d(template constant)/d theta_p (k_grad_src)
  float4* lam;          // [n][n_seg]: (Re lambda, Im lambda, mu, 0) per segment (k_grad_a)
};

// The track at the start of tranche m: the mixed kernel's double-float evaluation
// (retarded time, u = 1 - t'/t_c, y = u^(-1/8), f, the phase in cycles), plus the FP32
// intermediates the reverse-mode step needs.
struct Trk {
  bool ok;
  int kc;
  float aa, eps, sig, e2;  // f/df - k_c; fdot dT/df; df sqrt(2/fdot); sigma eps
  float cps, sps;          // e^{i Psi}
  float cph, sph;          // e^{i phi}
  float P;                 // A / sqrt(2 fdot)
  float f, fdot, amp, u, tpr, y, y2, onec, fsrc, fdsrc, d1, d2, ca, sa;  // tpr = t'/t_c = 1 - u
  df ud, yd, tprd;  // u, y, t'/t_c as double-floats (for the phase terms)
  float Tr[2], Ti[2];      // response (no amplitude)
};

template <bool TDI>
__device__ __forceinline__ Trk track_df(const GradArgs& a, const TplMix* cp, int m) {
  Trk k;
  k.ok = false;
  if (!a.mask[m]) return k;
  const float4* cq = reinterpret_cast<const float4*>(cp);
  const float4 c0 = ldg_nc4(cq), c1 = ldg_nc4(cq + 1), c2 = ldg_nc4(cq + 2), c3 = ldg_nc4(cq + 3);
  const df tc_inv = {c0.x, c0.y}, F0 = {c0.z, c0.w};
  const df P5 = {c1.x, c1.y}, P3 = {c1.z, c1.w};
  const df Kc = {c2.x, c2.y};
  const float dopc = c2.z, dops = c2.w;
  const df C2 = {c3.x, c3.y};
  const float fd_k = c3.z, C2x5 = c3.w;
  const TrancheF tr = a.tabF[m];
  float d0 = 0.f, d1 = 0.f, d2 = 0.f;
  if (a.response) {
    d0 = fmaf(dopc, tr.ca_hi, dops * tr.sa_hi);
    d1 = (float)kOmega * (dops * tr.ca_hi - dopc * tr.sa_hi);
    d2 = -(float)(kOmega * kOmega) * d0;
  }
  const df tp = df_add_f(df{tr.t_hi, tr.t_lo}, d0);
  const df tpr = df_mul(tp, tc_inv);
  const df u = df_sub(df{1.0f, 0.0f}, tpr);
  if (!(u.hi > 0.f)) return k;
  const float y0 = pow_m18(u.hi);
  const df y02 = two_prod(y0, y0);
  const df p = df_mul(u, df_sqr(df_sqr(y02)));
  const float r = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);
  const df y = quick_two_sum(y0, y0 * r * 0.125f);
  const df y2 = df_sqr(y);
  const df y3 = df_mul(y2, y);
  const df c2y2d = df_mul(C2, y2);
  const float c2y2 = c2y2d.hi;
  const df onec = df_add(df{1.0f, 0.0f}, c2y2d);
  const df fs = df_mul(df_mul(F0, y3), onec);
  const df f = df_add_f(fs, fs.hi * d1);
  const float y2f = y2.hi, y3f = y3.hi;
  const float fds = fd_k * (y3f * y3f * y3f * y2f) * fmaf(C2x5, y2f, 3.0f);
  const float fdot = fds * (1.0f + d1) * (1.0f + d1) + fs.hi * d2;
  const df x = df_mul(f, df{a.mc.dT_hi, a.mc.dT_lo});
  const bool inband = x.hi > (float)kNFHalf && x.hi < a.mc.x_hi;
  float kcf = rint_small(inband ? x.hi : 0.0f);
  if (kcf < x.hi || (kcf == x.hi && x.lo > 0.f)) kcf += 1.0f;
  const int kc = int_small(kcf);
  if (!inband || !(fdot > 0.f) || kc - kNFHalf < 1 || kc + kNFHalf > a.g.n_bins - 1) return k;
  k.ok = true;
  k.kc = kc;
  k.aa = __fadd_rn(__fsub_rn(x.hi, kcf), x.lo);
  k.f = f.hi;
  k.fdot = fdot;
  k.sig = a.mc.sig_k * rsqrt_approx(fdot);
  k.eps = fdot * a.mc.dTf * a.mc.dTf;
  k.e2 = k.sig * k.eps;
  const float psi = fmaf(2.0f, k.aa, k.eps);
  __sincosf(3.141592654f * (psi - 2.0f * rint_small(0.5f * psi)), &k.sps, &k.cps);
  const df ph = df_sub(Kc, df_mul(df_mul(u, y3), df_add(P5, df_mul(P3, y2))));
  float cyc = __fadd_rn(__fsub_rn(ph.hi, rintf(ph.hi)), ph.lo);
  cyc = __fsub_rn(cyc, rint_small(cyc));
  __sincosf(6.283185307f * cyc, &k.sph, &k.cph);
  k.amp = y2f * pow_2_3(onec.hi);  // (f/F0)^(2/3) = y^2 (1 + C2 y^2)^(2/3)
  k.P = k.amp * rsqrt_approx(2.0f * fdot);
  k.u = u.hi;
  k.tpr = tpr.hi;
  k.ud = u;
  k.yd = y;
  k.tprd = tpr;
  k.y = y.hi;
  k.y2 = y2f;
  k.onec = onec.hi;
  k.fsrc = fs.hi;
  k.fdsrc = fds;
  k.d1 = d1;
  k.d2 = d2;
  k.ca = tr.ca_hi;
  k.sa = tr.sa_hi;
  if (a.response) {
    const float4* pq = reinterpret_cast<const float4*>(cp->pp);
    const float4 q0 = ldg_nc4(pq), q1 = ldg_nc4(pq + 1), q2 = ldg_nc4(pq + 2);
    const float pp[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
    const float px[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
    if (TDI) {
      const float4 nq = ldg_nc4(pq + 3);  // direction to the source
      Cplx<float> TA, TE;
      tdi_transfer<float>(f.hi, tr.ca_hi, tr.sa_hi, nq.x, nq.y, nq.z, pp, px, TA, TE);
      k.Tr[0] = TA.re;
      k.Ti[0] = TA.im;
      k.Tr[1] = TE.re;
      k.Ti[1] = TE.im;
    } else {
      float fpA = 0.f, fxA = 0.f, fpE = 0.f, fxE = 0.f;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        fpA = fmaf(tr.D[q].x, pp[q], fpA);
        fxA = fmaf(tr.D[q].x, px[q], fxA);
        fpE = fmaf(tr.D[q].y, pp[q], fpE);
        fxE = fmaf(tr.D[q].y, px[q], fxE);
      }
      k.Tr[0] = fpA;
      k.Ti[0] = -fxA;
      k.Tr[1] = fpE;
      k.Ti[1] = -fxE;
    }
  } else {
    k.Tr[0] = k.Tr[1] = 1.0f;
    k.Ti[0] = k.Ti[1] = 0.0f;
  }
  return k;
}

// FP32 copies of the template constants the reverse-mode step uses (radians for P5, P3),
// and double-float ones for its phase terms (P5, P3 in cycles).
struct SrcF {
  float tc, tc_inv, inv8tc, F0, C2, P5, P3;
  df tc_inv_d, P5c, P3c;
};

// Reverse-mode step of the track for one tranche: given the tranche's sensitivities
// of Upsilon to (f, fdot, phi, ln A, T_alpha), its contribution to the adjoints g of
// the template constants (tc F0 C2 P5 P3 phi0 dop_c dop_s pp[6] px[6]). The phase's
// shares of the t_c, P5 and P3 adjoints, gph = (tc, P5, P3), are formed in double-float
// arithmetic (gph[0] in cycles, the others per radian of phase): they are large and
// cancel each other in the final contraction (the phase's leading term 2 pi f0 t does
// not depend on M_c or eta), so FP32 rounding there would dominate.
__device__ __forceinline__ void track_adjoint(const GradArgs& a, const SrcF& s, const Trk& k,
                                              const TrancheF& tr, float cf, float cfd, float cphi,
                                              float cP, const float cTr[2], const float cTi[2],
                                              float g[kSrcFields], df gph[3]) {
  const float op1 = 1.0f + k.d1;
  const float g_fsrc = cf * op1 + cfd * k.d2;
  const float g_fdsrc = cfd * op1 * op1;
  const float g_d1 = cf * k.fsrc + 2.0f * cfd * k.fdsrc * op1;
  const float g_d2 = cfd * k.fsrc;
  const float y = k.y, y2 = k.y2, y3 = y2 * y, y5 = y3 * y2, y10 = y5 * y5;
  const float dfs_dy = s.F0 * y2 * fmaf(5.0f * s.C2, y2, 3.0f);
  const float dfd_dy = s.F0 * y10 * fmaf(65.0f * s.C2, y2, 33.0f) * s.inv8tc;
  const float ionec = rcp_approx(k.onec);
  const float dlnA_dy = 2.0f * rcp_approx(y) + (4.0f / 3.0f) * s.C2 * y * ionec;
  const float g_y = g_fsrc * dfs_dy + g_fdsrc * dfd_dy + cP * dlnA_dy;
  g[2] = g_fsrc * s.F0 * y5 + g_fdsrc * s.F0 * y10 * y3 * 5.0f * s.inv8tc +
         cP * (2.0f / 3.0f) * y2 * ionec;
  g[1] = s.F0 != 0.0f ? (g_fsrc * k.fsrc + g_fdsrc * k.fdsrc) * rcp_approx(s.F0) : 0.0f;
  // phase: Phi = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)), u^(5/8) = u y^3
  const df y2d = df_sqr(k.yd), y3d = df_mul(y2d, k.yd);
  const df u58 = df_mul(k.ud, y3d);
  gph[1] = df_mul_f(one_minus(u58), cphi);
  gph[2] = df_mul_f(one_minus(df_mul(u58, y2d)), cphi);
  // dPhi/du [cycles] = -(5/8) P5 y^3 - (3/8) P3 y^5
  const df dph = df_add(df_mul_f(df_mul(s.P5c, y3d), 0.625f),
                        df_mul_f(df_mul(df_mul(s.P3c, y3d), y2d), 0.375f));
  const df gu_ph = df_mul_f(dph, -cphi);                       // cycles
  gph[0] = df_mul(df_mul(gu_ph, k.tprd), s.tc_inv_d);          // du/dtc = t'/tc^2
  g[3] = 0.0f;
  g[4] = 0.0f;
  g[5] = cphi;
  const float g_u = -g_y * y * rcp_approx(8.0f * k.u);
  g[0] = (g_u * k.tpr - g_fdsrc * k.fdsrc) * s.tc_inv;
  const float g_u_all = g_u + (float)(2.0 * kPi) * gu_ph.hi;  // for the delay amplitudes
  for (int q = 6; q < kSrcFields; ++q) g[q] = 0.0f;
  if (a.response) {
    const float g_tp = -g_u_all * s.tc_inv;
    const float w1 = (float)kOmega, w2 = (float)(kOmega * kOmega);
    g[6] = g_tp * k.ca - g_d1 * w1 * k.sa - g_d2 * w2 * k.ca;
    g[7] = g_tp * k.sa + g_d1 * w1 * k.ca - g_d2 * w2 * k.sa;
    if (a.response != 2) {  // T_alpha = D_alpha : (pp - i px); TDI: tdi_adjoint
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        g[8 + q] = cTr[0] * tr.D[q].x + cTr[1] * tr.D[q].y;
        g[14 + q] = -(cTi[0] * tr.D[q].x + cTi[1] * tr.D[q].y);
      }
    }
  }
}

// TDI-1.5 response: its share of the adjoints of A+ e+, Ax ex (linear), of the source
// direction (g[6], g[7] through n_x = dop_c / (R/c), n_y = dop_s / (R/c), and g[20] for
// n_z), and the response's own dependence on f, returned as an addition to dUpsilon/df.
// Derivatives of the arm coefficients in (f, n) by the four-direction dual.
__device__ __forceinline__ float tdi_adjoint(const TplMix* cp, const Trk& k, const float cTr[2],
                                             const float cTi[2], float g[kSrcFields]) {
  const float4* pq = reinterpret_cast<const float4*>(cp->pp);
  const float4 q0 = ldg_nc4(pq), q1 = ldg_nc4(pq + 1), q2 = ldg_nc4(pq + 2), nq = ldg_nc4(pq + 3);
  const float pp[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
  const float px[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
  TdiArms<DF4> arm;
  float q[3][6];
  tdi_arms<DF4, float>(DF4(k.f, 0), k.ca, k.sa, DF4(nq.x, 1), DF4(nq.y, 2), DF4(nq.z, 3), arm, q);
  float dfT = 0.f, dn[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    // P_arm = q . (pp - i px)
    float Pr = 0.f, Pi = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      Pr = fmaf(q[r][j], pp[j], Pr);
      Pi = fmaf(-q[r][j], px[j], Pi);
    }
    // sum over channels of Re(conj(c) dC) P and of the linear parts
    float wr = 0.f, wi = 0.f;  // sum_c (cTr C.re + cTi C.im), sum_c (cTr C.im - cTi C.re)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const Cplx<DF4>& C = arm.C[c][r];
      wr += cTr[c] * C.re.v + cTi[c] * C.im.v;
      wi += cTr[c] * C.im.v - cTi[c] * C.re.v;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        // d(C P) = dC P; Re and Im against (cTr, cTi)
        const float tr_ = C.re.d[d] * Pr - C.im.d[d] * Pi;
        const float ti_ = C.re.d[d] * Pi + C.im.d[d] * Pr;
        const float v = cTr[c] * tr_ + cTi[c] * ti_;
        if (d == 0)
          dfT += v;
        else
          dn[d - 1] += v;
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      g[8 + j] += q[r][j] * wr;
      g[14 + j] += q[r][j] * wi;
    }
  }
  g[6] += dn[0] * (float)(1.0 / kAuS);
  g[7] += dn[1] * (float)(1.0 / kAuS);
  g[20] += dn[2];
  return dfT;
}

}  // namespace

// Work item (i, h): template i's segments split into a.parts contiguous groups of
// (nearly) equal count; item h covers the tranches of group h inside [m_lo, m_hi).
// Upsilon and the gradient are sums over segments, so the items' partial sums add up
// to the template's (in a fixed order, by k_grad_reduce).
// Tranche range [mA, mB) of work item (template with range [m_lo, m_hi), group h);
// false for an empty group.
__device__ __forceinline__ bool item_range(const GradArgs& a, int parts, int m_lo, int m_hi, int h,
                                           int& mA, int& mB) {
  mA = m_lo;
  mB = m_hi;
  if (parts > 1 && mB > mA) {
    const int s_lo = mA / a.seg_len, n_s = (mB - 1) / a.seg_len - s_lo + 1;
    mA = max(mA, (s_lo + (h * n_s) / parts) * a.seg_len);
    mB = min(mB, (s_lo + ((h + 1) * n_s) / parts) * a.seg_len);
  }
  return mB > mA;
}

// Pass A of work item (i, [mA, mB)): Z_n, N_n of its segments folded in the warp's seg
// slots, then the adjoint weights (lambda, mu) of those segments stored to a.lam. Returns
// the item's share of Upsilon (on every lane).
template <bool TDI>
__device__ __forceinline__ double grad_pass_a(const GradArgs& a, int64_t i, int mA, int mB, int lane,
                                              float4* seg) {
  const int nch = a.g.n_chan;
  const int64_t pitch2 = 2 * (int64_t)a.pitch;  // float4 units per pixel row
  const TplMix* cp = a.tplm + i;
  for (int q = lane; q < a.n_seg; q += 32) seg[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();

  // ---- pass A: Z_n, N_n ----
  for (int m0 = mA; m0 < mB; m0 += 32) {
    const int m = m0 + lane;
    const bool inr = m < mB;
    float Zr = 0.f, Zi = 0.f, Nn = 0.f;
    Trk L;
    L.ok = false;
    if (inr) L = track_df<TDI>(a, cp, m);
    int JLO, JHI;
    general_range(L.ok, L.aa, L.eps, L.sig, JLO, JHI);
    {
      if (L.ok) {
        const int g0 = max(0, min(kNF, JLO + kNFHalf)), g1 = max(g0, min(kNF, JHI + kNFHalf + 1));
        const float4* Pp = a.P + (int64_t)(L.kc - kNFHalf) * pitch2 + 2 * (int64_t)m;
        // asymptotic bins: A1 = sum u/v1, A2 = sum u/v2, Q = sum w |pi W|^2 (channels
        // paired); sum conj(u) W over them = (i/pi)(conj(A1) - e^{i Psi} conj(A2))
        float2 A1r = f2(0.f), A1i = f2(0.f), A2r = f2(0.f), A2i = f2(0.f), Q = f2(0.f);
        const float m2c = -2.0f * L.cps;
        auto asym = [&](const float4& u, const float4& w, float v1) {
          const float q1 = rcp_approx(v1), q2 = rcp_approx(v1 + L.e2);
          const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w);
          A1r = __ffma2_rn(ur, f2(q1), A1r);
          A1i = __ffma2_rn(ui, f2(q1), A1i);
          A2r = __ffma2_rn(ur, f2(q2), A2r);
          A2i = __ffma2_rn(ui, f2(q2), A2i);
          Q = __ffma2_rn(make_float2(w.x, w.y), f2(fmaf(q1, fmaf(m2c, q2, q1), q2 * q2)), Q);
        };
        // general bins: direct sums of conj(u) W and w |W|^2
        float gzr[2] = {0.f, 0.f}, gzi[2] = {0.f, 0.f}, gnn[2] = {0.f, 0.f};
        auto general = [&](const float4& u, const float4& w, float v1) {
          const BinW b = bin_w<false>(v1, v1 + L.e2, L.cps, L.sps);
          const float ww = b.wr * b.wr + b.wi * b.wi;
          gzr[0] += u.x * b.wr + u.z * b.wi;
          gzi[0] += u.x * b.wi - u.z * b.wr;
          gnn[0] += w.x * ww;
          gzr[1] += u.y * b.wr + u.w * b.wi;
          gzi[1] += u.y * b.wi - u.w * b.wr;
          gnn[1] += w.y * ww;
        };
        // fully unrolled window when the warp's general bins lie in jp = -G .. G-1: those
        // first, then the asymptotic bins with their loads kGradDepth bins ahead
        auto unrolled = [&](auto gtag) {
          constexpr int G = decltype(gtag)::value;
          constexpr int kAsym = kNF - 2 * G;
          auto asym_bin = [](int k) { return k < kNFHalf - G ? k : k + 2 * G; };
          float4 ru[kGradDepth], rw[kGradDepth];
#pragma unroll
          for (int q = 0; q < kGradDepth; ++q) {
            ru[q] = __ldg(Pp + asym_bin(q) * pitch2);
            rw[q] = __ldg(Pp + asym_bin(q) * pitch2 + 1);
          }
#pragma unroll
          for (int h = 0; h < 2 * G; ++h) {
            const int jp = h - G;
            const float4 u = __ldg(Pp + (kNFHalf + jp) * pitch2), w = __ldg(Pp + (kNFHalf + jp) * pitch2 + 1);
            general(u, w, (L.aa - (float)jp) * L.sig);
          }
#pragma unroll
          for (int k = 0; k < kAsym; ++k) {
            const float4 u = ru[k % kGradDepth], w = rw[k % kGradDepth];
            if (k + kGradDepth < kAsym) {
              ru[k % kGradDepth] = __ldg(Pp + asym_bin(k + kGradDepth) * pitch2);
              rw[k % kGradDepth] = __ldg(Pp + asym_bin(k + kGradDepth) * pitch2 + 1);
            }
            asym(u, w, (L.aa - (float)(asym_bin(k) - kNFHalf)) * L.sig);
          }
        };
        if (JLO >= -1 && JHI <= 0) {
          unrolled(GradBins<1>{});
        } else if (JLO >= -2 && JHI <= 1) {
          unrolled(GradBins<2>{});
        } else {
          const int g0 = max(0, min(kNF, JLO + kNFHalf)), g1 = max(g0, min(kNF, JHI + kNFHalf + 1));
          // the asymptotic bins j in [0, g0) and [g1, kNF) as one counted loop
          const int n_as = kNF - (g1 - g0);
#pragma unroll kGradUnroll
          for (int i = 0; i < n_as; ++i) {
            const int j = i < g0 ? i : i + (g1 - g0);
            asym(__ldg(Pp + j * pitch2), __ldg(Pp + j * pitch2 + 1),
                 (L.aa - (small_int_f(j) - (float)kNFHalf)) * L.sig);
          }
          for (int j = g0; j < g1; ++j)
            general(__ldg(Pp + j * pitch2), __ldg(Pp + j * pitch2 + 1),
                    (L.aa - (small_int_f(j) - (float)kNFHalf)) * L.sig);
        }
        float zr[2], zi[2], nn[2];
        {
          const float ip = (float)(1.0 / kPi), ip2 = ip * ip;
          const float c = L.cps, sn = L.sps;
          zr[0] = ip * (A1i.x + sn * A2r.x - c * A2i.x) + gzr[0];
          zi[0] = ip * (A1r.x - c * A2r.x - sn * A2i.x) + gzi[0];
          nn[0] = ip2 * Q.x + gnn[0];
          zr[1] = ip * (A1i.y + sn * A2r.y - c * A2i.y) + gzr[1];
          zi[1] = ip * (A1r.y - c * A2r.y - sn * A2i.y) + gzi[1];
          nn[1] = ip2 * Q.y + gnn[1];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c >= nch) break;
          const float ar = L.Tr[c] * zr[c] - L.Ti[c] * zi[c];
          const float ai = L.Tr[c] * zi[c] + L.Ti[c] * zr[c];
          Zr += L.P * (ar * L.cph - ai * L.sph);
          Zi += L.P * (ar * L.sph + ai * L.cph);
          Nn += L.P * L.P * (L.Tr[c] * L.Tr[c] + L.Ti[c] * L.Ti[c]) * nn[c];
        }
      }
    }
    const int key = inr ? m / a.seg_len : 0x7fffffff;
    for (int o = 1; o < 32; o <<= 1) {
      const float zr2 = __shfl_down_sync(kFullG, Zr, o);
      const float zi2 = __shfl_down_sync(kFullG, Zi, o);
      const float n2 = __shfl_down_sync(kFullG, Nn, o);
      const int k2 = __shfl_down_sync(kFullG, key, o);
      if (lane + o < 32 && k2 == key) {
        Zr += zr2;
        Zi += zi2;
        Nn += n2;
      }
    }
    const int kprev = __shfl_up_sync(kFullG, key, 1);
    if (inr && (lane == 0 || kprev != key)) {
      float4 v = seg[key];
      v.x += Zr;
      v.y += Zi;
      v.z += Nn;
      seg[key] = v;
    }
  }
  __syncwarp();
  // adjoint weights of the item's segments, lambda = 2 s conj(Z)/N, mu = -s |Z|^2/N^2
  double ups = 0.0;
  const int qa = mA / a.seg_len, qb = (mB - 1) / a.seg_len;
  for (int q = qa + lane; q <= qb; q += 32) {
    const float4 v = seg[q];
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v.z > 0.f) {
      const double zz = (double)v.x * v.x + (double)v.y * v.y;
      const double inz = 1.0 / (double)v.z, t = a.scale * inz;
      ups += t * zz;
      o.x = (float)(2.0 * t * v.x);
      o.y = (float)(-2.0 * t * v.y);
      o.z = (float)(-t * zz * inz);
    }
    a.lam[(int64_t)i * a.n_seg + q] = o;
  }
  for (int o = 16; o > 0; o >>= 1) ups += __shfl_xor_sync(kFullG, ups, o);
  __syncwarp();
  return ups;
}

// Pass B of work item (i, h): the adjoints of the template constants from the stored
// (lambda, mu), contracted with the constants' theta-derivatives.
template <bool TDI>
__device__ __forceinline__ void grad_one(const GradArgs& a, int64_t i, int h, int lane) {
  const int nch = a.g.n_chan;
  const int64_t pitch2 = 2 * (int64_t)a.pitch;  // float4 units per pixel row
  const TplConst tc = a.tpl[i];
  const TplMix* cp = a.tplm + i;
  int mA, mB;
  if (!item_range(a, a.parts, tc.m_lo, tc.m_hi, h, mA, mB)) {  // empty group: zero gradient
    if (lane >= 1 && lane < 9) {
      if (a.parts > 1)
        a.part_out[((int64_t)h * 9 + lane) * a.n_tpl + i] = 0.0;
      else
        a.out_grad[(int64_t)(lane - 1) * a.n_tpl + i] = 0.0;
    }
    return;
  }
  SrcF sf;
  sf.tc = (float)tc.tc;
  sf.tc_inv = (float)(1.0 / tc.tc);
  sf.inv8tc = (float)(0.125 / tc.tc);
  sf.F0 = (float)tc.F0;
  sf.C2 = (float)tc.C2;
  sf.P5 = (float)tc.P5;
  sf.P3 = (float)tc.P3;
  sf.tc_inv_d = df_make(1.0 / tc.tc);
  sf.P5c = df_make(tc.P5 * (0.5 / kPi));
  sf.P3c = df_make(tc.P3 * (0.5 / kPi));

  // ---- pass B: adjoints of the template constants ----
  // per 32-tranche block the lanes' FP32 contributions are summed over the warp; lane
  // k < 21 accumulates field k across blocks in FP64, lanes 21-23 the phase shares of
  // t_c, P5, P3 (one FP64 add per lane and block: the FP64 pipe is slow)
  double Gown = 0.0;
  const float twopidT = a.twopidT, pidT2 = a.pidT2;
  for (int m0 = mA; m0 < mB; m0 += 32) {
    const int m = m0 + lane;
    float gl[kSrcFields];
    for (int k = 0; k < kSrcFields; ++k) gl[k] = 0.0f;
    df gph[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    Trk L;
    L.ok = false;
    if (m < mB) L = track_df<TDI>(a, cp, m);
    int JLO, JHI;
    general_range(L.ok, L.aa, L.eps, L.sig, JLO, JHI);
    if (L.ok) {
      const float4 lm = __ldg(a.lam + (int64_t)i * a.n_seg + m / a.seg_len);
      const float lr = lm.x, li = lm.y, mu = lm.z;
      // general bins j in [g0, g1) (warp-uniform); the rest take the asymptotic form
      const int g0 = max(0, min(kNF, JLO + kNFHalf)), g1 = max(g0, min(kNF, JHI + kNFHalf + 1));
      const float4* Pp = a.P + (int64_t)(L.kc - kNFHalf) * pitch2 + 2 * (int64_t)m;
      // per channel: complex sums S0..S3, S1v, S2v and real sums R0..R3, R1v, R2v
      float S[2][6][2], R[2][6];
      {
        // asymptotic bins (q = 1/v, channels paired): complex sums of u with weights
        // q1, q2, q1^2, q2^2, v1 q2^2 and real sums of w with weights q1^2, q2^2, q1 q2,
        // q1^3, q1^2 q2, q1 q2^2, q2^3, v1 q2^3
        float2 A1r = f2(0.f), A1i = f2(0.f), A2r = f2(0.f), A2i = f2(0.f), B1r = f2(0.f),
               B1i = f2(0.f), B2r = f2(0.f), B2i = f2(0.f), C2r = f2(0.f), C2i = f2(0.f);
        float2 Q11 = f2(0.f), Q22 = f2(0.f), Q12 = f2(0.f), Q111 = f2(0.f), Q112 = f2(0.f),
               Q122 = f2(0.f), Q222 = f2(0.f), V222 = f2(0.f);
        const int n_as = kNF - (g1 - g0);
#pragma unroll kGradUnroll
        for (int i = 0; i < n_as; ++i) {
          const int j = i < g0 ? i : i + (g1 - g0);
          const float4 u4 = __ldg(Pp + j * pitch2), w4 = __ldg(Pp + j * pitch2 + 1);
          const float v1 = (L.aa - (small_int_f(j) - (float)kNFHalf)) * L.sig;
          const float q1 = rcp_approx(v1), q2 = rcp_approx(v1 + L.e2);
          const float q11 = q1 * q1, q22 = q2 * q2, q12 = q1 * q2;
          const float vq22 = v1 * q22;
          const float2 ur = make_float2(u4.x, u4.y), ui = make_float2(u4.z, u4.w);
          const float2 wv = make_float2(w4.x, w4.y);
          A1r = __ffma2_rn(ur, f2(q1), A1r);
          A1i = __ffma2_rn(ui, f2(q1), A1i);
          A2r = __ffma2_rn(ur, f2(q2), A2r);
          A2i = __ffma2_rn(ui, f2(q2), A2i);
          B1r = __ffma2_rn(ur, f2(q11), B1r);
          B1i = __ffma2_rn(ui, f2(q11), B1i);
          B2r = __ffma2_rn(ur, f2(q22), B2r);
          B2i = __ffma2_rn(ui, f2(q22), B2i);
          C2r = __ffma2_rn(ur, f2(vq22), C2r);
          C2i = __ffma2_rn(ui, f2(vq22), C2i);
          Q11 = __ffma2_rn(wv, f2(q11), Q11);
          Q22 = __ffma2_rn(wv, f2(q22), Q22);
          Q12 = __ffma2_rn(wv, f2(q12), Q12);
          Q111 = __ffma2_rn(wv, f2(q11 * q1), Q111);
          Q112 = __ffma2_rn(wv, f2(q11 * q2), Q112);
          Q122 = __ffma2_rn(wv, f2(q12 * q2), Q122);
          Q222 = __ffma2_rn(wv, f2(q22 * q2), Q222);
          V222 = __ffma2_rn(wv, f2(vq22 * q2), V222);
        }
        // the asymptotic bins' S and R: with k = 1/pi and e = e^{i Psi} = c + i s,
        //   W = k i (q1 - e q2), dW/dv1 = -k i q1^2, dW/dv2 = k i e q2^2, dW/dPsi = k e q2,
        //   v1 dW/dv1 = -k i q1, v1 dW/dv2 = k i e v1 q2^2,
        // so each sum of conj(u) X is a constant times the conjugate of a sum above; and
        //   |W|^2 = k^2 (q1^2 + q2^2 - 2 c q1 q2), 2 Re(conj(W) dW/dv1) = -2k^2 (q1^3 - c q1^2 q2),
        //   2 Re(conj(W) dW/dv2) = 2k^2 (c q1 q2^2 - q2^3), 2 Re(conj(W) dW/dPsi) = 2k^2 s q1 q2,
        //   and v1 times the v1, v2 ones: -2k^2 (q1^2 - c q1 q2) and 2k^2 (c q2^2 - v1 q2^3)
        const float k1 = (float)(1.0 / kPi), k2 = k1 * k1;
        const float c = L.cps, sn = L.sps;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          const float a1r = ch ? A1r.y : A1r.x, a1i = ch ? A1i.y : A1i.x;
          const float a2r = ch ? A2r.y : A2r.x, a2i = ch ? A2i.y : A2i.x;
          const float b1r = ch ? B1r.y : B1r.x, b1i = ch ? B1i.y : B1i.x;
          const float b2r = ch ? B2r.y : B2r.x, b2i = ch ? B2i.y : B2i.x;
          const float c2r = ch ? C2r.y : C2r.x, c2i = ch ? C2i.y : C2i.x;
          S[ch][0][0] = k1 * (a1i + sn * a2r - c * a2i);
          S[ch][0][1] = k1 * (a1r - c * a2r - sn * a2i);
          S[ch][1][0] = -k1 * b1i;
          S[ch][1][1] = -k1 * b1r;
          S[ch][2][0] = -k1 * (sn * b2r - c * b2i);
          S[ch][2][1] = k1 * (c * b2r + sn * b2i);
          S[ch][3][0] = k1 * (c * a2r + sn * a2i);
          S[ch][3][1] = k1 * (sn * a2r - c * a2i);
          S[ch][4][0] = -k1 * a1i;
          S[ch][4][1] = -k1 * a1r;
          S[ch][5][0] = -k1 * (sn * c2r - c * c2i);
          S[ch][5][1] = k1 * (c * c2r + sn * c2i);
          const float q11 = ch ? Q11.y : Q11.x, q22 = ch ? Q22.y : Q22.x, q12 = ch ? Q12.y : Q12.x;
          const float q111 = ch ? Q111.y : Q111.x, q112 = ch ? Q112.y : Q112.x;
          const float q122 = ch ? Q122.y : Q122.x, q222 = ch ? Q222.y : Q222.x;
          const float v222 = ch ? V222.y : V222.x;
          R[ch][0] = k2 * (q11 + q22 - 2.f * c * q12);
          R[ch][1] = -2.f * k2 * (q111 - c * q112);
          R[ch][2] = 2.f * k2 * (c * q122 - q222);
          R[ch][3] = 2.f * k2 * sn * q12;
          R[ch][4] = -2.f * k2 * (q11 - c * q12);
          R[ch][5] = 2.f * k2 * (c * q22 - v222);
        }
      }
      // general bins: the paper's Fresnel form and its derivatives per bin
      for (int j = g0; j < g1; ++j) {
        const float4 u4 = __ldg(Pp + j * pitch2), w4 = __ldg(Pp + j * pitch2 + 1);
        const float v1 = (L.aa - (small_int_f(j) - (float)kNFHalf)) * L.sig;
        const BinW b = bin_w<true>(v1, v1 + L.e2, L.cps, L.sps);
        const float X[6][2] = {{b.wr, b.wi}, {b.a1r, b.a1i}, {b.a2r, b.a2i}, {b.a3r, b.a3i},
                               {b.a1r * v1, b.a1i * v1}, {b.a2r * v1, b.a2i * v1}};
        const float r1 = 2.f * (b.wr * b.a1r + b.wi * b.a1i);
        const float r2 = 2.f * (b.wr * b.a2r + b.wi * b.a2i);
        const float r3 = 2.f * (b.wr * b.a3r + b.wi * b.a3i);
        const float Rx[6] = {b.wr * b.wr + b.wi * b.wi, r1, r2, r3, r1 * v1, r2 * v1};
        const float ur[2] = {u4.x, u4.y}, ui[2] = {u4.z, u4.w}, wc[2] = {w4.x, w4.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            S[c][q][0] += ur[c] * X[q][0] + ui[c] * X[q][1];
            S[c][q][1] += ur[c] * X[q][1] - ui[c] * X[q][0];
            R[c][q] += wc[c] * Rx[q];
          }
        }
      }
      // sensitivities of this tranche's dUpsilon to (f, fdot, phi, A, T_alpha)
      const float P = L.P;
      const float Er = P * L.cph, Ei = P * L.sph;  // E = P e^{i phi}
      const float rt = L.sig * a.mc.dTf;  // sqrt(2 / fdot) = sigma / df
      const float ifd2 = 0.5f * rcp_approx(L.fdot);
      const float e2 = L.e2;
      float Zmr = 0, Zmi = 0, Nm = 0, cf = 0, cfd = 0, cTr[2] = {0, 0}, cTi[2] = {0, 0};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nch) break;
        const float Qr = Er * S[c][0][0] - Ei * S[c][0][1];
        const float Qi = Er * S[c][0][1] + Ei * S[c][0][0];
        const float zr = L.Tr[c] * Qr - L.Ti[c] * Qi, zi = L.Tr[c] * Qi + L.Ti[c] * Qr;
        Zmr += zr;
        Zmi += zi;
        const float T2 = L.Tr[c] * L.Tr[c] + L.Ti[c] * L.Ti[c];
        Nm += T2 * P * P * R[c][0];
        // dT terms: Re(lambda dT Q) + mu P^2 R0 d|T|^2
        cTr[c] = (lr * Qr - li * Qi) + mu * 2.0f * L.Tr[c] * P * P * R[c][0];
        cTi[c] = -(lr * Qi + li * Qr) + mu * 2.0f * L.Ti[c] * P * P * R[c][0];
        // dS0 = K1 df + K2 dfdot (complex), dR0 likewise (real)
        const float K1r = (S[c][1][0] + S[c][2][0]) * rt + S[c][3][0] * twopidT;
        const float K1i = (S[c][1][1] + S[c][2][1]) * rt + S[c][3][1] * twopidT;
        const float K2r = (-S[c][4][0] - S[c][5][0] + e2 * S[c][2][0]) * ifd2 + S[c][3][0] * pidT2;
        const float K2i = (-S[c][4][1] - S[c][5][1] + e2 * S[c][2][1]) * ifd2 + S[c][3][1] * pidT2;
        const float TEr = L.Tr[c] * Er - L.Ti[c] * Ei, TEi = L.Tr[c] * Ei + L.Ti[c] * Er;
        const float a1r = TEr * K1r - TEi * K1i, a1i = TEr * K1i + TEi * K1r;
        const float a2r = TEr * K2r - TEi * K2i, a2i = TEr * K2i + TEi * K2r;
        cf += lr * a1r - li * a1i;
        cfd += lr * a2r - li * a2i;
        const float RK1 = (R[c][1] + R[c][2]) * rt + R[c][3] * twopidT;
        const float RK2 = (-R[c][4] - R[c][5] + e2 * R[c][2]) * ifd2 + R[c][3] * pidT2;
        cf += mu * T2 * P * P * RK1;
        cfd += mu * T2 * P * P * RK2;
      }
      const float cphi = -(lr * Zmi + li * Zmr);               // Re(i lambda z)
      const float cP = (lr * Zmr - li * Zmi) + 2.0f * mu * Nm;  // coefficient of dP/P
      cfd += -cP * ifd2;
      if (TDI) {
        float tg[kSrcFields];
        for (int k = 0; k < kSrcFields; ++k) tg[k] = 0.0f;
        cf += tdi_adjoint(cp, L, cTr, cTi, tg);  // the transfer depends on f too
        track_adjoint(a, sf, L, a.tabF[m], cf, cfd, cphi, cP, cTr, cTi, gl, gph);
        for (int k = 0; k < kSrcFields; ++k) gl[k] += tg[k];
      } else {
        track_adjoint(a, sf, L, a.tabF[m], cf, cfd, cphi, cP, cTr, cTi, gl, gph);
      }
    }
    // warp sums (the phase shares in double-float; gph[0] is in cycles), each kept by
    // the lane that owns it
    float own_f = 0.0f;
    df own_d = {0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      df v = gph[k];
      for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, df{__shfl_xor_sync(kFullG, v.hi, o), __shfl_xor_sync(kFullG, v.lo, o)});
      if (lane == kSrcFields + k) own_d = v;
    }
    own_f = transpose_sum<kSrcFields>(gl, lane);
    const double sc = lane == kSrcFields ? 2.0 * kPi : 1.0;
    Gown += (double)own_f + sc * ((double)own_d.hi + (double)own_d.lo);
  }
  // d Upsilon / d theta_p = sum_k G_k d(constant_k)/d theta_p, with the phase shares
  // added to t_c, P5, P3
  double v = 0.0;
  for (int k = 0; k < kSrcFields; ++k) {
    double Gk = __shfl_sync(kFullG, Gown, k);
    if (k == 0) Gk += __shfl_sync(kFullG, Gown, kSrcFields);
    if (k == 3) Gk += __shfl_sync(kFullG, Gown, kSrcFields + 1);
    if (k == 4) Gk += __shfl_sync(kFullG, Gown, kSrcFields + 2);
    if (lane < 8) v = fma(Gk, a.dsrc[((int64_t)i * 8 + lane) * kSrcFields + k], v);
  }
  if (lane < 8) {
    if (a.parts > 1)
      a.part_out[((int64_t)h * 9 + 1 + lane) * a.n_tpl + i] = v;
    else
      a.out_grad[(int64_t)lane * a.n_tpl + i] = v;
  }
}

// Derivatives of the template constants with respect to theta (FP64 forward mode), one
// thread per (template, direction p): computed once per call, not once per work item.
__global__ void k_grad_src(const double* __restrict__ theta, int64_t n, int pn_order,
                           double* __restrict__ dsrc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * 8) return;
  const int64_t i = t >> 3;
  const int p = (int)(t & 7);
  D1 thd[8];
  for (int q = 0; q < 8; ++q) thd[q] = mk(theta[(int64_t)q * n + i], q == p ? 1.0 : 0.0);
  double* o = dsrc + t * kSrcFields;
  // the chirp constants depend on (Mc, eta, f0) only, the rest on (phi0, lambda, beta,
  // psi, iota) only: each direction evaluates its own half
  SrcT<D1> sd;
  if (p < 3) {
    source_chirp<D1>(thd, pn_order, sd);
    o[0] = sd.tc.d;
    o[1] = sd.F0.d;
    o[2] = sd.C2.d;
    o[3] = sd.P5.d;
    o[4] = sd.P3.d;
    for (int k = 5; k < kSrcFields; ++k) o[k] = 0.0;
  } else {
    source_geometry<D1>(thd, sd);
    for (int k = 0; k < 5; ++k) o[k] = 0.0;
    o[5] = sd.phi0.d;
    o[6] = sd.dop_c.d;
    o[7] = sd.dop_s.d;
    for (int q = 0; q < 6; ++q) {
      o[8 + q] = sd.pp[q].d;
      o[14 + q] = sd.px[q].d;
    }
    o[20] = sd.nz.d;
  }
}

size_t grad_src_bytes(int64_t n) { return (size_t)n * 8 * kSrcFields * sizeof(double); }

// Sum of the work items' partial sums, h = 0 .. parts-1 in order (deterministic).
__global__ void k_grad_reduce(const double* __restrict__ part, int parts_a, int parts, int64_t n,
                              double* __restrict__ out_stat, double* __restrict__ out_grad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 9 * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, i = t - r * n;
    const int np = r == 0 ? parts_a : parts;
    if (np <= 1) continue;  // that pass wrote its output directly
    double v = 0.0;
    for (int h = 0; h < np; ++h) v += part[((int64_t)h * 9 + r) * n + i];
    if (r == 0)
      out_stat[i] = v;
    else
      out_grad[(r - 1) * n + i] = v;
  }
}

#ifndef TFS_GRAD_MINB
#define TFS_GRAD_MINB 4
#endif

// Persistent launch: every warp takes templates from the queue until it is empty, so
// the long templates (first in the sorted queue) do not leave a tail of idle SMs.
// TDI: the TDI-1.5 response (code 2), as its own instantiation.
// Pass A (Upsilon and the adjoint weights) in a kernel of its own: it needs far fewer
// registers than pass B, and runs at twice the resident warps.
#ifndef TFS_GRADA_MINB
#define TFS_GRADA_MINB 8
#endif
template <bool TDI>
__global__ void __launch_bounds__(kGradWarps * 32, TDI ? 4 : TFS_GRADA_MINB) k_grad_a(GradArgs a) {
  extern __shared__ float4 s_seg[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* seg = s_seg + (size_t)warp * a.n_seg;
  for (;;) {
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(kFullG, t, 0);
    if ((int64_t)t >= a.n_tpl * a.parts_a) break;  // whole warp leaves together
    const int64_t q = (int64_t)(t / (unsigned)a.parts_a);
    const int h = (int)(t - (unsigned)q * (unsigned)a.parts_a);
    const int64_t i = a.perm ? (int64_t)a.perm[q] : q;
    int mA, mB;
    double ups = 0.0;
    if (item_range(a, a.parts_a, a.tpl[i].m_lo, a.tpl[i].m_hi, h, mA, mB))
      ups = grad_pass_a<TDI>(a, i, mA, mB, lane, seg);
    if (lane == 0) {
      if (a.parts_a > 1)
        a.part_out[(int64_t)h * 9 * a.n_tpl + i] = ups;
      else
        a.out_stat[i] = ups;
    }
    __syncwarp();  // seg is rewritten by the next item
  }
}

// Pass B, after k_grad_a has stored every item's (lambda, mu).
template <bool TDI>
__global__ void __launch_bounds__(kGradWarps * 32, TDI ? 2 : TFS_GRAD_MINB) k_grad(GradArgs a) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(a.counter + 1, 1u);
    t = __shfl_sync(kFullG, t, 0);
    if ((int64_t)t >= a.n_tpl * a.parts) break;  // whole warp leaves together
    const int64_t q = (int64_t)(t / (unsigned)a.parts);
    const int h = (int)(t - (unsigned)q * (unsigned)a.parts);
    const int64_t i = a.perm ? (int64_t)a.perm[q] : q;
    grad_one<TDI>(a, i, h, lane);
  }
}

// Resident warps of the gradient kernel and the number of work items per template:
// a small batch (fewer than ~3 waves of templates) splits each template's segments into
// up to 4 groups so that the persistent queue still ends in a short tail.
// A batch is split until its work items fill about kGradWaves waves of resident warps.
#ifndef TFS_GRAD_WAVES
#define TFS_GRAD_WAVES 3
#endif
constexpr int kGradWaves = TFS_GRAD_WAVES;

cudaError_t grad_plan(int response, int n_seg, int n_sm, int64_t n, int* parts, int* parts_a) {
  auto split = [&](int per_sm) {
    const int64_t resident = (int64_t)n_sm * std::max(per_sm, 1) * kGradWarps;
    int p = 1;
    while (p < kGradMaxParts && p < n_seg && n * p < kGradWaves * resident) ++p;
    return p;
  };
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, response == 2 ? k_grad<true> : k_grad<false>, kGradWarps * 32, 0);
  if (e != cudaSuccess) return e;
  *parts = split(per_sm);
  // pass A's occupancy with its shared segment slots
  const size_t smem = (size_t)kGradWarps * n_seg * sizeof(float4);
  auto kern_a = response == 2 ? k_grad_a<true> : k_grad_a<false>;
  e = cudaFuncSetAttribute(kern_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern_a, kGradWarps * 32, smem);
  if (e != cudaSuccess) return e;
  *parts_a = split(per_sm);
  return cudaSuccess;
}

cudaError_t launch_grad(const GridDesc& g, const MixConst& mc, int response, int pn_order,
                        int pitch, const TrancheF* tabF, const float4* P, const uint8_t* mask,
                        const double* theta, const TplConst* tpl, const TplMix* tplm, int64_t n,
                        int n_seg, double scale, double* out_stat, double* out_grad,
                        unsigned* counter, const int32_t* perm, int parts, int parts_a,
                        double* part_buf, double* src_buf, float4* lam_buf, int n_sm,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (parts < 1 || parts > kGradMaxParts || parts_a < 1 || parts_a > kGradMaxParts ||
      ((parts > 1 || parts_a > 1) && !part_buf) || !src_buf || !lam_buf)
    return cudaErrorInvalidValue;
  k_grad_src<<<(unsigned)((n * 8 + 127) / 128), 128, 0, s>>>(theta, n, pn_order, src_buf);
  GradArgs a;
  a.g = g;
  a.mc = mc;
  a.response = response;
  a.pitch = pitch;
  a.tabF = tabF;
  a.P = P;
  a.mask = mask;
  a.theta = theta;
  a.tpl = tpl;
  a.tplm = tplm;
  a.pn_order = pn_order;
  a.n_tpl = n;
  a.n_seg = n_seg;
  a.seg_len = g.n_tranche / n_seg;
  a.scale = scale;
  a.twopidT = (float)(2.0 * kPi * g.dT);
  a.pidT2 = (float)(kPi * g.dT * g.dT);
  a.out_stat = out_stat;
  a.out_grad = out_grad;
  a.counter = counter;
  a.perm = perm;
  a.parts = parts;
  a.parts_a = parts_a;
  a.part_out = part_buf;
  a.dsrc = src_buf;
  a.lam = lam_buf;
  cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned), s);  // tickets of A and B
  if (e != cudaSuccess) return e;
  // pass A: Upsilon and (lambda, mu) per segment
  {
    const size_t smem = (size_t)kGradWarps * n_seg * sizeof(float4);
    auto kern = response == 2 ? k_grad_a<true> : k_grad_a<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGradWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t need = (n * parts_a + kGradWarps - 1) / kGradWarps;
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)n_sm * std::max(per_sm, 1)));
    kern<<<(unsigned)ctas, kGradWarps * 32, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // pass B: the gradient
  {
    auto kern = response == 2 ? k_grad<true> : k_grad<false>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGradWarps * 32, 0);
    if (e != cudaSuccess) return e;
    const int64_t need = (n * parts + kGradWarps - 1) / kGradWarps;
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)n_sm * std::max(per_sm, 1)));
    kern<<<(unsigned)ctas, kGradWarps * 32, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || (parts == 1 && parts_a == 1)) return e;
  const int64_t blocks = std::min<int64_t>((9 * n + 255) / 256, (int64_t)n_sm * 8);
  k_grad_reduce<<<(unsigned)blocks, 256, 0, s>>>(part_buf, parts_a, parts, n, out_stat, out_grad);
  return cudaGetLastError();
}

}  // namespace tfs
