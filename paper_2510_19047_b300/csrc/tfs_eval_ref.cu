// One-thread-per-template evaluation kernels (the paper's GPU mapping: "devoting one
// GPU thread to each set of source parameters", Sec. "Hardware acceleration and
// computational cost"), each updating Upsilon tranche by tranche without storing
// the waveform:
//
//   k_eval_fp64  - FP64 throughout, the Fresnel-kernel transform in the
//                  phase-cancelled form (see below), the absolute phase of each
//                  tranche from double-double chirp constants. The parity path.
//   k_eval_plain - the printed Eq. fresnel-ft evaluated bin by bin: Fresnel C, S of
//                  v_1, v_2 and the factor exp(i(phi - pi fdot zeta^2)), with FP32
//                  pixels and FP32 Fresnel/trig; the large trig arguments are reduced
//                  in FP64 first, the phase track is FP64.
//
// Phase-cancelled form. With C + iS = sgn(v) [(1+i)/2 - G(|v|) e^{i pi v^2/2}],
// G = g + i f (the paper's auxiliary functions), v_1 = sqrt(2 fdot) zeta and
// pi v_1^2/2 = pi fdot zeta^2, Eq. fresnel-ft becomes
//   h~_k = A/sqrt(2 fdot) e^{i phi} W_k,
//   W_k  = s_1 G(|v_1|) - s_2 G(|v_2|) e^{i Psi} + [s_1 != s_2] (1+i) e^{-i pi v_1^2/2},
//   Psi  = pi (v_2^2 - v_1^2)/2 = 2 pi (f_nm - f_k) dT + pi fdot dT^2,
// and e^{i Psi} = e^{i(2 pi a + pi fdot dT^2)} (a = f_nm/df - k_c) is the same for all
// bins of a tranche: the two ~1e5-rad arguments cancel exactly instead of numerically.
#include <math.h>

#include "tfs_dd.cuh"
#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_tdi.cuh"

namespace tfs {

namespace {

struct TrackD {
  double tp, d0, f, fdot, fsrc;
};

// Retarded time, frequency and its derivative at the start of tranche m (FP64).
__device__ __forceinline__ TrackD track_fp64(const TplConst& c, const TrancheD& tr, int resp) {
  TrackD r;
  double d1 = 0.0, d2 = 0.0;
  r.d0 = 0.0;
  if (resp) {
    r.d0 = c.dop_c * tr.ca + c.dop_s * tr.sa;
    d1 = kOmega * (c.dop_s * tr.ca - c.dop_c * tr.sa);
    d2 = -kOmega * kOmega * r.d0;
  }
  r.tp = tr.t + r.d0;
  const double u = 1.0 - r.tp / c.tc;
  const double y = pow(u, -0.125), y2 = y * y, y3 = y2 * y;
  r.fsrc = c.F0 * y3 * (1.0 + c.C2 * y2);
  const double fdsrc = c.F0 * y3 * y3 * y3 * y2 * (3.0 + 5.0 * c.C2 * y2) / (8.0 * c.tc);
  r.f = r.fsrc * (1.0 + d1);
  r.fdot = fdsrc * (1.0 + d1) * (1.0 + d1) + r.fsrc * d2;
  return r;
}

// Phase advanced, in cycles, from barycentre time ta to ta + dt (both before t_c), for
// the plain path's FP64 phase track:
// [P5 (ua^(5/8) - ub^(5/8)) + P3 (ua^(3/8) - ub^(3/8))] / 2 pi with ub = ua (1 + rho),
// rho = -dt / (t_c - ta), written with log1p/expm1 so that it keeps full relative
// precision for small steps.
__device__ __forceinline__ double phase_step_cycles(const TplConst& c, double ta, double dt) {
  const double ua = 1.0 - ta / c.tc;
  const double rho = -dt / (c.tc - ta);
  const double l = log1p(rho);
  const double q = pow(ua, 0.125), q2 = q * q, q3 = q2 * q, q5 = q3 * q2;
  const double s = c.P5 * q5 * (-expm1(0.625 * l)) + c.P3 * q3 * (-expm1(0.375 * l));
  return s * (0.5 / kPi);
}

__device__ __forceinline__ void kahan_add(double& acc, double& comp, double x) {
  const double y = x - comp;
  const double t = acc + y;
  comp = (t - acc) - y;
  acc = t;
}

// Segment levels of one template.
struct LevelState {
  int n;
  int seg_len[kMaxLevels];
  int anchor;
};

__device__ __forceinline__ LevelState levels_of(const EvalArgs& a, int64_t i) {
  LevelState L;
  if (a.nseg_pt) {
    L.n = 1;
    L.seg_len[0] = a.g.n_tranche / a.nseg_pt[i];
    L.anchor = L.seg_len[0];
  } else {
    L.n = a.lv.n;
    for (int l = 0; l < kMaxLevels; ++l) L.seg_len[l] = a.lv.seg_len[l];
    L.anchor = a.lv.anchor_len;
  }
  return L;
}

// Response factors of Eq. tdi2: T_alpha = F+ A+ - i Fx Ax in the long-wavelength limit
// (resp 1), or the TDI-1.5 transfer at the tranche's frequency f (resp 2), evaluated
// in the arithmetic type T.
template <class T, bool TDI>
__device__ __forceinline__ void response_factors(const TplConst& c, const TrancheD& tr, double f,
                                                 int resp, T Tr[2], T Ti[2]) {
  if (!resp) {
    Tr[0] = Tr[1] = T(1);
    Ti[0] = Ti[1] = T(0);
    return;
  }
  if (TDI) {
    T pp[6], px[6];
    for (int k = 0; k < 6; ++k) {
      pp[k] = T(c.pp[k]);
      px[k] = T(c.px[k]);
    }
    Cplx<T> TA, TE;
    tdi_transfer<T>(T(f), T(tr.ca), T(tr.sa), T(c.dop_c / kAuS), T(c.dop_s / kAuS), T(c.nz), pp,
                    px, TA, TE);
    Tr[0] = TA.re;
    Ti[0] = TA.im;
    Tr[1] = TE.re;
    Ti[1] = TE.im;
    return;
  }
  const double* DA = tr.DA;
  const double* DE = tr.DE;
  double fpA = 0, fxA = 0, fpE = 0, fxE = 0;
  for (int p = 0; p < 6; ++p) {
    fpA += DA[p] * c.pp[p];
    fxA += DA[p] * c.px[p];
    fpE += DE[p] * c.pp[p];
    fxE += DE[p] * c.px[p];
  }
  Tr[0] = T(fpA);
  Ti[0] = T(-fxA);
  Tr[1] = T(fpE);
  Ti[1] = T(-fxE);
}

// W_k of the phase-cancelled form at v_1 = (aa - jp) sig, v_2 = v_1 + e2 (FP64).
__device__ __forceinline__ void w_fp64(double aa, int jp, double sig, double e2, double cpsi,
                                       double spsi, double& wr, double& wi) {
  const double v1 = (aa - (double)jp) * sig;
  const double v2 = v1 + e2;
  double f1, g1, f2, g2;
  fresnel_fg<double>(fabs(v1), f1, g1);
  fresnel_fg<double>(fabs(v2), f2, g2);
  const double s1 = v1 < 0.0 ? -1.0 : 1.0, s2 = v2 < 0.0 ? -1.0 : 1.0;
  wr = s1 * g1 - s2 * (g2 * cpsi - f2 * spsi);
  wi = s1 * f1 - s2 * (g2 * spsi + f2 * cpsi);
  if (s1 != s2) {
    double sp, cp;
    sincospi(0.5 * v1 * v1, &sp, &cp);
    wr += cp + sp;  // (1+i) e^{-i pi v1^2/2}
    wi += cp - sp;
  }
}

}  // namespace

// -------------------------------------------------------------------------------------
// FP64 parity kernel
// -------------------------------------------------------------------------------------
// TDI: the TDI-1.5 response (code 2) as its own instantiation (the long-wavelength
// kernel carries none of its code).
template <bool TDI>
__global__ void __launch_bounds__(128) k_eval_fp64(EvalArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_tpl) return;
  const TplConst c = a.tpl[i];
  const LevelState L = levels_of(a, i);
  const GridDesc g = a.g;
  const int nch = g.n_chan;
  double zr[kMaxLevels], zi[kMaxLevels], nn[kMaxLevels], ups[kMaxLevels];
  int neff[kMaxLevels], cur[kMaxLevels];
  for (int l = 0; l < kMaxLevels; ++l) {
    zr[l] = zi[l] = nn[l] = ups[l] = 0.0;
    neff[l] = 0;
    cur[l] = -1;
  }
  int nact = 0, nnc = 0;
  const dd tcd = {c.tc, c.tc_lo}, P5d = {c.P5, c.P5_lo}, P3d = {c.P3, c.P3_lo};
  const dd ph0 = dd_mul_d(kInv2PiDD, c.phi0);
  for (int m = c.m_lo; m < c.m_hi; ++m) {
    for (int l = 0; l < L.n; ++l) {
      const int s = m / L.seg_len[l];
      if (s != cur[l]) {
        if (nn[l] > 0.0) {
          ups[l] += (zr[l] * zr[l] + zi[l] * zi[l]) / nn[l];
          ++neff[l];
        }
        zr[l] = zi[l] = nn[l] = 0.0;
        cur[l] = s;
      }
    }
    if (!a.mask[m]) continue;
    const TrancheD tr = a.tabD[m];
    const TrackD tk = track_fp64(c, tr, a.response);
    if (!(tk.tp < c.tc)) break;  // t' grows with t: every later tranche is past t_c
    if (!(tk.fdot > 0.0)) continue;
    const double x = tk.f * g.dT;  // f / df
    const double kcd = ceil(x);
    const int kc = (int)kcd;
    if (kc - kNFHalf < 1 || kc + kNFHalf > g.n_bins - 1) continue;
    // absolute phase Phi(t'_nm) / 2 pi in cycles, formed in double-double and reduced
    // to [0, 1): ~1e-16 cycles however far the track has advanced
    const double cyc = dd_frac(dd_add(chirp_cycles_dd(tcd, P5d, P3d, tr.t, tk.d0), ph0));
    ++nact;
    if (tk.fdot * g.dT > 10.0 * g.df) ++nnc;

    double Tr[2], Ti[2];
    response_factors<double, TDI>(c, tr, tk.f, a.response, Tr, Ti);
    const double aa = x - kcd;                    // in (-1, 0]
    const double sig = g.df * sqrt(2.0 / tk.fdot);  // v = sig * (f_nm - f_k)/df
    const double e2 = sqrt(2.0 * tk.fdot) * g.dT;   // v_2 - v_1
    double spsi, cpsi;
    sincospi(2.0 * aa + tk.fdot * g.dT * g.dT, &spsi, &cpsi);
    double zcr[2] = {0, 0}, zci[2] = {0, 0}, ncc[2] = {0, 0};
    for (int j = 0; j < kNF; ++j) {
      const int k = kc - kNFHalf + j;
      double wr, wi;
      w_fp64(aa, j - kNFHalf, sig, e2, cpsi, spsi, wr, wi);
      const double ww = wr * wr + wi * wi;
      for (int ch = 0; ch < nch; ++ch) {
        const int64_t px = ((int64_t)ch * g.n_tranche + m) * g.n_bins + k;
        const double2 u = a.u64[px];
        zcr[ch] += u.x * wr + u.y * wi;  // conj(u) W
        zci[ch] += u.x * wi - u.y * wr;
        ncc[ch] += a.w64[px] * ww;
      }
    }
    const double amp = pow(tk.fsrc / c.F0, 2.0 / 3.0);
    const double P = amp / sqrt(2.0 * tk.fdot);
    double sph, cph;
    sincospi(2.0 * cyc, &sph, &cph);
    double Zr = 0.0, Zi = 0.0, N = 0.0;
    for (int ch = 0; ch < nch; ++ch) {
      const double ar = Tr[ch] * zcr[ch] - Ti[ch] * zci[ch];
      const double ai = Tr[ch] * zci[ch] + Ti[ch] * zcr[ch];
      Zr += ar * cph - ai * sph;
      Zi += ar * sph + ai * cph;
      N += (Tr[ch] * Tr[ch] + Ti[ch] * Ti[ch]) * ncc[ch];
    }
    for (int l = 0; l < L.n; ++l) {
      zr[l] += P * Zr;
      zi[l] += P * Zi;
      nn[l] += P * P * N;
    }
  }
  for (int l = 0; l < L.n; ++l) {
    if (nn[l] > 0.0) {
      ups[l] += (zr[l] * zr[l] + zi[l] * zi[l]) / nn[l];
      ++neff[l];
    }
    a.out_stat[(int64_t)l * a.n_tpl + i] = ups[l] * a.out_scale;
    if (a.out_neff) a.out_neff[(int64_t)l * a.n_tpl + i] = neff[l];
  }
  if (a.out_diag) {
    a.out_diag[i] = nact;
    a.out_diag[a.n_tpl + i] = nnc;
  }
}

// -------------------------------------------------------------------------------------
// FP64 multi-harmonic kernel (Sec. "Outlook": {A, f, fdot, phi} per harmonic, then the
// Fresnel expressions per harmonic). Harmonic h of a tranche has frequency nu_h f_nm,
// derivative nu_h fdot_nm, phase nu_h Phi(t'_nm) and amplitude c_h A; its 21-bin
// window is the phase-cancelled W_k about ceil(nu_h f_nm / delta f). The tranche's
// template y_k = sum_h Y_h W^h_k (Y_h = T_alpha c_h A / sqrt(2 nu_h fdot) e^{i phi_h})
// gives Z = sum_h Y_h sum_k conj(u_k) W^h_k and
// N = sum_h |Y_h|^2 sum_k w_k |W^h_k|^2 + 2 Re sum_{a<b} conj(Y_a) Y_b sum_k w_k conj(W^a_k) W^b_k,
// the last sum over the bins two windows share. The phases are absolute: the anchor
// block's phase since t' = 0 plus the compensated phase advanced inside the block.
// -------------------------------------------------------------------------------------
namespace {

// One harmonic's window geometry and template factor Y in one tranche.
struct HarmD {
  bool on;
  int kc;
  double aa, sig, e2, cpsi, spsi;
  double Yr[2], Yi[2];
};

template <bool TDI>
__device__ __forceinline__ HarmD harm_fp64(const EvalArgs& a, const TplConst& c,
                                           const TrancheD& tr, const TrackD& tk, double amp,
                                           dd cyc_abs, const double Tlr[2], const double Tli[2],
                                           int h) {
  HarmD r;
  r.on = false;
  const GridDesc& g = a.g;
  const double nu = a.harm.nu[h];
  const double fh = nu * tk.f, fdh = nu * tk.fdot;
  const double x = fh * g.dT;
  const double kcd = ceil(x);
  r.kc = (int)kcd;
  if (r.kc - kNFHalf < 1 || r.kc + kNFHalf > g.n_bins - 1) return r;
  r.on = true;
  r.aa = x - kcd;
  r.sig = g.df * sqrt(2.0 / fdh);
  r.e2 = sqrt(2.0 * fdh) * g.dT;
  sincospi(2.0 * r.aa + fdh * g.dT * g.dT, &r.spsi, &r.cpsi);
  double Tr[2] = {Tlr[0], Tlr[1]}, Ti[2] = {Tli[0], Tli[1]};
  if (TDI) response_factors<double, true>(c, tr, fh, a.response, Tr, Ti);
  // nu Phi / 2 pi, reduced to [0, 1) in double-double
  const double cyc = dd_frac(dd_mul_d(cyc_abs, nu));
  double sph, cph;
  sincospi(2.0 * cyc, &sph, &cph);
  const double P = amp / sqrt(2.0 * fdh);
  const double er = P * (cph * a.harm.cr[h] - sph * a.harm.ci[h]);
  const double ei = P * (cph * a.harm.ci[h] + sph * a.harm.cr[h]);
  for (int ch = 0; ch < 2; ++ch) {
    r.Yr[ch] = Tr[ch] * er - Ti[ch] * ei;
    r.Yi[ch] = Tr[ch] * ei + Ti[ch] * er;
  }
  return r;
}

}  // namespace

template <bool TDI>
__global__ void __launch_bounds__(128) k_eval_fp64_harm(EvalArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_tpl) return;
  const TplConst c = a.tpl[i];
  const LevelState L = levels_of(a, i);
  const GridDesc g = a.g;
  const int nch = g.n_chan;
  const int H = a.harm.n;
  double zr[kMaxLevels], zi[kMaxLevels], nn[kMaxLevels], ups[kMaxLevels];
  int neff[kMaxLevels], cur[kMaxLevels];
  for (int l = 0; l < kMaxLevels; ++l) {
    zr[l] = zi[l] = nn[l] = ups[l] = 0.0;
    neff[l] = 0;
    cur[l] = -1;
  }
  int nact = 0, nnc = 0;
  const dd tcd = {c.tc, c.tc_lo}, P5d = {c.P5, c.P5_lo}, P3d = {c.P3, c.P3_lo};
  const dd ph0 = dd_mul_d(kInv2PiDD, c.phi0);
  HarmD hd[TFS_MAX_HARMONICS];
  for (int m = c.m_lo; m < c.m_hi; ++m) {
    for (int l = 0; l < L.n; ++l) {
      const int s = m / L.seg_len[l];
      if (s != cur[l]) {
        if (nn[l] > 0.0) {
          ups[l] += (zr[l] * zr[l] + zi[l] * zi[l]) / nn[l];
          ++neff[l];
        }
        zr[l] = zi[l] = nn[l] = 0.0;
        cur[l] = s;
      }
    }
    if (!a.mask[m]) continue;
    const TrancheD tr = a.tabD[m];
    const TrackD tk = track_fp64(c, tr, a.response);
    if (!(tk.tp < c.tc)) break;
    if (!(tk.fdot > 0.0)) continue;
    // absolute phase Phi(t'_nm) / 2 pi in cycles (double-double, not reduced)
    const dd cyc = dd_add(chirp_cycles_dd(tcd, P5d, P3d, tr.t, tk.d0), ph0);

    double Tlr[2] = {1.0, 1.0}, Tli[2] = {0.0, 0.0};
    if (!TDI) response_factors<double, false>(c, tr, tk.f, a.response, Tlr, Tli);
    const double amp = pow(tk.fsrc / c.F0, 2.0 / 3.0);
    double Zr = 0.0, Zi = 0.0, N = 0.0;
    bool any = false;
    for (int h = 0; h < H; ++h) {
      hd[h] = harm_fp64<TDI>(a, c, tr, tk, amp, cyc, Tlr, Tli, h);
      const HarmD& q = hd[h];
      if (!q.on) continue;
      any = true;
      double zcr[2] = {0, 0}, zci[2] = {0, 0}, ncc[2] = {0, 0};
      for (int j = 0; j < kNF; ++j) {
        const int k = q.kc - kNFHalf + j;
        double wr, wi;
        w_fp64(q.aa, j - kNFHalf, q.sig, q.e2, q.cpsi, q.spsi, wr, wi);
        const double ww = wr * wr + wi * wi;
        for (int ch = 0; ch < nch; ++ch) {
          const int64_t px = ((int64_t)ch * g.n_tranche + m) * g.n_bins + k;
          const double2 u = a.u64[px];
          zcr[ch] += u.x * wr + u.y * wi;  // conj(u) W
          zci[ch] += u.x * wi - u.y * wr;
          ncc[ch] += a.w64[px] * ww;
        }
      }
      for (int ch = 0; ch < nch; ++ch) {
        Zr += q.Yr[ch] * zcr[ch] - q.Yi[ch] * zci[ch];
        Zi += q.Yr[ch] * zci[ch] + q.Yi[ch] * zcr[ch];
        N += (q.Yr[ch] * q.Yr[ch] + q.Yi[ch] * q.Yi[ch]) * ncc[ch];
      }
    }
    if (!any) continue;
    // cross terms of windows that share bins
    for (int ha = 0; ha < H; ++ha) {
      if (!hd[ha].on) continue;
      for (int hb = ha + 1; hb < H; ++hb) {
        if (!hd[hb].on) continue;
        const HarmD &A = hd[ha], &B = hd[hb];
        const int k0 = max(A.kc, B.kc) - kNFHalf, k1 = min(A.kc, B.kc) + kNFHalf;
        for (int k = k0; k <= k1; ++k) {
          double war, wai, wbr, wbi;
          w_fp64(A.aa, k - A.kc, A.sig, A.e2, A.cpsi, A.spsi, war, wai);
          w_fp64(B.aa, k - B.kc, B.sig, B.e2, B.cpsi, B.spsi, wbr, wbi);
          // conj(W^a) W^b
          const double xr = war * wbr + wai * wbi, xi = war * wbi - wai * wbr;
          for (int ch = 0; ch < nch; ++ch) {
            const int64_t px = ((int64_t)ch * g.n_tranche + m) * g.n_bins + k;
            // Re(conj(Y_a) Y_b (xr + i xi))
            const double yr = A.Yr[ch] * B.Yr[ch] + A.Yi[ch] * B.Yi[ch];
            const double yi = A.Yr[ch] * B.Yi[ch] - A.Yi[ch] * B.Yr[ch];
            N += 2.0 * a.w64[px] * (yr * xr - yi * xi);
          }
        }
      }
    }
    ++nact;
    if (tk.fdot * g.dT > 10.0 * g.df) ++nnc;
    for (int l = 0; l < L.n; ++l) {
      zr[l] += Zr;
      zi[l] += Zi;
      nn[l] += N;
    }
  }
  for (int l = 0; l < L.n; ++l) {
    if (nn[l] > 0.0) {
      ups[l] += (zr[l] * zr[l] + zi[l] * zi[l]) / nn[l];
      ++neff[l];
    }
    a.out_stat[(int64_t)l * a.n_tpl + i] = ups[l] * a.out_scale;
    if (a.out_neff) a.out_neff[(int64_t)l * a.n_tpl + i] = neff[l];
  }
  if (a.out_diag) {
    a.out_diag[i] = nact;
    a.out_diag[a.n_tpl + i] = nnc;
  }
}

// -------------------------------------------------------------------------------------
// Plain FP32 kernel: Eq. fresnel-ft as printed, bin by bin.
// -------------------------------------------------------------------------------------

// x - 2 round(x/2) in FP64, returned as FP32 in [-1, 1]: sin(pi x), cos(pi x) of the
// result equal those of x.
__device__ __forceinline__ float reduce_mod2(double x) { return (float)(x - 2.0 * rint(0.5 * x)); }

// Paper's Fresnel C(v), S(v) with the trig argument pi v^2/2 reduced in FP64.
__device__ __forceinline__ void fresnel_cs_plain(double v, float& C, float& S) {
  const float a = fabsf((float)v);
  float f, gg;
  fresnel_fg<float>(a, f, gg);
  float sn, cs;
  sincospif(reduce_mod2(0.5 * v * v), &sn, &cs);
  C = 0.5f + f * sn - gg * cs;
  S = 0.5f - f * cs - gg * sn;
  if (v < 0.0) {
    C = -C;
    S = -S;
  }
}

template <bool TDI>
__global__ void __launch_bounds__(128) k_eval_plain(EvalArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_tpl) return;
  const TplConst c = a.tpl[i];
  const LevelState L = levels_of(a, i);
  const GridDesc g = a.g;
  const int nch = g.n_chan;
  float zr[kMaxLevels], zi[kMaxLevels], nn[kMaxLevels];
  double ups[kMaxLevels];
  int neff[kMaxLevels], cur[kMaxLevels];
  for (int l = 0; l < kMaxLevels; ++l) {
    zr[l] = zi[l] = nn[l] = 0.0f;
    ups[l] = 0.0;
    neff[l] = 0;
    cur[l] = -1;
  }
  int nact = 0, nnc = 0;
  int blk = -1, m_prev = 0;
  double acc = 0.0, comp = 0.0, tp_prev = 0.0, d0_prev = 0.0;
  for (int m = c.m_lo; m < c.m_hi; ++m) {
    for (int l = 0; l < L.n; ++l) {
      const int s = m / L.seg_len[l];
      if (s != cur[l]) {
        if (nn[l] > 0.0f) {
          ups[l] += ((double)zr[l] * zr[l] + (double)zi[l] * zi[l]) / (double)nn[l];
          ++neff[l];
        }
        zr[l] = zi[l] = nn[l] = 0.0f;
        cur[l] = s;
      }
    }
    if (!a.mask[m]) continue;
    const TrancheD tr = a.tabD[m];
    const TrackD tk = track_fp64(c, tr, a.response);
    if (!(tk.tp < c.tc)) break;
    if (!(tk.fdot > 0.0)) continue;
    const int kc = (int)ceil(tk.f * g.dT);
    if (kc - kNFHalf < 1 || kc + kNFHalf > g.n_bins - 1) continue;
    const int b = m / L.anchor;
    if (b != blk) {
      blk = b;
      m_prev = b * L.anchor;
      const TrancheD ta = a.tabD[m_prev];
      d0_prev = a.response ? c.dop_c * ta.ca + c.dop_s * ta.sa : 0.0;
      tp_prev = ta.t + d0_prev;
      acc = comp = 0.0;
    }
    const double dt_ab = (double)(m - m_prev) * g.dT + (tk.d0 - d0_prev);
    kahan_add(acc, comp, phase_step_cycles(c, tp_prev, dt_ab));
    tp_prev = tk.tp;
    d0_prev = tk.d0;
    m_prev = m;
    const double cyc = (acc - floor(acc)) - comp;
    ++nact;
    if (tk.fdot * g.dT > 10.0 * g.df) ++nnc;

    float Tr[2], Ti[2];
    response_factors<float, TDI>(c, tr, tk.f, a.response, Tr, Ti);
    const double s2d = sqrt(2.0 * tk.fdot);
    const double inv_fdot = 1.0 / tk.fdot;
    const float P = (float)(pow(tk.fsrc / c.F0, 2.0 / 3.0) / s2d);
    float zcr[2] = {0, 0}, zci[2] = {0, 0}, ncc[2] = {0, 0};
    for (int j = 0; j < kNF; ++j) {
      const int k = kc - kNFHalf + j;
      const double zeta = (tk.f - (double)k * g.df) * inv_fdot;
      const double v1 = s2d * zeta, v2 = s2d * (g.dT + zeta);
      float C1, S1, C2, S2;
      fresnel_cs_plain(v1, C1, S1);
      fresnel_cs_plain(v2, C2, S2);
      // exp(i (phi - pi fdot zeta^2)), argument in cycles reduced in FP64
      float sn, cs;
      sincospif(reduce_mod2(2.0 * cyc - tk.fdot * zeta * zeta), &sn, &cs);
      const float Fr = C2 - C1, Fi = S2 - S1;
      const float hr = P * (cs * Fr - sn * Fi);
      const float hi = P * (cs * Fi + sn * Fr);
      const float hh = hr * hr + hi * hi;
      for (int ch = 0; ch < nch; ++ch) {
        const int64_t px = ((int64_t)ch * g.n_tranche + m) * g.n_bins + k;
        const float2 u = a.u32[px];
        zcr[ch] += u.x * hr + u.y * hi;
        zci[ch] += u.x * hi - u.y * hr;
        ncc[ch] += a.w32[px] * hh;
      }
    }
    for (int ch = 0; ch < nch; ++ch) {
      const float ar = Tr[ch] * zcr[ch] - Ti[ch] * zci[ch];
      const float ai = Tr[ch] * zci[ch] + Ti[ch] * zcr[ch];
      const float n = (Tr[ch] * Tr[ch] + Ti[ch] * Ti[ch]) * ncc[ch];
      for (int l = 0; l < L.n; ++l) {
        zr[l] += ar;
        zi[l] += ai;
        nn[l] += n;
      }
    }
  }
  for (int l = 0; l < L.n; ++l) {
    if (nn[l] > 0.0f) {
      ups[l] += ((double)zr[l] * zr[l] + (double)zi[l] * zi[l]) / (double)nn[l];
      ++neff[l];
    }
    a.out_stat[(int64_t)l * a.n_tpl + i] = ups[l] * a.out_scale;
    if (a.out_neff) a.out_neff[(int64_t)l * a.n_tpl + i] = neff[l];
  }
  if (a.out_diag) {
    a.out_diag[i] = nact;
    a.out_diag[a.n_tpl + i] = nnc;
  }
}

cudaError_t launch_eval_fp64(const EvalArgs& a, cudaStream_t s) {
  if (a.n_tpl <= 0) return cudaSuccess;
  if (a.harm.n > 0) {
    if (a.response == 2)
      k_eval_fp64_harm<true><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
    else
      k_eval_fp64_harm<false><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (a.response == 2)
    k_eval_fp64<true><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
  else
    k_eval_fp64<false><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------------------
// Plain multi-harmonic kernel: the paper's mapping and printed Eq. fresnel-ft, with
// harmonic h of the tranche at frequency nu_h f_nm, derivative nu_h fdot_nm, phase
// nu_h Phi(t'_nm) (absolute, as in k_eval_fp64_harm) and amplitude c_h A. Every bin of
// the union of the harmonics' windows is visited once: its template value is the sum
// of the harmonics whose window holds it, so the norm keeps the cross terms.
// -------------------------------------------------------------------------------------
namespace {

// One harmonic's Eq. fresnel-ft geometry in one tranche (FP64 frequency, FP32 factors).
struct HarmP {
  bool on;
  int kc;
  double f, fdot, s2d, inv_fdot;
  double cyc;        // phase / 2 pi, reduced to [0, 1)
  float Yr[2], Yi[2];  // T_alpha c_h A / sqrt(2 fdot) per channel
};

template <bool TDI>
__device__ __forceinline__ HarmP harm_plain(const EvalArgs& a, const TplConst& c,
                                            const TrancheD& tr, const TrackD& tk, double amp,
                                            double ph_int, double ph_frac, const float Tlr[2],
                                            const float Tli[2], int h) {
  HarmP r;
  r.on = false;
  const GridDesc& g = a.g;
  const double nu = a.harm.nu[h];
  r.f = nu * tk.f;
  r.fdot = nu * tk.fdot;
  r.kc = (int)ceil(r.f * g.dT);
  if (r.kc - kNFHalf < 1 || r.kc + kNFHalf > g.n_bins - 1) return r;
  r.on = true;
  r.s2d = sqrt(2.0 * r.fdot);
  r.inv_fdot = 1.0 / r.fdot;
  const double p = nu * ph_int;
  r.cyc = (p - floor(p)) + fma(nu, ph_int, -p) + nu * ph_frac;
  r.cyc -= floor(r.cyc);
  float Tr[2] = {Tlr[0], Tlr[1]}, Ti[2] = {Tli[0], Tli[1]};
  if (TDI) response_factors<float, true>(c, tr, r.f, a.response, Tr, Ti);
  const float P = (float)(amp / r.s2d);
  const float cr = (float)a.harm.cr[h] * P, ci = (float)a.harm.ci[h] * P;
  for (int ch = 0; ch < 2; ++ch) {
    r.Yr[ch] = Tr[ch] * cr - Ti[ch] * ci;
    r.Yi[ch] = Tr[ch] * ci + Ti[ch] * cr;
  }
  return r;
}

// The printed transform of one harmonic at bin k: (C2 - C1 + i (S2 - S1)) times
// exp(i (phi - pi fdot zeta^2)), without the amplitude.
__device__ __forceinline__ void plain_bin(const HarmP& q, double df, double dT, int k, float& hr,
                                          float& hi) {
  const double zeta = (q.f - (double)k * df) * q.inv_fdot;
  const double v1 = q.s2d * zeta, v2 = q.s2d * (dT + zeta);
  float C1, S1, C2, S2;
  fresnel_cs_plain(v1, C1, S1);
  fresnel_cs_plain(v2, C2, S2);
  float sn, cs;
  sincospif(reduce_mod2(2.0 * q.cyc - q.fdot * zeta * zeta), &sn, &cs);
  const float Fr = C2 - C1, Fi = S2 - S1;
  hr = cs * Fr - sn * Fi;
  hi = cs * Fi + sn * Fr;
}

}  // namespace

template <bool TDI>
__global__ void __launch_bounds__(128) k_eval_plain_harm(EvalArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_tpl) return;
  const TplConst c = a.tpl[i];
  const LevelState L = levels_of(a, i);
  const GridDesc g = a.g;
  const int nch = g.n_chan;
  const int H = a.harm.n;
  float zr[kMaxLevels], zi[kMaxLevels], nn[kMaxLevels];
  double ups[kMaxLevels];
  int neff[kMaxLevels], cur[kMaxLevels];
  for (int l = 0; l < kMaxLevels; ++l) {
    zr[l] = zi[l] = nn[l] = 0.0f;
    ups[l] = 0.0;
    neff[l] = 0;
    cur[l] = -1;
  }
  int nact = 0, nnc = 0;
  int blk = -1, m_prev = 0;
  double acc = 0.0, comp = 0.0, tp_prev = 0.0, d0_prev = 0.0, ph_a = 0.0;
  HarmP hp[TFS_MAX_HARMONICS];
  for (int m = c.m_lo; m < c.m_hi; ++m) {
    for (int l = 0; l < L.n; ++l) {
      const int s = m / L.seg_len[l];
      if (s != cur[l]) {
        if (nn[l] > 0.0f) {
          ups[l] += ((double)zr[l] * zr[l] + (double)zi[l] * zi[l]) / (double)nn[l];
          ++neff[l];
        }
        zr[l] = zi[l] = nn[l] = 0.0f;
        cur[l] = s;
      }
    }
    if (!a.mask[m]) continue;
    const TrancheD tr = a.tabD[m];
    const TrackD tk = track_fp64(c, tr, a.response);
    if (!(tk.tp < c.tc)) break;
    if (!(tk.fdot > 0.0)) continue;
    const int b = m / L.anchor;
    if (b != blk) {
      blk = b;
      m_prev = b * L.anchor;
      const TrancheD ta = a.tabD[m_prev];
      d0_prev = a.response ? c.dop_c * ta.ca + c.dop_s * ta.sa : 0.0;
      tp_prev = ta.t + d0_prev;
      acc = comp = 0.0;
      ph_a = c.phi0 * (0.5 / kPi) + phase_step_cycles(c, 0.0, tp_prev);
    }
    const double dt_ab = (double)(m - m_prev) * g.dT + (tk.d0 - d0_prev);
    kahan_add(acc, comp, phase_step_cycles(c, tp_prev, dt_ab));
    tp_prev = tk.tp;
    d0_prev = tk.d0;
    m_prev = m;
    const double ph_int = floor(ph_a) + floor(acc);
    const double ph_frac = (ph_a - floor(ph_a)) + ((acc - floor(acc)) - comp);
    float Tlr[2] = {1.0f, 1.0f}, Tli[2] = {0.0f, 0.0f};
    if (!TDI) response_factors<float, false>(c, tr, tk.f, a.response, Tlr, Tli);
    const double amp = pow(tk.fsrc / c.F0, 2.0 / 3.0);
    bool any = false;
    for (int h = 0; h < H; ++h) {
      hp[h] = harm_plain<TDI>(a, c, tr, tk, amp, ph_int, ph_frac, Tlr, Tli, h);
      any = any || hp[h].on;
    }
    if (!any) continue;
    ++nact;
    if (tk.fdot * g.dT > 10.0 * g.df) ++nnc;
    float Zr = 0.f, Zi = 0.f, N = 0.f;
    for (int h = 0; h < H; ++h) {
      if (!hp[h].on) continue;
      for (int j = 0; j < kNF; ++j) {
        const int k = hp[h].kc - kNFHalf + j;
        bool seen = false;  // bin k already visited through an earlier harmonic's window
        for (int e = 0; e < h; ++e) seen = seen || (hp[e].on && abs(k - hp[e].kc) <= kNFHalf);
        if (seen) continue;
        float yr[2] = {0.f, 0.f}, yi[2] = {0.f, 0.f};
        for (int e = h; e < H; ++e) {
          if (!hp[e].on || abs(k - hp[e].kc) > kNFHalf) continue;
          float hr, hi;
          plain_bin(hp[e], g.df, g.dT, k, hr, hi);
          for (int ch = 0; ch < nch; ++ch) {
            yr[ch] += hp[e].Yr[ch] * hr - hp[e].Yi[ch] * hi;
            yi[ch] += hp[e].Yr[ch] * hi + hp[e].Yi[ch] * hr;
          }
        }
        for (int ch = 0; ch < nch; ++ch) {
          const int64_t px = ((int64_t)ch * g.n_tranche + m) * g.n_bins + k;
          const float2 u = a.u32[px];
          Zr += u.x * yr[ch] + u.y * yi[ch];  // conj(u) y
          Zi += u.x * yi[ch] - u.y * yr[ch];
          N += a.w32[px] * (yr[ch] * yr[ch] + yi[ch] * yi[ch]);
        }
      }
    }
    for (int l = 0; l < L.n; ++l) {
      zr[l] += Zr;
      zi[l] += Zi;
      nn[l] += N;
    }
  }
  for (int l = 0; l < L.n; ++l) {
    if (nn[l] > 0.0f) {
      ups[l] += ((double)zr[l] * zr[l] + (double)zi[l] * zi[l]) / (double)nn[l];
      ++neff[l];
    }
    a.out_stat[(int64_t)l * a.n_tpl + i] = ups[l] * a.out_scale;
    if (a.out_neff) a.out_neff[(int64_t)l * a.n_tpl + i] = neff[l];
  }
  if (a.out_diag) {
    a.out_diag[i] = nact;
    a.out_diag[a.n_tpl + i] = nnc;
  }
}

cudaError_t ref_occupancy(const EvalArgs& a, int path, int* per_sm) {
  const bool tdi = a.response == 2, harm = a.harm.n > 0;
  const void* k;
  if (path == TFS_PATH_FP64)
    k = harm ? (tdi ? (const void*)k_eval_fp64_harm<true> : (const void*)k_eval_fp64_harm<false>)
             : (tdi ? (const void*)k_eval_fp64<true> : (const void*)k_eval_fp64<false>);
  else
    k = harm ? (tdi ? (const void*)k_eval_plain_harm<true> : (const void*)k_eval_plain_harm<false>)
             : (tdi ? (const void*)k_eval_plain<true> : (const void*)k_eval_plain<false>);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, 128, 0);
}

cudaError_t launch_eval_plain(const EvalArgs& a, cudaStream_t s) {
  if (a.n_tpl <= 0) return cudaSuccess;
  if (a.harm.n > 0) {
    if (a.response == 2)
      k_eval_plain_harm<true><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
    else
      k_eval_plain_harm<false><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (a.response == 2)
    k_eval_plain<true><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
  else
    k_eval_plain<false><<<(unsigned)((a.n_tpl + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tfs
