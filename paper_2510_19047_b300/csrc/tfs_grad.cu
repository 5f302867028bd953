// Gradient-ascent update of candidate templates (refinement of candidates by
// d Upsilon / d theta).
#include <math.h>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_source.cuh"

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
// template, one lane per tranche. Pass A forms Z_n, N_n in shared memory; pass B
// recomputes the track (it is never stored), the per-bin sums of the Fresnel-kernel
// derivatives with respect to v_1, v_2 and Psi, and turns them into the tranche's
// sensitivities to (f, fdot, phi, A, T_alpha). A reverse-mode step through the FP64
// closed-form track adds the tranche's share to the adjoints of the 20 template
// constants (t_c, F0, C2, P5, P3, phi0, the delay amplitudes, A+ e+, Ax ex); at the end
// they are contracted with the constants' derivatives with respect to theta (forward
// mode, one direction per parameter, once per template). The window position and the
// Fresnel branch are held fixed: the almost-everywhere derivative.
// ---------------------------------------------------------------------------------
namespace {

constexpr unsigned kFullG = 0xffffffffu;
constexpr int kGradWarps = 4;
constexpr int kSrcFields = 20;  // tc F0 C2 P5 P3 phi0 dop_c dop_s pp[6] px[6]

// The paper's auxiliary Fresnel functions and their derivatives at a = |v|.
__device__ __forceinline__ void fg_deriv(float a, float& f, float& g, float& fp, float& gp) {
  if (a > 6.0f) {
    f = 1.0f / ((float)kPi * a);
    g = 0.0f;
    fp = -f / a;
    gp = 0.0f;
  } else {
    const float N = fmaf(0.926f, a, 1.0f);
    const float D = fmaf(a, fmaf(3.104f, a, 1.792f), 2.0f);
    f = N / D;
    fp = (0.926f * D - N * fmaf(6.208f, a, 1.792f)) / (D * D);
    const float E = fmaf(a, fmaf(a, fmaf(6.670f, a, 3.492f), 4.142f), 2.0f);
    g = 1.0f / E;
    gp = -fmaf(a, fmaf(20.01f, a, 6.984f), 4.142f) * g * g;
  }
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
    sincospif(0.5f * v1 * v1, &sp, &cp);
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

struct GradArgs {
  GridDesc g;
  int response, pn_order;
  const TrancheD* tabD;
  const float2* u32;
  const float* w32;
  const uint8_t* mask;
  const double* theta;  // [8][n]
  const TplConst* tpl;  // set-up constants (ranges)
  int64_t n_tpl;
  int seg_len, n_seg;
  double scale;         // Upsilon = scale * sum |Z|^2 / N
  double* out_stat;
  double* out_grad;     // [8][n]
};

// x^(-1/8) to ~2^-21 relative (x > 0), the seed of the FP64 Newton steps below.
__device__ __forceinline__ float seed_m18(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.125f * l));
  return r;
}

// The track at the start of tranche m in FP64 without transcendental calls: the same
// chirp model as the set-up (f = F0 y^3 (1 + C2 y^2), Phi = phi0 + P5 (1 - u^(5/8)) +
// P3 (1 - u^(3/8)), y = u^(-1/8), u = 1 - t'/t_c, t' = t + n.r/c) with y from a float
// seed and two Newton steps, and the intermediates the adjoint needs.
struct Trk {
  bool ok;
  int kc;
  double f, fdot, phi, amp;  // phi absolute [rad]; amp = (f_src/F0)^(2/3)
  double Tr[2], Ti[2];
  double u, y, y2, onec, fsrc, fdsrc, d1, d2;
};

struct SrcAux {
  double tc_inv, inv8tc;
};

__device__ __forceinline__ Trk track64(const GradArgs& a, const SrcT<double>& s, const SrcAux& x,
                                       int m) {
  Trk k;
  k.ok = false;
  if (!a.mask[m]) return k;
  const TrancheD& tr = a.tabD[m];
  double d0 = 0.0, d1 = 0.0, d2 = 0.0;
  if (a.response) {
    d0 = s.dop_c * tr.ca + s.dop_s * tr.sa;
    d1 = kOmega * (s.dop_s * tr.ca - s.dop_c * tr.sa);
    d2 = -kOmega * kOmega * d0;
  }
  const double tp = tr.t + d0;
  const double u = fma(-tp, x.tc_inv, 1.0);
  if (!(u > 0.0)) return k;
  double y = (double)seed_m18((float)u);
#pragma unroll
  for (int it = 0; it < 2; ++it) {  // y <- y (1 + (1 - u y^8) / 8)
    const double y2 = y * y, y4 = y2 * y2;
    y = fma(y * 0.125, fma(-u, y4 * y4, 1.0), y);
  }
  const double y2 = y * y, y3 = y2 * y;
  const double onec = fma(s.C2, y2, 1.0);
  const double fsrc = s.F0 * y3 * onec;
  const double y5 = y3 * y2, y11 = y5 * y5 * y;
  const double fdsrc = s.F0 * y11 * fma(5.0 * s.C2, y2, 3.0) * x.inv8tc;
  const double f = fsrc * (1.0 + d1);
  const double fdot = fdsrc * (1.0 + d1) * (1.0 + d1) + fsrc * d2;
  if (!(fdot > 0.0)) return k;
  const int kc = (int)ceil(f * a.g.dT);
  if (kc - kNFHalf < 1 || kc + kNFHalf > a.g.n_bins - 1) return k;
  k.ok = true;
  k.kc = kc;
  k.f = f;
  k.fdot = fdot;
  const double u58 = u * y3;  // u^(5/8)
  k.phi = s.phi0 + s.P5 * (1.0 - u58) + s.P3 * (1.0 - u58 * y2);
  const float cb = cbrtf((float)onec);
  k.amp = y2 * (double)(cb * cb);
  k.u = u;
  k.y = y;
  k.y2 = y2;
  k.onec = onec;
  k.fsrc = fsrc;
  k.fdsrc = fdsrc;
  k.d1 = d1;
  k.d2 = d2;
  if (a.response) {
    double fpA = 0, fxA = 0, fpE = 0, fxE = 0;
    for (int q = 0; q < 6; ++q) {
      fpA = fma(s.pp[q], tr.DA[q], fpA);
      fxA = fma(s.px[q], tr.DA[q], fxA);
      fpE = fma(s.pp[q], tr.DE[q], fpE);
      fxE = fma(s.px[q], tr.DE[q], fxE);
    }
    k.Tr[0] = fpA;
    k.Ti[0] = -fxA;
    k.Tr[1] = fpE;
    k.Ti[1] = -fxE;
  } else {
    k.Tr[0] = k.Tr[1] = 1.0;
    k.Ti[0] = k.Ti[1] = 0.0;
  }
  return k;
}

// e^{i phi} with phi in FP64 reduced to cycles first; FP32 sine and cosine.
__device__ __forceinline__ void phase_factor(double phi, float& s, float& c) {
  double cyc = phi * (0.5 / kPi);
  cyc -= rint(cyc);
  __sincosf(6.283185307f * (float)cyc, &s, &c);
}

// Reverse-mode step of the track for one tranche: given the tranche's sensitivities
// of Upsilon to (f, fdot, phi, ln A, T_alpha), add its contribution to the adjoints G
// of the template constants (tc F0 C2 P5 P3 phi0 dop_c dop_s pp[6] px[6]).
__device__ __forceinline__ void track_adjoint(const GradArgs& a, const SrcT<double>& s,
                                              const SrcAux& x, const Trk& k, int m, double cf,
                                              double cfd, double cphi, double cP,
                                              const double cTr[2], const double cTi[2],
                                              double G[kSrcFields]) {
  const double op1 = 1.0 + k.d1;
  const double g_fsrc = cf * op1 + cfd * k.d2;
  const double g_fdsrc = cfd * op1 * op1;
  const double g_d1 = cf * k.fsrc + 2.0 * cfd * k.fdsrc * op1;
  const double g_d2 = cfd * k.fsrc;
  const double y = k.y, y2 = k.y2, y3 = y2 * y, y5 = y3 * y2;
  const double y10 = y5 * y5;
  // f_src = F0 y^3 onec, fdot_src = F0 y^11 (3 + 5 C2 y^2) / (8 t_c), ln A = 2 ln y + (2/3) ln onec
  const double dfs_dy = s.F0 * y2 * fma(5.0 * s.C2, y2, 3.0);
  const double dfd_dy = s.F0 * y10 * fma(65.0 * s.C2, y2, 33.0) * x.inv8tc;
  const double dlnA_dy = 2.0 / y + (4.0 / 3.0) * s.C2 * y / k.onec;
  const double g_y = g_fsrc * dfs_dy + g_fdsrc * dfd_dy + cP * dlnA_dy;
  G[2] += g_fsrc * s.F0 * y5 + g_fdsrc * s.F0 * y10 * y3 * 5.0 * x.inv8tc +
          cP * (2.0 / 3.0) * y2 / k.onec;
  if (s.F0 != 0.0) G[1] += (g_fsrc * k.fsrc + g_fdsrc * k.fdsrc) / s.F0;
  const double u58 = k.u * y3;
  G[3] += cphi * (1.0 - u58);
  G[4] += cphi * (1.0 - u58 * y2);
  G[5] += cphi;
  const double g_u = -g_y * y / (8.0 * k.u) - cphi * (0.625 * s.P5 * y3 + 0.375 * s.P3 * y5);
  G[0] += (g_u * (1.0 - k.u) - g_fdsrc * k.fdsrc) * x.tc_inv;  // du/dtc = (1 - u)/tc
  if (a.response) {
    const TrancheD& tr = a.tabD[m];
    const double g_tp = -g_u * x.tc_inv;
    const double w2 = kOmega * kOmega;
    G[6] += g_tp * tr.ca - g_d1 * kOmega * tr.sa - g_d2 * w2 * tr.ca;
    G[7] += g_tp * tr.sa + g_d1 * kOmega * tr.ca - g_d2 * w2 * tr.sa;
    for (int q = 0; q < 6; ++q) {
      G[8 + q] += cTr[0] * tr.DA[q] + cTr[1] * tr.DE[q];
      G[14 + q] -= cTi[0] * tr.DA[q] + cTi[1] * tr.DE[q];
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(kGradWarps * 32) k_grad(GradArgs a) {
  extern __shared__ float4 s_seg[];
  __shared__ double s_dsrc[kGradWarps][8][kSrcFields];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kGradWarps + warp;
  if (i >= a.n_tpl) return;  // whole warp leaves together
  float4* seg = s_seg + (size_t)warp * a.n_seg;
  const GridDesc g = a.g;
  const int nch = g.n_chan;
  double th[8];
  for (int p = 0; p < 8; ++p) th[p] = a.theta[(int64_t)p * a.n_tpl + i];
  const TplConst tc = a.tpl[i];
  const SrcT<double> s = source_of<double>(th, a.pn_order);
  SrcAux xa;
  xa.tc_inv = 1.0 / s.tc;
  xa.inv8tc = 0.125 * xa.tc_inv;
  for (int q = lane; q < a.n_seg; q += 32) seg[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  // directional derivatives of the template constants: lane p < 8 takes direction p
  if (lane < 8) {
    D1 thd[8];
    for (int p = 0; p < 8; ++p) thd[p] = mk(th[p], p == lane ? 1.0 : 0.0);
    const SrcT<D1> sd = source_of<D1>(thd, a.pn_order);
    double* o = s_dsrc[warp][lane];
    o[0] = sd.tc.d;
    o[1] = sd.F0.d;
    o[2] = sd.C2.d;
    o[3] = sd.P5.d;
    o[4] = sd.P3.d;
    o[5] = sd.phi0.d;
    o[6] = sd.dop_c.d;
    o[7] = sd.dop_s.d;
    for (int q = 0; q < 6; ++q) {
      o[8 + q] = sd.pp[q].d;
      o[14 + q] = sd.px[q].d;
    }
  }
  __syncwarp();

  // ---- pass A: Z_n, N_n ----
  for (int m0 = tc.m_lo; m0 < tc.m_hi; m0 += 32) {
    const int m = m0 + lane;
    const bool inr = m < tc.m_hi;
    float Zr = 0.f, Zi = 0.f, Nn = 0.f;
    if (inr) {
      const Trk L = track64(a, s, xa, m);
      if (L.ok) {
        const double x = L.f * g.dT;
        const float aa = (float)(x - (double)L.kc);
        const float sig = (float)(g.df * sqrt(2.0 / L.fdot));
        const float e2 = (float)(sqrt(2.0 * L.fdot) * g.dT);
        float sps, cps;
        sincospif((float)(2.0 * (x - L.kc) + L.fdot * g.dT * g.dT), &sps, &cps);
        float zr[2] = {0, 0}, zi[2] = {0, 0}, nn[2] = {0, 0};
        for (int j = 0; j < kNF; ++j) {
          const int k = L.kc - kNFHalf + j;
          const float v1 = (aa - (float)(j - kNFHalf)) * sig;
          const BinW b = bin_w<false>(v1, v1 + e2, cps, sps);
          const float ww = b.wr * b.wr + b.wi * b.wi;
          for (int c = 0; c < nch; ++c) {
            const int64_t px = ((int64_t)c * g.n_tranche + m) * g.n_bins + k;
            const float2 u = a.u32[px];
            zr[c] += u.x * b.wr + u.y * b.wi;
            zi[c] += u.x * b.wi - u.y * b.wr;
            nn[c] += a.w32[px] * ww;
          }
        }
        const float P = (float)(L.amp / sqrt(2.0 * L.fdot));
        float sph, cph;
        phase_factor(L.phi, sph, cph);
        for (int c = 0; c < nch; ++c) {
          const float ar = (float)L.Tr[c] * zr[c] - (float)L.Ti[c] * zi[c];
          const float ai = (float)L.Tr[c] * zi[c] + (float)L.Ti[c] * zr[c];
          Zr += P * (ar * (float)cph - ai * (float)sph);
          Zi += P * (ar * (float)sph + ai * (float)cph);
          Nn += P * P * (float)(L.Tr[c] * L.Tr[c] + L.Ti[c] * L.Ti[c]) * nn[c];
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
  // adjoint weights per segment, replacing (Z, N) by (lambda, mu)
  double ups = 0.0;
  for (int q = lane; q < a.n_seg; q += 32) {
    const float4 v = seg[q];
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v.z > 0.f) {
      const double zz = (double)v.x * v.x + (double)v.y * v.y;
      ups += a.scale * zz / v.z;
      o.x = (float)(2.0 * a.scale * v.x / v.z);   // lambda = 2 s conj(Z)/N
      o.y = (float)(-2.0 * a.scale * v.y / v.z);
      o.z = (float)(-a.scale * zz / ((double)v.z * v.z));  // mu
    }
    seg[q] = o;
  }
  for (int o = 16; o > 0; o >>= 1) ups += __shfl_xor_sync(kFullG, ups, o);
  if (lane == 0) a.out_stat[i] = ups;
  __syncwarp();

  // ---- pass B: adjoints of the template constants ----
  double G[kSrcFields];
  for (int k = 0; k < kSrcFields; ++k) G[k] = 0.0;
  for (int m0 = tc.m_lo; m0 < tc.m_hi; m0 += 32) {
    const int m = m0 + lane;
    if (m >= tc.m_hi) continue;
    const Trk L = track64(a, s, xa, m);
    if (!L.ok) continue;
    const float4 lm = seg[m / a.seg_len];
    const double lr = lm.x, li = lm.y, mu = lm.z;
    const double x = L.f * g.dT;
    const float aa = (float)(x - (double)L.kc);
    const float sig = (float)(g.df * sqrt(2.0 / L.fdot));
    const float e2 = (float)(sqrt(2.0 * L.fdot) * g.dT);
    float sps, cps;
    sincospif((float)(2.0 * (x - L.kc) + L.fdot * g.dT * g.dT), &sps, &cps);
    // per channel: complex sums S0..S3, S1v, S2v and real sums R0..R3, R1v, R2v
    float S[2][6][2], R[2][6];
    for (int c = 0; c < 2; ++c)
      for (int q = 0; q < 6; ++q) {
        S[c][q][0] = S[c][q][1] = 0.f;
        R[c][q] = 0.f;
      }
    for (int j = 0; j < kNF; ++j) {
      const int k = L.kc - kNFHalf + j;
      const float v1 = (aa - (float)(j - kNFHalf)) * sig;
      const BinW b = bin_w<true>(v1, v1 + e2, cps, sps);
      const float X[6][2] = {{b.wr, b.wi}, {b.a1r, b.a1i}, {b.a2r, b.a2i}, {b.a3r, b.a3i},
                             {b.a1r * v1, b.a1i * v1}, {b.a2r * v1, b.a2i * v1}};
      const float r1 = 2.f * (b.wr * b.a1r + b.wi * b.a1i);
      const float r2 = 2.f * (b.wr * b.a2r + b.wi * b.a2i);
      const float r3 = 2.f * (b.wr * b.a3r + b.wi * b.a3i);
      const float Rx[6] = {b.wr * b.wr + b.wi * b.wi, r1, r2, r3, r1 * v1, r2 * v1};
      for (int c = 0; c < nch; ++c) {
        const int64_t px = ((int64_t)c * g.n_tranche + m) * g.n_bins + k;
        const float2 u = a.u32[px];
        const float w = a.w32[px];
        for (int q = 0; q < 6; ++q) {
          S[c][q][0] += u.x * X[q][0] + u.y * X[q][1];
          S[c][q][1] += u.x * X[q][1] - u.y * X[q][0];
          R[c][q] += w * Rx[q];
        }
      }
    }
    // sensitivities of this tranche's dUpsilon to (f, fdot, phi, A, T_alpha)
    const double P = L.amp / sqrt(2.0 * L.fdot);
    float sphf, cphf;
    phase_factor(L.phi, sphf, cphf);
    const double sph = sphf, cph = cphf;
    const double Er = P * cph, Ei = P * sph;  // E = P e^{i phi}
    const double rt = sqrt(2.0 / L.fdot), ifd2 = 0.5 / L.fdot;
    const double twopidT = 2.0 * kPi * g.dT, pidT2 = kPi * g.dT * g.dT;
    double Zmr = 0, Zmi = 0, Nm = 0, cf = 0, cfd = 0, cTr[2] = {0, 0}, cTi[2] = {0, 0};
    for (int c = 0; c < nch; ++c) {
      // Q = E S0; z = T Q
      const double Qr = Er * S[c][0][0] - Ei * S[c][0][1];
      const double Qi = Er * S[c][0][1] + Ei * S[c][0][0];
      const double zr = L.Tr[c] * Qr - L.Ti[c] * Qi, zi = L.Tr[c] * Qi + L.Ti[c] * Qr;
      Zmr += zr;
      Zmi += zi;
      const double T2 = L.Tr[c] * L.Tr[c] + L.Ti[c] * L.Ti[c];
      const double n = T2 * P * P * R[c][0];
      Nm += n;
      // dT terms: Re(lambda dT Q) + mu P^2 R0 d|T|^2
      cTr[c] = (lr * Qr - li * Qi) + mu * 2.0 * L.Tr[c] * P * P * R[c][0];
      cTi[c] = -(lr * Qi + li * Qr) + mu * 2.0 * L.Ti[c] * P * P * R[c][0];
      // dS0 = K1 df + K2 dfdot (complex), dR0 likewise (real)
      double K1r = (S[c][1][0] + S[c][2][0]) * rt + S[c][3][0] * twopidT;
      double K1i = (S[c][1][1] + S[c][2][1]) * rt + S[c][3][1] * twopidT;
      double K2r = (-S[c][4][0] - S[c][5][0] + e2 * S[c][2][0]) * ifd2 + S[c][3][0] * pidT2;
      double K2i = (-S[c][4][1] - S[c][5][1] + e2 * S[c][2][1]) * ifd2 + S[c][3][1] * pidT2;
      // T E K
      const double TEr = L.Tr[c] * Er - L.Ti[c] * Ei, TEi = L.Tr[c] * Ei + L.Ti[c] * Er;
      const double a1r = TEr * K1r - TEi * K1i, a1i = TEr * K1i + TEi * K1r;
      const double a2r = TEr * K2r - TEi * K2i, a2i = TEr * K2i + TEi * K2r;
      cf += lr * a1r - li * a1i;
      cfd += lr * a2r - li * a2i;
      const double RK1 = (R[c][1] + R[c][2]) * rt + R[c][3] * twopidT;
      const double RK2 = (-R[c][4] - R[c][5] + e2 * R[c][2]) * ifd2 + R[c][3] * pidT2;
      cf += mu * T2 * P * P * RK1;
      cfd += mu * T2 * P * P * RK2;
    }
    const double cphi = -(lr * Zmi + li * Zmr);       // Re(i lambda z)
    const double cP = (lr * Zmr - li * Zmi) + 2.0 * mu * Nm;  // coefficient of dP/P
    cfd += -cP * ifd2;
    track_adjoint(a, s, xa, L, m, cf, cfd, cphi, cP, cTr, cTi, G);
  }
  // d Upsilon / d theta_p = sum_k G_k d(constant_k)/d theta_p
  double grad[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < kSrcFields; ++k) {
    double v = G[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullG, v, o);
    for (int p = 0; p < 8; ++p) grad[p] = fma(v, s_dsrc[warp][p][k], grad[p]);
  }
  if (lane < 8) {
    double v = grad[0];
    for (int p = 1; p < 8; ++p)
      if (lane == p) v = grad[p];
    a.out_grad[(int64_t)lane * a.n_tpl + i] = v;
  }
}

cudaError_t launch_grad(const GridDesc& g, int response, int pn_order, const TrancheD* tabD,
                        const float2* u32, const float* w32, const uint8_t* mask,
                        const double* theta, const TplConst* tpl, int64_t n, int n_seg,
                        double scale, double* out_stat, double* out_grad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  GradArgs a;
  a.g = g;
  a.response = response;
  a.pn_order = pn_order;
  a.tabD = tabD;
  a.u32 = u32;
  a.w32 = w32;
  a.mask = mask;
  a.theta = theta;
  a.tpl = tpl;
  a.n_tpl = n;
  a.n_seg = n_seg;
  a.seg_len = g.n_tranche / n_seg;
  a.scale = scale;
  a.out_stat = out_stat;
  a.out_grad = out_grad;
  const size_t smem = (size_t)kGradWarps * n_seg * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_grad<<<(unsigned)((n + kGradWarps - 1) / kGradWarps), kGradWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tfs
