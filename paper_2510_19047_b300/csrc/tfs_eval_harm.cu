// Mixed-precision evaluation of Upsilon_{N_seg} for multi-harmonic templates (Sec.
// "Outlook": the quantities {A, f, fdot, phi} of each harmonic, then the Fresnel
// expressions per harmonic). Same mapping and arithmetic as tfs_eval_mixed.cu: one
// warp per template, one lane per tranche, persistent CTAs on the sorted queue,
// FP16/BF16/FP32 pixels with FP32 sums and a double-float phase track.
//
// Per tranche (lane) the track is computed once: x = f_nm / df (double-float), fdot,
// the amplitude, S = (P5 u^(5/8) + P3 u^(3/8)) / 2 pi (double-float cycles) and the
// long-wavelength response. Harmonic h then has x_h = nu_h x, fdot_h = nu_h fdot,
// window centre ceil(x_h), sigma_h = df sqrt(2 / fdot_h), Psi_h, and phase
// frac(nu_h K) - nu_h S cycles (K = (phi0 + P5 + P3) / 2 pi; frac(nu_h K) per template
// from the FP64 set-up), amplitude c_h A and, for TDI-1.5, the transfer at nu_h f_nm.
// Its window sums are the mixed kernel's: the general bins of every lane joined over
// the warp, the rest in the asymptotic form from two reciprocals.
//
// N_n holds the cross terms 2 Re(conj(T_a) T_b sum_k w_k conj(W''^a_k) W''^b_k) of the
// bins two windows share. Windows of nu_a, nu_b can share bins only where
// |nu_a - nu_b| f_nm / df < 21; lanes that may see such a pair evaluate the shared bins
// one by one with the general W'' (a rare path at the bank's frequencies for harmonics
// nu = j / 2).
#include <math.h>
#include <stddef.h>

#include <algorithm>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_mixed_bins.cuh"
#include "tfs_tdi.cuh"

namespace tfs {

namespace {

// The harmonic-independent part of a tranche's track.
struct TrackH {
  df x;        // f_nm / df
  df S;        // (P5 u^(5/8) + P3 u^(3/8)) / 2 pi
  float fdot;  // fdot_nm
  float amp;   // (f / F0)^(2/3)
  float f;     // f_nm (FP32, for the TDI transfer)
  float fpA, fxA, fpE, fxE;  // long-wavelength F+, Fx of A and E
};
constexpr int kTrkF = 11;  // floats of a TrackH

// A lane's TrackH in shared memory (field k at t[32 k]): held there across the
// harmonic loop instead of in registers.
__device__ __forceinline__ void put_track(float* t, const TrackH& k) {
  const float v[kTrkF] = {k.x.hi, k.x.lo, k.S.hi, k.S.lo, k.fdot, k.amp, k.f, k.fpA, k.fxA, k.fpE,
                          k.fxE};
#pragma unroll
  for (int i = 0; i < kTrkF; ++i) t[32 * i] = v[i];
}
__device__ __forceinline__ TrackH get_track(const float* t) {
  TrackH k;
  k.x = df{t[0], t[32]};
  k.S = df{t[64], t[96]};
  k.fdot = t[128];
  k.amp = t[160];
  k.f = t[192];
  k.fpA = t[224];
  k.fxA = t[256];
  k.fpE = t[288];
  k.fxE = t[320];
  return k;
}

// One harmonic's window geometry and template factors T_alpha (amplitude, phase, c_h
// and response included) in one tranche.
struct HarmM {
  bool act;
  int kc;
  float aa, eps, sig, cpsi, spsi;
  float a1;  // x - (k_c - 1)
  float Tr0, Ti0, Tr1, Ti1;
};

// x1 = x - (k_c + j) of window bin j; j = -1 comes from a1
__device__ __forceinline__ float bin_x1(const HarmM& q, float j) {
  return j == -1.0f ? q.a1 : q.aa - j;
}

// The bin below f_nm (x1 = x - (k_c - 1)) and Psi are formed from rb = x - rint(x), to
// full relative precision when f_nm is just above a bin, as in the single-mode kernel.
template <bool TDI>
__device__ __forceinline__ HarmM harm_of(const EvalArgs& a, const TrackH& tk, const TplMix* cptr,
                                         float2 Kh, int h, float sig_k, float dTf, int m) {
  HarmM q;
  q.act = false;
  const df nu = {a.harm.nu_hi[h], a.harm.nu_lo[h]};
  const df x = df_mul(tk.x, nu);
  const bool inband = x.hi > (float)kNFHalf && x.hi < (float)(a.g.n_bins - kNFHalf);
  float kcf = rint_small(inband ? x.hi : 0.0f);  // ceil(x) = rint(x) (+1 if below x)
  // rb = x - rint(x) in [-1/2, 1/2]; rb > 0 exactly when ceil(x) = rint(x) + 1
  const float rb = __fadd_rn(__fsub_rn(x.hi, kcf), x.lo);
  q.kc = int_small(rb > 0.f ? kcf + 1.0f : kcf);
  q.aa = rb > 0.f ? rb - 1.0f : rb;
  q.a1 = rb > 0.f ? rb : rb + 1.0f;
  if (!inband || q.kc - kNFHalf < 1 || q.kc + kNFHalf > a.g.n_bins - 1) return q;
  q.act = true;
  const float fdh = nu.hi * tk.fdot;
  q.sig = sig_k * rsqrt_approx(fdh);
  q.eps = fdh * dTf * dTf;
  const float psi = fmaf(2.0f, rb, q.eps);  // Psi / pi (mod 2), reduced to [-1, 1]
  __sincosf(3.141592654f * (psi - 2.0f * rint_small(0.5f * psi)), &q.spsi, &q.cpsi);
  // phase frac(nu K) - nu S in cycles, reduced in two steps as in the mixed kernel
  const df ph = df_sub(df{Kh.x, Kh.y}, df_mul(tk.S, nu));
  float cyc = __fadd_rn(__fsub_rn(ph.hi, rintf(ph.hi)), ph.lo);
  cyc = __fsub_rn(cyc, rint_small(cyc));
  float sph, cph;
  __sincosf(6.283185307f * cyc, &sph, &cph);
  // c_h A e^{i phi_h}
  const float cr = a.harm.crf[h], ci = a.harm.cif[h];
  const float er = tk.amp * (cph * cr - sph * ci), ei = tk.amp * (cph * ci + sph * cr);
  q.Tr0 = q.Tr1 = er;
  q.Ti0 = q.Ti1 = ei;
  if (a.response) {
    float fpA = tk.fpA, fxA = tk.fxA, fpE = tk.fpE, fxE = tk.fxE;
    if (TDI) {  // TDI-1.5 transfer at (t_nm, nu_h f_nm)
      const float4* pq = reinterpret_cast<const float4*>(cptr->pp);
      const float4 q0 = ldg_nc4(pq), q1 = ldg_nc4(pq + 1), q2 = ldg_nc4(pq + 2);
      const float4 nq = ldg_nc4(pq + 3);  // (nx, ny, nz, pad)
      const float pp[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
      const float px[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
      Cplx<float> TA, TE;
      tdi_transfer_geom<float>(nu.hi * tk.f, tdi_geom_load(a.tdiF + (int64_t)m * kTdiGeomF4), nq.x,
                               nq.y, nq.z, pp, px, TA, TE);
      fpA = TA.re;
      fxA = -TA.im;
      fpE = TE.re;
      fxE = -TE.im;
    }
    // (F+ - i Fx)(er + i ei)
    q.Tr0 = fmaf(fpA, er, fxA * ei);
    q.Ti0 = fmaf(fpA, ei, -fxA * er);
    q.Tr1 = fmaf(fpE, er, fxE * ei);
    q.Ti1 = fmaf(fpE, ei, -fxE * er);
  }
  return q;
}

// The cross terms 2 Re sum_alpha conj(T_a) T_b sum_k w_k conj(W''^a_k) W''^b_k of every
// pair of harmonics whose windows share bins, in one tranche (bin by bin, general W'').
template <int NCH, int PIX, bool TDI>
__device__ __noinline__ float cross_terms(const EvalArgs& a, const TrackH& tk, const TplMix* cptr,
                                          const float2* Kp, int m, float sig_k, float dTf) {
  using Ld = PixLoad<PIX>;
  const typename Ld::P* PX = (const typename Ld::P*)a.Umix;
  float N = 0.0f;
  for (int ha = 0; ha < a.harm.n; ++ha) {
    const HarmM A = harm_of<TDI>(a, tk, cptr, Kp[ha], ha, sig_k, dTf, m);
    if (!A.act) continue;
    for (int hb = ha + 1; hb < a.harm.n; ++hb) {
      const HarmM B = harm_of<TDI>(a, tk, cptr, Kp[hb], hb, sig_k, dTf, m);
      if (!B.act || abs(A.kc - B.kc) > 2 * kNFHalf) continue;
      // conj(T_a) T_b per channel
      const float y0r = A.Tr0 * B.Tr0 + A.Ti0 * B.Ti0, y0i = A.Tr0 * B.Ti0 - A.Ti0 * B.Tr0;
      const float y1r = A.Tr1 * B.Tr1 + A.Ti1 * B.Ti1, y1i = A.Tr1 * B.Ti1 - A.Ti1 * B.Tr1;
      const int k0 = max(A.kc, B.kc) - kNFHalf, k1 = min(A.kc, B.kc) + kNFHalf;
      for (int k = k0; k <= k1; ++k) {
        const float ja = (float)(k - A.kc), jb = (float)(k - B.kc);
        float war, wai, wbr, wbi;
        const float xa = bin_x1(A, ja), xb = bin_x1(B, jb);
        w_general(xa, xa + A.eps, A.sig, A.sig * (float)kPi, A.cpsi, A.spsi, true, war, wai);
        w_general(xb, xb + B.eps, B.sig, B.sig * (float)kPi, B.cpsi, B.spsi, true, wbr, wbi);
        const float xr = war * wbr + wai * wbi, xi = war * wbi - wai * wbr;  // conj(Wa) Wb
        float2 ur, ui, w;
        Ld::cvt(Ld::raw(PX + (int64_t)k * a.pitch + m), ur, ui, w);
        N += 2.0f * w.x * (y0r * xr - y0i * xi);
        if (NCH == 2) N += 2.0f * w.y * (y1r * xr - y1i * xi);
      }
    }
  }
  return N;
}

}  // namespace

#ifndef TFS_HARM_MINB
#define TFS_HARM_MINB 3
#endif
constexpr int kHarmDepth = 3;  // pixel-load lead of the unrolled window path, in bins

// PITCH: the pixel plane's m-pitch as a compile-time constant (immediate row offsets),
// or 0 for a runtime pitch.
template <int NCH, int PIX, int PITCH, bool TDI>
__global__ void __launch_bounds__(256, TFS_HARM_MINB) k_eval_harm(EvalArgs a) {
  extern __shared__ float4 s_acc[];
  using Ld = PixLoad<PIX>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // per warp: the fine-segment sums, then the lanes' TrackH (kTrkF x 32 floats)
  float4* acc = s_acc + (size_t)warp * (a.fine_cap + kTrkF * 32 / 4);
  float* tks = reinterpret_cast<float*>(acc + a.fine_cap) + lane;
  const GridDesc g = a.g;
  const typename Ld::P* __restrict__ PX = (const typename Ld::P*)a.Umix;
  const int pitch = PITCH ? PITCH : a.pitch;
  const int H = a.harm.n;
  // grid constants as FP32 launch parameters (as in the single-mode kernel)
  const df dTd = {a.mc.dT_hi, a.mc.dT_lo};
  const float dTf = a.mc.dTf;
  const float sig_k = a.mc.sig_k;  // sigma = df sqrt(2/fdot)
  const float ncomp = a.mc.ncomp;  // fdot > 10 df / dT: non-compact
  // windows of two harmonics can share bins only below x = 21 / dnu_min (+ margin);
  // equal nu (dnu_min tiny) always, a single harmonic never
  const float x_ov = H > 1 ? 21.5f / a.harm.dnu_min : 0.0f;

  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= a.n_work) break;
    const int idx = a.perm ? a.perm[t] : t;
    const TplMix* __restrict__ cptr = a.tplm + idx;
    const float2* __restrict__ Kp = a.harm_K + (int64_t)idx * H;
    const int m_lo = cptr->m_lo, m_hi = cptr->m_hi;

    int nl, fine_len;
    int seg_len[kMaxLevels];
    if (a.nseg_pt) {
      nl = 1;
      seg_len[0] = g.n_tranche / a.nseg_pt[idx];
      fine_len = seg_len[0];
    } else {
      nl = a.lv.n;
#pragma unroll
      for (int l = 0; l < kMaxLevels; ++l) seg_len[l] = a.lv.seg_len[l];
      fine_len = a.lv.fine_len;
    }
    const int n_fine = g.n_tranche / fine_len;
    // m / fine_len = umulhi(m, ceil(2^32 / fine_len)), exact while m * fine_len < 2^32
    // (n_tranche < 2^16, checked by the host)
    const unsigned fmagic = fine_len > 1 ? 0xFFFFFFFFu / (unsigned)fine_len + 1u : 0u;
    for (int q = lane; q < n_fine; q += 32) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int nact = 0, nnc = 0;
    __syncwarp();

    // the template's range walked over unmasked tranches only (a gap idles no lane);
    // lane l of a block takes the block's l-th unmasked tranche
    const int r_lo = a.rank[m_lo], r_hi = a.rank[m_hi];
    for (int i0 = r_lo; i0 < r_hi; i0 += 32) {
      const int il = i0 + lane;
      const bool inr = il < r_hi;
      const int m = inr ? a.live[il] : 0;
      bool act = inr;
      {
      TrackH tk;
      tk.x = df{0.f, 0.f};
      tk.S = df{0.f, 0.f};
      tk.fdot = 1.f;
      tk.amp = tk.f = 0.f;
      tk.fpA = tk.fxA = tk.fpE = tk.fxE = 0.f;
      if (act) {
        const float4* cq = reinterpret_cast<const float4*>(cptr);
        const float4 c0 = ldg_nc4(cq), c1 = ldg_nc4(cq + 1), c2 = ldg_nc4(cq + 2),
                     c3 = ldg_nc4(cq + 3);
        const df tc_inv = {c0.x, c0.y}, F0 = {c0.z, c0.w};
        const df P5 = {c1.x, c1.y}, P3 = {c1.z, c1.w};
        const float dopc = c2.z, dops = c2.w;
        const df C2 = {c3.x, c3.y};
        const float fd_k = c3.z, C2x5 = c3.w;
        const TrancheF tr = a.tabF[m];
        const df tt = {tr.t_hi, tr.t_lo};
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (a.response) {
          d0 = fmaf(dopc, tr.ca_hi, dops * tr.sa_hi);
          d1 = (float)kOmega * (dops * tr.ca_hi - dopc * tr.sa_hi);
          d2 = -(float)(kOmega * kOmega) * d0;
        }
        const df tp = quick_add_f(tt, d0);
        const df u = one_minus(df_mul_u(tp, tc_inv));  // 1 - t'/t_c
        if (!(u.hi > 0.f)) {
          act = false;
        } else {
          // y = u^(-1/8): FP32 seed, one Newton step with a double-float residual
          const float y0 = pow_m18(u.hi);
          const df y02 = two_prod(y0, y0);
          const df y08 = df_sqr_u(df_sqr_u(y02));
          const df p = df_mul_u(u, y08);
          const float r = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);
          const df y = quick_two_sum(y0, y0 * r * 0.125f);
          // products that only feed further df arithmetic stay unnormalised (~46 bits)
          const df y2 = df_sqr_u(y);
          const df y3 = df_mul_u(y2, y);
          const df c2y2d = df_mul_u(C2, y2);
          const float c2y2 = c2y2d.hi;
          const df fs = df_mul_u(df_mul_u(F0, y3), one_plus_u(c2y2d));
          const df f = quick_add_f(fs, fs.hi * d1);
          const float y2f = y2.hi, y3f = y3.hi;
          const float fds = fd_k * (y3f * y3f * y3f * y2f) * fmaf(C2x5, y2f, 3.0f);
          tk.fdot = fds * (1.0f + d1) * (1.0f + d1) + fs.hi * d2;
          tk.x = df_mul(f, dTd);
          tk.f = f.hi;
          if (!(tk.fdot > 0.f)) {
            act = false;
          } else {
            tk.S = df_mul(df_mul_u(u, y3), df_add(P5, df_mul_u(P3, y2)));
            tk.amp = y2f * fmaf(c2y2, fmaf(c2y2, fmaf(c2y2, 4.0f / 81.0f, -1.0f / 9.0f), 2.0f / 3.0f),
                                1.0f);
            if (a.response && !TDI) {
              const float4* pq = reinterpret_cast<const float4*>(cptr->pp);
              const float4 q0 = ldg_nc4(pq), q1 = ldg_nc4(pq + 1), q2 = ldg_nc4(pq + 2);
              const float pp[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
              const float px[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
              // (F+_A, F+_E) and (Fx_A, Fx_E) as packed pairs
              float2 fp = make_float2(0.f, 0.f), fx = make_float2(0.f, 0.f);
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                fp = __ffma2_rn(tr.D[q], make_float2(pp[q], pp[q]), fp);
                fx = __ffma2_rn(tr.D[q], make_float2(px[q], px[q]), fx);
              }
              tk.fpA = fp.x;
              tk.fpE = fp.y;
              tk.fxA = fx.x;
              tk.fxE = fx.y;
            }
          }
        }
      }
      put_track(tks, tk);
      }
      float Zr = 0.f, Zi = 0.f, Nn = 0.f;
      bool any = false;
      for (int h = 0; h < H; ++h) {
        HarmM q;
        q.act = false;
        if (act) q = harm_of<TDI>(a, get_track(tks), cptr, Kp[h], h, sig_k, dTf, m);
        // general-bin range of the harmonic, joined over the warp (as in the mixed kernel)
        int jlo = 100, jhi = -100;
        if (q.act) {
          const float r6 = 6.0f * rcp_approx(q.sig);
          jlo = (int)ceilf(q.aa - r6 - 0.01f);
          jhi = (int)floorf(q.aa + q.eps + r6 + 0.01f);
        }
        const int JLO = __reduce_min_sync(kFull, jlo), JHI = __reduce_max_sync(kFull, jhi);
        if (!q.act) continue;
        any = true;
        const typename Ld::P* Pp = PX + (int64_t)(q.kc - kNFHalf) * pitch + m;
        const float spi = q.sig * (float)kPi;
        const float ae = q.aa + q.eps;
        const float m2c = -2.0f * q.cpsi;
        const float2 xae = make_float2(q.aa, ae);
        BinAcc s;
        s.u1r = s.u1i = s.u2r = s.u2i = s.nn = make_float2(0.f, 0.f);
        // fully unrolled window, no per-bin branch: the general form on the 2G bins
        // jp = -G .. G-1 next to f_nm (first, so that their temporaries are dead before
        // the asymptotic bins run), the asymptotic form on the others; only jp >= 0 can
        // hold the sweep, and jp = -1 takes its offset from rb (a1)
        auto unrolled = [&](auto gtag) {
          constexpr int G = decltype(gtag)::value;
          constexpr int kAsym = kNF - 2 * G;
          // the k-th asymptotic bin: 0 .. kNFHalf-G-1, then kNFHalf+G .. kNF-1
          auto asym_bin = [](int k) { return k < kNFHalf - G ? k : k + 2 * G; };
          typename Ld::P ring[kHarmDepth];
#pragma unroll
          for (int r = 0; r < kHarmDepth; ++r) ring[r] = Ld::raw(Pp + (int64_t)asym_bin(r) * pitch);
#pragma unroll
          for (int hb = 0; hb < 2 * G; ++hb) {
            const int jp = hb - G;
            const typename Ld::P gp = Ld::raw(Pp + (int64_t)(kNFHalf + jp) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(gp, cur_r, cur_i, cur_w);
            constexpr float kZero = 0.0f;
            const float c = kZero + (float)jp;
            float wr, wi;
            w_general(jp == -1 ? q.a1 : q.aa - c, jp == -1 ? q.a1 + q.eps : ae - c, q.sig, spi,
                      q.cpsi, q.spsi, jp >= 0, wr, wi);
            acc_general(s, cur_r, cur_i, cur_w, wr, wi);
          }
#pragma unroll
          for (int k = 0; k < kAsym; ++k) {
            const typename Ld::P pj = ring[k % kHarmDepth];
            if (k + kHarmDepth < kAsym)
              ring[k % kHarmDepth] = Ld::raw(Pp + (int64_t)asym_bin(k + kHarmDepth) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(pj, cur_r, cur_i, cur_w);
            constexpr float kZero = 0.0f;
            const float c = kZero + (float)(asym_bin(k) - kNFHalf);
            acc_asym(s, cur_r, cur_i, cur_w, __fadd2_rn(xae, make_float2(-c, -c)), m2c);
          }
        };
        if (JLO >= -1 && JHI <= 0) {
          unrolled(GeneralBins<1>{});
        } else if (JLO >= -2 && JHI <= 1) {
          unrolled(GeneralBins<2>{});
        } else if (JLO >= -3 && JHI <= 2) {
          unrolled(GeneralBins<3>{});
        } else {
          typename Ld::P cur = Ld::raw(Pp);
          float jpf = -(float)kNFHalf;
          for (int j = 0; j < kNF; ++j, jpf += 1.0f) {
            typename Ld::P nxt;
            if (j + 1 < kNF) nxt = Ld::raw(Pp + (int64_t)(j + 1) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(cur, cur_r, cur_i, cur_w);
            const int jp = j - kNFHalf;
            const float2 xx = __fadd2_rn(xae, make_float2(-jpf, -jpf));
            const float x1 = xx.x, x2 = xx.y;
            if (jp >= JLO && jp <= JHI) {
              float wr, wi;
              const bool near = jp == -1;
              w_general(near ? q.a1 : x1, near ? q.a1 + q.eps : x2, q.sig, spi, q.cpsi, q.spsi,
                        true, wr, wi);
              acc_general(s, cur_r, cur_i, cur_w, wr, wi);
            } else {
              acc_asym(s, cur_r, cur_i, cur_w, xx, m2c);
            }
            if (j + 1 < kNF) cur = nxt;
          }
        }
        // sum conj(u) W'' = i conj(U1) - i e^{i Psi} conj(U2), both channels at once
        const float2 ncp = make_float2(-q.cpsi, -q.cpsi);
        const float2 zr = __ffma2_rn(make_float2(q.spsi, q.spsi), s.u2r, __ffma2_rn(ncp, s.u2i, s.u1i));
        const float2 zi = __ffma2_rn(ncp, s.u2r, __ffma2_rn(make_float2(-q.spsi, -q.spsi), s.u2i, s.u1r));
        Zr += q.Tr0 * zr.x - q.Ti0 * zi.x;
        Zi += q.Tr0 * zi.x + q.Ti0 * zr.x;
        Nn += (q.Tr0 * q.Tr0 + q.Ti0 * q.Ti0) * s.nn.x;
        if (NCH == 2) {
          Zr += q.Tr1 * zr.y - q.Ti1 * zi.y;
          Zi += q.Tr1 * zi.y + q.Ti1 * zr.y;
          Nn += (q.Tr1 * q.Tr1 + q.Ti1 * q.Ti1) * s.nn.y;
        }
      }
      // cross terms of windows that share bins (a rare path, out of line)
      if (any && tks[0] < x_ov) Nn += cross_terms<NCH, PIX, TDI>(a, get_track(tks), cptr, Kp, m, sig_k, dTf);
      if (any) {
        ++nact;
        if (tks[128] > ncomp) ++nnc;
      }
      // inclusive prefix sums across the warp; a lane whose next lane lies in another
      // finest segment (or past the block) adds its prefix to its own segment's slot and
      // subtracts it from the next segment's, so that each slot gains the sum of its
      // segment's lanes, in a fixed order
      const int key = inr ? (fine_len > 1 ? (int)__umulhi((unsigned)m, fmagic) : m) : 0x7fffffff;
      const int key_up = __shfl_down_sync(kFull, key, 1);
      const bool nin = lane < 31 && il + 1 < r_hi;
      const int keyn = nin ? key_up : 0x7fffffff;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float zr2 = __shfl_up_sync(kFull, Zr, o);
        const float zi2 = __shfl_up_sync(kFull, Zi, o);
        const float n2 = __shfl_up_sync(kFull, Nn, o);
        if (lane >= o) {
          Zr += zr2;
          Zi += zi2;
          Nn += n2;
        }
      }
      const bool seg_end = inr && keyn != key;
      if (seg_end) {
        float4 v = acc[key];
        v.x += Zr;
        v.y += Zi;
        v.z += Nn;
        acc[key] = v;
      }
      __syncwarp();
      if (seg_end && nin) {
        float4 v = acc[keyn];
        v.x -= Zr;
        v.y -= Zi;
        v.z -= Nn;
        acc[keyn] = v;
      }
    }
    __syncwarp();
    for (int l = 0; l < nl; ++l) {
      const int r = seg_len[l] / fine_len;
      const int ns = g.n_tranche / seg_len[l];
      float ups = 0.f;
      int ne = 0;
      for (int n = lane; n < ns; n += 32) {
        float zr = 0.f, zi = 0.f, nn = 0.f;
        for (int q = 0; q < r; ++q) {
          const float4 v = acc[n * r + q];
          zr += v.x;
          zi += v.y;
          nn += v.z;
        }
        if (nn > 0.f) {
          ups += __fdividef(fmaf(zr, zr, zi * zi), nn);
          ++ne;
        }
      }
      for (int o = 16; o > 0; o >>= 1) ups += __shfl_xor_sync(kFull, ups, o);
      ne = __reduce_add_sync(kFull, ne);
      if (lane == 0) {
        a.out_stat[(int64_t)l * a.n_tpl + idx] = (double)ups * a.out_scale;
        if (a.out_neff) a.out_neff[(int64_t)l * a.n_tpl + idx] = ne;
      }
    }
    nact = __reduce_add_sync(kFull, nact);
    nnc = __reduce_add_sync(kFull, nnc);
    if (lane == 0 && a.out_diag) {
      a.out_diag[idx] = nact;
      a.out_diag[a.n_tpl + idx] = nnc;
    }
    __syncwarp();
  }
}

namespace {

template <int NCH, int PIX, int PITCH>
cudaError_t launch_harm_one(const EvalArgs& a, int n_sm, cudaStream_t s, int* shape) {
  constexpr int kWarps = 8;
  const size_t smem = (size_t)kWarps * (a.fine_cap * sizeof(float4) + kTrkF * 32 * sizeof(float));
  auto kern = a.response == 2 ? k_eval_harm<NCH, PIX, PITCH, true> : k_eval_harm<NCH, PIX, PITCH, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  const int64_t need = (a.n_work + kWarps - 1) / kWarps;
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)n_sm * std::max(per_sm, 1)));
  kern<<<(unsigned)ctas, kWarps * 32, smem, s>>>(a);
  if (shape) {
    shape[0] = kWarps * 32;
    shape[1] = (int)ctas;
    shape[2] = per_sm;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eval_harm(const EvalArgs& a, int n_chan, int pix, int n_sm, cudaStream_t s,
                             int* shape) {
  if (a.n_work <= 0) return cudaSuccess;
  const bool fixed = a.pitch == kMixedPitch;
  if (n_chan == 1) {
    if (pix == TFS_PIX_F32)
      return fixed ? launch_harm_one<1, TFS_PIX_F32, kMixedPitch>(a, n_sm, s, shape)
                   : launch_harm_one<1, TFS_PIX_F32, 0>(a, n_sm, s, shape);
    if (pix == TFS_PIX_F16)
      return fixed ? launch_harm_one<1, TFS_PIX_F16, kMixedPitch>(a, n_sm, s, shape)
                   : launch_harm_one<1, TFS_PIX_F16, 0>(a, n_sm, s, shape);
    return fixed ? launch_harm_one<1, TFS_PIX_BF16, kMixedPitch>(a, n_sm, s, shape)
                 : launch_harm_one<1, TFS_PIX_BF16, 0>(a, n_sm, s, shape);
  }
  if (pix == TFS_PIX_F32)
    return fixed ? launch_harm_one<2, TFS_PIX_F32, kMixedPitch>(a, n_sm, s, shape)
                 : launch_harm_one<2, TFS_PIX_F32, 0>(a, n_sm, s, shape);
  if (pix == TFS_PIX_F16)
    return fixed ? launch_harm_one<2, TFS_PIX_F16, kMixedPitch>(a, n_sm, s, shape)
                 : launch_harm_one<2, TFS_PIX_F16, 0>(a, n_sm, s, shape);
  return fixed ? launch_harm_one<2, TFS_PIX_BF16, kMixedPitch>(a, n_sm, s, shape)
               : launch_harm_one<2, TFS_PIX_BF16, 0>(a, n_sm, s, shape);
}

}  // namespace tfs
