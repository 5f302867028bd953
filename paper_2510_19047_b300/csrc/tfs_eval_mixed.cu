// Mixed-precision evaluation of Upsilon_{N_seg} (Eq. Upsilon-seg): one warp per
// template, one lane per tranche, persistent CTAs that take templates from a
// length/frequency-sorted queue.
//
// Per tranche (lane):
//   * the track (Sec. "Time-frequency waveform representation": phi_nm, f_nm,
//     fdot_nm at the tranche start) in double-float arithmetic: retarded time
//     t' = t + n.r/c (the delay itself in FP32), u = 1 - t'/t_c, y = u^(-1/8) by one
//     Newton step, f, and the phase in cycles (accurate to ~1e-5 cycles over 1e7
//     cycles); fdot, amplitude and response in FP32;
//   * the Fresnel-kernel transform (Eq. fresnel-ft) in the phase-cancelled form
//     h~_k = A/sqrt(2 fdot) e^{i phi} W_k (see tfs_eval_ref.cu), scaled as
//     W''_k = sigma pi W_k with sigma = df sqrt(2/fdot) so that v = sigma x,
//     x = (f_nm - f_k)/df. Where |v_1|, |v_2| > 6 on the same side (the printed
//     asymptotic form) W''_k = i/x_1 - i e^{i Psi}/x_2: two reciprocals per bin. The
//     bins that need the rational form or the in-sweep term are found per lane and
//     joined over the warp, so every branch is warp-uniform;
//   * the tranche inner products (Eq. inner-tranche-tf) against FP16/BF16/FP32 pixels
//     u = d~/S, w = 1/S read from frequency-major planes (lanes read consecutive
//     tranches of one frequency row: coalesced), accumulated in FP32.
// Per warp: the template's range is walked over unmasked tranches only (32 per block,
// so that gaps idle no lane); tranche sums are folded into the template's finest common
// segments by warp prefix sums differenced at segment boundaries into shared memory (a
// fixed order: deterministic), and at the end into every requested N_seg (Eqs.
// overlap-n, Upsilon-seg).
#include <math.h>
#include <stddef.h>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_mixed_bins.cuh"
#include "tfs_tdi.cuh"

namespace tfs {

namespace {

static_assert(offsetof(TplMix, tcinv_hi) == 0 && offsetof(TplMix, P5_hi) == 16 &&
                  offsetof(TplMix, K_hi) == 32 && offsetof(TplMix, dopc) == 40 &&
                  offsetof(TplMix, C2_hi) == 48 && offsetof(TplMix, fd_k) == 56 &&
                  offsetof(TplMix, pp) == 64 && offsetof(TplMix, px) == 88 &&
                  offsetof(TplMix, nx) == 112,
              "TplMix layout assumed by the 16-byte loads of the mixed kernel");

}  // namespace

// Tile and schedule variants the launch autotuner chooses among (mixed_shape in
// tfs_api.cu): the bin unroll of the general-bin loop path, the pixel-load lead of the
// unrolled path (a ring of packed elements in registers, in bins), and the CTAs of 256
// threads per SM the register allocation targets (4: 64 registers, 3: 85).
template <int V>
struct MixedVariant;
template <>
struct MixedVariant<0> {
  static constexpr int unroll = 3, depth = 3, minb = 4;
};
template <>
struct MixedVariant<1> {
  static constexpr int unroll = 2, depth = 2, minb = 4;
};
template <>
struct MixedVariant<2> {
  static constexpr int unroll = 3, depth = 5, minb = 3;
};

// PITCH: the m-pitch of the pixel plane as a compile-time constant (kMixedPitch) so that
// the 21 window rows are immediate offsets from one address, or 0 for a runtime pitch.
// TDI: the TDI-1.5 response (response code 2) instead of the long-wavelength one, as
// its own instantiation so the long-wavelength kernel carries none of its code.
// V: the tile/schedule variant (MixedVariant).
template <int NCH, int PIX, int PITCH, bool TDI, int V>
__global__ void __launch_bounds__(256, MixedVariant<V>::minb) k_eval_mixed(EvalArgs a) {
  constexpr int kBinUnroll = MixedVariant<V>::unroll;
  constexpr int kDepth = MixedVariant<V>::depth;  // pixel-load lead of the unrolled path
  extern __shared__ float4 s_acc[];
  using Ld = PixLoad<PIX>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4* acc = s_acc + (size_t)warp * a.fine_cap;
  const GridDesc g = a.g;
  const typename Ld::P* __restrict__ PX = (const typename Ld::P*)a.Umix;
  const int pitch = PITCH ? PITCH : a.pitch;
  // grid constants as FP32 launch parameters: derived from the FP64 grid here, the
  // compiler re-derives them inside the tranche loop on the narrow FP64 pipe
  const df dTd = {a.mc.dT_hi, a.mc.dT_lo};
  const float dTf = a.mc.dTf, dTf2 = dTf * dTf;
  const float sig_k = a.mc.sig_k;  // sigma = df sqrt(2/fdot)
  const float ncomp = a.mc.ncomp;  // fdot > 10 df / dT: non-compact
  // The bin next to f_nm below it (x1 = f_nm/df - (k_c - 1)) and Psi are formed from
  // rb = f_nm/df - rint(f_nm/df), which keeps full relative precision when f_nm is just
  // above a bin. From aa = f_nm/df - k_c ~ -1 they would keep ~6e-8 bins absolute only,
  // against a sweep x2 - x1 = eps = 2/sigma^2 of ~5e-5 bins for slow chirps: a ~1e-3
  // relative error of W'' on that bin, invisible in one tranche's |Z|^2/N but adding up
  // over a long segment's coherent tranches.
  // precision-study pixel types: the template's values held at FP16 precision
  constexpr bool kR16 = PIX == TFS_PIX_F16_ALL || PIX == TFS_PIX_BF16_ALL;

  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= a.n_work) break;
    const int idx = a.perm ? a.perm[t] : t;
    const TplMix* __restrict__ cptr = a.tplm + idx;
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
      float Zr = 0.f, Zi = 0.f, Nn = 0.f;
      int kc = 0;
      float aa = 0.f, a1 = 0.f, eps = 0.f, sig = 1.f, spsi = 0.f, cpsi = 1.f;
      // T_alpha A e^{i phi}: response times amplitude and phase factor, per channel
      float Tr0 = 0.f, Ti0 = 0.f, Tr1 = 0.f, Ti1 = 0.f;
      if (act) {
        // the template's constants are re-read per tranche (L1 hits) instead of being
        // held in registers across the tranche loop
        const float4* cq = reinterpret_cast<const float4*>(cptr);
        const float4 c0 = ldg_nc4(cq), c1 = ldg_nc4(cq + 1), c2 = ldg_nc4(cq + 2),
                     c3 = ldg_nc4(cq + 3);
        const df tc_inv = {c0.x, c0.y}, F0 = {c0.z, c0.w};
        const df P5 = {c1.x, c1.y}, P3 = {c1.z, c1.w};  // phase coefficients in cycles
        const df Kc = {c2.x, c2.y};
        const float dopc = c2.z, dops = c2.w;
        const df C2 = {c3.x, c3.y};
        const float fd_k = c3.z, C2x5 = c3.w;  // fdot_src = fd_k y^11 (3 + 5 C2 y^2)
        const TrancheF tr = a.tabF[m];
        const df tt = {tr.t_hi, tr.t_lo};
        // barycentre delay n.r/c (|d0| <= 500 s) in FP32: its rounding, < 1e-4 s, moves
        // the phase by < 1e-5 cycles
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (a.response) {
          d0 = fmaf(dopc, tr.ca_hi, dops * tr.sa_hi);
          d1 = (float)kOmega * (dops * tr.ca_hi - dopc * tr.sa_hi);
          d2 = -(float)(kOmega * kOmega) * d0;
        }
        // |t| >= |d0| except at t = 0, where the quick sum is exact as well
        const df tp = quick_add_f_u(tt, d0);
        const df u = one_minus_u(df_mul_u(tp, tc_inv));  // 1 - t'/t_c
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
          // products that only feed further df arithmetic stay unnormalised (~46 bits);
          // their hi words enter FP32 terms (fdot, amplitude) only
          const df y2 = df_sqr_u(y);
          const df y3 = df_mul_u(y2, y);
          const df c2y2d = df_mul_u(C2, y2);
          const float c2y2 = c2y2d.hi;
          const df onec = one_plus_u(c2y2d);  // |C2 y^2| < 1
          const df fs = df_mul_u(df_mul_u(F0, y3), onec);  // source-frame frequency
          const df f = quick_add_f_u(fs, fs.hi * d1);   // detector frame: f (1 + dt'/dt - 1)
          const float y2f = y2.hi, y3f = y3.hi;
          const float fds = fd_k * (y3f * y3f * y3f * y2f) * fmaf(C2x5, y2f, 3.0f);
          const float fdot = fds * (1.0f + d1) * (1.0f + d1) + fs.hi * d2;
          const df x = df_mul(f, dTd);  // f_nm / df
          // the window test first on the float, so that x is small enough for the
          // FMA-pipe ceiling below (n_bins < 2^22)
          const bool inband = x.hi > (float)kNFHalf && x.hi < (float)(g.n_bins - kNFHalf);
          float kcf = rint_small(inband ? x.hi : 0.0f);  // ceil(x) = rint(x) (+1 if below x)
          // rb = x - rint(x) in [-1/2, 1/2]; rb > 0 exactly when ceil(x) = rint(x) + 1
          const float rb = __fadd_rn(__fsub_rn(x.hi, kcf), x.lo);
          kc = int_small(rb > 0.f ? kcf + 1.0f : kcf);
          aa = rb > 0.f ? rb - 1.0f : rb;  // f_nm/df - k_c, in (-1, 0]
          a1 = rb > 0.f ? rb : rb + 1.0f;  // f_nm/df - (k_c - 1)
          if (!inband || !(fdot > 0.f) || kc - kNFHalf < 1 || kc + kNFHalf > g.n_bins - 1) {
            act = false;
          } else {
            ++nact;
            if (fdot > ncomp) ++nnc;
            // phase in cycles: K - P5 u^(5/8) - P3 u^(3/8) = K - u y^3 (P5 + P3 y^2)
            // (u^(5/8) = u y^3, u^(3/8) = u y^5); the fractional part is taken in two
            // steps because the hi word can be an integer-valued float (|Phi| > 2^23)
            const df u58 = df_mul_u(u, y3);
            const df ph = df_sub_u(Kc, df_mul_u(u58, df_add_u(P5, df_mul_u(P3, y2))));
            float cyc = __fadd_rn(__fsub_rn(ph.hi, rintf(ph.hi)), ph.lo);
            cyc = __fsub_rn(cyc, rint_small(cyc));
            // cyc is in [-1/2, 1/2]: the hardware sine/cosine are accurate to ~4e-7 there
            float sph, cph;
            __sincosf(6.283185307f * cyc, &sph, &cph);
            // amplitude (f/F0)^(2/3) = y^2 (1 + C2 y^2)^(2/3), series to O(e^4)
            const float amp =
                y2f * fmaf(c2y2, fmaf(c2y2, fmaf(c2y2, 4.0f / 81.0f, -1.0f / 9.0f), 2.0f / 3.0f),
                           1.0f);
            const float amp_c = amp * cph, amp_s = amp * sph;
            Tr0 = Tr1 = amp_c;
            Ti0 = Ti1 = amp_s;
            sig = sig_k * rsqrt_approx(fdot);
            eps = fdot * dTf2;  // fdot dT / df: sweep width in bins
            // Psi / 2 pi = aa + eps / 2 = rb + eps / 2 (mod 1), reduced to [-1/2, 1/2]
            const float hpsi = fmaf(0.5f, eps, rb);
            __sincosf(6.283185307f * (hpsi - rint_small(hpsi)), &spsi, &cpsi);
            if (a.response) {
              // (F+_A, F+_E) and (Fx_A, Fx_E) as packed pairs
              float2 fp = make_float2(0.f, 0.f), fx = make_float2(0.f, 0.f);
              // the polarisation tensors are read here, per tranche, from L1 rather than
              // held in registers across the tranche loop
              const float4* pq = reinterpret_cast<const float4*>(a.tplm[idx].pp);
              const float4 q0 = ldg_nc4(pq), q1 = ldg_nc4(pq + 1), q2 = ldg_nc4(pq + 2);
              const float pp[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
              const float px[6] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
              if (TDI) {  // TDI-1.5 transfer at (t_nm, f_nm)
                const float4 nq = ldg_nc4(pq + 3);  // (nx, ny, nz, pad)
                Cplx<float> TA, TE;
                tdi_transfer_geom<float>(f.hi, tdi_geom_load(a.tdiF + (int64_t)m * kTdiGeomF4), nq.x,
                                         nq.y, nq.z, pp, px, TA, TE);
                fp = make_float2(TA.re, TE.re);
                fx = make_float2(-TA.im, -TE.im);
              } else {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                  fp = __ffma2_rn(tr.D[q], make_float2(pp[q], pp[q]), fp);
                  fx = __ffma2_rn(tr.D[q], make_float2(px[q], px[q]), fx);
                }
              }
              // (F+ - i Fx)(amp_c + i amp_s), both channels at once
              const float2 ac = make_float2(amp_c, amp_c), as = make_float2(amp_s, amp_s);
              const float2 Tr = __ffma2_rn(fp, ac, __fmul2_rn(fx, as));
              const float2 Ti = __ffma2_rn(fp, as, __fmul2_rn(fx, make_float2(-amp_c, -amp_c)));
              Tr0 = Tr.x;
              Tr1 = Tr.y;
              Ti0 = Ti.x;
              Ti1 = Ti.y;
            }
            if (kR16) {
              Tr0 = round_f16(Tr0);
              Ti0 = round_f16(Ti0);
              Tr1 = round_f16(Tr1);
              Ti1 = round_f16(Ti1);
            }
          }
        }
      }
      // Window-relative bins jp = j - 10 that need the general (rational or in-sweep)
      // form: |v| <= 6 for v1 or v2, or the sweep [x1, x2] contains 0. Joined over the
      // warp so that every branch below is warp-uniform.
      // jlo = ceil(aa - r6 - 0.01) and jhi = floor(aa + eps + r6 + 0.01), r6 = 6/sigma;
      // the common case jlo >= -1, jhi <= 0 is tested on the floats
      const float r6 = act ? 6.0f * rcp_approx(sig) : 0.0f;
      const bool central = !act || (aa - r6 - 0.01f > -2.0f && aa + eps + r6 + 0.01f < 1.0f);
      int JLO = -1, JHI = 0;
      if (!__all_sync(kFull, central)) {
        int jlo = 100, jhi = -100;
        if (act) {
          jlo = (int)ceilf(aa - r6 - 0.01f);
          jhi = (int)floorf(aa + eps + r6 + 0.01f);
        }
        JLO = __reduce_min_sync(kFull, jlo);
        JHI = __reduce_max_sync(kFull, jhi);
      }
      if (act) {
        const typename Ld::P* Pp = PX + (int64_t)(kc - kNFHalf) * pitch + m;
        const float spi = sig * (float)kPi;
        const float ae = aa + eps;
        const float m2c = -2.0f * cpsi;
        const float2 xae = make_float2(aa, ae);
        BinAcc s;
        s.u1r = s.u1i = s.u2r = s.u2i = s.nn = make_float2(0.f, 0.f);
        // pixel loads run one bin ahead of the arithmetic
        typename Ld::P cur = Ld::raw(Pp);
        // Fully unrolled window, no per-bin branch: the general form on the 2G bins
        // jp = -G .. G-1 next to f_nm, the asymptotic form on the others (for jp >= G,
        // x2 < -r6 < 0; for jp < -G, x1 > G > r6). Only jp >= 0 can hold the sweep
        // (x1 < 0 <= x2), and jp = -1 takes its offset from rb (a1). The general bins
        // come first, so that a1 and the general form's temporaries are dead before the
        // asymptotic bins run; pixel loads of those run kDepth bins ahead (a ring of
        // packed elements in registers, started before the general bins so that their
        // latency is covered).
        auto unrolled = [&](auto gtag) {
          constexpr int G = decltype(gtag)::value;
          constexpr int kAsym = kNF - 2 * G;
          // the k-th asymptotic bin: 0 .. kNFHalf-G-1, then kNFHalf+G .. kNF-1
          auto asym_bin = [](int k) { return k < kNFHalf - G ? k : k + 2 * G; };
          typename Ld::P ring[kDepth];
          ring[0] = cur;
#pragma unroll
          for (int q = 1; q < kDepth; ++q) ring[q] = Ld::raw(Pp + (int64_t)asym_bin(q) * pitch);
#pragma unroll
          for (int h = 0; h < 2 * G; ++h) {
            const int jp = h - G;
            const typename Ld::P gp = Ld::raw(Pp + (int64_t)(kNFHalf + jp) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(gp, cur_r, cur_i, cur_w);
            constexpr float kZero = 0.0f;
            const float c = kZero + (float)jp;
            float wr, wi;
            w_general(jp == -1 ? a1 : aa - c, jp == -1 ? a1 + eps : ae - c, sig, spi, cpsi, spsi,
                      jp >= 0, wr, wi);
            if (kR16) {
              wr = round_f16(wr);
              wi = round_f16(wi);
            }
            acc_general(s, cur_r, cur_i, cur_w, wr, wi);
          }
#pragma unroll
          for (int k = 0; k < kAsym; ++k) {
            const typename Ld::P pj = ring[k % kDepth];
            if (k + kDepth < kAsym) ring[k % kDepth] = Ld::raw(Pp + (int64_t)asym_bin(k + kDepth) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(pj, cur_r, cur_i, cur_w);
            constexpr float kZero = 0.0f;
            const float c = kZero + (float)(asym_bin(k) - kNFHalf);
            acc_asym<kR16>(s, cur_r, cur_i, cur_w, __fadd2_rn(xae, make_float2(-c, -c)), m2c);
          }
        };
        if (JLO >= -1 && JHI <= 0) {
          unrolled(GeneralBins<1>{});  // ~72 % of the units on the two-year bank
        } else if (JLO >= -2 && JHI <= 1) {
          unrolled(GeneralBins<2>{});  // ~18 %
        } else {
          float jpf = -(float)kNFHalf;  // jp as an exact float (no int-to-float per bin)
#pragma unroll kBinUnroll
          for (int j = 0; j < kNF; ++j, jpf += 1.0f) {
            typename Ld::P nxt;
            if (j + 1 < kNF) nxt = Ld::raw(Pp + (int64_t)(j + 1) * pitch);
            float2 cur_r, cur_i, cur_w;
            Ld::cvt(cur, cur_r, cur_i, cur_w);
            const int jp = j - kNFHalf;
            // x1 = (f_nm - f_k)/df formed directly from aa: aa + 10 - j would round aa
            // to ulp(10) and ruin 1/x1 for the bins next to f_nm
            const float2 xx = __fadd2_rn(xae, make_float2(-jpf, -jpf));
            const float x1 = xx.x, x2 = xx.y;
            if (jp >= JLO && jp <= JHI) {
              float wr, wi;
              const bool near = jp == -1;
              w_general(near ? a1 : x1, near ? a1 + eps : x2, sig, spi, cpsi, spsi, true, wr, wi);
              if (kR16) {
                wr = round_f16(wr);
                wi = round_f16(wi);
              }
              acc_general(s, cur_r, cur_i, cur_w, wr, wi);
            } else {
              acc_asym<kR16>(s, cur_r, cur_i, cur_w, xx, m2c);
            }
            if (j + 1 < kNF) cur = nxt;
          }
        }
        // Z = i conj(U1) - i e^{i Psi} conj(U2), both channels at once
        const float2 ncp = make_float2(-cpsi, -cpsi);
        const float2 zr = __ffma2_rn(make_float2(spsi, spsi), s.u2r, __ffma2_rn(ncp, s.u2i, s.u1i));
        const float2 zi = __ffma2_rn(ncp, s.u2r, __ffma2_rn(make_float2(-spsi, -spsi), s.u2i, s.u1r));
        const float zr0 = zr.x, zi0 = zi.x, n0 = s.nn.x, zr1 = zr.y, zi1 = zi.y, n1 = s.nn.y;
        float ar = Tr0 * zr0 - Ti0 * zi0, ai = Tr0 * zi0 + Ti0 * zr0;
        float nt = (Tr0 * Tr0 + Ti0 * Ti0) * n0;
        if (NCH == 2) {
          ar += Tr1 * zr1 - Ti1 * zi1;
          ai += Tr1 * zi1 + Ti1 * zr1;
          nt += (Tr1 * Tr1 + Ti1 * Ti1) * n1;
        }
        Zr = ar;
        Zi = ai;
        Nn = nt;
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

// The instantiation of (channels, pixel type, pitch, response, variant). Variants other
// than 0 are compiled for the two-channel, fixed-pitch planes only (the configuration of
// long A/E grids); other configurations map every variant to variant 0.
template <int NCH, int PIX, int PITCH>
static void (*kernel_of(int resp, int variant))(EvalArgs) {
  constexpr bool kTuned = NCH == 2 && PITCH == kMixedPitch && PIX <= TFS_PIX_BF16;
  const int v = kTuned ? variant : 0;
  if (resp == 2) {
    if (v == 1) return k_eval_mixed<NCH, PIX, PITCH, true, kTuned ? 1 : 0>;
    if (v == 2) return k_eval_mixed<NCH, PIX, PITCH, true, kTuned ? 2 : 0>;
    return k_eval_mixed<NCH, PIX, PITCH, true, 0>;
  }
  if (v == 1) return k_eval_mixed<NCH, PIX, PITCH, false, kTuned ? 1 : 0>;
  if (v == 2) return k_eval_mixed<NCH, PIX, PITCH, false, kTuned ? 2 : 0>;
  return k_eval_mixed<NCH, PIX, PITCH, false, 0>;
}

template <int NCH, int PIX, int PITCH>
static cudaError_t launch_one(const EvalArgs& a, int variant, int warps, int ctas, cudaStream_t s) {
  const size_t smem = (size_t)warps * a.fine_cap * sizeof(float4);
  kernel_of<NCH, PIX, PITCH>(a.response, variant)<<<ctas, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// Sets the dynamic shared-memory limit of the instantiation and returns how many CTAs
// of this shape fit on one SM.
template <int NCH, int PIX, int PITCH>
static cudaError_t occ_one(int variant, int warps, int fine_cap, int resp, int* n) {
  const size_t smem = (size_t)warps * fine_cap * sizeof(float4);
  auto kern = kernel_of<NCH, PIX, PITCH>(resp, variant);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, warps * 32, smem);
}

// Instantiation for (channels, pixel type, pitch); CALL(NCH, PIX, PITCH) is an expression.
#define TFS_MIXED_DISPATCH_PIX(CALL, N, pix, fixed)                                         \
  do {                                                                                      \
    if ((pix) == TFS_PIX_F32)                                                               \
      return (fixed) ? CALL(N, TFS_PIX_F32, kMixedPitch) : CALL(N, TFS_PIX_F32, 0);         \
    if ((pix) == TFS_PIX_F16)                                                               \
      return (fixed) ? CALL(N, TFS_PIX_F16, kMixedPitch) : CALL(N, TFS_PIX_F16, 0);         \
    if ((pix) == TFS_PIX_BF16)                                                              \
      return (fixed) ? CALL(N, TFS_PIX_BF16, kMixedPitch) : CALL(N, TFS_PIX_BF16, 0);       \
    if ((pix) == TFS_PIX_F16_ALL)                                                           \
      return (fixed) ? CALL(N, TFS_PIX_F16_ALL, kMixedPitch) : CALL(N, TFS_PIX_F16_ALL, 0); \
    return (fixed) ? CALL(N, TFS_PIX_BF16_ALL, kMixedPitch) : CALL(N, TFS_PIX_BF16_ALL, 0);  \
  } while (0)
#define TFS_MIXED_DISPATCH(CALL, n_chan, pix, pitch)                                        \
  do {                                                                                      \
    const bool fixed_ = (pitch) == kMixedPitch;                                             \
    if ((n_chan) == 1) TFS_MIXED_DISPATCH_PIX(CALL, 1, pix, fixed_);                        \
    TFS_MIXED_DISPATCH_PIX(CALL, 2, pix, fixed_);                                           \
  } while (0)

// Launch only (no attribute calls, so it can be captured into a CUDA graph);
// mixed_occupancy() must have been called for the same shape first.
cudaError_t launch_eval_mixed(const EvalArgs& a, int n_chan, int pix, int variant, int warps,
                              int ctas, cudaStream_t s) {
  if (a.n_tpl <= 0) return cudaSuccess;
#define TFS_CALL(N, P, Q) launch_one<N, P, Q>(a, variant, warps, ctas, s)
  TFS_MIXED_DISPATCH(TFS_CALL, n_chan, pix, a.pitch);
#undef TFS_CALL
}

cudaError_t mixed_occupancy(int n_chan, int pix, int pitch, int resp, int variant, int warps,
                            int fine_cap, int* ctas_per_sm) {
#define TFS_CALL(N, P, Q) occ_one<N, P, Q>(variant, warps, fine_cap, resp, ctas_per_sm)
  TFS_MIXED_DISPATCH(TFS_CALL, n_chan, pix, pitch);
#undef TFS_CALL
}

int mixed_variants(int n_chan, int pitch) { return n_chan == 2 && pitch == kMixedPitch ? 3 : 1; }

}  // namespace tfs
