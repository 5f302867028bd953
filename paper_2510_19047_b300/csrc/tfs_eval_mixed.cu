// Mixed-precision evaluation of Upsilon_{N_seg} (Eq. Upsilon-seg): one warp per
// template, one lane per tranche, persistent CTAs that take templates from a
// length/frequency-sorted queue.
//
// Per tranche (lane):
//   * the track (Sec. "Time-frequency waveform representation": phi_nm, f_nm,
//     fdot_nm at the tranche start) in double-float arithmetic: retarded time
//     t' = t + n.r/c, u = 1 - t'/t_c, y = u^(-1/8) by one Newton step, f, and the phase
//     in cycles (accurate to ~1e-8 cycles over 1e6 cycles); fdot, amplitude and
//     response in FP32;
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
// Per warp: tranche sums are folded into the template's finest common segments by a
// deterministic segmented shuffle reduction into shared memory, and at the end into
// every requested N_seg (Eqs. overlap-n, Upsilon-seg).
#include <math.h>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"

namespace tfs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Pixel loads: one element per (bin, tranche) holds both channels of u and w,
// ur = (Re u_A, Re u_E), ui = (Im u_A, Im u_E), w = (w_A, w_E): one 128-bit load for
// FP16/BF16 pixels, two for FP32.
template <int PIX>
struct PixLoad;
template <>
struct PixLoad<TFS_PIX_F32> {
  struct __align__(16) P {
    float4 u, w;
  };
  __device__ static void load(const P* p, float2& ur, float2& ui, float2& w) {
    const float4 a = __ldg(&p->u), b = __ldg(&p->w);
    ur = make_float2(a.x, a.y);
    ui = make_float2(a.z, a.w);
    w = make_float2(b.x, b.y);
  }
};
template <>
struct PixLoad<TFS_PIX_F16> {
  using P = uint4;
  __device__ static float2 cv(unsigned int x) {
    __half2 h = *reinterpret_cast<__half2*>(&x);
    return __half22float2(h);
  }
  __device__ static void load(const P* p, float2& ur, float2& ui, float2& w) {
    const uint4 v = __ldg(p);
    ur = cv(v.x);
    ui = cv(v.y);
    w = cv(v.z);
  }
};
template <>
struct PixLoad<TFS_PIX_BF16> {
  using P = uint4;
  __device__ static float2 cv(unsigned int x) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&x);
    return __bfloat1622float2(h);
  }
  __device__ static void load(const P* p, float2& ur, float2& ui, float2& w) {
    const uint4 v = __ldg(p);
    ur = cv(v.x);
    ui = cv(v.y);
    w = cv(v.z);
  }
};

__device__ __forceinline__ df two_prod(float a, float b) {
  df r;
  r.hi = __fmul_rn(a, b);
  r.lo = __fmaf_rn(a, b, -r.hi);
  return r;
}

// Paper's auxiliary Fresnel functions in FP32 with approximate division.
__device__ __forceinline__ void fg_fast(float a, float& f, float& g) {
  if (a > 6.0f) {
    f = __fdividef(1.0f, (float)kPi * a);
    g = 0.0f;
  } else {
    f = __fdividef(fmaf(0.926f, a, 1.0f), fmaf(a, fmaf(3.104f, a, 1.792f), 2.0f));
    g = __fdividef(1.0f, fmaf(a, fmaf(a, fmaf(6.670f, a, 3.492f), 4.142f), 2.0f));
  }
}

}  // namespace

#ifndef TFS_MIXED_UNROLL
#define TFS_MIXED_UNROLL 3
#endif
#ifndef TFS_MIXED_MINB
#define TFS_MIXED_MINB 4
#endif
#ifndef TFS_MIXED_PREFETCH
#define TFS_MIXED_PREFETCH 1
#endif
constexpr int kBinUnroll = TFS_MIXED_UNROLL;
constexpr int kPrefetch = TFS_MIXED_PREFETCH;

template <int NCH, int PIX>
__global__ void __launch_bounds__(256, TFS_MIXED_MINB) k_eval_mixed(EvalArgs a) {
  extern __shared__ float4 s_acc[];
  using Ld = PixLoad<PIX>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4* acc = s_acc + (size_t)warp * a.fine_cap;
  const GridDesc g = a.g;
  const typename Ld::P* __restrict__ PX = (const typename Ld::P*)a.Umix;
  const int pitch = a.pitch;
  const df dTd = df_make(g.dT);
  const float dTf = (float)g.dT;
  const float sig_k = (float)(sqrt(2.0) * g.df);       // sigma = df sqrt(2/fdot)
  const float ncomp = (float)(10.0 * g.df / g.dT);      // fdot > 10 df / dT: non-compact
  const df one = {1.0f, 0.0f};

  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= a.n_work) break;
    const int idx = a.perm ? a.perm[t] : t;
    const TplMix c = a.tplm[idx];

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
    for (int q = lane; q < n_fine; q += 32) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    const df tc_inv = {c.tcinv_hi, c.tcinv_lo};
    const df F0 = {c.F0_hi, c.F0_lo};
    const float C2 = c.C2;
    const float fd_k = c.fd_k;  // fdot_src = fd_k y^11 (3 + 5 C2 y^2)
    const df P5 = {c.P5_hi, c.P5_lo};  // phase coefficients in cycles
    const df P3 = {c.P3_hi, c.P3_lo};
    const df Kc = {c.K_hi, c.K_lo};
    const df dopc = {c.dopc_hi, c.dopc_lo}, dops = {c.dops_hi, c.dops_lo};
    int nact = 0, nnc = 0;
    __syncwarp();

    for (int m0 = c.m_lo; m0 < c.m_hi; m0 += 32) {
      const int m = m0 + lane;
      const bool inr = m < c.m_hi;
      bool act = inr && a.mask[m];
      float Zr = 0.f, Zi = 0.f, Nn = 0.f;
      int kc = 0;
      float aa = 0.f, eps = 0.f, sig = 1.f, spsi = 0.f, cpsi = 1.f, amp_c = 0.f, amp_s = 0.f;
      float Tr0 = 1.f, Ti0 = 0.f, Tr1 = 1.f, Ti1 = 0.f;
      if (act) {
        const TrancheF tr = a.tabF[m];
        const df tt = {tr.t_hi, tr.t_lo};
        df d0 = {0.f, 0.f};
        float d1 = 0.f, d2 = 0.f;
        if (a.response) {
          const df ca = {tr.ca_hi, tr.ca_lo}, sa = {tr.sa_hi, tr.sa_lo};
          d0 = df_add(df_mul(dopc, ca), df_mul(dops, sa));
          d1 = (float)kOmega * (dops.hi * ca.hi - dopc.hi * sa.hi);
          d2 = -(float)(kOmega * kOmega) * d0.hi;
        }
        const df tp = df_add(tt, d0);
        const df u = df_sub(one, df_mul(tp, tc_inv));  // 1 - t'/t_c
        if (!(u.hi > 0.f)) {
          act = false;
        } else {
          // y = u^(-1/8): FP32 seed, one Newton step with a double-float residual
          const float y0 = rsqrtf(sqrtf(sqrtf(u.hi)));
          const df y02 = two_prod(y0, y0);
          const df y08 = df_sqr(df_sqr(y02));
          const df p = df_mul(u, y08);
          const float r = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);
          const df y = quick_two_sum(y0, y0 * r * 0.125f);
          const df y2 = df_sqr(y);
          const df y3 = df_mul(y2, y);
          const float c2y2 = C2 * y2.hi;
          const df onec = two_sum(1.0f, c2y2);
          const df fs = df_mul(df_mul(F0, y3), onec);  // source-frame frequency
          const df f = df_add_f(fs, fs.hi * d1);        // detector frame: f (1 + dt'/dt - 1)
          const float y2f = y2.hi, y3f = y3.hi;
          const float fds = fd_k * (y3f * y3f * y3f * y2f) * fmaf(5.0f * C2, y2f, 3.0f);
          const float fdot = fds * (1.0f + d1) * (1.0f + d1) + fs.hi * d2;
          const df x = df_mul(f, dTd);  // f_nm / df
          float kcf = ceilf(x.hi);
          if (kcf == x.hi && x.lo > 0.f) kcf += 1.0f;
          kc = (int)kcf;
          aa = __fadd_rn(__fsub_rn(x.hi, kcf), x.lo);  // f_nm/df - k_c, in (-1, 0]
          if (!(fdot > 0.f) || kc - kNFHalf < 1 || kc + kNFHalf > g.n_bins - 1) {
            act = false;
          } else {
            ++nact;
            if (fdot > ncomp) ++nnc;
            // phase in cycles: K - P5 u^(5/8) - P3 u^(3/8), with u^(5/8) = u y^3 and
            // u^(3/8) = u y^5; the fractional part is taken in two steps because the hi
            // word can be an integer-valued float (|Phi| > 2^23 cycles)
            const df u58 = df_mul(u, y3);
            const df u38 = df_mul(u58, y2);
            const df ph = df_sub(df_sub(Kc, df_mul(P5, u58)), df_mul(P3, u38));
            float cyc = __fadd_rn(__fsub_rn(ph.hi, rintf(ph.hi)), ph.lo);
            cyc = __fsub_rn(cyc, rintf(cyc));
            // cyc is in [-1/2, 1/2]: the hardware sine/cosine are accurate to ~4e-7 there
            float sph, cph;
            __sincosf(6.283185307f * cyc, &sph, &cph);
            // amplitude (f/F0)^(2/3) = y^2 (1 + C2 y^2)^(2/3), series to O(e^4)
            const float amp =
                y2f * fmaf(c2y2, fmaf(c2y2, fmaf(c2y2, 4.0f / 81.0f, -1.0f / 9.0f), 2.0f / 3.0f),
                           1.0f);
            amp_c = amp * cph;
            amp_s = amp * sph;
            sig = sig_k * rsqrtf(fdot);
            eps = fdot * dTf * dTf;  // fdot dT / df: sweep width in bins
            const float psi = fmaf(2.0f, aa, eps);  // Psi / pi, reduced to [-1, 1]
            __sincosf(3.141592654f * (psi - 2.0f * rintf(0.5f * psi)), &spsi, &cpsi);
            if (a.response) {
              float fpA = 0.f, fxA = 0.f, fpE = 0.f, fxE = 0.f;
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                fpA = fmaf(tr.DA[q], c.pp[q], fpA);
                fxA = fmaf(tr.DA[q], c.px[q], fxA);
                fpE = fmaf(tr.DE[q], c.pp[q], fpE);
                fxE = fmaf(tr.DE[q], c.px[q], fxE);
              }
              Tr0 = fpA;
              Ti0 = -fxA;
              Tr1 = fpE;
              Ti1 = -fxE;
            }
          }
        }
      }
      // window-relative bins that need the exact (rational or in-sweep) branch
      int jlo = 100, jhi = -100;
      if (act) {
        const float r6 = __fdividef(6.0f, sig);
        jlo = (int)ceilf(aa - r6 - 0.01f);
        jhi = (int)floorf(aa + eps + r6 + 0.01f);
      }
      const int JLO = __reduce_min_sync(kFull, jlo);
      const int JHI = __reduce_max_sync(kFull, jhi);
      if (act) {
        const typename Ld::P* Pp = PX + (int64_t)(kc - kNFHalf) * pitch + m;
        float2 zr = make_float2(0.f, 0.f), zi = zr, nn = zr;  // (channel A, channel E)
        const float spi = sig * (float)kPi;
        // pixel loads run kPrefetch bins ahead of the arithmetic
        float2 cur_r, cur_i, cur_w, p1_r, p1_i, p1_w;
        Ld::load(Pp, cur_r, cur_i, cur_w);
        if (kPrefetch > 1) Ld::load(Pp + pitch, p1_r, p1_i, p1_w);
        float jpf = -(float)kNFHalf;  // j - 10 as an exact float (no int-to-float per bin)
#pragma unroll kBinUnroll
        for (int j = 0; j < kNF; ++j, jpf += 1.0f) {
          float2 nxt_r, nxt_i, nxt_w;
          if (j + kPrefetch < kNF) Ld::load(Pp + (int64_t)(j + kPrefetch) * pitch, nxt_r, nxt_i, nxt_w);
          const int jp = j - kNFHalf;
          // x1 = (f_nm - f_k)/df, formed directly from aa: aa + 10 - j would round aa
          // to ulp(10) and ruin 1/x1 for the bins next to f_nm
          const float x1 = aa - jpf;
          const float x2 = x1 + eps;
          float wr, wi;
          if (jp >= JLO && jp <= JHI) {
            const float v1 = sig * x1, v2 = sig * x2;
            float f1, g1, f2, g2;
            fg_fast(fabsf(v1), f1, g1);
            fg_fast(fabsf(v2), f2, g2);
            const float s1 = v1 < 0.f ? -1.f : 1.f, s2 = v2 < 0.f ? -1.f : 1.f;
            wr = s1 * g1 - s2 * (g2 * cpsi - f2 * spsi);
            wi = s1 * f1 - s2 * (g2 * spsi + f2 * cpsi);
            if (s1 != s2) {
              float sp, cp;
              sincospif(0.5f * v1 * v1, &sp, &cp);
              wr += cp + sp;
              wi += cp - sp;
            }
            wr *= spi;
            wi *= spi;
          } else {
            const float q1 = __fdividef(1.0f, x1), q2 = __fdividef(1.0f, x2);
            wr = spsi * q2;
            wi = fmaf(-cpsi, q2, q1);
          }
          const float ww = fmaf(wr, wr, wi * wi);
          const float2 wr2 = make_float2(wr, wr), wi2 = make_float2(wi, wi);
          const float2 nwr2 = make_float2(-wr, -wr), ww2 = make_float2(ww, ww);
          // conj(u) W for both channels at once
          zr = __ffma2_rn(cur_r, wr2, __ffma2_rn(cur_i, wi2, zr));
          zi = __ffma2_rn(cur_r, wi2, __ffma2_rn(cur_i, nwr2, zi));
          nn = __ffma2_rn(cur_w, ww2, nn);
          if (kPrefetch > 1) {
            cur_r = p1_r;
            cur_i = p1_i;
            cur_w = p1_w;
            if (j + kPrefetch < kNF) {
              p1_r = nxt_r;
              p1_i = nxt_i;
              p1_w = nxt_w;
            }
          } else if (j + 1 < kNF) {
            cur_r = nxt_r;
            cur_i = nxt_i;
            cur_w = nxt_w;
          }
        }
        const float zr0 = zr.x, zi0 = zi.x, n0 = nn.x, zr1 = zr.y, zi1 = zi.y, n1 = nn.y;
        float ar = Tr0 * zr0 - Ti0 * zi0, ai = Tr0 * zi0 + Ti0 * zr0;
        float nt = (Tr0 * Tr0 + Ti0 * Ti0) * n0;
        if (NCH == 2) {
          ar += Tr1 * zr1 - Ti1 * zi1;
          ai += Tr1 * zi1 + Ti1 * zr1;
          nt += (Tr1 * Tr1 + Ti1 * Ti1) * n1;
        }
        Zr = ar * amp_c - ai * amp_s;
        Zi = ar * amp_s + ai * amp_c;
        Nn = (amp_c * amp_c + amp_s * amp_s) * nt;
      }
      // segmented (by finest segment) suffix sums across the warp; the first lane
      // of each run adds its segment's sum to shared memory
      const int key = inr ? m / fine_len : 0x7fffffff;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float zr2 = __shfl_down_sync(kFull, Zr, o);
        const float zi2 = __shfl_down_sync(kFull, Zi, o);
        const float n2 = __shfl_down_sync(kFull, Nn, o);
        const int k2 = __shfl_down_sync(kFull, key, o);
        if (lane + o < 32 && k2 == key) {
          Zr += zr2;
          Zi += zi2;
          Nn += n2;
        }
      }
      const int kprev = __shfl_up_sync(kFull, key, 1);
      if (inr && (lane == 0 || kprev != key)) {
        float4 v = acc[key];
        v.x += Zr;
        v.y += Zi;
        v.z += Nn;
        acc[key] = v;
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

template <int NCH, int PIX>
static cudaError_t launch_one(const EvalArgs& a, int warps, int ctas, cudaStream_t s) {
  const size_t smem = (size_t)warps * a.fine_cap * sizeof(float4);
  k_eval_mixed<NCH, PIX><<<ctas, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// Launch only (no attribute calls, so it can be captured into a CUDA graph);
// mixed_occupancy() must have been called for the same shape first.
cudaError_t launch_eval_mixed(const EvalArgs& a, int n_chan, int pix, int warps, int ctas,
                              cudaStream_t s) {
  if (a.n_tpl <= 0) return cudaSuccess;
  if (n_chan == 1) {
    if (pix == TFS_PIX_F32) return launch_one<1, TFS_PIX_F32>(a, warps, ctas, s);
    if (pix == TFS_PIX_F16) return launch_one<1, TFS_PIX_F16>(a, warps, ctas, s);
    return launch_one<1, TFS_PIX_BF16>(a, warps, ctas, s);
  }
  if (pix == TFS_PIX_F32) return launch_one<2, TFS_PIX_F32>(a, warps, ctas, s);
  if (pix == TFS_PIX_F16) return launch_one<2, TFS_PIX_F16>(a, warps, ctas, s);
  return launch_one<2, TFS_PIX_BF16>(a, warps, ctas, s);
}

// Sets the dynamic shared-memory limit of the instantiation and returns how many CTAs
// of this shape fit on one SM.
template <int NCH, int PIX>
static cudaError_t occ_one(int warps, int fine_cap, int* n) {
  const size_t smem = (size_t)warps * fine_cap * sizeof(float4);
  auto kern = k_eval_mixed<NCH, PIX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, warps * 32, smem);
}

cudaError_t mixed_occupancy(int n_chan, int pix, int warps, int fine_cap, int* ctas_per_sm) {
  if (n_chan == 1) {
    if (pix == TFS_PIX_F32) return occ_one<1, TFS_PIX_F32>(warps, fine_cap, ctas_per_sm);
    if (pix == TFS_PIX_F16) return occ_one<1, TFS_PIX_F16>(warps, fine_cap, ctas_per_sm);
    return occ_one<1, TFS_PIX_BF16>(warps, fine_cap, ctas_per_sm);
  }
  if (pix == TFS_PIX_F32) return occ_one<2, TFS_PIX_F32>(warps, fine_cap, ctas_per_sm);
  if (pix == TFS_PIX_F16) return occ_one<2, TFS_PIX_F16>(warps, fine_cap, ctas_per_sm);
  return occ_one<2, TFS_PIX_BF16>(warps, fine_cap, ctas_per_sm);
}

}  // namespace tfs
