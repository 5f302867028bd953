// Kernel argument blocks and host-side launchers of libtfs.
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

// Everything an evaluation kernel needs, passed by value.
// FP32 forms of grid constants for the mixed kernel, rounded once on the host (the
// kernel then needs no FP64 instruction, even where it re-derives a value per tranche).
struct MixConst {
  float dT_hi, dT_lo;  // dT as a double-float
  float dTf;           // (float) dT
  float sig_k;         // sqrt(2) df: sigma = sig_k / sqrt(fdot)
  float ncomp;         // 10 df / dT: fdot above it counts as non-compact
  float x_hi;          // n_bins - 10: window centres below it are in band
};

// Harmonic set of the templates (n = 0: the dominant mode alone).
struct HarmSet {
  int n;
  double nu[TFS_MAX_HARMONICS];
  double cr[TFS_MAX_HARMONICS], ci[TFS_MAX_HARMONICS];
  // the same for the mixed path: nu as double-float, c in FP32, and the smallest
  // |nu_a - nu_b| over pairs (windows can share bins only where dnu_min f/df < 21)
  float nu_hi[TFS_MAX_HARMONICS], nu_lo[TFS_MAX_HARMONICS];
  float crf[TFS_MAX_HARMONICS], cif[TFS_MAX_HARMONICS];
  float dnu_min;
};

struct EvalArgs {
  GridDesc g;
  MixConst mc;
  int response;
  int pitch;                    // m-dimension pitch of the mixed planes
  const TrancheD* tabD;         // [N_t]
  const TrancheF* tabF;         // [N_t]
  const float4* tdiF;           // [N_t][7]: the constellation geometry of the TDI transfer
  const double2* u64;           // [c][m][k] FP64 u = d~ w
  const double* w64;            // [c][m][k] FP64 w
  const float2* u32;            // [c][m][k] scaled FP32 u
  const float* w32;             // [c][m][k] scaled FP32 w
  const void* Umix;             // [k][pitch] mixed plane (u and w of both channels)
  const uint8_t* mask;          // [N_t]
  const int32_t* live;          // [n_live] unmasked tranches in increasing order
  const int32_t* rank;          // [N_t + 1] unmasked tranches before tranche m
  const TplConst* tpl;          // [n_tpl]
  const TplMix* tplm;           // [n_tpl] (mixed path)
  const int32_t* perm;          // processing order (mixed path), may be null
  int64_t n_tpl;
  int64_t n_work;               // queue entries the mixed launch processes (<= n_tpl)
  Levels lv;                    // global levels (per-template mode: lv.n == 0)
  const int32_t* nseg_pt;       // per-template N_seg or null
  int fine_cap;                 // smem fine-segment slots per warp (mixed path)
  double* out_stat;             // [levels][n_tpl]
  int32_t* out_neff;            // [levels][n_tpl] or null
  int32_t* out_diag;            // [2][n_tpl] or null
  double out_scale;             // Upsilon = out_scale * sum |Z|^2 / N
  int* counter;                 // work ticket of the persistent launch
  int* dev_err;                 // checked-mode status word
  int checked;
  HarmSet harm;                 // harmonics (FP64 and mixed paths)
  const float2* harm_K;         // [n_tpl][harm.n] frac(nu_h Phi_const) as double-float (mixed path)
};

cudaError_t launch_tranche_table(const GridDesc& g, TrancheD* td, TrancheF* tf, float4* tdi,
                                 cudaStream_t s);
cudaError_t launch_absmax(int64_t n, const double* d_re, const double* d_im, const double* w,
                          unsigned long long* umax, unsigned long long* wmax, int* bad,
                          int n_sm, cudaStream_t s);
cudaError_t launch_pack_ref(int64_t n, const double* d_re, const double* d_im, const double* w,
                            double su, double sw, double2* u64, double* w64, float2* u32,
                            float* w32, int n_sm, cudaStream_t s);
// P: the mixed plane, 16 B (FP16/BF16) or 32 B (FP32) per pixel, [n_bins][pitch].
cudaError_t launch_pack_mixed(int pix, const GridDesc& g, int pitch, const double* d_re,
                              const double* d_im, const double* w, double su, double sw, void* P,
                              int n_sm, cudaStream_t s);
// mix may be null (only the mixed path reads it). [nu_min, nu_max]: the harmonics'
// frequency factors, which widen the tranche range that can be active.
cudaError_t launch_setup(const double* theta, int64_t n, int pn_order, const GridDesc& g,
                         TplConst* out, TplMix* mix, cudaStream_t s, double nu_min = 1.0,
                         double nu_max = 1.0);

cudaError_t launch_check_tpl(const TplConst* tpl, int64_t n, int n_tranche, int* err, cudaStream_t s);
cudaError_t launch_eval_fp64(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_eval_plain(const EvalArgs& a, cudaStream_t s);
// CTAs of 128 threads resident per SM for the FP64 (path 0) or plain (path 1) kernel.
cudaError_t ref_occupancy(const EvalArgs& a, int path, int* per_sm);
// Persistent mixed-precision launch; grid = ctas, block = 32 * warps; variant selects
// the compiled tile/schedule variant (0 .. mixed_variants() - 1).
cudaError_t launch_eval_mixed(const EvalArgs& a, int n_chan, int pix, int variant, int warps,
                              int ctas, cudaStream_t s);
cudaError_t mixed_occupancy(int n_chan, int pix, int pitch, int resp, int variant, int warps,
                            int fine_cap, int* ctas_per_sm);
// Number of compiled variants for this configuration.
int mixed_variants(int n_chan, int pitch);
// Multi-harmonic mixed launch (persistent, a.counter zeroed by the caller); a.harm_K
// from launch_harm_phase. Chooses its own grid (n_sm x resident CTAs of 8 warps).
cudaError_t launch_eval_harm(const EvalArgs& a, int n_chan, int pix, int n_sm, cudaStream_t s,
                             int* shape = nullptr);  // shape: threads per CTA, CTAs, CTAs per SM
// K[i][h] = frac(nu_h (phi0 + P5 + P3) / 2 pi) of template i as double-float.
cudaError_t launch_harm_phase(const TplConst* tpl, int64_t n, const HarmSet& h, float2* K,
                              cudaStream_t s);

// Particle-swarm state of S swarms x P particles (all device pointers): positions,
// velocities and personal bests SoA [8][S*P] (particle i of swarm s at s*P + i), personal
// best values [S*P], swarm bests [8][S] and values [S]; tile corners [S][8].
struct PsoArgs {
  int n_swarm, n_part;
  double *x, *v, *pbest, *pval, *gbest, *gval;
  const double *lo, *hi;
  double inertia, c1, c2;
  uint2 key;        // Philox key (the seed)
  double* history;  // [iterations][S] swarm best after each step, or null
};
cudaError_t launch_pso_init(const PsoArgs& a, int n_sm, cudaStream_t s);
cudaError_t launch_pso_step(const PsoArgs& a, const double* f, int64_t iter, int move,
                            cudaStream_t s);

// Noise-only data grid from the weights w (FP64 [c][m][k]) into d_re, d_im.
cudaError_t launch_noise(int64_t n, const double* w, double df, uint64_t seed, double* d_re,
                         double* d_im, int n_sm, cudaStream_t s);

// One refinement step of n candidates (device pointers; see k_refine_update).
struct RefineArgs {
  int64_t n;
  const double *stat, *grad;            // U [n] and dU/dtheta [8][n] at theta
  double *theta, *best_theta, *best_grad, *best_stat, *eta;
  const double* sigma;                  // [8][n]
  double lo[8], hi[8];
  double eta_up, eta_down;
  double* mean_out;                     // mean of U_best, or null
  double* part;                         // [blocks] partial sums (when mean_out is set)
  unsigned* done;                       // block counter, zero between calls
};
cudaError_t launch_refine_update(const RefineArgs& a, cudaStream_t s);

struct AscentParams {
  double step[8], lo[8], hi[8];
};
cudaError_t launch_ascent(double* theta, const double* grad, int64_t n, const AscentParams& p,
                          cudaStream_t s);
// Adjoint gradient at one N_seg: out_stat [n], out_grad [8][n] (device pointers).
// Work items per template of the gradient kernel (1 .. kGradMaxParts) for a batch of n:
// parts > 1 needs a [parts][9][n] FP64 buffer for the partial sums.
constexpr int kGradMaxParts = 4;
cudaError_t grad_plan(int response, int n_seg, int n_sm, int64_t n, int* parts, int* parts_a);
cudaError_t launch_grad(const GridDesc& g, const MixConst& mc, int response, int pn_order,
                        int pitch, const TrancheF* tabF, const float4* P, const uint8_t* mask,
                        const double* theta, const TplConst* tpl, const TplMix* tplm, int64_t n,
                        int n_seg, double scale, double* out_stat, double* out_grad,
                        unsigned* counter, const int32_t* perm, int parts, int parts_a,
                        double* part_buf, double* src_buf, float4* lam_buf, int n_sm,
                        cudaStream_t s);
// Bytes of launch_grad's src_buf for n templates (the constants' theta-derivatives);
// lam_buf holds n * n_seg float4 (the segments' adjoint weights).
size_t grad_src_bytes(int64_t n);

}  // namespace tfs
