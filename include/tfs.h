/*
 * tfs.h -- C ABI of libtfs, a B300 (sm_103a) library that evaluates the
 * time-frequency semi-coherent detection statistic of arXiv:2510.19047
 * ("Global time-frequency search for stellar-mass binary black holes in LISA")
 * for large banks of inspiral templates, and its gradient.
 *
 * What is computed (paper notation):
 *   For every template theta and segment n (segment length T_seg = N_t dT / N_seg,
 *   Eq. Upsilon-seg), the tranche-decomposed complex inner products
 *     Z_n = sum_alpha sum_{m in n} T_alpha,nm sum_{k in window} conj(d~_alpha,nm[k])
 *           h~_nm[k] / S_alpha,nm[k] delta f                 (Eqs. inner-tf, inner-tranche-tf)
 *     N_n = sum_alpha sum_{m in n} |T_alpha,nm|^2 sum_k |h~_nm[k]|^2 / S_alpha,nm[k] delta f
 *   with h~_nm the Fresnel-kernel transform of the quadratic-phase tranche
 *   (Eq. fresnel-ft, Eq. kernel-function, the paper's Fresnel forms for |z| > 6 and
 *   |z| <= 6), N_F = 21 bins about k_c = ceil(f_nm / delta f), and
 *     Upsilon_{N_seg} = sum_{n: N_n > 0} 4 |Z_n|^2 / N_n           (Eqs. overlap-n, Upsilon-seg)
 *   A tranche is active iff it is not masked (gaps: a tranche that overlaps a gap
 *   is left out of Eq. inner-tf), t'_nm < t_c, fdot_nm > 0 and its window lies in
 *   bins [1, N_bins - 1].
 *
 * Templates: theta is structure-of-arrays double [8][n_tpl] in the order
 *   (M_c [M_sun], eta, f_0 [Hz], phi_0 [rad], lambda, beta, psi, iota [rad]);
 *   f_0, phi_0 are the GW frequency and phase at barycentre time t' = 0.
 *   Chirp: Newtonian (pn_order 0) or 1PN TaylorT3 (pn_order 1). Response: none
 *   (T = 1, one or two identical channels), the long-wavelength A/E response of a
 *   rigid constellation on a 1 AU orbit with Doppler delay t' = t + n.r(t)/c
 *   (response 1), or the TDI-1.5 A/E transfer of the same rigidly rotating,
 *   constant-arm (2.5e9 m) constellation built from single-link observables and
 *   evaluated at each tranche's (t_nm, f_nm) (response 2; Eq. tdi2).
 *
 * Pointers: every array argument may be a host pointer or a device pointer of the
 *   context's device (the library asks the CUDA runtime which). Inputs are read
 *   or copied, never retained after the call returns. Outputs are owned by the
 *   caller. A call runs on `stream` (a cudaStream_t, NULL = legacy default stream);
 *   it returns before the GPU finishes only if every output pointer is a device
 *   pointer, otherwise it synchronises the stream before returning.
 *
 * Errors: every entry point returns TFS_OK (0) or a negative tfs_status; a
 *   human-readable message is then available from tfs_last_error(). No C++
 *   exception crosses this interface. Functions are not re-entrant on one
 *   context; distinct contexts are independent.
 */
#ifndef TFS_H
#define TFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tfs_ctx tfs_ctx; /* opaque; owns all device memory it allocates */

typedef enum tfs_status {
  TFS_OK = 0,
  TFS_ERR_ARG = -1,          /* bad argument: null pointer, size, value out of range */
  TFS_ERR_STATE = -2,        /* data or noise weights not loaded yet */
  TFS_ERR_NSEG = -3,         /* N_t is not divisible by a requested N_seg */
  TFS_ERR_OOM = -4,          /* device allocation failed or over the context's cap */
  TFS_ERR_CUDA = -5,         /* a CUDA runtime call failed (message has the detail) */
  TFS_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  TFS_ERR_DEVICE_CHECK = -7  /* checked mode: a kernel saw an out-of-range index */
} tfs_status;

typedef enum tfs_path {
  TFS_PATH_FP64 = 0,  /* all-FP64 parity path, one thread per template */
  TFS_PATH_PLAIN = 1, /* the paper's mapping: one thread per template, Eq. fresnel-ft
                         evaluated bin by bin as printed, FP32 pixels, FP64 phase */
  TFS_PATH_MIXED = 2  /* warp per template, lane per tranche, phase-cancelled Fresnel
                         kernel, FP16/BF16 u with FP32 w, FP32 accumulation, double-float
                         phase track, length-sorted persistent launch */
} tfs_path;

typedef enum tfs_pixel {
  TFS_PIX_F32 = 0,      /* u = d~/S and w = 1/S in FP32 */
  TFS_PIX_F16 = 1,      /* u in FP16, w in FP32 */
  TFS_PIX_BF16 = 2,     /* u in BF16, w in FP32 */
  TFS_PIX_F16_ALL = 3,  /* u and w in FP16, and the template's per-bin kernel values and
                           per-tranche prefactor (response x amplitude x phase factor)
                           rounded to FP16 before the products; FP32 accumulation */
  TFS_PIX_BF16_ALL = 4  /* u and w in BF16, template values rounded to FP16 as above */
} tfs_pixel;

typedef struct tfs_options {
  int path;          /* tfs_path used by tfs_eval_statistic (default MIXED) */
  int pixel;         /* tfs_pixel: storage of d~/S and 1/S for the mixed path (default F16);
                        the _ALL types (precision studies) also round the template values to
                        FP16 and are not available with harmonics */
  int pn_order;      /* 0 Newtonian chirp, 1 1PN TaylorT3 (default 1) */
  int response;      /* 0 none (T = 1, t' = t), 1 long-wavelength A/E (default 1),
                        2 TDI-1.5 A/E */
  int checked;       /* 1: kernels bounds-check every pixel index (slower) */
  int sort;          /* 1: length/frequency-sort templates before the mixed launch (default 1) */
  int warps_per_cta; /* mixed path CTA size in warps; 0 = autotuned on first use */
  int use_graph;     /* 1: replay the mixed evaluation as a CUDA graph per batch shape */
  int profile;       /* 1: time each kernel of a call with CUDA events (tfs_last_profile) */
  int tile_variant;  /* with warps_per_cta set: the mixed kernel's compiled tile/schedule
                        variant, 0..2 (default 0; 1 and 2 exist for two channels on the
                        fixed plane pitch, TFS_ERR_ARG otherwise); the autotuner picks
                        its own when warps_per_cta is 0 */
  int64_t max_device_bytes; /* cap on the context's device allocations, 0 = none */
} tfs_options;

/* Default options (see the field comments). */
void tfs_default_options(tfs_options* opt);

/* Create a context on CUDA device `device` (the device becomes current for the
 * calling thread). opt may be NULL for defaults. *out receives the handle. */
int tfs_create(tfs_ctx** out, int device, const tfs_options* opt);

/* Free every device allocation of the context and the context itself. NULL is ok. */
int tfs_destroy(tfs_ctx* ctx);

/* Replace the context's options (takes effect at the next call). */
int tfs_set_options(tfs_ctx* ctx, const tfs_options* opt);
int tfs_get_options(const tfs_ctx* ctx, tfs_options* opt);

/* Load the time-frequency data grid d~_alpha,m[k] (Eq. inner-tranche-tf):
 *   n_chan 1 or 2 (A, E), n_tranche N_t in [1, 65535], n_bins in [22, 2^21] complex bins per tranche
 *   (bin k at f_k = k / dT), dt the sample cadence (dT / dt >= 2 n_bins), dT the
 *   tranche length [s], t0 the start time of tranche 0 [s].
 *   d_re, d_im: double [n_chan][n_tranche][n_bins], host or device, copied.
 * Any previously loaded data and noise weights are dropped. */
int tfs_load_tf_data(tfs_ctx* ctx, int n_chan, int n_tranche, int n_bins, double dt,
                     double dT, double t0, const double* d_re, const double* d_im);

/* Set the noise weights 1/S_alpha,m[k] (one-sided PSD per tranche; the paper lets the
 * PSD change between tranches, "Search extension to data with gaps") and the tranche
 * mask (gaps: 0 = tranche overlaps a gap and is left out).
 *   inv_psd: double [n_chan][n_tranche][n_bins], >= 0 and finite, host or device.
 *   tranche_mask: uint8 [n_tranche], or NULL for "keep all".
 * Forms the weighted data u = d~ w once, in every storage the paths use. */
int tfs_set_noise_weights(tfs_ctx* ctx, const double* inv_psd, const uint8_t* tranche_mask);

/* Replace the loaded data by a noise-only realisation drawn from the current noise
 * weights, for false-alarm backgrounds (Secs. "Search results on the full dataset" and
 * "Injected and recovered signals": the paper builds the background of the search
 * maximum from independent noise-only realisations). Per pixel d~ = sqrt(S / (4 delta f)) (g1 + i g2) with S = 1/w (d~ = 0
 * where w = 0), so E|d~|^2 = S / (2 delta f), the data's convention; g1, g2 are
 * independent standard normals from the Box-Muller transform
 *   g1 + i g2 = sqrt(-2 ln(1 - a)) e^{2 pi i b}
 * of the two uniforms a, b in [0, 1) (top 53 bits of each half) of one Philox4x32-10
 * block keyed by `seed` (low, high 32 bits) with counter (pixel index low 32 bits, high
 * 32 bits, 0, 0x4E4F4953); pixel index = (chan * N_t + tranche) * n_bins + bin. The
 * weights and mask stay; u = d~ w is re-formed in every storage. Synchronous.
 * TFS_ERR_STATE before load_tf_data and set_noise_weights. */
int tfs_noise_realisation(tfs_ctx* ctx, uint64_t seed);

/* Upsilon_{N_seg} (Eq. Upsilon-seg) for n_tpl templates.
 *   theta: double [8][n_tpl] (SoA, order above).
 *   per_template == 0: n_seg[0..n_levels-1] are 1..4 segment counts applied to every
 *     template, all evaluated in one pass; out_stat is double [n_levels][n_tpl] and
 *     out_neff (optional) int32 [n_levels][n_tpl].
 *   per_template == 1: n_seg is int32 [n_tpl], one segment count per template
 *     (n_levels is ignored); out_stat double [n_tpl], out_neff int32 [n_tpl].
 *   Every N_seg must divide N_t (else TFS_ERR_NSEG).
 *   out_neff: number of segments with N_n > 0 (the chi^2 test has 2 N_eff dof).
 *   out_diag (optional): int32 [2][n_tpl] = active tranches, active tranches that
 *     violate the compactness condition fdot dT <= 10 delta f (Appendix A). */
int tfs_eval_statistic(tfs_ctx* ctx, const double* theta, int64_t n_tpl, const int32_t* n_seg,
                       int n_levels, int per_template, double* out_stat, int32_t* out_neff,
                       int32_t* out_diag, void* stream);

/* Upsilon_{N_seg} and its gradient d Upsilon / d theta (out_grad double [8][n_tpl]) by
 * the adjoint of Eq. Upsilon-seg: a forward pass keeps Z_n, N_n per segment, a second
 * pass recomputes the track and accumulates
 *   dUpsilon = sum_n [8 Re(conj(Z_n) dZ_n) / N_n - 4 |Z_n|^2 dN_n / N_n^2].
 * The window position and the Fresnel branch are held fixed (the almost-everywhere
 * derivative). FP32 arithmetic with a double-float phase track; with response 2 the
 * TDI-1.5 transfer's dependence on f and on the source direction is included.
 * A batch smaller than about three waves of the kernel (a few thousand templates on a
 * B300) splits each template's segments into up to four work items whose partial sums
 * are added in a fixed order: results are deterministic for a given batch size, and a
 * template's values may differ in the last bits between a small and a large batch.
 * A template with no active tranche gets Upsilon = 0 and a zero gradient. The context
 * keeps per template 1344 bytes of the constants' theta-derivatives and 16 N_seg bytes
 * of per-segment adjoint weights (device memory, grown as needed). */
int tfs_grad_statistic(tfs_ctx* ctx, const double* theta, int64_t n_tpl, int32_t n_seg,
                       double* out_stat, double* out_grad, void* stream);

/* Harmonic content of the templates (Sec. "Outlook": the time-frequency waveform
 * extends to several harmonics by computing {A, f, fdot, phi} for each harmonic and
 * applying the Fresnel expressions to each). n_harm = 0, the default, evaluates the
 * single dominant mode described above. With n_harm in [1, TFS_MAX_HARMONICS],
 * harmonic h of every template has phase nu[h] Phi(t'), frequency nu[h] f_nm,
 * derivative nu[h] fdot_nm and amplitude c[h] A with c[h] = c_re[h] + i c_im[h], and
 * the dominant mode's polarisation content (with response 2 the transfer is taken at
 * the harmonic's frequency). Each harmonic has its own 21-bin window about
 * ceil(nu[h] f_nm / delta f), used only where it lies inside [1, N_bins - 1]; the
 * tranche's template is the sum of the windows, so a bin inside two windows carries
 * both and N_n keeps the cross terms. Phases are absolute (phi_0 included): the
 * harmonics' relative phases do not cancel per segment. A tranche is active when it
 * passes the tests above with at least one window in band.
 *   nu: double [n_harm], each in (0, 16]; c_re, c_im: double [n_harm], finite; host
 *   pointers, copied (NULL allowed when n_harm = 0).
 * Applies to tfs_eval_statistic on every path; tfs_grad_statistic returns TFS_ERR_ARG
 * while n_harm > 0. */
#define TFS_MAX_HARMONICS 8
int tfs_set_harmonics(tfs_ctx* ctx, int n_harm, const double* nu, const double* c_re,
                      const double* c_im);

/* Indices of the k largest values of stat[n] (ties broken by the lower index; -0.0
 * equals +0.0; NaN ranks below every number), in decreasing order of stat, into
 * out_index int64 [k]: the survivors of one stage of
 * the adaptive N_seg ladder (Sec. "Time-frequency search statistic": N_seg is reduced
 * as the search progresses). stat and out_index may be host or device pointers. */
int tfs_select_top(tfs_ctx* ctx, const double* stat, int64_t n, int64_t k, int64_t* out_index,
                   void* stream);

/* Same selection as tfs_select_top, for callers that cannot allocate device memory:
 * code between the launches of a pipeline that must not synchronise the device
 * (cudaMalloc/cudaFree synchronise it), or a framework that owns all device memory
 * through its own pool under a fixed budget. This function has no counterpart in the
 * paper; it is a deployment variant. It calls no allocator and needs no context: the
 * radix-sort scratch is a static device array of about 1.6 MB (room for
 * n <= 65536 values) that every GPU loading this library keeps until the process
 * exits.
 *   stat: double [n] and out_index: int64 [k], both device pointers of the current
 *   device; n > 65536, host pointers or k outside [0, n] return TFS_ERR_ARG; a CUDA
 *   failure returns TFS_ERR_CUDA (no message: there is no context).
 * The first call on a device looks up the array's device address (once per device,
 * with that device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not call this function again on a device
 * after cudaDeviceReset there (the kept address belongs to the destroyed context). Every
 * call reuses the same array and overwrites every byte it reads, so nothing carries
 * over from the previous call, but calls whose GPU work overlaps (two streams, or two
 * host threads on one device) race on it: serialise them. Asynchronous on `stream`. */
int tfs_select_top_noalloc(const double* stat, int64_t n, int64_t k, int64_t* out_index,
                           void* stream);

/* One projected gradient-ascent step on a batch of templates, in place:
 *   theta[p][i] += step[p] * grad[p][i], then clamped to [lo[p], hi[p]];
 *   phi_0, lambda, psi are wrapped to [0, 2 pi) / [0, pi) instead of clamped.
 * theta, grad: double [8][n] device or host; step, lo, hi: double [8] host. */
int tfs_ascent_step(tfs_ctx* ctx, double* theta, const double* grad, int64_t n,
                    const double* step, const double* lo, const double* hi, void* stream);

/* Particle-swarm maximisation of Upsilon over parameter tiles: the paper searches
 * each tile of its (M_c, f_in) grid with a particle swarm (Sec. "Implementation
 * details"). S swarms of P particles run together; the caller evaluates Upsilon for
 * all S*P positions (one tfs_eval_statistic call on x) between steps. Global-best swarm
 * with an inertia weight: per particle and coordinate
 *   v <- inertia v + c1 r1 (pbest - x) + c2 r2 (gbest - x),   x <- x + v,
 * r1, r2 uniform in [0, 1), drawn from Philox4x32-10 keyed by `seed` with counter
 * (particle, coordinate, step): the run is a deterministic function of the seed.
 * For an angle whose tile spans its whole period (phi_0, lambda: 2 pi; psi: pi) the
 * differences take the shorter way round and x wraps into [0, period); every other
 * coordinate is clipped to the tile, which zeroes its velocity; a coordinate whose
 * tile has zero width stays fixed.
 *   n_swarm S >= 1, n_part P >= 1 (S P < 2^31); lo, hi: double [S][8] tile corners,
 *   host or device, read at each call; x, v, pbest: double [8][S*P] (SoA: particle i
 *   of swarm s at column s*P + i, the layout tfs_eval_statistic takes); pval double
 *   [S*P]; gbest double [8][S]; gval double [S]. All state arrays are device memory of
 *   the context's device, owned by the caller (TFS_ERR_ARG otherwise). */
typedef struct tfs_swarm {
  int n_swarm, n_part;
  const double *lo, *hi;
  double inertia, c1, c2;
  uint64_t seed;
  double *x, *v, *pbest, *pval, *gbest, *gval;
} tfs_swarm;

/* Initial swarm: x uniform in the tile, v uniform in +-0.1 of the tile width,
 * pbest = x, pval = gval = -inf, gbest at the tile centre. Asynchronous on `stream`. */
int tfs_pso_init(tfs_ctx* ctx, const tfs_swarm* sw, void* stream);

/* One swarm step with f = double [S*P] (device) the objective at the current x:
 * personal bests where f > pval; each swarm's best replaced by its largest pval (the
 * lowest particle index among equals) where that is larger; then, if `move` is
 * non-zero, the velocity and position update above with the draws of step `iter`
 * (>= 0). history: null, or device double [>= iter + 1][S] whose row `iter` receives
 * gval after the update. Asynchronous on `stream`. */
int tfs_pso_step(tfs_ctx* ctx, const tfs_swarm* sw, const double* f, int64_t iter, int move,
                 double* history, void* stream);

/* Batched gradient-ascent refinement of n candidates (the gradient of Eq. Upsilon-seg
 * from tfs_grad_statistic drives the step). State, all device memory of the context's
 * device, owned by the caller: theta double [8][n] (the point just evaluated; replaced
 * by the next point), best_theta, best_grad double [8][n], best_stat double [n] (start
 * at -inf), eta double [n] (step lengths in units of sigma), sigma double [8][n]
 * (per-candidate parameter scales, 0 freezes a parameter); lo, hi: bounds of the
 * clamped parameters (M_c, eta, f_0, beta, iota; phi_0 and lambda wrap to [0, 2 pi),
 * psi to [0, pi)); eta_up, eta_down > 0. */
typedef struct tfs_refine {
  int64_t n;
  double *theta, *best_theta, *best_grad, *best_stat, *eta;
  const double* sigma;
  double lo[8], hi[8];
  double eta_up, eta_down;
} tfs_refine;

/* One refinement step from U = stat [n] and dU/dtheta = grad [8][n] (device) at theta:
 * where U >= best_stat the candidate accepts (best_* take the current values and eta
 * is multiplied by eta_up), else it rejects (eta *= eta_down); then
 *   theta = project(best_theta + eta sigma (sigma best_grad) / |sigma best_grad|).
 * mean_best: null, or a device double that receives the mean of best_stat (summed in a
 * fixed order). Asynchronous on `stream`. */
int tfs_refine_step(tfs_ctx* ctx, const tfs_refine* rf, const double* stat, const double* grad,
                    double* mean_best, void* stream);

/* Per-kernel GPU times [ms] of the last tfs_eval_statistic / tfs_grad_statistic call
 * made with options.profile = 1: ms[0] set-up, ms[1] sort, ms[2] statistic kernel,
 * ms[3] output fold/copy. Returns TFS_ERR_STATE if nothing was profiled. */
int tfs_last_profile(const tfs_ctx* ctx, double ms[4]);

/* Shape of the statistic kernel launch of the last tfs_eval_statistic call:
 * out[0] the compiled tile/schedule variant of the mixed kernel that the autotuner
 * picked (0 on the other paths), out[1] threads per CTA, out[2] CTAs launched, out[3]
 * CTAs resident per SM, out[4] SMs of the device, out[5] autotuner trials timed so far
 * by this context. TFS_ERR_STATE before the first evaluation. */
int tfs_last_launch_shape(const tfs_ctx* ctx, int32_t out[6]);

/* Kernel launches issued by the last call (for launch accounting). */
int64_t tfs_last_launch_count(const tfs_ctx* ctx);

/* Message of the last error on this context ("" if none). Never NULL. */
const char* tfs_last_error(const tfs_ctx* ctx);

/* Library version, major * 10000 + minor * 100 + patch. */
int tfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TFS_H */
