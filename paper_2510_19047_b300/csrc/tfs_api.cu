// C ABI of libtfs (declared in include/tfs.h): the context, data loading, noise
// weights, and dispatch of the evaluation paths. Host code only; the kernels live in
// tfs_setup.cu, tfs_eval_ref.cu, tfs_eval_mixed.cu, tfs_sort.cu and tfs_grad.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <string>
#include <vector>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"
#include "tfs_sort.cuh"

using namespace tfs;

namespace {

constexpr int kMixedMaxFine = 1024;  // shared-memory segment slots per warp, mixed path

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// The shape of a mixed launch: compiled variant, warps per CTA, CTAs, CTAs per SM.
struct MixedShape {
  int variant = 0, warps = 8, ctas = 1, per_sm = 1;
};

}  // namespace

struct tfs_ctx {
  int device = 0;
  int n_sm = 0;
  tfs_options opt{};
  std::string err;
  int64_t alloc_bytes = 0;
  int64_t launches = 0;
  // data
  bool has_data = false, has_weights = false;
  GridDesc g{};
  double dt = 0;
  DevBuf d_re, d_im, w_in, mask, tabD, tabF;
  DevBuf tdiF;  // per-tranche constellation geometry of the TDI transfer
  // packed pixels
  DevBuf u64, w64, u32, w32, Umix;
  DevBuf Ugrad;            // FP32 mixed-layout plane for the gradient (when Umix is not FP32)
  DevBuf gpart;            // the gradient's per-work-item partial sums (small batches)
  DevBuf gsrc;             // the gradient's table of d(template constant)/d theta
  bool ugrad_ok = false;
  int pitch = 0;
  int pix_built = -1;
  double su = 1.0, sw = 1.0;
  // per-call scratch
  DevBuf theta, tpl, tplm, perm, sortbuf, stat, neff, diag, counter, deverr, nseg, idx64, grad;
  DevBuf segZ;  // the gradient's per-segment adjoint weights (lambda, mu)
  // search steps: tile corners of the swarms, partial sums and block counter of the
  // refinement step's mean
  DevBuf tile_lo, tile_hi, rpart, rdone;
  DevBuf tune_perm;  // the autotuner's strided sample of the queue
  DevBuf live, rank;  // unmasked tranches in order; unmasked tranches before each tranche
  // harmonic content of the templates (n = 0: the dominant mode) and its per-template
  // constant phases (mixed path)
  HarmSet harm{};
  DevBuf harmK;
  // profiling
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double prof[4] = {0, 0, 0, 0};
  bool prof_valid = false;
  int mixed_warps = 0;
  // autotuned mixed launch shapes: (n_chan, pixel, fine_cap, per_template, response) ->
  // (variant, warps, CTAs per SM); trials timed so far
  std::map<std::tuple<int, int, int, int, int>, MixedShape> tuned;
  int64_t tune_trials = 0;
  // shape of the last statistic launch: variant, threads per CTA, CTAs, CTAs per SM, SMs
  int shape[5] = {0, 0, 0, 0, 0};
  // CUDA graph of the mixed evaluation, replayed while its key is unchanged
  cudaStream_t cstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<long long> gkey;
};

namespace {

int fail(tfs_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TFS_ERR_OOM : TFS_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

void buf_free(tfs_ctx* c, DevBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    c->alloc_bytes -= (int64_t)b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
}

// Grow-only device buffer with the context's allocation cap.
int buf_ensure(tfs_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return TFS_OK;
  buf_free(c, b);
  if (c->opt.max_device_bytes > 0 && c->alloc_bytes + (int64_t)bytes > c->opt.max_device_bytes)
    return fail(c, TFS_ERR_OOM,
                "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap of " +
                    std::to_string(c->opt.max_device_bytes) + " bytes");
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(c, TFS_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  b.bytes = bytes;
  c->alloc_bytes += (int64_t)bytes;
  return TFS_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself if it is device memory, else a
// copy into `tmp`.
int device_view(tfs_ctx* c, const void* src, size_t bytes, DevBuf& tmp, cudaStream_t s,
                const void** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return TFS_OK;
  }
  int r = buf_ensure(c, tmp, bytes);
  if (r) return r;
  CUDA_TRY(c, cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, s));
  *out = tmp.p;
  return TFS_OK;
}

int64_t lcm64(int64_t a, int64_t b) { return a / std::gcd(a, b) * b; }

double pow2_scale(double maxval) {
  // power of two that brings the largest value to ~2^14 (FP16 keeps 4x headroom)
  if (!(maxval > 0.0) || !std::isfinite(maxval)) return 1.0;
  return std::ldexp(1.0, 14 - (int)std::ceil(std::log2(maxval)));
}

MixConst mix_const(const GridDesc& g) {
  MixConst m;
  m.dT_hi = (float)g.dT;
  m.dT_lo = (float)(g.dT - (double)m.dT_hi);
  m.dTf = (float)g.dT;
  m.sig_k = (float)(std::sqrt(2.0) * g.df);
  m.ncomp = (float)(10.0 * g.df / g.dT);
  m.x_hi = (float)(g.n_bins - kNFHalf);
  return m;
}

int pack_mixed(tfs_ctx* c, cudaStream_t s) {
  const int pix = c->opt.pixel;
  const size_t pe = pix == TFS_PIX_F32 ? 32 : 16;
  const size_t npix = (size_t)c->g.n_bins * c->pitch;
  int r = buf_ensure(c, c->Umix, npix * pe);
  if (r) return r;
  CUDA_TRY(c, launch_pack_mixed(pix, c->g, c->pitch, (const double*)c->d_re.p,
                                (const double*)c->d_im.p, (const double*)c->w_in.p, c->su, c->sw,
                                c->Umix.p, c->n_sm, s));
  c->launches++;
  c->pix_built = pix;
  return TFS_OK;
}

int make_levels(tfs_ctx* c, const int32_t* n_seg, int n_levels, Levels* lv) {
  if (n_levels < 1 || n_levels > kMaxLevels)
    return fail(c, TFS_ERR_ARG, "n_levels must be 1..4");
  lv->n = n_levels;
  int64_t anchor = 1, fine = 0;
  for (int l = 0; l < kMaxLevels; ++l) lv->seg_len[l] = c->g.n_tranche;
  for (int l = 0; l < n_levels; ++l) {
    const int ns = n_seg[l];
    if (ns < 1) return fail(c, TFS_ERR_ARG, "N_seg must be >= 1");
    if (c->g.n_tranche % ns != 0)
      return fail(c, TFS_ERR_NSEG,
                  "N_t = " + std::to_string(c->g.n_tranche) + " is not divisible by N_seg = " +
                      std::to_string(ns));
    lv->seg_len[l] = c->g.n_tranche / ns;
    anchor = lcm64(anchor, lv->seg_len[l]);
    fine = std::gcd<int64_t>(fine, lv->seg_len[l]);
  }
  lv->anchor_len = (int)anchor;  // divides N_t since every segment length does
  lv->fine_len = (int)fine;
  lv->n_fine = c->g.n_tranche / (int)fine;
  return TFS_OK;
}

void prof_record(tfs_ctx* c, int i, cudaStream_t s) {
  if (!c->opt.profile) return;
  // inside a stream capture the record becomes an external event node, which records
  // the event each time the graph runs (so that the kernel times stay measurable)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                             : cudaEventRecordDefault;
  if (cudaEventRecordWithFlags(c->ev[i], s, flags) != cudaSuccess) cudaGetLastError();
}

// Per-kernel times of the call just synchronised; a failed query leaves the profile
// invalid and clears its error, so that no later launch check reports it.
void read_profile(tfs_ctx* c) {
  c->prof_valid = true;
  for (int i = 0; i < 4; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      c->prof_valid = false;
    }
    c->prof[i] = ms;
  }
}


// The launches of one mixed evaluation after the per-template set-up: optional
// length/frequency sort, counter reset, persistent statistic kernel.
int issue_mixed(tfs_ctx* c, EvalArgs& a, int64_t n_tpl, const MixedShape& sh, cudaStream_t s) {
  if (c->opt.sort) {
    int nl = 0;
    CUDA_TRY(c, sort_templates((const TplConst*)c->tpl.p, n_tpl, (int32_t*)c->perm.p, c->sortbuf.p,
                               c->n_sm, s, &nl));
    c->launches += nl;
    a.perm = (const int32_t*)c->perm.p;
  } else {
    a.perm = nullptr;
  }
  prof_record(c, 2, s);
  CUDA_TRY(c, cudaMemsetAsync(c->counter.p, 0, 16, s));
  CUDA_TRY(c, launch_eval_mixed(a, c->g.n_chan, c->opt.pixel, sh.variant, sh.warps, sh.ctas, s));
  c->launches += 1;
  return TFS_OK;
}

// Launch shape of the mixed kernel. With options.warps_per_cta set: that CTA size,
// options.tile_variant, as many CTAs as fit. Otherwise the autotuner's pick, timed once per
// (channels, pixel type, segment slots, per-template mode, response) on 24576 templates
// taken at a fixed stride from the current (already sorted) queue: every compiled tile/schedule
// variant (bin unroll, pixel-load lead, register target) x {4, 8} warps per CTA x
// {full, full - 1} CTAs per SM, the fastest of two runs each.
int mixed_shape(tfs_ctx* c, EvalArgs a, int64_t n_tpl, int fine_cap, int per_template,
                cudaStream_t s, MixedShape* out) {
  const int n_chan = c->g.n_chan, pix = c->opt.pixel;
  auto ctas_for = [&](int warps, int per_sm) {
    const int64_t need = (n_tpl + warps - 1) / warps;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->n_sm * per_sm, need));
  };
  if (c->opt.warps_per_cta) {
    const int v = c->opt.tile_variant;
    if (v >= mixed_variants(n_chan, c->pitch))
      return fail(c, TFS_ERR_ARG, "options.tile_variant " + std::to_string(v) +
                                      " is not compiled for this channel count and plane pitch");
    int per_sm = 0;
    CUDA_TRY(c, mixed_occupancy(n_chan, pix, c->pitch, c->opt.response, v, c->opt.warps_per_cta,
                                fine_cap, &per_sm));
    if (per_sm < 1) return fail(c, TFS_ERR_ARG, "mixed kernel does not fit on an SM with these shapes");
    out->variant = v;
    out->warps = c->opt.warps_per_cta;
    out->per_sm = per_sm;
    out->ctas = ctas_for(out->warps, per_sm);
    return TFS_OK;
  }
  const auto key = std::make_tuple(n_chan, pix, fine_cap, per_template, c->opt.response);
  auto it = c->tuned.find(key);
  if (it == c->tuned.end()) {
    // trial batch: every stride-th entry of the (longest-first) queue, so that it spans
    // the batch's whole range of track lengths
    const int64_t cnt = std::min<int64_t>(n_tpl, 24576);
    a.n_work = cnt;
    if (a.perm && cnt < n_tpl) {
      const int64_t stride = n_tpl / cnt;
      int r;
      if ((r = buf_ensure(c, c->tune_perm, (size_t)cnt * 4))) return r;
      CUDA_TRY(c, cudaMemcpy2DAsync(c->tune_perm.p, 4, a.perm, (size_t)stride * 4, 4, (size_t)cnt,
                                    cudaMemcpyDeviceToDevice, s));
      a.perm = (const int32_t*)c->tune_perm.p;
    }
    float best = 1e30f;
    MixedShape pick;
    cudaEvent_t e0 = c->ev[0], e1 = c->ev[1];
    const int nv = mixed_variants(n_chan, c->pitch);
    for (int v = 0; v < nv; ++v) {
      for (int warps : {4, 8}) {
        int occ = 0;
        CUDA_TRY(c, mixed_occupancy(n_chan, pix, c->pitch, c->opt.response, v, warps, fine_cap, &occ));
        for (int per_sm = occ; per_sm >= std::max(1, occ - 1); --per_sm) {
          const int ctas = ctas_for(warps, per_sm);
          float ms = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            CUDA_TRY(c, cudaMemsetAsync(c->counter.p, 0, 16, s));
            CUDA_TRY(c, cudaEventRecord(e0, s));
            CUDA_TRY(c, launch_eval_mixed(a, n_chan, pix, v, warps, ctas, s));
            CUDA_TRY(c, cudaEventRecord(e1, s));
            CUDA_TRY(c, cudaEventSynchronize(e1));
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
          }
          c->tune_trials++;
          if (ms < best) {
            best = ms;
            pick.variant = v;
            pick.warps = warps;
            pick.per_sm = per_sm;
          }
        }
      }
    }
    it = c->tuned.emplace(key, pick).first;
  }
  int occ = 0;
  const MixedShape& t = it->second;
  CUDA_TRY(c, mixed_occupancy(n_chan, pix, c->pitch, c->opt.response, t.variant, t.warps, fine_cap, &occ));
  out->variant = t.variant;
  out->warps = t.warps;
  out->per_sm = std::min(occ, t.per_sm);
  out->ctas = ctas_for(t.warps, out->per_sm);
  return TFS_OK;
}

}  // namespace

extern "C" {

int tfs_version(void) { return 10000; }

void tfs_default_options(tfs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->path = TFS_PATH_MIXED;
  o->pixel = TFS_PIX_F16;
  o->pn_order = 1;
  o->response = 1;
  o->checked = 0;
  o->sort = 1;
  o->warps_per_cta = 0;
  o->tile_variant = 0;
  o->use_graph = 0;
  o->profile = 0;
  o->max_device_bytes = 0;
}

static int check_options(tfs_ctx* c, const tfs_options* o) {
  if (o->path < 0 || o->path > 2) return fail(c, TFS_ERR_ARG, "options.path must be 0, 1 or 2");
  if (o->pixel < 0 || o->pixel > 4) return fail(c, TFS_ERR_ARG, "options.pixel must be 0 .. 4");
  if (o->pn_order < 0 || o->pn_order > 1) return fail(c, TFS_ERR_ARG, "options.pn_order must be 0 or 1");
  if (o->response < 0 || o->response > 2)
    return fail(c, TFS_ERR_ARG, "options.response must be 0, 1 or 2");
  if (o->warps_per_cta < 0 || o->warps_per_cta > 8 ||
      (o->warps_per_cta && (o->warps_per_cta & (o->warps_per_cta - 1))))
    return fail(c, TFS_ERR_ARG, "options.warps_per_cta must be 0 or a power of two <= 8");
  if (o->tile_variant < 0 || o->tile_variant > 2)
    return fail(c, TFS_ERR_ARG, "options.tile_variant must be 0, 1 or 2");
  if (o->max_device_bytes < 0) return fail(c, TFS_ERR_ARG, "options.max_device_bytes must be >= 0");
  return TFS_OK;
}

int tfs_create(tfs_ctx** out, int device, const tfs_options* opt) {
  if (!out) return TFS_ERR_ARG;
  *out = nullptr;
  tfs_ctx* c = new (std::nothrow) tfs_ctx();
  if (!c) return TFS_ERR_OOM;
  tfs_default_options(&c->opt);
  if (opt) {
    int r = check_options(c, opt);
    if (r) {
      delete c;
      return r;
    }
    c->opt = *opt;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete c;
    return TFS_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TFS_ERR_CUDA;
  }
  c->device = device;
  for (int i = 0; i < 5; ++i) cudaEventCreate(&c->ev[i]);
  cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking);
  *out = c;
  return TFS_OK;
}

int tfs_destroy(tfs_ctx* c) {
  if (!c) return TFS_OK;
  cudaSetDevice(c->device);
  DevBuf* all[] = {&c->d_re, &c->d_im, &c->w_in, &c->mask, &c->tabD, &c->tabF, &c->tdiF, &c->u64,
                   &c->w64, &c->u32, &c->w32, &c->Umix, &c->theta, &c->tpl, &c->tplm,
                   &c->perm, &c->sortbuf, &c->stat, &c->neff, &c->diag, &c->counter,
                   &c->deverr, &c->nseg, &c->idx64, &c->grad, &c->segZ, &c->Ugrad, &c->gpart, &c->gsrc,
                   &c->harmK, &c->tile_lo, &c->tile_hi, &c->rpart, &c->rdone, &c->tune_perm,
                   &c->live, &c->rank};
  for (DevBuf* b : all) buf_free(c, *b);
  for (int i = 0; i < 5; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  delete c;
  return TFS_OK;
}

int tfs_set_options(tfs_ctx* c, const tfs_options* o) {
  if (!c || !o) return TFS_ERR_ARG;
  int r = check_options(c, o);
  if (r) return r;
  c->opt = *o;
  c->mixed_warps = 0;
  return TFS_OK;
}

int tfs_get_options(const tfs_ctx* c, tfs_options* o) {
  if (!c || !o) return TFS_ERR_ARG;
  *o = c->opt;
  return TFS_OK;
}

int tfs_set_harmonics(tfs_ctx* c, int n_harm, const double* nu, const double* c_re,
                      const double* c_im) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (n_harm < 0 || n_harm > TFS_MAX_HARMONICS)
    return fail(c, TFS_ERR_ARG, "n_harm must be in [0, " + std::to_string(TFS_MAX_HARMONICS) + "]");
  if (n_harm > 0 && (!nu || !c_re || !c_im)) return fail(c, TFS_ERR_ARG, "null argument");
  if (n_harm > 0 && (is_device_ptr(nu) || is_device_ptr(c_re) || is_device_ptr(c_im)))
    return fail(c, TFS_ERR_ARG, "harmonics must be given in host memory");
  HarmSet h{};
  h.n = n_harm;
  h.dnu_min = 0.f;
  for (int i = 0; i < n_harm; ++i) {
    if (!(nu[i] > 0.0 && nu[i] <= 16.0)) return fail(c, TFS_ERR_ARG, "nu must be in (0, 16]");
    if (!std::isfinite(c_re[i]) || !std::isfinite(c_im[i]))
      return fail(c, TFS_ERR_ARG, "harmonic amplitudes must be finite");
    h.nu[i] = nu[i];
    h.cr[i] = c_re[i];
    h.ci[i] = c_im[i];
    h.nu_hi[i] = (float)nu[i];
    h.nu_lo[i] = (float)(nu[i] - (double)h.nu_hi[i]);
    h.crf[i] = (float)c_re[i];
    h.cif[i] = (float)c_im[i];
  }
  double dmin = 0.0;
  for (int i = 0; i < n_harm; ++i)
    for (int j = i + 1; j < n_harm; ++j) {
      const double d = std::fabs(nu[i] - nu[j]);
      if (dmin == 0.0 || d < dmin) dmin = d;
      if (d == 0.0) dmin = -1.0;  // equal nu: the windows always coincide
    }
  // windows of two harmonics can share bins only below f/df = 21 / dnu_min; equal nu
  // (always) is a tiny positive value
  h.dnu_min = dmin < 0.0 ? 1e-30f : (float)dmin;
  c->harm = h;
  return TFS_OK;
}

const char* tfs_last_error(const tfs_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t tfs_last_launch_count(const tfs_ctx* c) { return c ? c->launches : -1; }

int tfs_last_profile(const tfs_ctx* c, double ms[4]) {
  if (!c || !ms) return TFS_ERR_ARG;
  if (!c->prof_valid) return TFS_ERR_STATE;
  for (int i = 0; i < 4; ++i) ms[i] = c->prof[i];
  return TFS_OK;
}

int tfs_load_tf_data(tfs_ctx* c, int n_chan, int n_tranche, int n_bins, double dt, double dT,
                     double t0, const double* d_re, const double* d_im) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (n_chan < 1 || n_chan > 2) return fail(c, TFS_ERR_ARG, "n_chan must be 1 or 2");
  if (n_tranche < 1 || n_tranche > 65535)
    return fail(c, TFS_ERR_ARG, "n_tranche must be in [1, 65535]");
  if (n_bins < 2 * kNFHalf + 2 || n_bins > (1 << 21))
    return fail(c, TFS_ERR_ARG, "n_bins must be in [22, 2^21]");
  if (!(dT > 0.0) || !(dt > 0.0) || !std::isfinite(dT) || !std::isfinite(t0))
    return fail(c, TFS_ERR_ARG, "dt and dT must be positive and finite");
  if (dT / dt + 1e-9 < 2.0 * n_bins)
    return fail(c, TFS_ERR_ARG, "n_bins exceeds dT / (2 dt) (bins above the Nyquist frequency)");
  if (!d_re || !d_im) return fail(c, TFS_ERR_ARG, "d_re and d_im must not be null");
  CUDA_TRY(c, cudaSetDevice(c->device));
  c->has_data = c->has_weights = false;
  c->g.n_chan = n_chan;
  c->g.n_tranche = n_tranche;
  c->g.n_bins = n_bins;
  c->g.dT = dT;
  c->g.df = 1.0 / dT;
  c->g.t0 = t0;
  c->dt = dt;
  // the mixed plane's m-pitch: the kernel's compile-time pitch when the grid fits it
  c->pitch = n_tranche <= kMixedPitch ? kMixedPitch : (n_tranche + 31) / 32 * 32;
  const size_t n = (size_t)n_chan * n_tranche * n_bins;
  int r;
  if ((r = buf_ensure(c, c->d_re, n * 8)) || (r = buf_ensure(c, c->d_im, n * 8)) ||
      (r = buf_ensure(c, c->tabD, (size_t)n_tranche * sizeof(TrancheD))) ||
      (r = buf_ensure(c, c->tabF, (size_t)n_tranche * sizeof(TrancheF))) ||
      (r = buf_ensure(c, c->tdiF, (size_t)n_tranche * 7 * sizeof(float4))))
    return r;
  const cudaMemcpyKind k1 = is_device_ptr(d_re) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind k2 = is_device_ptr(d_im) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(c, cudaMemcpy(c->d_re.p, d_re, n * 8, k1));
  CUDA_TRY(c, cudaMemcpy(c->d_im.p, d_im, n * 8, k2));
  CUDA_TRY(c, launch_tranche_table(c->g, (TrancheD*)c->tabD.p, (TrancheF*)c->tabF.p,
                                   (float4*)c->tdiF.p, 0));
  c->launches = 1;
  CUDA_TRY(c, cudaDeviceSynchronize());
  c->has_data = true;
  return TFS_OK;
}

static int pack_all(tfs_ctx* c);

int tfs_set_noise_weights(tfs_ctx* c, const double* inv_psd, const uint8_t* tranche_mask) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (!c->has_data) return fail(c, TFS_ERR_STATE, "load_tf_data must be called first");
  if (!inv_psd) return fail(c, TFS_ERR_ARG, "inv_psd must not be null");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const size_t n = (size_t)c->g.n_chan * c->g.n_tranche * c->g.n_bins;
  int r;
  if ((r = buf_ensure(c, c->w_in, n * 8)) || (r = buf_ensure(c, c->mask, c->g.n_tranche)) ||
      (r = buf_ensure(c, c->u64, n * 16)) || (r = buf_ensure(c, c->w64, n * 8)) ||
      (r = buf_ensure(c, c->u32, n * 8)) || (r = buf_ensure(c, c->w32, n * 4)) ||
      (r = buf_ensure(c, c->counter, 64)))
    return r;
  CUDA_TRY(c, cudaMemcpy(c->w_in.p, inv_psd, n * 8,
                         is_device_ptr(inv_psd) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  if (tranche_mask) {
    CUDA_TRY(c, cudaMemcpy(c->mask.p, tranche_mask, c->g.n_tranche,
                           is_device_ptr(tranche_mask) ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice));
  } else {
    CUDA_TRY(c, cudaMemset(c->mask.p, 1, c->g.n_tranche));
  }
  // the unmasked tranches in order, and for each tranche the count of unmasked ones
  // before it: the mixed kernel walks a template's range over these only, so that no
  // lane of a warp idles on a gap
  {
    const int nt = c->g.n_tranche;
    std::vector<uint8_t> hmask(nt);
    CUDA_TRY(c, cudaMemcpy(hmask.data(), c->mask.p, nt, cudaMemcpyDeviceToHost));
    std::vector<int32_t> live, rank(nt + 1);
    for (int m = 0; m < nt; ++m) {
      rank[m] = (int32_t)live.size();
      if (hmask[m]) live.push_back(m);
    }
    rank[nt] = (int32_t)live.size();
    if ((r = buf_ensure(c, c->live, std::max<size_t>(live.size(), 1) * 4)) ||
        (r = buf_ensure(c, c->rank, (size_t)(nt + 1) * 4)))
      return r;
    if (!live.empty())
      CUDA_TRY(c, cudaMemcpy(c->live.p, live.data(), live.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->rank.p, rank.data(), (size_t)(nt + 1) * 4, cudaMemcpyHostToDevice));
  }
  c->has_weights = false;
  if ((r = pack_all(c))) return r;
  c->has_weights = true;
  return TFS_OK;
}

// Validates the data under the weights, finds the storage scales and forms u = d~ w and
// w in every storage the paths use (synchronous).
static int pack_all(tfs_ctx* c) {
  const size_t n = (size_t)c->g.n_chan * c->g.n_tranche * c->g.n_bins;
  int r;
  // validate and find the ranges of u = d w and w
  unsigned long long* mx = (unsigned long long*)c->counter.p;
  int* bad = (int*)((char*)c->counter.p + 16);
  CUDA_TRY(c, cudaMemset(c->counter.p, 0, 64));
  CUDA_TRY(c, launch_absmax((int64_t)n, (const double*)c->d_re.p, (const double*)c->d_im.p,
                            (const double*)c->w_in.p, mx, mx + 1, bad, c->n_sm, 0));
  unsigned long long hm[2];
  int hbad = 0;
  CUDA_TRY(c, cudaMemcpy(hm, mx, 16, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(&hbad, bad, 4, cudaMemcpyDeviceToHost));
  c->launches = 1;
  if (hbad)
    return fail(c, TFS_ERR_ARG,
                std::to_string(hbad) +
                    " pixels have a negative or non-finite weight, or non-finite data under a "
                    "positive weight");
  double umax, wmax;
  std::memcpy(&umax, &hm[0], 8);
  std::memcpy(&wmax, &hm[1], 8);
  c->su = pow2_scale(umax);
  c->sw = pow2_scale(wmax);
  CUDA_TRY(c, launch_pack_ref((int64_t)n, (const double*)c->d_re.p, (const double*)c->d_im.p,
                              (const double*)c->w_in.p, c->su, c->sw, (double2*)c->u64.p,
                              (double*)c->w64.p, (float2*)c->u32.p, (float*)c->w32.p, c->n_sm, 0));
  r = pack_mixed(c, 0);
  if (r) return r;
  c->ugrad_ok = false;
  CUDA_TRY(c, cudaDeviceSynchronize());
  return TFS_OK;
}

int tfs_noise_realisation(tfs_ctx* c, uint64_t seed) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (!c->has_data || !c->has_weights)
    return fail(c, TFS_ERR_STATE, "load_tf_data and set_noise_weights must be called first");
  CUDA_TRY(c, cudaSetDevice(c->device));
  cudaGetLastError();
  const int64_t n = (int64_t)c->g.n_chan * c->g.n_tranche * c->g.n_bins;
  CUDA_TRY(c, launch_noise(n, (const double*)c->w_in.p, c->g.df, seed, (double*)c->d_re.p,
                           (double*)c->d_im.p, c->n_sm, 0));
  c->has_weights = false;
  int r = pack_all(c);
  if (r) return r;
  c->launches += 1;
  c->has_weights = true;
  return TFS_OK;
}

static int eval_impl(tfs_ctx* c, const double* theta, int64_t n_tpl, const int32_t* n_seg,
                     int n_levels, int per_template, double* out_stat, int32_t* out_neff,
                     int32_t* out_diag, cudaStream_t s) {
  const GridDesc& g = c->g;
  Levels lv{};
  int r;
  int fine_cap = 0;
  const int32_t* nseg_dev = nullptr;
  if (!per_template) {
    if (!n_seg) return fail(c, TFS_ERR_ARG, "n_seg must not be null");
    int32_t hs[kMaxLevels] = {0, 0, 0, 0};
    if (n_levels < 1 || n_levels > kMaxLevels) return fail(c, TFS_ERR_ARG, "n_levels must be 1..4");
    if (is_device_ptr(n_seg)) {
      CUDA_TRY(c, cudaMemcpy(hs, n_seg, n_levels * 4, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(hs, n_seg, n_levels * 4);
    }
    if ((r = make_levels(c, hs, n_levels, &lv))) return r;
    fine_cap = lv.n_fine;
  } else {
    n_levels = 1;
    std::vector<int32_t> hs(n_tpl > 0 ? n_tpl : 1);
    if (n_tpl > 0) {
      if (!n_seg) return fail(c, TFS_ERR_ARG, "n_seg must not be null");
      CUDA_TRY(c, cudaMemcpy(hs.data(), n_seg, n_tpl * 4,
                             is_device_ptr(n_seg) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    }
    int mx = 1;
    for (int64_t i = 0; i < n_tpl; ++i) {
      if (hs[i] < 1) return fail(c, TFS_ERR_ARG, "N_seg must be >= 1");
      if (g.n_tranche % hs[i] != 0)
        return fail(c, TFS_ERR_NSEG, "N_t = " + std::to_string(g.n_tranche) +
                                         " is not divisible by N_seg = " + std::to_string(hs[i]));
      mx = std::max(mx, (int)hs[i]);
    }
    lv.n = 0;
    fine_cap = mx;
    if ((r = buf_ensure(c, c->nseg, (size_t)std::max<int64_t>(n_tpl, 1) * 4))) return r;
    if (n_tpl > 0)
      CUDA_TRY(c, cudaMemcpyAsync(c->nseg.p, hs.data(), n_tpl * 4, cudaMemcpyHostToDevice, s));
    nseg_dev = (const int32_t*)c->nseg.p;
  }
  const int path = c->opt.path;
  if (path == TFS_PATH_MIXED && fine_cap > kMixedMaxFine)
    return fail(c, TFS_ERR_ARG,
                "the mixed path folds at most 1024 finest segments per template (N_t / gcd of "
                "segment lengths); use the plain or FP64 path for finer segmentations");
  c->launches = 0;
  c->prof_valid = false;
  if (n_tpl == 0) return TFS_OK;
  const bool harm = c->harm.n > 0;
  const bool graph = path == TFS_PATH_MIXED && c->opt.use_graph && !harm;
  // inputs: device theta is read in place, host theta is copied; a graph always reads
  // the context's own copy so that its pointers stay fixed between replays
  const void* th = nullptr;
  if (graph) {
    if ((r = buf_ensure(c, c->theta, (size_t)n_tpl * 64))) return r;
    CUDA_TRY(c, cudaMemcpyAsync(c->theta.p, theta, (size_t)n_tpl * 64,
                                is_device_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                s));
    th = c->theta.p;
  } else if ((r = device_view(c, theta, (size_t)n_tpl * 8 * 8, c->theta, s, &th))) {
    return r;
  }
  if ((r = buf_ensure(c, c->tpl, (size_t)n_tpl * sizeof(TplConst)))) return r;
  // outputs: device pointers are written directly, host ones (and graph replays) go
  // through the context's scratch
  const bool dev_stat = !graph && is_device_ptr(out_stat);
  const bool dev_neff = !graph && (!out_neff || is_device_ptr(out_neff));
  const bool dev_diag = !graph && (!out_diag || is_device_ptr(out_diag));
  double* o_stat = out_stat;
  int32_t* o_neff = out_neff;
  int32_t* o_diag = out_diag;
  if (!dev_stat) {
    if ((r = buf_ensure(c, c->stat, (size_t)n_levels * n_tpl * 8))) return r;
    o_stat = (double*)c->stat.p;
  }
  if (!dev_neff) {
    if ((r = buf_ensure(c, c->neff, (size_t)n_levels * n_tpl * 4))) return r;
    o_neff = (int32_t*)c->neff.p;
  }
  if (!dev_diag) {
    if ((r = buf_ensure(c, c->diag, (size_t)2 * n_tpl * 4))) return r;
    o_diag = (int32_t*)c->diag.p;
  }
  if ((r = buf_ensure(c, c->counter, 64))) return r;
  TplMix* mix = nullptr;
  if (path == TFS_PATH_MIXED) {
    if ((r = buf_ensure(c, c->tplm, (size_t)n_tpl * sizeof(TplMix)))) return r;
    mix = (TplMix*)c->tplm.p;
    if (c->pix_built != c->opt.pixel && (r = pack_mixed(c, s))) return r;
    if (c->opt.sort && ((r = buf_ensure(c, c->perm, (size_t)n_tpl * 4)) ||
                        (r = buf_ensure(c, c->sortbuf, sort_scratch_bytes(n_tpl)))))
      return r;
  }

  EvalArgs a{};
  a.g = g;
  a.mc = mix_const(g);
  a.response = c->opt.response;
  a.pitch = c->pitch;
  a.tabD = (const TrancheD*)c->tabD.p;
  a.tabF = (const TrancheF*)c->tabF.p;
  a.tdiF = (const float4*)c->tdiF.p;
  a.u64 = (const double2*)c->u64.p;
  a.w64 = (const double*)c->w64.p;
  a.u32 = (const float2*)c->u32.p;
  a.w32 = (const float*)c->w32.p;
  a.Umix = c->Umix.p;
  a.mask = (const uint8_t*)c->mask.p;
  a.live = (const int32_t*)c->live.p;
  a.rank = (const int32_t*)c->rank.p;
  a.tpl = (const TplConst*)c->tpl.p;
  a.tplm = mix;
  a.perm = nullptr;
  a.n_tpl = n_tpl;
  a.n_work = n_tpl;
  a.lv = lv;
  a.nseg_pt = nseg_dev;
  a.fine_cap = fine_cap;
  a.out_stat = o_stat;
  a.out_neff = o_neff;
  a.out_diag = o_diag;
  a.counter = (int*)c->counter.p;
  a.dev_err = (int*)c->counter.p + 8;
  a.checked = c->opt.checked;
  a.out_scale = path == TFS_PATH_FP64 ? 4.0 * g.df : 4.0 * g.df * c->sw / (c->su * c->su);
  a.harm = c->harm;
  a.harm_K = nullptr;

  double nu_min = 1.0, nu_max = 1.0;
  if (harm) {
    nu_min = nu_max = c->harm.nu[0];
    for (int h = 1; h < c->harm.n; ++h) {
      nu_min = std::min(nu_min, c->harm.nu[h]);
      nu_max = std::max(nu_max, c->harm.nu[h]);
    }
  }
  auto setup = [&](cudaStream_t st) -> int {
    prof_record(c, 0, st);
    CUDA_TRY(c, launch_setup((const double*)th, n_tpl, c->opt.pn_order, g, (TplConst*)c->tpl.p, mix, st,
                             nu_min, nu_max));
    c->launches++;
    prof_record(c, 1, st);
    return TFS_OK;
  };

  if (c->opt.checked) {
    // range check of the per-template constants before any kernel reads pixels
    if ((r = setup(s))) return r;
    CUDA_TRY(c, cudaMemsetAsync(a.dev_err, 0, 4, s));
    CUDA_TRY(c, launch_check_tpl((const TplConst*)c->tpl.p, n_tpl, g.n_tranche, a.dev_err, s));
    int herr = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&herr, a.dev_err, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (herr) return fail(c, TFS_ERR_DEVICE_CHECK, "a template's tranche range lies outside the grid");
  }

  if (path == TFS_PATH_MIXED && harm && c->opt.pixel > TFS_PIX_BF16)
    return fail(c, TFS_ERR_ARG, "the precision-study pixel types (3, 4) are not available with harmonics");
  if (path == TFS_PATH_MIXED && harm) {
    // multi-harmonic mixed launch: set-up, constant phases per harmonic, sort, kernel
    if ((r = buf_ensure(c, c->harmK, (size_t)n_tpl * c->harm.n * sizeof(float2)))) return r;
    if (!c->opt.checked && (r = setup(s))) return r;
    CUDA_TRY(c, launch_harm_phase((const TplConst*)c->tpl.p, n_tpl, c->harm, (float2*)c->harmK.p, s));
    c->launches += 1;
    a.harm_K = (const float2*)c->harmK.p;
    if (c->opt.sort) {
      int nl = 0;
      CUDA_TRY(c, sort_templates((const TplConst*)c->tpl.p, n_tpl, (int32_t*)c->perm.p, c->sortbuf.p,
                                 c->n_sm, s, &nl));
      c->launches += nl;
      a.perm = (const int32_t*)c->perm.p;
    }
    prof_record(c, 2, s);
    CUDA_TRY(c, cudaMemsetAsync(c->counter.p, 0, 16, s));
    int hs[3] = {0, 0, 0};
    CUDA_TRY(c, launch_eval_harm(a, g.n_chan, c->opt.pixel, c->n_sm, s, hs));
    c->launches += 1;
    c->shape[0] = 0;
    c->shape[1] = hs[0];
    c->shape[2] = hs[1];
    c->shape[3] = hs[2];
  } else if (path == TFS_PATH_MIXED) {
    MixedShape sh;
    const bool must_time = !c->opt.warps_per_cta &&
                           !c->tuned.count(std::make_tuple(g.n_chan, c->opt.pixel, fine_cap, per_template,
                                                           c->opt.response));
    // the direct launch needs the set-up first; a graph replays its own set-up, so it
    // runs eagerly only when the autotuner times the kernel on this batch
    if (!c->opt.checked && (!graph || must_time) && (r = setup(s))) return r;
    if (c->opt.sort && must_time) {
      // the autotuner times the sorted queue, so sort once before choosing
      EvalArgs t = a;
      int nl = 0;
      CUDA_TRY(c, sort_templates((const TplConst*)c->tpl.p, n_tpl, (int32_t*)c->perm.p, c->sortbuf.p,
                                 c->n_sm, s, &nl));
      t.perm = (const int32_t*)c->perm.p;
      if ((r = mixed_shape(c, t, n_tpl, fine_cap, per_template, s, &sh))) return r;
    } else if ((r = mixed_shape(c, a, n_tpl, fine_cap, per_template, s, &sh))) {
      return r;
    }
    c->shape[0] = sh.variant;
    c->shape[1] = sh.warps * 32;
    c->shape[2] = sh.ctas;
    c->shape[3] = sh.per_sm;
    c->launches = 0;
    if (!graph) {
      c->launches = 1;  // set-up
      if ((r = issue_mixed(c, a, n_tpl, sh, s))) return r;
    } else {
      std::vector<long long> key = {n_tpl, n_levels, per_template, fine_cap, sh.variant, sh.warps, sh.ctas,
                                    c->opt.pixel, c->opt.sort, c->opt.profile, c->opt.pn_order,
                                    c->opt.response, (long long)th, (long long)o_stat,
                                    (long long)o_neff, (long long)o_diag, (long long)c->tpl.p,
                                    (long long)c->tplm.p, (long long)c->perm.p,
                                    (long long)c->sortbuf.p, (long long)c->Umix.p,
                                    (long long)c->nseg.p, lv.seg_len[0], lv.seg_len[1],
                                    lv.seg_len[2], lv.seg_len[3]};
      if (!c->gexec || key != c->gkey) {
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
        cudaGraph_t gr = nullptr;
        CUDA_TRY(c, cudaStreamBeginCapture(c->cstream, cudaStreamCaptureModeThreadLocal));
        int rr = setup(c->cstream);
        if (!rr) rr = issue_mixed(c, a, n_tpl, sh, c->cstream);
        prof_record(c, 3, c->cstream);
        const cudaError_t ce = cudaStreamEndCapture(c->cstream, &gr);
        if (rr) {
          if (gr) cudaGraphDestroy(gr);
          return rr;
        }
        CUDA_TRY(c, ce);
        const cudaError_t ie = cudaGraphInstantiate(&c->gexec, gr, 0);
        cudaGraphDestroy(gr);
        CUDA_TRY(c, ie);
        c->gkey = key;
      }
      // the replay follows the work already queued on the caller's stream
      CUDA_TRY(c, cudaGraphLaunch(c->gexec, s));
      c->launches = 1 + (c->opt.sort ? 1 + 4 * 3 : 0) + 1;
    }
  } else {
    if (!c->opt.checked && (r = setup(s))) return r;
    prof_record(c, 2, s);
    CUDA_TRY(c, path == TFS_PATH_PLAIN ? launch_eval_plain(a, s) : launch_eval_fp64(a, s));
    c->launches += 1;
    int per_sm = 0;
    CUDA_TRY(c, ref_occupancy(a, path, &per_sm));
    c->shape[0] = 0;
    c->shape[1] = 128;
    c->shape[2] = (int)((n_tpl + 127) / 128);
    c->shape[3] = per_sm;
  }
  if (!graph) prof_record(c, 3, s);
  if (!dev_stat)
    CUDA_TRY(c, cudaMemcpyAsync(out_stat, o_stat, (size_t)n_levels * n_tpl * 8,
                                is_device_ptr(out_stat) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!dev_neff && out_neff)
    CUDA_TRY(c, cudaMemcpyAsync(out_neff, o_neff, (size_t)n_levels * n_tpl * 4,
                                is_device_ptr(out_neff) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!dev_diag && out_diag)
    CUDA_TRY(c, cudaMemcpyAsync(out_diag, o_diag, (size_t)2 * n_tpl * 4,
                                is_device_ptr(out_diag) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  prof_record(c, 4, s);
  const bool host_out = !is_device_ptr(out_stat) || (out_neff && !is_device_ptr(out_neff)) ||
                        (out_diag && !is_device_ptr(out_diag));
  if (host_out || c->opt.profile) CUDA_TRY(c, cudaStreamSynchronize(s));
  if (c->opt.profile) read_profile(c);
  return TFS_OK;
}

int tfs_eval_statistic(tfs_ctx* c, const double* theta, int64_t n_tpl, const int32_t* n_seg,
                       int n_levels, int per_template, double* out_stat, int32_t* out_neff,
                       int32_t* out_diag, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (!c->has_data || !c->has_weights)
    return fail(c, TFS_ERR_STATE, "load_tf_data and set_noise_weights must be called first");
  if (n_tpl < 0 || n_tpl > INT32_MAX) return fail(c, TFS_ERR_ARG, "n_tpl must be in [0, 2^31)");
  if (n_tpl > 0 && (!theta || !out_stat))
    return fail(c, TFS_ERR_ARG, "theta and out_stat must not be null");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaGetLastError();  // a launch check below must not report an earlier, unrelated error
  return eval_impl(c, theta, n_tpl, n_seg, n_levels, per_template, out_stat, out_neff, out_diag,
                   (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Ladder selection and gradient-ascent step
// ---------------------------------------------------------------------------------
extern "C" {

int tfs_last_launch_shape(const tfs_ctx* c, int32_t out[6]) {
  if (!c || !out) return TFS_ERR_ARG;
  if (!c->shape[1]) return TFS_ERR_STATE;
  for (int i = 0; i < 4; ++i) out[i] = c->shape[i];
  out[4] = c->n_sm;
  out[5] = (int32_t)std::min<int64_t>(c->tune_trials, INT32_MAX);
  return TFS_OK;
}

int tfs_select_top(tfs_ctx* c, const double* stat, int64_t n, int64_t k, int64_t* out_index,
                   void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (n < 0 || n > INT32_MAX || k < 0 || k > n) return fail(c, TFS_ERR_ARG, "need 0 <= k <= n < 2^31");
  if (k == 0) return TFS_OK;
  if (!stat || !out_index) return fail(c, TFS_ERR_ARG, "stat and out_index must not be null");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  c->launches = 0;
  int r;
  const void* sv = nullptr;
  if ((r = device_view(c, stat, (size_t)n * 8, c->stat, s, &sv))) return r;
  if ((r = buf_ensure(c, c->sortbuf, topk_scratch_bytes(n)))) return r;
  const bool dev_out = is_device_ptr(out_index);
  int64_t* o = out_index;
  if (!dev_out) {
    if ((r = buf_ensure(c, c->idx64, (size_t)k * 8))) return r;
    o = (int64_t*)c->idx64.p;
  }
  int nl = 0;
  CUDA_TRY(c, select_top((const double*)sv, n, k, o, c->sortbuf.p, s, &nl));
  c->launches += nl;
  if (!dev_out) {
    CUDA_TRY(c, cudaMemcpyAsync(out_index, o, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
  }
  return TFS_OK;
}

int tfs_ascent_step(tfs_ctx* c, double* theta, const double* grad, int64_t n, const double* step,
                    const double* lo, const double* hi, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (n < 0) return fail(c, TFS_ERR_ARG, "n must be >= 0");
  if (n == 0) return TFS_OK;
  if (!theta || !grad || !step || !lo || !hi) return fail(c, TFS_ERR_ARG, "null argument");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  AscentParams p;
  for (int i = 0; i < 8; ++i) {
    p.step[i] = step[i];
    p.lo[i] = lo[i];
    p.hi[i] = hi[i];
  }
  int r;
  const bool dev_theta = is_device_ptr(theta);
  double* th = theta;
  if (!dev_theta) {
    if ((r = buf_ensure(c, c->theta, (size_t)n * 64))) return r;
    th = (double*)c->theta.p;
    CUDA_TRY(c, cudaMemcpyAsync(th, theta, (size_t)n * 64, cudaMemcpyHostToDevice, s));
  }
  const void* gv = nullptr;
  if ((r = device_view(c, grad, (size_t)n * 64, c->grad, s, &gv))) return r;
  c->launches = 0;
  CUDA_TRY(c, launch_ascent(th, (const double*)gv, n, p, s));
  c->launches = 1;
  if (!dev_theta) {
    CUDA_TRY(c, cudaMemcpyAsync(theta, th, (size_t)n * 64, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
  }
  return TFS_OK;
}

int tfs_grad_statistic(tfs_ctx* c, const double* theta, int64_t n_tpl, int32_t n_seg,
                       double* out_stat, double* out_grad, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (!c->has_data || !c->has_weights)
    return fail(c, TFS_ERR_STATE, "load_tf_data and set_noise_weights must be called first");
  if (n_tpl < 0 || n_tpl > INT32_MAX) return fail(c, TFS_ERR_ARG, "n_tpl must be in [0, 2^31)");
  if (n_seg < 1) return fail(c, TFS_ERR_ARG, "N_seg must be >= 1");
  if (c->g.n_tranche % n_seg != 0)
    return fail(c, TFS_ERR_NSEG, "N_t = " + std::to_string(c->g.n_tranche) +
                                     " is not divisible by N_seg = " + std::to_string(n_seg));
  if (n_seg > kMixedMaxFine) return fail(c, TFS_ERR_ARG, "the gradient kernel supports N_seg <= 1024");
  if (c->harm.n > 0)
    return fail(c, TFS_ERR_ARG, "the gradient supports the dominant mode only (n_harm = 0)");
  if (n_tpl == 0) return TFS_OK;
  if (!theta || !out_stat || !out_grad) return fail(c, TFS_ERR_ARG, "null argument");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaGetLastError();  // a launch check below must not report an earlier, unrelated error
  cudaStream_t s = (cudaStream_t)stream;
  int r;
  const void* th = nullptr;
  if ((r = device_view(c, theta, (size_t)n_tpl * 64, c->theta, s, &th))) return r;
  if ((r = buf_ensure(c, c->tpl, (size_t)n_tpl * sizeof(TplConst)))) return r;
  if ((r = buf_ensure(c, c->tplm, (size_t)n_tpl * sizeof(TplMix)))) return r;
  if ((r = buf_ensure(c, c->counter, 64))) return r;
  if (c->opt.sort && ((r = buf_ensure(c, c->perm, (size_t)n_tpl * 4)) ||
                      (r = buf_ensure(c, c->sortbuf, sort_scratch_bytes(n_tpl)))))
    return r;
  // the FP32 pixel plane: the mixed plane itself when it is FP32, else a copy packed once
  // per set of noise weights
  const void* plane = c->Umix.p;
  if (c->pix_built != TFS_PIX_F32) {
    if (!c->ugrad_ok) {
      const size_t npix = (size_t)c->g.n_bins * c->pitch;
      if ((r = buf_ensure(c, c->Ugrad, npix * 32))) return r;
      CUDA_TRY(c, launch_pack_mixed(TFS_PIX_F32, c->g, c->pitch, (const double*)c->d_re.p,
                                    (const double*)c->d_im.p, (const double*)c->w_in.p, c->su,
                                    c->sw, c->Ugrad.p, c->n_sm, s));
      c->ugrad_ok = true;
    }
    plane = c->Ugrad.p;
  }
  const bool dev_stat = is_device_ptr(out_stat), dev_grad = is_device_ptr(out_grad);
  double* os = out_stat;
  double* og = out_grad;
  if (!dev_stat) {
    if ((r = buf_ensure(c, c->stat, (size_t)n_tpl * 8))) return r;
    os = (double*)c->stat.p;
  }
  if (!dev_grad) {
    if ((r = buf_ensure(c, c->grad, (size_t)n_tpl * 64))) return r;
    og = (double*)c->grad.p;
  }
  c->launches = 0;
  prof_record(c, 0, s);
  CUDA_TRY(c, launch_setup((const double*)th, n_tpl, c->opt.pn_order, c->g, (TplConst*)c->tpl.p,
                           (TplMix*)c->tplm.p, s));
  prof_record(c, 1, s);
  c->launches = 1;
  // longest templates first, as for the statistic kernel's queue
  const int32_t* perm = nullptr;
  if (c->opt.sort) {
    int nl = 0;
    CUDA_TRY(c, sort_templates((const TplConst*)c->tpl.p, n_tpl, (int32_t*)c->perm.p, c->sortbuf.p,
                               c->n_sm, s, &nl));
    c->launches += nl;
    perm = (const int32_t*)c->perm.p;
  }
  prof_record(c, 2, s);
  const double scale = 4.0 * c->g.df * c->sw / (c->su * c->su);
  int parts = 1, parts_a = 1;
  CUDA_TRY(c, grad_plan(c->opt.response, n_seg, c->n_sm, n_tpl, &parts, &parts_a));
  const int parts_max = std::max(parts, parts_a);
  if (parts_max > 1 && (r = buf_ensure(c, c->gpart, (size_t)parts_max * 9 * n_tpl * 8))) return r;
  if ((r = buf_ensure(c, c->gsrc, grad_src_bytes(n_tpl)))) return r;
  if ((r = buf_ensure(c, c->segZ, (size_t)n_tpl * n_seg * 16))) return r;
  CUDA_TRY(c, launch_grad(c->g, mix_const(c->g), c->opt.response, c->opt.pn_order, c->pitch,
                          (const TrancheF*)c->tabF.p, (const float4*)plane,
                          (const uint8_t*)c->mask.p, (const double*)th, (const TplConst*)c->tpl.p,
                          (const TplMix*)c->tplm.p, n_tpl, n_seg, scale, os, og,
                          (unsigned*)c->counter.p, perm, parts, parts_a, (double*)c->gpart.p,
                          (double*)c->gsrc.p, (float4*)c->segZ.p, c->n_sm, s));
  c->launches += parts_max > 1 ? 4 : 3;
  prof_record(c, 3, s);
  if (!dev_stat) CUDA_TRY(c, cudaMemcpyAsync(out_stat, os, (size_t)n_tpl * 8, cudaMemcpyDeviceToHost, s));
  if (!dev_grad) CUDA_TRY(c, cudaMemcpyAsync(out_grad, og, (size_t)n_tpl * 64, cudaMemcpyDeviceToHost, s));
  prof_record(c, 4, s);
  if (!dev_stat || !dev_grad || c->opt.profile) CUDA_TRY(c, cudaStreamSynchronize(s));
  if (c->opt.profile) read_profile(c);
  return TFS_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------------
// Search steps: particle swarm and refinement bookkeeping
// ---------------------------------------------------------------------------------
namespace {

// Device pointer of the context's device (the search-step calls take device state only).
bool on_ctx_device(const tfs_ctx* c, const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == c->device;
}

int pso_args(tfs_ctx* c, const tfs_swarm* sw, cudaStream_t s, PsoArgs* a) {
  if (!sw) return fail(c, TFS_ERR_ARG, "null swarm");
  if (sw->n_swarm < 1 || sw->n_part < 1 || (int64_t)sw->n_swarm * sw->n_part > INT32_MAX)
    return fail(c, TFS_ERR_ARG, "need n_swarm >= 1, n_part >= 1, n_swarm * n_part < 2^31");
  if (!sw->lo || !sw->hi) return fail(c, TFS_ERR_ARG, "null tile corners");
  double* st[6] = {sw->x, sw->v, sw->pbest, sw->pval, sw->gbest, sw->gval};
  for (double* p : st)
    if (!on_ctx_device(c, p))
      return fail(c, TFS_ERR_ARG, "swarm state must be device memory of the context's device");
  if (!(std::isfinite(sw->inertia) && std::isfinite(sw->c1) && std::isfinite(sw->c2)))
    return fail(c, TFS_ERR_ARG, "inertia, c1, c2 must be finite");
  const size_t nb = (size_t)sw->n_swarm * 8 * sizeof(double);
  int r;
  const void *lo = nullptr, *hi = nullptr;
  if ((r = device_view(c, sw->lo, nb, c->tile_lo, s, &lo))) return r;
  if ((r = device_view(c, sw->hi, nb, c->tile_hi, s, &hi))) return r;
  a->n_swarm = sw->n_swarm;
  a->n_part = sw->n_part;
  a->x = sw->x;
  a->v = sw->v;
  a->pbest = sw->pbest;
  a->pval = sw->pval;
  a->gbest = sw->gbest;
  a->gval = sw->gval;
  a->lo = (const double*)lo;
  a->hi = (const double*)hi;
  a->inertia = sw->inertia;
  a->c1 = sw->c1;
  a->c2 = sw->c2;
  a->key = make_uint2((uint32_t)sw->seed, (uint32_t)(sw->seed >> 32));
  a->history = nullptr;
  return TFS_OK;
}

}  // namespace

extern "C" {

int tfs_pso_init(tfs_ctx* c, const tfs_swarm* sw, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  PsoArgs a;
  int r = pso_args(c, sw, s, &a);
  if (r) return r;
  c->launches = 0;
  CUDA_TRY(c, launch_pso_init(a, c->n_sm, s));
  c->launches = 1;
  return TFS_OK;
}

int tfs_pso_step(tfs_ctx* c, const tfs_swarm* sw, const double* f, int64_t iter, int move,
                 double* history, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (iter < 0) return fail(c, TFS_ERR_ARG, "iter must be >= 0");
  if (!on_ctx_device(c, f)) return fail(c, TFS_ERR_ARG, "f must be device memory of the context's device");
  if (history && !on_ctx_device(c, history))
    return fail(c, TFS_ERR_ARG, "history must be null or device memory of the context's device");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  PsoArgs a;
  int r = pso_args(c, sw, s, &a);
  if (r) return r;
  a.history = history;
  c->launches = 0;
  CUDA_TRY(c, launch_pso_step(a, f, iter, move ? 1 : 0, s));
  c->launches = 1;
  return TFS_OK;
}

int tfs_refine_step(tfs_ctx* c, const tfs_refine* rf, const double* stat, const double* grad,
                    double* mean_best, void* stream) {
  if (!c) return TFS_ERR_ARG;
  c->err.clear();
  if (!rf) return fail(c, TFS_ERR_ARG, "null refinement state");
  if (rf->n < 0) return fail(c, TFS_ERR_ARG, "n must be >= 0");
  if (rf->n == 0) return TFS_OK;
  const void* ptrs[9] = {stat, grad, rf->theta, rf->best_theta, rf->best_grad, rf->best_stat,
                         rf->eta, rf->sigma, nullptr};
  for (int i = 0; i < 8; ++i)
    if (!on_ctx_device(c, ptrs[i]))
      return fail(c, TFS_ERR_ARG, "refinement arrays must be device memory of the context's device");
  if (mean_best && !on_ctx_device(c, mean_best))
    return fail(c, TFS_ERR_ARG, "mean_best must be null or device memory of the context's device");
  if (!(rf->eta_up > 0.0) || !(rf->eta_down > 0.0))
    return fail(c, TFS_ERR_ARG, "eta_up and eta_down must be > 0");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, TFS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  RefineArgs a;
  a.n = rf->n;
  a.stat = stat;
  a.grad = grad;
  a.theta = rf->theta;
  a.best_theta = rf->best_theta;
  a.best_grad = rf->best_grad;
  a.best_stat = rf->best_stat;
  a.eta = rf->eta;
  a.sigma = rf->sigma;
  for (int q = 0; q < 8; ++q) {
    a.lo[q] = rf->lo[q];
    a.hi[q] = rf->hi[q];
  }
  a.eta_up = rf->eta_up;
  a.eta_down = rf->eta_down;
  a.mean_out = mean_best;
  a.part = nullptr;
  a.done = nullptr;
  int r;
  if (mean_best) {
    const int64_t blocks = (rf->n + 255) / 256;
    if ((r = buf_ensure(c, c->rpart, (size_t)blocks * 8))) return r;
    if (!c->rdone.p) {
      if ((r = buf_ensure(c, c->rdone, 16))) return r;
      CUDA_TRY(c, cudaMemsetAsync(c->rdone.p, 0, 16, s));
    }
    a.part = (double*)c->rpart.p;
    a.done = (unsigned*)c->rdone.p;
  }
  c->launches = 0;
  CUDA_TRY(c, launch_refine_update(a, s));
  c->launches = 1;
  return TFS_OK;
}

}  // extern "C"
