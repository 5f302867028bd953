// Search-stage kernels around the statistic: the particle-swarm update of the per-tile
// stochastic optimiser (Sec. "Implementation details": the maximum of Upsilon in each
// parameter tile is found with a particle swarm) and the bookkeeping and step of the
// batched gradient-ascent refinement of candidates. Both run between launches of the
// statistic or gradient kernels, so that every step of a search stays on the device.
//
// Random numbers of the swarm come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator:
// each draw is a pure function of (counter, key), so any draw can be recomputed
// independently of the order in which threads run.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"

namespace tfs {

namespace {

// One Philox4x32-10 block: ten rounds of the S-box
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key bumped by the Weyl constants
// (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Two doubles in [0, 1) from one block: the top 53 bits of (x, y) and of (z, w).
__device__ __forceinline__ void philox_uniform2(uint4 c, uint2 k, double& a, double& b) {
  const uint4 r = philox4x32_10(c, k);
  const uint64_t ab = ((uint64_t)r.x << 32) | r.y, cd = ((uint64_t)r.z << 32) | r.w;
  a = (double)(ab >> 11) * 0x1.0p-53;
  b = (double)(cd >> 11) * 0x1.0p-53;
}

// Counter of the draw for (particle, coordinate, purpose, iteration).
__device__ __forceinline__ uint4 pso_counter(int64_t particle, int q, int purpose, int64_t iter) {
  return make_uint4((uint32_t)particle, (uint32_t)q | ((uint32_t)purpose << 8) |
                                            ((uint32_t)((uint64_t)particle >> 32) << 16),
                    (uint32_t)iter, (uint32_t)((uint64_t)iter >> 32));
}

__device__ __forceinline__ double period_of(int q) {
  return q == 3 || q == 4 ? 2.0 * kPi : (q == 6 ? kPi : 0.0);
}

}  // namespace

// Initial swarm: x uniform in the tile, v uniform in +-0.1 of its width (zero where the
// tile has no width), personal and swarm bests empty (-inf).
__global__ void k_pso_init(PsoArgs a) {
  const int64_t np = (int64_t)a.n_swarm * a.n_part;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / a.n_part);
    for (int q = 0; q < 8; ++q) {
      const double lo = a.lo[s * 8 + q], span = a.hi[s * 8 + q] - lo;
      double r1, r2;
      philox_uniform2(pso_counter(i, q, 0, 0), a.key, r1, r2);
      a.x[q * np + i] = lo + span * r1;
      a.v[q * np + i] = 0.1 * span * (2.0 * r2 - 1.0);
      a.pbest[q * np + i] = a.x[q * np + i];
    }
    a.pval[i] = -INFINITY;
  }
  // the swarm best starts empty at the tile centre (the first step replaces it)
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.n_swarm;
       s += (int64_t)gridDim.x * blockDim.x) {
    a.gval[s] = -INFINITY;
    for (int q = 0; q < 8; ++q)
      a.gbest[q * a.n_swarm + s] = 0.5 * (a.lo[s * 8 + q] + a.hi[s * 8 + q]);
  }
}

// One swarm per CTA. With f the objective at the current positions:
//   1. personal bests: where f > pval, pval = f and pbest = x;
//   2. swarm best: the largest pval (lowest particle index among equals) replaces the
//      swarm's best if it is larger;
//   3. (move) v <- w v + c1 r1 (pbest - x) + c2 r2 (gbest - x), x <- x + v, with r1, r2
//      uniform per particle and coordinate; for an angle whose tile spans its whole
//      period (phi_0, lambda: 2 pi; psi: pi) the differences take the shorter way round
//      and x wraps into [0, period); every other coordinate is clipped to the tile and
//      its velocity is zeroed where it was clipped; a coordinate of zero width stays.
// The history slot (if any) receives the swarm best after step 2.
__global__ void k_pso_step(PsoArgs a, const double* __restrict__ f, int64_t iter, int move) {
  __shared__ double s_val[256];
  __shared__ int s_idx[256];
  const int s = blockIdx.x;
  const int64_t np = (int64_t)a.n_swarm * a.n_part;
  const int64_t base = (int64_t)s * a.n_part;
  double best = -INFINITY;
  int bidx = 0x7fffffff;
  for (int p = threadIdx.x; p < a.n_part; p += blockDim.x) {
    const int64_t i = base + p;
    const double fi = f[i];
    double pv = a.pval[i];
    if (fi > pv) {
      pv = fi;
      a.pval[i] = fi;
      for (int q = 0; q < 8; ++q) a.pbest[q * np + i] = a.x[q * np + i];
    }
    if (pv > best) {  // p increases along the thread's loop: ties keep the lower index
      best = pv;
      bidx = p;
    }
  }
  s_val[threadIdx.x] = best;
  s_idx[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = s_val[threadIdx.x + o];
      const int i2 = s_idx[threadIdx.x + o];
      const double v1 = s_val[threadIdx.x];
      const int i1 = s_idx[threadIdx.x];
      if (v2 > v1 || (v2 == v1 && i2 < i1)) {
        s_val[threadIdx.x] = v2;
        s_idx[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gv = s_val[0];
    const int gi = s_idx[0];
    if (gi != 0x7fffffff && gv > a.gval[s]) {
      a.gval[s] = gv;
      for (int q = 0; q < 8; ++q) a.gbest[q * a.n_swarm + s] = a.pbest[q * np + base + gi];
    }
    if (a.history) a.history[iter * a.n_swarm + s] = a.gval[s];
  }
  __syncthreads();
  if (!move) return;
  for (int p = threadIdx.x; p < a.n_part; p += blockDim.x) {
    const int64_t i = base + p;
    for (int q = 0; q < 8; ++q) {
      const double lo = a.lo[s * 8 + q], hi = a.hi[s * 8 + q], span = hi - lo;
      const double per = period_of(q);
      const bool periodic = per > 0.0 && span >= per * (1.0 - 1e-12);
      const double x = a.x[q * np + i];
      double dp = a.pbest[q * np + i] - x, dg = a.gbest[q * a.n_swarm + s] - x;
      if (periodic) {  // the shorter way round
        dp = dp + 0.5 * per - per * floor((dp + 0.5 * per) / per) - 0.5 * per;
        dg = dg + 0.5 * per - per * floor((dg + 0.5 * per) / per) - 0.5 * per;
      }
      double r1, r2;
      philox_uniform2(pso_counter(i, q, 1, iter), a.key, r1, r2);
      double v = a.inertia * a.v[q * np + i] + a.c1 * r1 * dp + a.c2 * r2 * dg;
      if (span == 0.0) v = 0.0;
      double xn = x + v;
      if (periodic && span != 0.0) {
        xn = xn - per * floor(xn / per);
      } else {
        const double c = fmin(fmax(xn, lo), hi);
        if (c != xn) v = 0.0;
        xn = c;
      }
      a.x[q * np + i] = xn;
      a.v[q * np + i] = v;
    }
  }
}

cudaError_t launch_pso_init(const PsoArgs& a, int n_sm, cudaStream_t s) {
  const int64_t np = (int64_t)a.n_swarm * a.n_part;
  const int blocks = (int)std::min<int64_t>((np + 255) / 256, (int64_t)n_sm * 8);
  k_pso_init<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pso_step(const PsoArgs& a, const double* f, int64_t iter, int move,
                            cudaStream_t s) {
  k_pso_step<<<a.n_swarm, 256, 0, s>>>(a, f, iter, move);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Noise-only data for false-alarm backgrounds (Sec. "Search results on the full dataset":
// the background comes from independent noise-only realisations): per pixel
//   d~ = sqrt(S / (4 df)) (g1 + i g2),  S = 1/w (d~ = 0 where w = 0),
// so that E|d~|^2 = S / (2 df), with g1, g2 independent standard normals from the
// Box-Muller transform of the two uniforms of one Philox4x32-10 block keyed by the seed,
// counter (pixel index low, high, 0, kNoiseTag).
// ---------------------------------------------------------------------------------
constexpr uint32_t kNoiseTag = 0x4E4F4953u;

__global__ void k_noise(int64_t n, const double* __restrict__ w, double df, uint2 key,
                        double* __restrict__ d_re, double* __restrict__ d_im) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double u1, u2;
    philox_uniform2(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, kNoiseTag), key,
                    u1, u2);
    const double wi = w[i];
    double re = 0.0, im = 0.0;
    if (wi > 0.0) {
      const double r = sqrt(-2.0 * log(1.0 - u1)) * sqrt(1.0 / (4.0 * df * wi));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      re = r * cs;
      im = r * sn;
    }
    d_re[i] = re;
    d_im[i] = im;
  }
}

cudaError_t launch_noise(int64_t n, const double* w, double df, uint64_t seed, double* d_re,
                         double* d_im, int n_sm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 16);
  k_noise<<<blocks, 256, 0, s>>>(n, w, df, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)),
                                d_re, d_im);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Refinement by projected gradient ascent, one thread per candidate. With U and g the
// statistic and its gradient at the current parameters theta:
//   accept when U >= U_best (theta_best, g_best, U_best take the current values, the
//   step length eta grows by eta_up), else reject (eta shrinks by eta_down);
//   then theta = theta_best + eta sigma (sigma g_best) / |sigma g_best|,
// with sigma the per-parameter scales, projected as the ascent step projects (angles
// phi_0, lambda wrapped to [0, 2 pi), psi to [0, pi), the rest clamped to [lo, hi]).
// Each block adds its candidates' U_best in a fixed order; the last block to finish
// adds the blocks' sums in block order and writes their mean.
// ---------------------------------------------------------------------------------
__global__ void k_refine_update(RefineArgs a) {
  __shared__ double s_sum[256];
  __shared__ bool s_last;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = a.n;
  double ub = 0.0;
  if (i < n) {
    const double u = a.stat[i];
    ub = a.best_stat[i];
    double eta = a.eta[i];
    if (u >= ub) {
      ub = u;
      a.best_stat[i] = u;
      for (int q = 0; q < 8; ++q) {
        a.best_theta[q * n + i] = a.theta[q * n + i];
        a.best_grad[q * n + i] = a.grad[q * n + i];
      }
      eta *= a.eta_up;
    } else {
      eta *= a.eta_down;
    }
    a.eta[i] = eta;
    double sg[8], nrm = 0.0;
    for (int q = 0; q < 8; ++q) {
      sg[q] = a.sigma[q * n + i] * a.best_grad[q * n + i];
      nrm += sg[q] * sg[q];
    }
    const double scale = eta / fmax(sqrt(nrm), 1e-300);
    for (int q = 0; q < 8; ++q) {
      double x = a.best_theta[q * n + i] + a.sigma[q * n + i] * sg[q] * scale;
      if (q == 3 || q == 4) {
        x = x - 2.0 * kPi * floor(x / (2.0 * kPi));
      } else if (q == 6) {
        x = x - kPi * floor(x / kPi);
      } else {
        x = fmin(fmax(x, a.lo[q]), a.hi[q]);
      }
      a.theta[q * n + i] = x;
    }
  }
  if (!a.mean_out) return;
  s_sum[threadIdx.x] = i < n ? ub : 0.0;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = s_sum[0];
    __threadfence();
    s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += ((volatile double*)a.part)[b];
    *a.mean_out = tot / (double)n;
    *a.done = 0u;  // ready for the next call
  }
}

cudaError_t launch_refine_update(const RefineArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  k_refine_update<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tfs
