// Gradient-ascent update of candidate templates (refinement of candidates by
// d Upsilon / d theta).
#include <math.h>

#include "tfs_internal.cuh"
#include "tfs_kernels.cuh"

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

}  // namespace tfs
