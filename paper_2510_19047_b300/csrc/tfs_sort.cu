// Stable least-significant-digit radix sort (8-bit digits) of (key, index) pairs.
// Per pass: a per-tile digit histogram, one exclusive scan over (digit, tile) in
// digit-major order, and a scatter in which every tile ranks its items stably
// (warp match + per-warp counts + a prefix over the warps of the tile).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "tfs_sort.cuh"

namespace tfs {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;  // items per thread and tile (rounds of 256)
constexpr int kTile = kThreads * kItems;
constexpr int kDigits = 256;
constexpr int kWarps = kThreads / 32;

template <class K>
__global__ void k_hist(const K* __restrict__ keys, int64_t n, int shift, int ntiles,
                       unsigned* __restrict__ hist) {
  __shared__ unsigned h[kDigits];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + r * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m unsigned ints by one block of 1024 threads.
__global__ void k_scan(unsigned* __restrict__ v, int64_t m) {
  __shared__ unsigned part[1024];
  const int64_t per = (m + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = lo + per < m ? lo + per : m;
  unsigned s = 0;
  for (int64_t i = lo; i < hi; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned x = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int64_t i = lo; i < hi; ++i) {
    const unsigned x = v[i];
    v[i] = run;
    run += x;
  }
}

template <class K, class V>
__global__ void k_scatter(const K* __restrict__ kin, const V* __restrict__ vin, K* __restrict__ kout,
                          V* __restrict__ vout, int64_t n, int shift, int ntiles,
                          const unsigned* __restrict__ offs) {
  __shared__ unsigned wcount[kWarps][kDigits];
  __shared__ unsigned running[kDigits];
  __shared__ unsigned total[kDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kItems; ++r) {
    for (int w = 0; w < kWarps; ++w) wcount[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = base + r * kThreads + threadIdx.x;
    const bool ok = i < n;
    K key = 0;
    V val = 0;
    unsigned d = kDigits;  // out-of-range items form their own group and are not written
    if (ok) {
      key = kin[i];
      val = vin[i];
      d = (unsigned)(key >> shift) & 0xffu;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt);
    if (ok && rank == 0) wcount[warp][d] = __popc(peers);
    __syncthreads();
    {
      unsigned acc = 0;
      for (int w = 0; w < kWarps; ++w) {
        const unsigned x = wcount[w][threadIdx.x];
        wcount[w][threadIdx.x] = acc;
        acc += x;
      }
      total[threadIdx.x] = acc;
    }
    __syncthreads();
    if (ok) {
      const unsigned pos = running[d] + wcount[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    running[threadIdx.x] += total[threadIdx.x];
    __syncthreads();
  }
}

template <class K, class V>
cudaError_t radix_sort(K* k0, V* v0, K* k1, V* v1, unsigned* hist, int64_t n, int key_bits,
                       cudaStream_t s, int* launches, bool* result_in_1) {
  const int ntiles = (int)((n + kTile - 1) / kTile);
  K *ki = k0, *ko = k1;
  V *vi = v0, *vo = v1;
  int passes = 0;
  for (int shift = 0; shift < key_bits; shift += 8) {
    k_hist<K><<<ntiles, kThreads, 0, s>>>(ki, n, shift, ntiles, hist);
    k_scan<<<1, 1024, 0, s>>>(hist, (int64_t)kDigits * ntiles);
    k_scatter<K, V><<<ntiles, kThreads, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, hist);
    std::swap(ki, ko);
    std::swap(vi, vo);
    ++passes;
    *launches += 3;
  }
  *result_in_1 = (passes & 1) != 0;
  return cudaGetLastError();
}

__global__ void k_template_keys(const TplConst* __restrict__ tpl, int64_t n, uint32_t* keys,
                                int32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    keys[i] = tpl[i].key;
    vals[i] = (int32_t)i;
  }
}

// Ascending order of the key = decreasing order of the statistic; NaN sorts last; -0.0
// and +0.0 are one key, so that they tie like other equal values (by the lower index).
__global__ void k_stat_keys(const double* __restrict__ stat, int64_t n, uint64_t* keys,
                            int32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double x = stat[i] == 0.0 ? 0.0 : stat[i];
    uint64_t b = (uint64_t)__double_as_longlong(x);
    b = (b >> 63) ? ~b : (b | 0x8000000000000000ull);  // monotone in x
    keys[i] = isnan(x) ? ~0ull : ~b;
    vals[i] = (int32_t)i;
  }
}

__global__ void k_copy_idx(const int32_t* __restrict__ v, int64_t k, int64_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < k) out[i] = v[i];
}

}  // namespace

size_t sort_scratch_bytes(int64_t n) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  return (size_t)n * (4 + 4 + 4) + (size_t)kDigits * ntiles * 4 + 256;
}

cudaError_t sort_templates(const TplConst* tpl, int64_t n, int32_t* perm, void* scratch, int n_sm,
                           cudaStream_t s, int* launches) {
  (void)n_sm;
  if (n <= 0) return cudaSuccess;
  char* p = (char*)scratch;
  uint32_t* k0 = (uint32_t*)p;
  uint32_t* k1 = k0 + n;
  int32_t* v0 = (int32_t*)(k1 + n);
  unsigned* hist = (unsigned*)(v0 + n);
  k_template_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tpl, n, k0, v0);
  *launches += 1;
  bool in1 = false;
  cudaError_t e = radix_sort<uint32_t, int32_t>(k0, v0, k1, perm, hist, n, 32, s, launches, &in1);
  if (e != cudaSuccess) return e;
  // 4 passes: the result is back in (k0, v0)
  if (!in1) {
    e = cudaMemcpyAsync(perm, v0, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

size_t topk_scratch_bytes(int64_t n) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  return (size_t)n * (8 + 8 + 4 + 4) + (size_t)kDigits * ntiles * 4 + 256;
}

cudaError_t select_top(const double* stat, int64_t n, int64_t k, int64_t* out_idx, void* scratch,
                       cudaStream_t s, int* launches) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  char* p = (char*)scratch;
  uint64_t* k0 = (uint64_t*)p;
  uint64_t* k1 = k0 + n;
  int32_t* v0 = (int32_t*)(k1 + n);
  int32_t* v1 = v0 + n;
  unsigned* hist = (unsigned*)(v1 + n);
  k_stat_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(stat, n, k0, v0);
  *launches += 1;
  bool in1 = false;
  cudaError_t e = radix_sort<uint64_t, int32_t>(k0, v0, k1, v1, hist, n, 64, s, launches, &in1);
  if (e != cudaSuccess) return e;
  const int32_t* res = in1 ? v1 : v0;
  k_copy_idx<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(res, k, out_idx);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace tfs

// ---------------------------------------------------------------------------------
// Top-k selection that allocates nothing, for callers that cannot call cudaMalloc:
// code running between the launches of a pipeline that must not synchronise the
// device (cudaMalloc and cudaFree synchronise), or inside a framework whose memory
// is owned by its own pool under a fixed budget. The radix-sort scratch lives in a
// file-scope device array that every GPU loading this library keeps until exit.
// ---------------------------------------------------------------------------------
namespace tfs {
namespace {

constexpr int64_t kStaticTopMax = 1 << 16;  // largest n the static scratch holds
constexpr size_t kStaticTopBytes =
    (size_t)kStaticTopMax * (8 + 8 + 4 + 4) +
    (size_t)kDigits * ((kStaticTopMax + kTile - 1) / kTile) * 4 + 256;

static __device__ __align__(256) unsigned char g_top_scratch[kStaticTopBytes];

constexpr int kMaxDevices = 64;
std::mutex g_top_mutex;
void* g_top_ptr[kMaxDevices] = {};

// Device address of g_top_scratch on the current device (looked up once per device).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_top_mutex);
  if (!g_top_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_top_scratch);
    if (e != cudaSuccess) return e;
    g_top_ptr[dev] = p;
  }
  *out = g_top_ptr[dev];
  return cudaSuccess;
}

// Device (or managed) memory of the current device.
bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace tfs

extern "C" int tfs_select_top_noalloc(const double* stat, int64_t n, int64_t k,
                                      int64_t* out_index, void* stream) {
  using namespace tfs;
  if (n < 0 || k < 0 || k > n) return TFS_ERR_ARG;
  if (n > kStaticTopMax) return TFS_ERR_ARG;  // beyond the static scratch
  if (k == 0) return TFS_OK;
  if (!stat || !out_index || !on_device(stat) || !on_device(out_index)) return TFS_ERR_ARG;
  void* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return TFS_ERR_CUDA;
  int launches = 0;
  if (select_top(stat, n, k, out_index, scratch, (cudaStream_t)stream, &launches) != cudaSuccess)
    return TFS_ERR_CUDA;
  return TFS_OK;
}
