// gpe_sums_noalloc: the FP64 grid sums behind gpe_energy (sum |psi|^2, sum V |psi|^2,
// sum |psi|^4) for callers that cannot allocate device memory.
//
// Some callers can't call cudaMalloc: a host application whose memory pool already
// reserves the whole device, a plugin that may only use memory its host hands it, or a
// time-critical loop that must not risk the device-wide synchronisation an allocation
// can cause.  This entry point allocates nothing (no cudaMalloc/cudaFree, no library
// call that allocates): the block partials of the reduction live in the file-scope
// array g_partials below, which every GPU that loads this library holds until the
// process exits.
//
// Set-up: host code cannot pass g_partials itself to a kernel (in host code the name is
// only a host-side stand-in for the device symbol), so the first call on each device
// looks up the array's device address with cudaGetSymbolAddress, with that device
// current, and caches it.  That first call should come before any stream capture.  A
// cached address is checked on every call (cudaPointerGetAttributes, no allocation) and
// looked up again if the device's context was reset since (cudaDeviceReset).
//
// All calls share the array and it keeps the last call's contents.  Every call writes
// each partial it reads before reading it, so nothing needs clearing.  Calls whose work
// overlaps on the GPU (different streams, or other threads) race on the array and must
// be serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNoallocBlocks = 16384;              // partial slots
constexpr int kNoallocThreads = 256;
constexpr int kNoallocPerThread = 16;              // elements per thread per block
constexpr long long kNoallocMax = (long long)kNoallocBlocks * kNoallocThreads * kNoallocPerThread;  // 2^26

// [kNoallocBlocks][4] FP64 block partials: 512 KiB
static __device__ __align__(256) double g_partials[kNoallocBlocks * 4];

std::mutex g_mu;
double* g_addr[64] = {};  // device address of g_partials, per device ordinal

template <typename T>
__global__ void __launch_bounds__(kNoallocThreads)
    k_sums_partial(const ddi::cx_t<T>* __restrict__ psi, const T* __restrict__ V, long long count, double* part) {
  double v[3] = {0.0, 0.0, 0.0};
  const long long base = (long long)blockIdx.x * kNoallocThreads * kNoallocPerThread;
  for (int k = 0; k < kNoallocPerThread; ++k) {
    const long long i = base + (long long)k * kNoallocThreads + threadIdx.x;
    if (i < count) {
      const ddi::cx_t<T> a = psi[i];
      const double r = (double)a.x * a.x + (double)a.y * a.y;
      v[0] += r;
      v[1] += (double)V[i] * r;
      v[2] += r * r;
    }
  }
  __shared__ double sh[3][kNoallocThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 3; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[q][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) s += sh[threadIdx.x][w];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// sums the first `blocks` partials into out[0..2] in a fixed order (deterministic): thread t
// adds the contiguous chunk t of the partials in index order, then the chunk sums are added
// pairwise in a fixed tree
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) k_sums_final(const double* part, int blocks, double* out) {
  __shared__ double sh[3][kFinalThreads];
  const int t = threadIdx.x;
  const int per = (blocks + kFinalThreads - 1) / kFinalThreads;
  const int b0 = t * per, b1 = min(blocks, b0 + per);
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = b0; b < b1; ++b)
    for (int q = 0; q < 3; ++q) v[q] += part[(size_t)b * 4 + q];
  for (int q = 0; q < 3; ++q) sh[q][t] = v[q];
  __syncthreads();
  for (int o = kFinalThreads / 2; o > 0; o >>= 1) {
    if (t < o)
      for (int q = 0; q < 3; ++q) sh[q][t] += sh[q][t + o];
    __syncthreads();
  }
  if (t < 3) out[t] = sh[t][0];
}

// device address of g_partials on the current device dev (looked up once, re-checked)
int partials_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev]) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, g_addr[dev]) == cudaSuccess && at.type == cudaMemoryTypeDevice &&
        at.device == dev) {
      *out = g_addr[dev];
      return DDI_OK;
    }
    cudaGetLastError();
    g_addr[dev] = nullptr;  // the context was reset: look the array up again
  }
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_partials);
  if (e != cudaSuccess) {
    ddi::set_error("gpe_sums_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return DDI_ERR_CUDA;
  }
  g_addr[dev] = static_cast<double*>(ptr);
  *out = g_addr[dev];
  return DDI_OK;
}

}  // namespace

extern "C" int gpe_sums_noalloc(const void* psi, const void* V, int64_t count, int precision, double* sums,
                                void* stream) {
  return ddi::guarded("gpe_sums_noalloc", [&]() -> int {
    if (!psi || !V || !sums || count < 0 || (precision != DDI_FP64 && precision != DDI_FP32)) {
      ddi::set_error("gpe_sums_noalloc: psi, V, sums must be non-NULL device pointers, count >= 0, "
                     "precision DDI_FP64 or DDI_FP32");
      return DDI_ERR_ARG;
    }
    if (count > kNoallocMax) {
      ddi::set_error("gpe_sums_noalloc: count %lld exceeds the maximum %lld grid points of its fixed scratch",
                     (long long)count, kNoallocMax);
      return DDI_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      cudaGetLastError();
      ddi::set_error("gpe_sums_noalloc: no usable current device");
      return DDI_ERR_CUDA;
    }
    double* part = nullptr;
    DDI_TRY(partials_address(dev, &part));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long per = (long long)kNoallocThreads * kNoallocPerThread;
    const int blocks = count == 0 ? 0 : (int)((count + per - 1) / per);
    if (blocks > 0) {
      if (precision == DDI_FP64) {
        k_sums_partial<double><<<blocks, kNoallocThreads, 0, s>>>(static_cast<const double2*>(psi),
                                                                  static_cast<const double*>(V), count, part);
      } else {
        k_sums_partial<float><<<blocks, kNoallocThreads, 0, s>>>(static_cast<const float2*>(psi),
                                                                 static_cast<const float*>(V), count, part);
      }
      DDI_LAUNCH_CHECK();
    }
    k_sums_final<<<1, kFinalThreads, 0, s>>>(part, blocks, sums);
    DDI_LAUNCH_CHECK();
    return DDI_OK;
  });
}
