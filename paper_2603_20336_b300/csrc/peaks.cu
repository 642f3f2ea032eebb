// Measured peaks of the two resources the FP32 and table-lookup kernels are
// bound by (the denominators of their roofline fractions):
//  - FP32 fused multiply-add throughput: every thread of a full grid runs 16
//    independent FMA chains as packed two-lane instructions (fma.rn.f32x2, the
//    form the FP32 scorers use);
//  - L2-resident gather bandwidth: warps read 128-byte rows at hashed row indices
//    of a 64 MB buffer that stays in L2 (the access pattern of the qCH table
//    lookups), one coalesced 128-byte row per warp load.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fp32_peak_kernel(int iters, float seed, float* out) {
  uint64_t a[8], b = pack2(1.0000001f, 0.9999999f), c = pack2(seed * 1e-7f, seed * -1e-7f);
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = pack2(seed + i, seed - i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = ffma2(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += lo2(a[i]) + hi2(a[i]);
  if (s == 1.2345f) out[0] = s;  // keeps the chains live
}

// rows_mask + 1 rows of 32 floats (a power of two); eight independent hashed
// row reads in flight per lane at a time
__global__ void __launch_bounds__(kPeakThreads) l2_gather_kernel(const float* __restrict__ buf, uint32_t rows_mask,
                                                                  int reads_per_warp, float* out) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float acc[8] = {};
  for (int r = 0; r < reads_per_warp; r += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      uint32_t h = (warp * 2654435761u) ^ ((uint32_t)(r + u) * 0x9E3779B9u);
      h ^= h >> 15;
      h *= 0x2C1B3C6Du;
      h ^= h >> 12;
      acc[u] += __ldcg(buf + (size_t)(h & rows_mask) * 32 + lane);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += acc[u];
  if (s == 1.2345f) out[0] = s;
}

}  // namespace
}  // namespace gem

using namespace gem;

extern "C" gem_status gem_measure_peaks(float* fp32_tflops, float* l2_gather_gbs, void* stream) {
  if (!fp32_tflops || !l2_gather_gbs) return fail(GEM_ERR_INVALID, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, n_sm = 0;
  GEM_CUDA_TRY(cudaGetDevice(&dev));
  GEM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t rows = (int64_t)(64 << 20) / 128;  // 64 MB of 128-byte rows (2^19: a power of two)
  float* buf = nullptr;
  if (cudaMalloc(&buf, rows * 128 + 256) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEM_ERR_OOM, "64 MB probe buffer");
  }
  float* out = buf + rows * 32;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gem_status r = GEM_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && r == GEM_OK) r = cuda_fail(e, what);
  };
  check(cudaMemsetAsync(buf, 0, rows * 128 + 256, st), "cudaMemsetAsync");
  // FP32: grid of 8 CTAs per SM, best of three timed launches
  const int grid = n_sm * 8, iters = 1 << 14;
  float best_ms = 1e30f;
  for (int rep = 0; rep < 4 && r == GEM_OK; ++rep) {
    check(cudaEventRecord(e0, st), "cudaEventRecord");
    fp32_peak_kernel<<<grid, kPeakThreads, 0, st>>>(iters, 1.f + rep, out);
    check(cudaEventRecord(e1, st), "cudaEventRecord");
    check(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (rep > 0) best_ms = std::min(best_ms, ms);
  }
  *fp32_tflops = (float)((double)grid * kPeakThreads * iters * 8 * 2 * 2 / (best_ms * 1e-3) / 1e12);
  // L2 gathers: the buffer is read once to bring it into L2, then timed
  const int reads = 2048;
  best_ms = 1e30f;
  for (int rep = 0; rep < 4 && r == GEM_OK; ++rep) {
    check(cudaEventRecord(e0, st), "cudaEventRecord");
    l2_gather_kernel<<<grid, kPeakThreads, 0, st>>>(buf, (uint32_t)(rows - 1), reads, out);
    check(cudaEventRecord(e1, st), "cudaEventRecord");
    check(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (rep > 0) best_ms = std::min(best_ms, ms);
  }
  *l2_gather_gbs = (float)((double)grid * (kPeakThreads / 32) * reads * 128 / (best_ms * 1e-3) / 1e9);
  note_launches(8);
  check(cudaGetLastError(), "probe kernels");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return r;
}
