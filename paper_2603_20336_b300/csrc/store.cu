// The CSR doc-set store: device copies of the vectors in FP32 / BF16 / E4M3
// (+ per-vector scale), the offsets, chunk maps for the persistent kernels and
// TMA tensor maps of the low-precision copies.
#include <cuda_fp8.h>

#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

// One warp per set: every padded row r of set d takes source row
// off[d] + min(r, len - 1), so pad rows repeat the set's last vector.
__global__ void quantize_bf16_kernel(const float* __restrict__ src, const int64_t* __restrict__ off,
                                     const int64_t* __restrict__ pad_off, int64_t n_sets,
                                     __nv_bfloat16* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < n_sets;
       d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t s0 = off[d], len = off[d + 1] - s0;
    const int64_t p0 = pad_off[d], plen = pad_off[d + 1] - p0;
    for (int64_t r = 0; r < plen; ++r) {
      const float4 v = reinterpret_cast<const float4*>(src + (s0 + min(r, len - 1)) * kDim)[lane];
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
      __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
      uint2 w;
      w.x = *reinterpret_cast<uint32_t*>(&lo);
      w.y = *reinterpret_cast<uint32_t*>(&hi);
      reinterpret_cast<uint2*>(dst + (p0 + r) * kDim)[lane] = w;
    }
  }
}

// One warp per set, padded as above.  Per vector: s = max_k |x_k| / 448 (IEEE
// division), codes = E4M3(x_k / s) round to nearest even, saturating; a zero
// vector gets s = 1.
__global__ void quantize_fp8_kernel(const float* __restrict__ src, const int64_t* __restrict__ off,
                                    const int64_t* __restrict__ pad_off, int64_t n_sets,
                                    uint8_t* __restrict__ dst, float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < n_sets;
       d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t s0 = off[d], len = off[d + 1] - s0;
    const int64_t p0 = pad_off[d], plen = pad_off[d + 1] - p0;
    for (int64_t r = 0; r < plen; ++r) {
      const float4 v = reinterpret_cast<const float4*>(src + (s0 + min(r, len - 1)) * kDim)[lane];
      float a = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
      const float sc = (a == 0.f) ? 1.f : __fdiv_rn(a, 448.f);
      const float xs[4] = {v.x, v.y, v.z, v.w};
      uint32_t packed = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(__fdiv_rn(xs[j], sc), __NV_SATFINITE, __NV_E4M3);
        packed |= (uint32_t)c << (8 * j);
      }
      reinterpret_cast<uint32_t*>(dst + (p0 + r) * kDim)[lane] = packed;
      if (lane == 0) scale[p0 + r] = sc;
    }
  }
}

// One warp per set, padded as above, one scale for the whole set: the smallest
// power of two s >= FLT_MIN with max |x| over the set <= 448 s (s = 1 for a zero
// set), so that x / s is exact; codes = E4M3(x / s) round to nearest even, saturating.
// A common scale factors out of every maximum over the set's vectors.
__global__ void quantize_fp8_set_kernel(const float* __restrict__ src, const int64_t* __restrict__ off,
                                        const int64_t* __restrict__ pad_off, int64_t n_sets,
                                        uint8_t* __restrict__ dst, float* __restrict__ set_scale) {
  const int lane = threadIdx.x & 31;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < n_sets;
       d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t s0 = off[d], len = off[d + 1] - s0;
    const int64_t p0 = pad_off[d], plen = pad_off[d + 1] - p0;
    float a = 0.f;
    for (int64_t r = 0; r < len; ++r) {
      const float4 v = reinterpret_cast<const float4*>(src + (s0 + r) * kDim)[lane];
      a = fmaxf(a, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    float sc = 1.f;
    if (a > 0.f) {
      // a in [2^(e-1), 2^e): 448 * 2^(e-10) < a <= 448 * 2^(e-8), so the smallest
      // power of two s >= 2^-126 with a <= 448 s is found by at most two doublings
      // (448 s is exact; it may round up to +inf only where s already holds a)
      int e = 0;
      frexpf(a, &e);
      sc = ldexpf(1.f, max(e - 10, -126));
      while (a > 448.f * sc) sc *= 2.f;
    }
    const float inv = 1.f / sc;        // a power of two: x * inv == x / sc exactly
    for (int64_t r = 0; r < plen; ++r) {
      const float4 v = reinterpret_cast<const float4*>(src + (s0 + min(r, len - 1)) * kDim)[lane];
      const float xs[4] = {v.x, v.y, v.z, v.w};
      uint32_t packed = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(xs[j] * inv, __NV_SATFINITE, __NV_E4M3);
        packed |= (uint32_t)c << (8 * j);
      }
      reinterpret_cast<uint32_t*>(dst + (p0 + r) * kDim)[lane] = packed;
    }
    if (lane == 0) set_scale[d] = sc;
  }
}

// lazy deletion (Sec. 4.6): count ids outside [0, n_sets) into bad[0]
__global__ void check_ids_kernel(const int64_t* __restrict__ ids, int64_t n, int64_t n_sets, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (ids[i] < 0 || ids[i] >= n_sets) atomicAdd(bad, 1);
}

// set (deleted) or clear the bit of every id; ids are in range
__global__ void mark_deleted_kernel(const int64_t* __restrict__ ids, int64_t n, bool deleted, uint32_t* dead) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = ids[i];
    const uint32_t bit = 1u << (id & 31);
    if (deleted) atomicOr(dead + (id >> 5), bit);
    else atomicAnd(dead + (id >> 5), ~bit);
  }
}

__global__ void iota_offsets_kernel(int64_t* off, int n, int64_t step) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    off[i] = (int64_t)i * step;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

std::mutex g_store_mutex;  // guards the lazily built per-store caches

}  // namespace

bool encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, void* base, uint64_t inner,
                    uint64_t rows, uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows,
                    CUtensorMapSwizzle swz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, dtype, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tmap_1d_f32(CUtensorMap* map, void* base, uint64_t n, uint32_t box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[1] = {n};
  cuuint64_t strides[1] = {n * 4};
  cuuint32_t boxd[1] = {box};
  cuuint32_t estr[1] = {1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, base, dims, strides, boxd, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_quantize_bf16(const float* src, const int64_t* off, const int64_t* pad_off,
                          int64_t n_sets, __nv_bfloat16* dst, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((n_sets * 32 + 255) / 256, 148 * 16);
  if (grid > 0) { quantize_bf16_kernel<<<grid, 256, 0, st>>>(src, off, pad_off, n_sets, dst); note_launches(1); }
}

void launch_quantize_fp8(const float* src, const int64_t* off, const int64_t* pad_off,
                         int64_t n_sets, uint8_t* dst, float* scale, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((n_sets * 32 + 255) / 256, 148 * 16);
  if (grid > 0) {
    quantize_fp8_kernel<<<grid, 256, 0, st>>>(src, off, pad_off, n_sets, dst, scale);
    note_launches(1);
  }
}

void launch_quantize_fp8_set(const float* src, const int64_t* off, const int64_t* pad_off,
                             int64_t n_sets, uint8_t* dst, float* set_scale, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((n_sets * 32 + 255) / 256, 148 * 16);
  if (grid > 0) {
    quantize_fp8_set_kernel<<<grid, 256, 0, st>>>(src, off, pad_off, n_sets, dst, set_scale);
    note_launches(1);
  }
}

void launch_iota_offsets(int64_t* off, int32_t n, int64_t step, cudaStream_t st) {
  iota_offsets_kernel<<<(n + 256) / 256, 256, 0, st>>>(off, n, step);
  note_launches(1);
}

gem_status launch_mark_deleted(gem_store* s, const int64_t* ids, int64_t n, bool deleted, cudaStream_t st) {
  const size_t words = (size_t)((s->n_sets + 31) / 32);
  if (!s->d_dead) {
    // one extra word counts the ids out of range
    GEM_CUDA_TRY(cudaMalloc(&s->d_dead, sizeof(uint32_t) * (words + 1)));
    GEM_CUDA_TRY(cudaMemsetAsync(s->d_dead, 0, sizeof(uint32_t) * (words + 1), st));
  }
  if (n == 0) return GEM_OK;
  int* bad = reinterpret_cast<int*>(s->d_dead + words);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)s->n_sm * 8);
  GEM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
  check_ids_kernel<<<grid, 256, 0, st>>>(ids, n, s->n_sets, bad);
  GEM_CUDA_TRY(cudaGetLastError());
  int h_bad = 0;
  GEM_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  GEM_CUDA_TRY(cudaStreamSynchronize(st));
  note_launches(1);
  if (h_bad) return GEM_ERR_INVALID;
  mark_deleted_kernel<<<grid, 256, 0, st>>>(ids, n, deleted, s->d_dead);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status store_chunk_map(const gem_store* s, int chunk_rows, const ChunkMap** out) {
  std::lock_guard<std::mutex> lk(g_store_mutex);
  auto it = s->chunks.find(chunk_rows);
  if (it != s->chunks.end()) { *out = &it->second; return GEM_OK; }
  std::vector<int> starts;
  starts.reserve(s->n_sets / 64 + 2);
  int64_t d = 0;
  const auto& off = s->h_pad_offsets;
  while (d < s->n_sets) {
    starts.push_back((int)d);
    const int64_t limit = off[d] + chunk_rows;
    int64_t e = d + 1;
    while (e < s->n_sets && off[e + 1] <= limit) ++e;
    d = e;
  }
  starts.push_back((int)s->n_sets);
  ChunkMap cm;
  cm.chunk_rows = chunk_rows;
  cm.n_chunks = (int)starts.size() - 1;
  int dev_prev = 0;
  cudaGetDevice(&dev_prev);
  cudaSetDevice(s->device);
  cudaError_t e1 = cudaMalloc(&cm.d_chunk_doc, sizeof(int) * starts.size());
  if (e1 == cudaSuccess)
    e1 = cudaMemcpy(cm.d_chunk_doc, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice);
  cudaSetDevice(dev_prev);
  if (e1 != cudaSuccess) return cuda_fail(e1, "chunk map upload");
  auto res = s->chunks.emplace(chunk_rows, cm);
  *out = &res.first->second;
  return GEM_OK;
}

gem_status store_tmap_bf16(const gem_store* s, int box_rows, const CUtensorMap** out) {
  std::lock_guard<std::mutex> lk(g_store_mutex);
  if (!s->d_bf16) return fail(GEM_ERR_STATE, "store keeps no bf16 copy");
  auto it = s->tmap_bf16.find(box_rows);
  if (it == s->tmap_bf16.end()) {
    CUtensorMap m;
    if (!encode_tmap_2d(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, s->d_bf16, kDim, s->n_pad_vecs, kDim * 2, 64,
                        box_rows, CU_TENSOR_MAP_SWIZZLE_128B))
      return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the bf16 store");
    it = s->tmap_bf16.emplace(box_rows, m).first;
  }
  *out = &it->second;
  return GEM_OK;
}

gem_status store_tmap_fp8(const gem_store* s, int box_rows, const CUtensorMap** out) {
  std::lock_guard<std::mutex> lk(g_store_mutex);
  if (!s->d_fp8) return fail(GEM_ERR_STATE, "store keeps no fp8 copy");
  auto it = s->tmap_fp8.find(box_rows);
  if (it == s->tmap_fp8.end()) {
    CUtensorMap m;
    if (!encode_tmap_2d(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, s->d_fp8, kDim, s->n_pad_vecs, kDim, 128,
                        box_rows, CU_TENSOR_MAP_SWIZZLE_128B))
      return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the fp8 store");
    it = s->tmap_fp8.emplace(box_rows, m).first;
  }
  *out = &it->second;
  return GEM_OK;
}

gem_status store_tmap_fp8_set(const gem_store* s, int box_rows, const CUtensorMap** out) {
  std::lock_guard<std::mutex> lk(g_store_mutex);
  if (!s->d_fp8s) return fail(GEM_ERR_STATE, "store keeps no per-set-scale fp8 copy");
  auto it = s->tmap_fp8s.find(box_rows);
  if (it == s->tmap_fp8s.end()) {
    CUtensorMap m;
    if (!encode_tmap_2d(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, s->d_fp8s, kDim, s->n_pad_vecs, kDim, 128,
                        box_rows, CU_TENSOR_MAP_SWIZZLE_128B))
      return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the per-set-scale fp8 store");
    it = s->tmap_fp8s.emplace(box_rows, m).first;
  }
  *out = &it->second;
  return GEM_OK;
}

gem_status store_tmap_fp8_scale(const gem_store* s, int box_rows, const CUtensorMap** out) {
  std::lock_guard<std::mutex> lk(g_store_mutex);
  if (!s->d_fp8_scale) return fail(GEM_ERR_STATE, "store keeps no fp8 copy");
  auto it = s->tmap_fp8_scale.find(box_rows);
  if (it == s->tmap_fp8_scale.end()) {
    CUtensorMap m;
    // the scale allocation has 1024 spare entries past the last padded row
    if (!encode_tmap_1d_f32(&m, s->d_fp8_scale, s->n_pad_vecs + 1024, box_rows))
      return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the fp8 scales");
    it = s->tmap_fp8_scale.emplace(box_rows, m).first;
  }
  *out = &it->second;
  return GEM_OK;
}

}  // namespace gem
