// Query plan for the tensor-core scoring kernels.
//
// Each query set is cut into parts of at most 32 vectors.  A part of r rows
// occupies a slot of g = next_pow2(r) rows, so every slot lies inside one warp's
// 32 TMEM lanes at an offset that is a multiple of g and its per-row maxima can be
// summed with a fixed butterfly of g lanes.  Slots are packed by (pass, g desc,
// query): pass p holds the p-th part of every query long enough to have one, and
// each pass starts on a query-block boundary so a scoring launch covers one pass.
// Pass p > 0 adds its part sums onto the scores pass p-1 wrote, so the sum over a
// query's vectors always runs part 0, part 1, ... in that order.
//
// Everything is computed on the device from the device-resident q_offsets, so a
// call never reads metadata back to the host.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

struct PlanPtrs {
  int* hdr;
  int* part_query;
  int* part_rows;
  int* part_g;
  int* part_pass;
  int* part_slot;
  int64_t* part_row0;
  int* row_part;
};

__device__ __forceinline__ int slot_class(int rows) {  // g = 32 >> class
  int g = 1;
  while (g < rows) g <<= 1;
  return 5 - (31 - __clz(g));
}

// The part of query b (m vectors) that pass p holds, as a combo index
// p * kClasses + class, or -1.
__device__ __forceinline__ int part_combo(int m, int p) {
  int np = (m + 31) >> 5;
  if (p >= np) return -1;
  int rows = (p < np - 1) ? 32 : m - 32 * (np - 1);
  return p * kClasses + slot_class(rows);
}

__global__ void __launch_bounds__(1024, 1)
plan_kernel(const int64_t* __restrict__ qo, int B, int64_t n_rows, int m_res, int max_q_len,
            int64_t packed_cap, int64_t max_parts, PlanPtrs pp, int* status) {
  __shared__ int cnt[kCombos];
  __shared__ int start_row[kCombos];
  __shared__ int part_base[kCombos];
  __shared__ int run_base[kCombos];
  __shared__ int chunk_tot[kCombos];
  __shared__ int warp_tot[32][kCombos];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kCombos) { cnt[tid] = 0; run_base[tid] = 0; }
  if (tid == 0) bad = (qo[0] != 0 || qo[B] != n_rows) ? 1 : 0;
  __syncthreads();
  const int n_chunks = (B + 1023) / 1024;
  const unsigned lt_mask = (1u << lane) - 1u;

  // 1. parts per (pass, slot class)
  for (int c = 0; c < n_chunks; ++c) {
    int b = c * 1024 + tid;
    int m = 0;
    if (b < B) {
      int64_t mm = qo[b + 1] - qo[b];
      if (mm < 1 || mm > max_q_len) { atomicOr(&bad, 1); mm = 0; }
      m = (int)mm;
    }
    for (int p = 0; p < kMaxPasses; ++p) {
      int combo = part_combo(m, p);
      for (int cl = 0; cl < kClasses; ++cl) {
        unsigned bal = __ballot_sync(0xffffffffu, combo == p * kClasses + cl);
        if (lane == 0 && bal) atomicAdd(&cnt[p * kClasses + cl], __popc(bal));
      }
    }
  }
  __syncthreads();

  // 2. slot rows and part ids of each (pass, class) run
  if (tid == 0) {
    int64_t row = 0, pid = 0;
    int passes = 0;
    for (int p = 0; p < kMaxPasses; ++p) {
      pp.hdr[kHdrQbBegin + p] = (int)(row / m_res);
      int64_t before = row;
      for (int cl = 0; cl < kClasses; ++cl) {
        int k = p * kClasses + cl;
        start_row[k] = (int)row;
        part_base[k] = (int)pid;
        row += (int64_t)cnt[k] * (32 >> cl);
        pid += cnt[k];
      }
      if (row > before) passes = p + 1;
      row = (row + m_res - 1) / m_res * m_res;
    }
    if (row > packed_cap || pid > max_parts) bad |= 2;
    if (bad) {
      set_status(status, kDevInvalid);
      for (int p = 0; p <= kMaxPasses; ++p) pp.hdr[kHdrQbBegin + p] = 0;
      pp.hdr[kHdrParts] = 0;
      pp.hdr[kHdrPackedRows] = 0;
      pp.hdr[kHdrQBlocks] = 0;
      pp.hdr[kHdrPasses] = 0;
    } else {
      pp.hdr[kHdrQbBegin + kMaxPasses] = (int)(row / m_res);
      pp.hdr[kHdrParts] = (int)pid;
      pp.hdr[kHdrPackedRows] = (int)row;
      pp.hdr[kHdrQBlocks] = (int)(row / m_res);
      pp.hdr[kHdrPasses] = passes;
    }
  }
  __syncthreads();
  if (bad) return;

  // 3. ranks inside each run (queries in ascending order) -> part tables
  for (int c = 0; c < n_chunks; ++c) {
    int b = c * 1024 + tid;
    int m = (b < B) ? (int)(qo[b + 1] - qo[b]) : 0;
    for (int k = 0; k < kCombos; ++k) {
      unsigned bal = __ballot_sync(0xffffffffu, part_combo(m, k / kClasses) == k);
      if (lane == 0) warp_tot[warp][k] = __popc(bal);
    }
    __syncthreads();
    if (tid < kCombos) {
      int acc = 0;
      for (int w = 0; w < 32; ++w) {
        int t = warp_tot[w][tid];
        warp_tot[w][tid] = acc;
        acc += t;
      }
      chunk_tot[tid] = acc;
    }
    __syncthreads();
    for (int p = 0; p < kMaxPasses; ++p) {
      int combo = part_combo(m, p);
      for (int cl = 0; cl < kClasses; ++cl) {
        int k = p * kClasses + cl;
        unsigned bal = __ballot_sync(0xffffffffu, combo == k);
        if (combo == k) {
          int rank = run_base[k] + warp_tot[warp][k] + __popc(bal & lt_mask);
          int g = 32 >> cl;
          int id = part_base[k] + rank;
          int slot = start_row[k] + rank * g;
          int np = (m + 31) >> 5;
          pp.part_query[id] = b;
          pp.part_row0[id] = qo[b] + 32LL * p;
          pp.part_rows[id] = (p < np - 1) ? 32 : m - 32 * (np - 1);
          pp.part_g[id] = g;
          pp.part_pass[id] = p;
          pp.part_slot[id] = slot;
          for (int r = 0; r < g; ++r) pp.row_part[slot + r] = id;
        }
      }
    }
    __syncthreads();
    if (tid < kCombos) run_base[tid] += chunk_tot[tid];
    __syncthreads();
  }
}

// One warp per packed row: copy the part's row (or zeros) as bf16, round to
// nearest even.
__global__ void pack_bf16_kernel(const float* __restrict__ q, const int* __restrict__ hdr,
                                 const int* __restrict__ row_part, const int* __restrict__ part_slot,
                                 const int* __restrict__ part_rows, const int64_t* __restrict__ part_row0,
                                 __nv_bfloat16* __restrict__ out) {
  const int n_rows = hdr[kHdrPackedRows];
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows;
       r += (gridDim.x * blockDim.x) >> 5) {
    int p = row_part[r];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p >= 0) {
      int i = r - part_slot[p];
      if (i < part_rows[p]) v = reinterpret_cast<const float4*>(q + (part_row0[p] + i) * kDim)[lane];
    }
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 w;
    w.x = *reinterpret_cast<uint32_t*>(&lo);
    w.y = *reinterpret_cast<uint32_t*>(&hi);
    reinterpret_cast<uint2*>(out + (int64_t)r * kDim)[lane] = w;
  }
}

// One warp per packed row: per-row scale s = amax / 448 and E4M3 codes of x / s
// (round to nearest even, saturating).  Zero rows get s = 1.
__global__ void pack_fp8_kernel(const float* __restrict__ q, const int* __restrict__ hdr,
                                const int* __restrict__ row_part, const int* __restrict__ part_slot,
                                const int* __restrict__ part_rows, const int64_t* __restrict__ part_row0,
                                uint8_t* __restrict__ out, float* __restrict__ scale) {
  const int n_rows = hdr[kHdrPackedRows];
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows;
       r += (gridDim.x * blockDim.x) >> 5) {
    int p = row_part[r];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p >= 0) {
      int i = r - part_slot[p];
      if (i < part_rows[p]) v = reinterpret_cast<const float4*>(q + (part_row0[p] + i) * kDim)[lane];
    }
    float a = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    float s = (a == 0.f) ? 1.f : __fdiv_rn(a, 448.f);
    uint32_t packed = 0;
    float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(__fdiv_rn(xs[j], s), __NV_SATFINITE, __NV_E4M3);
      packed |= (uint32_t)c << (8 * j);
    }
    reinterpret_cast<uint32_t*>(out + (int64_t)r * kDim)[lane] = packed;
    if (lane == 0) scale[r] = s;
  }
}

}  // namespace

gem_status launch_plan(gem_workspace* ws, const float* q, const int64_t* q_offsets,
                       int32_t n_queries, int64_t n_q_rows, int m_res, int compute,
                       cudaStream_t st) {
  PlanPtrs pp{ws->d_plan_hdr, ws->d_part_query, ws->d_part_rows, ws->d_part_g,
              ws->d_part_pass, ws->d_part_slot, ws->d_part_row0, ws->d_row_part};
  GEM_CUDA_TRY(cudaMemsetAsync(ws->d_row_part, 0xFF, sizeof(int) * ws->packed_cap, st));
  plan_kernel<<<1, 1024, 0, st>>>(q_offsets, n_queries, n_q_rows, m_res, ws->max_q_len,
                                  ws->packed_cap, ws->max_parts, pp, ws->d_status);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  const int threads = 256;
  int64_t warps_needed = ws->packed_cap;
  int blocks = (int)std::min<int64_t>((warps_needed * 32 + threads - 1) / threads,
                                      (int64_t)ws->store->n_sm * 8);
  if (blocks < 1) blocks = 1;
  if (compute == GEM_FP8_E4M3) {
    pack_fp8_kernel<<<blocks, threads, 0, st>>>(q, ws->d_plan_hdr, ws->d_row_part, ws->d_part_slot,
                                                ws->d_part_rows, ws->d_part_row0, ws->d_qpack_fp8,
                                                ws->d_qpack_scale);
  } else {
    pack_bf16_kernel<<<blocks, threads, 0, st>>>(q, ws->d_plan_hdr, ws->d_row_part, ws->d_part_slot,
                                                 ws->d_part_rows, ws->d_part_row0, ws->d_qpack_bf16);
  }
  GEM_CUDA_TRY(cudaGetLastError());
  return GEM_OK;
}

}  // namespace gem
