// Exact MaxSim in FP32 on the SIMT pipes, with a compensated sum over query
// vectors.  Serves the FP32 exhaustive form and the exact rerank of a candidate
// pool (the final step of Algorithm 5, CH of Sec. 3.1 Eq. 1).
//
// Arithmetic order (fixed, independent of launch shape):
//   dot(q_i, p_j): one FP32 fused multiply-add chain over k = 0 .. 127
//   m_i = max_j dot(q_i, p_j)
//   CH  = Kahan sum of m_i over i = 0 .. m_q - 1 in ascending order
//
// Mapping: one CTA per work unit, lane = query row (32 rows per pass, the row's
// 128 components held in registers), one warp per document; the document's
// vectors are staged 8 at a time in the warp's shared-memory slice and read as
// broadcasts.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kF32Warps = 4;
constexpr int kF32Threads = kF32Warps * 32;
constexpr int kVecBlock = 8;          // document vectors staged per step
constexpr int kQStride = kDim + 4;    // padded query row stride in shared memory (floats)
constexpr int kSegDocs = 128;         // documents per unit in the all-sets form

struct F32Args {
  const float* q;
  const int64_t* q_off;
  int n_queries;
  const float* docs;       // FP32 master [n_vecs * 128]
  const int64_t* doc_off;  // [n_sets + 1]
  int64_t n_sets;
  const int64_t* cand_off; // null: all sets
  const int64_t* cand_ids;
  float* scores;
  int* status;
};

// CH of query rows qs[0 .. m_q) (shared, stride kQStride) against one set.
// Called by a full warp; returns the score in every lane.
__device__ __forceinline__ float warp_chamfer(const float* __restrict__ qs, int m_q, const float* __restrict__ P,
                              int m_p, float* __restrict__ stage, float* __restrict__ rowmax,
                              float (&qr)[kDim], int& loaded_rg) {
  const int lane = threadIdx.x & 31;
  const int n_rg = (m_q + 31) >> 5;
  for (int rg = 0; rg < n_rg; ++rg) {
    if (rg != loaded_rg) {
      const int i = rg * 32 + lane;
#pragma unroll
      for (int k = 0; k < kDim; ++k) qr[k] = (i < m_q) ? qs[i * kQStride + k] : 0.f;
      loaded_rg = rg;
    }
    float best = -INFINITY;
    for (int j0 = 0; j0 < m_p; j0 += kVecBlock) {
      const int nv = min(kVecBlock, m_p - j0);
      __syncwarp();
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v) {
        if (v < nv) {
          float4 x = reinterpret_cast<const float4*>(P + (int64_t)(j0 + v) * kDim)[lane];
          reinterpret_cast<float4*>(stage + v * kDim)[lane] = x;
        }
      }
      __syncwarp();
      float acc[kVecBlock];
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v) acc[v] = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < kDim / 4; ++k4) {
#pragma unroll
        for (int v = 0; v < kVecBlock; ++v) {
          const float4 p = reinterpret_cast<const float4*>(stage + v * kDim)[k4];
          acc[v] = __fmaf_rn(qr[4 * k4 + 0], p.x, acc[v]);
          acc[v] = __fmaf_rn(qr[4 * k4 + 1], p.y, acc[v]);
          acc[v] = __fmaf_rn(qr[4 * k4 + 2], p.z, acc[v]);
          acc[v] = __fmaf_rn(qr[4 * k4 + 3], p.w, acc[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv) best = fmaxf(best, acc[v]);
    }
    const int i = rg * 32 + lane;
    if (i < m_q) rowmax[i] = best;
  }
  __syncwarp();
  float s = 0.f;
  if (lane == 0) {
    float c = 0.f;  // Kahan compensation
    for (int i = 0; i < m_q; ++i) {
      const float y = __fsub_rn(rowmax[i], c);
      const float t = __fadd_rn(s, y);
      c = __fsub_rn(__fsub_rn(t, s), y);
      s = t;
    }
  }
  return __shfl_sync(0xffffffffu, s, 0);
}

__global__ void __launch_bounds__(kF32Threads)
f32_score_kernel(F32Args a, int max_q_len) {
  extern __shared__ float sm[];
  float* qs = sm;                                              // [max_q_len * kQStride]
  float* stage_all = qs + max_q_len * kQStride;                // [warps][kVecBlock * 128]
  float* rowmax_all = stage_all + kF32Warps * kVecBlock * kDim;  // [warps][max_q_len]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + warp * kVecBlock * kDim;
  float* rowmax = rowmax_all + warp * max_q_len;
  float qr[kDim];

  const bool all_sets = (a.cand_ids == nullptr);
  const int64_t n_seg = all_sets ? (a.n_sets + kSegDocs - 1) / kSegDocs : 1;
  const int64_t n_units = all_sets ? n_seg * a.n_queries : a.n_queries;

  for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = (int)(all_sets ? (u % a.n_queries) : u);
    const int64_t q0 = a.q_off[b];
    const int m_q = (int)(a.q_off[b + 1] - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m_q * (kDim / 4); idx += blockDim.x) {
      const int i = idx / (kDim / 4), k4 = idx % (kDim / 4);
      float4 x = reinterpret_cast<const float4*>(a.q + (q0 + i) * kDim)[k4];
      reinterpret_cast<float4*>(qs + i * kQStride)[k4] = x;
    }
    __syncthreads();
    int loaded_rg = -1;
    int64_t t0, t1;
    if (all_sets) {
      const int64_t seg = u / a.n_queries;
      t0 = seg * kSegDocs;
      t1 = min(a.n_sets, t0 + kSegDocs);
    } else {
      t0 = a.cand_off[b];
      t1 = a.cand_off[b + 1];
    }
    for (int64_t t = t0 + warp; t < t1; t += kF32Warps) {
      const int64_t id = all_sets ? t : a.cand_ids[t];
      float score;
      if (id < 0) {
        score = -INFINITY;
      } else if (id >= a.n_sets) {
        if (lane == 0) set_status(a.status, kDevBounds);
        score = __int_as_float(0x7fc00000);
      } else {
        const int64_t r0 = a.doc_off[id];
        const int m_p = (int)(a.doc_off[id + 1] - r0);
        score = warp_chamfer(qs, m_q, a.docs + r0 * kDim, m_p, stage, rowmax, qr, loaded_rg);
      }
      if (lane == 0) {
        if (all_sets) a.scores[(int64_t)b * a.n_sets + t] = score;
        else a.scores[t] = score;
      }
    }
  }
}

}  // namespace

gem_status launch_f32_score(const gem_store* s, gem_workspace* ws, const float* q,
                            const int64_t* q_offsets, int32_t n_queries, const int64_t* cand_offsets,
                            const int64_t* cand_ids, int64_t n_cands, float* scores, cudaStream_t st) {
  (void)n_cands;
  F32Args a;
  a.q = q;
  a.q_off = q_offsets;
  a.n_queries = n_queries;
  a.docs = s->d_f32;
  a.doc_off = s->d_offsets;
  a.n_sets = s->n_sets;
  a.cand_off = cand_offsets;
  a.cand_ids = cand_ids;
  a.scores = scores;
  a.status = ws->d_status;
  const int mq = ws->max_q_len;
  const size_t smem = sizeof(float) * ((size_t)mq * kQStride + kF32Warps * kVecBlock * kDim +
                                       (size_t)kF32Warps * mq);
  GEM_CUDA_TRY(cudaFuncSetAttribute(f32_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32_score_kernel, kF32Threads,
                                                             smem));
  if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "f32 scoring kernel does not fit on an SM");
  int64_t units = cand_ids ? n_queries : ((s->n_sets + kSegDocs - 1) / kSegDocs) * n_queries;
  int grid = (int)std::min<int64_t>(units, (int64_t)s->n_sm * per_sm);
  if (grid < 1) return GEM_OK;
  f32_score_kernel<<<grid, kF32Threads, smem, st>>>(a, mq);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
