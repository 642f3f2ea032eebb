// Per-pair exact MaxSim on the SIMT pipes, shared by every FP32 scorer so that
// all of them produce bit-identical scores for the same (query, set) pair.
//
// Arithmetic order (fixed, independent of launch shape):
//   dot(q_i, p_j): one FP32 fused multiply-add chain over k = 0 .. 127
//   m_i = max_j dot(q_i, p_j)
//   CH  = Kahan (compensated) sum of m_i over i = 0 .. m_q - 1 in ascending order
//
// Mapping: lane = query row (32 rows per pass, the row's 128 components held in
// registers); the set's vectors are staged 8 at a time in the warp's shared
// slice and read as broadcasts.  In the codes form every stored vector p_j is
// replaced by its centroid C[code_j] (the caller stages centroids of the query
// codes as the query rows), which gives the quantized estimate in similarity form.
#pragma once
#include "internal.h"

namespace gem {

constexpr int kVecBlock = 8;        // set vectors staged per step
constexpr int kQStride = kDim + 4;  // padded query row stride in shared memory (floats)

// One row of the set (or its centroid in the codes form) as this lane's float4.
__device__ __forceinline__ float4 set_row4(const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                           const float* __restrict__ centroids, int j, int lane) {
  const float* src = row_code ? centroids + (int64_t)row_code[j] * kDim : P + (int64_t)j * kDim;
  return reinterpret_cast<const float4*>(src)[lane];
}

// CH of query rows qs[0 .. m_q) (row stride q_stride floats, shared or global
// memory) against one set.  Called by a full warp; returns the score in every
// lane.  P: the set's first row; row_code == nullptr: rows are P[j * 128],
// otherwise rows are centroids[row_code[j] * 128].  The next 8 set vectors are
// loaded into registers while the current 8 are multiplied, so the loads of a
// set overlap its arithmetic; the arithmetic order is unchanged.
template <bool CodedQ>
__device__ __forceinline__ float warp_chamfer_impl(const float* __restrict__ qs, int q_stride,
                                                   const int32_t* __restrict__ q_code, int m_q,
                                              const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                              const float* __restrict__ centroids, int m_p,
                                              float* __restrict__ stage, float* __restrict__ rowmax,
                                              float (&qr)[kDim], int& loaded_rg) {
  const int lane = threadIdx.x & 31;
  const int n_rg = (m_q + 31) >> 5;
  for (int rg = 0; rg < n_rg; ++rg) {
    if (rg != loaded_rg) {
      const int i = rg * 32 + lane;
#pragma unroll
      for (int k = 0; k < kDim; ++k) {
        if constexpr (CodedQ) qr[k] = (i < m_q) ? centroids[(int64_t)q_code[i] * kDim + k] : 0.f;
        else qr[k] = (i < m_q) ? qs[(int64_t)i * q_stride + k] : 0.f;
      }
      loaded_rg = rg;
    }
    float best = -INFINITY;
    float4 pf[kVecBlock];
    {
      const int nv0 = min(kVecBlock, m_p);
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv0) pf[v] = set_row4(P, row_code, centroids, v, lane);
    }
    for (int j0 = 0; j0 < m_p; j0 += kVecBlock) {
      const int nv = min(kVecBlock, m_p - j0);
      __syncwarp();
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv) reinterpret_cast<float4*>(stage + v * kDim)[lane] = pf[v];
      __syncwarp();
      const int j1 = j0 + kVecBlock;
      const int nv1 = min(kVecBlock, m_p - j1);
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv1) pf[v] = set_row4(P, row_code, centroids, j1 + v, lane);
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

__device__ __forceinline__ float warp_chamfer(const float* __restrict__ qs, int q_stride, int m_q,
                                              const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                              const float* __restrict__ centroids, int m_p,
                                              float* __restrict__ stage, float* __restrict__ rowmax,
                                              float (&qr)[kDim], int& loaded_rg) {
  return warp_chamfer_impl<false>(qs, q_stride, nullptr, m_q, P, row_code, centroids, m_p, stage, rowmax, qr,
                                  loaded_rg);
}

// Codes form with the query rows given as centroid indices (row i is
// centroids[q_code[i] * 128]).
__device__ __forceinline__ float warp_chamfer_coded_q(const float* __restrict__ centroids,
                                                      const int32_t* __restrict__ q_code, int m_q,
                                                      const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                                      int m_p, float* __restrict__ stage, float* __restrict__ rowmax,
                                                      float (&qr)[kDim], int& loaded_rg) {
  return warp_chamfer_impl<true>(nullptr, 0, q_code, m_q, P, row_code, centroids, m_p, stage, rowmax, qr,
                                 loaded_rg);
}

}  // namespace gem
