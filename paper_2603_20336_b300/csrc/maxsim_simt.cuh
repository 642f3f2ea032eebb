// Per-pair exact MaxSim on the SIMT pipes, shared by every FP32 scorer so that
// all of them produce bit-identical scores for the same (query, set) pair.
//
// Arithmetic order (fixed, independent of launch shape):
//   dot(q_i, p_j) = c0 + c1, c_h = e_h + o_h, where e_h and o_h are FP32 fused
//                   multiply-add chains over the even and the odd k of the half
//                   k in [64 h, 64 h + 64), each in ascending k (the two chains of
//                   a half advance together in packed two-lane FMAs)
//   m_i = max_j dot(q_i, p_j)
//   CH  = Kahan (compensated) sum of m_i over i = 0 .. m_q - 1 in ascending order
// With Sim = -(L2 distance) (the L2 form of Definition 1) the chains sum
// (q_ik - p_jk)^2 instead (the difference rounded, then one fused multiply-add),
// m_i = -sqrt(min_j d2(q_i, p_j)) with the correctly rounded square root, and the
// same Kahan sum follows.
//
// Mapping: lane l holds query rows 2(l/2) and 2(l/2)+1 of the current 32-row
// group, components k in [64 (l%2), 64 (l%2) + 64), in registers; the set's
// vectors are staged 8 at a time in the warp's shared slice (the upper half of a
// staged vector is shifted by 16 bytes so both half-warps' broadcast reads fall
// in different banks), so one 16-byte shared load feeds 4 packed FMAs (8
// products).  The query components are kept as packed pairs (k, k + 1).  The two
// halves of a dot meet through one xor shuffle.  In the codes form every
// stored vector p_j is replaced by its centroid C[code_j] and the query rows by
// the centroids of the query codes, which gives the quantized estimate in
// similarity form.
#pragma once
#include "internal.h"
#include "ptx.cuh"

namespace gem {

constexpr int kVecBlock = 8;         // set vectors staged per step
constexpr int kQStride = kDim + 4;   // padded query row stride in shared memory (floats)
constexpr int kStageStride = kDim + 4;  // staged set vector: [k 0..63][4 pad][k 64..127]

// Query registers of a lane: row a's 64 components as 32 packed pairs
// (k, k + 1), then row b's.
constexpr int kQPairs = kDim / 2;
constexpr int kRowPairs = kDim / 4;

// One block of up to kVecBlock staged set vectors against this lane's two query
// rows: best_a / best_b take the max of the block's dot products (L2: of the
// negated squared distances).
template <bool L2>
__device__ __forceinline__ void block_terms(const float* __restrict__ stage, int rd_off,
                                            const uint64_t (&qr)[kQPairs], int nv, float& best_a, float& best_b) {
  uint64_t acc_a[kVecBlock], acc_b[kVecBlock];  // packed (even k, odd k) chains
#pragma unroll
  for (int v = 0; v < kVecBlock; ++v) { acc_a[v] = 0ull; acc_b[v] = 0ull; }
#pragma unroll
  for (int k4 = 0; k4 < kDim / 8; ++k4) {
#pragma unroll
    for (int v = 0; v < kVecBlock; ++v) {
      // components (4 k4, 4 k4 + 1) and (4 k4 + 2, 4 k4 + 3) of this half
      const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(stage + v * kStageStride + rd_off + 4 * k4);
      if constexpr (L2) {
        uint64_t d = fsub2(qr[2 * k4], p.x);
        acc_a[v] = ffma2(d, d, acc_a[v]);
        d = fsub2(qr[2 * k4 + 1], p.y);
        acc_a[v] = ffma2(d, d, acc_a[v]);
        d = fsub2(qr[kRowPairs + 2 * k4], p.x);
        acc_b[v] = ffma2(d, d, acc_b[v]);
        d = fsub2(qr[kRowPairs + 2 * k4 + 1], p.y);
        acc_b[v] = ffma2(d, d, acc_b[v]);
      } else {
        acc_a[v] = ffma2(qr[2 * k4], p.x, acc_a[v]);
        acc_a[v] = ffma2(qr[2 * k4 + 1], p.y, acc_a[v]);
        acc_b[v] = ffma2(qr[kRowPairs + 2 * k4], p.x, acc_b[v]);
        acc_b[v] = ffma2(qr[kRowPairs + 2 * k4 + 1], p.y, acc_b[v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < kVecBlock; ++v) {
    const float ca = __fadd_rn(lo2(acc_a[v]), hi2(acc_a[v]));  // e_h + o_h
    const float cb = __fadd_rn(lo2(acc_b[v]), hi2(acc_b[v]));
    // c0 + c1 in the lane holding c0 and c1 + c0 in its partner: the same sum
    const float da = ca + __shfl_xor_sync(0xffffffffu, ca, 1);
    const float db = cb + __shfl_xor_sync(0xffffffffu, cb, 1);
    if (v < nv) {
      best_a = fmaxf(best_a, L2 ? -da : da);
      best_b = fmaxf(best_b, L2 ? -db : db);
    }
  }
}

// The per-query-vector term m_i from the block maxima.
template <bool L2>
__device__ __forceinline__ float row_term(float best) {
  return L2 ? -__fsqrt_rn(-best) : best;
}

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
template <bool CodedQ, bool L2>
__device__ __forceinline__ float warp_chamfer_impl(const float* __restrict__ qs, int q_stride,
                                                   const int32_t* __restrict__ q_code, int m_q,
                                                   const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                                   const float* __restrict__ centroids, int m_p,
                                                   float* __restrict__ stage, float* __restrict__ rowmax,
                                                   uint64_t (&qr)[kQPairs], int& loaded_rg) {
  const int lane = threadIdx.x & 31;
  const int half = lane & 1;           // component half of this lane
  const int pair = lane >> 1;          // query rows 2 pair, 2 pair + 1
  const int n_rg = (m_q + 31) >> 5;
  // where this lane's float4 of a set vector goes in the staged layout
  const int st_off = 4 * lane + (lane >= 16 ? 4 : 0);
  const int rd_off = half * (kDim / 2 + 4);
  for (int rg = 0; rg < n_rg; ++rg) {
    const int ia = rg * 32 + 2 * pair, ib = ia + 1;
    if (rg != loaded_rg) {
#pragma unroll
      for (int k2 = 0; k2 < kRowPairs; ++k2) {
        const int kk = half * (kDim / 2) + 2 * k2;
        if constexpr (CodedQ) {
          qr[k2] = (ia < m_q) ? pack2(centroids[(int64_t)q_code[ia] * kDim + kk],
                                      centroids[(int64_t)q_code[ia] * kDim + kk + 1]) : 0ull;
          qr[kRowPairs + k2] = (ib < m_q) ? pack2(centroids[(int64_t)q_code[ib] * kDim + kk],
                                                  centroids[(int64_t)q_code[ib] * kDim + kk + 1]) : 0ull;
        } else {
          qr[k2] = (ia < m_q) ? pack2(qs[(int64_t)ia * q_stride + kk], qs[(int64_t)ia * q_stride + kk + 1]) : 0ull;
          qr[kRowPairs + k2] =
              (ib < m_q) ? pack2(qs[(int64_t)ib * q_stride + kk], qs[(int64_t)ib * q_stride + kk + 1]) : 0ull;
        }
      }
      loaded_rg = rg;
    }
    float best_a = -INFINITY, best_b = -INFINITY;
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
        if (v < nv) *reinterpret_cast<float4*>(stage + v * kStageStride + st_off) = pf[v];
      __syncwarp();
      const int j1 = j0 + kVecBlock;
      const int nv1 = min(kVecBlock, m_p - j1);
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv1) pf[v] = set_row4(P, row_code, centroids, j1 + v, lane);
      block_terms<L2>(stage, rd_off, qr, nv, best_a, best_b);
    }
    if (half == 0 && ia < m_q) rowmax[ia] = row_term<L2>(best_a);
    if (half == 1 && ib < m_q) rowmax[ib] = row_term<L2>(best_b);
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

template <bool L2 = false>
__device__ __forceinline__ float warp_chamfer(const float* __restrict__ qs, int q_stride, int m_q,
                                              const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                              const float* __restrict__ centroids, int m_p,
                                              float* __restrict__ stage, float* __restrict__ rowmax,
                                              uint64_t (&qr)[kQPairs], int& loaded_rg) {
  return warp_chamfer_impl<false, L2>(qs, q_stride, nullptr, m_q, P, row_code, centroids, m_p, stage, rowmax, qr,
                                      loaded_rg);
}

// Codes form with the query rows given as centroid indices (row i is
// centroids[q_code[i] * 128]).
__device__ __forceinline__ float warp_chamfer_coded_q(const float* __restrict__ centroids,
                                                      const int32_t* __restrict__ q_code, int m_q,
                                                      const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                                      int m_p, float* __restrict__ stage, float* __restrict__ rowmax,
                                                      uint64_t (&qr)[kQPairs], int& loaded_rg) {
  return warp_chamfer_impl<true, false>(nullptr, 0, q_code, m_q, P, row_code, centroids, m_p, stage, rowmax, qr,
                                        loaded_rg);
}

}  // namespace gem
