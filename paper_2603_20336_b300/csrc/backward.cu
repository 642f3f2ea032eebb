// MaxSim forward with argmax side output, and its backward.
//
// Forward, per (query b, set d) pair: S = sum_i max_j <q_i, p_j> (Eq. 1) and
// j*(i) = argmax_j <q_i, p_j> (lowest j on ties).  Compute GEM_BF16 rounds every
// component of q and p to bfloat16 (nearest even) before the FP32 fused
// multiply-add chain over k; GEM_F32 uses the FP32 values.  The sum over i is a
// Kahan sum in ascending i.
//
// Backward, for an upstream gradient g[t] per pair t (the score is piecewise
// linear; the gradient is taken at the forward's argmax, treating the bf16
// rounding as the identity):
//   dL/dq_i   += g[t] * p_{j*(t,i)}                     (FP32 values of p)
//   dL/dp_j   += g[t] * sum over i with j*(t,i) = j of q_i
// grad_q is accumulated per query row over its query's pairs in ascending pair
// order (one FMA chain per output element, deterministic).  grad_docs: every row
// is written once by the set it belongs to; a set that occurs in exactly one
// pair gets its rows' sums written directly (no atomics, deterministic), a set
// in several pairs is zeroed and each pair adds its contribution with 16-byte
// atomic adds.
#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kFbWarps = 4;
constexpr int kFbStride = kDim + 4;
constexpr int kFbBlock = 8;

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct FwdArgs {
  const float* q;
  const int64_t* q_off;
  int n_queries;
  const float* docs;
  const int64_t* d_off;
  int64_t n_docs;
  const int64_t* pair_off;
  const int64_t* pair_ids;
  int bf16;
  int max_q_len;
  float* scores;
  int32_t* argmax;   // [n_pairs * max_q_len]
  int* status;
};

// One CTA per query (grid-stride), one warp per pair; lane = query row.
__global__ void __launch_bounds__(kFbWarps * 32) maxsim_fwd_kernel(FwdArgs a) {
  extern __shared__ float sm[];
  float* qs = sm;                                          // [max_q_len * kFbStride]
  float* stage_all = qs + a.max_q_len * kFbStride;         // [warps][kFbBlock * 128]
  float* rmax_all = stage_all + kFbWarps * kFbBlock * kDim;  // [warps][max_q_len]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + warp * kFbBlock * kDim;
  float* rmax = rmax_all + warp * a.max_q_len;
  for (int b = blockIdx.x; b < a.n_queries; b += gridDim.x) {
    const int64_t q0 = a.q_off[b];
    const int m_q = (int)(a.q_off[b + 1] - q0);
    __syncthreads();
    if (m_q < 1 || m_q > a.max_q_len) {
      if (threadIdx.x == 0) set_status(a.status, kDevInvalid);
      continue;
    }
    for (int idx = threadIdx.x; idx < m_q * kDim; idx += blockDim.x) {
      const int i = idx / kDim, k = idx % kDim;
      const float v = a.q[(q0 + i) * kDim + k];
      qs[i * kFbStride + k] = a.bf16 ? round_bf16(v) : v;
    }
    __syncthreads();
    for (int64_t t = a.pair_off[b] + warp; t < a.pair_off[b + 1]; t += kFbWarps) {
      const int64_t d = a.pair_ids[t];
      if (d < 0 || d >= a.n_docs) {
        if (lane == 0) {
          set_status(a.status, kDevBounds);
          a.scores[t] = __int_as_float(0x7fc00000);
        }
        continue;
      }
      const int64_t r0 = a.d_off[d];
      const int m_p = (int)(a.d_off[d + 1] - r0);
      for (int rg = 0; rg < (m_q + 31) / 32; ++rg) {
        const int i = rg * 32 + lane;
        float best = -INFINITY;
        int best_j = 0;
        for (int j0 = 0; j0 < m_p; j0 += kFbBlock) {
          const int nv = min(kFbBlock, m_p - j0);
          __syncwarp();
          for (int v = 0; v < nv; ++v) {
            float4 x = reinterpret_cast<const float4*>(a.docs + (r0 + j0 + v) * kDim)[lane];
            if (a.bf16) x = make_float4(round_bf16(x.x), round_bf16(x.y), round_bf16(x.z), round_bf16(x.w));
            reinterpret_cast<float4*>(stage + v * kDim)[lane] = x;
          }
          __syncwarp();
          if (i < m_q) {
            for (int v = 0; v < nv; ++v) {
              float acc = 0.f;
#pragma unroll 8
              for (int k = 0; k < kDim; ++k) acc = __fmaf_rn(qs[i * kFbStride + k], stage[v * kDim + k], acc);
              if (acc > best) { best = acc; best_j = j0 + v; }
            }
          }
        }
        if (i < m_q) {
          rmax[i] = best;
          a.argmax[t * a.max_q_len + i] = best_j;
        }
      }
      __syncwarp();
      if (lane == 0) {
        float s = 0.f, c = 0.f;
        for (int i = 0; i < m_q; ++i) {
          const float y = __fsub_rn(rmax[i], c);
          const float tt = __fadd_rn(s, y);
          c = __fsub_rn(__fsub_rn(tt, s), y);
          s = tt;
        }
        a.scores[t] = s;
      }
      __syncwarp();
    }
  }
}

struct BwdArgs {
  const float* q;
  const int64_t* q_off;
  int n_queries;
  const float* docs;
  const int64_t* d_off;
  int64_t n_docs;
  const int64_t* pair_off;
  const int64_t* pair_ids;
  const int32_t* argmax;
  int max_q_len;
  const float* g;
  float* grad_q;
  float* grad_docs;
};

// grad_q: one warp per query row (row i of query b), lane = 4 components.  The
// query's pairs are taken 32 at a time: lane l loads pair t0 + l's set row
// (through the argmax) and weight in parallel, then the warp adds the rows in
// ascending pair order, eight rows' loads in flight at a time.
__global__ void __launch_bounds__(256) maxsim_bwd_q_kernel(BwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_slots = (int64_t)a.n_queries * a.max_q_len;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < n_slots; w += n_warps) {
    const int b = (int)(w / a.max_q_len);
    const int i = (int)(w % a.max_q_len);
    const int64_t q0 = a.q_off[b];
    if (i >= a.q_off[b + 1] - q0) continue;  // warp-uniform
    const int64_t r = q0 + i;
    const int64_t t_end = a.pair_off[b + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t t0 = a.pair_off[b]; t0 < t_end; t0 += 32) {
      const int cnt = (int)min((int64_t)32, t_end - t0);
      int64_t row = -1;  // set row of pair t0 + lane, -1: skipped
      float gt = 0.f;
      if (lane < cnt) {
        const int64_t t = t0 + lane;
        const int64_t d = a.pair_ids[t];
        if (d >= 0 && d < a.n_docs) {
          const int64_t s0 = a.d_off[d];
          const int j = a.argmax[t * a.max_q_len + i];
          if (j >= 0 && j < a.d_off[d + 1] - s0) {  // an argmax outside the set adds nothing
            row = s0 + j;
            gt = a.g[t];
          }
        }
      }
      for (int e0 = 0; e0 < cnt; e0 += 8) {
        float4 p[8];
        float w[8];
        bool v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u;
          const int64_t re = __shfl_sync(0xffffffffu, (long long)row, e & 31);
          w[u] = __shfl_sync(0xffffffffu, gt, e & 31);
          v[u] = e < cnt && re >= 0;
          p[u] = v[u] ? reinterpret_cast<const float4*>(a.docs + re * kDim)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (v[u]) {
            acc.x = __fmaf_rn(w[u], p[u].x, acc.x);
            acc.y = __fmaf_rn(w[u], p[u].y, acc.y);
            acc.z = __fmaf_rn(w[u], p[u].z, acc.z);
            acc.w = __fmaf_rn(w[u], p[u].w, acc.w);
          }
        }
      }
    }
    reinterpret_cast<float4*>(a.grad_q + r * kDim)[lane] = acc;
  }
}

// grad_docs: one CTA per pair (grid-stride over queries' pairs); thread per
// (set row j, 4 components): sum of q_i over the rows i whose argmax is j.
__global__ void __launch_bounds__(256) maxsim_bwd_p_kernel(BwdArgs a, int64_t n_pairs) {
  __shared__ int js[256];
  for (int64_t t = blockIdx.x; t < n_pairs; t += gridDim.x) {
    // query of pair t
    int lo = 0, hi = a.n_queries - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.pair_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const int64_t d = a.pair_ids[t];
    if (d < 0 || d >= a.n_docs) continue;
    const int64_t q0 = a.q_off[b];
    const int m_q = (int)(a.q_off[b + 1] - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < m_q; i += blockDim.x) js[i] = a.argmax[t * a.max_q_len + i];
    __syncthreads();
    const int64_t r0 = a.d_off[d];
    const int m_p = (int)(a.d_off[d + 1] - r0);
    const float gt = a.g[t];
    for (int idx = threadIdx.x; idx < m_p * (kDim / 4); idx += blockDim.x) {
      const int j = idx / (kDim / 4), k4 = idx % (kDim / 4);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      bool any = false;
      for (int i = 0; i < m_q; ++i) {
        if (js[i] != j) continue;
        const float4 qv = reinterpret_cast<const float4*>(a.q + (q0 + i) * kDim)[k4];
        acc.x += qv.x; acc.y += qv.y; acc.z += qv.z; acc.w += qv.w;
        any = true;
      }
      if (any) {
        float* out = a.grad_docs + (r0 + j) * kDim + 4 * k4;
        atomicAdd(out + 0, gt * acc.x);
        atomicAdd(out + 1, gt * acc.y);
        atomicAdd(out + 2, gt * acc.z);
        atomicAdd(out + 3, gt * acc.w);
      }
    }
  }
}

// The sort of a pair's (j*(i), i) keys, key = j * 32 + i (rows past m_q last):
// rows sharing an argmax row j become adjacent, in ascending i.
__device__ __forceinline__ uint32_t sorted_argmax_key(const BwdArgs& a, int64_t t, int m_q, int lane) {
  uint32_t key = lane < m_q ? ((uint32_t)a.argmax[t * a.max_q_len + lane] << 5) | (uint32_t)lane : 0xFFFFFFFFu;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const uint32_t other = __shfl_xor_sync(0xffffffffu, key, stride);
      const bool up = ((lane & size) == 0);
      const bool lower = ((lane & stride) == 0);
      key = (lower == up) ? min(key, other) : max(key, other);
    }
  }
  return key;
}

// grad_docs for query sets of at most 32 rows: one warp per pair.  The pair's
// (j*(i), i) are sorted by a warp bitonic sort, so the rows sharing an argmax
// row j are adjacent; lane k4 then walks the sorted rows in order, sums q_i's
// components 4 k4 .. 4 k4 + 3 over each run (ascending i, as the CTA-per-pair
// kernel does) and adds g_t times the sum to row j with one 16-byte atomic.
__global__ void __launch_bounds__(256) maxsim_bwd_p_warp_kernel(BwdArgs a, int64_t n_pairs, const int* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < n_pairs; t += n_warps) {
    int lo = 0, hi = a.n_queries - 1;  // query of pair t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.pair_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const int64_t d = a.pair_ids[t];
    if (d < 0 || d >= a.n_docs) continue;  // warp-uniform
    if (cnt != nullptr && cnt[d] < 2) continue;  // written by its owner
    const int64_t q0 = a.q_off[b];
    const int m_q = (int)(a.q_off[b + 1] - q0);
    if (m_q < 1 || m_q > 32) continue;
    const int64_t r0 = a.d_off[d];
    const int64_t m_p = a.d_off[d + 1] - r0;
    const float gt = a.g[t];
    const uint32_t key = sorted_argmax_key(a, t, m_q, lane);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = 0; e < m_q; ++e) {
      const uint32_t ke = __shfl_sync(0xffffffffu, key, e);
      const uint32_t kn = __shfl_sync(0xffffffffu, key, (e + 1) & 31);
      const int i = (int)(ke & 31u);
      const int64_t j = (int64_t)(ke >> 5);
      const float4 qv = reinterpret_cast<const float4*>(a.q + (q0 + i) * kDim)[lane];
      acc.x += qv.x; acc.y += qv.y; acc.z += qv.z; acc.w += qv.w;
      if ((e + 1 == m_q || (int64_t)(kn >> 5) != j) && j < m_p) {
        atomicAdd(reinterpret_cast<float4*>(a.grad_docs + (r0 + j) * kDim) + lane,
                  make_float4(gt * acc.x, gt * acc.y, gt * acc.z, gt * acc.w));
        acc = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}


// How many valid pairs name each set, and (when exactly one does) which.
__global__ void bwd_set_owner_kernel(BwdArgs a, int64_t n_pairs, int* cnt, int64_t* owner) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_pairs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = a.pair_ids[t];
    if (d < 0 || d >= a.n_docs) continue;
    atomicAdd(cnt + d, 1);
    owner[d] = t;  // meaningful only where the count ends at 1
  }
}

// grad_docs, query sets of at most 32 rows: one warp per set, every row of the
// set written once.  A set named by exactly one pair t: the pair's sorted
// (j*, i) keys are walked along the set's rows in order; a row that is the
// argmax of query rows i gets g_t times their sum (ascending i), any other row
// 0.  Any other set: zeros (the atomic pass adds the pairs of sets named more
// than once).  Rows outside the sets' range are zeroed too.
__global__ void __launch_bounds__(256) maxsim_bwd_p_owner_kernel(BwdArgs a, int64_t n_doc_rows, const int* cnt,
                                                                 const int64_t* owner) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  for (int64_t d = gw; d < a.n_docs; d += n_warps) {
    const int64_t r0 = a.d_off[d];
    const int64_t m_p = a.d_off[d + 1] - r0;
    float4* out = reinterpret_cast<float4*>(a.grad_docs + r0 * kDim) + lane;
    int m_q = 0;
    int64_t q0 = 0, t = -1;
    if (cnt[d] == 1) {
      t = owner[d];
      int lo = 0, hi = a.n_queries - 1;  // query of pair t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.pair_off[mid] <= t) lo = mid; else hi = mid - 1;
      }
      q0 = a.q_off[lo];
      m_q = (int)(a.q_off[lo + 1] - q0);
      if (m_q > 32) m_q = 0;
    }
    if (m_q < 1) {
      for (int64_t j = 0; j < m_p; ++j) out[j * (kDim / 4)] = zero;
      continue;
    }
    const float gt = a.g[t];
    const uint32_t key = sorted_argmax_key(a, t, m_q, lane);
    int e = 0;
    uint32_t ke = __shfl_sync(0xffffffffu, key, 0);
    for (int64_t j = 0; j < m_p; ++j) {
      float4 acc = zero;
      bool hit = false;
      while (e < m_q && (int64_t)(ke >> 5) == j) {
        const float4 qv = reinterpret_cast<const float4*>(a.q + (q0 + (ke & 31u)) * kDim)[lane];
        acc.x += qv.x; acc.y += qv.y; acc.z += qv.z; acc.w += qv.w;
        hit = true;
        ++e;
        ke = __shfl_sync(0xffffffffu, key, e & 31);
      }
      out[j * (kDim / 4)] = hit ? make_float4(gt * acc.x, gt * acc.y, gt * acc.z, gt * acc.w) : zero;
    }
  }
  // rows before the first set and after the last
  const int64_t lo_end = a.d_off[0], hi_begin = a.d_off[a.n_docs];
  for (int64_t row = gw; row < lo_end; row += n_warps)
    reinterpret_cast<float4*>(a.grad_docs + row * kDim)[lane] = zero;
  for (int64_t row = hi_begin + gw; row < n_doc_rows; row += n_warps)
    reinterpret_cast<float4*>(a.grad_docs + row * kDim)[lane] = zero;
}

}  // namespace

gem_status launch_maxsim_fwd(const float* q, const int64_t* q_off, int32_t n_queries, const float* docs,
                             const int64_t* d_off, int64_t n_docs, const int64_t* pair_off,
                             const int64_t* pair_ids, int32_t max_q_len, int bf16, float* scores,
                             int32_t* argmax, int* status, int n_sm, cudaStream_t st) {
  FwdArgs a{q, q_off, n_queries, docs, d_off, n_docs, pair_off, pair_ids, bf16, max_q_len, scores, argmax, status};
  const size_t smem = sizeof(float) * ((size_t)max_q_len * kFbStride + kFbWarps * kFbBlock * kDim +
                                       (size_t)kFbWarps * max_q_len);
  GEM_CUDA_TRY(cudaFuncSetAttribute(maxsim_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(n_queries, n_sm * 8);
  maxsim_fwd_kernel<<<grid, kFbWarps * 32, smem, st>>>(a);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_maxsim_bwd(const float* q, const int64_t* q_off, int32_t n_queries, const float* docs,
                             const int64_t* d_off, int64_t n_docs, int64_t n_doc_rows, const int64_t* pair_off,
                             const int64_t* pair_ids, int64_t n_pairs, const int32_t* argmax, int32_t max_q_len,
                             const float* g, float* grad_q, float* grad_docs, int n_sm, cudaStream_t st) {
  BwdArgs a{q, q_off, n_queries, docs, d_off, n_docs, pair_off, pair_ids, argmax, max_q_len, g, grad_q, grad_docs};
  if (grad_q) {
    const int64_t warps = (int64_t)n_queries * max_q_len;
    maxsim_bwd_q_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)n_sm * 16)), 256, 0,
                          st>>>(a);
    GEM_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  if (grad_docs && n_pairs > 0 && max_q_len <= 32) {
    // every row written once by its set: counts and owners, the owners' rows
    // (zeros elsewhere), then the atomic adds of sets named by several pairs
    uint8_t* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), (size_t)n_docs * 12 + 16, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(GEM_ERR_OOM, "scratch of the backward");
    }
    int64_t* owner = reinterpret_cast<int64_t*>(scratch);
    int* cnt = reinterpret_cast<int*>(scratch + (size_t)n_docs * 8);
    e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_docs, st);
    if (e == cudaSuccess) {
      bwd_set_owner_kernel<<<(int)std::min<int64_t>((n_pairs + 255) / 256, (int64_t)n_sm * 8), 256, 0, st>>>(
          a, n_pairs, cnt, owner);
      maxsim_bwd_p_owner_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_docs + 7) / 8, (int64_t)n_sm * 16)),
                                  256, 0, st>>>(a, n_doc_rows, cnt, owner);
      maxsim_bwd_p_warp_kernel<<<(int)std::min<int64_t>((n_pairs + 7) / 8, (int64_t)n_sm * 16), 256, 0, st>>>(
          a, n_pairs, cnt);
      e = cudaGetLastError();
      note_launches(3);
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "backward grad_docs launches");
  } else if (grad_docs) {
    GEM_CUDA_TRY(cudaMemsetAsync(grad_docs, 0, sizeof(float) * n_doc_rows * kDim, st));
    if (n_pairs > 0) {
      maxsim_bwd_p_kernel<<<(int)std::min<int64_t>(n_pairs, (int64_t)n_sm * 16), 256, 0, st>>>(a, n_pairs);
      GEM_CUDA_TRY(cudaGetLastError());
      note_launches(1);
    }
  }
  return GEM_OK;
}

}  // namespace gem
