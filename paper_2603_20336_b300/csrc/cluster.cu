// Cluster filter (Sec. 4.5.1, Eq. 15; Algorithm 5, first two steps).
//
// The relevance S = C_index Q^T scores every coarse centroid against every query
// vector; each query vector keeps its top-t centroids (largest inner product, ties
// to the lower centroid index) and C_query is the union over the query set's
// vectors, returned as a bitmask over the k2 centroids and as a sorted id list.
//
// One CTA per query set, kCfWarps warps.  The query vectors (32 per pass) and the
// centroids (tiles of kCfTile) pass through shared memory with a padded row stride,
// so that the float4 reads of 8 lanes fall in distinct banks.  Warp w takes the
// pass's query vectors w, w + 8, w + 16, w + 24; lane l scores centroids l and
// l + 32 of every tile, each dot one FP32 fused multiply-add chain over
// k = 0 .. 127 in order, and keeps its own top-t of each of its vectors in
// registers.  After the last tile the warp merges the 32 lists of a vector with t
// rounds of a warp arg-max and sets the winners' bits in the set's bitmask.
#include <cuda_runtime.h>

#include "internal.h"

namespace gem {
namespace {

constexpr int kCfWarps = 8;
constexpr int kCfThreads = kCfWarps * 32;
constexpr int kCfTile = 64;              // centroids per shared-memory tile
constexpr int kCfRows = 32;              // query vectors per pass
constexpr int kCfStride = kDim + 4;      // padded row stride (floats)
constexpr int kCfRowsPerWarp = kCfRows / kCfWarps;
constexpr int kCfMaxT = 8;               // largest t

// (v, i) ranks before (w, j): larger value, then lower index
__device__ __forceinline__ bool cf_before(float v, int i, float w, int j) {
  return v > w || (v == w && i < j);
}

template <int T>
__global__ void __launch_bounds__(kCfThreads)
cluster_filter_kernel(const float* __restrict__ q, const int64_t* __restrict__ q_off, int n_queries,
                      const float* __restrict__ C, int k2, int words, int cap,
                      uint32_t* __restrict__ out_mask, int32_t* __restrict__ out_list,
                      int32_t* __restrict__ out_count) {
  extern __shared__ float cf_smem[];
  float* qs = cf_smem;                                    // [kCfRows][kCfStride]
  float* cs = qs + kCfRows * kCfStride;                   // [kCfTile][kCfStride]
  uint32_t* mask = reinterpret_cast<uint32_t*>(cs + kCfTile * kCfStride);  // [words]
  __shared__ int scan[kCfThreads];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int b = blockIdx.x; b < n_queries; b += gridDim.x) {
    const int64_t r0 = q_off[b];
    const int m_q = (int)(q_off[b + 1] - r0);
    for (int w = threadIdx.x; w < words; w += kCfThreads) mask[w] = 0u;

    for (int p0 = 0; p0 < m_q; p0 += kCfRows) {
      const int np = min(kCfRows, m_q - p0);
      __syncthreads();  // previous pass done with qs (and the mask is cleared)
      for (int idx = threadIdx.x; idx < np * (kDim / 4); idx += kCfThreads) {
        const int i = idx / (kDim / 4), k4 = idx % (kDim / 4);
        reinterpret_cast<float4*>(qs + i * kCfStride)[k4] =
            reinterpret_cast<const float4*>(q + (r0 + p0 + i) * kDim)[k4];
      }
      // this lane's top-t of each of its vectors (sorted, value desc / index asc)
      float val[kCfRowsPerWarp][T];
      int id[kCfRowsPerWarp][T];
#pragma unroll
      for (int r = 0; r < kCfRowsPerWarp; ++r)
#pragma unroll
        for (int j = 0; j < T; ++j) { val[r][j] = -INFINITY; id[r][j] = 0x7fffffff; }

      for (int c0 = 0; c0 < k2; c0 += kCfTile) {
        const int nc = min(kCfTile, k2 - c0);
        __syncthreads();  // everyone done with the previous tile
        for (int idx = threadIdx.x; idx < nc * (kDim / 4); idx += kCfThreads) {
          const int i = idx / (kDim / 4), k4 = idx % (kDim / 4);
          reinterpret_cast<float4*>(cs + i * kCfStride)[k4] =
              reinterpret_cast<const float4*>(C + (int64_t)(c0 + i) * kDim)[k4];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kCfRowsPerWarp; ++r) {
          const int row = warp + r * kCfWarps;
          if (row >= np) continue;  // warp-uniform
          const float* qr = qs + row * kCfStride;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c >= nc) continue;
            const float* cr = cs + c * kCfStride;
            float acc = 0.f;
#pragma unroll 8
            for (int k4 = 0; k4 < kDim / 4; ++k4) {
              const float4 a = reinterpret_cast<const float4*>(qr)[k4];
              const float4 x = reinterpret_cast<const float4*>(cr)[k4];
              acc = __fmaf_rn(a.x, x.x, acc);
              acc = __fmaf_rn(a.y, x.y, acc);
              acc = __fmaf_rn(a.z, x.z, acc);
              acc = __fmaf_rn(a.w, x.w, acc);
            }
            // insert (indices arrive in increasing order per lane, so an equal
            // value goes after the entries already kept)
            if (acc > val[r][T - 1]) {
              float cv = acc;
              int ci = c0 + c;
#pragma unroll
              for (int j = 0; j < T; ++j) {
                if (cv > val[r][j]) {
                  const float tv = val[r][j];
                  const int ti = id[r][j];
                  val[r][j] = cv;
                  id[r][j] = ci;
                  cv = tv;
                  ci = ti;
                }
              }
            }
          }
        }
      }
      // merge the 32 lists of each vector: t rounds of a warp arg-max
#pragma unroll
      for (int r = 0; r < kCfRowsPerWarp; ++r) {
        const int row = warp + r * kCfWarps;
        if (row >= np) continue;  // warp-uniform
#pragma unroll
        for (int round = 0; round < T; ++round) {
          float bv = val[r][0];
          int bi = id[r][0];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (cf_before(ov, oi, bv, bi)) { bv = ov; bi = oi; }
          }
          if (bi == 0x7fffffff) break;  // fewer than t centroids (cannot happen for t <= k2)
          if (id[r][0] == bi) {
            // the winning lane drops its head
#pragma unroll
            for (int j = 0; j + 1 < T; ++j) { val[r][j] = val[r][j + 1]; id[r][j] = id[r][j + 1]; }
            val[r][T - 1] = -INFINITY;
            id[r][T - 1] = 0x7fffffff;
          }
          if (lane == 0) atomicOr(&mask[bi >> 5], 1u << (bi & 31));
        }
      }
    }
    __syncthreads();
    // bitmask out; sorted ids via a block scan over per-thread word ranges
    uint32_t* om = out_mask + (int64_t)b * words;
    for (int w = threadIdx.x; w < words; w += kCfThreads) om[w] = mask[w];
    const int per = (words + kCfThreads - 1) / kCfThreads;
    const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(mask[w]);
    scan[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int i = 0; i < kCfThreads; ++i) { const int c = scan[i]; scan[i] = run; run += c; }
      out_count[b] = run;
    }
    __syncthreads();
    int pos = scan[threadIdx.x];
    int32_t* ol = out_list + (int64_t)b * cap;
    for (int w = w0; w < w1; ++w) {
      uint32_t bits = mask[w];
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        if (pos < cap) ol[pos] = w * 32 + bit;
        ++pos;
      }
    }
    __syncthreads();  // the mask is cleared for the next query set only after this
  }
}

}  // namespace

gem_status launch_cluster_filter(const float* q, const int64_t* q_offsets, int32_t n_queries, const float* centroids,
                                 int32_t k2, int32_t t, int32_t cap, uint32_t* out_mask, int32_t* out_list,
                                 int32_t* out_count, int n_sm, cudaStream_t st) {
  const int words = (k2 + 31) / 32;
  const size_t smem = sizeof(float) * (size_t)(kCfRows + kCfTile) * kCfStride + sizeof(uint32_t) * (size_t)words;
  if (n_queries == 0) return GEM_OK;
  const int grid = std::min(n_queries, n_sm * 4);
  auto go = [&](auto kern) -> gem_status {
    GEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kCfThreads, smem, st>>>(q, q_offsets, n_queries, centroids, k2, words, cap, out_mask, out_list,
                                         out_count);
    GEM_CUDA_TRY(cudaGetLastError());
    return GEM_OK;
  };
  gem_status r;
  switch (t) {
    case 1: r = go(cluster_filter_kernel<1>); break;
    case 2: r = go(cluster_filter_kernel<2>); break;
    case 3: r = go(cluster_filter_kernel<3>); break;
    case 4: r = go(cluster_filter_kernel<4>); break;
    case 5: r = go(cluster_filter_kernel<5>); break;
    case 6: r = go(cluster_filter_kernel<6>); break;
    case 7: r = go(cluster_filter_kernel<7>); break;
    case 8: r = go(cluster_filter_kernel<8>); break;
    default: return fail(GEM_ERR_INVALID, "t must be 1..8");
  }
  if (r != GEM_OK) return r;
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
