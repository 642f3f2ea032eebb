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

#include <algorithm>
#include <cstdint>

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

// ---------------------------------------------------------------------------
// Cluster members and multi-entry points (Sec. 4.1.1 Eq. 4, Sec. 4.5.2,
// Algorithm 5): every stored vector's nearest C_index centroid, per cluster the
// sets of its vectors, and for a query's C_query one random member set per
// cluster.  The draw for (query b, cluster c) is the member s with the smallest
// H(seed, b, c, s) (then the lower s), H = out(out(out(seed + b) + c) + s) with
// out(x) one SplitMix64 output from state x; the minimum does not depend on the
// order (or repetition) of the members, so the lists are built with atomics.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t splitmix_out(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void count_codes_kernel(const int32_t* __restrict__ codes, int64_t n, int64_t* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(counts + codes[i]), 1ull);
}

// exclusive scan of counts [k] into off [k + 1] by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) scan_counts_kernel(const int64_t* __restrict__ counts, int k,
                                                         int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  __shared__ int64_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < k; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    const int64_t v = c < k ? counts[c] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // Hillis-Steele inclusive scan
      const int64_t add = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (c < k) off[c] = base + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) base += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[k] = base;
}

// one warp per set: every vector of set `d` adds d to the member list of its cluster
__global__ void scatter_members_kernel(const int32_t* __restrict__ codes, const int64_t* __restrict__ offsets,
                                       int64_t n_sets, const int64_t* __restrict__ member_off,
                                       int64_t* __restrict__ cursor, int32_t* __restrict__ members) {
  const int lane = threadIdx.x & 31;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < n_sets;
       d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    for (int64_t v = offsets[d] + lane; v < offsets[d + 1]; v += 32) {
      const int c = codes[v];
      const int64_t pos = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + c), 1ull);
      members[member_off[c] + pos] = (int32_t)d;
    }
  }
}

// one warp per (query b, slot j): the draw for cluster lists[b * stride + j]
__global__ void entry_points_kernel(const int32_t* __restrict__ lists, const int32_t* __restrict__ counts,
                                    int n_queries, int stride, const int64_t* __restrict__ member_off,
                                    const int32_t* __restrict__ members, int k2, uint64_t seed,
                                    int64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t n_items = (int64_t)n_queries * stride;
  for (int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; it < n_items;
       it += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int b = (int)(it / stride), j = (int)(it % stride);
    int64_t pick = -1;
    if (j < counts[b]) {
      const int c = lists[it];
      if (c >= 0 && c < k2) {
        const uint64_t h2 = splitmix_out(splitmix_out(seed + (uint64_t)b) + (uint64_t)c);
        uint64_t best_h = ~0ull;
        int64_t best_s = INT64_MAX;
        for (int64_t m = member_off[c] + lane; m < member_off[c + 1]; m += 32) {
          const int64_t sidx = members[m];
          const uint64_t h = splitmix_out(h2 + (uint64_t)sidx);
          if (h < best_h || (h == best_h && sidx < best_s)) { best_h = h; best_s = sidx; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const uint64_t oh = __shfl_xor_sync(0xffffffffu, best_h, o);
          const int64_t os = __shfl_xor_sync(0xffffffffu, best_s, o);
          if (oh < best_h || (oh == best_h && os < best_s)) { best_h = oh; best_s = os; }
        }
        pick = best_s == INT64_MAX ? -1 : best_s;
      }
    }
    if (lane == 0) out[it] = pick;
  }
}

}  // namespace

gem_status launch_cluster_index(gem_store* s, cudaStream_t st) {
  int64_t* counts = nullptr;
  if (cudaMalloc(&counts, sizeof(int64_t) * s->k2) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEM_ERR_OOM, "cluster counts");
  }
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * s->k2, st);
  if (e == cudaSuccess) {
    count_codes_kernel<<<1024, 256, 0, st>>>(s->d_icodes, s->n_vecs, counts);
    scan_counts_kernel<<<1, 1024, 0, st>>>(counts, s->k2, s->d_member_off);
    e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * s->k2, st);
  }
  if (e == cudaSuccess) {
    scatter_members_kernel<<<1024, 256, 0, st>>>(s->d_icodes, s->d_offsets, s->n_sets, s->d_member_off, counts,
                                                  s->d_members);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(counts);
  if (e != cudaSuccess) return cuda_fail(e, "cluster members");
  note_launches(3);
  return GEM_OK;
}

gem_status launch_entry_points(const gem_store* s, const int32_t* lists, const int32_t* counts, int32_t n_queries,
                               int32_t stride, uint64_t seed, int64_t* out, cudaStream_t st) {
  const int64_t warps = (int64_t)n_queries * stride;
  if (warps == 0) return GEM_OK;
  const int grid = (int)std::min<int64_t>((warps + 7) / 8, 4096);
  entry_points_kernel<<<grid, 256, 0, st>>>(lists, counts, n_queries, stride, s->d_member_off, s->d_members, s->k2,
                                            seed, out);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

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
