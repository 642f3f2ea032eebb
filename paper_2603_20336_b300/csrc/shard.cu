// Doc-range sharding of the store: the k-argmax of Eq. 2 over a database D
// split by set id into contiguous ranges, one store per shard (one GPU each, or
// several on one GPU).
//
// Protocol (exact: the result is bit for bit that of gem_search on the whole
// store, because every (query, set) score depends on the two sets alone):
//   1. gem_shard_first_pass on every shard: first-pass scores of the shard's
//      sets and their top `depth` per query, ids made global (+ id_base);
//   2. the per-shard lists are gathered shard-major [n_shards][n_queries][depth]
//      and gem_merge_topk keeps the top `depth` of their union per query: the
//      whole store's rerank pool, since every member of it is in its own
//      shard's top `depth`;
//   3. gem_shard_rerank on every shard writes the exact FP32 score of the pool
//      entries the shard owns (the others keep the -inf the caller filled in);
//      across GPUs an element-wise max combines them;
//   4. gem_topk of the pool scores with the pool ids gives the top k.
// Candidate lists (the scoring step of a beam expansion, Algorithm 5) are
// routed the same way: every shard scores the listed ids it owns
// (gem_shard_score_ids) into a buffer filled with -inf, and an element-wise max
// across shards gives gem_score_ids on the whole store.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace gem {
namespace {

__global__ void offset_ids_kernel(int64_t* __restrict__ ids, int64_t n, int64_t base) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (ids[i] >= 0) ids[i] += base;
}

// global -> local ids of this shard; entries it does not own become -1
__global__ void local_ids_kernel(const int64_t* __restrict__ g, int64_t n, int64_t base, int64_t n_sets,
                                 int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = g[i] - base;
    out[i] = (g[i] >= 0 && l >= 0 && l < n_sets) ? l : -1;
  }
}

// the owned entries' scores into out; the rest of out is left as it is
__global__ void scatter_owned_kernel(const int64_t* __restrict__ local, const float* __restrict__ sc, int64_t n,
                                     float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (local[i] >= 0) out[i] = sc[i];
}

int grid_for(int64_t n, int n_sm) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, n_sm * 8)); }

}  // namespace
}  // namespace gem

using namespace gem;

extern "C" {

gem_status gem_shard_ranges(const int64_t* offsets_host, int64_t n_sets, int32_t n_shards, int64_t* bounds_host) {
  GEM_NVTX_RANGE("gem_shard_ranges");
  if (!offsets_host || !bounds_host) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_sets < 1 || n_shards < 1 || n_shards > n_sets) return fail(GEM_ERR_INVALID, "need 1 <= n_shards <= n_sets");
  if (offsets_host[0] != 0) return fail(GEM_ERR_INVALID, "offsets[0] != 0");
  for (int64_t i = 0; i < n_sets; ++i)
    if (offsets_host[i + 1] <= offsets_host[i]) return fail(GEM_ERR_INVALID, "empty or non-monotone set");
  const int64_t V = offsets_host[n_sets];
  bounds_host[0] = 0;
  for (int32_t s = 1; s < n_shards; ++s) {
    // the set boundary closest to s/n_shards of the vectors, every shard non-empty
    const int64_t target = V / n_shards * s + (V % n_shards) * s / n_shards;
    int64_t b = std::lower_bound(offsets_host, offsets_host + n_sets + 1, target) - offsets_host;
    if (b > 0 && target - offsets_host[b - 1] < offsets_host[b] - target) --b;
    b = std::max(b, bounds_host[s - 1] + 1);
    b = std::min(b, n_sets - (n_shards - s));
    bounds_host[s] = b;
  }
  bounds_host[n_shards] = n_sets;
  return GEM_OK;
}

gem_status gem_shard_first_pass(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                                int32_t n_queries, int64_t n_q_rows, int32_t compute, int32_t depth, int64_t id_base,
                                int64_t* out_ids, float* out_scores, void* stream) {
  GEM_NVTX_RANGE("gem_shard_first_pass");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!out_ids || !out_scores) return fail(GEM_ERR_INVALID, "NULL output");
  if (!w->d_scores) return fail(GEM_ERR_STATE, "workspace was created with max_k = 0");
  if (depth < 1 || depth > kMaxK) return fail(GEM_ERR_INVALID, "depth must be 1..4096");
  if (id_base < 0) return fail(GEM_ERR_INVALID, "id_base < 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  r = search_first_pass(s, w, q, q_offsets, n_queries, n_q_rows, compute, st);
  if (r != GEM_OK) return r;
  r = launch_topk(w, w->d_scores, nullptr, n_queries, s->n_sets, nullptr, depth, out_ids, out_scores, st);
  if (r != GEM_OK) return r;
  if (id_base > 0) {
    const int64_t n = (int64_t)n_queries * depth;
    offset_ids_kernel<<<grid_for(n, s->n_sm), 256, 0, st>>>(out_ids, n, id_base);
    GEM_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  return GEM_OK;
}

gem_status gem_shard_rerank(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                            int32_t n_queries, int64_t n_q_rows, const int64_t* pool_ids, int32_t depth,
                            int64_t id_base, float* pool_scores, void* stream) {
  GEM_NVTX_RANGE("gem_shard_rerank");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!pool_ids || !pool_scores) return fail(GEM_ERR_INVALID, "NULL argument");
  if (!w->d_pool_off || !w->d_pool_ids) return fail(GEM_ERR_STATE, "workspace was created with max_k or max_cands 0");
  if (depth < 1 || (int64_t)depth * n_queries > w->max_cands)
    return fail(GEM_ERR_INVALID, "n_queries * depth must be 1..max_cands");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "the rerank needs the fp32 copy");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)n_queries * depth;
  local_ids_kernel<<<grid_for(n, s->n_sm), 256, 0, st>>>(pool_ids, n, id_base, s->n_sets, w->d_pool_ids);
  launch_iota_offsets(w->d_pool_off, n_queries, depth, st);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  r = launch_f32_score_pool(s, w, q, q_offsets, n_queries, depth, w->d_pool_ids, w->d_pool_scores, st);
  if (r != GEM_OK) return r;
  scatter_owned_kernel<<<grid_for(n, s->n_sm), 256, 0, st>>>(w->d_pool_ids, w->d_pool_scores, n, pool_scores);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status gem_shard_score_ids(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                               int32_t n_queries, int64_t n_q_rows, const int64_t* cand_offsets,
                               const int64_t* cand_ids, int64_t n_cands, int32_t compute, int64_t id_base,
                               float* scores, void* stream) {
  GEM_NVTX_RANGE("gem_shard_score_ids");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!cand_offsets || (n_cands > 0 && (!cand_ids || !scores))) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_cands < 0) return fail(GEM_ERR_INVALID, "n_cands < 0");
  if (n_cands == 0) return GEM_OK;
  if (!w->d_pool_ids || n_cands > w->max_cands) return fail(GEM_ERR_INVALID, "n_cands exceeds the workspace's max_cands");
  if (id_base < 0) return fail(GEM_ERR_INVALID, "id_base < 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  local_ids_kernel<<<grid_for(n_cands, s->n_sm), 256, 0, st>>>(cand_ids, n_cands, id_base, s->n_sets, w->d_pool_ids);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  r = gem_score_ids(s, w, q, q_offsets, n_queries, n_q_rows, cand_offsets, w->d_pool_ids, n_cands, compute,
                    w->d_pool_scores, stream);
  if (r != GEM_OK) return r;
  scatter_owned_kernel<<<grid_for(n_cands, s->n_sm), 256, 0, st>>>(w->d_pool_ids, w->d_pool_scores, n_cands, scores);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status gem_merge_topk(const float* scores, const int64_t* ids, int32_t n_lists, int32_t rows, int32_t k_in,
                          int32_t k, int64_t* out_ids, float* out_scores, void* stream) {
  GEM_NVTX_RANGE("gem_merge_topk");
  if (!scores || !ids || !out_ids) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_lists < 1 || rows < 0 || k_in < 1) return fail(GEM_ERR_INVALID, "bad shape");
  if (k < 1 || k > kMaxK) return fail(GEM_ERR_INVALID, "k must be 1..4096");
  int dev = 0, n_sm = 0;
  GEM_CUDA_TRY(cudaGetDevice(&dev));
  GEM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  return launch_merge_topk(scores, ids, n_lists, rows, k_in, k, out_ids, out_scores, n_sm,
                           reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
