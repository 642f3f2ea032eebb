// Exact MaxSim in FP32 on the SIMT pipes, with a compensated sum over query
// vectors.  Serves the FP32 exhaustive form and the exact rerank of a candidate
// pool (the final step of Algorithm 5, CH of Sec. 3.1 Eq. 1).
//
// One CTA per work unit (query, segment of sets), one warp per set; the per-pair
// arithmetic is warp_chamfer (maxsim_simt.cuh).
#include "internal.h"
#include "maxsim_simt.cuh"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kF32Warps = 4;
constexpr int kF32Threads = kF32Warps * 32;
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
  const int32_t* codes;      // codes form: store codes, centroids and query codes
  const float* centroids;
  const int32_t* qcodes;
};

// All sets: one CTA per (segment of kSegDocs sets, query), the query staged in
// shared memory; consecutive CTAs share a segment, so its sets stay in L2.
template <bool L2>
__global__ void __launch_bounds__(kF32Threads, 2)
f32_all_kernel(F32Args a, int max_q_len) {
  extern __shared__ float sm[];
  float* qs = sm;                                              // [max_q_len * kQStride]
  float* stage_all = qs + max_q_len * kQStride;                // [warps][kVecBlock * 128]
  float* rowmax_all = stage_all + kF32Warps * kVecBlock * kStageStride;  // [warps][max_q_len]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + warp * kVecBlock * kStageStride;
  float* rowmax = rowmax_all + warp * max_q_len;
  uint64_t qr[kQPairs];
  const int64_t n_seg = (a.n_sets + kSegDocs - 1) / kSegDocs;
  const int64_t n_units = n_seg * a.n_queries;
  for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = (int)(u % a.n_queries);
    const int64_t q0 = a.q_off[b];
    const int m_q = (int)(a.q_off[b + 1] - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m_q * (kDim / 4); idx += blockDim.x) {
      const int i = idx / (kDim / 4), k4 = idx % (kDim / 4);
      const float* src = a.qcodes ? a.centroids + (int64_t)a.qcodes[q0 + i] * kDim : a.q + (q0 + i) * kDim;
      reinterpret_cast<float4*>(qs + i * kQStride)[k4] = reinterpret_cast<const float4*>(src)[k4];
    }
    __syncthreads();
    int loaded_rg = -1;
    const int64_t t0 = (u / a.n_queries) * kSegDocs;
    const int64_t t1 = min(a.n_sets, t0 + kSegDocs);
    for (int64_t t = t0 + warp; t < t1; t += kF32Warps) {
      const int64_t r0 = a.doc_off[t];
      const int m_p = (int)(a.doc_off[t + 1] - r0);
      const float score = warp_chamfer<L2>(qs, kQStride, m_q, a.docs + r0 * kDim, a.qcodes ? a.codes + r0 : nullptr,
                                           a.centroids, m_p, stage, rowmax, qr, loaded_rg);
      if (lane == 0) a.scores[(int64_t)b * a.n_sets + t] = score;
    }
  }
}

// Id lists: every warp takes one contiguous range of the n_cands candidates
// (equal shares, whatever the list lengths) and streams it (stream_pairs in
// maxsim_simt.cuh: bit-identical to warp_chamfer); a pool in segment order is
// taken in groups of kPoolGroup positions, grid-strided.  CODES: the codes
// forms, whose stored rows are the centroids the store codes name (and whose
// query rows, given query codes, are centroids too).
template <bool L2, bool CODES = false>
__global__ void __launch_bounds__(kF32Threads, 2)
f32_ids_stream_kernel(StreamArgs a, int64_t n_cands) {
  extern __shared__ float sm[];
  const int warp = threadIdx.x >> 5;
  float* ring = sm + warp * kRing * ring_block(false);
  float* rowmax = sm + kF32Warps * kRing * ring_block(false) + warp * kStreamRowmax;
  const int64_t n_warps = (int64_t)gridDim.x * kF32Warps;
  const int64_t gw = (int64_t)blockIdx.x * kF32Warps + warp;
  if (a.perm) {
    // a pool in segment order: the warps claim kPoolGroup positions at a time,
    // in order, from a counter, so they move through the positions together and
    // the sets in use at any moment come from one or two segments of set ids
    const int lane = threadIdx.x & 31;
    for (;;) {
      unsigned long long claim = 0;
      if (lane == 0) claim = atomicAdd(a.counter, 1ull);
      const int64_t p0 = (int64_t)__shfl_sync(0xffffffffu, claim, 0) * kPoolGroup;
      if (p0 >= n_cands) break;
      stream_pairs<L2, false, CODES>(a, p0, min(n_cands, p0 + kPoolGroup), ring, rowmax);
    }
    return;
  }
  const int64_t chunk = (n_cands + n_warps - 1) / n_warps;
  const int64_t t_begin = min(n_cands, gw * chunk);
  const int64_t t_end = min(n_cands, t_begin + chunk);
  stream_pairs<L2, false, CODES>(a, t_begin, t_end, ring, rowmax);
}

// Order of a rerank pool (per_query entries per query) for the exact rescoring:
// by segment of set ids first (K equal ranges of ids), then by query, so that
// at any time the warps work inside one segment and a set several queries share
// is read from DRAM about once (the segment's sets fit in L2), while each warp
// still takes runs of one query's entries.  A counting sort on the key
// segment * n_queries + query: count, exclusive scan, scatter (the order inside
// a key depends on atomics; the scores do not, each entry is scored alone).
__device__ __forceinline__ int pool_key(const int64_t* ids, int64_t i, int per_query, int n_queries, int64_t n_sets,
                                        int segs) {
  const int64_t id = ids[i];
  const int seg = (id >= 0 && id < n_sets) ? (int)(id * segs / n_sets) : segs - 1;
  return seg * n_queries + (int)(i / per_query);
}

__global__ void pool_key_count_kernel(const int64_t* __restrict__ ids, int64_t n, int per_query, int n_queries,
                                      int64_t n_sets, int segs, int* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + pool_key(ids, i, per_query, n_queries, n_sets, segs), 1);
}

// one block of 1024 threads: cnt[0 .. nk) becomes its exclusive prefix sum
__global__ void __launch_bounds__(1024) pool_key_scan_kernel(int* __restrict__ cnt, int nk) {
  __shared__ int part[1024];
  constexpr int kPer = kPoolKeys / 1024;
  const int t = threadIdx.x;
  int sum = 0;
  for (int j = 0; j < kPer; ++j) {
    const int i = t * kPer + j;
    sum += i < nk ? cnt[i] : 0;
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the per-thread sums
    const int x = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int run = part[t] - sum;
  for (int j = 0; j < kPer; ++j) {
    const int i = t * kPer + j;
    if (i < nk) {
      const int v = cnt[i];
      cnt[i] = run;
      run += v;
    }
  }
}

__global__ void pool_key_scatter_kernel(const int64_t* __restrict__ ids, int64_t n, int per_query, int n_queries,
                                        int64_t n_sets, int segs, int* __restrict__ cursor,
                                        int32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    perm[atomicAdd(cursor + pool_key(ids, i, per_query, n_queries, n_sets, segs), 1)] = (int32_t)i;
}

}  // namespace

gem_status launch_f32_score(const gem_store* s, gem_workspace* ws, const float* q,
                            const int64_t* q_offsets, int32_t n_queries, const int64_t* cand_offsets,
                            const int64_t* cand_ids, int64_t n_cands, float* scores, cudaStream_t st,
                            const int32_t* qcodes, bool stored_codes) {
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
  a.codes = s->d_codes;
  a.centroids = s->d_codebook;
  a.qcodes = qcodes;
  // id lists, asymmetric codes form: stored rows by their codes, exact query rows
  const bool asym_codes = stored_codes && !qcodes && cand_ids;
  const int mq = ws->max_q_len;
  // Sim = -(L2 distance) on the exact rows only (the codes forms are inner products)
  const bool l2 = ws->sim == GEM_SIM_L2 && !qcodes && !asym_codes;
  int per_sm = 0;
  if (cand_ids == nullptr) {
    const size_t smem = sizeof(float) * ((size_t)mq * kQStride + kF32Warps * kVecBlock * kStageStride + (size_t)kF32Warps * mq);
    auto kern = l2 ? f32_all_kernel<true> : f32_all_kernel<false>;
    GEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32Threads, smem));
    if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "f32 scoring kernel does not fit on an SM");
    const int64_t units = ((s->n_sets + kSegDocs - 1) / kSegDocs) * n_queries;
    const int grid = (int)std::min<int64_t>(units, (int64_t)s->n_sm * per_sm);
    kern<<<grid, kF32Threads, smem, st>>>(a, mq);
  } else {
    StreamArgs sa{q, q_offsets, n_queries, cand_offsets, cand_ids, s->d_f32, s->d_offsets, s->n_sets,
                  scores, ws->d_status, mq};
    const bool coded = qcodes || asym_codes;
    if (coded) {
      sa.codes = s->d_codes;
      sa.centroids = s->d_codebook;
      sa.qcodes = qcodes;  // null: the asymmetric form (exact query rows)
    }
    const size_t smem = sizeof(float) * (kF32Warps * kRing * ring_block(false) + kF32Warps * kStreamRowmax);
    auto kern = coded ? f32_ids_stream_kernel<false, true>
                      : l2 ? f32_ids_stream_kernel<true> : f32_ids_stream_kernel<false>;
    GEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32Threads, smem));
    if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "f32 scoring kernel does not fit on an SM");
    const int64_t max_grid = (n_cands + kF32Warps - 1) / kF32Warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(max_grid, (int64_t)s->n_sm * per_sm));
    kern<<<grid, kF32Threads, smem, st>>>(sa, n_cands);
  }
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_f32_score_pool(const gem_store* s, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                                 int32_t n_queries, int32_t per_query, const int64_t* cand_ids, float* scores,
                                 cudaStream_t st) {
  const int64_t n = (int64_t)n_queries * per_query;
  // small pools (the three grouping launches would not pay) and pools the
  // workspace has no order buffer for: query order
  if (n < kPoolMinEntries || !ws->d_pool_perm || n > ws->max_cands)
    return launch_f32_score(s, ws, q, q_offsets, n_queries, ws->d_pool_off, cand_ids, n, scores, st);
  // segments: up to kPoolSegs, at most kPoolKeys keys
  const int segs = (int)std::max<int64_t>(1, std::min<int64_t>(kPoolSegs, kPoolKeys / n_queries));
  if (segs < 2) return launch_f32_score(s, ws, q, q_offsets, n_queries, ws->d_pool_off, cand_ids, n, scores, st);
  const int nk = segs * n_queries;
  GEM_CUDA_TRY(cudaMemsetAsync(ws->d_pool_bucket, 0, sizeof(int) * nk, st));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)s->n_sm * 8);
  pool_key_count_kernel<<<grid, 256, 0, st>>>(cand_ids, n, per_query, n_queries, s->n_sets, segs,
                                              ws->d_pool_bucket);
  pool_key_scan_kernel<<<1, 1024, 0, st>>>(ws->d_pool_bucket, nk);
  pool_key_scatter_kernel<<<grid, 256, 0, st>>>(cand_ids, n, per_query, n_queries, s->n_sets, segs,
                                                ws->d_pool_bucket, ws->d_pool_perm);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(3);
  const int mq = ws->max_q_len;
  const bool l2 = ws->sim == GEM_SIM_L2;
  StreamArgs sa{q, q_offsets, n_queries, ws->d_pool_off, cand_ids, s->d_f32, s->d_offsets, s->n_sets,
                scores, ws->d_status, mq};
  sa.perm = ws->d_pool_perm;
  sa.per_query = per_query;
  sa.counter = reinterpret_cast<unsigned long long*>(ws->d_unit_counter);
  GEM_CUDA_TRY(cudaMemsetAsync(sa.counter, 0, sizeof(unsigned long long), st));
  const size_t smem = sizeof(float) * (kF32Warps * kRing * ring_block(false) + kF32Warps * kStreamRowmax);
  auto kern = l2 ? f32_ids_stream_kernel<true> : f32_ids_stream_kernel<false>;
  GEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32Threads, smem));
  if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "f32 scoring kernel does not fit on an SM");
  const int64_t max_grid = (n + kF32Warps - 1) / kF32Warps;
  const int kgrid = (int)std::max<int64_t>(1, std::min<int64_t>(max_grid, (int64_t)s->n_sm * per_sm));
  kern<<<kgrid, kF32Threads, smem, st>>>(sa, n);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
