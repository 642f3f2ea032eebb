// Batched candidate-list scoring: the scoring step of one beam-search expansion
// (Algorithm 5: every unvisited neighbour P' of a popped node is scored against
// Q) for thousands of queries at once, in one persistent launch replayed from a
// CUDA graph.
//
// Per round the graph runs: header copy (pinned host -> device) -> work plan
// (segments of SEG candidates per query, prefix-summed) -> [query codes, codes
// form only] -> counter reset -> persistent scorer: every warp pulls (query,
// segment) items from an atomic counter and streams the segment's sets
// (stream_pairs; the codes form gathers the centroid rows the codes name).
// Either way a batched score is bit-identical to the score the same pair gets
// from gem_score_ids.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "maxsim_simt.cuh"
#include "ptx.cuh"


namespace gem {
namespace {

constexpr int kBatchWarps = 4;

// One block: items per query = ceil(list length / seg), exclusive prefix sum.
__global__ void __launch_bounds__(1024)
batch_plan_kernel(int64_t* __restrict__ hdr, const int64_t* __restrict__ co, int seg,
                  int64_t* __restrict__ item_off, int max_queries, int64_t max_cands, int* status) {
  __shared__ long long warp_sum[32];
  __shared__ long long carry;
  __shared__ int bad;
  const int B = (int)hdr[0];
  const int64_t n_cands = hdr[2];
  if (threadIdx.x == 0) {
    carry = 0;
    bad = (B < 1 || B > max_queries || co[0] != 0 || co[B] != n_cands || n_cands > max_cands) ? 1 : 0;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) { hdr[3] = 0; set_status(status, kDevInvalid); }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < B; c0 += 1024) {
    const int b = c0 + threadIdx.x;
    long long n = 0;
    if (b < B) {
      const int64_t len = co[b + 1] - co[b];
      if (len < 0) atomicOr(&bad, 1);
      n = len > 0 ? (len + seg - 1) / seg : 0;
    }
    long long x = n;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long ws = warp_sum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sum[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const long long before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - n;
    if (b < B) item_off[b] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    item_off[B] = carry;
    hdr[3] = bad ? 0 : carry;
    if (bad) set_status(status, kDevInvalid);
  }
}

struct BatchArgs {
  const float* q;
  const int64_t* q_off;
  const int64_t* co;
  const int64_t* ids;
  const int64_t* item_off;
  const int64_t* hdr;
  unsigned long long* counter;
  const float* docs;
  const int64_t* doc_off;
  int64_t n_sets;
  const int32_t* codes;      // codes form: store codes
  const float* centroids;    // codes form: C_quant
  const int32_t* qcodes;     // codes form: query codes
  int seg;
  int max_q_len;
  float* scores;
  int* status;
};

// A warp per item; the pairs of the item's segment stream through the warp's
// ring (bit-identical to gem_score_ids).  CODES: the codes form, whose staged rows
// are the centroids the store codes name and whose query rows are the centroids
// of the query codes.  A query longer than max_q_len (or empty) is skipped with a
// status and its scores stay unwritten.
template <bool CODES>
__global__ void __launch_bounds__(kBatchWarps * 32, 2) batch_stream_kernel(BatchArgs a) {
  extern __shared__ float sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ring = sm + warp * kRing * ring_block(true);
  float* rowmax = sm + kBatchWarps * kRing * ring_block(true) + warp * kStreamRowmax;
  const int B = (int)a.hdr[0];
  const long long total = a.hdr[3];
  StreamArgs sa{a.q, a.q_off, B, a.co, a.ids, a.docs, a.doc_off, a.n_sets, a.scores, a.status, a.max_q_len};
  if constexpr (CODES) {
    sa.codes = a.codes;
    sa.centroids = a.centroids;
    sa.qcodes = a.qcodes;
  }
  while (true) {
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd(a.counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    int lo = 0, hi = B - 1;  // query owning the item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.item_off[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const int m_q = (int)(a.q_off[b + 1] - a.q_off[b]);
    if (m_q < 1 || m_q > a.max_q_len) {
      if (lane == 0) set_status(a.status, kDevInvalid);
      continue;
    }
    const int64_t t0 = a.co[b] + (item - a.item_off[b]) * a.seg;
    const int64_t t1 = min(a.co[b + 1], t0 + a.seg);
    stream_pairs<false, true, CODES>(sa, t0, t1, ring, rowmax);
  }
}

size_t batch_smem() {
  return sizeof(float) * ((size_t)kBatchWarps * kRing * ring_block(true) + kBatchWarps * kStreamRowmax);
}

// The scorer of a mode, with its shared-memory attribute set once.
cudaError_t batch_kernel(int32_t mode, void (**kern)(BatchArgs)) {
  static bool attr_set[2] = {false, false};
  const int codes = mode == GEM_CODES ? 1 : 0;
  *kern = codes ? batch_stream_kernel<true> : batch_stream_kernel<false>;
  if (!attr_set[codes]) {
    cudaError_t e = cudaFuncSetAttribute(*kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
    if (e != cudaSuccess) return e;
    attr_set[codes] = true;
  }
  return cudaSuccess;
}

// The launch sequence of one round, on stream st (captured or direct).
gem_status enqueue_round(gem_batch* bt, cudaStream_t st) {
  const gem_store* s = bt->store;
  GEM_CUDA_TRY(cudaMemcpyAsync(bt->d_hdr, bt->h_hdr, sizeof(int64_t) * 3, cudaMemcpyHostToDevice, st));
  batch_plan_kernel<<<1, 1024, 0, st>>>(bt->d_hdr, bt->d_cand_off, bt->seg, bt->d_item_off, bt->max_queries,
                                        bt->max_cands, bt->d_status);
  GEM_CUDA_TRY(cudaGetLastError());
  int n_launch = 2;
  if (bt->mode == GEM_CODES) {
    // the round's query rows (their count on the device) to NN codes
    gem_status r = bt->d_asg_scratch
                       ? enqueue_assign_tc(bt->d_q, bt->max_q_rows, bt->d_hdr + 1, s->d_codebook, s->k1,
                                           bt->d_qcodes, nullptr, bt->d_asg_scratch, bt->d_status, s->n_sm, st)
                       : launch_assign_dev_n(bt->d_q, bt->max_q_rows, bt->d_hdr + 1, s->d_codebook, s->k1,
                                             bt->d_qcodes, st);
    if (r != GEM_OK) return r;
  }
  GEM_CUDA_TRY(cudaMemsetAsync(bt->d_counter, 0, sizeof(unsigned long long), st));
  BatchArgs a;
  a.q = bt->d_q;
  a.q_off = bt->d_q_off;
  a.co = bt->d_cand_off;
  a.ids = bt->d_cand_ids;
  a.item_off = bt->d_item_off;
  a.hdr = bt->d_hdr;
  a.counter = bt->d_counter;
  a.docs = s->d_f32;
  a.doc_off = s->d_offsets;
  a.n_sets = s->n_sets;
  a.codes = bt->mode == GEM_CODES ? s->d_codes : nullptr;
  a.centroids = s->d_codebook;
  a.qcodes = bt->mode == GEM_CODES ? bt->d_qcodes : nullptr;
  a.seg = bt->seg;
  a.max_q_len = bt->max_q_len;
  a.scores = bt->d_scores;
  a.status = bt->d_status;
  void (*kern)(BatchArgs) = nullptr;
  GEM_CUDA_TRY(batch_kernel(bt->mode, &kern));
  kern<<<bt->grid, kBatchWarps * 32, batch_smem(), st>>>(a);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(n_launch);
  return GEM_OK;
}

}  // namespace

gem_status batch_create(const gem_store* s, int32_t mode, int32_t max_queries, int64_t max_q_rows,
                        int32_t max_q_len, int64_t max_cands, int32_t seg, int32_t ctas_per_sm,
                        float* q, int64_t* q_offsets, int64_t* cand_offsets, int64_t* cand_ids,
                        float* scores, gem_batch** out) {
  gem_batch* bt = new gem_batch();
  bt->store = s;
  bt->device = s->device;
  bt->mode = mode;
  bt->max_queries = max_queries;
  bt->max_q_rows = max_q_rows;
  bt->max_q_len = max_q_len;
  bt->max_cands = max_cands;
  bt->seg = seg;
  auto bail = [&](gem_status r) { batch_destroy(bt); return r; };
  cudaError_t e;
#define BT_ALLOC(ptr, bytes)                                         \
  if ((e = cudaMalloc(reinterpret_cast<void**>(&bt->ptr), (bytes))) != cudaSuccess) { \
    cudaGetLastError();                                              \
    return bail(fail(GEM_ERR_OOM, "cudaMalloc failed for " #ptr)); \
  }
  bt->d_q = q;
  bt->d_q_off = q_offsets;
  bt->d_cand_off = cand_offsets;
  bt->d_cand_ids = cand_ids;
  bt->d_scores = scores;
  BT_ALLOC(d_hdr, sizeof(int64_t) * 4);
  BT_ALLOC(d_item_off, sizeof(int64_t) * (max_queries + 1));
  BT_ALLOC(d_counter, sizeof(unsigned long long));
  BT_ALLOC(d_status, sizeof(int));
  if (mode == GEM_CODES) BT_ALLOC(d_qcodes, sizeof(int32_t) * max_q_rows);
  if (mode == GEM_CODES && max_q_rows >= kAssignTcMinRows && s->k1 >= kAssignTcMinCentroids) {
    BT_ALLOC(d_asg_scratch, assign_tc_scratch_bytes(max_q_rows, s->k1));
    if ((e = assign_tc_prepare()) != cudaSuccess) return bail(cuda_fail(e, "smem attribute"));
  }
#undef BT_ALLOC
  if ((e = cudaMallocHost(reinterpret_cast<void**>(&bt->h_hdr), sizeof(int64_t) * 4)) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMallocHost"));
  if ((e = cudaMemset(bt->d_status, 0, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "memset"));
  if ((e = cudaEventCreateWithFlags(&bt->done, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(e, "event"));
  const size_t smem = batch_smem();
  void (*kern)(BatchArgs) = nullptr;
  if ((e = batch_kernel(mode, &kern)) != cudaSuccess) return bail(cuda_fail(e, "smem attribute"));
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchWarps * 32, smem)) != cudaSuccess)
    return bail(cuda_fail(e, "occupancy"));
  if (per_sm < 1) return bail(fail(GEM_ERR_UNSUPPORTED, "batched scorer does not fit on an SM"));
  bt->grid = s->n_sm * std::min(per_sm, ctas_per_sm > 0 ? ctas_per_sm : per_sm);
  // capture one round into a graph
  cudaStream_t cap;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return bail(cuda_fail(e, "stream"));
  bt->h_hdr[0] = 1;
  bt->h_hdr[1] = 1;
  bt->h_hdr[2] = 0;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  gem_status r = GEM_OK;
  if (e == cudaSuccess) {
    const int64_t before = gem_kernel_launches();
    r = enqueue_round(bt, cap);
    // launches inside a capture are counted when the graph is replayed
    bt->round_launches = (int)(gem_kernel_launches() - before);
    note_launches(-bt->round_launches);
    cudaError_t e2 = cudaStreamEndCapture(cap, &bt->graph);
    if (r == GEM_OK && e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && r == GEM_OK) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
  cudaStreamDestroy(cap);
  if (r != GEM_OK) return bail(r);
  if (e != cudaSuccess) return bail(cuda_fail(e, "graph capture"));
  *out = bt;
  return GEM_OK;
}

gem_status batch_run(gem_batch* bt, int32_t n_queries, int64_t n_q_rows, int64_t n_cands, int use_graph,
                     cudaStream_t st) {
  // the previous round must have copied its header before it is overwritten
  if (bt->launched) GEM_CUDA_TRY(cudaEventSynchronize(bt->done));
  bt->h_hdr[0] = n_queries;
  bt->h_hdr[1] = n_q_rows;
  bt->h_hdr[2] = n_cands;
  if (use_graph) {
    GEM_CUDA_TRY(cudaGraphLaunch(bt->exec, st));
    note_launches(bt->round_launches);
  } else {
    gem_status r = enqueue_round(bt, st);
    if (r != GEM_OK) return r;
  }
  GEM_CUDA_TRY(cudaEventRecord(bt->done, st));
  bt->launched = true;
  return GEM_OK;
}

void batch_destroy(gem_batch* bt) {
  if (!bt) return;
  if (bt->launched) cudaEventSynchronize(bt->done);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->done) cudaEventDestroy(bt->done);
  void* ptrs[] = {bt->d_hdr, bt->d_item_off, bt->d_counter, bt->d_qcodes, bt->d_asg_scratch, bt->d_status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (bt->h_hdr) cudaFreeHost(bt->h_hdr);
  delete bt;
}

// ---------------------------------------------------------------------------
// gem_score_ids_noalloc: the batched scorer with its work-plan scratch in a
// fixed device array instead of caller- or library-allocated memory.

namespace {

constexpr int kNoAllocMaxQueries = 16384;  // queries per call
constexpr int kNoAllocSeg = 32;

struct NoAllocScratch {
  int64_t hdr[4];                               // n_queries, n_q_rows, n_cands, items
  unsigned long long counter;                   // work-queue position
  int status;
  int pad;
  int64_t item_off[kNoAllocMaxQueries + 1];     // first work item of each query
};

// One copy per device, shared by every call (about 128 KB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Everything a call relies on starting at zero is written here first.
__global__ void noalloc_init_kernel(NoAllocScratch* sc, int n_queries, int64_t n_q_rows, int64_t n_cands) {
  sc->hdr[0] = n_queries;
  sc->hdr[1] = n_q_rows;
  sc->hdr[2] = n_cands;
  sc->hdr[3] = 0;
  sc->counter = 0;
  sc->status = 0;
}

std::mutex g_noalloc_mu;
std::map<int, NoAllocScratch*> g_noalloc_addr;  // device -> device address of the array

// Device address of this device's copy of the array, looked up once per device
// with that device current.  The name of the array is only a host-side handle.
gem_status noalloc_scratch(int dev, NoAllocScratch** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it == g_noalloc_addr.end()) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
    void (*kern)(BatchArgs) = nullptr;
    e = batch_kernel(GEM_F32, &kern);
    if (e != cudaSuccess) return cuda_fail(e, "shared memory attribute");
    it = g_noalloc_addr.emplace(dev, reinterpret_cast<NoAllocScratch*>(p)).first;
  }
  *out = it->second;
  return GEM_OK;
}

}  // namespace

gem_status score_ids_noalloc(const gem_store* s, const float* q, const int64_t* q_offsets, int32_t n_queries,
                             int64_t n_q_rows, int32_t max_q_len, const int64_t* cand_offsets,
                             const int64_t* cand_ids, int64_t n_cands, float* scores, cudaStream_t st) {
  if (n_queries > kNoAllocMaxQueries)
    return fail(GEM_ERR_INVALID, "gem_score_ids_noalloc takes at most 16384 queries per call");
  NoAllocScratch* sc = nullptr;
  gem_status r = noalloc_scratch(s->device, &sc);
  if (r != GEM_OK) return r;
  const size_t smem = batch_smem();
  void (*kern)(BatchArgs) = nullptr;
  GEM_CUDA_TRY(batch_kernel(GEM_F32, &kern));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchWarps * 32, smem));
  if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "batched scorer does not fit on an SM");
  noalloc_init_kernel<<<1, 1, 0, st>>>(sc, n_queries, n_q_rows, n_cands);
  batch_plan_kernel<<<1, 1024, 0, st>>>(sc->hdr, cand_offsets, kNoAllocSeg, sc->item_off, kNoAllocMaxQueries,
                                        n_cands, &sc->status);
  BatchArgs a;
  a.q = q;
  a.q_off = q_offsets;
  a.co = cand_offsets;
  a.ids = cand_ids;
  a.item_off = sc->item_off;
  a.hdr = sc->hdr;
  a.counter = &sc->counter;
  a.docs = s->d_f32;
  a.doc_off = s->d_offsets;
  a.n_sets = s->n_sets;
  a.codes = nullptr;
  a.centroids = nullptr;
  a.qcodes = nullptr;
  a.seg = kNoAllocSeg;
  a.max_q_len = max_q_len;
  a.scores = scores;
  a.status = &sc->status;
  kern<<<s->n_sm * per_sm, kBatchWarps * 32, smem, st>>>(a);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(3);
  return GEM_OK;
}

}  // namespace gem
