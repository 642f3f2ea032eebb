// Internal runtime types of libgem: the store, the workspace, the query plan and
// the kernel launchers.  Nothing here is part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "gem.h"

namespace gem {

constexpr int kDim = 128;         // vector dimension handled by every kernel
constexpr int kMaxPasses = 8;     // query sets of up to 8 * 32 = 256 vectors
constexpr int kClasses = 6;       // slot sizes 32, 16, 8, 4, 2, 1 rows
constexpr int kCombos = kMaxPasses * kClasses;
constexpr int kMaxK = 4096;       // largest top-k
constexpr int kPlanHdrInts = 64;
// The low-precision store copies pad every set to a multiple of kRowAlign rows
// with copies of the set's last vector, so set boundaries fall on 8-row steps.
constexpr int kRowAlign = 8;

// Plan header layout (device int32 array).
enum : int {
  kHdrParts = 0,       // number of query parts
  kHdrPackedRows = 1,  // rows of the packed query buffer in use (multiple of m_res)
  kHdrQBlocks = 2,     // total query blocks
  kHdrPasses = 3,      // passes with any work
  kHdrQbBegin = 4,     // kMaxPasses + 1 entries: first query block of each pass
};

// A document chunk map: contiguous runs of whole sets holding about
// `chunk_rows` vectors each (a set longer than that forms a chunk of its own).
struct ChunkMap {
  int chunk_rows = 0;
  int n_chunks = 0;
  int* d_chunk_doc = nullptr;  // [n_chunks + 1] first set of each chunk
};

struct TmapSet {
  bool valid = false;
  CUtensorMap map;
};

}  // namespace gem

struct gem_store {
  int device = 0;
  int n_sm = 0;
  int64_t n_sets = 0;
  int64_t n_vecs = 0;
  uint32_t keep = 0;
  std::vector<int64_t> h_offsets;
  int64_t* d_offsets = nullptr;
  // padded layout of the bf16 / fp8 copies
  int64_t n_pad_vecs = 0;
  std::vector<int64_t> h_pad_offsets;
  int64_t* d_pad_offsets = nullptr;
  // bit i set: a set ends with padded row 8 i + 7 (two words of slack at the end)
  uint32_t* d_end_bits = nullptr;
  float* d_f32 = nullptr;
  __nv_bfloat16* d_bf16 = nullptr;
  uint8_t* d_fp8 = nullptr;
  float* d_fp8_scale = nullptr;
  // E4M3 with one power-of-two scale per set (padded layout as d_fp8)
  uint8_t* d_fp8s = nullptr;
  float* d_set_scale = nullptr;   // [n_sets]
  int64_t max_set_len = 0;
  // stage-1 codebook C_quant and the codes NN(p) of every stored vector
  int k1 = 0;
  float* d_codebook = nullptr;   // [k1 * 128], unit rows
  int32_t* d_codes = nullptr;    // [n_vecs], original (unpadded) row order
  // coarse clusters C_index (Sec. 4.1.1): the nearest one of every stored vector
  // and, per cluster, the sets of its vectors (one entry per vector, in no fixed
  // order) behind member_off [k2 + 1]
  int k2 = 0;
  float* d_cindex = nullptr;      // [k2 * 128]
  int32_t* d_icodes = nullptr;    // [n_vecs]
  int64_t* d_member_off = nullptr;
  int32_t* d_members = nullptr;   // [n_vecs] set ids
  // lazy deletion (Sec. 4.6): bit s set = set s is deleted; null until the first
  // deletion.  Deleted sets are still scored and traversed, never returned.
  uint32_t* d_dead = nullptr;     // [ceil(n_sets / 32)]
  // tensor maps of the doc copies, keyed by tile rows (box height)
  mutable std::map<int, CUtensorMap> tmap_bf16;
  mutable std::map<int, CUtensorMap> tmap_fp8;
  mutable std::map<int, CUtensorMap> tmap_fp8_scale;
  mutable std::map<int, CUtensorMap> tmap_fp8s;
  mutable std::map<int, gem::ChunkMap> chunks;
};

struct gem_workspace {
  const gem_store* store = nullptr;
  int device = 0;
  int32_t max_queries = 0;
  int64_t max_q_rows = 0;
  int32_t max_q_len = 0;
  int64_t max_cands = 0;
  int32_t max_k = 0;
  int n_passes = 0;
  int tc_m_tiles = 2;          // schedule of the tensor-core kernels
  int tc_variant = GEM_TC_PLAIN;
  int qch_form = GEM_QCH_SYMMETRIC;  // every qCH estimate through this workspace
  int sim = GEM_SIM_IP;              // Sim of Definition 1 for the exact FP32 scorers
  int tc_chunk_rows = 1 << 16;

  int* d_status = nullptr;
  int* d_unit_counter = nullptr;  // 8 bytes: work-unit counter of the tensor-core kernels (low 32 bits)
                                  // and, as 64 bits, the chunk counter of the qCH scan

  // query plan
  int64_t packed_cap = 0;  // rows of the packed query buffers
  int64_t max_parts = 0;
  int* d_plan_hdr = nullptr;
  int* d_part_query = nullptr;
  int* d_part_rows = nullptr;
  int* d_part_g = nullptr;
  int* d_part_pass = nullptr;
  int* d_part_slot = nullptr;
  int64_t* d_part_row0 = nullptr;
  int* d_row_part = nullptr;
  __nv_bfloat16* d_qpack_bf16 = nullptr;
  uint8_t* d_qpack_fp8 = nullptr;
  float* d_qpack_scale = nullptr;
  CUtensorMap tmap_q_bf16;
  CUtensorMap tmap_q_fp8;

  // quantized estimate
  int32_t* d_qcodes = nullptr;     // [max_q_rows]
  // (ordered best value, ~index) per query row while the centroids of C_quant are
  // split over CTAs (few rows: see launch_assign_split)
  unsigned long long* d_assign_key = nullptr;  // [max_q_rows]
  float* d_tables = nullptr;       // [table_parts * k1 * 32]
  int table_parts = 0;

  // search pipeline
  float* d_scores = nullptr;       // [max_queries * n_sets]
  int64_t* d_pool_ids = nullptr;   // [max_cands]
  int64_t* d_pool_off = nullptr;   // [max_queries + 1]
  float* d_pool_scores = nullptr;  // [max_cands]
  int32_t* d_pool_perm = nullptr;  // [max_cands] rerank order: by segment of set ids, then query
  int* d_pool_bucket = nullptr;    // [kPoolKeys] counts, then cursors, of that order

  // threshold top-k of long dense rows (topk.cu): per row a key threshold, a
  // counter and a candidate buffer of topk_cap keys, for topk_rows rows at a time
  int topk_cap = 0;
  int topk_rows = 0;
  unsigned long long* d_topk_thr = nullptr;   // [topk_rows]
  unsigned* d_topk_cnt = nullptr;             // [topk_rows]
  unsigned long long* d_topk_cand = nullptr;  // [topk_rows * topk_cap]

  // host-buffer entry point staging
  float* d_q_in = nullptr;
  int64_t* d_qo_in = nullptr;
  int64_t* d_out_ids = nullptr;
  float* d_out_scores = nullptr;
};

// A batched candidate scorer: its own buffers and the captured CUDA graph of
// one round (batch.cu).
struct gem_batch {
  const gem_store* store = nullptr;
  int device = 0;
  int mode = GEM_F32;
  int32_t max_queries = 0;
  int64_t max_q_rows = 0;
  int32_t max_q_len = 0;
  int64_t max_cands = 0;
  int seg = 32;
  int grid = 0;
  int n_warps = 4;
  // caller-owned inputs and output (fixed addresses, read by the graph)
  float* d_q = nullptr;
  int64_t* d_q_off = nullptr;
  int64_t* d_cand_off = nullptr;
  int64_t* d_cand_ids = nullptr;
  float* d_scores = nullptr;
  // internal
  int64_t* h_hdr = nullptr;  // pinned: n_queries, n_q_rows, n_cands
  int64_t* d_hdr = nullptr;  // + [3] total items
  int64_t* d_item_off = nullptr;
  unsigned long long* d_counter = nullptr;
  int32_t* d_qcodes = nullptr;
  void* d_asg_scratch = nullptr;  // codes form: scratch of the tensor-core query assignment, or null
  int* d_status = nullptr;
  int round_launches = 0;         // kernels of one captured round
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

namespace gem {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
gem_status fail(gem_status code, const std::string& msg);
gem_status cuda_fail(cudaError_t e, const char* what);
// A named range on the host timeline for profilers (NVTX; a no-op when no tool
// is attached), from construction to the end of the scope.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GEM_NVTX_RANGE(name) ::gem::NvtxRange gem_nvtx_range_(name)

#define GEM_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) return ::gem::cuda_fail(e__, #expr); \
  } while (0)

// Counts kernels enqueued by this library (gem_kernel_launches).
void note_launches(int n);

// ---------------------------------------------------------------- TMA maps
bool encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, void* base, uint64_t inner,
                    uint64_t rows, uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows,
                    CUtensorMapSwizzle swz);
bool encode_tmap_1d_f32(CUtensorMap* map, void* base, uint64_t n, uint32_t box);

// ---------------------------------------------------------------- store helpers
gem_status store_chunk_map(const gem_store* s, int chunk_rows, const ChunkMap** out);
gem_status store_tmap_bf16(const gem_store* s, int box_rows, const CUtensorMap** out);
gem_status store_tmap_fp8(const gem_store* s, int box_rows, const CUtensorMap** out);
gem_status store_tmap_fp8_scale(const gem_store* s, int box_rows, const CUtensorMap** out);
gem_status store_tmap_fp8_set(const gem_store* s, int box_rows, const CUtensorMap** out);

// ---------------------------------------------------------------- launchers
// Query plan: split sets into <= 32-row parts, pack them into m_res-row blocks
// and convert to the tensor-core operand type (bf16 or e4m3 + scale).
gem_status launch_plan(gem_workspace* ws, const float* q, const int64_t* q_offsets,
                       int32_t n_queries, int64_t n_q_rows, int m_res, int compute,
                       cudaStream_t st);

// Tensor-core exact MaxSim over all stored sets.
gem_status launch_tc_score_all(const gem_store* s, gem_workspace* ws, int compute, int m_tiles,
                               int variant, int chunk_rows, float* scores, cudaStream_t st);

// FP32 SIMT exact MaxSim (Kahan over query vectors), all sets or id lists;
// qcodes != nullptr selects the codes form (centroids in place of vectors);
// stored_codes alone (id lists) the asymmetric codes form: exact query rows,
// stored vectors replaced by their centroids.
gem_status launch_f32_score(const gem_store* s, gem_workspace* ws, const float* q,
                            const int64_t* q_offsets, int32_t n_queries, const int64_t* cand_offsets,
                            const int64_t* cand_ids, int64_t n_cands, float* scores, cudaStream_t st,
                            const int32_t* qcodes = nullptr, bool stored_codes = false);
// Exact FP32 scores of a rerank pool of per_query candidates per query
// (cand_ids [n_queries * per_query]), taken segment of set ids by segment
// (the order is built in the workspace), so that a set several queries share is
// gathered from DRAM about once; scores land in pool order, bit-identical to
// launch_f32_score.  Pools below kPoolMinEntries are taken in query order.
constexpr int kPoolSegs = 64;
constexpr int kPoolKeys = 65536;  // segments x queries
constexpr int64_t kPoolMinEntries = 65536;
constexpr int kPoolGroup = 32;    // positions a warp takes at a time
gem_status launch_f32_score_pool(const gem_store* s, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                                 int32_t n_queries, int32_t per_query, const int64_t* cand_ids, float* scores,
                                 cudaStream_t st);

// MaxSim forward with argmax and backward (backward.cu).
gem_status launch_maxsim_fwd(const float* q, const int64_t* q_off, int32_t n_queries, const float* docs,
                             const int64_t* d_off, int64_t n_docs, const int64_t* pair_off,
                             const int64_t* pair_ids, int32_t max_q_len, int bf16, float* scores,
                             int32_t* argmax, int* status, int n_sm, cudaStream_t st);
gem_status launch_maxsim_fwd_tc(const float* q, const int64_t* q_off, int32_t n_queries, int64_t n_q_rows,
                                const float* docs, const int64_t* d_off, int64_t n_docs, int64_t n_doc_rows,
                                const int64_t* pair_off, const int64_t* pair_ids, int64_t n_pairs, int32_t max_q_len,
                                float* scores, int32_t* argmax, int* status, int n_sm, cudaStream_t st);
gem_status launch_maxsim_bwd(const float* q, const int64_t* q_off, int32_t n_queries, const float* docs,
                             const int64_t* d_off, int64_t n_docs, int64_t n_doc_rows, const int64_t* pair_off,
                             const int64_t* pair_ids, int64_t n_pairs, const int32_t* argmax, int32_t max_q_len,
                             const float* g, float* grad_q, float* grad_docs, int n_sm, cudaStream_t st);

// Batched candidate scoring (batch.cu).
gem_status batch_create(const gem_store* s, int32_t mode, int32_t max_queries, int64_t max_q_rows,
                        int32_t max_q_len, int64_t max_cands, int32_t seg, int32_t ctas_per_sm,
                        float* q, int64_t* q_offsets, int64_t* cand_offsets, int64_t* cand_ids,
                        float* scores, gem_batch** out);
gem_status batch_run(gem_batch* bt, int32_t n_queries, int64_t n_q_rows, int64_t n_cands, int use_graph,
                     cudaStream_t st);
void batch_destroy(gem_batch* bt);
gem_status autotune_score_all(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                              int32_t n_queries, int64_t n_q_rows, int32_t compute, float* scores,
                              const char* cache_file, int32_t* m_tiles, int32_t* variant, int32_t* chunk_rows, float* ms_out,
                              int32_t* from_cache, cudaStream_t st);
gem_status autotune_batch(const gem_store* s, int32_t mode, int32_t n_queries, int64_t n_q_rows, int32_t max_q_len,
                          int64_t n_cands, float* q, int64_t* q_offsets, int64_t* cand_offsets, int64_t* cand_ids,
                          float* scores, const char* cache_file, int32_t* seg, int32_t* ctas_per_sm, float* ms_out,
                          int32_t* from_cache, cudaStream_t st);
gem_status score_ids_noalloc(const gem_store* s, const float* q, const int64_t* q_offsets, int32_t n_queries,
                             int64_t n_q_rows, int32_t max_q_len, const int64_t* cand_offsets,
                             const int64_t* cand_ids, int64_t n_cands, float* scores, cudaStream_t st);

// Host-side checks shared by the query calls (store, workspace, sizes, device).
gem_status check_query_args(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                            int32_t n_queries, int64_t n_q_rows);
// The first pass of gem_search into w->d_scores [n_queries x n_sets]: exact CH
// in `compute` or, for GEM_CODES, the qCH estimate.
gem_status search_first_pass(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                             int32_t n_queries, int64_t n_q_rows, int32_t compute, cudaStream_t st);
// Per-row top-k of the union of n_lists lists laid out [n_lists][rows][k_in]
// (scores and ids; negative ids are empty slots).
gem_status launch_merge_topk(const float* scores, const int64_t* ids, int32_t n_lists, int32_t rows, int32_t k_in,
                             int32_t k, int64_t* out_ids, float* out_scores, int n_sm, cudaStream_t st);

// Candidate-buffer entries per row the threshold top-k needs for k <= max_k.
int topk_candidate_cap(int max_k);

// Per-row top-k by (score desc, id asc).
gem_status launch_topk(gem_workspace* ws, const float* scores, const int64_t* row_offsets,
                       int32_t rows, int64_t cols, const int64_t* ids, int32_t k,
                       int64_t* out_ids, float* out_scores, cudaStream_t st);

// Codes, k-means and the quantized estimate (codes.cu).
// qvec != nullptr: asymmetric tables from the exact query rows (qcodes unused)
gem_status launch_qch_tables(const gem_store* s, const int32_t* qcodes, const float* qvec, const int64_t* q_offsets,
                             int32_t n_queries, int max_np, float* T, cudaStream_t st);
gem_status launch_qch_scan_ids(const gem_store* s, const float* T, const int64_t* q_offsets, int32_t n_queries,
                               int max_np, const int64_t* cand_offsets, const int64_t* cand_ids, float* out,
                               int* status, unsigned long long* counter, cudaStream_t st);
gem_status launch_cluster_index(gem_store* s, cudaStream_t st);
gem_status launch_qemd(const gem_store* s, const int64_t* set_a, const int64_t* set_b, int64_t n_pairs, float* out,
                       int* status, cudaStream_t st);
gem_status launch_wait_selftest(int* status, long long budget, cudaStream_t st);
gem_status launch_mark_deleted(gem_store* s, const int64_t* ids, int64_t n, bool deleted, cudaStream_t st);
gem_status beam_search(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                       int32_t n_queries, const int64_t* graph_off, const int32_t* graph_nbrs, int32_t max_degree,
                       const uint32_t* cluster_mask, const int64_t* entries, int32_t entry_stride, int32_t ef,
                       int32_t max_rounds, int64_t* out_ids, float* out_scores, int32_t* out_rounds, cudaStream_t stm);
gem_status launch_entry_points(const gem_store* s, const int32_t* lists, const int32_t* counts, int32_t n_queries,
                               int32_t stride, uint64_t seed, int64_t* out, cudaStream_t st);
gem_status launch_cluster_filter(const float* q, const int64_t* q_offsets, int32_t n_queries, const float* centroids,
                                 int32_t k2, int32_t t, int32_t cap, uint32_t* out_mask, int32_t* out_list,
                                 int32_t* out_count, int n_sm, cudaStream_t st);
// NN codes of n rows (ties to the lowest index, FP32 chain per dot).  From
// kAssignTcMinRows rows and kAssignTcMinCentroids centroids on the tensor cores
// (assign_tc.cu: the same codes; allocates stream-ordered scratch and blocks
// until done), otherwise the FP32 SIMT kernel (asynchronous).
constexpr int64_t kAssignTcMinRows = 16384;
constexpr int kAssignTcMinCentroids = 64;
gem_status launch_assign(const float* X, int64_t n, const float* C, int k1, int32_t* codes, float* best,
                         cudaStream_t st);
gem_status launch_assign_tc(const float* X, int64_t n, const float* C, int k1, int32_t* codes, float* best,
                            int n_sm, cudaStream_t st);
// The same tensor-core assignment of the rows 0 .. *n_dev - 1 (at most max_n)
// as stream work only: scratch of assign_tc_scratch_bytes(max_n, k1) bytes from
// the caller, no allocation and no host wait, so that it can be captured into a
// graph.  A bounded wait that gives up writes its code to *status (null: a word
// of the scratch).  assign_tc_prepare() sets the kernel's shared-memory limit
// and is called once outside any capture.
size_t assign_tc_scratch_bytes(int64_t max_n, int k1);
cudaError_t assign_tc_prepare();
gem_status enqueue_assign_tc(const float* X, int64_t max_n, const int64_t* n_dev, const float* C, int k1,
                             int32_t* codes, float* best, void* scratch, int* status, int n_sm, cudaStream_t st);
// the SIMT assignment of the rows rows[0 .. *n_dev - 1] (at most max_n) of X
gem_status launch_assign_rows(const float* X, int64_t max_n, const int64_t* n_dev, const int32_t* rows,
                              const float* C, int k1, int32_t* codes, float* best, int n_sm, cudaStream_t st);
// the same codes as launch_assign; with few rows the centroids are split over
// CTAs and merged through scratch [n] (one 64-bit key per row)
gem_status launch_assign_split(const float* X, int64_t n, const float* C, int k1, int32_t* codes,
                               unsigned long long* scratch, int n_sm, cudaStream_t st);
gem_status launch_assign_dev_n(const float* X, int64_t max_n, const int64_t* n_dev, const float* C, int k1,
                               int32_t* codes, cudaStream_t st);
gem_status launch_kmeans_step(const float* X, int64_t n, const int32_t* codes, double* sums, int* counts,
                              int k1, float* C, cudaStream_t st);
gem_status launch_gather_rows(const float* src, const int64_t* rows, int64_t n, float* dst, cudaStream_t st);
gem_status launch_qch(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                      int32_t n_queries, int64_t n_q_rows, const int64_t* cand_offsets,
                      const int64_t* cand_ids, float* est, cudaStream_t st);

// FP32 -> bf16 / e4m3 store copies in the padded layout.
void launch_quantize_bf16(const float* src, const int64_t* off, const int64_t* pad_off,
                          int64_t n_sets, __nv_bfloat16* dst, cudaStream_t st);
void launch_quantize_fp8(const float* src, const int64_t* off, const int64_t* pad_off,
                         int64_t n_sets, uint8_t* dst, float* scale, cudaStream_t st);
void launch_quantize_fp8_set(const float* src, const int64_t* off, const int64_t* pad_off,
                             int64_t n_sets, uint8_t* dst, float* set_scale, cudaStream_t st);

// Build the uniform rerank-pool offsets b * depth.
void launch_iota_offsets(int64_t* off, int32_t n, int64_t step, cudaStream_t st);

}  // namespace gem
