/*
 * gem.h -- C ABI of the B300 (sm_103a) multi-vector scoring library.
 *
 * The library scores query vector sets against a CSR-packed store of document
 * vector sets under the Chamfer / MaxSim similarity of GEM (arXiv 2603.20336,
 * Sec. 3.1, Definition 1, Eq. 1):
 *
 *     CH(Q, P) = sum over q in Q of  max over p in P of <q, p>
 *
 * with Sim taken as the inner product (cosine on the unit-norm vectors the
 * paper's encoders emit).  Scores are similarities: higher is better.
 *
 * Conventions shared by every call
 *  - Vectors have d = 128 float32 components, rows packed contiguously.
 *  - A set collection is CSR-packed: set i owns rows offsets[i] .. offsets[i+1]-1;
 *    offsets is int64 with offsets[0] = 0 and strictly increasing (no empty set).
 *  - Unless a parameter says "host", every pointer is a device pointer that the
 *    caller allocated and owns; the library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is asynchronous on that stream; outputs are valid once the stream
 *    reaches the call.  Calls on a workspace allocate no device memory, so they
 *    may be captured into a CUDA graph.
 *  - Errors: invalid arguments are detected on the host before anything is
 *    enqueued and returned synchronously (the outputs are left untouched).
 *    Inconsistent device-resident metadata (non-monotone offsets, ids outside
 *    [0, n_sets)) and bounded-wait timeouts are recorded in the workspace's
 *    device status word; gem_stream_status() returns it.
 *    gem_last_error_message() describes the last synchronous error of the
 *    calling thread.
 *  - A store is immutable after creation and may be shared by concurrent calls;
 *    a workspace must be used by one stream at a time.
 *  - Test hook, off unless set: the environment variable GEM_FAULT_INJECT=alloc:N
 *    makes the N-th device allocation of gem_store_create / gem_workspace_create
 *    fail with GEM_ERR_OOM (counted from the first allocation after the variable
 *    took its value); the call unwinds what it had built.
 *  - Each entry point marks its host time with an NVTX range of its own name
 *    (gem_search also its four stages), which profilers can filter on.
 */
#ifndef GEM_H_
#define GEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GEM_OK = 0,
  GEM_ERR_INVALID = 1,     /* bad argument or inconsistent metadata */
  GEM_ERR_OOM = 2,         /* device allocation failed (creation calls only) */
  GEM_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  GEM_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
  GEM_ERR_UNSUPPORTED = 5, /* device is not sm_103, or an unsupported option */
  GEM_ERR_STATE = 6,       /* object lacks what the call needs (e.g. no bf16 copy) */
  GEM_ERR_BOUNDS = 7       /* a device-side index check failed */
} gem_status;

/* Arithmetic of the scoring pass. */
typedef enum {
  GEM_F32 = 0,      /* FP32 SIMT, fixed summation order, Kahan sum over query vectors */
  GEM_BF16 = 1,     /* BF16 operands on tcgen05 tensor cores, FP32 accumulation */
  GEM_FP8_E4M3 = 2, /* E4M3 operands with per-vector FP32 scales, FP32 accumulation */
  GEM_CODES = 3,    /* id lists only: the GEM_F32 arithmetic with every query and stored
                       vector replaced by its centroid (the quantized estimate) */
  GEM_FP8_E4M3_SET = 4  /* E4M3 operands, one power-of-two scale per stored set (per-vector
                           scales for the query rows), FP32 accumulation: the set's scale
                           multiplies once per set instead of once per stored vector */
} gem_dtype;

/* Launch variants of the tensor-core scoring kernels (gem_workspace_set_schedule). */
typedef enum {
  GEM_TC_PLAIN = 0,    /* query block in shared memory, one set of epilogue warps */
  GEM_TC_A_TMEM = 1,   /* query block in tensor memory (m_tiles = 2) */
  GEM_TC_TWO_SETS = 2  /* two sets of epilogue warps on alternate tiles (m_tiles = 2) */
} gem_tc_variant;

/* Sim of Definition 1 (Eq. 1) for the exact scorers (gem_workspace_set_similarity). */
typedef enum {
  GEM_SIM_IP = 0,  /* inner product (cosine on unit vectors): CH = sum_i max_j <q_i, p_j> */
  GEM_SIM_L2 = 1   /* negated L2 distance: CH = -sum_i min_j ||q_i - p_j||_2 */
} gem_sim;

/* Form of the quantized Chamfer estimate qCH (gem_workspace_set_qch_form). */
typedef enum {
  GEM_QCH_SYMMETRIC = 0,  /* Eq. 16 as written: both the query vectors and the stored
                             vectors replaced by their nearest centroids */
  GEM_QCH_ASYMMETRIC = 1  /* only the stored vectors replaced: sum_i max_j <q_i, C_{NN(p_j)}> */
} gem_qch_form;

/* Which copies of the vectors a store keeps (bit mask). */
enum {
  GEM_KEEP_F32 = 1u,   /* FP32 master copy (needed by GEM_F32 scoring and the rerank) */
  GEM_KEEP_BF16 = 2u,  /* BF16, round to nearest even */
  GEM_KEEP_FP8 = 4u,   /* E4M3 codes + per-vector FP32 scale s_j = max_k |x_jk| / 448 */
  GEM_KEEP_FP8_SET = 8u /* E4M3 codes + one scale per set: the smallest power of two s
                           (>= FLT_MIN) with max |x| over the set <= 448 s (1 for a zero
                           set); x / s is exact and only the E4M3 rounding remains */
};

/* Internal arrays a store can copy out (gem_store_export).  The bf16 and
 * E4M3 copies use a padded layout: set i owns rows pad_offsets[i] ..
 * pad_offsets[i+1]-1, its length rounded up to a multiple of 8, and the extra
 * rows repeat the set's last vector (a repeated vector leaves every maximum of
 * Eq. 1 unchanged). */
enum {
  GEM_EXPORT_BF16 = 0,        /* uint16 [n_pad_vecs * 128] bfloat16 bit patterns */
  GEM_EXPORT_FP8 = 1,         /* uint8  [n_pad_vecs * 128] E4M3 bit patterns */
  GEM_EXPORT_FP8_SCALE = 2,   /* float  [n_pad_vecs] per-vector scales */
  GEM_EXPORT_OFFSETS = 3,     /* int64  [n_sets + 1] */
  GEM_EXPORT_PAD_OFFSETS = 4, /* int64  [n_sets + 1] offsets of the padded layout */
  GEM_EXPORT_CODES = 5,       /* int32  [n_vecs] NN code of every stored vector */
  GEM_EXPORT_CODEBOOK = 6,    /* float  [k1 * 128] centroids of C_quant */
  GEM_EXPORT_INDEX_CODES = 7, /* int32  [n_vecs] nearest C_index centroid of every stored vector */
  GEM_EXPORT_F32 = 8,         /* float  [n_vecs * 128] FP32 master copy (original row order) */
  GEM_EXPORT_INDEX_CENTROIDS = 9, /* float [k2 * 128] centroids of C_index */
  GEM_EXPORT_DELETED = 10,    /* uint32 [ceil(n_sets / 32)] deletion bitmap (all zero if none) */
  GEM_EXPORT_FP8_SET = 11,    /* uint8  [n_pad_vecs * 128] E4M3 bit patterns of the per-set-scale copy */
  GEM_EXPORT_SET_SCALE = 12   /* float  [n_sets] the per-set scales of that copy */
};

typedef struct gem_store gem_store;
typedef struct gem_workspace gem_workspace;
typedef struct gem_batch gem_batch;

/* Library version, major * 10000 + minor * 100 + patch. */
int gem_version(void);

/* Human-readable text of the last synchronous error on the calling thread. */
const char* gem_last_error_message(void);

/* Checks that `device` is an sm_103 GPU (B300).  GEM_ERR_UNSUPPORTED otherwise. */
gem_status gem_device_check(int device);

/*
 * Builds a store of n_sets vector sets (the database D of Sec. 3.1, problem
 * statement).  vecs: float32 [offsets[n_sets] * dim]; offsets: int64 [n_sets+1].
 * inputs_on_host != 0: vecs and offsets are host pointers (copied in);
 * otherwise device pointers (copied; the caller keeps ownership).  dim must be
 * 128.  keep_mask: GEM_KEEP_* bits, at least one.  Sets must be non-empty.
 * The call synchronises `stream` once (it reads the offsets on the host to plan
 * the tile map).  On success *out owns all of its device memory.
 */
gem_status gem_store_create(const float* vecs, const int64_t* offsets, int64_t n_sets, int32_t dim,
                            uint32_t keep_mask, int inputs_on_host, void* stream, gem_store** out);
void gem_store_destroy(gem_store* store);

/* Sizes of a store (n_pad_vecs: rows of the padded bf16 / E4M3 layout).  Any
 * output pointer may be NULL. */
gem_status gem_store_info(const gem_store* store, int64_t* n_sets, int64_t* n_vecs,
                          int64_t* n_pad_vecs, uint32_t* keep_mask);

/* k1 = |C_quant| and k2 = |C_index| attached to the store (0 when absent). */
gem_status gem_store_codebook_sizes(const gem_store* store, int32_t* k1, int32_t* k2);

/*
 * gem_store_save / gem_store_load: a store on disk (the paper's index is
 * persisted between runs; it gives no format).  The file holds what cannot be
 * re-derived: the set offsets, the FP32 vectors, C_quant, C_index and the
 * deletion bitmap (layout in csrc/persist.cu: a 48-byte header with magic,
 * version and sizes, the arrays in that order, an 8-byte trailer).  Loading
 * rebuilds every other array with the same kernels as the original build (bf16
 * and E4M3 copies, codes, index codes, cluster members), so the loaded store
 * scores exactly as the saved one.  Host I/O; both calls block until done.
 *   save: the store must keep GEM_KEEP_F32 (else GEM_ERR_STATE).
 *   load: keep_mask chooses the copies of the new store (as in
 *         gem_store_create; GEM_KEEP_F32 is required when the file holds
 *         centroids).  The store is created on the current device.
 * Errors: GEM_ERR_INVALID (NULL, a path that cannot be opened, a failed write,
 * a file that is not a store, of another version, with a corrupt header or
 * offsets, or shorter or longer than its header says), GEM_ERR_OOM.
 */
gem_status gem_store_save(const gem_store* store, const char* path, void* stream);
gem_status gem_store_load(const char* path, uint32_t keep_mask, void* stream, gem_store** out);

/* Copies one internal array (GEM_EXPORT_*) into the device buffer dst of
 * dst_bytes bytes (must be at least the array's size). */
gem_status gem_store_export(const gem_store* store, int32_t what, void* dst, size_t dst_bytes,
                            void* stream);

/*
 * Nearest-centroid codes NN(x) = argmax_c <x, C_c> (Sec. 4.1.1 and Sec. 4.2.2:
 * each vector maps to its closest centroid of C_quant; with unit vectors and
 * centroids, closest under d_X = 1 - <x, c> is largest inner product).  Dot
 * products are FP32 fused multiply-add chains over k = 0..127; ties go to the
 * lowest index.  x float32 [n * 128], centroids float32 [k1 * 128], codes int32
 * [n]; best (may be NULL) receives the winning inner product.  Device pointers.
 * A NaN dot product counts as -inf, so every code lies in [0, k1) (a row whose
 * dots are all NaN gets code 0).
 * From 16,384 rows and 64 centroids the work runs on the tensor cores with the
 * same result (codes and best values bit for bit): rows and centroids split
 * into two bf16 parts, three products per dot, the centroids within the
 * products' error band of each row's maximum rechecked with the FP32 chain
 * above, and the FP32 kernel for rows with more near-ties than that.  That path
 * allocates stream-ordered scratch (512 bytes per centroid, 512 bytes per row
 * for up to 4M rows at a time, 4 bytes per row) and blocks until done; smaller
 * calls are asynchronous and allocate nothing.
 */
gem_status gem_assign_codes(const float* x, int64_t n, const float* centroids, int32_t k1,
                            int32_t* codes, float* best, void* stream);

/*
 * Stage-1 k-means of Sec. 4.1.1 (spherical Lloyd: assign with gem_assign_codes,
 * then each centroid becomes the L2-normalised mean of its vectors; a centroid
 * without vectors, or whose vectors sum to zero, keeps its value).  Runs on `sample` vectors of the store's
 * FP32 copy drawn with `seed` (all vectors if sample <= 0 or >= n_vecs),
 * initialised with k1 distinct sampled vectors, for `iters` iterations.
 * centroids_out float32 [k1 * 128] (device).  A build step: allocates its own
 * scratch and synchronises `stream`.  The paper sizes k1 as
 * 2^floor(log2(16 sqrt(#vectors))) (Sec. 5.1).
 */
gem_status gem_train_codebook(const gem_store* store, int32_t k1, int32_t iters, int64_t sample,
                              uint64_t seed, float* centroids_out, void* stream);

/*
 * Attaches C_quant (float32 [k1 * 128], device, unit rows expected) to the
 * store and assigns the code of every stored vector (needs GEM_KEEP_F32).  A
 * build step: synchronises `stream`; not concurrent with other calls on the
 * store.  Workspaces created afterwards can run gem_estimate_codes.
 */
gem_status gem_store_set_codebook(gem_store* store, const float* centroids, int32_t k1, void* stream);

/*
 * gem_kmeans: spherical k-means (Sec. 4.1.1, two-stage clustering) of the rows
 * of any device matrix x [n x 128] FP32; the second stage clusters the stage-1
 * codebook C_quant (k1 rows) into k2 coarse centroids C_index.  The initial
 * centroids are k distinct rows of x picked by a seeded shuffle; each of `iters`
 * Lloyd steps assigns every row to its nearest centroid (largest inner product,
 * ties to the lower index) and sets each centroid with members to the
 * renormalised mean of its members.  centroids_out [k x 128] FP32 device,
 * caller-owned.  Blocks until done (it frees its temporaries).
 * Errors: GEM_ERR_INVALID (NULL, k outside 1..n, iters < 0), GEM_ERR_OOM.
 */
gem_status gem_kmeans(const float* x, int64_t n, int32_t k, int32_t iters, uint64_t seed, float* centroids_out,
                      void* stream);

/*
 * gem_cluster_filter: C_query of every query set (Sec. 4.5.1, Eq. 15;
 * Algorithm 5, first two steps).  S = C_index Q^T scores the k2 centroids
 * against every query vector (one FP32 FMA chain over k = 0..127 per dot); each
 * query vector keeps its top-t centroids (largest score, ties to the lower
 * centroid index) and C_query is their union over the query set.
 *   q [n_q_rows x 128], q_offsets [n_queries + 1]  query sets (device)
 *   centroids [k2 x 128]                           C_index (device)
 *   t                                              1 .. min(8, k2)
 *   out_mask  uint32 [n_queries x ceil(k2 / 32)]   bit c of row b: centroid c in C_query(b)
 *   out_list  int32 [n_queries x max_q_len * t]    C_query(b) ascending in row b
 *   out_count int32 [n_queries]                    |C_query(b)|; entries past the
 *                                                  row capacity max_q_len * t
 *                                                  (queries longer than max_q_len)
 *                                                  are in the mask only
 * All buffers are device, caller-owned.  Asynchronous on `stream`.
 * Errors: GEM_ERR_INVALID (NULL, k2 outside 1..262144, t outside 1..min(8, k2)).
 */
gem_status gem_cluster_filter(const float* q, const int64_t* q_offsets, int32_t n_queries, int32_t max_q_len,
                              const float* centroids, int32_t k2, int32_t t, uint32_t* out_mask, int32_t* out_list,
                              int32_t* out_count, void* stream);

/*
 * gem_qemd: quantized earth mover's distance between pairs of stored sets
 * (Sec. 4.2.2, Eq. 14; EMD of Eq. 11-12 with every vector replaced by its
 * nearest C_quant centroid, Eq. 13): the minimum over transport plans T >= 0
 * whose rows sum to 1/m1 and columns to 1/m2 of sum_ij T_ij (1 - <C_a_i, C_b_j>).
 * It is the edge weight the paper builds its graph with; this call computes it
 * exactly (successive shortest paths on the transportation problem between the
 * sets' distinct codes, integer masses) with FP32 costs (one FMA chain per
 * centroid dot, clamped at 0) and an FP64 final sum.
 *   set_a, set_b int64 [n_pairs]   stored set ids (device)
 *   out float [n_pairs]            qEMD of (set_a[p], set_b[p]) (device)
 * Sets of at most 128 vectors.  Device-side: an id outside [0, n_sets) scores
 * NaN and records GEM_ERR_BOUNDS, a longer set scores NaN and records
 * GEM_ERR_INVALID in the workspace's status word.  Asynchronous on `stream`.
 * Errors: GEM_ERR_INVALID (NULL, n_pairs < 0), GEM_ERR_STATE (no codebook).
 */
gem_status gem_qemd(const gem_store* store, gem_workspace* ws, const int64_t* set_a, const int64_t* set_b,
                    int64_t n_pairs, float* out, void* stream);

/*
 * gem_store_mark_deleted: lazy deletion (Sec. 4.6).  deleted != 0 marks every
 * set in ids (int64 [n], device) deleted, deleted == 0 restores them.  A deleted
 * set stays in the store and in any graph over it: gem_beam_search still
 * traverses it, and every scoring call still scores it, but gem_topk,
 * gem_search and the R of gem_beam_search never return it.  Repeated ids are
 * fine.  Blocks until the ids are checked.  The bitmap is updated on `stream`:
 * calls on other streams that read this store see the change only once they
 * are ordered after it (the same rule as any other device write).
 * Errors: GEM_ERR_INVALID (NULL with n > 0, n < 0, an id outside [0, n_sets):
 * then no bit changes), GEM_ERR_OOM (the first call allocates ceil(n_sets / 32)
 * + 1 words).
 */
gem_status gem_store_mark_deleted(gem_store* store, const int64_t* ids, int64_t n, int32_t deleted, void* stream);

/*
 * gem_store_set_index_centroids: attach C_index (k2 coarse centroids, device
 * [k2 x 128] FP32, copied) to the store; every stored vector gets its nearest
 * C_index centroid (largest inner product, ties to the lower index; exported as
 * GEM_EXPORT_INDEX_CODES) and every cluster the list of sets with a vector in it
 * (the set's C(P), Sec. 4.1.1, Eq. 4).  Needs the FP32 copy.  Blocks until done.
 * Errors: GEM_ERR_INVALID (NULL, k2 outside 1..262144), GEM_ERR_STATE (no FP32
 * copy), GEM_ERR_OOM.
 */
gem_status gem_store_set_index_centroids(gem_store* store, const float* centroids, int32_t k2, void* stream);

/*
 * gem_entry_points: E of Algorithm 5 (Sec. 4.5.2): one random member set from
 * every cluster of each query's C_query.
 *   cluster_lists  int32 [n_queries x stride]  C_query(b) in row b (as written by
 *                                              gem_cluster_filter with stride =
 *                                              max_q_len * t)
 *   cluster_counts int32 [n_queries]           entries of row b in use (min with
 *                                              stride)
 *   out_sets       int64 [n_queries x stride]  the drawn set of each cluster; -1
 *                                              for unused slots and empty clusters
 * The draw for (query b, cluster c) is the member set s with the smallest
 * H(seed, b, c, s), then the lower s, where H = out(out(out(seed + b) + c) + s)
 * and out(x) is the SplitMix64 output from state x: uniform over the cluster's
 * member sets and reproducible for a given seed.  Device buffers, caller-owned;
 * asynchronous on `stream`.
 * Errors: GEM_ERR_INVALID (NULL, stride < 1), GEM_ERR_STATE (no C_index).
 */
gem_status gem_entry_points(const gem_store* store, const int32_t* cluster_lists, const int32_t* cluster_counts,
                            int32_t n_queries, int32_t stride, uint64_t seed, int64_t* out_sets, void* stream);

/*
 * gem_beam_search: cluster-guided multi-path beam search (Algorithm 5,
 * Sec. 4.5.3) of a batch of queries over a graph of the stored sets, scored by
 * qCH (the arithmetic of gem_estimate_codes, from centroid tables built once per
 * call; similarity qsim = m_q - qCH) and run in rounds.  Each round every non-empty queue W_e (one per entry set, in entry
 * order) pops its best set P; P scoring below tau (the worst score in R once R
 * holds ef sets) empties W_e, else every neighbour of P (in list order) that is
 * not visited and has a vector in a cluster of C_query is marked visited, scored,
 * and inserted (in that order) into W_e and R.  W_e and R keep the ef best sets
 * (higher score, then lower id).  Rounds run until every queue is empty or
 * max_rounds have run.
 *   graph_off int64 [n_sets + 1], graph_nbrs int32  neighbour lists (device), each
 *                                                   at most max_degree long, ids
 *                                                   in [0, n_sets), no repeats
 *   cluster_mask uint32 [n_queries x ceil(k2/32)]   C_query (gem_cluster_filter)
 *   entries int64 [n_queries x entry_stride]       entry sets (gem_entry_points);
 *                                                   -1 and repeats are skipped
 *   out_ids int64, out_scores float [n_queries x ef] R best first; -1 / -inf past
 *                                                   its size
 *   out_rounds (host int32, may be NULL)            rounds run
 * A set the store marks deleted (gem_store_mark_deleted) is scored, queued and
 * expanded like any other but never enters R.
 * Needs the store's codebook (before the workspace was created) and C_index
 * (gem_store_set_index_centroids).  Allocates its scratch and blocks until done.
 * Errors: GEM_ERR_INVALID (NULL, ef outside 1..4096, bad sizes, more than 65,535
 * query parts of 32 rows, a neighbour id out of range or a list longer than
 * max_degree), GEM_ERR_STATE, GEM_ERR_OOM (the tables take n_queries x
 * ceil(max_q_len / 32) x k1 x 128 bytes).
 */
gem_status gem_beam_search(const gem_store* store, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                           int32_t n_queries, int64_t n_q_rows, const int64_t* graph_off, const int32_t* graph_nbrs,
                           int32_t max_degree, const uint32_t* cluster_mask, const int64_t* entries,
                           int32_t entry_stride, int32_t ef, int32_t max_rounds, int64_t* out_ids, float* out_scores,
                           int32_t* out_rounds, void* stream);

/*
 * Scratch for scoring calls against `store`.  Bounds fix the memory once:
 *   max_queries  -- query sets per call
 *   max_q_rows   -- total query vectors per call
 *   max_q_len    -- vectors in the longest query set (1..256)
 *   max_cands    -- candidate ids per call (gem_score_ids and the rerank pool
 *                   of gem_search: n_queries * rerank_depth)
 *   max_k        -- largest k for gem_topk / gem_search (1..4096)
 */
gem_status gem_workspace_create(const gem_store* store, int32_t max_queries, int64_t max_q_rows,
                                int32_t max_q_len, int64_t max_cands, int32_t max_k,
                                gem_workspace** out);
void gem_workspace_destroy(gem_workspace* ws);

/*
 * Sim of Definition 1 for every exact score computed through this workspace
 * (gem_score_all, gem_score_ids, gem_search, gem_search_host).  Default
 * GEM_SIM_IP.  GEM_SIM_L2 (Sim(a, b) = -||a - b||_2, so higher is still better)
 * runs on the FP32 scorers only: each term is -sqrt(min_j sum_k (q_ik - p_jk)^2),
 * every difference rounded to FP32 and squared into the same two 64-term FMA
 * chains as the dot product, then the same Kahan sum over query vectors.  Under
 * GEM_SIM_L2, GEM_BF16 / GEM_FP8_E4M3 scoring, the codes form, gem_estimate_codes
 * and gem_beam_search return GEM_ERR_UNSUPPORTED (qCH is defined for the
 * inner-product Sim).  gem_batch and gem_maxsim_fwd / _bwd use the inner product.
 * Errors: GEM_ERR_INVALID (NULL, unknown sim).
 */
gem_status gem_workspace_set_similarity(gem_workspace* ws, int32_t sim);

/*
 * Form of every qCH estimate computed through this workspace: gem_estimate_codes,
 * gem_score_ids with GEM_CODES and gem_beam_search.  Default
 * GEM_QCH_SYMMETRIC.  The asymmetric form keeps the query vectors exact (the
 * tables hold <q_i, C_c>), so no query codes are assigned.
 * Errors: GEM_ERR_INVALID (NULL, unknown form).
 */
gem_status gem_workspace_set_qch_form(gem_workspace* ws, int32_t form);

/*
 * Schedule of the tensor-core scoring kernels on this workspace (the knobs the
 * autotuner varies; results do not depend on them):
 *   m_tiles     resident query rows per CTA / 128: 1, 2 or 4 (document tile
 *               width 256 / m_tiles columns)
 *   variant     GEM_TC_PLAIN: query rows in shared memory, one set of 4 *
 *               m_tiles epilogue warps;
 *               GEM_TC_A_TMEM: the query rows live in tensor memory and the MMAs read only
 *               the document tile from shared memory (m_tiles = 2 only; tile
 *               width 96);
 *               GEM_TC_TWO_SETS: two sets of epilogue warps take alternate tiles
 *               (m_tiles = 2 only)
 *   default: m_tiles 2, GEM_TC_PLAIN, chunk_rows 2^16
 *   chunk_rows  document rows per work unit (whole sets; 1024 .. 2^24)
 */
gem_status gem_workspace_set_schedule(gem_workspace* ws, int32_t m_tiles, int32_t variant, int32_t chunk_rows);

/*
 * Exact CH of every query set against every stored set (Eq. 1 for all P in D,
 * the scores ranked by Eq. 2).
 *   q          float32 [n_q_rows * 128] query vectors, CSR by q_offsets
 *   q_offsets  int64 [n_queries + 1] (device), q_offsets[n_queries] == n_q_rows
 *   compute    GEM_F32 (FP32 SIMT), GEM_BF16, GEM_FP8_E4M3 or GEM_FP8_E4M3_SET
 *              (tensor cores; the store must keep that copy)
 *   scores     float32 [n_queries * n_sets], row-major: scores[b * n_sets + n]
 */
gem_status gem_score_all(const gem_store* store, gem_workspace* ws, const float* q,
                         const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                         int32_t compute, float* scores, void* stream);

/*
 * Exact CH over per-query candidate lists (the candidate scoring of one
 * beam-search expansion, Algorithm 5).
 *   cand_offsets  int64 [n_queries + 1] (device), cand_offsets[n_queries] == n_cands
 *   cand_ids      int64 [n_cands]; ids of query b are cand_ids[cand_offsets[b] ..
 *                 cand_offsets[b+1]-1]; each must lie in [0, n_sets) (a negative id
 *                 is an empty slot and scores -inf; an id >= n_sets records
 *                 GEM_ERR_BOUNDS and scores NaN).  Duplicates are scored per position.
 *   scores        float32 [n_cands], aligned with cand_ids
 * compute GEM_F32 uses FP32 FMA in a fixed order per dot product and a Kahan
 * (compensated) sum over the query vectors in ascending order.
 */
gem_status gem_score_ids(const gem_store* store, gem_workspace* ws, const float* q,
                         const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                         const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                         int32_t compute, float* scores, void* stream);

/*
 * gem_rerank_pool: the exact rescoring of a rerank pool, the final step of
 * Algorithm 5 (exact CH of Sec. 3.1 Eq. 1 over the pool the first pass kept)
 * as its own call, the step gem_search runs between its two top-k selections.
 *   pool_ids     int64 [n_queries x depth], row b = query b's pool (-1 = empty
 *                entry: score -inf; an id >= n_sets: NaN and GEM_ERR_BOUNDS in
 *                gem_workspace_status)
 *   pool_scores  float32 [n_queries x depth] (output)
 * The scores are those of gem_score_ids with GEM_F32 over the rows as per-query
 * lists (bit-identical).  From 65,536 entries the pool is scored in the order of
 * its set ids (up to 64 ranges of ids, then query), so that a set in several
 * queries' pools is read from DRAM about once; the output order is unaffected.
 * Needs GEM_KEEP_F32 and a workspace with max_k > 0 and max_cands >= n_queries x
 * depth.  Device buffers, caller-owned; asynchronous on `stream`.
 */
gem_status gem_rerank_pool(const gem_store* store, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                           int32_t n_queries, int64_t n_q_rows, const int64_t* pool_ids, int32_t depth,
                           float* pool_scores, void* stream);

/*
 * Quantized Chamfer estimate (Sec. 4.5.3, Eq. 16) in similarity form:
 *   est = sum_i max_j <C_{NN(q_i)}, C_{NN(p_j)}> = m_q - qCH(Q, P)
 * The query vectors are coded on the fly; stored vectors use the store's codes.
 * cand_offsets == NULL: every stored set, est float32 [n_queries * n_sets]
 * row-major; otherwise est is aligned with cand_ids as in gem_score_ids.  The
 * store needs a codebook before the workspace is created.
 */
gem_status gem_estimate_codes(const gem_store* store, gem_workspace* ws, const float* q,
                              const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                              const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                              float* est, void* stream);

/*
 * Per-row top-k (the k-argmax of Eq. 2): sorted by score descending, ties by
 * lower id.  Rows are either dense (row_offsets == NULL: row r is
 * scores[r * cols .. r * cols + cols - 1]) or ragged (row_offsets int64
 * [rows + 1], device).  ids == NULL: an element's id is its index within its
 * row; otherwise ids is int64 aligned with scores.  Ids must be < 2^32.
 * out_ids int64 [rows * k], out_scores float32 [rows * k] (may be NULL); a row
 * with fewer than k elements is padded with id -1 and score -inf.  NaN scores
 * are not supported.  An element whose id is a set the workspace's store marks
 * deleted (gem_store_mark_deleted) is not a candidate.
 */
gem_status gem_topk(gem_workspace* ws, const float* scores, const int64_t* row_offsets, int32_t rows,
                    int64_t cols, const int64_t* ids, int32_t k, int64_t* out_ids, float* out_scores,
                    void* stream);

/*
 * Exhaustive search with an exact rerank (Eq. 2 answered as in the last step
 * of Algorithm 5): score every stored set with `compute`, keep the top
 * rerank_depth per query, rescore that pool with exact FP32 CH (Kahan sum over
 * query vectors) and return the top k of it.  rerank_depth == 0 skips the
 * rerank (the top k of the first pass is returned).  Needs GEM_KEEP_F32 when
 * rerank_depth > 0.  Deleted sets (gem_store_mark_deleted) are scored but never
 * returned.  out_ids int64 [n_queries * k], out_scores float32 [n_queries * k].
 * compute:
 *   GEM_F32, GEM_BF16, GEM_FP8_E4M3, GEM_FP8_E4M3_SET
 *                                    the first pass is exact CH in that arithmetic
 *                                    (as gem_score_all);
 *   GEM_CODES                        the first pass is the quantized estimate qsim
 *                                    (Sec. 4.5.3, Eq. 16; as gem_estimate_codes over
 *                                    every set, in the workspace's qCH form), the
 *                                    estimate-then-exact-rerank order of Algorithm 5.
 *                                    Needs the store's codebook before the workspace
 *                                    was created and Sim = inner product.
 */
gem_status gem_search(const gem_store* store, gem_workspace* ws, const float* q,
                      const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                      int32_t compute, int32_t rerank_depth, int32_t k, int64_t* out_ids,
                      float* out_scores, void* stream);

/*
 * gem_search with HOST buffers: q, q_offsets, out_ids and out_scores are host
 * pointers (pinned memory gives overlapped copies).  The call copies the
 * queries in, runs the search on `stream`, copies the results out and
 * synchronises the stream before returning.
 */
gem_status gem_search_host(const gem_store* store, gem_workspace* ws, const float* q_host,
                           const int64_t* q_offsets_host, int32_t n_queries, int32_t compute,
                           int32_t rerank_depth, int32_t k, int64_t* out_ids_host,
                           float* out_scores_host, void* stream);

/*
 * MaxSim forward over (query, set) pairs with the argmax side output, for
 * training: S_t = sum_i max_j <q_i, p_j> (Eq. 1) for every pair t, and
 * argmax[t * max_q_len + i] = j*(t, i), the set row attaining the max (lowest j
 * on ties).  Vector sets are raw device arrays (not a store) so that gradients
 * can flow to them: q float32 [n_q_rows * 128] CSR by q_offsets [n_queries + 1];
 * docs float32 [n_doc_rows * 128] CSR by doc_offsets [n_docs + 1]; the pairs of
 * query b are pair_ids[pair_offsets[b] .. pair_offsets[b+1]-1] (set ids).
 * compute GEM_BF16 rounds every component to bfloat16 before the FP32
 * accumulation; GEM_F32 uses the FP32 values.  scores float32 [n_pairs];
 * argmax int32 [n_pairs * max_q_len].  ws (may be NULL) receives device-side
 * errors (an id outside [0, n_docs) scores NaN).
 * GEM_BF16 with max_q_len <= 128 runs on the tensor cores: the query rows are
 * first rounded into stream-ordered scratch (2 bytes per component of q, freed
 * at the end of the call), the set rows are read once as FP32 and rounded on
 * chip, and the sum over i is taken in a fixed order (32-row butterflies, then
 * in ascending blocks of 32); otherwise an FP32 SIMT kernel with a Kahan sum in
 * ascending i runs.
 */
gem_status gem_maxsim_fwd(const float* q, const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                          const float* docs, const int64_t* doc_offsets, int64_t n_docs, int64_t n_doc_rows,
                          const int64_t* pair_offsets, const int64_t* pair_ids, int64_t n_pairs, int32_t max_q_len,
                          int32_t compute, float* scores, int32_t* argmax, gem_workspace* ws, void* stream);

/*
 * Backward of gem_maxsim_fwd for upstream gradients grad_scores [n_pairs]:
 *   grad_q[i of query b] = sum over b's pairs t (ascending) of g_t * p_{j*(t,i)}
 *   grad_docs[row j of set d] = sum over pairs t of d of g_t * (sum of q_i with j*(t,i) = j)
 * with the FP32 input values (the bf16 rounding of the forward is treated as the
 * identity).  grad_q float32 [n_q_rows * 128] and grad_docs float32
 * [n_doc_rows * 128] are overwritten (either may be NULL); an argmax entry
 * outside its set's rows adds nothing.  grad_q is deterministic (one FMA chain
 * per element, pairs ascending).  grad_docs: with max_q_len <= 32 every row is
 * written once by its set (a set named by one pair gets its sums directly, a
 * set named by several pairs is zeroed and its pairs add with atomics), using
 * 12 bytes per set of stream-ordered scratch; otherwise it is zeroed and every
 * pair adds with atomics.  It is deterministic when no set occurs in two pairs.
 */
gem_status gem_maxsim_bwd(const float* q, const int64_t* q_offsets, int32_t n_queries, const float* docs,
                          const int64_t* doc_offsets, int64_t n_docs, int64_t n_doc_rows,
                          const int64_t* pair_offsets, const int64_t* pair_ids, int64_t n_pairs,
                          const int32_t* argmax, int32_t max_q_len, const float* grad_scores, float* grad_q,
                          float* grad_docs, void* stream);

/*
 * Batched candidate scoring: the scoring step of one beam-search expansion
 * (Algorithm 5, the neighbours of each popped node scored against its query) for
 * many queries with uneven set sizes and uneven candidate lists, as one
 * persistent launch replayed from a CUDA graph.
 *   mode         GEM_F32 (exact) or GEM_CODES (quantized); scores are
 *                bit-identical to gem_score_ids with the same compute
 *   max_*        capacity of the batch's own device buffers
 *   seg          candidates per work item (1..1024; the autotuner's knob)
 *   ctas_per_sm  persistent CTAs per SM (0 = as many as fit)
 * GEM_CODES needs a store codebook.  Each run of it first assigns the run's
 * query rows to their NN codes (from 16,384 rows of capacity and 64 centroids
 * on the tensor cores, the same codes as gem_assign_codes), for which the batch
 * then holds about 512 (k1 + min(max_q_rows, 2^22)) + 4 max_q_rows bytes of its
 * own device memory (bf16 halves of the centroids and rows, a fallback list).  The caller owns the device buffers the graph reads and writes; their addresses are fixed for the batch's lifetime and
 * the caller refills them before each run: q float32 [max_q_rows * 128],
 * q_offsets and cand_offsets int64 [max_queries + 1], cand_ids int64
 * [max_cands] (same meaning as in gem_score_ids), scores float32 [max_cands]
 * (output).  gem_batch_run scores n_queries queries with n_q_rows vectors and
 * n_cands candidates on `stream`; it first waits until the previous run of the
 * same batch has finished.  use_graph = 0 runs the same launches without the
 * graph.  Inconsistent offsets are reported by gem_batch_status.
 */
gem_status gem_batch_create(const gem_store* store, int32_t mode, int32_t max_queries, int64_t max_q_rows,
                            int32_t max_q_len, int64_t max_cands, int32_t seg, int32_t ctas_per_sm,
                            float* q, int64_t* q_offsets, int64_t* cand_offsets, int64_t* cand_ids,
                            float* scores, gem_batch** out);
gem_status gem_batch_run(gem_batch* batch, int32_t n_queries, int64_t n_q_rows, int64_t n_cands,
                         int32_t use_graph, void* stream);
/* Synchronises the batch's last run and returns and clears its device status. */
gem_status gem_batch_status(gem_batch* batch);
void gem_batch_destroy(gem_batch* batch);

/*
 * Autotuner.  Times the candidate schedules of a kernel with CUDA events on the
 * given inputs and keeps the fastest; results never depend on the schedule
 * (bit-identical scores).  cache_path (NULL: $GEM_TUNE_CACHE, unset: no cache)
 * names a JSON file of earlier choices keyed by device name, dtype and size
 * buckets; a hit applies the stored choice without timing (*from_cache = 1).
 * Setup calls: they launch the kernels several times, may allocate, and
 * synchronise `stream`.
 *
 * gem_autotune_score_all: schedules of gem_score_all for compute GEM_BF16 or
 * GEM_FP8_E4M3 ((m_tiles, variant) in {(2, TWO_SETS), (2, PLAIN), (4, PLAIN),
 * (2, A_TMEM), (1, PLAIN)} x
 * chunk_rows in {2^14, 2^15, 2^16}); the choice is applied to `ws` (as
 * gem_workspace_set_schedule).  scores float32 [n_queries * n_sets] is scratch
 * for the timing runs.
 */
gem_status gem_autotune_score_all(const gem_store* store, gem_workspace* ws, const float* q,
                                  const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                                  int32_t compute, float* scores, const char* cache_path, int32_t* m_tiles,
                                  int32_t* variant, int32_t* chunk_rows, float* ms, int32_t* from_cache,
                                  void* stream);

/*
 * gem_autotune_batch: schedules of a gem_batch (seg in {8, 16, 32, 64} x
 * ctas_per_sm in {1, 2, all}) on one representative round held in the given
 * device buffers (as for gem_batch_create); returns the fastest pair for
 * gem_batch_create.
 */
gem_status gem_autotune_batch(const gem_store* store, int32_t mode, int32_t n_queries, int64_t n_q_rows,
                              int32_t max_q_len, int64_t n_cands, float* q, int64_t* q_offsets,
                              int64_t* cand_offsets, int64_t* cand_ids, float* scores, const char* cache_path,
                              int32_t* seg, int32_t* ctas_per_sm, float* ms, int32_t* from_cache, void* stream);

/*
 * gem_score_ids_noalloc: id-list scoring that allocates no device memory.  The
 * paper has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: processes whose device memory is owned by another allocator (a host
 * framework's caching allocator, a serving runtime that reserves its whole
 * memory budget at start-up) and that therefore cannot create a gem_workspace or
 * a gem_batch.  It computes what gem_score_ids computes with GEM_F32 (same
 * arithmetic, bit-identical scores) using the batched scorer, whose work-plan
 * scratch lives in a fixed array of about 128 KB in device memory, one per GPU,
 * that every GPU loading this library keeps until the process exits.
 *   n_queries   at most 16384 (larger calls fail with GEM_ERR_INVALID)
 *   max_q_len   bound on the vectors of any query set (1..256)
 * The other arguments are as in gem_score_ids: all device pointers, caller-owned.
 * The store still comes from gem_store_create (GEM_KEEP_F32 needed).
 * Every call on a device shares that one array and it keeps the last call's
 * contents (each call resets what it needs), so calls whose work overlaps on
 * the GPU (two streams, or two host threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address and
 * sets a kernel attribute; make that first call before any stream capture.
 * Device-side problems are not reported through a status word: an id outside
 * [0, n_sets) scores NaN, a negative id scores -inf, and inconsistent
 * cand_offsets leave scores unwritten, as does a query set longer than
 * max_q_len (all of that query's scores stay unwritten).
 */
gem_status gem_score_ids_noalloc(const gem_store* store, const float* q, const int64_t* q_offsets,
                                 int32_t n_queries, int64_t n_q_rows, int32_t max_q_len,
                                 const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                                 float* scores, void* stream);

/*
 * Doc-range sharding (Eq. 2 over a database D split by set id into contiguous
 * ranges, one store per shard: one per GPU, or several on one GPU).  The four
 * calls below answer gem_search exactly -- bit for bit the same ids and scores
 * as gem_search on the whole store with the same compute, rerank_depth and k --
 * because every (query, set) score depends on the two sets alone:
 *   1. gem_shard_first_pass on every shard (its top rerank_depth, global ids);
 *   2. the lists gathered shard-major [n_shards][n_queries][rerank_depth] and
 *      gem_merge_topk(k = rerank_depth): the whole store's rerank pool;
 *   3. pool scores filled with -inf, then gem_shard_rerank on every shard (it
 *      writes the entries it owns); across GPUs an element-wise max of the
 *      shards' pool scores combines them;
 *   4. gem_topk(pool scores, ids = pool ids, k).
 *
 * gem_shard_ranges: the shard boundaries, host only (no device work).
 *   offsets_host   int64 [n_sets + 1] CSR offsets of the whole store (host)
 *   bounds_host    int64 [n_shards + 1] (host, caller-owned): shard s owns the
 *                  sets bounds[s] .. bounds[s+1]-1; bounds[0] = 0, bounds[n_shards]
 *                  = n_sets; each boundary is the set boundary closest to
 *                  s/n_shards of the vectors (balanced by vector count, not set
 *                  count), every shard non-empty.
 * Errors: GEM_ERR_INVALID (NULL, n_shards outside 1..n_sets, bad offsets).
 */
gem_status gem_shard_ranges(const int64_t* offsets_host, int64_t n_sets, int32_t n_shards, int64_t* bounds_host);

/*
 * gem_shard_first_pass: step 1 on the shard `store` (its sets are the global
 * sets id_base .. id_base + n_sets - 1): the first pass of gem_search with
 * `compute` (exact CH, or the qCH estimate for GEM_CODES) and its top `depth`
 * per query by (score desc, id asc).  out_ids int64 [n_queries x depth] hold
 * global set ids (-1 past the shard's size), out_scores float32 [n_queries x
 * depth]; device, caller-owned.  Needs a workspace created with max_k > 0.
 * Errors: as gem_search; GEM_ERR_INVALID for depth outside 1..4096 or id_base < 0.
 */
gem_status gem_shard_first_pass(const gem_store* store, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                                int32_t n_queries, int64_t n_q_rows, int32_t compute, int32_t depth, int64_t id_base,
                                int64_t* out_ids, float* out_scores, void* stream);

/*
 * gem_shard_rerank: step 3 on one shard: for every entry of pool_ids (int64
 * [n_queries x depth], global set ids, -1 = empty) that lies in the shard's
 * range, pool_scores (float32, same shape) receives its exact FP32 CH (the
 * arithmetic of gem_score_ids with GEM_F32); every other entry is left as it
 * is.  Needs GEM_KEEP_F32 and a workspace with max_k > 0 and max_cands >=
 * n_queries x depth.  Device buffers, caller-owned; asynchronous on `stream`.
 */
gem_status gem_shard_rerank(const gem_store* store, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                            int32_t n_queries, int64_t n_q_rows, const int64_t* pool_ids, int32_t depth,
                            int64_t id_base, float* pool_scores, void* stream);

/*
 * gem_shard_score_ids: candidate lists routed to their owner shard (the scoring
 * step of a beam expansion, Algorithm 5, over a sharded store).  cand_offsets
 * int64 [n_queries + 1] and cand_ids int64 [n_cands] are as in gem_score_ids
 * but hold GLOBAL set ids (-1 = empty); for every entry in the shard's range
 * (id_base .. id_base + n_sets - 1) scores[j] receives what gem_score_ids with
 * `compute` (GEM_F32 or GEM_CODES) gives on the whole store, bit for bit; every
 * other entry is left as it is.  With scores filled with -inf beforehand, an
 * element-wise max over the shards' buffers gives the whole-store scores.
 * Needs a workspace with max_cands >= n_cands.  Device buffers, caller-owned;
 * asynchronous on `stream`.
 */
gem_status gem_shard_score_ids(const gem_store* store, gem_workspace* ws, const float* q, const int64_t* q_offsets,
                               int32_t n_queries, int64_t n_q_rows, const int64_t* cand_offsets,
                               const int64_t* cand_ids, int64_t n_cands, int32_t compute, int64_t id_base,
                               float* scores, void* stream);

/*
 * gem_merge_topk: step 2: per row, the top k (score desc, id asc) of the union
 * of n_lists lists laid out [n_lists][rows][k_in] (scores float32, ids int64;
 * negative ids are empty slots).  out_ids int64 [rows x k], out_scores float32
 * [rows x k] (may be NULL), padded with -1 / -inf.  Ids must be < 2^32 and, for
 * an exact answer, distinct within a row.  Device buffers; asynchronous.
 * Errors: GEM_ERR_INVALID (NULL, bad shape, k outside 1..4096).
 */
gem_status gem_merge_topk(const float* scores, const int64_t* ids, int32_t n_lists, int32_t rows, int32_t k_in,
                          int32_t k, int64_t* out_ids, float* out_scores, void* stream);

/*
 * gem_measure_peaks: measured denominators for the roofline fractions of the
 * FP32 and table-lookup kernels (the paper has no counterpart; a measurement
 * helper).  fp32_tflops: FP32 FMA throughput of a full grid of packed two-lane
 * FMA chains (fma.rn.f32x2, as the FP32 scorers issue them), 2 flop per FMA.
 * l2_gather_gbs: bandwidth of warps reading 128-byte rows at hashed indices of a
 * 64 MB buffer held in L2 (the qCH table-lookup pattern).  Best of three timed
 * launches each.  Allocates and frees a 64 MB buffer and blocks until done.
 */
gem_status gem_measure_peaks(float* fp32_tflops, float* l2_gather_gbs, void* stream);

/* Number of kernels this library has enqueued since it was loaded (all
 * devices and threads); lets a caller count the library's launches in a region. */
int64_t gem_kernel_launches(void);

/* Synchronises `stream`, then returns and clears the workspace's device status
 * word (GEM_OK if no device-side error was recorded since the last check). */
gem_status gem_stream_status(gem_workspace* ws, void* stream);

/* Failure-detection self-test: one warp waits, through the same bounded
 * mbarrier wait every pipelined kernel uses, on a barrier nothing arrives on.
 * After budget_cycles SM cycles (1 .. 2^32) the wait gives up, records
 * GEM_ERR_TIMEOUT in the workspace's status word and the kernel returns; the
 * next gem_stream_status returns GEM_ERR_TIMEOUT and the context stays usable.
 * Asynchronous on `stream`.  Errors: GEM_ERR_INVALID (NULL, budget out of range). */
gem_status gem_selftest_wait_timeout(gem_workspace* ws, int64_t budget_cycles, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GEM_H_ */
