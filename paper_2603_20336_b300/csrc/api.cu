// C-ABI entry points of libgem (declared in include/gem.h): argument checks,
// object lifetime and the dispatch of each call onto the kernels.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <numeric>
#include <random>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace gem {

namespace {
thread_local std::string g_last_error;

bool device_is_sm103(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  return p.major == 10 && p.minor == 3;
}

gem_status check_current_device(int want) {
  int dev = -1;
  GEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != want) return fail(GEM_ERR_INVALID, "current device differs from the store's device");
  return GEM_OK;
}

// Host-side fault injection for tests, off unless GEM_FAULT_INJECT is set:
// "alloc:N" makes the N-th device allocation of the store and workspace
// creation calls fail as if the device were out of memory, counting from the
// first allocation after the variable took its current value.
bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* env = std::getenv("GEM_FAULT_INJECT");
  const std::string cur = env ? env : "";
  std::lock_guard<std::mutex> lk(mu);
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.rfind("alloc:", 0) != 0) return false;
  return ++count == std::strtol(cur.c_str() + 6, nullptr, 10);
}

template <typename T>
gem_status dmalloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return GEM_OK;
  if (injected_alloc_failure()) return fail(GEM_ERR_OOM, std::string("injected allocation failure for ") + what);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GEM_ERR_OOM, std::string("cudaMalloc failed for ") + what);
  }
  return GEM_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
}

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

gem_status fail(gem_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

gem_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return GEM_ERR_CUDA;
}

}  // namespace gem

using namespace gem;

extern "C" {

int gem_version(void) { return 100; }

const char* gem_last_error_message(void) { return g_last_error.c_str(); }

gem_status gem_device_check(int device) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return fail(GEM_ERR_UNSUPPORTED, "no CUDA device with that index");
  }
  if (!device_is_sm103(device)) return fail(GEM_ERR_UNSUPPORTED, "device is not sm_103 (B300)");
  return GEM_OK;
}

// ----------------------------------------------------------------------------- store

void gem_store_destroy(gem_store* s) {
  if (!s) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  dfree(s->d_offsets);
  dfree(s->d_pad_offsets);
  dfree(s->d_end_bits);
  dfree(s->d_f32);
  dfree(s->d_bf16);
  dfree(s->d_fp8);
  dfree(s->d_fp8_scale);
  dfree(s->d_fp8s);
  dfree(s->d_set_scale);
  dfree(s->d_codebook);
  dfree(s->d_codes);
  dfree(s->d_cindex);
  dfree(s->d_icodes);
  dfree(s->d_member_off);
  dfree(s->d_members);
  dfree(s->d_dead);
  for (auto& kv : s->chunks) dfree(kv.second.d_chunk_doc);
  cudaSetDevice(prev);
  delete s;
}

gem_status gem_store_create(const float* vecs, const int64_t* offsets, int64_t n_sets, int32_t dim,
                            uint32_t keep_mask, int inputs_on_host, void* stream, gem_store** out) {
  GEM_NVTX_RANGE("gem_store_create");
  if (!out) return fail(GEM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!vecs || !offsets) return fail(GEM_ERR_INVALID, "vecs/offsets is NULL");
  if (n_sets < 1 || n_sets >= (int64_t)1 << 31) return fail(GEM_ERR_INVALID, "n_sets out of range");
  if (dim != kDim) return fail(GEM_ERR_UNSUPPORTED, "only dim = 128 is supported");
  if (keep_mask == 0 || (keep_mask & ~15u)) return fail(GEM_ERR_INVALID, "bad keep_mask");
  int dev = 0;
  GEM_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_is_sm103(dev)) return fail(GEM_ERR_UNSUPPORTED, "device is not sm_103 (B300)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  gem_store* s = new gem_store();
  s->device = dev;
  s->keep = keep_mask;
  s->n_sets = n_sets;
  {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, dev);
    s->n_sm = p.multiProcessorCount;
  }
  s->h_offsets.resize(n_sets + 1);
  if (inputs_on_host) {
    std::memcpy(s->h_offsets.data(), offsets, sizeof(int64_t) * (n_sets + 1));
  } else {
    cudaError_t e = cudaMemcpyAsync(s->h_offsets.data(), offsets, sizeof(int64_t) * (n_sets + 1),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { gem_store_destroy(s); return cuda_fail(e, "reading offsets"); }
  }
  if (s->h_offsets[0] != 0) { gem_store_destroy(s); return fail(GEM_ERR_INVALID, "offsets[0] != 0"); }
  for (int64_t i = 0; i < n_sets; ++i) {
    const int64_t len = s->h_offsets[i + 1] - s->h_offsets[i];
    if (len < 1) { gem_store_destroy(s); return fail(GEM_ERR_INVALID, "empty or non-monotone set"); }
    if (len > s->max_set_len) s->max_set_len = len;
  }
  s->n_vecs = s->h_offsets[n_sets];
  s->h_pad_offsets.resize(n_sets + 1);
  s->h_pad_offsets[0] = 0;
  for (int64_t i = 0; i < n_sets; ++i) {
    const int64_t len = s->h_offsets[i + 1] - s->h_offsets[i];
    s->h_pad_offsets[i + 1] = s->h_pad_offsets[i] + (len + kRowAlign - 1) / kRowAlign * kRowAlign;
  }
  s->n_pad_vecs = s->h_pad_offsets[n_sets];
  if (s->n_pad_vecs >= (int64_t)1 << 31) { gem_store_destroy(s); return fail(GEM_ERR_INVALID, "too many vectors"); }
  const int64_t V = s->n_vecs;
  const int64_t VP = s->n_pad_vecs;

  gem_status r;
  if ((r = dmalloc(&s->d_offsets, n_sets + 1, "offsets")) != GEM_OK) { gem_store_destroy(s); return r; }
  if ((r = dmalloc(&s->d_pad_offsets, n_sets + 1, "padded offsets")) != GEM_OK) { gem_store_destroy(s); return r; }
  std::vector<uint32_t> end_bits((size_t)(VP / kRowAlign / 32 + 2), 0u);
  for (int64_t i = 0; i < n_sets; ++i) {
    const int64_t b = s->h_pad_offsets[i + 1] / kRowAlign - 1;
    end_bits[(size_t)(b >> 5)] |= 1u << (b & 31);
  }
  if ((r = dmalloc(&s->d_end_bits, (int64_t)end_bits.size(), "set-end bitmap")) != GEM_OK) {
    gem_store_destroy(s);
    return r;
  }
  cudaError_t e = cudaMemcpyAsync(s->d_offsets, s->h_offsets.data(), sizeof(int64_t) * (n_sets + 1),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_pad_offsets, s->h_pad_offsets.data(), sizeof(int64_t) * (n_sets + 1),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_end_bits, end_bits.data(), sizeof(uint32_t) * end_bits.size(), cudaMemcpyHostToDevice,
                        st);
  // the FP32 source of the quantised copies lives on the device during the build
  float* src = nullptr;
  float* tmp = nullptr;
  if (e == cudaSuccess) {
    if (keep_mask & GEM_KEEP_F32) {
      if ((r = dmalloc(&s->d_f32, V * kDim, "f32 copy")) != GEM_OK) { gem_store_destroy(s); return r; }
      src = s->d_f32;
    } else if (inputs_on_host) {
      if ((r = dmalloc(&tmp, V * kDim, "staging copy")) != GEM_OK) { gem_store_destroy(s); return r; }
      src = tmp;
    } else {
      src = const_cast<float*>(vecs);
    }
    if (src != vecs)
      e = cudaMemcpyAsync(src, vecs, sizeof(float) * V * kDim,
                          inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess && (keep_mask & GEM_KEEP_BF16)) {
    if ((r = dmalloc(&s->d_bf16, VP * kDim, "bf16 copy")) != GEM_OK) { dfree(tmp); gem_store_destroy(s); return r; }
    launch_quantize_bf16(src, s->d_offsets, s->d_pad_offsets, n_sets, s->d_bf16, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (keep_mask & GEM_KEEP_FP8)) {
    if ((r = dmalloc(&s->d_fp8, VP * kDim, "fp8 copy")) != GEM_OK) { dfree(tmp); gem_store_destroy(s); return r; }
    // scales padded so that 1-D TMA boxes past the last vector stay in bounds
    if ((r = dmalloc(&s->d_fp8_scale, VP + 1024, "fp8 scales")) != GEM_OK) { dfree(tmp); gem_store_destroy(s); return r; }
    e = cudaMemsetAsync(s->d_fp8_scale, 0, sizeof(float) * (VP + 1024), st);
    if (e == cudaSuccess) {
      launch_quantize_fp8(src, s->d_offsets, s->d_pad_offsets, n_sets, s->d_fp8, s->d_fp8_scale, st);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && (keep_mask & GEM_KEEP_FP8_SET)) {
    if ((r = dmalloc(&s->d_fp8s, VP * kDim, "per-set fp8 copy")) != GEM_OK) { dfree(tmp); gem_store_destroy(s); return r; }
    if ((r = dmalloc(&s->d_set_scale, n_sets, "set scales")) != GEM_OK) { dfree(tmp); gem_store_destroy(s); return r; }
    launch_quantize_fp8_set(src, s->d_offsets, s->d_pad_offsets, n_sets, s->d_fp8s, s->d_set_scale, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(tmp);
  if (e != cudaSuccess) { gem_store_destroy(s); return cuda_fail(e, "building the store"); }
  *out = s;
  return GEM_OK;
}

gem_status gem_store_info(const gem_store* s, int64_t* n_sets, int64_t* n_vecs, int64_t* n_pad_vecs,
                          uint32_t* keep_mask) {
  if (!s) return fail(GEM_ERR_INVALID, "store is NULL");
  if (n_sets) *n_sets = s->n_sets;
  if (n_vecs) *n_vecs = s->n_vecs;
  if (n_pad_vecs) *n_pad_vecs = s->n_pad_vecs;
  if (keep_mask) *keep_mask = s->keep;
  return GEM_OK;
}

gem_status gem_store_export(const gem_store* s, int32_t what, void* dst, size_t dst_bytes, void* stream) {
  if (!s || !dst) return fail(GEM_ERR_INVALID, "store or dst is NULL");
  const void* src = nullptr;
  size_t bytes = 0;
  switch (what) {
    case GEM_EXPORT_BF16: src = s->d_bf16; bytes = sizeof(uint16_t) * s->n_pad_vecs * kDim; break;
    case GEM_EXPORT_FP8: src = s->d_fp8; bytes = (size_t)s->n_pad_vecs * kDim; break;
    case GEM_EXPORT_FP8_SCALE: src = s->d_fp8_scale; bytes = sizeof(float) * s->n_pad_vecs; break;
    case GEM_EXPORT_OFFSETS: src = s->d_offsets; bytes = sizeof(int64_t) * (s->n_sets + 1); break;
    case GEM_EXPORT_PAD_OFFSETS: src = s->d_pad_offsets; bytes = sizeof(int64_t) * (s->n_sets + 1); break;
    case GEM_EXPORT_CODES: src = s->d_codes; bytes = sizeof(int32_t) * s->n_vecs; break;
    case GEM_EXPORT_CODEBOOK: src = s->d_codebook; bytes = sizeof(float) * (size_t)s->k1 * kDim; break;
    case GEM_EXPORT_INDEX_CODES: src = s->d_icodes; bytes = sizeof(int32_t) * s->n_vecs; break;
    case GEM_EXPORT_F32: src = s->d_f32; bytes = sizeof(float) * s->n_vecs * kDim; break;
    case GEM_EXPORT_INDEX_CENTROIDS: src = s->d_cindex; bytes = sizeof(float) * (size_t)s->k2 * kDim; break;
    case GEM_EXPORT_FP8_SET: src = s->d_fp8s; bytes = (size_t)s->n_pad_vecs * kDim; break;
    case GEM_EXPORT_SET_SCALE: src = s->d_set_scale; bytes = sizeof(float) * s->n_sets; break;
    case GEM_EXPORT_DELETED: {
      bytes = sizeof(uint32_t) * (size_t)((s->n_sets + 31) / 32);
      if (dst_bytes < bytes) return fail(GEM_ERR_INVALID, "dst too small");
      cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
      if (s->d_dead) GEM_CUDA_TRY(cudaMemcpyAsync(dst, s->d_dead, bytes, cudaMemcpyDeviceToDevice, st));
      else GEM_CUDA_TRY(cudaMemsetAsync(dst, 0, bytes, st));
      return GEM_OK;
    }
    default: return fail(GEM_ERR_INVALID, "unknown export");
  }
  if (!src) return fail(GEM_ERR_STATE, "store does not keep that array");
  if (dst_bytes < bytes) return fail(GEM_ERR_INVALID, "dst too small");
  GEM_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
  return GEM_OK;
}

// ----------------------------------------------------------------------------- workspace

void gem_workspace_destroy(gem_workspace* w) {
  if (!w) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(w->device);
  void* ptrs[] = {w->d_status, w->d_unit_counter, w->d_plan_hdr, w->d_part_query, w->d_part_rows, w->d_part_g,
                  w->d_part_pass, w->d_part_slot, w->d_part_row0, w->d_row_part, w->d_qpack_bf16,
                  w->d_qpack_fp8, w->d_qpack_scale, w->d_scores, w->d_pool_ids, w->d_pool_off,
                  w->d_pool_scores, w->d_q_in, w->d_qo_in, w->d_out_ids, w->d_out_scores,
                  w->d_qcodes, w->d_assign_key, w->d_tables, w->d_topk_thr, w->d_topk_cnt, w->d_topk_cand,
                  w->d_pool_perm, w->d_pool_bucket};
  for (void* p : ptrs) dfree(p);
  cudaSetDevice(prev);
  delete w;
}

gem_status gem_workspace_create(const gem_store* s, int32_t max_queries, int64_t max_q_rows,
                                int32_t max_q_len, int64_t max_cands, int32_t max_k,
                                gem_workspace** out) {
  GEM_NVTX_RANGE("gem_workspace_create");
  if (!out) return fail(GEM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!s) return fail(GEM_ERR_INVALID, "store is NULL");
  if (max_queries < 1 || max_queries > (1 << 20)) return fail(GEM_ERR_INVALID, "max_queries out of range");
  if (max_q_rows < 1 || max_q_rows > ((int64_t)1 << 28)) return fail(GEM_ERR_INVALID, "max_q_rows out of range");
  if (max_q_len < 1 || max_q_len > 32 * kMaxPasses) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  if (max_cands < 0) return fail(GEM_ERR_INVALID, "max_cands < 0");
  if (max_k < 0 || max_k > kMaxK) return fail(GEM_ERR_INVALID, "max_k must be 0..4096");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;

  gem_workspace* w = new gem_workspace();
  w->store = s;
  w->device = s->device;
  w->max_queries = max_queries;
  w->max_q_rows = max_q_rows;
  w->max_q_len = max_q_len;
  w->max_cands = max_cands;
  w->max_k = max_k;
  w->n_passes = (max_q_len + 31) / 32;
  // every part of r rows takes a slot of g < 2r rows; each pass is padded to a
  // whole query block of at most 512 rows
  w->packed_cap = ((2 * max_q_rows + 512 * (kMaxPasses + 1)) + 511) / 512 * 512;
  w->max_parts = std::min<int64_t>(max_q_rows, (int64_t)max_queries * kMaxPasses);
#define WS_ALLOC(ptr, count)                                                 \
  if ((r = dmalloc(&w->ptr, (size_t)(count), #ptr)) != GEM_OK) {            \
    gem_workspace_destroy(w);                                               \
    return r;                                                               \
  }
  WS_ALLOC(d_status, 1);
  WS_ALLOC(d_unit_counter, 2);
  WS_ALLOC(d_plan_hdr, kPlanHdrInts);
  WS_ALLOC(d_part_query, w->max_parts);
  WS_ALLOC(d_part_rows, w->max_parts);
  WS_ALLOC(d_part_g, w->max_parts);
  WS_ALLOC(d_part_pass, w->max_parts);
  WS_ALLOC(d_part_slot, w->max_parts);
  WS_ALLOC(d_part_row0, w->max_parts);
  WS_ALLOC(d_row_part, w->packed_cap);
  if (s->d_bf16) WS_ALLOC(d_qpack_bf16, w->packed_cap * kDim);
  if (s->d_fp8 || s->d_fp8s) {
    WS_ALLOC(d_qpack_fp8, w->packed_cap * kDim);
    WS_ALLOC(d_qpack_scale, w->packed_cap);
  }
  if (max_k > 0) {
    WS_ALLOC(d_scores, (size_t)max_queries * s->n_sets);
    WS_ALLOC(d_pool_off, max_queries + 1);
    WS_ALLOC(d_q_in, max_q_rows * kDim);
    WS_ALLOC(d_qo_in, max_queries + 1);
    WS_ALLOC(d_out_ids, (size_t)max_queries * max_k);
    WS_ALLOC(d_out_scores, (size_t)max_queries * max_k);
    // candidate buffers of the threshold top-k: at most 512 MB, whole rows
    w->topk_cap = topk_candidate_cap(max_k);
    const int64_t row_bytes = (int64_t)w->topk_cap * 8;
    w->topk_rows = (int)std::max<int64_t>(1, std::min<int64_t>(max_queries, ((int64_t)512 << 20) / row_bytes));
    WS_ALLOC(d_topk_thr, w->topk_rows);
    WS_ALLOC(d_topk_cnt, w->topk_rows);
    WS_ALLOC(d_topk_cand, (size_t)w->topk_rows * w->topk_cap);
  }
  if (max_cands > 0) {
    WS_ALLOC(d_pool_ids, max_cands);
    WS_ALLOC(d_pool_scores, max_cands);
    if (max_cands < INT32_MAX) {
      WS_ALLOC(d_pool_perm, max_cands);
      WS_ALLOC(d_pool_bucket, kPoolKeys);
    }
  }
  if (s->k1 > 0) {
    // tables of up to 16 query parts (8 MB each at k1 = 65536)
    const int max_np = (max_q_len + 31) / 32;
    w->table_parts = std::max(max_np, std::min(16, max_queries * max_np));
    WS_ALLOC(d_qcodes, max_q_rows);
    WS_ALLOC(d_assign_key, max_q_rows);
    WS_ALLOC(d_tables, (size_t)w->table_parts * s->k1 * 32);
  }
#undef WS_ALLOC
  cudaError_t e = cudaMemset(w->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w->d_plan_hdr, 0, sizeof(int) * kPlanHdrInts);
  if (e != cudaSuccess) { gem_workspace_destroy(w); return cuda_fail(e, "workspace init"); }
  if (w->d_qpack_bf16 &&
      !encode_tmap_2d(&w->tmap_q_bf16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w->d_qpack_bf16, kDim,
                      w->packed_cap, kDim * 2, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B)) {
    gem_workspace_destroy(w);
    return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the packed queries");
  }
  if (w->d_qpack_fp8 &&
      !encode_tmap_2d(&w->tmap_q_fp8, CU_TENSOR_MAP_DATA_TYPE_UINT8, w->d_qpack_fp8, kDim,
                      w->packed_cap, kDim, 128, 128, CU_TENSOR_MAP_SWIZZLE_128B)) {
    gem_workspace_destroy(w);
    return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the packed fp8 queries");
  }
  *out = w;
  return GEM_OK;
}

gem_status gem_assign_codes(const float* x, int64_t n, const float* centroids, int32_t k1,
                            int32_t* codes, float* best, void* stream) {
  GEM_NVTX_RANGE("gem_assign_codes");
  if (!x || !centroids || !codes) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n < 0 || k1 < 1) return fail(GEM_ERR_INVALID, "bad sizes");
  return launch_assign(x, n, centroids, k1, codes, best, reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_train_codebook(const gem_store* s, int32_t k1, int32_t iters, int64_t sample,
                              uint64_t seed, float* centroids_out, void* stream) {
  GEM_NVTX_RANGE("gem_train_codebook");
  if (!s || !centroids_out) return fail(GEM_ERR_INVALID, "NULL argument");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "training reads the fp32 copy");
  if (iters < 0) return fail(GEM_ERR_INVALID, "iters < 0");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  const int64_t n = (sample <= 0 || sample >= s->n_vecs) ? s->n_vecs : sample;
  if (k1 < 1 || k1 > n) return fail(GEM_ERR_INVALID, "k1 must be 1..sample size");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // sample rows (without replacement) and the initial centroids: a seeded
  // shuffle of the sample; both are host-side index choices only
  std::mt19937_64 rng(seed);
  std::vector<int64_t> rows;
  if (n == s->n_vecs) {
    rows.resize(n);
    std::iota(rows.begin(), rows.end(), 0);
  } else {
    std::vector<int64_t> all(s->n_vecs);
    std::iota(all.begin(), all.end(), 0);
    for (int64_t i = 0; i < n; ++i) {
      std::uniform_int_distribution<int64_t> pick(i, s->n_vecs - 1);
      std::swap(all[i], all[pick(rng)]);
    }
    rows.assign(all.begin(), all.begin() + n);
  }
  std::vector<int64_t> init(rows.begin(), rows.end());
  for (int64_t i = 0; i < k1; ++i) {
    std::uniform_int_distribution<int64_t> pick(i, n - 1);
    std::swap(init[i], init[pick(rng)]);
  }
  init.resize(k1);
  float* X = nullptr;
  int64_t* d_rows = nullptr;
  int32_t* codes = nullptr;
  double* sums = nullptr;
  int* counts = nullptr;
  auto cleanup = [&]() { dfree(X); dfree(d_rows); dfree(codes); dfree(sums); dfree(counts); };
  if ((r = dmalloc(&X, (size_t)n * kDim, "sample")) != GEM_OK ||
      (r = dmalloc(&d_rows, (size_t)std::max<int64_t>(n, k1), "sample rows")) != GEM_OK ||
      (r = dmalloc(&codes, (size_t)n, "sample codes")) != GEM_OK ||
      (r = dmalloc(&sums, (size_t)k1 * kDim, "centroid sums")) != GEM_OK ||
      (r = dmalloc(&counts, (size_t)k1, "centroid counts")) != GEM_OK) {
    cleanup();
    return r;
  }
  cudaError_t e = cudaMemcpyAsync(d_rows, init.data(), sizeof(int64_t) * k1, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) r = launch_gather_rows(s->d_f32, d_rows, k1, centroids_out, st);
  if (e == cudaSuccess && r == GEM_OK)
    e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && r == GEM_OK) r = launch_gather_rows(s->d_f32, d_rows, n, X, st);
  for (int it = 0; it < iters && e == cudaSuccess && r == GEM_OK; ++it) {
    r = launch_assign(X, n, centroids_out, k1, codes, nullptr, st);
    if (r == GEM_OK) r = launch_kmeans_step(X, n, codes, sums, counts, k1, centroids_out, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "codebook training");
  return r;
}

static int current_sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

gem_status gem_kmeans(const float* x, int64_t n, int32_t k, int32_t iters, uint64_t seed, float* centroids_out,
                      void* stream) {
  GEM_NVTX_RANGE("gem_kmeans");
  if (!x || !centroids_out) return fail(GEM_ERR_INVALID, "NULL argument");
  if (k < 1 || k > n) return fail(GEM_ERR_INVALID, "k must be 1..n");
  if (iters < 0) return fail(GEM_ERR_INVALID, "iters < 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // initial centroids: k distinct rows of x from a seeded shuffle (a host-side
  // index choice only)
  std::mt19937_64 rng(seed);
  std::vector<int64_t> init(n);
  std::iota(init.begin(), init.end(), 0);
  for (int64_t i = 0; i < k; ++i) {
    std::uniform_int_distribution<int64_t> pick(i, n - 1);
    std::swap(init[i], init[pick(rng)]);
  }
  init.resize(k);
  int64_t* d_rows = nullptr;
  int32_t* codes = nullptr;
  double* sums = nullptr;
  int* counts = nullptr;
  auto cleanup = [&]() { dfree(d_rows); dfree(codes); dfree(sums); dfree(counts); };
  gem_status r;
  if ((r = dmalloc(&d_rows, (size_t)k, "initial rows")) != GEM_OK || (r = dmalloc(&codes, (size_t)n, "codes")) != GEM_OK ||
      (r = dmalloc(&sums, (size_t)k * kDim, "centroid sums")) != GEM_OK ||
      (r = dmalloc(&counts, (size_t)k, "centroid counts")) != GEM_OK) {
    cleanup();
    return r;
  }
  cudaError_t e = cudaMemcpyAsync(d_rows, init.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) r = launch_gather_rows(x, d_rows, k, centroids_out, st);
  for (int it = 0; it < iters && e == cudaSuccess && r == GEM_OK; ++it) {
    r = launch_assign(x, n, centroids_out, k, codes, nullptr, st);
    if (r == GEM_OK) r = launch_kmeans_step(x, n, codes, sums, counts, k, centroids_out, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "k-means");
  return r;
}

gem_status gem_cluster_filter(const float* q, const int64_t* q_offsets, int32_t n_queries, int32_t max_q_len,
                              const float* centroids, int32_t k2, int32_t t, uint32_t* out_mask, int32_t* out_list,
                              int32_t* out_count, void* stream) {
  GEM_NVTX_RANGE("gem_cluster_filter");
  if (!q || !q_offsets || !centroids || !out_mask || !out_list || !out_count)
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_queries < 0 || max_q_len < 1) return fail(GEM_ERR_INVALID, "bad sizes");
  if (k2 < 1 || k2 > (1 << 18)) return fail(GEM_ERR_INVALID, "k2 must be 1..262144");
  if (t < 1 || t > 8 || t > k2) return fail(GEM_ERR_INVALID, "t must be 1..min(8, k2)");
  return launch_cluster_filter(q, q_offsets, n_queries, centroids, k2, t, max_q_len * t, out_mask, out_list,
                               out_count, current_sm_count(), reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_store_set_index_centroids(gem_store* s, const float* centroids, int32_t k2, void* stream) {
  if (!s || !centroids) return fail(GEM_ERR_INVALID, "NULL argument");
  if (k2 < 1 || k2 > (1 << 18)) return fail(GEM_ERR_INVALID, "k2 must be 1..262144");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "cluster codes are assigned from the fp32 copy");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dfree(s->d_cindex);
  dfree(s->d_member_off);
  s->d_cindex = nullptr;
  s->d_member_off = nullptr;
  s->k2 = 0;
  if (!s->d_icodes && (r = dmalloc(&s->d_icodes, (size_t)s->n_vecs, "index codes")) != GEM_OK) return r;
  if (!s->d_members && (r = dmalloc(&s->d_members, (size_t)s->n_vecs, "cluster members")) != GEM_OK) return r;
  if ((r = dmalloc(&s->d_cindex, (size_t)k2 * kDim, "C_index")) != GEM_OK) return r;
  if ((r = dmalloc(&s->d_member_off, (size_t)k2 + 1, "member offsets")) != GEM_OK) return r;
  GEM_CUDA_TRY(cudaMemcpyAsync(s->d_cindex, centroids, sizeof(float) * (size_t)k2 * kDim, cudaMemcpyDeviceToDevice,
                               st));
  if ((r = launch_assign(s->d_f32, s->n_vecs, s->d_cindex, k2, s->d_icodes, nullptr, st)) != GEM_OK) return r;
  s->k2 = k2;
  return launch_cluster_index(s, st);
}

gem_status gem_store_mark_deleted(gem_store* s, const int64_t* ids, int64_t n, int32_t deleted, void* stream) {
  if (!s || (n > 0 && !ids)) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n < 0) return fail(GEM_ERR_INVALID, "n < 0");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  r = launch_mark_deleted(s, ids, n, deleted != 0, reinterpret_cast<cudaStream_t>(stream));
  if (r == GEM_ERR_INVALID) return fail(r, "set id out of range");
  return r;
}

gem_status gem_entry_points(const gem_store* s, const int32_t* cluster_lists, const int32_t* cluster_counts,
                            int32_t n_queries, int32_t stride, uint64_t seed, int64_t* out_sets, void* stream) {
  GEM_NVTX_RANGE("gem_entry_points");
  if (!s || !cluster_lists || !cluster_counts || !out_sets) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_queries < 0 || stride < 1) return fail(GEM_ERR_INVALID, "bad sizes");
  if (s->k2 <= 0) return fail(GEM_ERR_STATE, "store has no C_index (gem_store_set_index_centroids)");
  return launch_entry_points(s, cluster_lists, cluster_counts, n_queries, stride, seed, out_sets,
                             reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_store_set_codebook(gem_store* s, const float* centroids, int32_t k1, void* stream) {
  if (!s || !centroids) return fail(GEM_ERR_INVALID, "NULL argument");
  if (k1 < 1) return fail(GEM_ERR_INVALID, "k1 < 1");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "codes are assigned from the fp32 copy");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dfree(s->d_codebook);
  s->d_codebook = nullptr;
  s->k1 = 0;
  if (!s->d_codes && (r = dmalloc(&s->d_codes, (size_t)s->n_vecs, "codes")) != GEM_OK) return r;
  if ((r = dmalloc(&s->d_codebook, (size_t)k1 * kDim, "codebook")) != GEM_OK) return r;
  GEM_CUDA_TRY(cudaMemcpyAsync(s->d_codebook, centroids, sizeof(float) * (size_t)k1 * kDim,
                               cudaMemcpyDeviceToDevice, st));
  if ((r = launch_assign(s->d_f32, s->n_vecs, s->d_codebook, k1, s->d_codes, nullptr, st)) != GEM_OK) return r;
  GEM_CUDA_TRY(cudaStreamSynchronize(st));
  s->k1 = k1;
  return GEM_OK;
}

gem_status gem_workspace_set_similarity(gem_workspace* w, int32_t sim) {
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  if (sim != GEM_SIM_IP && sim != GEM_SIM_L2) return fail(GEM_ERR_INVALID, "unknown similarity");
  w->sim = sim;
  return GEM_OK;
}

gem_status gem_workspace_set_qch_form(gem_workspace* w, int32_t form) {
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  if (form != GEM_QCH_SYMMETRIC && form != GEM_QCH_ASYMMETRIC) return fail(GEM_ERR_INVALID, "unknown qCH form");
  w->qch_form = form;
  return GEM_OK;
}

gem_status gem_workspace_set_schedule(gem_workspace* w, int32_t m_tiles, int32_t variant, int32_t chunk_rows) {
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  if (m_tiles != 1 && m_tiles != 2 && m_tiles != 4) return fail(GEM_ERR_INVALID, "m_tiles must be 1, 2 or 4");
  if (variant < GEM_TC_PLAIN || variant > GEM_TC_TWO_SETS) return fail(GEM_ERR_INVALID, "unknown variant");
  if (variant == GEM_TC_A_TMEM && m_tiles != 2) return fail(GEM_ERR_INVALID, "a_tmem needs m_tiles = 2");
  if (variant == GEM_TC_TWO_SETS && m_tiles == 4) return fail(GEM_ERR_INVALID, "two_sets needs m_tiles 1 or 2");
  if (chunk_rows < 1024 || chunk_rows > (1 << 24)) return fail(GEM_ERR_INVALID, "chunk_rows out of range");
  w->tc_m_tiles = m_tiles;
  w->tc_variant = variant;
  w->tc_chunk_rows = chunk_rows;
  return GEM_OK;
}

// ----------------------------------------------------------------------------- scoring

}  // extern "C"

gem_status gem::check_query_args(const gem_store* s, gem_workspace* w, const float* q,
                                   const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows) {
  if (!s || !w) return fail(GEM_ERR_INVALID, "store or workspace is NULL");
  if (w->store != s) return fail(GEM_ERR_INVALID, "workspace was created for another store");
  if (!q || !q_offsets) return fail(GEM_ERR_INVALID, "q or q_offsets is NULL");
  if (n_queries < 1 || n_queries > w->max_queries) return fail(GEM_ERR_INVALID, "n_queries out of range");
  if (n_q_rows < n_queries || n_q_rows > w->max_q_rows) return fail(GEM_ERR_INVALID, "n_q_rows out of range");
  return check_current_device(s->device);
}

extern "C" {

static gem_status score_all_impl(const gem_store* s, gem_workspace* w, const float* q,
                                 const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                                 int32_t compute, float* scores, cudaStream_t st) {
  if (compute == GEM_F32) {
    if (!s->d_f32) return fail(GEM_ERR_STATE, "store keeps no fp32 copy");
    return launch_f32_score(s, w, q, q_offsets, n_queries, nullptr, nullptr, 0, scores, st);
  }
  if (w->sim == GEM_SIM_L2 && (compute == GEM_BF16 || compute == GEM_FP8_E4M3 || compute == GEM_FP8_E4M3_SET))
    return fail(GEM_ERR_UNSUPPORTED, "Sim = L2 distance is scored by GEM_F32 only");
  if (compute == GEM_BF16) {
    if (!s->d_bf16) return fail(GEM_ERR_STATE, "store keeps no bf16 copy");
    const int mt = w->tc_m_tiles;
    gem_status r = launch_plan(w, q, q_offsets, n_queries, n_q_rows, 128 * mt, compute, st);
    if (r != GEM_OK) return r;
    return launch_tc_score_all(s, w, compute, mt, w->tc_variant, w->tc_chunk_rows, scores, st);
  }
  if (compute == GEM_FP8_E4M3 || compute == GEM_FP8_E4M3_SET) {
    if (compute == GEM_FP8_E4M3 && !s->d_fp8) return fail(GEM_ERR_STATE, "store keeps no fp8 copy");
    if (compute == GEM_FP8_E4M3_SET && !s->d_fp8s) return fail(GEM_ERR_STATE, "store keeps no per-set-scale fp8 copy");
    const int mt = w->tc_m_tiles;
    // the query rows take per-row E4M3 scales in both forms
    gem_status r = launch_plan(w, q, q_offsets, n_queries, n_q_rows, 128 * mt, GEM_FP8_E4M3, st);
    if (r != GEM_OK) return r;
    return launch_tc_score_all(s, w, compute, mt, w->tc_variant, w->tc_chunk_rows, scores, st);
  }
  return fail(GEM_ERR_INVALID, "unknown compute dtype");
}

gem_status gem_score_all(const gem_store* s, gem_workspace* w, const float* q,
                         const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                         int32_t compute, float* scores, void* stream) {
  GEM_NVTX_RANGE("gem_score_all");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!scores) return fail(GEM_ERR_INVALID, "scores is NULL");
  return score_all_impl(s, w, q, q_offsets, n_queries, n_q_rows, compute, scores,
                        reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_score_ids(const gem_store* s, gem_workspace* w, const float* q,
                         const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                         const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                         int32_t compute, float* scores, void* stream) {
  GEM_NVTX_RANGE("gem_score_ids");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!cand_offsets || (n_cands > 0 && (!cand_ids || !scores)))
    return fail(GEM_ERR_INVALID, "candidate arrays or scores is NULL");
  if (n_cands < 0) return fail(GEM_ERR_INVALID, "n_cands < 0");
  if (n_cands == 0) return GEM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (compute == GEM_F32) {
    if (!s->d_f32) return fail(GEM_ERR_STATE, "store keeps no fp32 copy");
    return launch_f32_score(s, w, q, q_offsets, n_queries, cand_offsets, cand_ids, n_cands, scores, st);
  }
  if (compute == GEM_CODES) {
    if (w->sim == GEM_SIM_L2) return fail(GEM_ERR_UNSUPPORTED, "qCH is defined for the inner-product Sim");
    if (!s->d_f32 || s->k1 == 0 || !w->d_qcodes)
      return fail(GEM_ERR_STATE, "the codes form needs a codebook before the workspace is created");
    if (w->qch_form == GEM_QCH_ASYMMETRIC)
      return launch_f32_score(s, w, q, q_offsets, n_queries, cand_offsets, cand_ids, n_cands, scores, st, nullptr,
                              true);
    r = launch_assign_split(q, n_q_rows, s->d_codebook, s->k1, w->d_qcodes, w->d_assign_key, s->n_sm, st);
    if (r != GEM_OK) return r;
    return launch_f32_score(s, w, q, q_offsets, n_queries, cand_offsets, cand_ids, n_cands, scores, st,
                            w->d_qcodes);
  }
  if (compute == GEM_BF16 || compute == GEM_FP8_E4M3 || compute == GEM_FP8_E4M3_SET)
    return fail(GEM_ERR_UNSUPPORTED, "id-list scoring runs in GEM_F32 or GEM_CODES");
  return fail(GEM_ERR_INVALID, "unknown compute dtype");
}

gem_status gem_rerank_pool(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                           int32_t n_queries, int64_t n_q_rows, const int64_t* pool_ids, int32_t depth,
                           float* pool_scores, void* stream) {
  GEM_NVTX_RANGE("gem_rerank_pool");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!pool_ids || !pool_scores) return fail(GEM_ERR_INVALID, "pool_ids or pool_scores is NULL");
  if (!w->d_pool_off) return fail(GEM_ERR_STATE, "workspace was created with max_k or max_cands 0");
  if (depth < 1 || (int64_t)depth * n_queries > w->max_cands)
    return fail(GEM_ERR_INVALID, "n_queries * depth must be 1..max_cands");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "the rerank needs the fp32 copy");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch_iota_offsets(w->d_pool_off, n_queries, depth, st);
  GEM_CUDA_TRY(cudaGetLastError());
  return launch_f32_score_pool(s, w, q, q_offsets, n_queries, depth, pool_ids, pool_scores, st);
}

gem_status gem_beam_search(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                           int32_t n_queries, int64_t n_q_rows, const int64_t* graph_off, const int32_t* graph_nbrs,
                           int32_t max_degree, const uint32_t* cluster_mask, const int64_t* entries,
                           int32_t entry_stride, int32_t ef, int32_t max_rounds, int64_t* out_ids, float* out_scores,
                           int32_t* out_rounds, void* stream) {
  GEM_NVTX_RANGE("gem_beam_search");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!graph_off || !graph_nbrs || !cluster_mask || !entries || !out_ids || !out_scores)
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (ef < 1 || ef > 4096) return fail(GEM_ERR_INVALID, "ef must be 1..4096");
  if (entry_stride < 1 || max_degree < 1 || max_rounds < 0) return fail(GEM_ERR_INVALID, "bad sizes");
  if (s->k1 == 0 || !w->d_qcodes)
    return fail(GEM_ERR_STATE, "the search scores by qCH: a codebook is needed before the workspace is created");
  if (s->k2 == 0) return fail(GEM_ERR_STATE, "the cluster test needs C_index (gem_store_set_index_centroids)");
  if (w->sim == GEM_SIM_L2) return fail(GEM_ERR_UNSUPPORTED, "qCH is defined for the inner-product Sim");
  if ((int64_t)n_queries * ((w->max_q_len + 31) / 32) > 65535)
    return fail(GEM_ERR_INVALID, "more than 65,535 query parts of 32 rows in one search");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (w->qch_form == GEM_QCH_SYMMETRIC) {
    r = launch_assign_split(q, n_q_rows, s->d_codebook, s->k1, w->d_qcodes, w->d_assign_key, s->n_sm, st);
    if (r != GEM_OK) return r;
  }
  return beam_search(s, w, q, q_offsets, n_queries, graph_off, graph_nbrs, max_degree, cluster_mask, entries,
                     entry_stride, ef, max_rounds, out_ids, out_scores, out_rounds, st);
}

gem_status gem_estimate_codes(const gem_store* s, gem_workspace* w, const float* q,
                              const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                              const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                              float* est, void* stream) {
  GEM_NVTX_RANGE("gem_estimate_codes");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!est) return fail(GEM_ERR_INVALID, "est is NULL");
  if (w->sim == GEM_SIM_L2) return fail(GEM_ERR_UNSUPPORTED, "qCH is defined for the inner-product Sim");
  if (s->k1 == 0 || !w->d_tables)
    return fail(GEM_ERR_STATE, "store had no codebook when the workspace was created");
  if (cand_offsets && n_cands > 0 && !cand_ids) return fail(GEM_ERR_INVALID, "cand_ids is NULL");
  if (cand_offsets && n_cands == 0) return GEM_OK;
  return launch_qch(s, w, q, q_offsets, n_queries, n_q_rows, cand_offsets, cand_ids, est,
                    reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_topk(gem_workspace* w, const float* scores, const int64_t* row_offsets, int32_t rows,
                    int64_t cols, const int64_t* ids, int32_t k, int64_t* out_ids, float* out_scores,
                    void* stream) {
  GEM_NVTX_RANGE("gem_topk");
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  if (!scores || !out_ids) return fail(GEM_ERR_INVALID, "scores or out_ids is NULL");
  if (rows < 0 || (!row_offsets && cols < 0)) return fail(GEM_ERR_INVALID, "bad shape");
  if (k < 1 || k > kMaxK) return fail(GEM_ERR_INVALID, "k must be 1..4096");
  gem_status r = check_current_device(w->device);
  if (r != GEM_OK) return r;
  return launch_topk(w, scores, row_offsets, rows, cols, ids, k, out_ids, out_scores,
                     reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

gem_status gem::search_first_pass(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                             int32_t n_queries, int64_t n_q_rows, int32_t compute, cudaStream_t st) {
  if (compute == GEM_CODES) {
    // first pass by the quantized estimate (Algorithm 5 scores by qCH and
    // reranks by exact CH): qsim of every stored set in the workspace's form
    if (w->sim == GEM_SIM_L2) return fail(GEM_ERR_UNSUPPORTED, "qCH is defined for the inner-product Sim");
    if (s->k1 == 0 || !w->d_tables)
      return fail(GEM_ERR_STATE, "the codes pass needs a codebook before the workspace is created");
    return launch_qch(s, w, q, q_offsets, n_queries, n_q_rows, nullptr, nullptr, w->d_scores, st);
  }
  return score_all_impl(s, w, q, q_offsets, n_queries, n_q_rows, compute, w->d_scores, st);
}

extern "C" {

static gem_status search_impl(const gem_store* s, gem_workspace* w, const float* q,
                              const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                              int32_t compute, int32_t rerank_depth, int32_t k, int64_t* out_ids,
                              float* out_scores, cudaStream_t st) {
  if (k < 1 || k > w->max_k) return fail(GEM_ERR_INVALID, "k must be 1..max_k");
  if (rerank_depth < 0 || rerank_depth > kMaxK) return fail(GEM_ERR_INVALID, "rerank_depth must be 0..4096");
  if (rerank_depth > 0 && rerank_depth < k) return fail(GEM_ERR_INVALID, "rerank_depth < k");
  if (rerank_depth > 0 && (int64_t)rerank_depth * n_queries > w->max_cands)
    return fail(GEM_ERR_INVALID, "n_queries * rerank_depth exceeds max_cands");
  if (rerank_depth > 0 && !s->d_f32) return fail(GEM_ERR_STATE, "the rerank needs the fp32 copy");
  gem_status r;
  {
    GEM_NVTX_RANGE("search: first pass");
    r = search_first_pass(s, w, q, q_offsets, n_queries, n_q_rows, compute, st);
  }
  if (r != GEM_OK) return r;
  if (rerank_depth == 0)
    return launch_topk(w, w->d_scores, nullptr, n_queries, s->n_sets, nullptr, k, out_ids, out_scores, st);
  {
    GEM_NVTX_RANGE("search: top-R");
    r = launch_topk(w, w->d_scores, nullptr, n_queries, s->n_sets, nullptr, rerank_depth, w->d_pool_ids,
                    nullptr, st);
  }
  if (r != GEM_OK) return r;
  launch_iota_offsets(w->d_pool_off, n_queries, rerank_depth, st);
  GEM_CUDA_TRY(cudaGetLastError());
  {
    GEM_NVTX_RANGE("search: FP32 rerank");
    r = launch_f32_score_pool(s, w, q, q_offsets, n_queries, rerank_depth, w->d_pool_ids, w->d_pool_scores, st);
  }
  if (r != GEM_OK) return r;
  GEM_NVTX_RANGE("search: top-k");
  return launch_topk(w, w->d_pool_scores, nullptr, n_queries, rerank_depth, w->d_pool_ids, k, out_ids,
                     out_scores, st);
}

gem_status gem_search(const gem_store* s, gem_workspace* w, const float* q,
                      const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                      int32_t compute, int32_t rerank_depth, int32_t k, int64_t* out_ids,
                      float* out_scores, void* stream) {
  GEM_NVTX_RANGE("gem_search");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!out_ids) return fail(GEM_ERR_INVALID, "out_ids is NULL");
  if (!w->d_scores) return fail(GEM_ERR_STATE, "workspace was created with max_k = 0");
  return search_impl(s, w, q, q_offsets, n_queries, n_q_rows, compute, rerank_depth, k, out_ids,
                     out_scores, reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_search_host(const gem_store* s, gem_workspace* w, const float* q_host,
                           const int64_t* q_offsets_host, int32_t n_queries, int32_t compute,
                           int32_t rerank_depth, int32_t k, int64_t* out_ids_host,
                           float* out_scores_host, void* stream) {
  GEM_NVTX_RANGE("gem_search_host");
  if (!s || !w || !q_host || !q_offsets_host || !out_ids_host)
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (!w->d_scores) return fail(GEM_ERR_STATE, "workspace was created with max_k = 0");
  if (n_queries < 1 || n_queries > w->max_queries) return fail(GEM_ERR_INVALID, "n_queries out of range");
  const int64_t n_q_rows = q_offsets_host[n_queries];
  if (q_offsets_host[0] != 0) return fail(GEM_ERR_INVALID, "q_offsets[0] != 0");
  for (int32_t b = 0; b < n_queries; ++b) {
    const int64_t m = q_offsets_host[b + 1] - q_offsets_host[b];
    if (m < 1 || m > w->max_q_len) return fail(GEM_ERR_INVALID, "query set length out of range");
  }
  gem_status r = check_query_args(s, w, w->d_q_in, w->d_qo_in, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (k < 1 || k > w->max_k) return fail(GEM_ERR_INVALID, "k must be 1..max_k");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GEM_CUDA_TRY(cudaMemcpyAsync(w->d_q_in, q_host, sizeof(float) * n_q_rows * kDim, cudaMemcpyHostToDevice, st));
  GEM_CUDA_TRY(cudaMemcpyAsync(w->d_qo_in, q_offsets_host, sizeof(int64_t) * (n_queries + 1),
                               cudaMemcpyHostToDevice, st));
  r = search_impl(s, w, w->d_q_in, w->d_qo_in, n_queries, n_q_rows, compute, rerank_depth, k, w->d_out_ids,
                  w->d_out_scores, st);
  if (r != GEM_OK) return r;
  GEM_CUDA_TRY(cudaMemcpyAsync(out_ids_host, w->d_out_ids, sizeof(int64_t) * n_queries * k,
                               cudaMemcpyDeviceToHost, st));
  if (out_scores_host)
    GEM_CUDA_TRY(cudaMemcpyAsync(out_scores_host, w->d_out_scores, sizeof(float) * n_queries * k,
                                 cudaMemcpyDeviceToHost, st));
  GEM_CUDA_TRY(cudaStreamSynchronize(st));
  return GEM_OK;
}

gem_status gem_maxsim_fwd(const float* q, const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                          const float* docs, const int64_t* doc_offsets, int64_t n_docs, int64_t n_doc_rows,
                          const int64_t* pair_offsets, const int64_t* pair_ids, int64_t n_pairs, int32_t max_q_len,
                          int32_t compute, float* scores, int32_t* argmax, gem_workspace* ws, void* stream) {
  GEM_NVTX_RANGE("gem_maxsim_fwd");
  if (!q || !q_offsets || !docs || !doc_offsets || !pair_offsets || !scores || !argmax || (n_pairs > 0 && !pair_ids))
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_queries < 1 || n_docs < 1 || n_pairs < 0 || n_q_rows < n_queries || n_doc_rows < n_docs)
    return fail(GEM_ERR_INVALID, "bad sizes");
  if (max_q_len < 1 || max_q_len > 256) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  if (compute != GEM_F32 && compute != GEM_BF16) return fail(GEM_ERR_INVALID, "compute must be GEM_F32 or GEM_BF16");
  if (n_pairs == 0) return GEM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (compute == GEM_BF16 && max_q_len <= 128)
    return launch_maxsim_fwd_tc(q, q_offsets, n_queries, n_q_rows, docs, doc_offsets, n_docs, n_doc_rows,
                                pair_offsets, pair_ids, n_pairs, max_q_len, scores, argmax,
                                ws ? ws->d_status : nullptr, current_sm_count(), st);
  return launch_maxsim_fwd(q, q_offsets, n_queries, docs, doc_offsets, n_docs, pair_offsets, pair_ids, max_q_len,
                           compute == GEM_BF16, scores, argmax, ws ? ws->d_status : nullptr, current_sm_count(), st);
}

gem_status gem_maxsim_bwd(const float* q, const int64_t* q_offsets, int32_t n_queries, const float* docs,
                          const int64_t* doc_offsets, int64_t n_docs, int64_t n_doc_rows,
                          const int64_t* pair_offsets, const int64_t* pair_ids, int64_t n_pairs,
                          const int32_t* argmax, int32_t max_q_len, const float* grad_scores, float* grad_q,
                          float* grad_docs, void* stream) {
  GEM_NVTX_RANGE("gem_maxsim_bwd");
  if (!q || !q_offsets || !docs || !doc_offsets || !pair_offsets || !argmax || !grad_scores ||
      (n_pairs > 0 && !pair_ids))
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_queries < 1 || n_docs < 1 || n_pairs < 0 || n_doc_rows < n_docs) return fail(GEM_ERR_INVALID, "bad sizes");
  if (max_q_len < 1 || max_q_len > 256) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  return launch_maxsim_bwd(q, q_offsets, n_queries, docs, doc_offsets, n_docs, n_doc_rows, pair_offsets, pair_ids,
                           n_pairs, argmax, max_q_len, grad_scores, grad_q, grad_docs, current_sm_count(),
                           reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_batch_create(const gem_store* s, int32_t mode, int32_t max_queries, int64_t max_q_rows,
                            int32_t max_q_len, int64_t max_cands, int32_t seg, int32_t ctas_per_sm,
                            float* q, int64_t* q_offsets, int64_t* cand_offsets, int64_t* cand_ids,
                            float* scores, gem_batch** out) {
  GEM_NVTX_RANGE("gem_batch_create");
  if (!out) return fail(GEM_ERR_INVALID, "out is NULL");
  if (!q || !q_offsets || !cand_offsets || (max_cands > 0 && (!cand_ids || !scores)))
    return fail(GEM_ERR_INVALID, "batch buffer is NULL");
  *out = nullptr;
  if (!s) return fail(GEM_ERR_INVALID, "store is NULL");
  if (mode != GEM_F32 && mode != GEM_CODES) return fail(GEM_ERR_INVALID, "mode must be GEM_F32 or GEM_CODES");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "batched scoring reads the fp32 copy");
  if (mode == GEM_CODES && s->k1 == 0) return fail(GEM_ERR_STATE, "GEM_CODES needs a store codebook");
  if (max_queries < 1 || max_q_rows < 1 || max_cands < 0) return fail(GEM_ERR_INVALID, "bad capacity");
  if (max_q_len < 1 || max_q_len > 32 * kMaxPasses) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  if (seg < 1 || seg > 1024) return fail(GEM_ERR_INVALID, "seg must be 1..1024");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  return batch_create(s, mode, max_queries, max_q_rows, max_q_len, max_cands, seg, ctas_per_sm, q, q_offsets,
                      cand_offsets, cand_ids, scores, out);
}

gem_status gem_batch_run(gem_batch* b, int32_t n_queries, int64_t n_q_rows, int64_t n_cands,
                         int32_t use_graph, void* stream) {
  GEM_NVTX_RANGE("gem_batch_run");
  if (!b) return fail(GEM_ERR_INVALID, "batch is NULL");
  if (n_queries < 1 || n_queries > b->max_queries) return fail(GEM_ERR_INVALID, "n_queries out of range");
  if (n_q_rows < n_queries || n_q_rows > b->max_q_rows) return fail(GEM_ERR_INVALID, "n_q_rows out of range");
  if (n_cands < 0 || n_cands > b->max_cands) return fail(GEM_ERR_INVALID, "n_cands out of range");
  gem_status r = check_current_device(b->device);
  if (r != GEM_OK) return r;
  return batch_run(b, n_queries, n_q_rows, n_cands, use_graph, reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_batch_status(gem_batch* b) {
  if (!b) return fail(GEM_ERR_INVALID, "batch is NULL");
  if (b->launched) GEM_CUDA_TRY(cudaEventSynchronize(b->done));
  int code = 0;
  GEM_CUDA_TRY(cudaMemcpy(&code, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  GEM_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
  if (code != 0) set_error("device-side check failed in a batched run");
  return (gem_status)code;
}

void gem_batch_destroy(gem_batch* b) { batch_destroy(b); }

gem_status gem_autotune_score_all(const gem_store* s, gem_workspace* w, const float* q,
                                  const int64_t* q_offsets, int32_t n_queries, int64_t n_q_rows,
                                  int32_t compute, float* scores, const char* cache_path, int32_t* m_tiles,
                                  int32_t* variant, int32_t* chunk_rows, float* ms, int32_t* from_cache,
                                  void* stream) {
  GEM_NVTX_RANGE("gem_autotune_score_all");
  gem_status r = check_query_args(s, w, q, q_offsets, n_queries, n_q_rows);
  if (r != GEM_OK) return r;
  if (!scores || !m_tiles || !variant || !chunk_rows || !ms || !from_cache)
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (compute == GEM_BF16 && !s->d_bf16) return fail(GEM_ERR_STATE, "store keeps no bf16 copy");
  if (compute == GEM_FP8_E4M3 && !s->d_fp8) return fail(GEM_ERR_STATE, "store keeps no fp8 copy");
  if (compute == GEM_FP8_E4M3_SET && !s->d_fp8s) return fail(GEM_ERR_STATE, "store keeps no per-set-scale fp8 copy");
  if (compute != GEM_BF16 && compute != GEM_FP8_E4M3 && compute != GEM_FP8_E4M3_SET)
    return fail(GEM_ERR_INVALID, "compute must be bf16 or fp8");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  r = autotune_score_all(s, w, q, q_offsets, n_queries, n_q_rows, compute, scores, cache_path, m_tiles, variant,
                         chunk_rows, ms, from_cache, st);
  if (r == GEM_OK) GEM_CUDA_TRY(cudaStreamSynchronize(st));
  return r;
}

gem_status gem_autotune_batch(const gem_store* s, int32_t mode, int32_t n_queries, int64_t n_q_rows,
                              int32_t max_q_len, int64_t n_cands, float* q, int64_t* q_offsets,
                              int64_t* cand_offsets, int64_t* cand_ids, float* scores, const char* cache_path,
                              int32_t* seg, int32_t* ctas_per_sm, float* ms, int32_t* from_cache, void* stream) {
  GEM_NVTX_RANGE("gem_autotune_batch");
  if (!s || !q || !q_offsets || !cand_offsets || !cand_ids || !scores || !seg || !ctas_per_sm || !ms || !from_cache)
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (mode != GEM_F32 && mode != GEM_CODES) return fail(GEM_ERR_INVALID, "mode must be GEM_F32 or GEM_CODES");
  if (!s->d_f32 || (mode == GEM_CODES && s->k1 == 0)) return fail(GEM_ERR_STATE, "store lacks fp32 copy or codebook");
  if (n_queries < 1 || n_q_rows < n_queries || n_cands < 1) return fail(GEM_ERR_INVALID, "bad sizes");
  if (max_q_len < 1 || max_q_len > 32 * kMaxPasses) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  r = autotune_batch(s, mode, n_queries, n_q_rows, max_q_len, n_cands, q, q_offsets, cand_offsets, cand_ids, scores,
                     cache_path, seg, ctas_per_sm, ms, from_cache, st);
  if (r == GEM_OK) GEM_CUDA_TRY(cudaStreamSynchronize(st));
  return r;
}

gem_status gem_score_ids_noalloc(const gem_store* s, const float* q, const int64_t* q_offsets,
                                 int32_t n_queries, int64_t n_q_rows, int32_t max_q_len,
                                 const int64_t* cand_offsets, const int64_t* cand_ids, int64_t n_cands,
                                 float* scores, void* stream) {
  GEM_NVTX_RANGE("gem_score_ids_noalloc");
  if (!s || !q || !q_offsets || !cand_offsets || (n_cands > 0 && (!cand_ids || !scores)))
    return fail(GEM_ERR_INVALID, "NULL argument");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "id-list scoring reads the fp32 copy");
  if (n_queries < 1 || n_q_rows < n_queries || n_cands < 0) return fail(GEM_ERR_INVALID, "bad sizes");
  if (max_q_len < 1 || max_q_len > 32 * kMaxPasses) return fail(GEM_ERR_INVALID, "max_q_len must be 1..256");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  if (n_cands == 0) return GEM_OK;
  return score_ids_noalloc(s, q, q_offsets, n_queries, n_q_rows, max_q_len, cand_offsets, cand_ids, n_cands,
                           scores, reinterpret_cast<cudaStream_t>(stream));
}

int64_t gem_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

gem_status gem_qemd(const gem_store* s, gem_workspace* w, const int64_t* set_a, const int64_t* set_b, int64_t n_pairs,
                    float* out, void* stream) {
  GEM_NVTX_RANGE("gem_qemd");
  if (!s || !w) return fail(GEM_ERR_INVALID, "NULL argument");
  if (n_pairs < 0) return fail(GEM_ERR_INVALID, "n_pairs < 0");
  if (n_pairs > 0 && (!set_a || !set_b || !out)) return fail(GEM_ERR_INVALID, "NULL argument");
  if (s->k1 == 0 || !s->d_codes) return fail(GEM_ERR_STATE, "qEMD needs the store's codebook (gem_store_set_codebook)");
  gem_status r = check_current_device(s->device);
  if (r != GEM_OK) return r;
  if (n_pairs == 0) return GEM_OK;
  return launch_qemd(s, set_a, set_b, n_pairs, out, w->d_status, reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_selftest_wait_timeout(gem_workspace* w, int64_t budget_cycles, void* stream) {
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  if (budget_cycles < 1 || budget_cycles > ((int64_t)1 << 32)) return fail(GEM_ERR_INVALID, "budget out of range");
  gem_status r = check_current_device(w->device);
  if (r != GEM_OK) return r;
  return launch_wait_selftest(w->d_status, budget_cycles, reinterpret_cast<cudaStream_t>(stream));
}

gem_status gem_stream_status(gem_workspace* w, void* stream) {
  if (!w) return fail(GEM_ERR_INVALID, "workspace is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GEM_CUDA_TRY(cudaStreamSynchronize(st));
  int code = 0;
  GEM_CUDA_TRY(cudaMemcpy(&code, w->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  GEM_CUDA_TRY(cudaMemset(w->d_status, 0, sizeof(int)));
  if (code != 0) {
    set_error(code == GEM_ERR_TIMEOUT ? "a device-side wait timed out"
              : code == GEM_ERR_BOUNDS ? "a device-side index check failed"
                                       : "device-side metadata check failed");
    return (gem_status)code;
  }
  return GEM_OK;
}

}  // extern "C"
