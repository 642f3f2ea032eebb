// Per-row exact top-k (the k-argmax of Eq. 2, Sec. 3.1): score descending,
// ties by lower id.
//
// Each element gets a 64-bit key (order-preserving map of the FP32 score in the
// high word, 0xFFFFFFFF - id in the low word), so "larger key" is exactly
// "better (score, id)" and all keys of a row are distinct.  Elements with a
// negative id, or the id of a set the store marks deleted (Sec. 4.6), are not
// candidates.
//
// Two paths give the same result:
//  - Row path: one CTA per row runs an MSB-first radix select with 8-bit digits
//    on the keys, reading the row once per digit and stopping as soon as the
//    selected bucket holds exactly the remaining count; a final pass gathers the
//    k winners into shared memory, a bitonic sort orders them and the CTA writes
//    ids and scores.
//  - Threshold path (long dense rows, the workspace's candidate buffer): a
//    sample of every row (256 runs of 32 consecutive elements) gives a key
//    threshold T whose expected count above it in the row is 4k + 256; one
//    streaming pass over all rows (many CTAs per row, coalesced 16-byte loads)
//    appends every key >= T to the row's candidate buffer; the row path then
//    selects from that buffer.  Every key of the top k is >= T whenever at
//    least k keys are (the k-th best key is then >= T), so a row whose count is
//    at least k and fits the buffer is exact; any other row (an unlucky sample)
//    falls back to the row path over the whole row.  The score matrix is read
//    about once instead of once per digit.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kTopkThreads = 512;
constexpr int kSampleRuns = 256;                  // runs of the threshold sample
constexpr int kSampleRun = 32;                    // consecutive elements per run
constexpr int kSample = kSampleRuns * kSampleRun; // sampled keys per row
constexpr int kFilterThreads = 256;
constexpr int kFilterPerThread = 32;              // eight 16-byte loads
constexpr int kFilterChunk = kFilterThreads * kFilterPerThread;

__device__ __forceinline__ uint32_t score_key(float f) {
  // -0 and +0 are equal scores: both map to the key of +0, so the id decides
  uint32_t u = __float_as_uint(f == 0.f ? 0.f : f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_score(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

__device__ __forceinline__ uint64_t make_key(float s, int64_t id) {
  return ((uint64_t)score_key(s) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)id);
}

__device__ __forceinline__ bool is_dead(const uint32_t* dead, int64_t n_sets, int64_t id) {
  return dead && id < n_sets && ((dead[id >> 5] >> (id & 31)) & 1u);
}

// A row of scores in global memory (ids may be implicit).
struct RowView {
  const float* s;
  const int64_t* ids;  // null: id = index
  int64_t n;
  const uint32_t* dead;  // null: no set deleted
  int64_t n_sets;
  __device__ __forceinline__ bool key(int64_t t, uint64_t& k) const {
    int64_t id = ids ? ids[t] : t;
    if (id < 0) return false;
    if (is_dead(dead, n_sets, id)) return false;
    k = make_key(s[t], id);
    return true;
  }
};

// A row of ready-made keys (every entry valid).
struct KeyView {
  const uint64_t* keys;
  int64_t n;
  __device__ __forceinline__ bool key(int64_t t, uint64_t& k) const {
    k = keys[t];
    return true;
  }
};

// Row r of the union of n_lists lists laid out [list][rows][k_in]: element t
// is entry t % k_in of list t / k_in (negative ids are empty slots).
struct SegView {
  const float* s;
  const int64_t* ids;
  int64_t n;          // n_lists * k_in
  int64_t list_stride;  // rows * k_in
  int k_in;
  __device__ __forceinline__ bool key(int64_t t, uint64_t& k) const {
    const int64_t idx = (t / k_in) * list_stride + (t % k_in);
    const int64_t id = ids[idx];
    if (id < 0) return false;
    k = make_key(s[idx], id);
    return true;
  }
};

struct SelectSmem {
  int hist[256];
  int suffix[257];
  int digit, count_at, taken, eq_taken;
  unsigned long long n_valid;
};

// hist[digit] += 1 for every active lane, one shared atomic per distinct digit
// of the warp (the keys of a row share their leading digits, so plain atomics
// would serialise on one counter).  Every lane of the warp must call it.
__device__ __forceinline__ void hist_add(int* hist, int digit, bool active) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const unsigned peers = __match_any_sync(act, digit);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[digit], __popc(peers));
}

// Radix select: the leading `bits` bits (`prefix`) of the k_eff-th largest key,
// k_rem of the selection still to come from the keys with that prefix, and
// whether all of them are taken.  All threads of the CTA call it.
template <class View>
__device__ void radix_prefix(const View& v, int k_eff, long long n_valid, SelectSmem& sm, uint64_t& prefix,
                             int& bits, int& k_rem, bool& take_all) {
  prefix = 0;
  bits = 0;
  k_rem = k_eff;
  take_all = (k_eff == n_valid);
  while (!take_all && bits < 64) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) sm.hist[d] = 0;
    __syncthreads();
    const int shift = 56 - bits;
    for (int64_t t0 = 0; t0 < v.n; t0 += blockDim.x) {  // warp-uniform trip count
      const int64_t t = t0 + threadIdx.x;
      uint64_t key = 0;
      bool active = t < v.n && v.key(t, key);
      if (active && bits > 0 && (key >> (64 - bits)) != prefix) active = false;
      hist_add(sm.hist, (int)((key >> shift) & 0xFF), active);
    }
    __syncthreads();
    // suffix sums: suffix[d] = number of matching keys with digit >= d
    if (threadIdx.x < 256) sm.suffix[threadIdx.x] = sm.hist[threadIdx.x];
    if (threadIdx.x == 0) sm.suffix[256] = 0;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
      int add = 0;
      if (threadIdx.x < 256 && threadIdx.x + o < 256) add = sm.suffix[threadIdx.x + o];
      __syncthreads();
      if (threadIdx.x < 256) sm.suffix[threadIdx.x] += add;
      __syncthreads();
    }
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
      if (sm.suffix[d] >= k_rem && sm.suffix[d + 1] < k_rem) {
        sm.digit = d;
        sm.count_at = sm.hist[d];
        sm.taken = sm.suffix[d + 1];  // keys strictly above this digit
      }
    }
    __syncthreads();
    const int d = sm.digit;
    k_rem -= sm.taken;
    prefix = (prefix << 8) | (uint64_t)d;
    bits += 8;
    if (sm.count_at == k_rem) take_all = true;
    __syncthreads();
  }
}

// The top k of one row into out_ids / out_scores (k entries, padded with -1 /
// -inf).  count_valid: the view may hold invalid entries (ids, deletions).
template <class View>
__device__ void select_row(const View& v, bool count_valid, int k, int sort_n, uint64_t* sel, SelectSmem& sm,
                           int64_t* __restrict__ out_ids, float* __restrict__ out_scores) {
  if (threadIdx.x == 0) sm.n_valid = count_valid ? 0ull : (unsigned long long)v.n;
  __syncthreads();
  if (count_valid) {
    unsigned long long c = 0;
    for (int64_t t = threadIdx.x; t < v.n; t += blockDim.x) {
      uint64_t key;
      c += v.key(t, key) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&sm.n_valid, c);
  }
  __syncthreads();
  const long long n_valid = (long long)sm.n_valid;
  const int k_eff = (int)min((long long)k, n_valid);
  uint64_t prefix;
  int bits, k_rem;
  bool take_all;
  radix_prefix(v, k_eff, n_valid, sm, prefix, bits, k_rem, take_all);

  // gather: keys above the prefix bucket, plus k_rem from the bucket
  if (threadIdx.x == 0) { sm.taken = 0; sm.eq_taken = 0; }
  __syncthreads();
  for (int64_t t = threadIdx.x; t < v.n; t += blockDim.x) {
    uint64_t key;
    if (!v.key(t, key)) continue;
    bool pick;
    if (bits == 0) {
      pick = true;  // every valid key is selected
    } else {
      const uint64_t hi = key >> (64 - bits);
      if (hi > prefix) pick = true;
      else if (hi == prefix) pick = take_all || (atomicAdd(&sm.eq_taken, 1) < k_rem);
      else pick = false;
    }
    if (pick) {
      const int slot = atomicAdd(&sm.taken, 1);
      if (slot < sort_n) sel[slot] = key;
    }
  }
  __syncthreads();
  const int n_sel = min(sm.taken, k_eff);
  for (int i = n_sel + threadIdx.x; i < sort_n; i += blockDim.x) sel[i] = 0;
  __syncthreads();
  // bitonic sort, descending
  for (int size = 2; size <= sort_n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < sort_n; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool desc = ((i & size) == 0);
          const uint64_t a = sel[i], b = sel[j];
          if (desc ? (a < b) : (a > b)) { sel[i] = b; sel[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int64_t oid = -1;
    float osc = -INFINITY;
    if (i < n_sel) {
      const uint64_t key = sel[i];
      oid = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
      osc = key_score((uint32_t)(key >> 32));
    }
    out_ids[i] = oid;
    if (out_scores) out_scores[i] = osc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kTopkThreads)
topk_kernel(const float* __restrict__ scores, const int64_t* __restrict__ row_off, int rows,
            int64_t cols, const int64_t* __restrict__ ids, int k, int sort_n,
            int64_t* __restrict__ out_ids, float* __restrict__ out_scores,
            const uint32_t* __restrict__ dead, int64_t n_sets) {
  extern __shared__ uint64_t sel[];  // [sort_n]
  __shared__ SelectSmem sm;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    RowView v;
    const int64_t base = row_off ? row_off[r] : (int64_t)r * cols;
    v.n = row_off ? row_off[r + 1] - base : cols;
    v.s = scores + base;
    v.ids = ids ? ids + base : nullptr;
    v.dead = dead;
    v.n_sets = n_sets;
    select_row(v, v.ids != nullptr || v.dead != nullptr, k, sort_n, sel, sm, out_ids + (int64_t)r * k,
               out_scores ? out_scores + (int64_t)r * k : nullptr);
  }
}

// Threshold path, step 1: a key threshold per dense row from a sample of
// kSample keys (all of the row when it is shorter): the leading digits of the
// sample's r-th largest key, r = ceil(target * sample / cols), so that about
// `target` keys of the row lie at or above it.  Invalid elements enter the
// sample as key 0 (below every valid key).  Also clears the row's counter.
__global__ void __launch_bounds__(kTopkThreads)
topk_sample_kernel(const float* __restrict__ scores, int rows, int64_t cols, const int64_t* __restrict__ ids,
                   const uint32_t* __restrict__ dead, int64_t n_sets, int target,
                   unsigned long long* __restrict__ thr, unsigned* __restrict__ cnt) {
  extern __shared__ uint64_t skeys[];  // [kSample]
  __shared__ SelectSmem sm;
  const int m = (int)min((int64_t)kSample, cols);
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* s = scores + (int64_t)r * cols;
    const int64_t* id_row = ids ? ids + (int64_t)r * cols : nullptr;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      int64_t t = i;
      if (cols > kSample) {  // run q starts at q (cols - 32) / (runs - 1): runs span the row
        const int q = i / kSampleRun;
        t = (int64_t)q * (cols - kSampleRun) / (kSampleRuns - 1) + (i % kSampleRun);
      }
      const int64_t id = id_row ? id_row[t] : t;
      skeys[i] = (id < 0 || is_dead(dead, n_sets, id)) ? 0ull : make_key(s[t], id);
    }
    __syncthreads();
    const int64_t want = ((int64_t)target * m + cols - 1) / cols;
    const int r_target = (int)max((int64_t)1, min((int64_t)m, want));
    KeyView v{skeys, m};
    uint64_t prefix;
    int bits, k_rem;
    bool take_all;
    radix_prefix(v, r_target, m, sm, prefix, bits, k_rem, take_all);
    if (threadIdx.x == 0) {
      thr[r] = bits == 0 ? 0ull : (prefix << (64 - bits));
      cnt[r] = 0u;
    }
    __syncthreads();
  }
}

// Threshold path, step 2: one streaming pass; every valid key >= thr[row] is
// appended to the row's candidate buffer (cap entries; the counter keeps
// counting past it).  Work items are (row, 8,192-element chunk); four CTAs per
// SM (at most 64 registers) keep 128 KB of loads in flight per SM.  The test is a
// float comparison with the threshold's score (keys order like their scores,
// and -0 equals +0 in both); only an element whose score equals it compares
// ids.  Each thread counts its picks, the warp scans the counts and takes one
// slot range with a single atomic.
__global__ void __launch_bounds__(kFilterThreads, 4)
topk_filter_kernel(const float* __restrict__ scores, int rows, int64_t cols, const int64_t* __restrict__ ids,
                   const uint32_t* __restrict__ dead, int64_t n_sets, const unsigned long long* __restrict__ thr,
                   unsigned* __restrict__ cnt, unsigned long long* __restrict__ cand, int cap, bool vec4) {
  const int64_t cpr = (cols + kFilterChunk - 1) / kFilterChunk;
  const int64_t items = (int64_t)rows * cpr;
  const int lane = threadIdx.x & 31;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int r = (int)(item / cpr);
    const int64_t c0 = (item % cpr) * kFilterChunk;
    const float* s = scores + (int64_t)r * cols;
    const int64_t* id_row = ids ? ids + (int64_t)r * cols : nullptr;
    const unsigned long long T = thr[r];
    const bool take_all = (T == 0ull);
    const float fT = take_all ? 0.f : key_score((uint32_t)(T >> 32));
    const uint32_t T_lo = (uint32_t)T;
    float v[kFilterPerThread];
    // eight coalesced 16-byte loads per thread, all in flight before use
#pragma unroll
    for (int j = 0; j < kFilterPerThread / 4; ++j) {
      const int64_t t = c0 + ((int64_t)j * kFilterThreads + threadIdx.x) * 4;
      if (vec4 && t + 3 < cols) {
        const float4 f = __ldcs(reinterpret_cast<const float4*>(s + t));
        v[4 * j] = f.x; v[4 * j + 1] = f.y; v[4 * j + 2] = f.z; v[4 * j + 3] = f.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[4 * j + e] = (t + e < cols) ? s[t + e] : 0.f;
      }
    }
    uint32_t picks = 0;  // bit 4 j + e: element (j, e) is a candidate
    if (!take_all && !id_row && !dead && c0 + kFilterChunk <= cols) {
      // the common case: ids are positions, every element valid; a score equal
      // to the threshold's decides by id
      uint32_t eq = 0;
#pragma unroll
      for (int i = 0; i < kFilterPerThread; ++i) {
        picks |= (v[i] >= fT) ? (1u << i) : 0u;
        eq |= (v[i] == fT) ? (1u << i) : 0u;
      }
      uint32_t check = picks & eq;
      while (check) {
        const int b = __ffs(check) - 1;
        check &= check - 1;
        const int64_t t = c0 + ((int64_t)(b >> 2) * kFilterThreads + threadIdx.x) * 4 + (b & 3);
        if ((0xFFFFFFFFu - (uint32_t)t) < T_lo) picks &= ~(1u << b);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kFilterPerThread / 4; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t t = c0 + ((int64_t)j * kFilterThreads + threadIdx.x) * 4 + e;
          const float sv = v[4 * j + e];
          bool p = take_all || sv >= fT;
          if (p && t < cols && (id_row || dead || (!take_all && sv == fT))) {
            const int64_t id = id_row ? id_row[t] : t;
            p = id >= 0 && !is_dead(dead, n_sets, id) &&
                (take_all || sv > fT || (0xFFFFFFFFu - (uint32_t)id) >= T_lo);
          }
          picks |= (p && t < cols) ? (1u << (4 * j + e)) : 0u;
        }
      }
    }
    // warp: inclusive scan of the pick counts, one atomic for the warp's slots
    const unsigned c = __popc(picks);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;  // warp-uniform
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(cnt + r, total);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - c;
    while (picks) {
      const int b = __ffs(picks) - 1;
      picks &= picks - 1;
      const int64_t t = c0 + ((int64_t)(b >> 2) * kFilterThreads + threadIdx.x) * 4 + (b & 3);
      const int64_t id = id_row ? id_row[t] : t;
      float sv = 0.f;  // v[b] by selects (no dynamic register indexing)
#pragma unroll
      for (int i = 0; i < kFilterPerThread; ++i) sv = (i == b) ? v[i] : sv;
      if (base < (unsigned)cap) cand[(int64_t)r * cap + base] = make_key(sv, id);
      ++base;
    }
  }
}

// Threshold path, step 3: the row path over the candidates of each row, or
// over the whole row when its count is below k or overflowed the buffer.
__global__ void __launch_bounds__(kTopkThreads)
topk_select_kernel(const float* __restrict__ scores, int rows, int64_t cols, const int64_t* __restrict__ ids,
                   int k, int sort_n, int64_t* __restrict__ out_ids, float* __restrict__ out_scores,
                   const uint32_t* __restrict__ dead, int64_t n_sets, const unsigned* __restrict__ cnt,
                   const unsigned long long* __restrict__ cand, int cap) {
  extern __shared__ uint64_t sel[];  // [sort_n]
  __shared__ SelectSmem sm;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const unsigned c = cnt[r];
    int64_t* oi = out_ids + (int64_t)r * k;
    float* os = out_scores ? out_scores + (int64_t)r * k : nullptr;
    if (c >= (unsigned)k && c <= (unsigned)cap) {
      KeyView v{reinterpret_cast<const uint64_t*>(cand) + (int64_t)r * cap, (int64_t)c};
      select_row(v, false, k, sort_n, sel, sm, oi, os);
    } else {
      RowView v;
      v.n = cols;
      v.s = scores + (int64_t)r * cols;
      v.ids = ids ? ids + (int64_t)r * cols : nullptr;
      v.dead = dead;
      v.n_sets = n_sets;
      select_row(v, v.ids != nullptr || v.dead != nullptr, k, sort_n, sel, sm, oi, os);
    }
  }
}

// Merge of per-shard top lists: one CTA per row over the row's n_lists * k_in entries.
__global__ void __launch_bounds__(kTopkThreads)
merge_topk_kernel(const float* __restrict__ scores, const int64_t* __restrict__ ids, int n_lists, int rows,
                  int k_in, int k, int sort_n, int64_t* __restrict__ out_ids, float* __restrict__ out_scores) {
  extern __shared__ uint64_t sel[];  // [sort_n]
  __shared__ SelectSmem sm;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    SegView v;
    v.s = scores + (int64_t)r * k_in;
    v.ids = ids + (int64_t)r * k_in;
    v.n = (int64_t)n_lists * k_in;
    v.list_stride = (int64_t)rows * k_in;
    v.k_in = k_in;
    select_row(v, true, k, sort_n, sel, sm, out_ids + (int64_t)r * k, out_scores ? out_scores + (int64_t)r * k : nullptr);
  }
}

int sort_size(int k) {
  int n = 1;
  while (n < k) n <<= 1;
  return n;
}

}  // namespace

gem_status launch_merge_topk(const float* scores, const int64_t* ids, int32_t n_lists, int32_t rows, int32_t k_in,
                             int32_t k, int64_t* out_ids, float* out_scores, int n_sm, cudaStream_t st) {
  if (rows == 0) return GEM_OK;
  const int sort_n = sort_size(k);
  const size_t smem = sizeof(uint64_t) * sort_n;
  GEM_CUDA_TRY(cudaFuncSetAttribute(merge_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  merge_topk_kernel<<<std::min(rows, n_sm * 4), kTopkThreads, smem, st>>>(scores, ids, n_lists, rows, k_in, k, sort_n,
                                                                          out_ids, out_scores);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

int topk_candidate_cap(int max_k) { return max_k > 0 ? 2 * (4 * max_k + 256) : 0; }

gem_status launch_topk(gem_workspace* ws, const float* scores, const int64_t* row_offsets,
                       int32_t rows, int64_t cols, const int64_t* ids, int32_t k,
                       int64_t* out_ids, float* out_scores, cudaStream_t st) {
  if (rows == 0) return GEM_OK;
  const int sort_n = sort_size(k);
  const size_t smem = sizeof(uint64_t) * sort_n;
  const gem_store* s = ws->store;
  const int target = 4 * k + 256;
  const bool threshold_path = row_offsets == nullptr && ws->d_topk_cand != nullptr &&
                              2 * target <= ws->topk_cap && cols >= 8LL * target;
  if (threshold_path) {
    GEM_CUDA_TRY(cudaFuncSetAttribute(topk_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(uint64_t) * kSample)));
    GEM_CUDA_TRY(cudaFuncSetAttribute(topk_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const bool vec4 = (cols % 4 == 0) && (reinterpret_cast<uintptr_t>(scores) % 16 == 0);
    for (int r0 = 0; r0 < rows; r0 += ws->topk_rows) {
      const int nr = std::min(ws->topk_rows, rows - r0);
      const float* sc = scores + (int64_t)r0 * cols;
      const int64_t* id0 = ids ? ids + (int64_t)r0 * cols : nullptr;
      topk_sample_kernel<<<std::min(nr, s->n_sm * 4), kTopkThreads, sizeof(uint64_t) * kSample, st>>>(
          sc, nr, cols, id0, s->d_dead, s->n_sets, target, ws->d_topk_thr, ws->d_topk_cnt);
      const int64_t items = (int64_t)nr * ((cols + kFilterChunk - 1) / kFilterChunk);
      topk_filter_kernel<<<(unsigned)std::min<int64_t>(items, (int64_t)s->n_sm * 8), kFilterThreads, 0, st>>>(
          sc, nr, cols, id0, s->d_dead, s->n_sets, ws->d_topk_thr, ws->d_topk_cnt, ws->d_topk_cand, ws->topk_cap,
          vec4);
      topk_select_kernel<<<std::min(nr, s->n_sm * 4), kTopkThreads, smem, st>>>(
          sc, nr, cols, id0, k, sort_n, out_ids + (int64_t)r0 * k, out_scores ? out_scores + (int64_t)r0 * k : nullptr,
          s->d_dead, s->n_sets, ws->d_topk_cnt, ws->d_topk_cand, ws->topk_cap);
      GEM_CUDA_TRY(cudaGetLastError());
      note_launches(3);
    }
    return GEM_OK;
  }
  GEM_CUDA_TRY(cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_kernel, kTopkThreads, smem));
  if (per_sm < 1) per_sm = 1;
  const int grid = std::min<int>(rows, s->n_sm * per_sm);
  topk_kernel<<<grid, kTopkThreads, smem, st>>>(scores, row_offsets, rows, cols, ids, k, sort_n, out_ids, out_scores,
                                                s->d_dead, s->n_sets);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
