// Per-row exact top-k (the k-argmax of Eq. 2, Sec. 3.1): score descending,
// ties by lower id.
//
// Each element gets a 64-bit key (order-preserving map of the FP32 score in the
// high word, 0xFFFFFFFF - id in the low word), so "larger key" is exactly
// "better (score, id)".  One CTA per row runs an MSB-first radix select with
// 8-bit digits on that key, reading the row once per digit and stopping as soon
// as the selected bucket holds exactly the remaining count; a final pass gathers
// the k winners into shared memory, a bitonic sort orders them and the CTA
// writes ids and scores.  Elements with a negative id, or the id of a set the
// store marks deleted (Sec. 4.6), are not candidates.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kTopkThreads = 512;

__device__ __forceinline__ uint32_t score_key(float f) {
  // -0 and +0 are equal scores: both map to the key of +0, so the id decides
  uint32_t u = __float_as_uint(f == 0.f ? 0.f : f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_score(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

struct RowView {
  const float* s;
  const int64_t* ids;  // null: id = index
  int64_t n;
  const uint32_t* dead;  // null: no set deleted
  int64_t n_sets;
  __device__ __forceinline__ bool key(int64_t t, uint64_t& k) const {
    int64_t id = ids ? ids[t] : t;
    if (id < 0) return false;
    if (dead && id < n_sets && ((dead[id >> 5] >> (id & 31)) & 1u)) return false;
    k = ((uint64_t)score_key(s[t]) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)id);
    return true;
  }
};

__global__ void __launch_bounds__(kTopkThreads)
topk_kernel(const float* __restrict__ scores, const int64_t* __restrict__ row_off, int rows,
            int64_t cols, const int64_t* __restrict__ ids, int k, int sort_n,
            int64_t* __restrict__ out_ids, float* __restrict__ out_scores,
            const uint32_t* __restrict__ dead, int64_t n_sets) {
  extern __shared__ uint64_t sel[];  // [sort_n]
  __shared__ int hist[256];
  __shared__ int suffix[257];
  __shared__ int s_digit, s_count_at, s_taken, s_eq_taken;
  __shared__ long long s_n_valid;

  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    RowView v;
    int64_t base = row_off ? row_off[r] : (int64_t)r * cols;
    v.n = row_off ? row_off[r + 1] - base : cols;
    v.s = scores + base;
    v.ids = ids ? ids + base : nullptr;
    v.dead = dead;
    v.n_sets = n_sets;

    // count valid elements (every element is valid when there are no ids and
    // no deleted sets: no pass over the row is needed)
    if (threadIdx.x == 0) s_n_valid = (v.ids == nullptr && v.dead == nullptr) ? v.n : 0;
    __syncthreads();
    if (v.ids != nullptr || v.dead != nullptr) {
      long long c = 0;
      for (int64_t t = threadIdx.x; t < v.n; t += blockDim.x) {
        uint64_t key;
        c += v.key(t, key) ? 1 : 0;
      }
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&s_n_valid, (unsigned long long)c);
    }
    __syncthreads();
    const long long n_valid = s_n_valid;
    const int k_eff = (int)min((long long)k, n_valid);

    // radix select: prefix of `bits` determined bits; k_rem still needed from
    // the elements matching the prefix
    uint64_t prefix = 0;
    int bits = 0;
    int k_rem = k_eff;
    bool take_all_matching = (k_eff == n_valid);
    while (!take_all_matching && bits < 64) {
      for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
      __syncthreads();
      const int shift = 56 - bits;
      for (int64_t t = threadIdx.x; t < v.n; t += blockDim.x) {
        uint64_t key;
        if (!v.key(t, key)) continue;
        if (bits > 0 && (key >> (64 - bits)) != prefix) continue;
        atomicAdd(&hist[(key >> shift) & 0xFF], 1);
      }
      __syncthreads();
      // suffix sums: suffix[d] = number of matching elements with digit >= d
      if (threadIdx.x < 256) suffix[threadIdx.x] = hist[threadIdx.x];
      if (threadIdx.x == 0) suffix[256] = 0;
      __syncthreads();
      for (int o = 1; o < 256; o <<= 1) {
        int add = 0;
        if (threadIdx.x < 256 && threadIdx.x + o < 256) add = suffix[threadIdx.x + o];
        __syncthreads();
        if (threadIdx.x < 256) suffix[threadIdx.x] += add;
        __syncthreads();
      }
      if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        if (suffix[d] >= k_rem && suffix[d + 1] < k_rem) {
          s_digit = d;
          s_count_at = hist[d];
          s_taken = suffix[d + 1];  // elements strictly above this digit
        }
      }
      __syncthreads();
      const int d = s_digit;
      k_rem -= s_taken;
      prefix = (prefix << 8) | (uint64_t)d;
      bits += 8;
      if (s_count_at == k_rem) take_all_matching = true;
      __syncthreads();
    }

    // gather: keys above the prefix bucket, plus k_rem from the bucket
    if (threadIdx.x == 0) { s_taken = 0; s_eq_taken = 0; }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < v.n; t += blockDim.x) {
      uint64_t key;
      if (!v.key(t, key)) continue;
      bool pick;
      if (bits == 0) {
        pick = true;  // every valid element is selected
      } else {
        const uint64_t hi = key >> (64 - bits);
        if (hi > prefix) pick = true;
        else if (hi == prefix) pick = take_all_matching || (atomicAdd(&s_eq_taken, 1) < k_rem);
        else pick = false;
      }
      if (pick) {
        int slot = atomicAdd(&s_taken, 1);
        if (slot < sort_n) sel[slot] = key;
      }
    }
    __syncthreads();
    const int n_sel = min(s_taken, k_eff);
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
      out_ids[(int64_t)r * k + i] = oid;
      if (out_scores) out_scores[(int64_t)r * k + i] = osc;
    }
    __syncthreads();
  }
}

}  // namespace

gem_status launch_topk(gem_workspace* ws, const float* scores, const int64_t* row_offsets,
                       int32_t rows, int64_t cols, const int64_t* ids, int32_t k,
                       int64_t* out_ids, float* out_scores, cudaStream_t st) {
  if (rows == 0) return GEM_OK;
  int sort_n = 1;
  while (sort_n < k) sort_n <<= 1;
  const size_t smem = sizeof(uint64_t) * sort_n;
  GEM_CUDA_TRY(cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_kernel, kTopkThreads, smem));
  if (per_sm < 1) per_sm = 1;
  const int grid = std::min<int>(rows, ws->store->n_sm * per_sm);
  topk_kernel<<<grid, kTopkThreads, smem, st>>>(scores, row_offsets, rows, cols, ids, k, sort_n,
                                                out_ids, out_scores, ws->store->d_dead, ws->store->n_sets);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
