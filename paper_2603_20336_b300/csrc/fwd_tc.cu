// MaxSim forward over (query, set) pairs on the sm_103a tensor cores, with the
// argmax side output the backward needs (GEM_BF16, query sets of at most 128
// vectors):
//   S_t = sum_i max_j <q_i, p_j>  (Eq. 1),  j*(t, i) = argmax_j, lowest j on ties,
// every component rounded to bfloat16 (nearest even) and products accumulated in
// FP32 -- the arithmetic of the SIMT forward, with the sum over i taken in a
// fixed order (a butterfly within each warp of 32 rows, then the warps in order).
//
// The query rows are first rounded to bf16 into scratch.  Work unit = 16
// consecutive pairs; a persistent CTA per SM draws units from a counter.  The
// query block (A, 128 rows) stays in shared memory while its pairs run.  Each
// set is read once, as FP32: TMA brings it in boxes of 32 rows (at most 31 rows
// read past its end) into a four-slot staging ring, and four converter warps
// round each box to bf16 into the 128-byte-swizzled operand layout of a
// two-stage ring of 256-row tiles (a proxy fence makes the writes visible to the
// tensor cores).  One MMA per K step covers the tile with N = 32 x boxes.  The
// accumulator (128 query rows x 256 rows of the set) is double-buffered in TMEM;
// four epilogue warps, one thread per query row, take the running max and argmax
// over the set's valid columns, write the argmax row and add the row maxima (a
// butterfly per warp, the four warp sums in order through shared memory).
#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kFtN = 256;                       // set rows per tile
constexpr int kFtBox = 32;                      // rows per TMA box
constexpr int kFtStages = 2;
constexpr int kFtPairsPerUnit = 16;
constexpr int kFtEpiWarps = 4;
constexpr int kFtConvWarps = 4;                       // FP32 -> bf16 converters, one staging slot each
constexpr int kFtConv0 = kFtEpiWarps + 2;             // first converter warp
constexpr int kFtThreads = (kFtEpiWarps + 2 + kFtConvWarps) * 32;   // + producer, MMA warp, converters
constexpr int kFtABytes = 128 * kDim * 2;             // 32 KB
constexpr int kFtStageBytes = kFtN * kDim * 2;        // 64 KB
constexpr int kFtStgBytes = kFtBox * kDim * 4;        // one FP32 box: 16 KB
constexpr int kFtUnitRing = 2;
constexpr int kFtNBars = 2 * kFtStages + 4 + 2 + 1 + 2 * kFtUnitRing + 4 + 2 * kFtConvWarps;
constexpr int kFtBarBytes =
    (kFtNBars * 8 + 16 + 4 * kFtUnitRing + 2 * 4 * 4 + 2 * 4 * kFtConvWarps + 127) / 128 * 128;
constexpr int kFtSmem = 1024 + kFtABytes + kFtStages * kFtStageBytes + kFtConvWarps * kFtStgBytes + kFtBarBytes;
static_assert(kFtSmem <= 232448, "shared memory over the per-block limit");

struct FtArgs {
  const int64_t* q_off;
  int n_queries;
  const int64_t* d_off;
  int64_t n_docs;
  const int64_t* pair_off;
  const int64_t* pair_ids;
  int64_t n_pairs;
  int max_q_len;
  float* scores;
  int32_t* argmax;
  int* status;
  int* unit_counter;
};

// the query owning pair t (pair_off is non-decreasing)
__device__ __forceinline__ int query_of(const int64_t* pair_off, int n_queries, int64_t t) {
  int lo = 0, hi = n_queries - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pair_off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// What every role derives for pair t: its query, the set's first row and
// length, and the number of 256-row tiles (0: nothing to score).
struct PairInfo {
  int b;
  int m_q;
  int64_t q0;
  int64_t r0;
  int m_p;
  int tiles;
  bool bad_id;
};

__device__ __forceinline__ PairInfo pair_info(const FtArgs& a, int64_t t) {
  PairInfo p;
  p.b = query_of(a.pair_off, a.n_queries, t);
  p.q0 = a.q_off[p.b];
  p.m_q = (int)(a.q_off[p.b + 1] - p.q0);
  const int64_t d = a.pair_ids[t];
  p.bad_id = d < 0 || d >= a.n_docs;
  p.r0 = p.bad_id ? 0 : a.d_off[d];
  const int64_t m = p.bad_id ? 0 : a.d_off[d + 1] - p.r0;
  p.m_p = (int)min(m, (int64_t)INT32_MAX);
  const bool bad_q = p.m_q < 1 || p.m_q > a.max_q_len;
  p.tiles = (p.bad_id || bad_q || m < 1) ? 0 : (int)((m + kFtN - 1) / kFtN);
  return p;
}

// pair i's info from the lane that loaded it (every lane of the warp calls it)
__device__ __forceinline__ PairInfo shfl_pair(const PairInfo& m, int i) {
  PairInfo p;
  p.b = __shfl_sync(0xffffffffu, m.b, i);
  p.m_q = __shfl_sync(0xffffffffu, m.m_q, i);
  p.q0 = __shfl_sync(0xffffffffu, (long long)m.q0, i);
  p.r0 = __shfl_sync(0xffffffffu, (long long)m.r0, i);
  p.m_p = __shfl_sync(0xffffffffu, m.m_p, i);
  p.tiles = __shfl_sync(0xffffffffu, m.tiles, i);
  p.bad_id = __shfl_sync(0xffffffffu, (int)m.bad_id, i) != 0;
  return p;
}

// the infos of a unit's pairs t0 .. t0 + cnt - 1, lane i holding pair t0 + i:
// one round of parallel loads per unit instead of a chain of dependent loads
// per pair
__device__ __forceinline__ PairInfo unit_pairs(const FtArgs& a, int64_t t0, int cnt, int lane) {
  PairInfo m{};
  if (lane < cnt) m = pair_info(a, t0 + lane);
  return m;
}

__global__ void __launch_bounds__(kFtThreads, 1)
fwd_tc_kernel(const __grid_constant__ CUtensorMap tm_q, const __grid_constant__ CUtensorMap tm_d, FtArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a_smem = smem;                        // [2 halves][128 rows][128 B]
  uint8_t* b_smem = smem + kFtABytes;            // [stage][2 halves][256 rows][128 B]
  uint8_t* stg_smem = b_smem + kFtStages * kFtStageBytes;  // [slot][32 rows][128 FP32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_smem + kFtConvWarps * kFtStgBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kFtStages;
  uint64_t* acc_full = bars + 2 * kFtStages;     // [2]
  uint64_t* acc_empty = acc_full + 2;            // [2]
  uint64_t* q_full = acc_empty + 2;
  uint64_t* q_empty = q_full + 1;
  uint64_t* done_bar = q_empty + 1;
  uint64_t* unit_full = done_bar + 1;            // [UNIT_RING]
  uint64_t* unit_empty = unit_full + kFtUnitRing;
  uint64_t* part_full = unit_empty + kFtUnitRing;  // [2] per pair parity, count 4
  uint64_t* part_empty = part_full + 2;            // [2] count 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(part_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* unit_ring = abort_flag + 1;                               // [UNIT_RING]
  float* parts = const_cast<float*>(reinterpret_cast<volatile float*>(unit_ring + kFtUnitRing));  // [2][4]
  uint64_t* stg_full = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(parts + 8) + 7) & ~uintptr_t(7));   // [slot]: the FP32 box landed
  uint64_t* stg_empty = stg_full + kFtConvWarps;                         // [slot]: converted
  volatile int* stg_desc = reinterpret_cast<volatile int*>(stg_empty + kFtConvWarps);  // [slot][2]: stage, box (-1: stop)

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long n_units = (a.n_pairs + kFtPairsPerUnit - 1) / kFtPairsPerUnit;
  if (blockIdx.x >= n_units) return;

  if (threadIdx.x == 0) {
    // full[s]: one arrival per 32-row box of the tile (a converter each, the
    // producer for the boxes past the set's end)
    for (int s = 0; s < kFtStages; ++s) { mbar_init(&full[s], kFtN / kFtBox); mbar_init(&empty[s], 1); }
    for (int c = 0; c < kFtConvWarps; ++c) { mbar_init(&stg_full[c], 1); mbar_init(&stg_empty[c], 1); }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kFtEpiWarps);
      mbar_init(&part_full[i], kFtEpiWarps);
      mbar_init(&part_empty[i], 1);
    }
    mbar_init(q_full, 1);
    mbar_init(q_empty, 1);
    mbar_init(done_bar, 1);
    for (int i = 0; i < kFtUnitRing; ++i) {
      mbar_init(&unit_full[i], 1);
      mbar_init(&unit_empty[i], 1 + kFtEpiWarps);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kFtEpiWarps + 1) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kFtEpiWarps) {
    // ------------------------------------------------------------------ producer
    // lane 0 issues; the warp loads each unit's pair infos in parallel
    if (lane == 0) {
      tma_prefetch_desc(&tm_q);
      tma_prefetch_desc(&tm_d);
    }
    int stage = 0;
    uint32_t phase = 0;
    uint64_t n_box = 0;  // FP32 boxes issued (box g goes to staging slot g % kFtConvWarps)
    uint32_t n_a = 0;  // query blocks loaded
    int cur_b = -1;
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    for (;;) {
      long long u = 0;
      int okl = 1;
      if (lane == 0) {
        u = atomicAdd(a.unit_counter, 1);
        okl = mbar_wait(&unit_empty[uslot], uphase ^ 1, a.status, abort_flag) ? 1 : 0;
        if (okl) {
          unit_ring[uslot] = (int)(u < n_units ? u : n_units);
          mbar_arrive(&unit_full[uslot]);
        }
      }
      u = __shfl_sync(0xffffffffu, u, 0);
      if (!__shfl_sync(0xffffffffu, okl, 0)) { ok = false; break; }
      if (++uslot == kFtUnitRing) { uslot = 0; uphase ^= 1; }
      if (u >= n_units) break;
      const int64_t t0 = u * kFtPairsPerUnit;
      const int cnt = (int)min((int64_t)kFtPairsPerUnit, a.n_pairs - t0);
      const PairInfo mine = unit_pairs(a, t0, cnt, lane);
      for (int i = 0; i < cnt && ok; ++i) {
        const PairInfo p = shfl_pair(mine, i);
        if (p.tiles == 0) continue;
        if (lane == 0) {
          if (p.b != cur_b) {
            if (n_a > 0 && !mbar_wait(q_empty, (n_a - 1) & 1, a.status, abort_flag)) okl = 0;
            if (okl) {
              mbar_arrive_expect_tx(q_full, kFtABytes);
              for (int h = 0; h < 2; ++h) tma_load_2d(a_smem + h * 16384, &tm_q, q_full, h * 64, (int)p.q0);
              ++n_a;
              cur_b = p.b;
            }
          }
          for (int tile = 0; tile < p.tiles && okl; ++tile) {
            const int rows = min(kFtN, p.m_p - tile * kFtN);
            const int nb = (rows + kFtBox - 1) / kFtBox;
            if (!mbar_wait(&empty[stage], phase ^ 1, a.status, abort_flag)) { okl = 0; break; }
            const int row0 = (int)(p.r0 + (int64_t)tile * kFtN);
            for (int bx = 0; bx < nb && okl; ++bx) {
              // the box's FP32 rows into the next staging slot; its converter
              // writes them, rounded, into this stage
              const int sl = (int)(n_box % kFtConvWarps);
              const uint32_t use = (uint32_t)(n_box / kFtConvWarps);
              if (use > 0 && !mbar_wait(&stg_empty[sl], (use - 1) & 1, a.status, abort_flag)) { okl = 0; break; }
              stg_desc[2 * sl] = stage;
              stg_desc[2 * sl + 1] = bx;
              mbar_arrive_expect_tx(&stg_full[sl], kFtStgBytes);
              tma_load_2d(stg_smem + sl * kFtStgBytes, &tm_d, &stg_full[sl], 0, row0 + bx * kFtBox);
              ++n_box;
            }
            for (int bx = nb; bx < kFtN / kFtBox; ++bx) mbar_arrive(&full[stage]);  // no rows there
            if (++stage == kFtStages) { stage = 0; phase ^= 1; }
          }
        }
        if (!__shfl_sync(0xffffffffu, okl, 0)) ok = false;
      }
    }
    if (lane == 0) {
      if (ok) {
        // stop every converter: a descriptor of -1 in its slot, once the slot is free
        for (int sl = 0; sl < kFtConvWarps; ++sl) {
          const uint64_t uses = n_box / kFtConvWarps + ((uint64_t)sl < n_box % kFtConvWarps ? 1 : 0);
          if (uses > 0 && !mbar_wait(&stg_empty[sl], (uint32_t)((uses - 1) & 1), a.status, abort_flag)) break;
          stg_desc[2 * sl] = -1;
          mbar_arrive(&stg_full[sl]);
        }
      } else {
        // drain: every load this thread issued must land before the CTA exits
        for (int sl = 0; sl < kFtConvWarps; ++sl) {
          const uint64_t uses = n_box / kFtConvWarps + ((uint64_t)sl < n_box % kFtConvWarps ? 1 : 0);
          if (uses) { int z = 0; mbar_wait(&stg_full[sl], (uint32_t)((uses - 1) & 1), nullptr, &z); }
        }
        int z = 0;
        if (n_a) mbar_wait(q_full, (n_a - 1) & 1, nullptr, &z);
      }
    }
  } else if (warp == kFtEpiWarps + 1) {
    // ------------------------------------------------------------------ MMA issuer
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    uint32_t n_a = 0;
    int cur_b = -1;
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    const uint64_t ad0 = sw128_desc(smem_u32(a_smem));
    for (;;) {
      const bool w = mbar_wait(&unit_full[uslot], uphase, a.status, abort_flag);
      if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
      const long long u = unit_ring[uslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&unit_empty[uslot]);
      if (++uslot == kFtUnitRing) { uslot = 0; uphase ^= 1; }
      if (u >= n_units) break;
      const int64_t t0 = u * kFtPairsPerUnit;
      const int cnt = (int)min((int64_t)kFtPairsPerUnit, a.n_pairs - t0);
      const PairInfo mine = unit_pairs(a, t0, cnt, lane);
      for (int i = 0; i < cnt && ok; ++i) {
        const PairInfo p = shfl_pair(mine, i);
        if (p.tiles == 0) continue;
        int okl = 1;
        if (lane == 0) {
          if (p.b != cur_b) {
            if (n_a > 0) mma_commit(q_empty);   // the previous block's MMAs release it
            if (!mbar_wait(q_full, n_a & 1, a.status, abort_flag)) okl = 0;
            tc_fence_after();
            ++n_a;
            cur_b = p.b;
          }
          for (int tile = 0; tile < p.tiles && okl; ++tile) {
            const int rows = min(kFtN, p.m_p - tile * kFtN);
            const int nb = (rows + kFtBox - 1) / kFtBox;
            if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1, a.status, abort_flag)) { okl = 0; break; }
            if (!mbar_wait(&full[stage], phase, a.status, abort_flag)) { okl = 0; break; }
            tc_fence_after();
            const uint64_t bd0 = sw128_desc(smem_u32(b_smem + stage * kFtStageBytes));
            const uint32_t idesc = make_idesc(128, nb * kFtBox, 1u, 1u);
            const uint32_t dt = tmem + acc * kFtN;
#pragma unroll
            for (int k = 0; k < kDim / 16; ++k) {
              const int half = (k * 32) / 128;
              const int within = (k * 32) % 128;
              mma_bf16(dt, ad0 + (uint64_t)((half * 16384 + within) >> 4),
                       bd0 + (uint64_t)((half * (kFtN * 128) + within) >> 4), idesc, k > 0);
            }
            mma_commit(&empty[stage]);
            mma_commit(&acc_full[acc]);
            if (++stage == kFtStages) { stage = 0; phase ^= 1; }
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
          }
        }
        if (!__shfl_sync(0xffffffffu, okl, 0)) ok = false;
      }
      if (!ok) break;
    }
    if (lane == 0) {
      mma_commit(done_bar);
      int z = 0;
      mbar_wait(done_bar, 0, nullptr, &z);
    }
  } else if (warp >= kFtConv0) {
    // ------------------------------------------------------------------ converters
    // warp c takes staging slot c: 32 FP32 rows -> bf16 (nearest even) at rows
    // 32 box .. 32 box + 31 of its stage, in the 128-byte swizzle (16-byte chunk
    // index XOR row % 8) the MMA descriptors expect
    const int sl = warp - kFtConv0;
    const float* stg = reinterpret_cast<const float*>(stg_smem + sl * kFtStgBytes);
    const int h = lane >> 4;                 // component half of this lane's 4 floats
    const int cc = (lane & 15) >> 1;         // 16-byte chunk within the half
    for (uint32_t n = 0;; ++n) {
      const bool w = mbar_wait(&stg_full[sl], n & 1, a.status, abort_flag);
      if (!__all_sync(0xffffffffu, w)) break;
      const int st_i = stg_desc[2 * sl];
      const int bx = stg_desc[2 * sl + 1];
      if (st_i < 0) break;
      uint8_t* dst = b_smem + st_i * kFtStageBytes + h * (kFtN * 128) + (lane & 1) * 8;
      // eight rows' loads in flight before their conversions and stores
#pragma unroll 1
      for (int r0 = 0; r0 < kFtBox; r0 += 8) {
        float4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = reinterpret_cast<const float4*>(stg + (r0 + u) * kDim)[lane];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          uint2 o;
          o.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[u].x)) |
                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[u].y)) << 16);
          o.y = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[u].z)) |
                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[u].w)) << 16);
          const int R = bx * kFtBox + r0 + u;
          *reinterpret_cast<uint2*>(dst + R * 128 + ((cc ^ (R & 7)) << 4)) = o;
        }
      }
      fence_proxy_async_shared();   // the writes, visible to the tensor cores
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&stg_empty[sl]);
        mbar_arrive(&full[st_i]);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const uint32_t t_lane = (uint32_t)(warp * 32) << 16;
    const int row = warp * 32 + lane;  // query row within the block
    int acc = 0;
    uint32_t acc_phase = 0;
    uint32_t n_pair = 0;  // pairs summed (part buffers alternate)
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    for (;;) {
      const bool w = mbar_wait(&unit_full[uslot], uphase, a.status, abort_flag);
      if (!__all_sync(0xffffffffu, w)) break;
      const long long u = unit_ring[uslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&unit_empty[uslot]);
      if (++uslot == kFtUnitRing) { uslot = 0; uphase ^= 1; }
      if (u >= n_units) break;
      const int64_t t0 = u * kFtPairsPerUnit;
      const int cnt = (int)min((int64_t)kFtPairsPerUnit, a.n_pairs - t0);
      const PairInfo mine_p = unit_pairs(a, t0, cnt, lane);
      for (int i = 0; i < cnt && ok; ++i) {
        const int64_t t = t0 + i;
        const PairInfo p = shfl_pair(mine_p, i);
        if (p.tiles == 0) {
          if (warp == 0 && lane == 0) {
            if (p.bad_id) {
              set_status(a.status, kDevBounds);
              a.scores[t] = __int_as_float(0x7fc00000);
            } else {
              set_status(a.status, kDevInvalid);
            }
          }
          continue;
        }
        const bool any_rows = warp * 32 < p.m_q;  // warp-uniform
        float best = -INFINITY;
        int best_j = 0;
        for (int tile = 0; tile < p.tiles; ++tile) {
          const int rows = min(kFtN, p.m_p - tile * kFtN);
          const int nb = (rows + kFtBox - 1) / kFtBox;
          const bool got = mbar_wait(&acc_full[acc], acc_phase, a.status, abort_flag);
          if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
          tc_fence_after();
          if (any_rows) {
            for (int c = 0; c < nb; ++c) {
              float v[32];
              tmem_ld32(tmem + t_lane + acc * kFtN + c * 32, v);
              const int j0 = tile * kFtN + c * 32;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const float x = (c * 32 + j < rows) ? v[j] : -INFINITY;
                if (x > best) { best = x; best_j = j0 + j; }
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[acc]);
          if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
        if (!ok) break;
        const bool mine = row < p.m_q;
        if (mine) a.argmax[t * a.max_q_len + row] = best_j;
        // the rows' maxima summed: a butterfly within the warp, the warps in order
        float s = mine ? best : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int pb = n_pair & 1;
        if (n_pair >= 2) {
          const bool e = mbar_wait(&part_empty[pb], ((n_pair >> 1) - 1) & 1, a.status, abort_flag);
          if (!__all_sync(0xffffffffu, e)) { ok = false; break; }
        }
        if (lane == 0) {
          parts[pb * 4 + warp] = s;
          mbar_arrive(&part_full[pb]);
        }
        if (warp == 0) {
          const bool f = mbar_wait(&part_full[pb], (n_pair >> 1) & 1, a.status, abort_flag);
          if (!__all_sync(0xffffffffu, f)) { ok = false; break; }
          if (lane == 0) {
            const volatile float* pv = parts + pb * 4;
            a.scores[t] = ((pv[0] + pv[1]) + pv[2]) + pv[3];
            mbar_arrive(&part_empty[pb]);
          }
        }
        ++n_pair;
      }
      if (!ok) break;
    }
  }

  __syncthreads();
  if (warp == kFtEpiWarps + 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// FP32 -> bf16 (nearest even), n rows of 128
__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n4, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(x)[i];
    uint2 o;
    o.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v.x)) |
          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v.y)) << 16);
    o.y = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v.z)) |
          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v.w)) << 16);
    reinterpret_cast<uint2*>(y)[i] = o;
  }
}

}  // namespace

gem_status launch_maxsim_fwd_tc(const float* q, const int64_t* q_off, int32_t n_queries, int64_t n_q_rows,
                                const float* docs, const int64_t* d_off, int64_t n_docs, int64_t n_doc_rows,
                                const int64_t* pair_off, const int64_t* pair_ids, int64_t n_pairs, int32_t max_q_len,
                                float* scores, int32_t* argmax, int* status, int n_sm, cudaStream_t st) {
  if (max_q_len > 128) return fail(GEM_ERR_UNSUPPORTED, "the tensor-core forward takes query sets of <= 128 rows");
  if (n_q_rows >= ((int64_t)1 << 31) || n_doc_rows >= ((int64_t)1 << 31))
    return fail(GEM_ERR_INVALID, "too many rows");
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t qb = up((size_t)n_q_rows * kDim * 2);
  uint8_t* base = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), qb + 256, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GEM_ERR_OOM, "scratch of the tensor-core forward");
  }
  auto* qh = reinterpret_cast<__nv_bfloat16*>(base);
  int* counter = reinterpret_cast<int*>(base + qb);
  auto done = [&](gem_status r) {
    cudaFreeAsync(base, st);
    return r;
  };
  CUtensorMap tm_q, tm_d;
  if (!encode_tmap_2d(&tm_q, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, qh, kDim, (uint64_t)n_q_rows, kDim * 2, 64, 128,
                      CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tm_d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<float*>(docs), kDim, (uint64_t)n_doc_rows,
                      kDim * 4, kDim, kFtBox, CU_TENSOR_MAP_SWIZZLE_NONE))
    return done(fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the forward operands"));
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFtSmem);
    if (e != cudaSuccess) return done(cuda_fail(e, "cudaFuncSetAttribute"));
    attr_set = true;
  }
  const int64_t nq4 = n_q_rows * kDim / 4;
  to_bf16_kernel<<<(int)std::min<int64_t>((nq4 + 255) / 256, n_sm * 16LL), 256, 0, st>>>(q, nq4, qh);
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return done(cuda_fail(e, "cudaMemsetAsync"));
  FtArgs aa;
  aa.q_off = q_off;
  aa.n_queries = n_queries;
  aa.d_off = d_off;
  aa.n_docs = n_docs;
  aa.pair_off = pair_off;
  aa.pair_ids = pair_ids;
  aa.n_pairs = n_pairs;
  aa.max_q_len = max_q_len;
  aa.scores = scores;
  aa.argmax = argmax;
  aa.status = status;
  aa.unit_counter = counter;
  const int64_t units = (n_pairs + kFtPairsPerUnit - 1) / kFtPairsPerUnit;
  fwd_tc_kernel<<<(unsigned)std::min<int64_t>(units, n_sm), kFtThreads, kFtSmem, st>>>(tm_q, tm_d, aa);
  e = cudaGetLastError();
  note_launches(2);
  if (e != cudaSuccess) return done(cuda_fail(e, "fwd_tc_kernel"));
  return done(GEM_OK);
}

}  // namespace gem
