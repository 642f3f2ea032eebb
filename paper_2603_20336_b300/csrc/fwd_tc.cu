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
// read past its end) into a six-slot staging ring (96 KB of loads in flight per
// SM).  Six converter warps take the boxes in turn: a converter reads its
// box and rounds it to bf16 in registers, frees the slot, waits until its
// tile's operand stage is free (the MMAs of the stage's previous tile have
// completed: a count of completed tiles the epilogue publishes) and writes the
// box into the 128-byte-swizzled layout of a three-stage ring of 128-row tiles
// (a proxy fence makes the writes visible to the tensor cores).  So a staging
// slot is held only for its load, and the loads run ahead of the tensor cores by
// up to six boxes whatever the tile sizes.  One MMA per K step covers the tile
// with N = 32 x boxes.  The accumulator (128 query rows x 128 rows of the set)
// has four buffers in TMEM; four epilogue warps, one thread per query row, take
// the running max and argmax over the set's valid columns, write the argmax row
// and add the row maxima (a butterfly per warp, the four warp sums in order
// through shared memory).
#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kFtN = 128;                       // set rows per tile
constexpr int kFtBox = 32;                      // rows per TMA box
constexpr int kFtBoxes = kFtN / kFtBox;         // boxes per tile
constexpr int kFtStages = 3;
constexpr int kFtPairsPerUnit = 16;
constexpr int kFtEpiWarps = 4;
constexpr int kFtConvWarps = 6;                       // FP32 -> bf16 converters: boxes c, c + C, ...
constexpr int kFtSlotsPerConv = 1;
constexpr int kFtSlots = kFtSlotsPerConv * kFtConvWarps;  // FP32 staging slots; converter c uses c + C s
constexpr int kFtAccs = 4;                            // TMEM accumulators
constexpr int kFtConv0 = kFtEpiWarps + 2;             // first converter warp
constexpr int kFtThreads = (kFtEpiWarps + 2 + kFtConvWarps) * 32;   // + producer, MMA warp, converters
constexpr int kFtABytes = 128 * kDim * 2;             // 32 KB
constexpr int kFtStageBytes = kFtN * kDim * 2;        // 32 KB
constexpr int kFtStgBytes = kFtBox * kDim * 4;        // one FP32 box: 16 KB
constexpr int kFtTmemCols = kFtAccs * kFtN < 32 ? 32 : kFtAccs * kFtN;   // a power of two >= 32
static_assert((kFtTmemCols & (kFtTmemCols - 1)) == 0 && kFtTmemCols <= 512, "TMEM allocation");
constexpr int kFtUnitRing = 2;
constexpr int kFtNBars = kFtStages + 2 * kFtAccs + 2 + 1 + 2 * kFtUnitRing + 4 + 2 * kFtSlots;
constexpr int kFtBarBytes =
    (kFtNBars * 8 + 16 + 4 * kFtUnitRing + 2 * 4 * 4 + 4 * 4 * kFtSlots + 8 + 127) / 128 * 128;
constexpr int kFtSmem = 1024 + kFtABytes + kFtStages * kFtStageBytes + kFtSlots * kFtStgBytes + kFtBarBytes;
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
  uint8_t* b_smem = smem + kFtABytes;            // [stage][2 halves][128 rows][128 B]
  uint8_t* stg_smem = b_smem + kFtStages * kFtStageBytes;  // [slot][32 rows][128 FP32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_smem + kFtSlots * kFtStgBytes);
  uint64_t* full = bars;                         // [kFtStages]
  uint64_t* acc_full = bars + kFtStages;         // [kFtAccs]
  uint64_t* acc_empty = acc_full + kFtAccs;      // [kFtAccs]
  uint64_t* q_full = acc_empty + kFtAccs;
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
  uint64_t* stg_empty = stg_full + kFtSlots;                             // [slot]: read out
  // [slot][4]: operand stage (-1: stop), box, arrivals on the stage's full
  // barrier beyond one (the tile's boxes with no rows), tile index
  volatile int* stg_desc = reinterpret_cast<volatile int*>(stg_empty + kFtSlots);
  // tiles whose MMAs have completed, in order (written by the epilogue when it
  // sees a tile's accumulator full): a tile's operand stage is free for tile
  // + kFtStages once tiles_done > tile.  A counter rather than a parity wait:
  // the converters run an unbounded number of tiles ahead of the MMA.
  volatile int* tiles_done = stg_desc + 4 * kFtSlots;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long n_units = (a.n_pairs + kFtPairsPerUnit - 1) / kFtPairsPerUnit;
  if (blockIdx.x >= n_units) return;

  if (threadIdx.x == 0) {
    // full[s]: one arrival per 32-row box of the tile, all from converters (the
    // converter of a tile's last box also arrives for the boxes past the set's
    // end)
    for (int s = 0; s < kFtStages; ++s) mbar_init(&full[s], kFtBoxes);
    for (int c = 0; c < kFtSlots; ++c) { mbar_init(&stg_full[c], 1); mbar_init(&stg_empty[c], 1); }
    for (int i = 0; i < kFtAccs; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kFtEpiWarps);
    }
    for (int i = 0; i < 2; ++i) {
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
    *tiles_done = 0;
    fence_barrier_init();
  }
  if (warp == kFtEpiWarps + 1) tmem_alloc(tmem_slot, kFtTmemCols);
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
    uint64_t n_tile = 0;  // tiles issued (tile n goes to operand stage n % kFtStages)
    uint64_t n_box = 0;   // FP32 boxes issued (box g: staging slot g % kFtSlots, converter g % kFtConvWarps)
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
            const int stage = (int)(n_tile % kFtStages);
            const int row0 = (int)(p.r0 + (int64_t)tile * kFtN);
            for (int bx = 0; bx < nb && okl; ++bx) {
              // the box's FP32 rows into the next staging slot; its converter
              // writes them, rounded, into this tile's stage
              const int sl = (int)(n_box % kFtSlots);
              const uint32_t use = (uint32_t)(n_box / kFtSlots);
              if (use > 0 && !mbar_wait(&stg_empty[sl], (use - 1) & 1, a.status, abort_flag)) { okl = 0; break; }
              const int extra = bx == nb - 1 ? kFtBoxes - nb : 0;  // boxes with no rows
              stg_desc[4 * sl] = stage;
              stg_desc[4 * sl + 1] = bx;
              stg_desc[4 * sl + 2] = extra;
              stg_desc[4 * sl + 3] = (int)n_tile;
              mbar_arrive_expect_tx(&stg_full[sl], kFtStgBytes);
              tma_load_2d(stg_smem + sl * kFtStgBytes, &tm_d, &stg_full[sl], 0, row0 + bx * kFtBox);
              ++n_box;
            }
            ++n_tile;
          }
        }
        if (!__shfl_sync(0xffffffffu, okl, 0)) ok = false;
      }
    }
    if (lane == 0) {
      if (ok) {
        // stop every converter: a descriptor of -1 in the slot it reads next
        // (converter c's k-th box went to slot c + C (k % S), use k / S), once
        // that slot's previous box has been read out
        for (int c = 0; c < kFtConvWarps; ++c) {
          const uint64_t n_c = n_box / kFtConvWarps + ((uint64_t)c < n_box % kFtConvWarps ? 1 : 0);
          const int sl = c + kFtConvWarps * (int)(n_c % kFtSlotsPerConv);
          const uint64_t prev = n_c / kFtSlotsPerConv;
          if (prev > 0 && !mbar_wait(&stg_empty[sl], (uint32_t)((prev - 1) & 1), a.status, abort_flag)) break;
          stg_desc[4 * sl] = -1;
          mbar_arrive(&stg_full[sl]);
        }
      } else {
        // drain: every load this thread issued must land before the CTA exits
        for (int sl = 0; sl < kFtSlots; ++sl) {
          const uint64_t uses = n_box / kFtSlots + ((uint64_t)sl < n_box % kFtSlots ? 1 : 0);
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
            mma_commit(&acc_full[acc]);
            if (++stage == kFtStages) { stage = 0; phase ^= 1; }
            if (++acc == kFtAccs) { acc = 0; acc_phase ^= 1; }
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
    // converter c takes boxes c, c + C, ... (C converters; its k-th box in
    // staging slot c + C (k % S), S slots each): the 32 FP32 rows read and
    // rounded to bf16 (nearest even) in registers, the slot freed, then, once
    // the tile's operand stage is free, the rows stored at rows 32 box ..
    // 32 box + 31 of the stage, in the 128-byte
    // swizzle (16-byte chunk index XOR row % 8) the MMA descriptors expect
    const int c = warp - kFtConv0;
    const int h = lane >> 4;                 // component half of this lane's 4 floats
    const int cc = (lane & 15) >> 1;         // 16-byte chunk within the half
    for (uint32_t n = 0;; ++n) {
      const int sl = c + kFtConvWarps * (int)(n % kFtSlotsPerConv);
      const bool w = mbar_wait(&stg_full[sl], (n / kFtSlotsPerConv) & 1, a.status, abort_flag);
      if (!__all_sync(0xffffffffu, w)) break;
      const int st_i = stg_desc[4 * sl];
      const int bx = stg_desc[4 * sl + 1];
      const int extra = stg_desc[4 * sl + 2];
      const int tile = stg_desc[4 * sl + 3];
      if (st_i < 0) break;
      const float* stg = reinterpret_cast<const float*>(stg_smem + sl * kFtStgBytes);
      uint2 o[kFtBox];
#pragma unroll
      for (int r0 = 0; r0 < kFtBox; r0 += 8) {
        float4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = reinterpret_cast<const float4*>(stg + (r0 + u) * kDim)[lane];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          o[r0 + u].x = pack_bf16x2(x[u].x, x[u].y);   // two components per conversion
          o[r0 + u].y = pack_bf16x2(x[u].z, x[u].w);
        }
      }
      // every lane has consumed its reads of the slot (the rounded values are in
      // registers); the proxy fence orders those reads before the next TMA write
      // into the slot, which the producer issues once the slot is released
      fence_proxy_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&stg_empty[sl]);
      // the stage's previous tile (tile - kFtStages) must be consumed by its MMAs
      bool e = true;
      if (tile >= kFtStages) {
        const long long t0 = clock64();
        while (*tiles_done <= tile - kFtStages) {
          if (*abort_flag) { e = false; break; }
          if (clock64() - t0 > kWaitBudgetCycles) {
            set_status(a.status, kDevTimeout);
            *abort_flag = 1;
            e = false;
            break;
          }
        }
        __threadfence_block();
      }
      if (!__all_sync(0xffffffffu, e)) break;
      uint8_t* dst = b_smem + st_i * kFtStageBytes + h * (kFtN * 128) + (lane & 1) * 8;
#pragma unroll
      for (int r = 0; r < kFtBox; ++r) {
        const int R = bx * kFtBox + r;
        *reinterpret_cast<uint2*>(dst + R * 128 + ((cc ^ (R & 7)) << 4)) = o[r];
      }
      fence_proxy_async_shared();   // the writes, visible to the tensor cores
      __syncwarp();
      if (lane == 0) {
        // this box, and for a tile's last box the boxes past the set's end
        for (int k = 0; k <= extra; ++k) mbar_arrive(&full[st_i]);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const uint32_t t_lane = (uint32_t)(warp * 32) << 16;
    const int row = warp * 32 + lane;  // query row within the block
    int acc = 0;
    uint32_t acc_phase = 0;
    int n_tiles_seen = 0;
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
          // the tile's MMAs are complete, so its operand stage may be refilled
          if (warp == 0 && lane == 0) {
            __threadfence_block();  // the completion seen above, ordered before the count
            *tiles_done = ++n_tiles_seen;
          }
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
          if (++acc == kFtAccs) { acc = 0; acc_phase ^= 1; }
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
    tmem_dealloc(tmem, kFtTmemCols);
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
