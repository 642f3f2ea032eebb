// Nearest-centroid codes NN(x) = argmax_c <x, C_c> (Sec. 4.1.1, Sec. 4.2.2) of
// many rows on the sm_103a tensor cores, with the same answer as the FP32 SIMT
// assignment (one fused multiply-add chain over k = 0 .. 127 per dot, ties to
// the lowest index).
//
// 1. Split.  Every FP32 component becomes hi = bf16(x) and lo = bf16(x - hi)
//    (x - hi is exact in FP32), for the rows and for the centroids.  The three
//    products hi.hi + lo.hi + hi.lo, accumulated in FP32 by tcgen05.mma, give
//    every <x, C_c> within
//      E_b = (3.01 * 2^-18 + 384 * 2^-23) * |x| |C_c|
//    of its exact value (the dropped lo.lo term and the residues of the split,
//    and 384 accumulations even if each truncates), while the FP32 chain of the
//    SIMT assignment is within E_f = 128 * 2^-24 * |x| |C_c|.
// 2. Candidates.  The epilogue keeps, per row, the running maximum m of the
//    tensor-core values over the k1 centroids and every centroid whose value
//    was within band of m when it was seen (band = 2 (E_b + E_f) |x| max_c
//    |C_c|, with 1% slack), evicting those that fall below m - band, at most
//    K = 6 at a time.  The FP32 winner c* scores at least m_final - band on the
//    tensor cores, and m only grows, so c* is always kept.
// 3. Recheck.  The kept candidates are rescored with the SIMT assignment's
//    exact FP32 chain and the best one (ties to the lower index) is the code:
//    the same code and best value as the SIMT kernel.  A row whose list
//    overflowed (more than K near-ties), or with a zero, infinite or NaN value or
//    norm, is listed and assigned afterwards by the SIMT kernel itself.
//
// Kernel layout: a persistent CTA per SM takes units of 256 rows (two M tiles)
// from a global counter; the A operands (hi and lo) of a unit sit in shared
// memory; the centroid tiles (128 centroids, hi then lo) stream through a ring
// of three shared-memory stages filled by TMA, so all CTAs read the same
// centroid tiles from L2.  Two MMA warps (one per M tile) issue 24 MMAs per
// tile into a double-buffered TMEM accumulator; eight epilogue warps, one
// thread per row, fold each 128-column tile into the row's candidate list.
#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kAtMT = 2;                      // M tiles per unit
constexpr int kAtRows = 128 * kAtMT;          // rows per unit
constexpr int kAtN = 128;                     // centroids per tile
constexpr int kAtStages = 3;                  // ring stages (one operand of a tile each)
constexpr int kAtK = 6;                       // candidates per row
constexpr int kAtEpiWarps = 4 * kAtMT;
constexpr int kAtNMW = kAtMT;                 // one MMA warp per M tile
constexpr int kAtThreads = (kAtEpiWarps + 1 + kAtNMW) * 32;
constexpr int kAtOpBytes = kAtRows * kDim * 2;   // one A operand of a unit (64 KB)
constexpr int kAtStageBytes = kAtN * kDim * 2;   // one operand of a centroid tile (32 KB)
constexpr int kAtUnitRing = 2;
constexpr int kAtNBars = 2 * kAtStages + 4 * kAtNMW + 2 + kAtNMW + 2 * kAtUnitRing;
constexpr int kAtBarBytes = (kAtNBars * 8 + 16 + 4 * kAtUnitRing + 127) / 128 * 128;
constexpr int kAtSmem = 1024 + 2 * kAtOpBytes + kAtStages * kAtStageBytes + kAtBarBytes;
static_assert(kAtSmem <= 232448, "shared memory over the per-block limit");
constexpr int kAtAccCols = kAtMT * kAtN;      // per accumulator buffer
constexpr int kAtTmemCols = 2 * kAtAccCols;
static_assert(kAtTmemCols <= 512, "TMEM over-committed");
constexpr uint32_t kAtIdesc = make_idesc(128, kAtN, 1u, 1u);
constexpr int kAtCh = 64;                     // accumulator columns per TMEM load
// 2 (E_b + E_f) per unit |x| |C|, with 1% slack for the FP32 norms
constexpr float kAtBand =
    2.0f * (3.01f / 262144.f + 384.f / 8388608.f + 128.f / 16777216.f) * 1.01f;

struct AtArgs {
  const float* X;          // FP32 rows of this launch [n_rows x 128]
  const float* C;          // FP32 centroids [k1 x 128]
  int64_t n_rows;          // rows of this launch (an upper bound when n_dev is set)
  const int64_t* n_dev;    // rows of the whole call, read on the device, or null
  int k1;
  const float* cmax;       // largest centroid norm (device scalar)
  int32_t* codes;          // [n_rows] of this launch
  float* best;             // [n_rows] or null
  int64_t row_base;        // index of this launch's first row in the whole call
  int32_t* fb_rows;        // rows left to the SIMT assignment (whole-call indices)
  unsigned long long* fb_count;
  int* status;
  int* unit_counter;
};

__device__ __forceinline__ bool better(float v, int i, float bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

__global__ void __launch_bounds__(kAtThreads, 1)
assign_tc_kernel(const __grid_constant__ CUtensorMap tm_xh, const __grid_constant__ CUtensorMap tm_xl,
                 const __grid_constant__ CUtensorMap tm_ch, const __grid_constant__ CUtensorMap tm_cl, AtArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a_hi = smem;                        // [MT][2 halves][128 rows][128 B]
  uint8_t* a_lo = smem + kAtOpBytes;
  uint8_t* b_smem = smem + 2 * kAtOpBytes;     // [stage][2 halves][N rows][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_smem + kAtStages * kAtStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kAtStages;
  uint64_t* acc_full = bars + 2 * kAtStages;   // [2 buffers][NMW]
  uint64_t* acc_empty = acc_full + 2 * kAtNMW;
  uint64_t* q_full = acc_empty + 2 * kAtNMW;
  uint64_t* q_empty = q_full + 1;
  uint64_t* done_bar = q_empty + 1;            // [NMW]
  uint64_t* unit_full = done_bar + kAtNMW;     // [UNIT_RING]
  uint64_t* unit_empty = unit_full + kAtUnitRing;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(unit_empty + kAtUnitRing);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* unit_ring = abort_flag + 1;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t n_rows =
      a.n_dev ? max((int64_t)0, min(a.n_rows, (int64_t)__ldg(a.n_dev) - a.row_base)) : a.n_rows;
  const long long n_units = (n_rows + kAtRows - 1) / kAtRows;
  const int n_tiles = (a.k1 + kAtN - 1) / kAtN;
  if (blockIdx.x >= n_units) return;  // uniform for the CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAtStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kAtNMW); }
    for (int i = 0; i < 2 * kAtNMW; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 4); }
    mbar_init(q_full, 1);
    mbar_init(q_empty, kAtNMW);
    for (int w = 0; w < kAtNMW; ++w) mbar_init(&done_bar[w], 1);
    for (int i = 0; i < kAtUnitRing; ++i) {
      mbar_init(&unit_full[i], 1);
      mbar_init(&unit_empty[i], kAtNMW + kAtEpiWarps);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kAtEpiWarps + 1) tmem_alloc(tmem_slot, kAtTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kAtEpiWarps) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      tma_prefetch_desc(&tm_xh);
      tma_prefetch_desc(&tm_xl);
      tma_prefetch_desc(&tm_ch);
      tma_prefetch_desc(&tm_cl);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued[kAtStages] = {};
      uint32_t q_issued = 0;
      bool ok = true;
      int uslot = 0;
      uint32_t uphase = 0;
      int it = 0;
      auto draw_unit = [&]() -> long long {
        const long long u = atomicAdd(a.unit_counter, 1);
        if (!mbar_wait(&unit_empty[uslot], uphase ^ 1, a.status, abort_flag)) {
          ok = false;
          return n_units;
        }
        unit_ring[uslot] = (int)(u < n_units ? u : n_units);
        mbar_arrive(&unit_full[uslot]);
        if (++uslot == kAtUnitRing) { uslot = 0; uphase ^= 1; }
        return u;
      };
      for (long long u = draw_unit(); u < n_units && ok; u = draw_unit(), ++it) {
        if (it > 0 && !mbar_wait(q_empty, (it - 1) & 1, a.status, abort_flag)) { ok = false; break; }
        mbar_arrive_expect_tx(q_full, 2 * kAtOpBytes);
        ++q_issued;
        for (int m = 0; m < kAtMT; ++m)
          for (int h = 0; h < 2; ++h) {
            const int row = (int)(u * kAtRows + m * 128);
            tma_load_2d(a_hi + (m * 2 + h) * 16384, &tm_xh, q_full, h * 64, row);
            tma_load_2d(a_lo + (m * 2 + h) * 16384, &tm_xl, q_full, h * 64, row);
          }
        for (int t = 0; t < n_tiles && ok; ++t) {
          for (int op = 0; op < 2; ++op) {  // hi, then lo
            if (!mbar_wait(&empty[stage], phase ^ 1, a.status, abort_flag)) { ok = false; break; }
            uint8_t* dst = b_smem + stage * kAtStageBytes;
            mbar_arrive_expect_tx(&full[stage], kAtStageBytes);
            for (int h = 0; h < 2; ++h)
              tma_load_2d(dst + h * (kAtN * 128), op ? &tm_cl : &tm_ch, &full[stage], h * 64, t * kAtN);
            issued[stage]++;
            if (++stage == kAtStages) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (!ok) {
        // drain: every load this thread issued must land before the CTA exits
        for (int s = 0; s < kAtStages; ++s)
          if (issued[s]) { int z = 0; mbar_wait(&full[s], (issued[s] - 1) & 1, nullptr, &z); }
        int z = 0;
        if (q_issued) mbar_wait(q_full, (q_issued - 1) & 1, nullptr, &z);
      }
    }
  } else if (warp > kAtEpiWarps) {
    // ------------------------------------------------------------------ MMA issuers
    const int mw = warp - kAtEpiWarps - 1;  // this warp's M tile
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      int it = 0;
      bool ok = true;
      int uslot = 0;
      uint32_t uphase = 0;
      auto take_unit = [&]() -> long long {
        if (!mbar_wait(&unit_full[uslot], uphase, a.status, abort_flag)) {
          ok = false;
          return n_units;
        }
        const long long u = unit_ring[uslot];
        mbar_arrive(&unit_empty[uslot]);
        if (++uslot == kAtUnitRing) { uslot = 0; uphase ^= 1; }
        return u;
      };
      for (long long u = take_unit(); u < n_units && ok; u = take_unit(), ++it) {
        if (!mbar_wait(q_full, it & 1, a.status, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint64_t ah0 = sw128_desc(smem_u32(a_hi + mw * 2 * 16384));
        const uint64_t al0 = sw128_desc(smem_u32(a_lo + mw * 2 * 16384));
        for (int t = 0; t < n_tiles; ++t) {
          if (!mbar_wait(&acc_empty[acc * kAtNMW + mw], acc_phase ^ 1, a.status, abort_flag)) { ok = false; break; }
          const uint32_t dt = tmem + acc * kAtAccCols + mw * kAtN;
          for (int op = 0; op < 2 && ok; ++op) {
            if (!mbar_wait(&full[stage], phase, a.status, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint64_t bd0 = sw128_desc(smem_u32(b_smem + stage * kAtStageBytes));
#pragma unroll
            for (int k = 0; k < kDim / 16; ++k) {
              const int half = (k * 32) / 128;
              const int within = (k * 32) % 128;
              const uint64_t bd = bd0 + (uint64_t)((half * (kAtN * 128) + within) >> 4);
              const uint64_t off = (uint64_t)((half * 16384 + within) >> 4);
              if (op == 0) {
                mma_bf16(dt, ah0 + off, bd, kAtIdesc, k > 0);  // hi . hi
                mma_bf16(dt, al0 + off, bd, kAtIdesc, 1);      // lo . hi
              } else {
                mma_bf16(dt, ah0 + off, bd, kAtIdesc, 1);      // hi . lo
              }
            }
            mma_commit(&empty[stage]);
            if (++stage == kAtStages) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&acc_full[acc * kAtNMW + mw]);
          if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
        if (ok) mma_commit(q_empty);
      }
      // all MMAs of this thread complete before the CTA releases TMEM
      mma_commit(&done_bar[mw]);
      int z = 0;
      mbar_wait(&done_bar[mw], 0, nullptr, &z);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int m_tile = warp >> 2;
    const int quad = warp & 3;  // the TMEM lane quarter this warp may read
    const int local_row = m_tile * 128 + quad * 32 + lane;
    const uint32_t t_lane = (uint32_t)(quad * 32) << 16;
    const float cmax = *a.cmax;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    int uslot = 0;
    uint32_t uphase = 0;
    auto take_unit = [&]() -> long long {
      const bool w = mbar_wait(&unit_full[uslot], uphase, a.status, abort_flag);
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        return n_units;
      }
      const long long u = unit_ring[uslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&unit_empty[uslot]);
      if (++uslot == kAtUnitRing) { uslot = 0; uphase ^= 1; }
      return u;
    };
    for (long long u = take_unit(); u < n_units && ok; u = take_unit()) {
      const int64_t row = u * kAtRows + local_row;
      const bool live = row < n_rows;
      // the row's norm (its band) from the FP32 row; the same FMA chain as the recheck
      float ss = 0.f;
      if (live) {
        const float4* xr = reinterpret_cast<const float4*>(a.X + row * kDim);
#pragma unroll 8
        for (int k4 = 0; k4 < kDim / 4; ++k4) {
          const float4 x = __ldg(xr + k4);
          ss = __fmaf_rn(x.x, x.x, ss);
          ss = __fmaf_rn(x.y, x.y, ss);
          ss = __fmaf_rn(x.z, x.z, ss);
          ss = __fmaf_rn(x.w, x.w, ss);
        }
      }
      const float band = kAtBand * sqrtf(ss) * cmax;
      // Running maximum m of the tensor-core values, and every column seen so
      // far whose value was within `band` of the maximum at the time: a column
      // within band of the final maximum is always among them (the maximum only
      // grows), and an entry that falls below max - band is evicted.  More than
      // kAtK such columns at once overflows the list: the row then goes to the
      // SIMT assignment.
      float m = -INFINITY, thr = -INFINITY;
      float lv[kAtK];
      int li[kAtK];
      int n_l = 0;
      bool overflow = false;
#pragma unroll
      for (int i = 0; i < kAtK; ++i) { lv[i] = -INFINITY; li[i] = -1; }
      for (int t = 0; t < n_tiles; ++t) {
        const bool got = mbar_wait(&acc_full[acc * kAtNMW + m_tile], acc_phase, a.status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tcol = tmem + t_lane + acc * kAtAccCols + m_tile * kAtN;
        const int valid = a.k1 - t * kAtN;  // columns of real centroids in this tile
#pragma unroll 1
        for (int c = 0; c < kAtN / 32; ++c) {
          float v[32];
          tmem_ld32(tcol + c * 32, v);
          if (c == kAtN / 32 - 1) {
            // the accumulator is in registers: hand the buffer back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc * kAtNMW + m_tile]);
          }
          if (valid < kAtN) {  // last tile: columns past k1 hold zero-filled rows
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (c * 32 + j >= valid) v[j] = -INFINITY;
          }
          // two-input maxima ignore NaN (a NaN centroid's column never counts)
          float cm[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) cm[j] = fmaxf(v[2 * j], v[2 * j + 1]);
#pragma unroll
          for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
            for (int j = 0; j < w; ++j) cm[j] = fmaxf(cm[j], cm[j + w]);
          // rare: the chunk holds a new maximum or a value within band of it.  A
          // row past the end (zero-filled: every column would tie) and a row
          // whose list has overflowed (it goes to the SIMT assignment) track nothing.
          if (live && !overflow && cm[0] >= thr) {
            uint32_t hits = 0;
            float tmp[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              tmp[j] = v[j];
              hits |= (v[j] >= thr) ? (1u << j) : 0u;
            }
#pragma unroll 1
            while (hits) {
              const int j = __ffs(hits) - 1;
              hits &= hits - 1;
              const float x = tmp[j];
              if (!(x >= thr)) continue;        // the threshold rose within this chunk
              if (x > m) {
                m = x;
                thr = m - band;
              }
              if (n_l == kAtK) {                // full: drop entries now below the band
                int k = 0;
#pragma unroll 1
                for (int e = 0; e < kAtK; ++e)
                  if (lv[e] >= thr) { lv[k] = lv[e]; li[k] = li[e]; ++k; }
                n_l = k;
              }
              if (n_l < kAtK) {
                lv[n_l] = x;
                li[n_l] = t * kAtN + c * 32 + j;
                ++n_l;
              } else {
                overflow = true;
              }
            }
          }
        }
        if (++acc == 2) { acc = 0; acc_phase ^= 1; }
      }
      if (!ok) break;
      if (!live) continue;
      // recheck the candidates within band of the final maximum with the SIMT
      // assignment's FP32 chain
      bool complete = !overflow && m == m && band == band && band < INFINITY && m > -INFINITY;
      int cidx[kAtK];
#pragma unroll
      for (int e = 0; e < kAtK; ++e) cidx[e] = (e < n_l && lv[e] >= thr) ? li[e] : -1;
      if (complete) {
        const float4* xr = reinterpret_cast<const float4*>(a.X + row * kDim);
        const float4* cr = reinterpret_cast<const float4*>(a.C);
        float dot[kAtK];
#pragma unroll
        for (int e = 0; e < kAtK; ++e) dot[e] = 0.f;
#pragma unroll 4
        for (int k4 = 0; k4 < kDim / 4; ++k4) {
          const float4 x = __ldg(xr + k4);
#pragma unroll
          for (int e = 0; e < kAtK; ++e) {
            const float4 c = __ldg(cr + (int64_t)(cidx[e] < 0 ? 0 : cidx[e]) * (kDim / 4) + k4);
            dot[e] = __fmaf_rn(x.x, c.x, dot[e]);
            dot[e] = __fmaf_rn(x.y, c.y, dot[e]);
            dot[e] = __fmaf_rn(x.z, c.z, dot[e]);
            dot[e] = __fmaf_rn(x.w, c.w, dot[e]);
          }
        }
        float bv = -INFINITY;
        int bi = 0x7fffffff;
#pragma unroll
        for (int e = 0; e < kAtK; ++e)
          if (cidx[e] >= 0 && better(dot[e], cidx[e], bv, bi)) { bv = dot[e]; bi = cidx[e]; }
        if (bi == 0x7fffffff) {
          complete = false;
        } else {
          a.codes[row] = bi;
          if (a.best) a.best[row] = bv;
        }
      }
      if (!complete) {
        const unsigned long long slot = atomicAdd(a.fb_count, 1ull);
        a.fb_rows[slot] = (int32_t)(a.row_base + row);
      }
    }
  }

  __syncthreads();
  if (warp == kAtEpiWarps + 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kAtTmemCols);
  }
}

// hi = bf16(x), lo = bf16(x - hi) for n rows of 128; norm_max != nullptr: the
// largest row norm (non-finite rows skipped) by an integer max of its bits
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t n, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, float* __restrict__ norm_max) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float4 x = reinterpret_cast<const float4*>(X + r * kDim)[lane];
    const float xs[4] = {x.x, x.y, x.z, x.w};
    __nv_bfloat16 h[4], l[4];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = __float2bfloat16_rn(xs[i]);
      l[i] = __float2bfloat16_rn(xs[i] - __bfloat162float(h[i]));
      ss = __fmaf_rn(xs[i], xs[i], ss);
    }
    uint2 hp, lp;
    hp.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
    hp.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
    lp.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
    lp.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
    reinterpret_cast<uint2*>(hi + r * kDim)[lane] = hp;
    reinterpret_cast<uint2*>(lo + r * kDim)[lane] = lp;
    if (norm_max) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float nrm = sqrtf(ss) * 1.0001f;
      if (lane == 0 && isfinite(nrm)) atomicMax(reinterpret_cast<int*>(norm_max), __float_as_int(nrm));
    }
  }
}

}  // namespace

namespace {

struct AtScratch {
  __nv_bfloat16 *c_hi, *c_lo, *x_hi, *x_lo;
  int32_t* fb_rows;
  unsigned long long* fb_count;
  float* cmax;
  int* unit_counter;
  int* status;
};

size_t at_up(size_t b) { return (b + 255) / 256 * 256; }
int64_t at_chunk(int64_t max_n) { return std::min<int64_t>(max_n, (int64_t)1 << 22); }

// One block: C hi/lo, X hi/lo of a chunk, the fallback list, the counters and
// the centroid-norm maximum.
AtScratch at_carve(void* scratch, int64_t max_n, int k1) {
  uint8_t* base = static_cast<uint8_t*>(scratch);
  const size_t c_op = at_up((size_t)k1 * kDim * 2), x_op = at_up((size_t)at_chunk(max_n) * kDim * 2),
               fb = at_up((size_t)max_n * 4);
  AtScratch sc;
  sc.c_hi = reinterpret_cast<__nv_bfloat16*>(base);
  sc.c_lo = reinterpret_cast<__nv_bfloat16*>(base + c_op);
  sc.x_hi = reinterpret_cast<__nv_bfloat16*>(base + 2 * c_op);
  sc.x_lo = reinterpret_cast<__nv_bfloat16*>(base + 2 * c_op + x_op);
  sc.fb_rows = reinterpret_cast<int32_t*>(base + 2 * c_op + 2 * x_op);
  uint8_t* small = base + 2 * c_op + 2 * x_op + fb;
  sc.fb_count = reinterpret_cast<unsigned long long*>(small);
  sc.cmax = reinterpret_cast<float*>(small + 8);
  sc.unit_counter = reinterpret_cast<int*>(small + 12);
  sc.status = reinterpret_cast<int*>(small + 16);
  return sc;
}

}  // namespace

size_t assign_tc_scratch_bytes(int64_t max_n, int k1) {
  return 2 * at_up((size_t)k1 * kDim * 2) + 2 * at_up((size_t)at_chunk(max_n) * kDim * 2) +
         at_up((size_t)max_n * 4) + 256;
}

cudaError_t assign_tc_prepare() {
  static bool attr_set = false;
  if (attr_set) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(assign_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAtSmem);
  if (e == cudaSuccess) attr_set = true;
  return e;
}

gem_status enqueue_assign_tc(const float* X, int64_t max_n, const int64_t* n_dev, const float* C, int k1,
                             int32_t* codes, float* best, void* scratch, int* status, int n_sm, cudaStream_t st) {
  if (max_n == 0) return GEM_OK;
  if (max_n >= ((int64_t)1 << 31)) return fail(GEM_ERR_INVALID, "too many rows");
  const int64_t chunk = at_chunk(max_n);
  const AtScratch sc = at_carve(scratch, max_n, k1);
  if (!status) status = sc.status;
  CUtensorMap tm_ch, tm_cl, tm_xh, tm_xl;
  if (!encode_tmap_2d(&tm_ch, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, sc.c_hi, kDim, (uint64_t)k1, kDim * 2, 64, kAtN,
                      CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tm_cl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, sc.c_lo, kDim, (uint64_t)k1, kDim * 2, 64, kAtN,
                      CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tm_xh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, sc.x_hi, kDim, (uint64_t)chunk, kDim * 2, 64, 128,
                      CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&tm_xl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, sc.x_lo, kDim, (uint64_t)chunk, kDim * 2, 64, 128,
                      CU_TENSOR_MAP_SWIZZLE_128B))
    return fail(GEM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the assignment operands");
  GEM_CUDA_TRY(assign_tc_prepare());
  // fallback count, centroid-norm maximum, unit counter and own status start at zero
  GEM_CUDA_TRY(cudaMemsetAsync(sc.fb_count, 0, 256, st));
  // every code is a valid index even if a bounded wait gives up mid-way
  GEM_CUDA_TRY(cudaMemsetAsync(codes, 0, sizeof(int32_t) * max_n, st));
  const int split_grid = (int)std::min<int64_t>(((int64_t)k1 * 32 + 255) / 256, (int64_t)n_sm * 16);
  split_bf16_kernel<<<split_grid, 256, 0, st>>>(C, k1, sc.c_hi, sc.c_lo, sc.cmax);
  int launches = 1;
  for (int64_t r0 = 0; r0 < max_n; r0 += chunk) {
    const int64_t nr = std::min(chunk, max_n - r0);
    const int g = (int)std::min<int64_t>((nr * 32 + 255) / 256, (int64_t)n_sm * 16);
    split_bf16_kernel<<<g, 256, 0, st>>>(X + r0 * kDim, nr, sc.x_hi, sc.x_lo, nullptr);
    GEM_CUDA_TRY(cudaMemsetAsync(sc.unit_counter, 0, sizeof(int), st));
    AtArgs aa;
    aa.X = X + r0 * kDim;
    aa.C = C;
    aa.n_rows = nr;
    aa.n_dev = n_dev;
    aa.k1 = k1;
    aa.cmax = sc.cmax;
    aa.codes = codes + r0;
    aa.best = best ? best + r0 : nullptr;
    aa.row_base = r0;
    aa.fb_rows = sc.fb_rows;
    aa.fb_count = sc.fb_count;
    aa.status = status;
    aa.unit_counter = sc.unit_counter;
    const int64_t units = (nr + kAtRows - 1) / kAtRows;
    assign_tc_kernel<<<(unsigned)std::min<int64_t>(units, n_sm), kAtThreads, kAtSmem, st>>>(tm_xh, tm_xl, tm_ch,
                                                                                           tm_cl, aa);
    launches += 2;
  }
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(launches);
  // the rows the candidates could not decide: the SIMT assignment itself
  return launch_assign_rows(X, max_n, reinterpret_cast<const int64_t*>(sc.fb_count), sc.fb_rows, C, k1, codes, best,
                            n_sm, st);
}

gem_status launch_assign_tc(const float* X, int64_t n, const float* C, int k1, int32_t* codes, float* best,
                            int n_sm, cudaStream_t st) {
  if (n == 0) return GEM_OK;
  if (n >= ((int64_t)1 << 31)) return fail(GEM_ERR_INVALID, "too many rows");
  void* base = nullptr;
  cudaError_t e = cudaMallocAsync(&base, assign_tc_scratch_bytes(n, k1), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GEM_ERR_OOM, "scratch of the tensor-core assignment");
  }
  const gem_status r = enqueue_assign_tc(X, n, nullptr, C, k1, codes, best, base, nullptr, n_sm, st);
  // a bounded wait that gave up is reported here (the call blocks)
  int h_status = 0;
  e = r == GEM_OK ? cudaMemcpyAsync(&h_status, at_carve(base, n, k1).status, sizeof(int), cudaMemcpyDeviceToHost, st)
                  : cudaSuccess;
  cudaFreeAsync(base, st);
  if (r != GEM_OK) return r;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core assignment");
  if (h_status != 0) return fail((gem_status)h_status, "a wait of the tensor-core assignment gave up");
  return GEM_OK;
}

}  // namespace gem
