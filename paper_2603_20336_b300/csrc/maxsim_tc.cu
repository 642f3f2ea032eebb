// Exact MaxSim over every stored set on the sm_103a tensor cores (tcgen05).
//
// CH(Q, P) = sum_i max_j <q_i, p_j>  (Sec. 3.1, Definition 1, Eq. 1) for all
// query parts of one pass of the plan against every set of the store.
//
// Work unit = (query block of M_RES = 128 * MT packed rows, document chunk).
// A persistent CTA per SM walks units chunk-major, so the CTAs running at any
// moment share a few chunks and the document tiles they stream are L2 hits
// after the first reader.
//
// Roles inside a CTA (warp specialisation):
//   warps 0 .. 4*MT-1  epilogue: warp w reads TMEM lanes 32*(w%4).. of M tile
//                      w/4; one thread owns one packed query row
//   warp 4*MT          TMA producer: query block once per unit, then the
//                      chunk's document tiles (N rows x 128) through a
//                      STAGES-deep shared-memory ring
//   warp 4*MT+1 (..)   MMA issuer(s): per tile, MT x (K/16) tcgen05.mma into a
//                      double-buffered TMEM accumulator (2 x MT x N columns);
//                      with MT >= 2 two issuers on alternate M tiles
//
// Epilogue: every thread walks its row's N accumulator columns in order.  The
// low-precision store copies pad each set to a multiple of 8 rows with copies of
// the set's own last vector (a repeated vector cannot change a maximum), so sets
// end only at 8-column subgroup boundaries.  Per subgroup the thread folds 8
// columns into a running max with three-input max instructions; when a set ends
// (a warp-uniform bit) the rows of each query slot are summed (a 32-row slot
// whose row maxima are all below 2 in magnitude: one integer warp reduction in
// fixed point; otherwise a g-lane xor butterfly, g = slot size) and one lane
// writes the score.  A set never spans two chunks, so no partial maximum leaves
// registers and no similarity matrix is written anywhere.
#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

// AT: the query block (operand A) lives in tensor memory, written by the
// epilogue warps once per unit, so the MMAs read only the document tile from
// shared memory; the tile narrows so that accumulators and A share the 512
// TMEM columns (bf16 MT=2: 2 x 2 x 96 + 2 x 64; e4m3 MT=2: 2 x 2 x 96 + 2 x 32).
// E: sets of 4 * MT epilogue warps; set e takes the tiles t with t % E == e of
// every unit (E = 2: each set owns one accumulator buffer), so more warps hide
// the epilogue's latencies; the running max of a set that crosses a tile
// boundary passes from set to set through shared memory.
// SS (with FP8): the stored sets carry one power-of-two scale each (the
// per-set-scale copy): no per-column scale ring, the set's scale multiplies the
// row maxima once at the set's end.
template <int MT, bool FP8, bool AT = false, int E = 1, bool SS = false>
struct TcCfg {
  static constexpr int M_RES = 128 * MT;
  static constexpr int A_COLS = AT ? (FP8 ? 32 : 64) : 0;  // TMEM columns of A per M tile
  // tile width: with A resident, 96 columns (a multiple of 32, so every TMEM
  // access starts on a 32-column boundary)
  static constexpr int N = AT ? 96 : 256 / MT;  // columns per tile
  static_assert(!AT || MT == 2, "A in tensor memory is laid out for two M tiles");
  static_assert(E == 1 || (E == 2 && !AT), "two epilogue sets only with A in shared memory");
  static constexpr int ROW_BYTES = FP8 ? 128 : 256;
  static constexpr int HALVES = FP8 ? 1 : 2;      // 128-byte swizzle atoms per row
  static constexpr int K_STEP = FP8 ? 32 : 16;    // K per MMA instruction
  static constexpr int K_STEPS = kDim / K_STEP;   // MMAs per tile and M tile
  static constexpr int Q_BYTES = AT ? 0 : M_RES * ROW_BYTES;
  static constexpr int STAGE_BYTES = N * ROW_BYTES;
  static constexpr int STAGES = AT ? (FP8 ? 12 : 8)
                                   : (MT == 1) ? (FP8 ? 6 : 3) : (MT == 2 ? (FP8 ? 8 : 4) : (FP8 ? 12 : 6));
  // fp8: per-column dequantisation scales of each tile, in a ring of their own
  // (the operand stage is recycled as soon as the MMA has read it)
  static constexpr int SC_SLOTS = (FP8 && !SS) ? 8 : 0;
  static constexpr int SC_BYTES = SC_SLOTS * N * 4;
  static constexpr int EPI_SET = 4 * MT;          // epilogue warps per set
  static constexpr int EPI_WARPS = E * EPI_SET;
  // MMA issuer warps: with two or more M tiles, two issuers (on different SM
  // sub-partitions) take alternate M tiles, each with its own accumulator barriers
  static constexpr int NMW = (MT >= 2 && !AT) ? 2 : 1;
  static constexpr int THREADS = (EPI_WARPS + 1 + NMW) * 32;
  // accumulator columns per TMEM load (more than 12 warps leave at most 96
  // registers a thread, so 32 columns at a time)
  static constexpr int CH = EPI_WARPS + 1 + NMW > 12 ? 32 : (E > 1 ? 64 : (N < 128 ? N : 128));
  static constexpr int CARRY_BYTES = E > 1 ? E * EPI_SET * 32 * 4 : 0;
  static constexpr int BASE_BYTES = 1024 /*align slack*/ + Q_BYTES + STAGES * STAGE_BYTES + SC_BYTES + CARRY_BYTES;
  static constexpr int UNIT_RING = 2;  // units drawn ahead by the producer
  static constexpr int N_BARS =
      2 * STAGES + 4 * NMW + 2 + NMW + 2 * SC_SLOTS + (E > 1 ? 2 * E * EPI_SET : 0) + 2 * UNIT_RING;
  static constexpr int BAR_BYTES = (N_BARS * 8 + 16 + 4 * UNIT_RING + 127) / 128 * 128;
  static constexpr int ACC_COLS = MT * N;         // per accumulator buffer
  static constexpr int A_BASE = 2 * ACC_COLS;     // first TMEM column of A (AT)
  static constexpr int TMEM_COLS = 512;
  static_assert(A_BASE + MT * A_COLS <= TMEM_COLS, "TMEM over-committed");
  static constexpr int SMEM_BYTES = BASE_BYTES + BAR_BYTES;
  static_assert(SMEM_BYTES <= 232448, "shared memory over the per-block limit");
  static constexpr uint32_t IDESC = make_idesc(128, N, FP8 ? 0u : 1u, FP8 ? 0u : 1u);
};

struct TcArgs {
  const int* hdr;
  const int* row_part;
  const int* part_query;
  const int* part_g;
  const int* part_pass;
  const float* q_scale;      // fp8 only: per packed row
  const uint32_t* qpack;     // AT: packed query rows as 32-bit words
  const int64_t* doc_off;    // padded row offsets [n_sets + 1]
  const uint32_t* end_bits;  // set-end bitmap over 8-row subgroups
  const int* chunk_doc;      // [n_chunks + 1]
  int n_chunks;
  int pass;
  int64_t n_sets;
  float* scores;             // [n_queries * n_sets]
  const float* set_scale;    // SS: [n_sets]
  int* status;
  int* unit_counter;         // next unit to hand out (zeroed before every launch)
};

// o[s] for a warp-uniform s < L, by a tree of selects on the bits of s (the
// array stays in registers).
template <int L>
__device__ __forceinline__ float pick(const float (&o)[L], int s) {
  constexpr int P = L <= 2 ? 2 : (L <= 4 ? 4 : (L <= 8 ? 8 : (L <= 16 ? 16 : 32)));
  static_assert(L <= 32, "at most 32 subgroups per tile");
  float a[P];
#pragma unroll
  for (int i = 0; i < P; ++i) a[i] = i < L ? o[i] : o[0];
#pragma unroll
  for (int w = P / 2, b = 0; w >= 1; w /= 2, ++b) {
    const bool hi = (s >> b) & 1;
#pragma unroll
    for (int i = 0; i < w; ++i) a[i] = hi ? a[2 * i + 1] : a[2 * i];
  }
  return a[0];
}

template <int MT, bool FP8, bool AT, int E, bool SS>
__global__ void __launch_bounds__(TcCfg<MT, FP8, AT, E, SS>::THREADS, 1)
tc_score_all_kernel(const __grid_constant__ CUtensorMap tm_q, const __grid_constant__ CUtensorMap tm_d,
                    const __grid_constant__ CUtensorMap tm_scale, TcArgs a) {
  using C = TcCfg<MT, FP8, AT, E, SS>;
  constexpr bool COL_SCALE = FP8 && !SS;  // a scale per stored vector (column)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* q_smem = smem;
  uint8_t* d_smem = smem + C::Q_BYTES;
  float* sc_smem = reinterpret_cast<float*>(d_smem + C::STAGES * C::STAGE_BYTES);
  float* carry_smem = reinterpret_cast<float*>(d_smem + C::STAGES * C::STAGE_BYTES + C::SC_BYTES);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(d_smem + C::STAGES * C::STAGE_BYTES + C::SC_BYTES + C::CARRY_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* acc_full = bars + 2 * C::STAGES;    // [2 buffers][NMW]
  uint64_t* acc_empty = acc_full + 2 * C::NMW;  // [2 buffers][NMW]
  uint64_t* q_full = acc_empty + 2 * C::NMW;
  uint64_t* q_empty = q_full + 1;
  uint64_t* done_bar = q_empty + 1;             // [NMW]
  uint64_t* sc_full = done_bar + C::NMW;
  uint64_t* sc_empty = sc_full + C::SC_SLOTS;
  uint64_t* carry_full = sc_empty + C::SC_SLOTS;                        // [E][EPI_SET] (E > 1)
  uint64_t* carry_empty = carry_full + (E > 1 ? E * C::EPI_SET : 0);   // [E][EPI_SET]
  uint64_t* unit_full = carry_empty + (E > 1 ? E * C::EPI_SET : 0);   // [UNIT_RING]
  uint64_t* unit_empty = unit_full + C::UNIT_RING;                     // [UNIT_RING]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(unit_empty + C::UNIT_RING);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* unit_ring = abort_flag + 1;                            // [UNIT_RING]

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int qb0 = a.hdr[kHdrQbBegin + a.pass];
  const int nqb = a.hdr[kHdrQbBegin + a.pass + 1] - qb0;
  const long long n_units = (long long)nqb * a.n_chunks;
  if (blockIdx.x >= n_units) return;  // uniform for the CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], C::NMW); }
    for (int i = 0; i < 2 * C::NMW; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], C::EPI_SET / C::NMW); }
    mbar_init(q_full, AT ? C::EPI_SET : 1);
    mbar_init(q_empty, C::NMW);
    for (int w = 0; w < C::NMW; ++w) mbar_init(&done_bar[w], 1);
    for (int s = 0; s < C::SC_SLOTS; ++s) { mbar_init(&sc_full[s], 1); mbar_init(&sc_empty[s], C::EPI_SET); }
    if constexpr (E > 1)
      for (int i = 0; i < E * C::EPI_SET; ++i) { mbar_init(&carry_full[i], 32); mbar_init(&carry_empty[i], 32); }
    for (int i = 0; i < C::UNIT_RING; ++i) {
      mbar_init(&unit_full[i], 1);
      mbar_init(&unit_empty[i], C::NMW + C::EPI_WARPS);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == C::EPI_WARPS + 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == C::EPI_WARPS) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      tma_prefetch_desc(&tm_q);
      tma_prefetch_desc(&tm_d);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued[C::STAGES];
      for (int s = 0; s < C::STAGES; ++s) issued[s] = 0;
      int sslot = 0;
      uint32_t sphase = 0;
      uint32_t sc_issued[C::SC_SLOTS > 0 ? C::SC_SLOTS : 1] = {};
      int it = 0;
      uint32_t q_issued = 0;
      bool ok = true;
      // Units are drawn in one global order from a counter, so all CTAs work
      // on the same few chunks (which then stay in L2), and handed to the MMA
      // and epilogue warps through a ring in shared memory.
      int uslot = 0;
      uint32_t uphase = 0;
      auto draw_unit = [&]() -> long long {
        const long long u = atomicAdd(a.unit_counter, 1);
        if (!mbar_wait(&unit_empty[uslot], uphase ^ 1, a.status, abort_flag)) {
          ok = false;
          return n_units;
        }
        unit_ring[uslot] = (int)(u < n_units ? u : n_units);
        mbar_arrive(&unit_full[uslot]);
        if (++uslot == C::UNIT_RING) { uslot = 0; uphase ^= 1; }
        return u;
      };
      for (long long u = draw_unit(); u < n_units && ok; u = draw_unit(), ++it) {
        const int chunk = (int)(u / nqb);
        const int qb = qb0 + (int)(u % nqb);
        if constexpr (!AT) {
          if (it > 0 && !mbar_wait(q_empty, (it - 1) & 1, a.status, abort_flag)) { ok = false; break; }
          mbar_arrive_expect_tx(q_full, C::Q_BYTES);
          ++q_issued;
          for (int m = 0; m < MT; ++m)
            for (int h = 0; h < C::HALVES; ++h)
              tma_load_2d(q_smem + (m * C::HALVES + h) * 16384, &tm_q, q_full, h * 64,
                          qb * C::M_RES + m * 128);
        } else {
          (void)qb;
        }
        const int64_t r0 = a.doc_off[a.chunk_doc[chunk]];
        const int64_t r1 = a.doc_off[a.chunk_doc[chunk + 1]];
        const int ntiles = (int)((r1 - r0 + C::N - 1) / C::N);
        for (int t = 0; t < ntiles; ++t) {
          if (!mbar_wait(&empty[stage], phase ^ 1, a.status, abort_flag)) { ok = false; break; }
          uint8_t* dst = d_smem + stage * C::STAGE_BYTES;
          const int row = (int)(r0 + (int64_t)t * C::N);
          mbar_arrive_expect_tx(&full[stage], C::STAGE_BYTES);
          for (int h = 0; h < C::HALVES; ++h)
            tma_load_2d(dst + h * (C::N * 128), &tm_d, &full[stage], h * 64, row);
          issued[stage]++;
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
          if constexpr (COL_SCALE) {
            // the tile's column scales (row is a multiple of 8: 16-byte aligned)
            if (!mbar_wait(&sc_empty[sslot], sphase ^ 1, a.status, abort_flag)) { ok = false; break; }
            mbar_arrive_expect_tx(&sc_full[sslot], C::N * 4);
            tma_load_1d(sc_smem + sslot * C::N, &tm_scale, &sc_full[sslot], row);
            sc_issued[sslot]++;
            if (++sslot == C::SC_SLOTS) { sslot = 0; sphase ^= 1; }
          }
        }
      }
      if (!ok) {
        // drain: every load this thread issued must land before the CTA exits
        for (int s = 0; s < C::STAGES; ++s)
          if (issued[s]) { int z = 0; mbar_wait(&full[s], (issued[s] - 1) & 1, nullptr, &z); }
        for (int s = 0; s < C::SC_SLOTS; ++s)
          if (sc_issued[s]) { int z = 0; mbar_wait(&sc_full[s], (sc_issued[s] - 1) & 1, nullptr, &z); }
        int z = 0;
        if (q_issued) mbar_wait(q_full, (q_issued - 1) & 1, nullptr, &z);
      }
    }
  } else if (warp > C::EPI_WARPS) {
    // ---------------------------------------------------------------- MMA issuer(s)
    // warp mw issues the MMAs of the M tiles m with m % NMW == mw
    const int mw = warp - C::EPI_WARPS - 1;
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
        if (++uslot == C::UNIT_RING) { uslot = 0; uphase ^= 1; }
        return u;
      };
      for (long long u = take_unit(); u < n_units && ok; u = take_unit(), ++it) {
        const int chunk = (int)(u / nqb);
        const int64_t r0 = a.doc_off[a.chunk_doc[chunk]];
        const int64_t r1 = a.doc_off[a.chunk_doc[chunk + 1]];
        const int ntiles = (int)((r1 - r0 + C::N - 1) / C::N);
        if (!mbar_wait(q_full, it & 1, a.status, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint64_t ad0 = sw128_desc(smem_u32(q_smem));
        for (int t = 0; t < ntiles; ++t) {
          if (!mbar_wait(&acc_empty[acc * C::NMW + mw], acc_phase ^ 1, a.status, abort_flag)) { ok = false; break; }
          if (!mbar_wait(&full[stage], phase, a.status, abort_flag)) { ok = false; break; }
          tc_fence_after();
          // descriptors: the start-address field (bits 0-13, address / 16) of a
          // base descriptor plus a compile-time offset (shared addresses stay
          // below 2^18 bytes, so the field never carries)
          const uint64_t bd0 = sw128_desc(smem_u32(d_smem + stage * C::STAGE_BYTES));
#pragma unroll
          for (int mi = 0; mi < MT / C::NMW; ++mi) {
            const int m = mi * C::NMW + mw;
#pragma unroll
            for (int k = 0; k < C::K_STEPS; ++k) {
              const int half = (k * C::K_STEP * (FP8 ? 1 : 2)) / 128;
              const int within = (k * C::K_STEP * (FP8 ? 1 : 2)) % 128;
              const uint64_t bd = bd0 + (uint64_t)((half * (C::N * 128) + within) >> 4);
              const uint32_t dt = tmem + acc * C::ACC_COLS + m * C::N;
              if constexpr (AT) {
                // A: 128 lanes x (K_STEP elements = 8 columns of 32-bit words) per step
                const uint32_t at = tmem + C::A_BASE + m * C::A_COLS + k * 8;
                if constexpr (FP8) mma_f8_ta(dt, at, bd, C::IDESC, k > 0);
                else mma_bf16_ta(dt, at, bd, C::IDESC, k > 0);
              } else {
                const uint64_t ad = ad0 + (uint64_t)((((m * C::HALVES + half) * 16384) + within) >> 4);
                if constexpr (FP8) mma_f8(dt, ad, bd, C::IDESC, k > 0);
                else mma_bf16(dt, ad, bd, C::IDESC, k > 0);
              }
            }
          }
          mma_commit(&empty[stage]);
          mma_commit(&acc_full[acc * C::NMW + mw]);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
          if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
        if (ok && !AT) mma_commit(q_empty);
      }
      // all MMAs of this thread complete before the CTA releases TMEM
      mma_commit(&done_bar[mw]);
      int z = 0;
      mbar_wait(&done_bar[mw], 0, nullptr, &z);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    constexpr int CH = C::CH;
    constexpr int NSUB = C::N / kRowAlign;  // 8-column subgroups per tile
    const int eset = warp / C::EPI_SET;     // this warp takes the tiles t with t % E == eset
    const int wpos = warp % C::EPI_SET;
    const int m_tile = wpos >> 2;
    const int quad = wpos & 3;              // = warp % 4: the TMEM lane quarter this warp may read
    const int local_row = m_tile * 128 + quad * 32 + lane;
    const uint32_t t_lane = (uint32_t)(quad * 32) << 16;
    // carries between sets (E > 1): this set writes slot eset, reads the previous set's slot
    const int prev_set = (eset + E - 1) % E;
    float* carry_out_buf = carry_smem + (eset * C::EPI_SET + wpos) * 32;
    float* carry_in_buf = carry_smem + (prev_set * C::EPI_SET + wpos) * 32;
    uint64_t* cfull_out = carry_full + eset * C::EPI_SET + wpos;
    uint64_t* cempty_out = carry_empty + eset * C::EPI_SET + wpos;
    uint64_t* cfull_in = carry_full + prev_set * C::EPI_SET + wpos;
    uint64_t* cempty_in = carry_empty + prev_set * C::EPI_SET + wpos;
    uint32_t n_pub = 0, n_recv = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    int sslot = 0;
    uint32_t sphase = 0;
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
      if (++uslot == C::UNIT_RING) { uslot = 0; uphase ^= 1; }
      return u;
    };
    for (long long u = take_unit(); u < n_units && ok; u = take_unit()) {
      const int chunk = (int)(u / nqb);
      const int qb = qb0 + (int)(u % nqb);
      const int prow = qb * C::M_RES + local_row;
      const int p = a.row_part[prow];
      int g = 1;
      bool add = false;
      float* dst = nullptr;  // score row of this row's query (rows of no part: none)
      float row_scale = 1.f;
      if (p >= 0) {
        g = a.part_g[p];
        add = a.part_pass[p] > 0;
        dst = a.scores + (int64_t)a.part_query[p] * a.n_sets;
      }
      if constexpr (FP8) row_scale = a.q_scale[prow];
      if constexpr (AT) {
        // This unit's query row goes into TMEM as operand A (lane = row, 32-bit
        // words of packed elements, lower k in the lower bits).  Every MMA of
        // the previous unit has completed: this warp consumed its last tile.
        constexpr int W = C::A_COLS;  // words per row
        const uint4* src = reinterpret_cast<const uint4*>(a.qpack + (int64_t)prow * W);
        uint32_t words[W];
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
          const uint4 x = src[i];
          words[4 * i] = x.x; words[4 * i + 1] = x.y; words[4 * i + 2] = x.z; words[4 * i + 3] = x.w;
        }
        const uint32_t ta = tmem + t_lane + C::A_BASE + m_tile * C::A_COLS;
        if constexpr (W == 64) tmem_st64(ta, words);
        else tmem_st32(ta, words);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(q_full);
      }
      const int d0 = a.chunk_doc[chunk];
      const int d1 = a.chunk_doc[chunk + 1];
      const int64_t r0 = a.doc_off[d0];
      const int64_t r1 = a.doc_off[d1];
      const int ntiles = (int)((r1 - r0 + C::N - 1) / C::N);
      int cur = d0;           // index of the next set to end
      float carry = -INFINITY;  // E = 1: running max entering the next tile
      // Set ends come from the store's end bitmap (bit i: a set ends with padded
      // row 8 i + 7).  The bits of tile t + 1 are loaded while tile t is folded.
      const int64_t sg_first = r0 / kRowAlign;
      auto load_bits = [&](int t) -> uint32_t {
        const int64_t gs = sg_first + (int64_t)t * NSUB;
        const uint32_t* w = a.end_bits + (gs >> 5);
        return (uint32_t)((((uint64_t)__ldg(w + 1) << 32) | __ldg(w)) >> (gs & 31));
      };
      uint32_t bits = load_bits(0);
      // Scores leave in groups: lane (set index mod g) of a slot keeps the score
      // of its set, and the kept scores are stored together when the group is
      // complete or the next group begins.
      float mine = 0.f;
      int mine_set = -1;
      auto flush = [&]() {
        if (mine_set >= 0 && dst != nullptr) {
          float* d = dst + mine_set;
          *d = add ? (*d + mine) : mine;
        }
        mine_set = -1;
      };

      // A set that ends: sum its row maxima over each query slot and keep the
      // score.  A 32-row slot whose row maxima are all below 2 in magnitude is
      // summed in 2^-24 fixed point by one warp reduction (|sum| < 2^30, exact
      // and independent of the order; rounding <= 2^-25 per row), any other
      // slot by a g-lane xor butterfly.
      auto set_end = [&](float m, float set_sc) {
        float val = m * row_scale;
        if constexpr (SS) val *= set_sc;
        float sum;
        if (__all_sync(0xffffffffu, g == 32 && fabsf(val) < 2.f)) {
          sum = (float)__reduce_add_sync(0xffffffffu, __float2int_rn(val * 16777216.f)) * (1.f / 16777216.f);
        } else {
          sum = val;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float other = __shfl_xor_sync(0xffffffffu, sum, o);
            if (o < g) sum += other;
          }
        }
        if (mine_set >= 0 && ((mine_set ^ cur) & ~(g - 1)) != 0) flush();  // another group
        const int j = cur & (g - 1);
        if ((lane & (g - 1)) == j) { mine = sum; mine_set = cur; }
        if (j == g - 1) flush();
        ++cur;
      };

      // Fold the 8-column subgroups of one loaded chunk into the running max,
      // branch-free: out[s] is the running max after subgroup s, and the max
      // restarts after a subgroup that ends a set.  fp8: each column is first
      // multiplied by its vector's scale s_j, read as a broadcast from the
      // tile's scale slot.  Columns past the chunk's last row (the next chunk's
      // rows or the tensor map's zero fill) are folded too: no set ends there.
      float run = -INFINITY;
      float out[NSUB];
      auto fold = [&](const float (&v)[CH], int sg0, uint32_t ends, const float* sc) {
#pragma unroll
        for (int s = 0; s < CH / 8; ++s) {
          float x[8];
          if constexpr (COL_SCALE) {
            const float4 s0 = reinterpret_cast<const float4*>(sc)[2 * s];
            const float4 s1 = reinterpret_cast<const float4*>(sc)[2 * s + 1];
            const float2 p0 = fmul2(make_float2(v[8 * s + 0], v[8 * s + 1]), make_float2(s0.x, s0.y));
            const float2 p1 = fmul2(make_float2(v[8 * s + 2], v[8 * s + 3]), make_float2(s0.z, s0.w));
            const float2 p2 = fmul2(make_float2(v[8 * s + 4], v[8 * s + 5]), make_float2(s1.x, s1.y));
            const float2 p3 = fmul2(make_float2(v[8 * s + 6], v[8 * s + 7]), make_float2(s1.z, s1.w));
            x[0] = p0.x; x[1] = p0.y; x[2] = p1.x; x[3] = p1.y;
            x[4] = p2.x; x[5] = p2.y; x[6] = p3.x; x[7] = p3.y;
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = v[8 * s + j];
          }
          run = fmax3(run, fmax3(x[0], x[1], x[2]), fmax3(x[3], x[4], x[5]));
          run = fmax3(run, x[6], x[7]);
          out[sg0 + s] = run;
          run = ((ends >> (sg0 + s)) & 1u) ? -INFINITY : run;
        }
      };
      // E > 1: hand the running max entering tile t + 1 to the next set / take
      // the one entering tile t from the previous set (bounded waits; every
      // lane passes its own row)
      auto publish = [&](float val) -> bool {
        const bool w = mbar_wait(cempty_out, (n_pub & 1) ^ 1, a.status, abort_flag);
        if (!__all_sync(0xffffffffu, w)) return false;
        carry_out_buf[lane] = val;
        mbar_arrive(cfull_out);
        ++n_pub;
        return true;
      };
      auto receive = [&](float& val) -> bool {
        const bool w = mbar_wait(cfull_in, n_recv & 1, a.status, abort_flag);
        if (!__all_sync(0xffffffffu, w)) return false;
        val = carry_in_buf[lane];
        mbar_arrive(cempty_in);
        ++n_recv;
        return true;
      };

      for (int t = 0; t < ntiles; ++t) {
        // Sets are padded to multiples of kRowAlign rows, so a set ends only at
        // the end of an 8-column subgroup: one bit per subgroup, cut at the
        // chunk's last row (the next chunk's sets are not this unit's).
        uint32_t ends = bits;
        {
          const int64_t n_sub = (r1 - r0) / kRowAlign - (int64_t)t * NSUB;
          if (n_sub < 32) ends &= (1u << n_sub) - 1u;
          if (NSUB < 32) ends &= (1u << (NSUB & 31)) - 1u;
        }
        // the same in every lane; the reduction makes that visible to the
        // compiler, so the tests below are uniform branches
        ends = __reduce_or_sync(0xffffffffu, ends);
        if (t + 1 < ntiles) bits = load_bits(t + 1);
        if (E > 1 && t % E != eset) {
          // another set's tile: only the set count and the ring positions move
          cur += __popc(ends);
          if constexpr (COL_SCALE) { if (++sslot == C::SC_SLOTS) { sslot = 0; sphase ^= 1; } }
          if (++acc == 2) { acc = 0; acc_phase ^= 1; }
          continue;
        }
        // SS: the scales of this tile's first two set ends, loaded before the
        // fold so that their latency hides behind it (a tile of N <= 256
        // columns rarely ends more than two sets)
        float sc_a = 1.f, sc_b = 1.f;
        if constexpr (SS) {
          if (ends != 0) {
            sc_a = __ldg(a.set_scale + cur);
            sc_b = __ldg(a.set_scale + min(cur + 1, d1 - 1));
          }
        }
        // every lane waits, then the warp agrees, so the .sync.aligned TMEM
        // loads below always run with the whole warp
        bool got = mbar_wait(&acc_full[acc * C::NMW + m_tile % C::NMW], acc_phase, a.status, abort_flag);
        if constexpr (COL_SCALE) got = got && mbar_wait(&sc_full[sslot], sphase, a.status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const float* sc = COL_SCALE ? sc_smem + sslot * C::N : nullptr;
        const uint32_t tcol = tmem + t_lane + acc * C::ACC_COLS + m_tile * C::N;
#pragma unroll
        for (int c = 0; c < C::N / CH; ++c) {
          float v[CH];
          tmem_ld_cols<CH>(tcol + c * CH, v);
          if (c == C::N / CH - 1) {
            // the accumulator is in registers: hand the buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc * C::NMW + m_tile % C::NMW]);
          }
          fold(v, c * (CH / 8), ends, COL_SCALE ? sc + c * CH : nullptr);
        }
        if constexpr (COL_SCALE) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&sc_empty[sslot]);
          if (++sslot == C::SC_SLOTS) { sslot = 0; sphase ^= 1; }
        }
        if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        // run: the max since this tile's last set end (or over the whole tile)
        float cin = -INFINITY;
        if constexpr (E > 1) {
          const bool more = t + 1 < ntiles;
          bool fine = true;
          if (ends != 0 && more) fine = publish(run);
          if (fine && t > 0) fine = receive(cin);
          if (fine && ends == 0 && more) fine = publish(fmaxf(cin, run));
          if (!fine) {
            ok = false;
            break;
          }
        } else {
          cin = carry;
          carry = ends != 0 ? run : fmaxf(carry, run);
        }
        run = -INFINITY;
        uint32_t e = ends;
        int k_end = 0;
#pragma unroll 1
        while (e) {
          const int sidx = __ffs(e) - 1;
          e &= e - 1;
          float set_sc = 1.f;
          if constexpr (SS) set_sc = k_end == 0 ? sc_a : k_end == 1 ? sc_b : __ldg(a.set_scale + cur);
          set_end(fmaxf(cin, pick(out, sidx)), set_sc);
          cin = -INFINITY;
          ++k_end;
        }
      }
      flush();  // the scores this warp still keeps
    }
  }

  __syncthreads();
  if (warp == C::EPI_WARPS + 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <int MT, bool FP8, bool AT = false, int E = 1, bool SS = false>
gem_status launch_tc(const gem_store* s, gem_workspace* ws, const CUtensorMap& tm_q,
                     const CUtensorMap& tm_d, const CUtensorMap& tm_scale, const ChunkMap* cm,
                     float* scores, cudaStream_t st) {
  using C = TcCfg<MT, FP8, AT, E, SS>;
  static bool attr_set = false;
  if (!attr_set) {
    GEM_CUDA_TRY(cudaFuncSetAttribute(tc_score_all_kernel<MT, FP8, AT, E, SS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
    attr_set = true;
  }
  TcArgs a;
  a.hdr = ws->d_plan_hdr;
  a.row_part = ws->d_row_part;
  a.part_query = ws->d_part_query;
  a.part_g = ws->d_part_g;
  a.part_pass = ws->d_part_pass;
  a.q_scale = ws->d_qpack_scale;
  a.qpack = FP8 ? reinterpret_cast<const uint32_t*>(ws->d_qpack_fp8)
                : reinterpret_cast<const uint32_t*>(ws->d_qpack_bf16);
  a.doc_off = s->d_pad_offsets;
  a.end_bits = s->d_end_bits;
  a.chunk_doc = cm->d_chunk_doc;
  a.n_chunks = cm->n_chunks;
  a.n_sets = s->n_sets;
  a.scores = scores;
  a.set_scale = s->d_set_scale;
  a.status = ws->d_status;
  a.unit_counter = ws->d_unit_counter;
  for (int pass = 0; pass < ws->n_passes; ++pass) {
    a.pass = pass;
    GEM_CUDA_TRY(cudaMemsetAsync(ws->d_unit_counter, 0, sizeof(int), st));
    tc_score_all_kernel<MT, FP8, AT, E, SS><<<s->n_sm, C::THREADS, C::SMEM_BYTES, st>>>(tm_q, tm_d, tm_scale, a);
    GEM_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  return GEM_OK;
}

template <bool FP8, bool SS = false>
gem_status launch_tc_dtype(const gem_store* s, gem_workspace* ws, int m_tiles, int variant, const ChunkMap* cm,
                           float* scores, cudaStream_t st) {
  const int n = variant == GEM_TC_A_TMEM ? TcCfg<2, FP8, true>::N : 256 / m_tiles;
  const CUtensorMap* td = nullptr;
  const CUtensorMap* tsc = nullptr;
  gem_status r = !FP8 ? store_tmap_bf16(s, n, &td) : SS ? store_tmap_fp8_set(s, n, &td) : store_tmap_fp8(s, n, &td);
  if (r != GEM_OK) return r;
  if (FP8 && !SS && (r = store_tmap_fp8_scale(s, n, &tsc)) != GEM_OK) return r;
  if (!FP8 || SS) tsc = td;  // unused
  const CUtensorMap& tq = FP8 ? ws->tmap_q_fp8 : ws->tmap_q_bf16;
  if (variant == GEM_TC_A_TMEM) return launch_tc<2, FP8, true, 1, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
  if (variant == GEM_TC_TWO_SETS) {
    if (m_tiles == 1) return launch_tc<1, FP8, false, 2, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
    return launch_tc<2, FP8, false, 2, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
  }
  switch (m_tiles) {
    case 1: return launch_tc<1, FP8, false, 1, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
    case 2: return launch_tc<2, FP8, false, 1, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
    case 4: return launch_tc<4, FP8, false, 1, SS>(s, ws, tq, *td, *tsc, cm, scores, st);
    default: return fail(GEM_ERR_INVALID, "m_tiles must be 1, 2 or 4");
  }
}

}  // namespace

gem_status launch_tc_score_all(const gem_store* s, gem_workspace* ws, int compute, int m_tiles,
                               int variant, int chunk_rows, float* scores, cudaStream_t st) {
  const ChunkMap* cm = nullptr;
  gem_status r = store_chunk_map(s, chunk_rows, &cm);
  if (r != GEM_OK) return r;
  if (variant == GEM_TC_A_TMEM && m_tiles != 2) return fail(GEM_ERR_INVALID, "a_tmem needs m_tiles = 2");
  if (variant == GEM_TC_TWO_SETS && m_tiles == 4) return fail(GEM_ERR_INVALID, "two_sets needs m_tiles 1 or 2");
  if (compute == GEM_BF16) return launch_tc_dtype<false>(s, ws, m_tiles, variant, cm, scores, st);
  if (compute == GEM_FP8_E4M3) return launch_tc_dtype<true>(s, ws, m_tiles, variant, cm, scores, st);
  if (compute == GEM_FP8_E4M3_SET) return launch_tc_dtype<true, true>(s, ws, m_tiles, variant, cm, scores, st);
  return fail(GEM_ERR_INVALID, "tensor-core scoring takes bf16 or fp8");
}

}  // namespace gem
