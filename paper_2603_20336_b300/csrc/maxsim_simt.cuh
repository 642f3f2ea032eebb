// Per-pair exact MaxSim on the SIMT pipes, shared by every FP32 scorer so that
// all of them produce bit-identical scores for the same (query, set) pair.
//
// Arithmetic order (fixed, independent of launch shape):
//   dot(q_i, p_j) = c0 + c1, c_h = e_h + o_h, where e_h and o_h are FP32 fused
//                   multiply-add chains over the even and the odd k of the half
//                   k in [64 h, 64 h + 64), each in ascending k (the two chains of
//                   a half advance together in packed two-lane FMAs)
//   m_i = max_j dot(q_i, p_j)
//   CH  = Kahan (compensated) sum of m_i over i = 0 .. m_q - 1 in ascending order
// With Sim = -(L2 distance) (the L2 form of Definition 1) the chains sum
// (q_ik - p_jk)^2 instead (the difference rounded, then one fused multiply-add),
// m_i = -sqrt(min_j d2(q_i, p_j)) with the correctly rounded square root, and the
// same Kahan sum follows.
//
// Mapping: lane l holds query rows 2(l/2) and 2(l/2)+1 of the current 32-row
// group, components k in [64 (l%2), 64 (l%2) + 64), in registers; the set's
// vectors are staged 8 at a time in the warp's shared slice (the upper half of a
// staged vector is shifted by 16 bytes so both half-warps' broadcast reads fall
// in different banks), so one 16-byte shared load feeds 4 packed FMAs (8
// products).  The query components are kept as packed pairs (k, k + 1).  The two
// halves of a dot meet through one xor shuffle.  In the codes form every
// stored vector p_j is replaced by its centroid C[code_j] and the query rows by
// the centroids of the query codes, which gives the quantized estimate in
// similarity form.
#pragma once
#include "internal.h"
#include "ptx.cuh"

namespace gem {

constexpr int kVecBlock = 8;         // set vectors staged per step
constexpr int kQStride = kDim + 4;   // padded query row stride in shared memory (floats)
constexpr int kStageStride = kDim + 4;  // staged set vector: [k 0..63][4 pad][k 64..127]

// Query registers of a lane: row a's 64 components as 32 packed pairs
// (k, k + 1), then row b's.
constexpr int kQPairs = kDim / 2;
constexpr int kRowPairs = kDim / 4;

// One block of up to kVecBlock staged set vectors against this lane's two query
// rows: best_a / best_b take the max of the block's dot products (L2: of the
// negated squared distances).
template <bool L2>
__device__ __forceinline__ void block_terms(const float* __restrict__ stage, int rd_off,
                                            const uint64_t (&qr)[kQPairs], int nv, float& best_a, float& best_b) {
  uint64_t acc_a[kVecBlock], acc_b[kVecBlock];  // packed (even k, odd k) chains
#pragma unroll
  for (int v = 0; v < kVecBlock; ++v) { acc_a[v] = 0ull; acc_b[v] = 0ull; }
#pragma unroll
  for (int k4 = 0; k4 < kDim / 8; ++k4) {
#pragma unroll
    for (int v = 0; v < kVecBlock; ++v) {
      // components (4 k4, 4 k4 + 1) and (4 k4 + 2, 4 k4 + 3) of this half
      const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(stage + v * kStageStride + rd_off + 4 * k4);
      if constexpr (L2) {
        uint64_t d = fsub2(qr[2 * k4], p.x);
        acc_a[v] = ffma2(d, d, acc_a[v]);
        d = fsub2(qr[2 * k4 + 1], p.y);
        acc_a[v] = ffma2(d, d, acc_a[v]);
        d = fsub2(qr[kRowPairs + 2 * k4], p.x);
        acc_b[v] = ffma2(d, d, acc_b[v]);
        d = fsub2(qr[kRowPairs + 2 * k4 + 1], p.y);
        acc_b[v] = ffma2(d, d, acc_b[v]);
      } else {
        acc_a[v] = ffma2(qr[2 * k4], p.x, acc_a[v]);
        acc_a[v] = ffma2(qr[2 * k4 + 1], p.y, acc_a[v]);
        acc_b[v] = ffma2(qr[kRowPairs + 2 * k4], p.x, acc_b[v]);
        acc_b[v] = ffma2(qr[kRowPairs + 2 * k4 + 1], p.y, acc_b[v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < kVecBlock; ++v) {
    const float ca = __fadd_rn(lo2(acc_a[v]), hi2(acc_a[v]));  // e_h + o_h
    const float cb = __fadd_rn(lo2(acc_b[v]), hi2(acc_b[v]));
    // c0 + c1 in the lane holding c0 and c1 + c0 in its partner: the same sum
    const float da = ca + __shfl_xor_sync(0xffffffffu, ca, 1);
    const float db = cb + __shfl_xor_sync(0xffffffffu, cb, 1);
    if (v < nv) {
      best_a = fmaxf(best_a, L2 ? -da : da);
      best_b = fmaxf(best_b, L2 ? -db : db);
    }
  }
}

// The per-query-vector term m_i from the block maxima.
template <bool L2>
__device__ __forceinline__ float row_term(float best) {
  return L2 ? -__fsqrt_rn(-best) : best;
}

// One row of the set (or its centroid in the codes form) as this lane's float4.
__device__ __forceinline__ float4 set_row4(const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                           const float* __restrict__ centroids, int j, int lane) {
  const float* src = row_code ? centroids + (int64_t)row_code[j] * kDim : P + (int64_t)j * kDim;
  return reinterpret_cast<const float4*>(src)[lane];
}

// CH of query rows qs[0 .. m_q) (row stride q_stride floats, shared or global
// memory) against one set.  Called by a full warp; returns the score in every
// lane.  P: the set's first row; row_code == nullptr: rows are P[j * 128],
// otherwise rows are centroids[row_code[j] * 128].  The next 8 set vectors are
// loaded into registers while the current 8 are multiplied, so the loads of a
// set overlap its arithmetic; the arithmetic order is unchanged.
template <bool L2 = false>
__device__ __forceinline__ float warp_chamfer(const float* __restrict__ qs, int q_stride, int m_q,
                                              const float* __restrict__ P, const int32_t* __restrict__ row_code,
                                              const float* __restrict__ centroids, int m_p,
                                              float* __restrict__ stage, float* __restrict__ rowmax,
                                              uint64_t (&qr)[kQPairs], int& loaded_rg) {
  const int lane = threadIdx.x & 31;
  const int half = lane & 1;           // component half of this lane
  const int pair = lane >> 1;          // query rows 2 pair, 2 pair + 1
  const int n_rg = (m_q + 31) >> 5;
  // where this lane's float4 of a set vector goes in the staged layout
  const int st_off = 4 * lane + (lane >= 16 ? 4 : 0);
  const int rd_off = half * (kDim / 2 + 4);
  for (int rg = 0; rg < n_rg; ++rg) {
    const int ia = rg * 32 + 2 * pair, ib = ia + 1;
    if (rg != loaded_rg) {
#pragma unroll
      for (int k2 = 0; k2 < kRowPairs; ++k2) {
        const int kk = half * (kDim / 2) + 2 * k2;
        qr[k2] = (ia < m_q) ? pack2(qs[(int64_t)ia * q_stride + kk], qs[(int64_t)ia * q_stride + kk + 1]) : 0ull;
        qr[kRowPairs + k2] =
            (ib < m_q) ? pack2(qs[(int64_t)ib * q_stride + kk], qs[(int64_t)ib * q_stride + kk + 1]) : 0ull;
      }
      loaded_rg = rg;
    }
    float best_a = -INFINITY, best_b = -INFINITY;
    float4 pf[kVecBlock];
    {
      const int nv0 = min(kVecBlock, m_p);
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv0) pf[v] = set_row4(P, row_code, centroids, v, lane);
    }
    for (int j0 = 0; j0 < m_p; j0 += kVecBlock) {
      const int nv = min(kVecBlock, m_p - j0);
      __syncwarp();
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv) *reinterpret_cast<float4*>(stage + v * kStageStride + st_off) = pf[v];
      __syncwarp();
      const int j1 = j0 + kVecBlock;
      const int nv1 = min(kVecBlock, m_p - j1);
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v)
        if (v < nv1) pf[v] = set_row4(P, row_code, centroids, j1 + v, lane);
      block_terms<L2>(stage, rd_off, qr, nv, best_a, best_b);
    }
    if (half == 0 && ia < m_q) rowmax[ia] = row_term<L2>(best_a);
    if (half == 1 && ib < m_q) rowmax[ib] = row_term<L2>(best_b);
  }
  __syncwarp();
  float s = 0.f;
  if (lane == 0) {
    float c = 0.f;  // Kahan compensation
    for (int i = 0; i < m_q; ++i) {
      const float y = __fsub_rn(rowmax[i], c);
      const float t = __fadd_rn(s, y);
      c = __fsub_rn(__fsub_rn(t, s), y);
      s = t;
    }
  }
  return __shfl_sync(0xffffffffu, s, 0);
}

// ------------------------------------------------------------------ streamed id lists

// The pairs of an id-list batch: query b's candidates are cand_ids[cand_off[b] ..
// cand_off[b + 1]), query rows q[q_off[b] .. q_off[b + 1]) of 128 floats.
struct StreamArgs {
  const float* q;
  const int64_t* q_off;
  int n_queries;
  const int64_t* cand_off;
  const int64_t* cand_ids;
  const float* docs;       // FP32 master [n_vecs * 128]
  const int64_t* doc_off;  // [n_sets + 1]
  int64_t n_sets;
  float* scores;
  int* status;
  int max_q_len;
  // optional processing order: position i takes pair perm[i], whose query is
  // perm[i] / per_query (a pool of per_query candidates per query); a chunk is
  // then a run of positions whose pairs share a query
  const int32_t* perm = nullptr;
  int per_query = 0;
  unsigned long long* counter = nullptr;  // with perm: group counter, zero at launch
  // codes form (optional): stored row r is centroids[codes[r]] and, with qcodes,
  // query row i is centroids[qcodes[i]] (the quantized estimate in similarity
  // form, the same per-dot arithmetic)
  const int32_t* codes = nullptr;
  const float* centroids = nullptr;
  const int32_t* qcodes = nullptr;
};

constexpr int kRing = 4;  // 8-vector stages in a warp's ring
// floats per ring stage: 8 staged vectors and 8 of padding, so that two stages
// read at once (the two half-warps of a short row group) fall in different banks
constexpr int kRingBlock = kVecBlock * kStageStride + 8;
__host__ __device__ constexpr int ring_block(bool dual) { return dual ? kRingBlock : kVecBlock * kStageStride; }
constexpr int kStreamRowmax = 1024;  // row maxima a warp keeps (chunk pairs x max_q_len)

// Pairs per chunk for queries of at most max_q_len rows.
__host__ __device__ constexpr int stream_chunk(int max_q_len) {
  return kStreamRowmax / max_q_len < 1 ? 1 : (kStreamRowmax / max_q_len > 32 ? 32 : kStreamRowmax / max_q_len);
}

// Exact scores of the pairs t_begin .. t_end - 1 by one warp, with the per-pair
// arithmetic of warp_chamfer (bit-identical scores).  The range is cut into
// chunks of at most stream_chunk(max_q_len) pairs of one query; a chunk is taken
// one 32-row group of the query at a time (the query registers are loaded once
// per chunk and group, or once per query when it has one group), and its pairs'
// row maxima collect in rowmax [chunk][max_q_len] until every group is done; then
// lane i takes the Kahan sum of pair i.  The set vectors of the whole range
// stream through a ring of kRing 8-vector stages with cp.async, kRing - 1 blocks
// ahead and across pair, group and chunk boundaries, so the gathers of the next
// sets overlap the arithmetic of the current one (a chunk's later groups re-read
// its sets from L2).  Scores: -inf for a negative id, NaN and a status for an id
// >= n_sets or a query longer than max_q_len.  DUAL: a row group of at most 16
// rows is taken by both half-warps on alternate 8-vector blocks (the same
// per-dot arithmetic; the maxima of the halves meet at the end, so the scores
// are unchanged); the rerank's instantiation keeps the plain loop.  CODES: the
// codes form of StreamArgs (stored rows, and with qcodes query rows, replaced by
// the centroids their codes name).
template <bool L2, bool DUAL = false, bool CODES = false>
__device__ __forceinline__ void stream_pairs(const StreamArgs& a, int64_t t_begin, int64_t t_end, float* ring,
                                             float* rowmax) {
  constexpr int RB = ring_block(DUAL);  // floats per ring stage
  if (t_begin >= t_end) return;
  const int lane = threadIdx.x & 31;
  const int half = lane & 1;
  const int pair = lane >> 1;
  const int st_off = 4 * lane + (lane >= 16 ? 4 : 0);
  const int rd_off = half * (kDim / 2 + 4);
  const int chunk_max = stream_chunk(a.max_q_len);
  int q_first = 0;  // the query owning t_begin
  if (!a.perm) {
    int hi = a.n_queries - 1;
    while (q_first < hi) {
      const int mid = (q_first + hi + 1) >> 1;
      if (a.cand_off[mid] <= t_begin) q_first = mid; else hi = mid - 1;
    }
  }
  // the pair at position i
  auto pair_at = [&](int64_t i) -> int64_t { return a.perm ? (int64_t)a.perm[i] : i; };
  // the chunk starting at pair c0 (b: a query at or before c0's); nrg = its
  // 32-row groups, 0 for a query longer than max_q_len
  struct Chunk {
    int64_t c0, c1;
    int b, nrg;
  };
  auto chunk_at = [&](int64_t c0, int b) -> Chunk {
    Chunk c;
    c.c0 = c0;
    if (c0 >= t_end) {
      c.c1 = c0;
      c.b = b;
      c.nrg = 0;
      return c;
    }
    if (a.perm) {
      // the run of positions from c0 whose pairs belong to c0's query (at most
      // chunk_max): lane i looks at position c0 + i
      b = (int)(pair_at(c0) / a.per_query);
      const int64_t pi = c0 + lane;
      const bool other = lane >= chunk_max || pi >= t_end || (int)(pair_at(pi) / a.per_query) != b;
      const uint32_t m = __ballot_sync(0xffffffffu, other);
      c.c1 = c0 + (m ? __ffs(m) - 1 : 32);
    } else {
      while (c0 >= a.cand_off[b + 1]) ++b;
      c.c1 = min(min(c0 + chunk_max, t_end), a.cand_off[b + 1]);
    }
    c.b = b;
    const int m = (int)(a.q_off[b + 1] - a.q_off[b]);
    c.nrg = m > a.max_q_len ? 0 : (m + 31) >> 5;
    return c;
  };
  // lane i: row offset and length of the chunk's pair i (length 0: nothing to
  // stream -- an invalid id, or a chunk with no groups)
  auto chunk_info = [&](const Chunk& c, int64_t& r0, int& mp) {
    const int64_t t = c.c0 + lane;
    r0 = 0;
    mp = 0;
    if (t < c.c1 && c.nrg > 0) {
      const int64_t id = a.cand_ids[pair_at(t)];
      if (id >= 0 && id < a.n_sets) {
        r0 = a.doc_off[id];
        mp = (int)(a.doc_off[id + 1] - r0);
      }
    }
  };

  // ---- producer: the blocks in the consumer's order (chunk, group, pair, block)
  Chunk pc = chunk_at(t_begin, q_first);
  int64_t p_r0;
  int p_mp;
  chunk_info(pc, p_r0, p_mp);
  Chunk pn = chunk_at(pc.c1, pc.b);  // the next chunk, its infos loaded a chunk ahead
  int64_t n_r0;
  int n_mp;
  chunk_info(pn, n_r0, n_mp);
  int rgp = 0, ip = 0, bp = 0;
  int mp_cur = __shfl_sync(0xffffffffu, p_mp, 0);
  int64_t r0_cur = __shfl_sync(0xffffffffu, p_r0, 0);
  uint32_t issued = 0;
  // move the cursor to the next block that holds vectors (warp-uniform)
  auto seek = [&]() {
    while (pc.c0 < t_end && bp * kVecBlock >= mp_cur) {
      bp = 0;
      if (++ip >= (int)(pc.c1 - pc.c0)) {  // a pass over the chunk is done
        ip = 0;
        if (++rgp >= pc.nrg) {             // the chunk is done
          rgp = 0;
          pc = pn;
          p_r0 = n_r0;
          p_mp = n_mp;
          if (pc.c0 >= t_end) break;
          pn = chunk_at(pc.c1, pc.b);
          chunk_info(pn, n_r0, n_mp);
        }
      }
      mp_cur = __shfl_sync(0xffffffffu, p_mp, ip);
      r0_cur = __shfl_sync(0xffffffffu, p_r0, ip);
    }
  };
  // CODES: the codes of a block are loaded one call ahead of its copies, so the
  // load's latency overlaps a block of arithmetic (lane v < pend_nv: code v)
  int pend_code = 0, pend_nv = 0;
  auto load_next = [&]() {
    seek();
    pend_nv = 0;
    if (pc.c0 < t_end) {
      const int64_t row = r0_cur + (int64_t)bp * kVecBlock;
      pend_nv = min(kVecBlock, mp_cur - bp * kVecBlock);
      pend_code = lane < pend_nv ? a.codes[row + lane] : 0;
      ++bp;
    }
  };
  auto issue = [&]() {
    float* dst = ring + (issued % kRing) * RB;
    if constexpr (CODES) {
#pragma unroll
      for (int v = 0; v < kVecBlock; ++v) {
        const int cv = __shfl_sync(0xffffffffu, pend_code, v);
        if (v < pend_nv) cp_async16(dst + v * kStageStride + st_off, a.centroids + (int64_t)cv * kDim + 4 * lane);
      }
      load_next();
    } else {
      seek();
      if (pc.c0 < t_end) {
        const int64_t row = r0_cur + (int64_t)bp * kVecBlock;
        const int nv = min(kVecBlock, mp_cur - bp * kVecBlock);
        const float* srcp = a.docs + row * kDim + 4 * lane;
#pragma unroll
        for (int v = 0; v < kVecBlock; ++v)
          if (v < nv) cp_async16(dst + v * kStageStride + st_off, srcp + v * kDim);
        ++bp;
      }
    }
    cp_async_commit();
    ++issued;
  };
  if constexpr (CODES) load_next();
#pragma unroll
  for (int i = 0; i < kRing - 1; ++i) issue();

  // ---- consumer
  uint64_t qr[kQPairs];
  int loaded_b = -1;  // query whose only row group is in qr
  uint32_t consumed = 0;
  for (Chunk cc = chunk_at(t_begin, q_first); cc.c0 < t_end; cc = chunk_at(cc.c1, cc.b)) {
    const int64_t q0 = a.q_off[cc.b];
    const int m_q = (int)(a.q_off[cc.b + 1] - q0);
    const int n = (int)(cc.c1 - cc.c0);
    const int64_t my_pair = lane < n ? pair_at(cc.c0 + lane) : 0;
    const int64_t my_id = lane < n ? a.cand_ids[my_pair] : -1;
    const int my_mp = (my_id >= 0 && my_id < a.n_sets) ? (int)(a.doc_off[my_id + 1] - a.doc_off[my_id]) : 0;
    for (int rg = 0; rg < cc.nrg; ++rg) {
      // a group of at most 16 rows: both half-warps hold its rows (lanes 16-31
      // as lanes 0-15) and take alternate 8-vector blocks of each set, so no
      // lane idles on empty rows; the two halves' row maxima meet at the end
      const bool dual = DUAL && m_q - rg * 32 <= 16;  // uniform over the warp
      const int ia = rg * 32 + 2 * (dual ? (pair & 7) : pair), ib = ia + 1;
      const int second = (dual && lane >= 16) ? 1 : 0;  // this lane takes the odd blocks
      if (cc.nrg > 1 || cc.b != loaded_b) {
        // rows ia and ib, components 64 half .. 64 half + 63, as packed pairs (codes
        // form with query codes: the rows of the centroids they name)
        const float* qa = a.q + (q0 + ia) * kDim;
        const float* qbr = a.q + (q0 + ib) * kDim;
        if (CODES && a.qcodes) {
          qa = ia < m_q ? a.centroids + (int64_t)a.qcodes[q0 + ia] * kDim : a.centroids;
          qbr = ib < m_q ? a.centroids + (int64_t)a.qcodes[q0 + ib] * kDim : a.centroids;
        }
        const float4* ra = reinterpret_cast<const float4*>(qa + half * (kDim / 2));
        const float4* rb = reinterpret_cast<const float4*>(qbr + half * (kDim / 2));
#pragma unroll
        for (int j = 0; j < kRowPairs / 2; ++j) {
          const float4 va = ia < m_q ? ra[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 vb = ib < m_q ? rb[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          qr[2 * j] = pack2(va.x, va.y);
          qr[2 * j + 1] = pack2(va.z, va.w);
          qr[kRowPairs + 2 * j] = pack2(vb.x, vb.y);
          qr[kRowPairs + 2 * j + 1] = pack2(vb.z, vb.w);
        }
        loaded_b = cc.nrg > 1 ? -1 : cc.b;
      }
      for (int i = 0; i < n; ++i) {
        const int m_p = __shfl_sync(0xffffffffu, my_mp, i);
        if (m_p == 0) continue;
        float best_a = -INFINITY, best_b = -INFINITY;
        const int nb = (m_p + kVecBlock - 1) / kVecBlock;
        if constexpr (!DUAL) {
          for (int blk = 0; blk < nb; ++blk) {
            issue();
            cp_async_wait<kRing - 1>();
            __syncwarp();
            const float* stage = ring + (consumed % kRing) * RB;
            block_terms<L2>(stage, rd_off, qr, min(kVecBlock, m_p - blk * kVecBlock), best_a, best_b);
            __syncwarp();
            ++consumed;
          }
        } else {
          // a dual group takes blocks blk (lanes 0-15) and blk + 1 (lanes 16-31)
          // at once: one block is issued before the two are read (into the stage
          // the last step freed) and, when there is a second, one after they are
          // consumed, so no stage is refilled while it is read
          for (int blk = 0; blk < nb; blk += dual ? 2 : 1) {
            const bool two = dual && blk + 1 < nb;
            issue();
            if (two) cp_async_wait<kRing - 2>(); else cp_async_wait<kRing - 1>();
            __syncwarp();
            const int mine = blk + second;
            const float* stage = ring + ((consumed + second) % kRing) * RB;
            block_terms<L2>(stage, rd_off, qr, mine < nb ? min(kVecBlock, m_p - mine * kVecBlock) : 0, best_a,
                            best_b);
            __syncwarp();
            consumed += two ? 2 : 1;
            if (two) issue();
          }
          if (dual) {
            best_a = fmaxf(best_a, __shfl_xor_sync(0xffffffffu, best_a, 16));
            best_b = fmaxf(best_b, __shfl_xor_sync(0xffffffffu, best_b, 16));
          }
        }
        float* rm = rowmax + i * a.max_q_len;
        if (!second && half == 0 && ia < m_q) rm[ia] = row_term<L2>(best_a);
        if (!second && half == 1 && ib < m_q) rm[ib] = row_term<L2>(best_b);
      }
    }
    __syncwarp();
    // lane i: the score of the chunk's pair i
    if (lane < n) {
      float score;
      if (my_id < 0) {
        score = -INFINITY;
      } else if (my_id >= a.n_sets || m_q > a.max_q_len) {
        set_status(a.status, my_id >= a.n_sets ? kDevBounds : kDevInvalid);
        score = __int_as_float(0x7fc00000);
      } else {
        const float* rm = rowmax + lane * a.max_q_len;
        float s = 0.f, c = 0.f;  // Kahan sum, compensation
        for (int i = 0; i < m_q; ++i) {
          const float y = __fsub_rn(rm[i], c);
          const float tt = __fadd_rn(s, y);
          c = __fsub_rn(__fsub_rn(tt, s), y);
          s = tt;
        }
        score = s;
      }
      a.scores[my_pair] = score;
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

}  // namespace gem
