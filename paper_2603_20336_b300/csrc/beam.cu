// Cluster-guided multi-path beam search (Algorithm 5, Sec. 4.5.3), batched over
// queries and run in rounds.
//
// Per query: one queue W_e per accepted entry set, the result set R and a visited
// bitmap over the stored sets.  A round is
//   expand   every non-empty W_e (in entry order) pops its best set P; if P scores
//            below tau (the worst score in R once R holds ef sets) W_e is emptied,
//            else every neighbour P' of P (in list order) that is not visited and
//            has a vector in a cluster of C_query is marked visited and queued
//   compact  the queued sets of all queries into one candidate list (CSR)
//   score    qsim = m_q - qCH of every queued set from the queries' centroid
//            tables, built once per search (the arithmetic of gem_estimate_codes)
//   insert   in queue order, each scored set into its W_e and into R
// and the host runs rounds until no queue is left.  W_e and R keep the ef best
// sets under the total order (higher score, then lower id); they are unsorted
// arrays, so pop and eviction are warp arg-max / arg-min searches (the insert
// keeps the worst entry in registers until it changes, appends a queue's run of
// candidates at once and discards by ballot the candidates R cannot take).  One warp owns one query
// in every kernel, so no two warps ever update the same query state; the expand
// tests a popped set's neighbours 32 at a time, one per lane.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace gem {
namespace {

constexpr int kBsWarps = 8;
constexpr int kBsThreads = kBsWarps * 32;

__device__ __forceinline__ bool bs_better(float a, int ia, float b, int ib) {
  return a > b || (a == b && ia < ib);
}

// Index (warp-uniform) of the best (want_best) or worst entry among sc/id[0, n),
// -1 if n == 0.
__device__ __forceinline__ int warp_arg(const float* sc, const int32_t* id, int n, bool want_best) {
  const int lane = threadIdx.x & 31;
  int bj = -1;
  float bs = 0.f;
  int bi = 0;
  for (int j = lane; j < n; j += 32) {
    const float s = sc[j];
    const int i = id[j];
    const bool take = bj < 0 || (want_best ? bs_better(s, i, bs, bi) : bs_better(bs, bi, s, i));
    if (take) { bj = j; bs = s; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
    const float os = __shfl_xor_sync(0xffffffffu, bs, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oj >= 0 && (bj < 0 || (want_best ? bs_better(os, oi, bs, bi) : bs_better(bs, bi, os, oi)))) {
      bj = oj; bs = os; bi = oi;
    }
  }
  return bj;
}

struct BeamState {
  int n_queries, S, ef, cap, vwords, mwords;
  int* nq;            // [B] queues per query
  float* qsc;         // [B * S * ef]
  int32_t* qid;
  int* qsize;         // [B * S]
  float* rsc;         // [B * ef]
  int32_t* rid;
  int* rsize;         // [B]
  uint32_t* visited;  // [B * vwords]
  int64_t* raw;       // [B * cap] queued sets of the round
  int32_t* rawq;      // [B * cap] their queue
  int* cnt;           // [B]
  int64_t* off;       // [B + 1]
  int64_t* cand;      // compacted queued sets
  int32_t* candq;     // their queue
  float* score;       // their scores
  int* flag;          // any queue non-empty at a round's start
  float* tables;      // [B * max_np * k1 * 32] qCH tables of the queries
  const uint32_t* dead;  // deleted sets (Sec. 4.6), or null
};

// Entries: accepted entry sets (not -1, not repeated) open one queue each and are
// queued for scoring like any expansion.
__global__ void bs_init_kernel(BeamState st, const int64_t* __restrict__ entries, int n_sets) {
  const int lane = threadIdx.x & 31;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < st.n_queries; b += (gridDim.x * blockDim.x) >> 5) {
    uint32_t* vis = st.visited + (int64_t)b * st.vwords;
    int c = 0;
    for (int e = 0; e < st.S; ++e) {
      const int64_t id = entries[(int64_t)b * st.S + e];
      if (id < 0 || id >= n_sets) continue;
      const bool seen = (vis[id >> 5] >> (id & 31)) & 1u;
      if (seen) continue;
      if (lane == 0) {
        vis[id >> 5] |= 1u << (id & 31);
        st.raw[(int64_t)b * st.cap + c] = id;
        st.rawq[(int64_t)b * st.cap + c] = c;
      }
      __syncwarp();
      ++c;
    }
    if (lane == 0) { st.nq[b] = c; st.cnt[b] = c; }
  }
}

// flag bits: 1 = some queue was non-empty at the round's start; 2 = a neighbour
// id outside [0, n_sets) or more queued sets than the round buffer holds
__global__ void bs_expand_kernel(BeamState st, const int64_t* __restrict__ graph_off,
                                 const int32_t* __restrict__ graph_nbrs, const int64_t* __restrict__ set_off,
                                 const int32_t* __restrict__ icodes, const uint32_t* __restrict__ qmask,
                                 int n_sets) {
  const int lane = threadIdx.x & 31;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < st.n_queries; b += (gridDim.x * blockDim.x) >> 5) {
    uint32_t* vis = st.visited + (int64_t)b * st.vwords;
    const uint32_t* mask = qmask + (int64_t)b * st.mwords;
    float* rsc = st.rsc + (int64_t)b * st.ef;
    int32_t* rid = st.rid + (int64_t)b * st.ef;
    const int nr = st.rsize[b];
    float tau = -INFINITY;
    if (nr >= st.ef) tau = rsc[warp_arg(rsc, rid, nr, false)];
    int c = 0;
    bool active = false, bad = false;
    const int nq = st.nq[b];
    for (int qi = 0; qi < nq; ++qi) {
      int* qs = st.qsize + (int64_t)b * st.S + qi;
      const int n = *qs;
      if (n == 0) continue;
      active = true;
      float* sc = st.qsc + ((int64_t)b * st.S + qi) * st.ef;
      int32_t* id = st.qid + ((int64_t)b * st.S + qi) * st.ef;
      const int j = warp_arg(sc, id, n, true);
      const float psc = sc[j];
      const int pid = id[j];
      __syncwarp();
      if (lane == 0) {
        sc[j] = sc[n - 1];
        id[j] = id[n - 1];
        *qs = psc < tau ? 0 : n - 1;
      }
      __syncwarp();
      if (psc < tau) continue;
      // the neighbours of P in list order, 32 at a time (lane i: the i-th of the
      // group), with the outcome of the sequential walk: a neighbour is queued
      // if it is not visited, has a vector in a cluster of C_query and is not a
      // repeat of an earlier one in the list; the walk stops at the first id
      // outside [0, n_sets) and once the round buffer is full
      const int64_t e1 = graph_off[pid + 1];
      for (int64_t eb = graph_off[pid]; eb < e1 && !bad; eb += 32) {
        const int64_t e = eb + lane;
        const bool in = e < e1;
        const int nb = in ? graph_nbrs[e] : 0;
        const unsigned badm = __ballot_sync(0xffffffffu, in && (nb < 0 || nb >= n_sets));
        const int n_ok = badm ? __ffs(badm) - 1 : 32;  // lanes before the first bad id
        bool take = in && lane < n_ok;
        const unsigned okm = __ballot_sync(0xffffffffu, take);
        // a repeat of an earlier neighbour of this group takes that one's outcome
#pragma unroll 1
        for (int j = 0; j < 32; ++j) {
          const int other = __shfl_sync(0xffffffffu, nb, j);
          if (j < lane && ((okm >> j) & 1u) && other == nb) take = false;
        }
        // visited (read past L1: earlier groups set bits with atomics)
        if (take) take = !((__ldcg(vis + (nb >> 5)) >> (nb & 31)) & 1u);
        if (take) {
          bool hit = false;
          const int64_t v1 = set_off[nb + 1];
          for (int64_t v = set_off[nb]; v < v1; ++v) {
            const int cl = icodes[v];
            if ((mask[cl >> 5] >> (cl & 31)) & 1u) { hit = true; break; }
          }
          take = hit;
        }
        const unsigned qm = __ballot_sync(0xffffffffu, take);
        const int rank = __popc(qm & ((1u << lane) - 1u));
        const int room = st.cap - c;
        if (take && rank < room) {
          atomicOr(vis + (nb >> 5), 1u << (nb & 31));
          st.raw[(int64_t)b * st.cap + c + rank] = nb;
          st.rawq[(int64_t)b * st.cap + c + rank] = qi;
        }
        const int n_new = __popc(qm);
        if (n_new > room) bad = true;  // the walk stops at the first set with no room
        c += min(n_new, room);
        if (badm) bad = true;
        __syncwarp();
      }
    }
    if (lane == 0) {
      st.cnt[b] = c;
      if (active) atomicOr(st.flag, 1);
      if (bad) atomicOr(st.flag, 2);
    }
  }
}

// exclusive scan of cnt [B] into off [B + 1] by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) bs_scan_kernel(const int* __restrict__ cnt, int n, int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  __shared__ int64_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const int64_t v = i < n ? cnt[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
      const int64_t add = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) off[i] = base + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) base += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = base;
}

__global__ void bs_compact_kernel(BeamState st) {
  const int lane = threadIdx.x & 31;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < st.n_queries; b += (gridDim.x * blockDim.x) >> 5) {
    const int64_t o = st.off[b];
    for (int j = lane; j < st.cnt[b]; j += 32) {
      st.cand[o + j] = st.raw[(int64_t)b * st.cap + j];
      st.candq[o + j] = st.rawq[(int64_t)b * st.cap + j];
    }
  }
}

// Insert (s, i) into the bounded set sc/id holding n entries (capacity cap):
// append while there is room, else replace the worst entry if (s, i) is better.
// n and the worst entry (index w, -1 when not known; its score and id) live in
// registers, so a set that cannot enter costs no memory read.  Ids within a
// query are distinct, so the worst entry is unique.  Warp-uniform.
__device__ __forceinline__ void cached_insert(float* sc, int32_t* id, int& n, int& w, float& ws, int& wi, int cap,
                                              float s, int i) {
  const int lane = threadIdx.x & 31;
  if (n < cap) {
    if (lane == 0) { sc[n] = s; id[n] = i; }
    ++n;
    w = -1;
  } else {
    if (w < 0) {
      w = warp_arg(sc, id, n, false);
      ws = sc[w];
      wi = id[w];
    }
    if (bs_better(s, i, ws, wi)) {
      if (lane == 0) { sc[w] = s; id[w] = i; }
      w = -1;
    }
  }
  __syncwarp();
}

__global__ void bs_insert_kernel(BeamState st) {
  const int lane = threadIdx.x & 31;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < st.n_queries; b += (gridDim.x * blockDim.x) >> 5) {
    float* rsc = st.rsc + (int64_t)b * st.ef;
    int32_t* rid = st.rid + (int64_t)b * st.ef;
    int rn = st.rsize[b], rw = -1, rwi = 0;
    float rws = 0.f;
    int cur = -1, qn = 0, qw = -1, qwi = 0;  // the queue of the current run of candidates
    float qws = 0.f;
    float* qsc = nullptr;
    int32_t* qid = nullptr;
    const int64_t j1 = st.off[b + 1];
    for (int64_t jb = st.off[b]; jb < j1; jb += 32) {
      // 32 candidates' (score, id, queue) in one load, then in order
      const int64_t jl = jb + lane;
      float sl = 0.f;
      int il = 0, ql = 0;
      if (jl < j1) { sl = st.score[jl]; il = (int)st.cand[jl]; ql = st.candq[jl]; }
      const int m = (int)(j1 - jb < 32 ? j1 - jb : 32);
      // the queues: runs of candidates of one queue, in order; a run that fits in
      // the queue's free room is appended at once
      for (int t = 0; t < m;) {
        const int qi = __shfl_sync(0xffffffffu, ql, t);
        const unsigned other = __ballot_sync(0xffffffffu, lane < m && ql != qi) & (0xffffffffu << t);
        const int e = other ? __ffs(other) - 1 : m;  // the run is [t, e)
        if (qi != cur) {
          if (cur >= 0 && lane == 0) st.qsize[(int64_t)b * st.S + cur] = qn;
          cur = qi;
          qsc = st.qsc + ((int64_t)b * st.S + qi) * st.ef;
          qid = st.qid + ((int64_t)b * st.S + qi) * st.ef;
          qn = st.qsize[(int64_t)b * st.S + qi];
          qw = -1;
        }
        if (qn + (e - t) <= st.ef) {
          if (lane >= t && lane < e) { qsc[qn + lane - t] = sl; qid[qn + lane - t] = il; }
          qn += e - t;
          qw = -1;
          __syncwarp();
        } else {
          for (int k = t; k < e; ++k)
            cached_insert(qsc, qid, qn, qw, qws, qwi, st.ef, __shfl_sync(0xffffffffu, sl, k),
                          __shfl_sync(0xffffffffu, il, k));
        }
        t = e;
      }
      // R (a deleted set keeps its place on the paths but never enters R): free
      // slots are filled in order; once R is full, the worst entry only improves,
      // so a candidate not better than it now never enters, and the first one
      // that is better replaces it
      const bool live = lane < m && (!st.dead || !((st.dead[il >> 5] >> (il & 31)) & 1u));
      unsigned pend = __ballot_sync(0xffffffffu, live);
      while (pend) {
        if (rn < st.ef) {
          const int rank = __popc(pend & ((1u << lane) - 1u));
          const bool take = ((pend >> lane) & 1u) && rank < st.ef - rn;
          if (take) { rsc[rn + rank] = sl; rid[rn + rank] = il; }
          const unsigned taken = __ballot_sync(0xffffffffu, take);
          rn += __popc(taken);
          rw = -1;
          pend &= ~taken;
          __syncwarp();
          continue;
        }
        if (rw < 0) {
          rw = warp_arg(rsc, rid, rn, false);
          rws = rsc[rw];
          rwi = rid[rw];
        }
        const unsigned better = __ballot_sync(0xffffffffu, ((pend >> lane) & 1u) && bs_better(sl, il, rws, rwi));
        if (!better) break;
        const int k = __ffs(better) - 1;
        const float ks = __shfl_sync(0xffffffffu, sl, k);
        const int ki = __shfl_sync(0xffffffffu, il, k);
        if (lane == 0) { rsc[rw] = ks; rid[rw] = ki; }
        rw = -1;
        pend &= (k == 31) ? 0u : (0xffffffffu << (k + 1));
        __syncwarp();
      }
    }
    if (lane == 0) {
      if (cur >= 0) st.qsize[(int64_t)b * st.S + cur] = qn;
      st.rsize[b] = rn;
    }
  }
}

// R of every query, best first; -1 / -inf past its size
__global__ void bs_output_kernel(BeamState st, int64_t* __restrict__ out_ids, float* __restrict__ out_scores) {
  const int lane = threadIdx.x & 31;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < st.n_queries; b += (gridDim.x * blockDim.x) >> 5) {
    float* rsc = st.rsc + (int64_t)b * st.ef;
    int32_t* rid = st.rid + (int64_t)b * st.ef;
    int n = st.rsize[b];
    for (int k = 0; k < st.ef; ++k) {
      if (k < st.rsize[b]) {
        const int j = warp_arg(rsc, rid, n, true);
        const float s = rsc[j];
        const int i = rid[j];
        __syncwarp();
        if (lane == 0) {
          out_ids[(int64_t)b * st.ef + k] = i;
          out_scores[(int64_t)b * st.ef + k] = s;
          rsc[j] = rsc[n - 1];
          rid[j] = rid[n - 1];
        }
        __syncwarp();
        --n;
      } else if (lane == 0) {
        out_ids[(int64_t)b * st.ef + k] = -1;
        out_scores[(int64_t)b * st.ef + k] = -INFINITY;
      }
    }
  }
}

template <typename T>
bool bs_alloc(T** p, size_t count) {
  if (cudaMalloc(p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

}  // namespace

gem_status beam_search(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                       int32_t n_queries, const int64_t* graph_off, const int32_t* graph_nbrs, int32_t max_degree,
                       const uint32_t* cluster_mask, const int64_t* entries, int32_t entry_stride, int32_t ef,
                       int32_t max_rounds, int64_t* out_ids, float* out_scores, int32_t* out_rounds, cudaStream_t stm) {
  BeamState st{};
  st.n_queries = n_queries;
  st.S = entry_stride;
  st.ef = ef;
  st.cap = std::max(entry_stride, entry_stride * max_degree);
  st.vwords = (int)((s->n_sets + 31) / 32);
  st.mwords = (s->k2 + 31) / 32;
  st.dead = s->d_dead;
  const size_t B = (size_t)n_queries;
  const int max_np = (w->max_q_len + 31) / 32;
  std::vector<void*> bufs;
  auto keep = [&](void* p) { bufs.push_back(p); return p != nullptr; };
  bool ok = keep(bs_alloc(&st.nq, B) ? (void*)st.nq : nullptr) &&
            keep(bs_alloc(&st.qsc, B * st.S * ef) ? (void*)st.qsc : nullptr) &&
            keep(bs_alloc(&st.qid, B * st.S * ef) ? (void*)st.qid : nullptr) &&
            keep(bs_alloc(&st.qsize, B * st.S) ? (void*)st.qsize : nullptr) &&
            keep(bs_alloc(&st.rsc, B * ef) ? (void*)st.rsc : nullptr) &&
            keep(bs_alloc(&st.rid, B * ef) ? (void*)st.rid : nullptr) &&
            keep(bs_alloc(&st.rsize, B) ? (void*)st.rsize : nullptr) &&
            keep(bs_alloc(&st.visited, B * st.vwords) ? (void*)st.visited : nullptr) &&
            keep(bs_alloc(&st.raw, B * st.cap) ? (void*)st.raw : nullptr) &&
            keep(bs_alloc(&st.rawq, B * st.cap) ? (void*)st.rawq : nullptr) &&
            keep(bs_alloc(&st.cnt, B) ? (void*)st.cnt : nullptr) &&
            keep(bs_alloc(&st.off, B + 1) ? (void*)st.off : nullptr) &&
            keep(bs_alloc(&st.cand, B * st.cap) ? (void*)st.cand : nullptr) &&
            keep(bs_alloc(&st.candq, B * st.cap) ? (void*)st.candq : nullptr) &&
            keep(bs_alloc(&st.score, B * st.cap) ? (void*)st.score : nullptr) &&
            keep(bs_alloc(&st.flag, 1) ? (void*)st.flag : nullptr) &&
            keep(bs_alloc(&st.tables, B * (size_t)max_np * s->k1 * 32) ? (void*)st.tables : nullptr);
  auto release = [&]() {
    for (void* p : bufs)
      if (p) cudaFree(p);
  };
  if (!ok) {
    release();
    return fail(GEM_ERR_OOM, "beam search scratch");
  }
  gem_status r = GEM_OK;
  cudaError_t e = cudaSuccess;
  const int grid = (int)std::min<int64_t>((n_queries + kBsWarps - 1) / kBsWarps, 4096);
  int64_t total = 0;
  int flag = 0;
  int rounds = 0;
  // score the queued sets of the round (codes form) and insert them
  auto score_insert = [&]() -> gem_status {
    bs_scan_kernel<<<1, 1024, 0, stm>>>(st.cnt, n_queries, st.off);
    bs_compact_kernel<<<grid, kBsThreads, 0, stm>>>(st);
    GEM_CUDA_TRY(cudaGetLastError());
    GEM_CUDA_TRY(cudaMemcpyAsync(&total, st.off + n_queries, sizeof(int64_t), cudaMemcpyDeviceToHost, stm));
    GEM_CUDA_TRY(cudaStreamSynchronize(stm));
    note_launches(2);
    if (total > 0) {
      gem_status rr = launch_qch_scan_ids(s, st.tables, q_offsets, n_queries, max_np, st.off, st.cand, st.score,
                                          w->d_status, reinterpret_cast<unsigned long long*>(w->d_unit_counter), stm);
      if (rr != GEM_OK) return rr;
      bs_insert_kernel<<<grid, kBsThreads, 0, stm>>>(st);
      GEM_CUDA_TRY(cudaGetLastError());
      note_launches(1);
    }
    return GEM_OK;
  };
  e = cudaMemsetAsync(st.qsize, 0, sizeof(int) * B * st.S, stm);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.rsize, 0, sizeof(int) * B, stm);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.visited, 0, sizeof(uint32_t) * B * st.vwords, stm);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "beam search state");
  }
  if (n_queries > 0) {
    r = launch_qch_tables(s, w->d_qcodes, w->qch_form == GEM_QCH_ASYMMETRIC ? q : nullptr, q_offsets, n_queries,
                          max_np, st.tables, stm);
    if (r != GEM_OK) {
      release();
      return r;
    }
    bs_init_kernel<<<grid, kBsThreads, 0, stm>>>(st, entries, (int)s->n_sets);
    note_launches(1);
    r = score_insert();
    while (r == GEM_OK && rounds < max_rounds) {
      e = cudaMemsetAsync(st.flag, 0, sizeof(int), stm);
      if (e != cudaSuccess) break;
      bs_expand_kernel<<<grid, kBsThreads, 0, stm>>>(st, graph_off, graph_nbrs, s->d_offsets, s->d_icodes,
                                                     cluster_mask, (int)s->n_sets);
      note_launches(1);
      e = cudaMemcpyAsync(&flag, st.flag, sizeof(int), cudaMemcpyDeviceToHost, stm);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
      if (e != cudaSuccess || !flag) break;
      if (flag & 2) {
        r = fail(GEM_ERR_INVALID, "a neighbour id is out of range or a list is longer than max_degree");
        break;
      }
      ++rounds;
      r = score_insert();
    }
    if (r == GEM_OK && e == cudaSuccess) {
      bs_output_kernel<<<grid, kBsThreads, 0, stm>>>(st, out_ids, out_scores);
      note_launches(1);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
    }
  }
  release();
  if (e != cudaSuccess) return cuda_fail(e, "beam search");
  if (r != GEM_OK) return r;
  if (out_rounds) *out_rounds = rounds;
  return GEM_OK;
}

}  // namespace gem
