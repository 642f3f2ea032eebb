// Quantized earth mover's distance between stored sets (Sec. 4.2, Eq. 11-14):
//
//   qEMD(P1, P2) = min_T sum_ij T_ij d_X(NN(p_i), NN(p'_j)),  d_X = 1 - <., .>,
//   T >= 0, every row of T sums to 1/m1 and every column to 1/m2.
//
// One CTA per pair of sets.  Vectors that share a code are one point whose mass
// is its multiplicity, so with n1 and n2 distinct codes the problem is a
// transportation problem with integer supplies s_i = w_i m2 at the n1 sources
// and integer demands r_j = w'_j m1 at the n2 sinks (the masses times m1 m2).
// It is solved exactly by successive shortest paths: a dense Dijkstra over the
// residual graph (forward edges source -> sink always, backward edges where
// flow is positive) with reduced costs under node potentials, then an
// augmentation by the bottleneck of the path.  Every augmentation moves at least
// one unit, so at most m1 m2 augmentations run, and every Dijkstra at most
// n1 + n2 extractions: the kernel always finishes.  The cost matrix (FP32, one
// FMA chain per centroid dot, clamped at 0) and the flows (16-bit: a flow never
// exceeds 128 x 128) live in shared memory; one __syncthreads per extraction.
// The result sum_ij flow_ij c_ij / (m1 m2) is summed in FP64 in a fixed order.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kQemdMax = 128;             // vectors per set
constexpr int kQemdThreads = 128;         // thread t owns source t and sink t
constexpr int kCStride = kQemdMax + 1;    // cost row stride (column reads conflict-free)
constexpr int kFStride = kQemdMax + 2;    // flow row stride (16-bit)
constexpr int kSink = kQemdMax;           // node id of sink j: kSink + j
constexpr int kStageRows = 32;            // centroid rows staged per step of the cost build

struct QemdSmem {
  float cost[kQemdMax * kCStride];
  // the flows; while the costs are built, the staging area of centroid rows
  uint16_t flow[kQemdMax * kFStride];
  float pot[2 * kQemdMax];        // node potentials (sources, then sinks)
  int prev[2 * kQemdMax];         // shortest-path tree of the current Dijkstra
  int sup[kQemdMax];              // remaining supplies
  int dem[kQemdMax];              // remaining demands
  int ua[kQemdMax], wa[kQemdMax];  // distinct codes of set A and their multiplicities
  int ub[kQemdMax], wb[kQemdMax];
  int srt[kQemdMax];
  unsigned long long red[2][kQemdThreads / 32];
  double dred[kQemdThreads / 32];
  int n1, n2, remaining;
};
static_assert(kQemdMax * kFStride * 2 >= kStageRows * kDim * 4, "staging area too small");

__device__ __forceinline__ uint32_t dist_key(float f) {
  const uint32_t u = __float_as_uint(f == 0.f ? 0.f : f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_dist(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Distinct codes of one set, ascending, with multiplicities; returns their count.
__device__ int distinct_codes(QemdSmem& s, const int32_t* __restrict__ codes, int m, int* u, int* w) {
  const int t = threadIdx.x;
  const int v = t < m ? codes[t] : 0;
  if (t < m) {
    // rank of element t in (code, position) order
    int r = 0;
    for (int k = 0; k < m; ++k) {
      const int x = codes[k];
      r += (x < v) || (x == v && k < t);
    }
    s.srt[r] = v;
  }
  __syncthreads();
  if (t == 0) {
    int n = 0;
    for (int k = 0; k < m; ++k) {
      if (k == 0 || s.srt[k] != s.srt[k - 1]) {
        u[n] = s.srt[k];
        w[n] = 1;
        ++n;
      } else {
        ++w[n - 1];
      }
    }
    s.srt[0] = n;
  }
  __syncthreads();
  const int n = s.srt[0];
  __syncthreads();
  return n;
}

__global__ void __launch_bounds__(kQemdThreads)
qemd_kernel(const float* __restrict__ C, const int32_t* __restrict__ codes, const int64_t* __restrict__ set_off,
            int64_t n_sets, const int64_t* __restrict__ set_a, const int64_t* __restrict__ set_b, int64_t n_pairs,
            float* __restrict__ out, int* status) {
  extern __shared__ __align__(16) unsigned char qemd_raw[];
  QemdSmem& s = *reinterpret_cast<QemdSmem*>(qemd_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int64_t pr = blockIdx.x; pr < n_pairs; pr += gridDim.x) {
    const int64_t a = set_a[pr], b = set_b[pr];
    if (a < 0 || a >= n_sets || b < 0 || b >= n_sets) {
      if (t == 0) {
        set_status(status, kDevBounds);
        out[pr] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    const int64_t a0 = set_off[a], b0 = set_off[b];
    const int m1 = (int)(set_off[a + 1] - a0), m2 = (int)(set_off[b + 1] - b0);
    if (m1 > kQemdMax || m2 > kQemdMax) {
      if (t == 0) {
        set_status(status, kDevInvalid);
        out[pr] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    __syncthreads();  // the previous pair's shared state is no longer read
    const int n1 = distinct_codes(s, codes + a0, m1, s.ua, s.wa);
    const int n2 = distinct_codes(s, codes + b0, m2, s.ub, s.wb);

    // cost[i][j] = max(0, 1 - <C_ua[i], C_ub[j]>): thread j keeps its sink's
    // centroid in registers; the sources' centroids pass through shared memory
    float br[kDim];
    if (t < n2) {
      const float4* src = reinterpret_cast<const float4*>(C + (int64_t)s.ub[t] * kDim);
#pragma unroll
      for (int k4 = 0; k4 < kDim / 4; ++k4) {
        const float4 x = src[k4];
        br[4 * k4] = x.x; br[4 * k4 + 1] = x.y; br[4 * k4 + 2] = x.z; br[4 * k4 + 3] = x.w;
      }
    }
    float* stage = reinterpret_cast<float*>(s.flow);
    for (int i0 = 0; i0 < n1; i0 += kStageRows) {
      const int rows = min(kStageRows, n1 - i0);
      for (int idx = t; idx < rows * (kDim / 4); idx += kQemdThreads) {
        const int i = idx / (kDim / 4), k4 = idx % (kDim / 4);
        reinterpret_cast<float4*>(stage + i * kDim)[k4] =
            reinterpret_cast<const float4*>(C + (int64_t)s.ua[i0 + i] * kDim)[k4];
      }
      __syncthreads();
      if (t < n2) {
        for (int i = 0; i < rows; ++i) {
          float acc = 0.f;
#pragma unroll
          for (int k4 = 0; k4 < kDim / 4; ++k4) {
            const float4 x = reinterpret_cast<const float4*>(stage + i * kDim)[k4];
            acc = __fmaf_rn(x.x, br[4 * k4], acc);
            acc = __fmaf_rn(x.y, br[4 * k4 + 1], acc);
            acc = __fmaf_rn(x.z, br[4 * k4 + 2], acc);
            acc = __fmaf_rn(x.w, br[4 * k4 + 3], acc);
          }
          s.cost[(i0 + i) * kCStride + t] = fmaxf(0.f, __fsub_rn(1.f, acc));
        }
      }
      __syncthreads();
    }
    for (int idx = t; idx < kQemdMax * kFStride; idx += kQemdThreads) s.flow[idx] = 0;
    if (t < n1) { s.sup[t] = s.wa[t] * m2; s.pot[t] = 0.f; }
    if (t < n2) { s.dem[t] = s.wb[t] * m1; s.pot[kSink + t] = 0.f; }
    if (t == 0) s.remaining = m1 * m2;
    __syncthreads();

    bool failed = false;
    while (s.remaining > 0) {
      // Dijkstra from every source with supply left
      float ds = (t < n1 && s.sup[t] > 0) ? 0.f : INFINITY;  // source t
      float dk = INFINITY;                                   // sink t
      bool fs = t >= n1, fk = t >= n2;                       // finalised (absent nodes count as done)
      s.prev[t] = -1;
      s.prev[kSink + t] = -1;
      int tsel = -1;
      float dt = 0.f;
      __syncthreads();
      for (int it = 0; it < n1 + n2; ++it) {
        const uint32_t ks = fs ? 0xFFFFFFFFu : dist_key(ds);
        const uint32_t kk = fk ? 0xFFFFFFFFu : dist_key(dk);
        uint32_t kb = ks;
        uint32_t ib = (uint32_t)t;
        if (kk < ks) { kb = kk; ib = (uint32_t)(kSink + t); }
        const uint32_t wmin = __reduce_min_sync(0xffffffffu, kb);
        const uint32_t widx = __reduce_min_sync(0xffffffffu, kb == wmin ? ib : 0xFFFFFFFFu);
        if (lane == 0) s.red[it & 1][warp] = ((unsigned long long)wmin << 32) | widx;
        __syncthreads();
        unsigned long long best = s.red[it & 1][0];
#pragma unroll
        for (int w = 1; w < kQemdThreads / 32; ++w) best = min(best, s.red[it & 1][w]);
        const uint32_t bk = (uint32_t)(best >> 32);
        const int u = (int)(best & 0xFFFFFFFFu);
        const float du = key_dist(bk);
        if (bk == 0xFFFFFFFFu || !isfinite(du)) {  // no node reachable: cannot happen with supply left
          failed = true;
          break;
        }
        if (u < kSink) {
          if (t == u) fs = true;
          // relax this thread's sink over the forward edge u -> t
          if (!fk) {
            const float nd = du + s.cost[u * kCStride + t] + s.pot[u] - s.pot[kSink + t];
            if (nd < dk) { dk = nd; s.prev[kSink + t] = u; }
          }
        } else {
          const int j = u - kSink;
          if (t == j) fk = true;
          if (s.dem[j] > 0) { tsel = u; dt = du; break; }
          // relax this thread's source over the backward edge j -> t
          if (!fs && s.flow[t * kFStride + j] > 0) {
            const float nd = du - s.cost[t * kCStride + j] + s.pot[u] - s.pot[t];
            if (nd < ds) { ds = nd; s.prev[t] = u; }
          }
        }
      }
      if (failed) break;
      // potentials: finalised nodes move by their distance, the others by dt
      if (t < n1) s.pot[t] += fs ? fminf(ds, dt) : dt;
      if (t < n2) s.pot[kSink + t] += fk ? fminf(dk, dt) : dt;
      __syncthreads();
      if (t == 0) {
        // the path's bottleneck, then the augmentation
        int bott = s.dem[tsel - kSink];
        int v = tsel;
        for (int p = s.prev[v]; p >= 0; v = p, p = s.prev[v])
          if (v < kSink) bott = min(bott, (int)s.flow[v * kFStride + (p - kSink)]);
        bott = min(bott, s.sup[v]);
        v = tsel;
        for (int p = s.prev[v]; p >= 0; v = p, p = s.prev[v]) {
          if (v >= kSink) s.flow[p * kFStride + (v - kSink)] += (uint16_t)bott;
          else s.flow[v * kFStride + (p - kSink)] -= (uint16_t)bott;
        }
        s.sup[v] -= bott;
        s.dem[tsel - kSink] -= bott;
        s.remaining -= bott;
      }
      __syncthreads();
    }
    if (failed) {
      if (t == 0) {
        set_status(status, kDevInvalid);
        out[pr] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    // sum_ij flow_ij c_ij in FP64: column per thread, then warps, then the block
    double acc = 0.0;
    if (t < n2)
      for (int i = 0; i < n1; ++i) acc += (double)s.flow[i * kFStride + t] * (double)s.cost[i * kCStride + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s.dred[warp] = acc;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < kQemdThreads / 32; ++w) tot += s.dred[w];
      out[pr] = (float)(tot / ((double)m1 * (double)m2));
    }
  }
}

}  // namespace

gem_status launch_qemd(const gem_store* s, const int64_t* set_a, const int64_t* set_b, int64_t n_pairs, float* out,
                       int* status, cudaStream_t st) {
  const size_t smem = sizeof(QemdSmem);
  GEM_CUDA_TRY(cudaFuncSetAttribute(qemd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qemd_kernel, kQemdThreads, smem));
  if (per_sm < 1) return fail(GEM_ERR_UNSUPPORTED, "qEMD kernel does not fit on an SM");
  const int grid = (int)std::min<int64_t>(n_pairs, (int64_t)s->n_sm * per_sm);
  qemd_kernel<<<grid, kQemdThreads, smem, st>>>(s->d_codebook, s->d_codes, s->d_offsets, s->n_sets, set_a, set_b,
                                                n_pairs, out, status);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
