// Nearest-centroid codes, the stage-1 k-means update and the quantized Chamfer
// estimate qCH.
//
//   NN(x) = argmax_c <x, C_c> over the centroids of C_quant   (Sec. 4.1.1, 4.2.2)
//   qCH(Q, P) = sum_i min_j d_X(NN(q_i), NN(p_j)),  d_X = 1 - <., .>   (Sec. 4.5.3, Eq. 16)
//
// The estimate is returned in similarity form qsim = sum_i max_j <C_{a_i}, C_{b_j}>
// = m_q - qCH, which ranks sets identically.  Per query part (<= 32 query
// vectors) a table T[c][i] = <C_{a_i}, C_c> over all k1 centroids is built once;
// a set's estimate is then sum_i max_j T[b_j][i], one coalesced 128-byte row
// gather per stored vector.  The full k1 x k1 centroid table of the paper would
// take 17 GB at k1 = 65536; the per-query table holds the only rows a query uses.
//
// Arithmetic: every dot product is one FP32 fused multiply-add chain over
// k = 0 .. 127; NN ties go to the lowest centroid index; the per-set sum runs
// over the part's rows with a fixed xor butterfly, parts in ascending order.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

constexpr int kAsgRows = 64;   // vectors per CTA tile
constexpr int kAsgCents = 64;  // centroids per CTA tile
constexpr int kAsgThreads = 256;

// (value, index) with "larger value, then lower index" as the order.
__device__ __forceinline__ bool better(float v, int i, float bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

// A NaN dot (a NaN component in a row or a centroid) counts as -inf, so every
// row still gets a code in [0, k1): the lowest index when all its dots are NaN.
__device__ __forceinline__ float nan_low(float v) { return (v != v) ? -INFINITY : v; }

// 64 vectors x 64 centroids per step; thread (ty, tx) owns rows 4ty..4ty+3 and
// centroids 4tx..4tx+3 of the step; operands are staged k-major in shared memory.
// keys: larger key = larger value, then lower index (the order of better());
// -0 and +0 are the same value
__device__ __forceinline__ unsigned long long best_key(float v, int i) {
  const uint32_t u = __float_as_uint(v == 0.f ? 0.f : v);
  const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)o << 32) | (0xFFFFFFFFu - (uint32_t)i);
}

// split != nullptr: blockIdx.y takes the centroids [y * span, (y + 1) * span) and
// the row's best over them is merged into split[row] by a 64-bit atomic max of
// best_key; every dot is the same FMA chain as in the unsplit form, so the
// merged argmax is the same.  rows != nullptr: row r of the launch is row
// rows[r] of X / codes / best_out (the rows the tensor-core assignment could
// not decide); n_dev != nullptr bounds n on the device.  CTAs stride over the
// 64-row blocks.
__global__ void __launch_bounds__(kAsgThreads)
assign_kernel(const float* __restrict__ X, int64_t n, const int64_t* __restrict__ n_dev,
              const float* __restrict__ C, int k1, int32_t* __restrict__ codes, float* __restrict__ best_out,
              unsigned long long* __restrict__ split = nullptr, int span = 0,
              const int32_t* __restrict__ rows = nullptr) {
  if (n_dev) n = min(n, *n_dev);
  const int c_begin = split ? (int)blockIdx.y * span : 0;
  const int c_end = split ? min(k1, c_begin + span) : k1;
  __shared__ __align__(16) float xs[kDim][kAsgRows];
  __shared__ __align__(16) float cs[kDim][kAsgCents];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t row0 = (int64_t)blockIdx.x * kAsgRows; row0 < n; row0 += (int64_t)gridDim.x * kAsgRows) {
  __syncthreads();  // the previous block's tiles are no longer read
  for (int idx = threadIdx.x; idx < kAsgRows * kDim; idx += kAsgThreads) {
    const int r = idx / kDim, k = idx % kDim;
    const int64_t src = row0 + r < n ? (rows ? (int64_t)rows[row0 + r] : row0 + r) : -1;
    xs[k][r] = src >= 0 ? X[src * kDim + k] : 0.f;
  }
  float bv[4];
  int bi[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) { bv[a] = -INFINITY; bi[a] = 0x7fffffff; }
  for (int c0 = c_begin; c0 < c_end; c0 += kAsgCents) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kAsgCents * kDim; idx += kAsgThreads) {
      const int c = idx / kDim, k = idx % kDim;
      cs[k][c] = (c0 + c < c_end) ? C[(int64_t)(c0 + c) * kDim + k] : 0.f;
    }
    __syncthreads();
    float acc[4][4] = {};
#pragma unroll 4
    for (int k = 0; k < kDim; ++k) {
      const float4 xv = *reinterpret_cast<const float4*>(&xs[k][ty * 4]);
      const float4 cv = *reinterpret_cast<const float4*>(&cs[k][tx * 4]);
      const float xr[4] = {xv.x, xv.y, xv.z, xv.w};
      const float cr[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = __fmaf_rn(xr[a], cr[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        const float v = nan_low(acc[a][b]);
        if (c < c_end && better(v, c, bv[a], bi[a])) { bv[a] = v; bi[a] = c; }
      }
  }
  // reduce over the 16 threads (tx) that share each row: lanes of a half warp
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv[a], o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi[a], o);
      if (better(ov, oi, bv[a], bi[a])) { bv[a] = ov; bi[a] = oi; }
    }
    const int64_t r = row0 + ty * 4 + a;
    if (tx == 0 && r < n) {
      if (split) {
        if (bi[a] != 0x7fffffff) atomicMax(split + r, best_key(bv[a], bi[a]));
      } else {
        const int64_t dst = rows ? (int64_t)rows[r] : r;
        codes[dst] = bi[a];
        if (best_out) best_out[dst] = bv[a];
      }
    }
  }
  }
}

// codes from the merged keys of the split form
// (a key of 0 -- no CTA merged anything into the row -- gives code 0, so a
// code is always a valid centroid index)
__global__ void assign_finish_kernel(const unsigned long long* __restrict__ split, int64_t n,
                                     int32_t* __restrict__ codes) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = split[r];
    codes[r] = key == 0ull ? 0 : (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
  }
}

// Spherical Lloyd update, step 1: per-centroid sums (FP64) and counts.
__global__ void kmeans_accumulate_kernel(const float* __restrict__ X, int64_t n,
                                         const int32_t* __restrict__ codes, double* __restrict__ sums,
                                         int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int c = codes[r];
    const float4 v = reinterpret_cast<const float4*>(X + r * kDim)[lane];
    double* s = sums + (int64_t)c * kDim + lane * 4;
    atomicAdd(s + 0, (double)v.x);
    atomicAdd(s + 1, (double)v.y);
    atomicAdd(s + 2, (double)v.z);
    atomicAdd(s + 3, (double)v.w);
    if (lane == 0) atomicAdd(counts + c, 1);
  }
}

// Step 2: C_c = sums_c / |sums_c| for centroids with members; others keep C_c.
__global__ void kmeans_finalize_kernel(const double* __restrict__ sums, const int* __restrict__ counts,
                                       int k1, float* __restrict__ C) {
  const int lane = threadIdx.x & 31;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < k1; c += (gridDim.x * blockDim.x) >> 5) {
    if (counts[c] == 0) continue;
    double v[4], ss = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = sums[(int64_t)c * kDim + lane * 4 + j];
      ss += v[j] * v[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
    if (ss > 0.0) {
      float4 w = make_float4((float)(v[0] * inv), (float)(v[1] * inv), (float)(v[2] * inv), (float)(v[3] * inv));
      reinterpret_cast<float4*>(C + (int64_t)c * kDim)[lane] = w;
    }
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int64_t* __restrict__ rows,
                                   int64_t n, float* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5)
    reinterpret_cast<float4*>(dst + r * kDim)[lane] =
        reinterpret_cast<const float4*>(src + rows[r] * kDim)[lane];
}

// Tables of one batch of queries q0 .. q0+nq-1.  Part p of the batch is part
// pi = p % max_np of query b = q0 + p / max_np (a part that query does not have
// is skipped): T[p][c][i] = <C_{a_i}, C_c> for the part's rows i, zero beyond.
// With qvec (the asymmetric form) the exact query rows replace the centroids
// of their codes: T[p][c][i] = <q_i, C_c>.  Block = (256 centroids, part).
__global__ void __launch_bounds__(256)
qch_table_kernel(const float* __restrict__ C, int k1, const int32_t* __restrict__ qcodes,
                 const float* __restrict__ qvec, const int64_t* __restrict__ q_off, int q0, int max_np,
                 float* __restrict__ T) {
  __shared__ __align__(16) float qa[32][kDim + 4];
  const int p = blockIdx.y;
  const int b = q0 + p / max_np, pi = p % max_np;
  const int64_t r0 = q_off[b] + 32LL * pi;
  const int64_t rr = q_off[b + 1] - r0;
  if (rr <= 0) return;
  const int rows = (int)min((int64_t)32, rr);
  for (int idx = threadIdx.x; idx < 32 * kDim; idx += blockDim.x) {
    const int i = idx / kDim, k = idx % kDim;
    qa[i][k] = (i >= rows) ? 0.f : qvec ? qvec[(r0 + i) * kDim + k] : C[(int64_t)qcodes[r0 + i] * kDim + k];
  }
  __syncthreads();
  const int c = blockIdx.x * 256 + threadIdx.x;
  if (c >= k1) return;
  float cr[kDim];
#pragma unroll
  for (int k4 = 0; k4 < kDim / 4; ++k4) {
    const float4 v = reinterpret_cast<const float4*>(C + (int64_t)c * kDim)[k4];
    cr[4 * k4] = v.x; cr[4 * k4 + 1] = v.y; cr[4 * k4 + 2] = v.z; cr[4 * k4 + 3] = v.w;
  }
  float* out = T + ((int64_t)p * k1 + c) * 32;
  for (int i0 = 0; i0 < 32; i0 += 4) {
    float d[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < kDim; ++k) acc = __fmaf_rn(qa[i0 + u][k], cr[k], acc);
      d[u] = (i0 + u < rows) ? acc : 0.f;
    }
    reinterpret_cast<float4*>(out)[i0 / 4] = make_float4(d[0], d[1], d[2], d[3]);
  }
}

// qsim of the batch's queries against sets: one warp per (query, set).  Lane i
// keeps max_j T[b_j][i] (a coalesced 128-byte gather per stored vector); the
// warp sums the lanes with a fixed xor butterfly; parts add in ascending order.
struct ScanArgs {
  const float* T;
  int k1;
  const int32_t* codes;     // store codes [n_vecs]
  const int64_t* doc_off;   // original offsets
  int64_t n_sets;
  const int64_t* q_off;
  int q0, nq, max_np;
  const int64_t* cand_off;  // null: all sets
  const int64_t* cand_ids;
  float* out;
  int* status;
  unsigned long long* counter;  // chunk counter, zero at launch
};

// A warp takes 32 consecutive (query, set) pairs at a time, claimed in order
// from a counter: lane i loads pair i's set rows (one coalesced round for the
// 32), then the warp walks the pairs with the first 32 codes of the next pair
// already loaded, gathering kScanUnroll table rows per step, and lane i keeps
// pair i's score for one store.
constexpr int kScanCtasPerSm = 3;  // resident CTAs of 256 threads at the kernel's 80 registers
constexpr int kScanUnroll = 16;    // table rows in flight per warp

__global__ void __launch_bounds__(256, kScanCtasPerSm) qch_scan_kernel(ScanArgs a) {
  const int lane = threadIdx.x & 31;
  const bool all_sets = (a.cand_ids == nullptr);
  const int64_t base = all_sets ? 0 : a.cand_off[a.q0];
  const int64_t total = all_sets ? (int64_t)a.nq * a.n_sets : a.cand_off[a.q0 + a.nq] - base;
  const int64_t n_chunks = (total + 31) / 32;
  // chunks are claimed in order from a counter, so the warps in flight work on
  // neighbouring pairs: a few queries' tables at a time, which stay in L2 (a
  // fixed grid stride lets the warps drift apart until the tables in use exceed
  // L2 and every row is read from DRAM several times)
  for (;;) {
    unsigned long long claim = 0;
    if (lane == 0) claim = atomicAdd(a.counter, 1ull);
    const int64_t ch = (int64_t)__shfl_sync(0xffffffffu, claim, 0);
    if (ch >= n_chunks) break;
    const int64_t w0 = ch * 32;
    const int cnt = (int)min((int64_t)32, total - w0);
    // lane i: pair w0 + i (its query, set id, output slot, set rows)
    int my_b = a.q0;
    int64_t my_id = -1, my_out = 0, my_r0 = 0, my_r1 = 0;
    if (lane < cnt) {
      const int64_t w = w0 + lane;
      if (all_sets) {
        my_b = a.q0 + (int)(w / a.n_sets);
        my_id = w % a.n_sets;
        my_out = (int64_t)my_b * a.n_sets + my_id;
      } else {
        my_out = base + w;
        my_id = a.cand_ids[my_out];
        int lo = a.q0, hi = a.q0 + a.nq - 1;  // query owning this candidate
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.cand_off[mid] <= my_out) lo = mid; else hi = mid - 1;
        }
        my_b = lo;
      }
      if (my_id >= 0 && my_id < a.n_sets) {
        my_r0 = a.doc_off[my_id];
        my_r1 = a.doc_off[my_id + 1];
      }
    }
    // codes of the next pair's first 32 rows, lane-wise
    int next_code;
    {
      const int64_t r0 = __shfl_sync(0xffffffffu, (long long)my_r0, 0);
      const int64_t r1 = __shfl_sync(0xffffffffu, (long long)my_r1, 0);
      next_code = (r0 + lane < r1) ? a.codes[r0 + lane] : 0;
    }
    float my_score = 0.f;
    for (int i = 0; i < cnt; ++i) {
      const int b = __shfl_sync(0xffffffffu, my_b, i);
      const int64_t id = __shfl_sync(0xffffffffu, (long long)my_id, i);
      const int64_t r0 = __shfl_sync(0xffffffffu, (long long)my_r0, i);
      const int64_t r1 = __shfl_sync(0xffffffffu, (long long)my_r1, i);
      const int code0 = next_code;
      {
        const int nx = i + 1 < cnt ? i + 1 : i;
        const int64_t n0 = __shfl_sync(0xffffffffu, (long long)my_r0, nx);
        const int64_t n1 = __shfl_sync(0xffffffffu, (long long)my_r1, nx);
        if (i + 1 < cnt) next_code = (n0 + lane < n1) ? a.codes[n0 + lane] : 0;
      }
      float score;
      if (id < 0) {
        score = -INFINITY;
      } else if (id >= a.n_sets) {
        if (lane == 0) set_status(a.status, kDevBounds);
        score = __int_as_float(0x7fc00000);
      } else {
        const int np = (int)((a.q_off[b + 1] - a.q_off[b] + 31) / 32);
        score = 0.f;
        for (int pi = 0; pi < np; ++pi) {
          const float* Tp = a.T + (int64_t)((b - a.q0) * a.max_np + pi) * a.k1 * 32;
          float run = -INFINITY;
          for (int64_t j0 = r0; j0 < r1; j0 += 32) {
            const int nj = (int)min((int64_t)32, r1 - j0);
            const int my_code = j0 == r0 ? code0 : ((lane < nj) ? a.codes[j0 + lane] : 0);
            // kScanUnroll table rows in flight per step (the max is exact, so the
            // order of the rows does not matter); rows past nj repeat row 0
            for (int j = 0; j < nj; j += kScanUnroll) {
              float v[kScanUnroll];
#pragma unroll
              for (int u = 0; u < kScanUnroll; ++u) {
                const int cb = __shfl_sync(0xffffffffu, my_code, j + u < nj ? j + u : 0);
                v[u] = Tp[(int64_t)cb * 32 + lane];
              }
#pragma unroll
              for (int u = 0; u < kScanUnroll; ++u) run = fmaxf(run, v[u]);
            }
          }
          float sum = run;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          score = (pi == 0) ? sum : score + sum;
        }
      }
      if (lane == i) my_score = score;
    }
    if (lane < cnt) a.out[my_out] = my_score;
  }
}

}  // namespace

gem_status launch_assign_rows(const float* X, int64_t max_n, const int64_t* n_dev, const int32_t* rows,
                              const float* C, int k1, int32_t* codes, float* best, int n_sm, cudaStream_t st) {
  if (max_n == 0) return GEM_OK;
  const int64_t blocks = std::min<int64_t>((max_n + kAsgRows - 1) / kAsgRows, (int64_t)n_sm * 4);
  assign_kernel<<<(unsigned)blocks, kAsgThreads, 0, st>>>(X, max_n, n_dev, C, k1, codes, best, nullptr, 0, rows);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_assign(const float* X, int64_t n, const float* C, int k1, int32_t* codes, float* best,
                         cudaStream_t st) {
  if (n == 0) return GEM_OK;
  if (n >= kAssignTcMinRows && k1 >= kAssignTcMinCentroids) {
    int dev = 0, n_sm = 0;
    GEM_CUDA_TRY(cudaGetDevice(&dev));
    GEM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    return launch_assign_tc(X, n, C, k1, codes, best, n_sm, st);
  }
  const int64_t blocks = (n + kAsgRows - 1) / kAsgRows;
  if (blocks > INT32_MAX) return fail(GEM_ERR_INVALID, "too many vectors");
  assign_kernel<<<(unsigned)blocks, kAsgThreads, 0, st>>>(X, n, nullptr, C, k1, codes, best);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_assign_split(const float* X, int64_t n, const float* C, int k1, int32_t* codes,
                               unsigned long long* scratch, int n_sm, cudaStream_t st) {
  if (n == 0) return GEM_OK;
  const int64_t blocks = (n + kAsgRows - 1) / kAsgRows;
  const int c_tiles = (k1 + kAsgCents - 1) / kAsgCents;
  // enough CTAs for two waves of the SMs, whole centroid tiles per split
  const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(c_tiles, (2LL * n_sm + blocks - 1) / blocks));
  if (splits == 1 || !scratch || blocks > 65535) return launch_assign(X, n, C, k1, codes, nullptr, st);
  const int span = (c_tiles + splits - 1) / splits * kAsgCents;
  const int ny = (k1 + span - 1) / span;
  GEM_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * n, st));
  assign_kernel<<<dim3((unsigned)blocks, (unsigned)ny), kAsgThreads, 0, st>>>(X, n, nullptr, C, k1, codes, nullptr,
                                                                               scratch, span);
  GEM_CUDA_TRY(cudaGetLastError());
  assign_finish_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(scratch, n, codes);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  return GEM_OK;
}

gem_status launch_assign_dev_n(const float* X, int64_t max_n, const int64_t* n_dev, const float* C, int k1,
                               int32_t* codes, cudaStream_t st) {
  if (max_n == 0) return GEM_OK;
  const int64_t blocks = (max_n + kAsgRows - 1) / kAsgRows;
  assign_kernel<<<(unsigned)blocks, kAsgThreads, 0, st>>>(X, max_n, n_dev, C, k1, codes, nullptr);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_kmeans_step(const float* X, int64_t n, const int32_t* codes, double* sums, int* counts,
                              int k1, float* C, cudaStream_t st) {
  GEM_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)k1 * kDim, st));
  GEM_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)k1, st));
  const int g1 = (int)std::min<int64_t>((n * 32 + 255) / 256, 148 * 32);
  kmeans_accumulate_kernel<<<std::max(g1, 1), 256, 0, st>>>(X, n, codes, sums, counts);
  const int g2 = (int)std::min<int64_t>(((int64_t)k1 * 32 + 255) / 256, 148 * 32);
  kmeans_finalize_kernel<<<std::max(g2, 1), 256, 0, st>>>(sums, counts, k1, C);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  return GEM_OK;
}

gem_status launch_gather_rows(const float* src, const int64_t* rows, int64_t n, float* dst, cudaStream_t st) {
  const int g = (int)std::min<int64_t>((n * 32 + 255) / 256, 148 * 32);
  gather_rows_kernel<<<std::max(g, 1), 256, 0, st>>>(src, rows, n, dst);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_qch_tables(const gem_store* s, const int32_t* qcodes, const float* qvec, const int64_t* q_offsets,
                             int32_t n_queries, int max_np, float* T, cudaStream_t st) {
  if (n_queries == 0) return GEM_OK;
  dim3 tg((s->k1 + 255) / 256, n_queries * max_np);
  qch_table_kernel<<<tg, 256, 0, st>>>(s->d_codebook, s->k1, qcodes, qvec, q_offsets, 0, max_np, T);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_qch_scan_ids(const gem_store* s, const float* T, const int64_t* q_offsets, int32_t n_queries,
                               int max_np, const int64_t* cand_offsets, const int64_t* cand_ids, float* out,
                               int* status, unsigned long long* counter, cudaStream_t st) {
  if (n_queries == 0) return GEM_OK;
  GEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  ScanArgs a;
  a.T = T;
  a.k1 = s->k1;
  a.codes = s->d_codes;
  a.doc_off = s->d_offsets;
  a.n_sets = s->n_sets;
  a.q_off = q_offsets;
  a.q0 = 0;
  a.nq = n_queries;
  a.max_np = max_np;
  a.cand_off = cand_offsets;
  a.cand_ids = cand_ids;
  a.out = out;
  a.status = status;
  a.counter = counter;
  qch_scan_kernel<<<s->n_sm * kScanCtasPerSm, 256, 0, st>>>(a);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

gem_status launch_qch(const gem_store* s, gem_workspace* w, const float* q, const int64_t* q_offsets,
                      int32_t n_queries, int64_t n_q_rows, const int64_t* cand_offsets,
                      const int64_t* cand_ids, float* est, cudaStream_t st) {
  const int k1 = s->k1;
  const bool asym = w->qch_form == GEM_QCH_ASYMMETRIC;
  // query codes NN(q_i) (the symmetric form)
  if (!asym) {
    gem_status r = launch_assign_split(q, n_q_rows, s->d_codebook, k1, w->d_qcodes, w->d_assign_key, s->n_sm, st);
    if (r != GEM_OK) return r;
  }
  const int max_np = (w->max_q_len + 31) / 32;
  const int q_per_batch = std::max(1, w->table_parts / max_np);
  for (int q0 = 0; q0 < n_queries; q0 += q_per_batch) {
    const int nq = std::min(q_per_batch, n_queries - q0);
    dim3 tg((k1 + 255) / 256, nq * max_np);
    qch_table_kernel<<<tg, 256, 0, st>>>(s->d_codebook, k1, w->d_qcodes, asym ? q : nullptr, q_offsets, q0, max_np,
                                         w->d_tables);
    ScanArgs a;
    a.T = w->d_tables;
    a.k1 = k1;
    a.codes = s->d_codes;
    a.doc_off = s->d_offsets;
    a.n_sets = s->n_sets;
    a.q_off = q_offsets;
    a.q0 = q0;
    a.nq = nq;
    a.max_np = max_np;
    a.cand_off = cand_offsets;
    a.cand_ids = cand_ids;
    a.out = est;
    a.status = w->d_status;
    a.counter = reinterpret_cast<unsigned long long*>(w->d_unit_counter);
    GEM_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st));
    qch_scan_kernel<<<s->n_sm * kScanCtasPerSm, 256, 0, st>>>(a);
    GEM_CUDA_TRY(cudaGetLastError());
    note_launches(2);
  }
  return GEM_OK;
}

}  // namespace gem
