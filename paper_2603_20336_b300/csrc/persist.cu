// Store persistence: gem_store_save writes what a store cannot re-derive (the
// set offsets, the FP32 vectors, C_quant, C_index and the deletion bitmap) to
// one file; gem_store_load reads it back and rebuilds everything else with the
// library's own deterministic kernels (bf16 / E4M3 copies, padded layout, codes,
// index codes, cluster member lists), so a loaded store scores exactly as the
// saved one did.
//
// Layout (little-endian):
//   header   "GEMSTORE", u32 version = 1, u32 dim = 128, i64 n_sets, i64 n_vecs,
//            i32 k1, i32 k2, u32 has_deleted, u32 reserved = 0
//   i64      offsets [n_sets + 1]
//   f32      vectors [n_vecs x 128]
//   f32      C_quant [k1 x 128]          (k1 > 0)
//   f32      C_index [k2 x 128]          (k2 > 0)
//   u32      deleted [ceil(n_sets / 32)] (has_deleted)
//   trailer  "GEMEND01"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace gem {
namespace {

constexpr char kMagic[8] = {'G', 'E', 'M', 'S', 'T', 'O', 'R', 'E'};
constexpr char kTrailer[8] = {'G', 'E', 'M', 'E', 'N', 'D', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr int64_t kChunkFloats = (int64_t)1 << 24;  // 64 MB per host staging step

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t dim;
  int64_t n_sets;
  int64_t n_vecs;
  int32_t k1;
  int32_t k2;
  uint32_t has_deleted;
  uint32_t reserved;
};
static_assert(sizeof(FileHeader) == 48, "file header layout");

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

bool put(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

// device -> file through a host buffer, kChunkFloats at a time
gem_status put_device(FILE* f, const float* d, int64_t n, cudaStream_t st) {
  std::vector<float> h((size_t)std::min<int64_t>(n, kChunkFloats));
  for (int64_t i = 0; i < n; i += kChunkFloats) {
    const int64_t c = std::min<int64_t>(kChunkFloats, n - i);
    GEM_CUDA_TRY(cudaMemcpyAsync(h.data(), d + i, sizeof(float) * c, cudaMemcpyDeviceToHost, st));
    GEM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!put(f, h.data(), sizeof(float) * c)) return fail(GEM_ERR_INVALID, "write failed");
  }
  return GEM_OK;
}

// host array -> new device array of n floats (caller frees)
gem_status to_device(const std::vector<float>& h, float** out, cudaStream_t st) {
  *out = nullptr;
  GEM_CUDA_TRY(cudaMalloc(out, sizeof(float) * std::max<size_t>(h.size(), 1)));
  GEM_CUDA_TRY(cudaMemcpyAsync(*out, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
  GEM_CUDA_TRY(cudaStreamSynchronize(st));
  return GEM_OK;
}

// n floats from the file into h; false when the file is short
bool get_floats(FILE* f, int64_t n, std::vector<float>& h) {
  h.resize((size_t)n);
  return get(f, h.data(), sizeof(float) * n);
}

bool all_finite(const std::vector<float>& h) {
  for (float x : h)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace
}  // namespace gem

using namespace gem;

extern "C" gem_status gem_store_save(const gem_store* s, const char* path, void* stream) {
  GEM_NVTX_RANGE("gem_store_save");
  if (!s || !path) return fail(GEM_ERR_INVALID, "NULL argument");
  if (!s->d_f32) return fail(GEM_ERR_STATE, "saving needs the FP32 copy (GEM_KEEP_F32)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  File file;
  file.f = fopen(path, "wb");
  if (!file.f) return fail(GEM_ERR_INVALID, std::string("cannot open for writing: ") + path);
  FileHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.dim = kDim;
  h.n_sets = s->n_sets;
  h.n_vecs = s->n_vecs;
  h.k1 = s->d_codebook ? s->k1 : 0;
  h.k2 = s->d_cindex ? s->k2 : 0;
  h.has_deleted = s->d_dead ? 1u : 0u;
  if (!put(file.f, &h, sizeof(h)) || !put(file.f, s->h_offsets.data(), sizeof(int64_t) * (s->n_sets + 1)))
    return fail(GEM_ERR_INVALID, "write failed");
  gem_status r = put_device(file.f, s->d_f32, s->n_vecs * kDim, st);
  if (r == GEM_OK && h.k1) r = put_device(file.f, s->d_codebook, (int64_t)h.k1 * kDim, st);
  if (r == GEM_OK && h.k2) r = put_device(file.f, s->d_cindex, (int64_t)h.k2 * kDim, st);
  if (r != GEM_OK) return r;
  if (h.has_deleted) {
    std::vector<uint32_t> bits((size_t)((s->n_sets + 31) / 32));
    GEM_CUDA_TRY(cudaMemcpyAsync(bits.data(), s->d_dead, sizeof(uint32_t) * bits.size(), cudaMemcpyDeviceToHost, st));
    GEM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!put(file.f, bits.data(), sizeof(uint32_t) * bits.size())) return fail(GEM_ERR_INVALID, "write failed");
  }
  if (!put(file.f, kTrailer, 8)) return fail(GEM_ERR_INVALID, "write failed");
  if (fclose(file.f) != 0) {
    file.f = nullptr;
    return fail(GEM_ERR_INVALID, "write failed");
  }
  file.f = nullptr;
  return GEM_OK;
}

extern "C" gem_status gem_store_load(const char* path, uint32_t keep_mask, void* stream, gem_store** out) {
  GEM_NVTX_RANGE("gem_store_load");
  if (!path || !out) return fail(GEM_ERR_INVALID, "NULL argument");
  *out = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  File file;
  file.f = fopen(path, "rb");
  if (!file.f) return fail(GEM_ERR_INVALID, std::string("cannot open: ") + path);
  FileHeader h{};
  if (!get(file.f, &h, sizeof(h)) || std::memcmp(h.magic, kMagic, 8) != 0)
    return fail(GEM_ERR_INVALID, "not a store file");
  if (h.version != kVersion) return fail(GEM_ERR_INVALID, "unknown store file version");
  if (h.dim != (uint32_t)kDim || h.n_sets < 1 || h.n_sets >= ((int64_t)1 << 31) || h.n_vecs < h.n_sets ||
      h.n_vecs > ((int64_t)1 << 36) || h.k1 < 0 || h.k2 < 0 || h.k2 > (1 << 18) || h.has_deleted > 1)
    return fail(GEM_ERR_INVALID, "corrupt store header");
  if ((h.k1 || h.k2) && !(keep_mask & GEM_KEEP_F32))
    return fail(GEM_ERR_INVALID, "the file has a codebook: codes are re-assigned from the FP32 copy (GEM_KEEP_F32)");
  const int64_t words = (h.n_sets + 31) / 32;
  // the file must be exactly as long as its header says
  const long long expect = (long long)sizeof(h) + 8LL * (h.n_sets + 1) + 4LL * h.n_vecs * kDim +
                           4LL * ((int64_t)h.k1 + h.k2) * kDim + (h.has_deleted ? 4LL * words : 0) + 8;
  if (fseeko(file.f, 0, SEEK_END) != 0 || (long long)ftello(file.f) != expect)
    return fail(GEM_ERR_INVALID, "store file truncated or corrupt");
  fseeko(file.f, (off_t)sizeof(h), SEEK_SET);
  std::vector<int64_t> off((size_t)(h.n_sets + 1));
  if (!get(file.f, off.data(), sizeof(int64_t) * off.size())) return fail(GEM_ERR_INVALID, "store file truncated");
  if (off[0] != 0 || off[h.n_sets] != h.n_vecs) return fail(GEM_ERR_INVALID, "corrupt store offsets");
  for (int64_t i = 0; i < h.n_sets; ++i)
    if (off[i + 1] <= off[i]) return fail(GEM_ERR_INVALID, "corrupt store offsets");
  // every float array is read and checked on the host before any device work:
  // a NaN or an infinity in the vectors or the centroids refuses the file
  std::vector<float> cq, ci;
  gem_store* s = nullptr;
  {
    std::vector<float> vecs;
    if (!get_floats(file.f, h.n_vecs * kDim, vecs) || !get_floats(file.f, (int64_t)h.k1 * kDim, cq) ||
        !get_floats(file.f, (int64_t)h.k2 * kDim, ci))
      return fail(GEM_ERR_INVALID, "store file truncated");
    if (!all_finite(vecs)) return fail(GEM_ERR_INVALID, "store file holds a non-finite vector component");
    if (!all_finite(cq) || !all_finite(ci)) return fail(GEM_ERR_INVALID, "store file holds a non-finite centroid");
    gem_status r = gem_store_create(vecs.data(), off.data(), h.n_sets, kDim, keep_mask, 1, stream, &s);
    if (r != GEM_OK) return r;
  }
  auto attach = [&](int32_t k, bool quant) -> gem_status {
    float* d = nullptr;
    gem_status r = to_device(quant ? cq : ci, &d, st);
    if (r == GEM_OK)
      r = quant ? gem_store_set_codebook(s, d, k, stream) : gem_store_set_index_centroids(s, d, k, stream);
    if (r == GEM_OK) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) r = cuda_fail(e, "attaching centroids");
    }
    if (d) cudaFree(d);
    return r;
  };
  gem_status r = GEM_OK;
  if (h.k1) r = attach(h.k1, true);
  if (r == GEM_OK && h.k2) r = attach(h.k2, false);
  if (r == GEM_OK && h.has_deleted) {
    std::vector<uint32_t> bits((size_t)words + 1, 0u);  // one extra word: the range-check counter
    if (!get(file.f, bits.data(), sizeof(uint32_t) * words)) {
      r = fail(GEM_ERR_INVALID, "store file truncated");
    } else {
      cudaError_t e = cudaMalloc(&s->d_dead, sizeof(uint32_t) * bits.size());
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_dead, bits.data(), sizeof(uint32_t) * bits.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) r = cuda_fail(e, "deletion bitmap");
    }
  }
  char tail[8] = {};
  if (r == GEM_OK && (!get(file.f, tail, 8) || std::memcmp(tail, kTrailer, 8) != 0))
    r = fail(GEM_ERR_INVALID, "store file trailer missing");
  if (r != GEM_OK) {
    gem_store_destroy(s);
    return r;
  }
  *out = s;
  return GEM_OK;
}

extern "C" gem_status gem_store_codebook_sizes(const gem_store* s, int32_t* k1, int32_t* k2) {
  if (!s) return fail(GEM_ERR_INVALID, "store is NULL");
  if (k1) *k1 = s->d_codebook ? s->k1 : 0;
  if (k2) *k2 = s->d_cindex ? s->k2 : 0;
  return GEM_OK;
}
