// Index persistence: the resident index written to and read from a host
// blob, so a serving process restarts without rebuilding it.
//
// Blob layout (little-endian): "SEDEFIDX", u32 version (1), u32 k, u64 nrec,
// u32 nseq, u32 reserved, i64 seq_off[nseq+1], u64 rec[nrec] (by position),
// u64 sorted[nrec] (by hash, position), u32 off[4^k + 1], u64 checksum of
// everything before it.
#include <cstring>

#include "common.cuh"

namespace {

constexpr char kMagic[8] = {'S', 'E', 'D', 'E', 'F', 'I', 'D', 'X'};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeader = 8 + 4 + 4 + 8 + 4 + 4;

int64_t blob_size(int k, int64_t nrec, int nseq) {
  return (int64_t)kHeader + 8 * (int64_t)(nseq + 1) + 16 * nrec +
         4 * ((int64_t(1) << (2 * k)) + 1) + 8;
}

uint64_t checksum(const unsigned char* p, size_t n) {
  uint64_t h = 0x9E3779B97F4A7C15ull;
  size_t x = 0;
  for (; x + 8 <= n; x += 8) {
    uint64_t w;
    std::memcpy(&w, p + x, 8);
    h = (h ^ w) * 0x100000001B3ull;
    h ^= h >> 29;
  }
  for (; x < n; ++x) h = (h ^ p[x]) * 0x100000001B3ull;
  return h;
}

}  // namespace

using namespace sedef;

extern "C" {

int64_t sedef_index_blob_size(int32_t k, int64_t nrec, int32_t nseq) {
  if (k < 2 || k > 15 || nrec < 0 || nseq < 0) return -1;
  return blob_size(k, nrec, nseq);
}

int sedef_index_save(sedef_ctx* ctx, const uint64_t* d_rec, const uint64_t* d_sorted,
                     const uint32_t* d_off, int64_t nrec, int32_t k, const int64_t* h_seq_off,
                     int32_t nseq, void* h_blob, int64_t cap) {
  if (!ctx || !h_blob || !h_seq_off || nseq < 0 || nrec < 0 || k < 2 || k > 15)
    return fail(SEDEF_ERR_INVALID, "sedef_index_save: bad arguments");
  if ((nrec > 0 && (!d_rec || !d_sorted)) || !d_off)
    return fail(SEDEF_ERR_INVALID, "sedef_index_save: NULL device array");
  const int64_t need = blob_size(k, nrec, nseq);
  if (cap < need) return fail(SEDEF_ERR_CAPACITY, "sedef_index_save: blob buffer too small");
  SEDEF_CUDA(cudaSetDevice(ctx_device(ctx)));
  unsigned char* b = (unsigned char*)h_blob;
  std::memcpy(b, kMagic, 8);
  const uint32_t ver = kVersion, kk = (uint32_t)k, ns = (uint32_t)nseq, zero = 0;
  const uint64_t nr = (uint64_t)nrec;
  std::memcpy(b + 8, &ver, 4);
  std::memcpy(b + 12, &kk, 4);
  std::memcpy(b + 16, &nr, 8);
  std::memcpy(b + 24, &ns, 4);
  std::memcpy(b + 28, &zero, 4);
  size_t o = kHeader;
  std::memcpy(b + o, h_seq_off, 8 * (size_t)(nseq + 1));
  o += 8 * (size_t)(nseq + 1);
  cudaStream_t st = ctx_stream(ctx);
  if (nrec > 0) {
    SEDEF_CUDA(cudaMemcpyAsync(b + o, d_rec, 8 * (size_t)nrec, cudaMemcpyDeviceToHost, st));
    o += 8 * (size_t)nrec;
    SEDEF_CUDA(cudaMemcpyAsync(b + o, d_sorted, 8 * (size_t)nrec, cudaMemcpyDeviceToHost, st));
    o += 8 * (size_t)nrec;
  }
  const size_t noff = 4 * ((size_t(1) << (2 * k)) + 1);
  SEDEF_CUDA(cudaMemcpyAsync(b + o, d_off, noff, cudaMemcpyDeviceToHost, st));
  o += noff;
  SEDEF_CUDA(cudaStreamSynchronize(st));
  const uint64_t c = checksum(b, o);
  std::memcpy(b + o, &c, 8);
  return SEDEF_OK;
}

int sedef_index_blob_info(const void* h_blob, int64_t size, int32_t* k, int64_t* nrec,
                          int32_t* nseq) {
  const unsigned char* b = (const unsigned char*)h_blob;
  if (!b || size < (int64_t)kHeader) return fail(SEDEF_ERR_INVALID, "index blob too short");
  if (std::memcmp(b, kMagic, 8) != 0) return fail(SEDEF_ERR_INVALID, "not an index blob");
  uint32_t ver, kk, ns;
  uint64_t nr;
  std::memcpy(&ver, b + 8, 4);
  std::memcpy(&kk, b + 12, 4);
  std::memcpy(&nr, b + 16, 8);
  std::memcpy(&ns, b + 24, 4);
  if (ver != kVersion) return fail(SEDEF_ERR_UNSUPPORTED, "index blob version");
  if (kk < 2 || kk > 15 || nr >= (uint64_t(1) << 32) || ns > (1u << 30))
    return fail(SEDEF_ERR_INVALID, "index blob header out of range");
  if (size != blob_size((int)kk, (int64_t)nr, (int)ns))
    return fail(SEDEF_ERR_INVALID, "index blob size does not match its header");
  const uint64_t c = checksum(b, (size_t)size - 8);
  uint64_t stored;
  std::memcpy(&stored, b + size - 8, 8);
  if (c != stored) return fail(SEDEF_ERR_INVALID, "index blob checksum mismatch");
  if (k) *k = (int32_t)kk;
  if (nrec) *nrec = (int64_t)nr;
  if (nseq) *nseq = (int32_t)ns;
  return SEDEF_OK;
}

int sedef_index_load(sedef_ctx* ctx, const void* h_blob, int64_t size, int64_t* h_seq_off,
                     int32_t nseq_cap, uint64_t* d_rec, uint64_t* d_sorted, uint32_t* d_off,
                     int64_t rec_cap) {
  int32_t k = 0, nseq = 0;
  int64_t nrec = 0;
  SEDEF_TRY(sedef_index_blob_info(h_blob, size, &k, &nrec, &nseq));
  if (!ctx || !h_seq_off || nseq > nseq_cap || nrec > rec_cap || !d_off ||
      (nrec > 0 && (!d_rec || !d_sorted)))
    return fail(SEDEF_ERR_INVALID, "sedef_index_load: buffers too small or NULL");
  SEDEF_CUDA(cudaSetDevice(ctx_device(ctx)));
  const unsigned char* b = (const unsigned char*)h_blob;
  size_t o = kHeader;
  std::memcpy(h_seq_off, b + o, 8 * (size_t)(nseq + 1));
  o += 8 * (size_t)(nseq + 1);
  cudaStream_t st = ctx_stream(ctx);
  if (nrec > 0) {
    SEDEF_CUDA(cudaMemcpyAsync(d_rec, b + o, 8 * (size_t)nrec, cudaMemcpyHostToDevice, st));
    o += 8 * (size_t)nrec;
    SEDEF_CUDA(cudaMemcpyAsync(d_sorted, b + o, 8 * (size_t)nrec, cudaMemcpyHostToDevice, st));
    o += 8 * (size_t)nrec;
  }
  SEDEF_CUDA(cudaMemcpyAsync(d_off, b + o, 4 * ((size_t(1) << (2 * k)) + 1),
                             cudaMemcpyHostToDevice, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // extern "C"
