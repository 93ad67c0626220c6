// a3 index: device-wide exclusive scan, stable LSD radix sort of uint64 keys
// (optionally with uint32 payloads) over a chosen bit range, and the offset
// table over all 4^k hashes.
//
// The sort takes 8-bit digits over only the significant bits (2k = 24 hash
// bits for the index: 3 passes).  Each pass: per-tile digit histograms
// (4096 keys per tile), one scan over the digit-major histogram array, and a
// scatter in which every warp ranks its keys with __match_any_sync, the CTA
// stages the tile in shared memory in digit order, and consecutive threads
// write consecutive output addresses (coalesced runs per digit).
#include "common.cuh"

namespace sedef {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_scan_tile(uint32_t (&v)[kScanItems], int* tmp,
                                                    uint32_t* total) {
  uint32_t s = 0;
#pragma unroll
  for (int x = 0; x < kScanItems; ++x) s += v[x];
  int tot;
  const int ex = block_exclusive_sum((int)s, tmp, &tot);
  uint32_t run = (uint32_t)ex;
#pragma unroll
  for (int x = 0; x < kScanItems; ++x) {
    const uint32_t t = v[x];
    v[x] = run;
    run += t;
  }
  *total = (uint32_t)tot;
  return (uint32_t)ex;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              int64_t n, uint32_t* __restrict__ sums) {
  __shared__ int tmp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int x = 0; x < kScanItems; ++x)
    if (base + x < n) s += in[base + x];
  int tot;
  block_exclusive_sum((int)s, tmp, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = (uint32_t)tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out, int64_t n,
                                                             const uint32_t* __restrict__ tile_off,
                                                             uint32_t* __restrict__ total) {
  __shared__ int tmp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
#pragma unroll
  for (int x = 0; x < kScanItems; ++x) v[x] = (base + x < n) ? in[base + x] : 0u;
  uint32_t tot;
  block_scan_tile(v, tmp, &tot);
  const uint32_t add = tile_off ? tile_off[blockIdx.x] : 0u;
#pragma unroll
  for (int x = 0; x < kScanItems; ++x)
    if (base + x < n) out[base + x] = v[x] + add;
  if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = add + tot;
}

// ------------------------------------------------------------- radix sort --

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ uint32_t digit_of(uint64_t key, int shift, uint32_t dmask) {
  return (uint32_t)(key >> shift) & dmask;
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                        int shift, uint32_t dmask, int64_t ntiles,
                                                        uint32_t* __restrict__ hist,
                                                        const uint32_t* __restrict__ dn) {
  __shared__ uint32_t h[256];
  n = live_n(n, dn);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = tile * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsItems; ++r) {
      const int64_t idx = base + (int64_t)r * kRsThreads + threadIdx.x;
      if (idx < n) atomicAdd(&h[digit_of(keys[idx], shift, dmask)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
  }
}

struct RsSmem {
  uint32_t wcnt[kRsWarps][256];
  uint32_t dstart[256];
  uint32_t gofs[256];
  int tmp[33];
  uint64_t keys[kRsTile];
  uint32_t vals[kRsTile];
};

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint64_t* __restrict__ kout,
                                                           uint32_t* __restrict__ vout, int64_t n,
                                                           int shift, uint32_t dmask, int64_t ntiles,
                                                           const uint32_t* __restrict__ hoff,
                                                           int iota_vals,
                                                           const uint32_t* __restrict__ dn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  n = live_n(n, dn);
  RsSmem& S = *reinterpret_cast<RsSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool has_vals = (vout != nullptr);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    for (int x = threadIdx.x; x < kRsWarps * 256; x += kRsThreads) (&S.wcnt[0][0])[x] = 0;
    __syncthreads();
    const int64_t base = tile * kRsTile + (int64_t)warp * (32 * kRsItems);
    uint64_t key[kRsItems];
    uint32_t val[kRsItems];
    uint32_t dig[kRsItems];
    uint32_t loc[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      const bool ok = idx < n;
      key[r] = ok ? kin[idx] : 0ull;
      if (has_vals) val[r] = ok ? (iota_vals ? (uint32_t)idx : vin[idx]) : 0u;
      dig[r] = ok ? digit_of(key[r], shift, dmask) : 256u;
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
      const uint32_t d = dig[r];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t rank = __popc(peers & lt);
      const uint32_t before = (d < 256) ? S.wcnt[warp][d] : 0u;
      __syncwarp();
      if (d < 256 && rank == 0) S.wcnt[warp][d] = before + __popc(peers);
      __syncwarp();
      loc[r] = before + rank;
    }
    __syncthreads();
    {
      const int d = threadIdx.x;  // 256 threads = 256 digits
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t c = S.wcnt[w][d];
        S.wcnt[w][d] = run;
        run += c;
      }
      int tot;
      const int ex = block_exclusive_sum((int)run, S.tmp, &tot);
      S.dstart[d] = (uint32_t)ex;
      S.gofs[d] = hoff[(int64_t)d * ntiles + tile];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
      const uint32_t d = dig[r];
      if (d < 256) {
        const uint32_t p = S.dstart[d] + S.wcnt[warp][d] + loc[r];
        S.keys[p] = key[r];
        if (has_vals) S.vals[p] = val[r];
      }
    }
    __syncthreads();
    const int64_t cnt = min((int64_t)kRsTile, n - tile * kRsTile);
    for (int x = threadIdx.x; x < cnt; x += kRsThreads) {
      const uint64_t kk = S.keys[x];
      const uint32_t d = digit_of(kk, shift, dmask);
      const uint32_t o = S.gofs[d] + (uint32_t)x - S.dstart[d];
      kout[o] = kk;
      if (has_vals) vout[o] = S.vals[x];
    }
  }
}

// --------------------------------------------------------- offset table ----

constexpr int kOffChunk = 4096;

__global__ void __launch_bounds__(256) k_offsets(const uint64_t* __restrict__ sorted, int64_t n,
                                                 int64_t nhash, uint32_t* __restrict__ off,
                                                 const uint32_t* __restrict__ dn) {
  n = live_n(n, dn);
  __shared__ uint32_t cnt[kOffChunk];
  __shared__ int64_t rng[2];
  __shared__ int tmp[33];
  const int64_t X0 = (int64_t)blockIdx.x * kOffChunk;
  for (int x = threadIdx.x; x < kOffChunk; x += 256) cnt[x] = 0;
  if (threadIdx.x < 2) {
    const uint64_t key = (uint64_t)(X0 + (threadIdx.x ? kOffChunk : 0));
    rng[threadIdx.x] = lower_bound_by(sorted, 0, n, key, [](uint64_t r) { return r >> 33; });
  }
  __syncthreads();
  const int64_t R0 = rng[0], R1 = rng[1];
  for (int64_t r = R0 + threadIdx.x; r < R1; r += 256)
    atomicAdd(&cnt[(int)((sorted[r] >> 33) - (uint64_t)X0)], 1u);
  __syncthreads();
  // exclusive scan of cnt[0..4096): 16 consecutive items per thread
  uint32_t v[16];
  uint32_t s = 0;
#pragma unroll
  for (int x = 0; x < 16; ++x) {
    v[x] = cnt[threadIdx.x * 16 + x];
    s += v[x];
  }
  int tot;
  const int ex = block_exclusive_sum((int)s, tmp, &tot);
  uint32_t run = (uint32_t)(R0 + ex);
#pragma unroll
  for (int x = 0; x < 16; ++x) {
    const int64_t h = X0 + threadIdx.x * 16 + x;
    if (h < nhash) off[h] = run;
    run += v[x];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off[nhash] = (uint32_t)n;
}

}  // namespace

int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total) {
  cudaStream_t st = ctx_stream(ctx);
  if (n <= 0) {
    if (d_total) SEDEF_CUDA(cudaMemsetAsync(d_total, 0, 4, st));
    return SEDEF_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    SEDEF_KERNEL(ctx, "k_scan_tiles", k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, d_total));
    return SEDEF_OK;
  }
  uint32_t* sums = (uint32_t*)ctx_alloc(ctx, (size_t)tiles * 4);
  uint32_t* soff = (uint32_t*)ctx_alloc(ctx, (size_t)tiles * 4);
  if (!sums || !soff) return SEDEF_ERR_OOM;
  SEDEF_KERNEL(ctx, "k_scan_reduce", k_scan_reduce<<<(int)tiles, kScanThreads, 0, st>>>(in, n, sums));
  SEDEF_TRY(scan_exclusive_u32(ctx, sums, soff, tiles, nullptr));
  SEDEF_KERNEL(ctx, "k_scan_tiles",
               k_scan_tiles<<<(int)tiles, kScanThreads, 0, st>>>(in, out, n, soff, d_total));
  return SEDEF_OK;
}

int radix_sort_u64(sedef_ctx* ctx, const uint64_t* keys_in, const uint32_t* vals_in,
                   uint64_t* keys_out, uint32_t* vals_out, int64_t n, int bit_lo, int bit_hi,
                   const uint32_t* dn) {
  cudaStream_t st = ctx_stream(ctx);
  if (n <= 0) return SEDEF_OK;
  const int passes = (bit_hi - bit_lo + 7) / 8;
  const bool iota = (vals_in == nullptr && vals_out != nullptr);
  if (passes <= 0) {
    SEDEF_CUDA(cudaMemcpyAsync(keys_out, keys_in, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
    return SEDEF_OK;
  }
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  uint32_t* hist = (uint32_t*)ctx_alloc(ctx, (size_t)ntiles * 256 * 4);
  uint32_t* hoff = (uint32_t*)ctx_alloc(ctx, (size_t)ntiles * 256 * 4);
  uint64_t* ktmp = (uint64_t*)ctx_alloc(ctx, (size_t)n * 8);
  uint32_t* vtmp = vals_out ? (uint32_t*)ctx_alloc(ctx, (size_t)n * 4) : nullptr;
  if (!hist || !hoff || !ktmp || (vals_out && !vtmp)) return SEDEF_ERR_OOM;
  const size_t smem = sizeof(RsSmem);
  SEDEF_TRY(ensure_smem_attr((const void*)k_rs_scatter, smem));
  int64_t grid = ntiles;
  const int64_t maxgrid = (int64_t)ctx_sm_count(ctx) * 3;
  if (grid > maxgrid) grid = maxgrid;
  int64_t hgrid = ntiles < (int64_t)ctx_sm_count(ctx) * 8 ? ntiles : (int64_t)ctx_sm_count(ctx) * 8;
  const uint64_t* ksrc = keys_in;
  const uint32_t* vsrc = vals_in;
  for (int p = 0; p < passes; ++p) {
    const int shift = bit_lo + 8 * p;
    const int bits = (bit_hi - shift) < 8 ? (bit_hi - shift) : 8;
    const uint32_t dmask = (1u << bits) - 1u;
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint64_t* kdst = to_out ? keys_out : ktmp;
    uint32_t* vdst = vals_out ? (to_out ? vals_out : vtmp) : nullptr;
    SEDEF_KERNEL(ctx, "k_rs_hist",
                 k_rs_hist<<<(int)hgrid, kRsThreads, 0, st>>>(ksrc, n, shift, dmask, ntiles, hist, dn));
    SEDEF_TRY(scan_exclusive_u32(ctx, hist, hoff, ntiles * 256, nullptr));
    SEDEF_KERNEL(ctx, "k_rs_scatter",
                 k_rs_scatter<<<(int)grid, kRsThreads, smem, st>>>(ksrc, vsrc, kdst, vdst, n, shift,
                                                                   dmask, ntiles, hoff,
                                                                   (p == 0 && iota) ? 1 : 0, dn));
    ksrc = kdst;
    vsrc = vdst;
  }
  return SEDEF_OK;
}

int build_offsets(sedef_ctx* ctx, const uint64_t* sorted, int64_t n, int k, uint32_t* off,
                  const uint32_t* dn) {
  cudaStream_t st = ctx_stream(ctx);
  const int64_t nhash = int64_t(1) << (2 * k);
  const int64_t chunks = (nhash + kOffChunk - 1) / kOffChunk;
  SEDEF_KERNEL(ctx, "k_offsets", k_offsets<<<(int)chunks, 256, 0, st>>>(sorted, n, nhash, off, dn));
  return SEDEF_OK;
}

}  // namespace sedef
