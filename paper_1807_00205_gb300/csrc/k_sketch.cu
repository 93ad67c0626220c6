// a1 pack and a2 sketch kernels.
//
// pack: 16 input bytes per thread (one 128-bit load), one packed word per
// thread and one mask/N word per lane pair (warp shuffle), so every global
// access is coalesced.  HBM-bound: 1 B read + 0.5 B written per base.
//
// sketch: one CTA per tile of 2048 consecutive windows.  The packed words,
// mask and N bits of the tile (plus halo) are staged in shared memory; every
// thread computes the canonical k-mer hashes of 8-9 positions from two 32-bit
// words (forward code by bit reversal, reverse complement by complementing),
// then the rightmost minimum of its 9 windows with a van Herk / Gil-Werman
// split (suffix minima, a shared middle, prefix minima), and keeps a window's
// argmin when it differs from the previous window's (winnowing argmins are
// non-decreasing, so this emits each selected position once, in order).  The
// window keys are (hash, reversed slot): 32 bits when the hash has at most 24
// bits and a thread's windows span at most 128 slots, else 64.  The eager
// pass writes its records in the same pass, finding each tile's offset by a
// decoupled look-back over the tiles taken before it; the planned (graph)
// pass and the allocation-free call count, scan and write instead.
#include <cstring>

#include "common.cuh"

namespace sedef {

namespace {

__device__ __forceinline__ void classify(uint32_t b, uint32_t& code, uint32_t& masked,
                                         uint32_t& isn) {
  const uint32_t l = b | 0x20u;
  const bool acgt = (l == 'a') | (l == 'c') | (l == 'g') | (l == 't');
  code = acgt ? (((l >> 1) ^ (l >> 2)) & 3u) : 0u;  // a=0 c=1 g=2 t=3
  masked = (b >= 'a' && b <= 'z') ? 1u : 0u;
  isn = acgt ? 0u : 1u;
}

template <bool kAligned>
__global__ void __launch_bounds__(256) k_pack(const uint8_t* __restrict__ seq, int64_t n,
                                              uint32_t* __restrict__ packed,
                                              uint32_t* __restrict__ mask,
                                              uint32_t* __restrict__ nbits) {
  const int64_t nchunk = (n + 15) >> 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nchunk; base += stride) {
    const int64_t c = base + threadIdx.x;
    uint32_t word = 0, m16 = 0, n16 = 0;
    if (c < nchunk) {
      const int64_t p0 = c << 4;
      uint32_t v[4];
      if (kAligned && p0 + 16 <= n) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(seq + p0));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
#pragma unroll
        for (int x = 0; x < 16; ++x) {
          uint32_t code, ms, isn;
          classify((v[x >> 2] >> (8 * (x & 3))) & 0xFFu, code, ms, isn);
          word |= code << (2 * x);
          m16 |= ms << x;
          n16 |= isn << x;
        }
      } else {
        for (int x = 0; x < 16; ++x) {
          if (p0 + x >= n) break;
          uint32_t code, ms, isn;
          classify(seq[p0 + x], code, ms, isn);
          word |= code << (2 * x);
          m16 |= ms << x;
          n16 |= isn << x;
        }
      }
    }
    const uint32_t om = __shfl_down_sync(0xffffffffu, m16, 1);
    const uint32_t on = __shfl_down_sync(0xffffffffu, n16, 1);
    if (c < nchunk) {
      packed[c] = word;
      if ((c & 1) == 0) {
        mask[c >> 1] = m16 | (om << 16);
        nbits[c >> 1] = n16 | (on << 16);
      }
    }
  }
}

constexpr int kSkThreads = 256;
constexpr int kSkWPT = 8;                          // windows per thread
constexpr int kSkTile = kSkThreads * kSkWPT;       // windows per CTA
constexpr int kSkMaxW = 256;
constexpr int kSkHashes = kSkTile + kSkMaxW;       // hash slots (tile + halo)
// Hash slot x lives at x + x/8: a thread's windows start kSkWPT = 8 slots
// after its neighbour's, and the padding turns that stride into 9 words, so
// the lanes of a warp read distinct banks.
constexpr int kSkHashesP = kSkHashes + kSkHashes / 8 + 1;
__device__ __forceinline__ int hslot(int x) { return x + (x >> 3); }
constexpr int kSkWords16 = (kSkHashes + 16) / 16 + 4;
constexpr int kSkWords32 = (kSkHashes + 16) / 32 + 4;

// Canonical hash of the k-mer whose first base is bit-offset `sh` into the
// 64-bit pair (lo, hi) of packed words.  Returns kInfHash for an ineligible
// k-mer (N inside, too few unmasked bases, palindrome).
__device__ __forceinline__ uint32_t bijective_hash(uint32_t x, int k, uint32_t M) {
  // A permutation of [0, 4^k): xor-shift-right and odd multipliers, all
  // modulo 2^(2k) (2k <= 30 bits, so 32-bit arithmetic is exact mod 2^(2k)).
  x &= M;
  x ^= x >> k;
  x = (x * 0x7F4A7C15u) & M;
  x ^= x >> (k - 1);
  x = (x * 0x6659FD93u) & M;
  x ^= x >> k;
  return x;
}

struct SketchArgs {
  const uint32_t* packed;
  const uint32_t* mask;
  const uint32_t* nbits;
  const int64_t* off;  // nseq + 1 sequence offsets (device)
  int nseq;
  int64_t N;
  int k, w, min_unmasked;
  uint32_t kmask;
  int64_t ntiles;
};

// Single-pass form: each CTA takes tiles in ticket order, publishes its
// tile's record count, and adds up its predecessors' counts (decoupled
// look-back) until one has published its inclusive prefix.  A tile's
// predecessors were all taken before it by CTAs that publish their count
// before they wait on anyone, so every wait ends; it is bounded all the
// same, and a wait that gives up raises *err for the host.
struct LookBack {
  unsigned long long* status;  // per tile: flag (2 bits) and value (62 bits); zeroed
  unsigned int* ticket;        // next tile to take; zeroed
  unsigned long long* total;   // records of all tiles (written by the last tile)
  int* err;                    // set when a wait gives up; zeroed
};

constexpr unsigned long long kLbAggregate = 1ull << 62, kLbPrefix = 2ull << 62;
constexpr unsigned long long kLbValue = (1ull << 62) - 1;
constexpr unsigned int kLbSpins = 1u << 20;  // polls of one predecessor before giving up

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Records before tile `tile`; warp 0 of the CTA calls it once per tile.  The
// warp reads the status of the 32 tiles below its window at once: the
// nearest one that has published its inclusive prefix ends the walk, and
// the counts of the tiles above it are summed by the warp (a look-back one
// tile at a time falls behind the tiles that are in flight).
__device__ long long look_back(const LookBack& lb, int64_t tile, int64_t ntiles,
                               unsigned long long count) {
  const int lane = threadIdx.x & 31;
  long long before = 0;
  if (tile > 0) {
    if (lane == 0) st_release_gpu(lb.status + tile, kLbAggregate | count);
    int64_t j = tile - 1;  // the walk's top tile
    unsigned int spins = 0;
    while (true) {
      const int64_t at = j - lane;
      // below tile 0 reads as a published prefix of zero
      const unsigned long long v = at >= 0 ? ld_acquire_gpu(lb.status + at) : kLbPrefix;
      const unsigned long long flag = v & ~kLbValue;
      const unsigned prefix = __ballot_sync(0xffffffffu, flag == kLbPrefix);
      const int p = prefix ? __ffs(prefix) - 1 : 31;  // lanes 0..p take part
      const unsigned need = p == 31 ? 0xffffffffu : ((1u << (p + 1)) - 1u);
      const unsigned waiting = __ballot_sync(0xffffffffu, flag == 0) & need;
      if (waiting) {
        if (++spins > kLbSpins) {
          if (lane == 0) atomicExch(lb.err, 1);
          break;
        }
        __nanosleep(64);
        continue;
      }
      spins = 0;
      long long part = lane <= p ? (long long)(v & kLbValue) : 0;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
      before += part;
      if (prefix) break;
      j -= 32;
    }
  }
  if (lane == 0) {
    st_release_gpu(lb.status + tile, kLbPrefix | ((unsigned long long)before + count));
    if (tile == ntiles - 1) *lb.total = (unsigned long long)before + count;
  }
  return before;
}

// Exclusive sum over the CTA.  Unlike block_exclusive_sum it ends without a
// barrier: the next tile reaches s_tmp only after at least two more.
__device__ __forceinline__ int tile_exclusive_sum(int v, int* tmp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int inc = warp_inclusive_sum(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int x = lane < kSkThreads / 32 ? tmp[lane] : 0;
    const int xi = warp_inclusive_sum(x);
    if (lane < kSkThreads / 32) tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  *total = tmp[32];
  return tmp[warp] + inc - v;
}

// Window minima for the windows starting at local slot B + t, t in
// [0, kSkWPT]: key[t] = min over slots [B + t, B + t + w) of kx(slot).
template <typename K, typename KX>
__device__ __forceinline__ void window_minima(int w, int B, KX kx, K (&key)[kSkWPT + 1]) {
  const K inf = ~K(0);
  if (w <= kSkWPT) {
#pragma unroll
    for (int t = 0; t <= kSkWPT; ++t) {
      K m = inf;
      for (int x = B + t; x < B + t + w; ++x) m = min(m, kx(x));
      key[t] = m;
    }
  } else {
    // suffix minima over [B+t, B+7], middle over [B+8, B+w-1], prefix
    // minima over [B+w, B+w+t-1]
    K suf[kSkWPT + 1];
    suf[kSkWPT] = inf;
#pragma unroll
    for (int t = kSkWPT - 1; t >= 0; --t) suf[t] = min(suf[t + 1], kx(B + t));
    K mid = inf;
    for (int x = B + kSkWPT; x < B + w; ++x) mid = min(mid, kx(x));
    K pre = inf;
#pragma unroll
    for (int t = 0; t <= kSkWPT; ++t) {
      if (t > 0) pre = min(pre, kx(B + w + t - 1));
      key[t] = min(min(suf[t], mid), pre);
    }
  }
}

// kMode 0: count the records of each tile; 1: write them at the tile
// offsets given; 2: one pass, offsets by look-back.  Four CTAs per SM (64
// registers a thread): while one CTA's warp 0 walks back, the others compute.
// kNarrow (2k <= 24 and w + kSkWPT <= 128): a window key is 32 bits, the
// hash (ineligible as 2^24) over 7 bits of the slot's reversed offset from
// the thread's first slot, so that equal hashes still go to the rightmost.
template <int kMode, bool kNarrow>
__global__ void __launch_bounds__(kSkThreads, 4) k_sketch(SketchArgs a, uint32_t* __restrict__ tile_count,
                                                       const uint32_t* __restrict__ tile_offset,
                                                       uint64_t* __restrict__ out, int64_t cap,
                                                       LookBack lb) {
  __shared__ uint32_t s_pk[kSkWords16];
  __shared__ uint32_t s_mk[kSkWords32];
  __shared__ uint32_t s_nb[kSkWords32];
  __shared__ uint32_t s_h[kSkHashesP];
  __shared__ uint8_t s_sg[kSkHashesP];
  __shared__ int s_tmp[33];
  __shared__ long long s_tile, s_base;
  __shared__ long long s_seg_lo, s_seg_hi;  // the sequence holding the tile's first position

  const int k = a.k, w = a.w;
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    int64_t tile = it;
    if (kMode == 2) {
      // every thread read the last tile's s_tile before the barriers of
      // that tile's body, so tid 0 may overwrite it now
      if (tid == 0) s_tile = (long long)atomicAdd(lb.ticket, 1u);
      __syncthreads();
      tile = s_tile;
    }
    if (tile >= a.ntiles) break;
    const int64_t Q0 = tile * kSkTile;
    const int64_t HB = Q0 - 1;                    // first hash position of the tile
    const int nh = kSkTile + w;                   // hash positions [HB, HB + nh)
    const int64_t b_lo = HB < 0 ? 0 : HB;
    const int64_t wb16 = b_lo >> 4, wb32 = b_lo >> 5;
    const int64_t nw16 = (a.N + 15) >> 4, nw32 = (a.N + 31) >> 5;
    const int64_t last = HB + nh + k;             // one past the last base read
    const int n16 = (int)(((last + 15) >> 4) - wb16 + 1);
    const int n32 = (int)(((last + 31) >> 5) - wb32 + 1);
    // no barrier here: the staging buffers were last read in the previous
    // tile's hash stage, which a barrier ends
    if (tid == 0) {
      const int s = seq_of(a.off, a.nseq, b_lo);
      s_seg_lo = a.off[s];
      s_seg_hi = a.off[s + 1];
    }
    for (int x = tid; x < n16; x += kSkThreads) {
      const int64_t g = wb16 + x;
      s_pk[x] = g < nw16 ? __ldg(a.packed + g) : 0u;
    }
    for (int x = tid; x < n32; x += kSkThreads) {
      const int64_t g = wb32 + x;
      s_mk[x] = g < nw32 ? __ldg(a.mask + g) : 0xFFFFFFFFu;
      s_nb[x] = g < nw32 ? __ldg(a.nbits + g) : 0xFFFFFFFFu;
    }
    __syncthreads();

    // ---- hashes of positions HB + x, x in [0, nh)
    {
      const int per = (nh + kSkThreads - 1) / kSkThreads;
      const int x0 = tid * per;
      int64_t segend = s_seg_hi, segstart = s_seg_lo;
      // every k-mer of this thread inside the tile's first sequence: no
      // per-position bounds checks
      const int xe = min(x0 + per, nh);
      const bool inside = HB + x0 >= segstart && HB + xe - 1 + k <= segend;
      for (int r = 0; r < per; ++r) {
        const int x = x0 + r;
        if (x >= nh) break;
        const int64_t p = HB + x;
        uint32_t h = kInfHash, sg = 0;
        if (inside || (p >= 0 && p + k <= a.N)) {
          if (!inside && (p >= segend || p < segstart)) {
            const int s = seq_of(a.off, a.nseq, p);
            segstart = a.off[s];
            segend = a.off[s + 1];
          }
          if (inside || p + k <= segend) {
            const int64_t lp = p - (wb16 << 4);
            const int wi = (int)(lp >> 4), sh = (int)(lp & 15) * 2;
            const uint64_t pair = (uint64_t)s_pk[wi] | ((uint64_t)s_pk[wi + 1] << 32);
            const uint32_t g = (uint32_t)(pair >> sh) & a.kmask;   // first base in the low bits
            const int64_t lb = p - (wb32 << 5);
            const int bi = (int)(lb >> 5), bs = (int)(lb & 31);
            const uint64_t kb = (1ull << k) - 1;
            const uint64_t nb = (((uint64_t)s_nb[bi] | ((uint64_t)s_nb[bi + 1] << 32)) >> bs) & kb;
            const uint64_t mk = (((uint64_t)s_mk[bi] | ((uint64_t)s_mk[bi + 1] << 32)) >> bs) & kb;
            // forward code: reverse the order of the k 2-bit groups
            uint32_t f = __brev(g);
            f = ((f >> 1) & 0x55555555u) | ((f & 0x55555555u) << 1);
            f >>= (32 - 2 * k);
            const uint32_t rc = g ^ a.kmask;  // complement each base, order reversed
            const int unmasked = k - __popcll(mk);
            if (nb == 0 && unmasked >= a.min_unmasked && f != rc) {
              h = bijective_hash(f < rc ? f : rc, k, a.kmask);
              sg = rc < f ? 1u : 0u;
            }
          }
        }
        s_h[hslot(x)] = h;
        s_sg[hslot(x)] = (uint8_t)sg;
      }
    }
    __syncthreads();

    // ---- windows q = HB + B + t, t in [0, 9): local hash range [B + t, B + t + w)
    const int B = tid * kSkWPT;
    uint32_t xs[kSkWPT + 1];  // slot of each window's minimizer
    uint32_t inf = 0;         // bit t: window t's minimum is ineligible
    if (kNarrow) {
      uint32_t key[kSkWPT + 1];
      auto kx = [&](int x) -> uint32_t {
        return (min(s_h[hslot(x)], 1u << 24) << 7) | (uint32_t)(127 - (x - B));
      };
      window_minima(w, B, kx, key);
#pragma unroll
      for (int t = 0; t <= kSkWPT; ++t) {
        xs[t] = (uint32_t)(B + 127) - (key[t] & 127u);
        if ((key[t] >> 7) >= (1u << 24)) inf |= 1u << t;
      }
    } else {
      uint64_t key[kSkWPT + 1];
      auto kx = [&](int x) -> uint64_t {
        return ((uint64_t)s_h[hslot(x)] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)x);
      };
      window_minima(w, B, kx, key);
#pragma unroll
      for (int t = 0; t <= kSkWPT; ++t) {
        xs[t] = 0xFFFFFFFFu - (uint32_t)key[t];
        if ((uint32_t)(key[t] >> 32) == kInfHash) inf |= 1u << t;
      }
    }
    // validity and selection flags for windows t = 1..8
    uint32_t flags = 0;
    {
      int64_t segend = s_seg_hi, segstart = s_seg_lo;
      // all nine windows inside the tile's first sequence
      const bool inside = HB + B >= segstart && HB + B + kSkWPT + w + k - 1 <= segend;
      bool prev_ok = false;
      uint32_t prev_arg = 0;
#pragma unroll
      for (int t = 0; t <= kSkWPT; ++t) {
        const int64_t q = HB + B + t;
        bool ok;
        if (inside) {
          ok = !((inf >> t) & 1u);
        } else {
          ok = false;
          if (q >= 0 && q + w + k - 1 <= a.N) {
            if (q >= segend || q < segstart) {
              const int s = seq_of(a.off, a.nseq, q);
              segstart = a.off[s];
              segend = a.off[s + 1];
            }
            ok = (q + w + k - 1 <= segend) && !((inf >> t) & 1u);
          }
        }
        const uint32_t arg = xs[t];
        if (t > 0 && ok && !(prev_ok && prev_arg == arg)) flags |= 1u << t;
        prev_ok = ok;
        prev_arg = arg;
      }
    }
    const int cnt = __popc(flags);
    int total;
    const int excl = tile_exclusive_sum(cnt, s_tmp, &total);
    if (kMode == 0) {
      if (tid == 0) tile_count[tile] = (uint32_t)total;
    } else {
      if (kMode == 2) {
        if (tid < 32) {
          const long long before = look_back(lb, tile, a.ntiles, (unsigned long long)total);
          if (tid == 0) s_base = before;
        }
        __syncthreads();
      }
      int64_t o = (kMode == 2 ? (int64_t)s_base : (int64_t)tile_offset[tile]) + excl;
#pragma unroll
      for (int t = 1; t <= kSkWPT; ++t) {
        if (flags >> t & 1u) {
          const uint32_t x = xs[t];
          const uint64_t pos = (uint64_t)(HB + x);
          if (o < cap)
            out[o] = ((uint64_t)s_h[hslot((int)x)] << 33) | (pos << 1) | (uint64_t)s_sg[hslot((int)x)];
          ++o;
        }
      }
    }
  }
}

// The 32-bit window keys hold a hash of 2k bits and a 7-bit slot offset.
bool narrow_keys(const Derived& D) { return 2 * D.k <= 24 && D.w + kSkWPT <= 128; }

}  // namespace

int launch_pack(sedef_ctx* ctx, const uint8_t* seq, int64_t n, uint32_t* packed, uint32_t* mask,
                uint32_t* nbits) {
  cudaStream_t st = ctx_stream(ctx);
  const int64_t nchunk = (n + 15) / 16;
  int64_t blocks = (nchunk + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  if (((uintptr_t)seq & 15) == 0)
    SEDEF_KERNEL(ctx, "k_pack", k_pack<true><<<(int)blocks, 256, 0, st>>>(seq, n, packed, mask, nbits));
  else
    SEDEF_KERNEL(ctx, "k_pack", k_pack<false><<<(int)blocks, 256, 0, st>>>(seq, n, packed, mask, nbits));
  return SEDEF_OK;
}

int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total);

int run_sketch(sedef_ctx* ctx, const uint32_t* packed, const uint32_t* mask, const uint32_t* nbits,
               const int64_t* h_off, int nseq, const Derived& D, uint64_t* rec, int64_t cap,
               int64_t* nrec, Planned* pl) {
  cudaStream_t st = ctx_stream(ctx);
  const int64_t N = h_off[nseq];
  SketchArgs a;
  a.packed = packed;
  a.mask = mask;
  a.nbits = nbits;
  a.nseq = nseq;
  a.N = N;
  a.k = D.k;
  a.w = D.w;
  a.min_unmasked = D.min_unmasked;
  a.kmask = D.kmask;
  const int64_t nwin = N;  // window starts q in [0, N)
  a.ntiles = (nwin + kSkTile - 1) / kSkTile;
  int64_t* d_off = (int64_t*)ctx_alloc(ctx, (size_t)(nseq + 1) * 8);
  if (!d_off) return SEDEF_ERR_OOM;
  if (pl) {
    int64_t* h = (int64_t*)host_buf(ctx, pl, (size_t)(nseq + 1) * 8);
    if (!h) return SEDEF_ERR_OOM;
    std::memcpy(h, h_off, (size_t)(nseq + 1) * 8);
    SEDEF_CUDA(cudaMemcpyAsync(d_off, h, (size_t)(nseq + 1) * 8, cudaMemcpyHostToDevice, st));
  } else {
    SEDEF_CUDA(cudaMemcpyAsync(d_off, h_off, (size_t)(nseq + 1) * 8, cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));  // h_off is caller memory: copy before returning
  }
  a.off = d_off;
  const bool narrow = narrow_keys(D);
  int64_t grid = a.ntiles;
  const int64_t maxgrid = (int64_t)ctx_sm_count(ctx) * 8;
  if (grid > maxgrid) grid = maxgrid;
  if (!pl) {
    // one pass: record offsets by look-back over the tiles
    if (a.ntiles == 0) {
      *nrec = 0;
      return SEDEF_OK;
    }
    unsigned long long* status = (unsigned long long*)ctx_alloc(ctx, (size_t)(a.ntiles + 4) * 8);
    if (!status) return SEDEF_ERR_OOM;
    LookBack lb;
    lb.status = status + 4;
    lb.ticket = (unsigned int*)status;
    lb.total = status + 1;
    lb.err = (int*)(status + 2);
    SEDEF_CUDA(cudaMemsetAsync(status, 0, (size_t)(a.ntiles + 4) * 8, st));
    if (narrow)
      SEDEF_KERNEL(ctx, "k_sketch",
                   k_sketch<2, true><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, nullptr, rec, cap, lb));
    else
      SEDEF_KERNEL(ctx, "k_sketch",
                   k_sketch<2, false><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, nullptr, rec, cap, lb));
    unsigned long long* h = (unsigned long long*)ctx_host(ctx, 16);
    if (!h) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(h, status + 1, 16, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
    if ((int)h[1] != 0) return fail(SEDEF_ERR_TIMEOUT, "sedef_sketch: a tile's offset wait gave up");
    *nrec = (int64_t)h[0];
    if (*nrec > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_sketch: record buffer too small");
    return SEDEF_OK;
  }
  // planned pass (one CUDA graph, no waits between CTAs): count, scan and
  // write; the write pass stores the records below the capacity and the
  // exact total stays on the device
  uint32_t* cnt = (uint32_t*)ctx_alloc(ctx, (size_t)(a.ntiles + 1) * 4);
  uint32_t* toff = (uint32_t*)ctx_alloc(ctx, (size_t)(a.ntiles + 1) * 4);
  if (!cnt || !toff) return SEDEF_ERR_OOM;
  if (narrow)
    SEDEF_KERNEL(ctx, "k_sketch_count",
                 k_sketch<0, true><<<(int)grid, kSkThreads, 0, st>>>(a, cnt, nullptr, nullptr, 0, LookBack{}));
  else
    SEDEF_KERNEL(ctx, "k_sketch_count",
                 k_sketch<0, false><<<(int)grid, kSkThreads, 0, st>>>(a, cnt, nullptr, nullptr, 0, LookBack{}));
  SEDEF_TRY(scan_exclusive_u32(ctx, cnt, toff, a.ntiles, toff + a.ntiles));
  pl->n_rec = toff + a.ntiles;
  SEDEF_TRY(plan_check(ctx, pl, toff + a.ntiles, cap, 0));
  *nrec = cap;
  if (narrow)
    SEDEF_KERNEL(ctx, "k_sketch_write",
                 k_sketch<1, true><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, toff, rec, cap, LookBack{}));
  else
    SEDEF_KERNEL(ctx, "k_sketch_write",
                 k_sketch<1, false><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, toff, rec, cap, LookBack{}));
  return SEDEF_OK;
}

}  // namespace sedef

// ------------------------------------------------ allocation-free sketch --
//
// sedef_sketch_noalloc: the sketch with its scratch (per-tile counts and
// offsets, the sequence offsets) in a fixed static device array instead of
// memory from a context, for callers that must not allocate device memory.
// The array's host-side name is only a stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.

namespace sedef {
namespace {

constexpr int64_t kNoallocMaxBases = int64_t(256) << 20;  // 268,435,456 bases
constexpr int kNoallocMaxSeqs = 4096;
constexpr int64_t kNoallocMaxTiles = (kNoallocMaxBases + kSkTile - 1) / kSkTile;
constexpr size_t kNoallocCountBytes = (size_t)(kNoallocMaxTiles + 1) * 4;
constexpr size_t kNoallocBytes = 2 * kNoallocCountBytes + (size_t)(kNoallocMaxSeqs + 1) * 8;

// Shared by every call in the process and kept between calls; about 1 MB on
// each device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];


// Exclusive scan of n counts by one block (n is at most 131,073 here).
__global__ void __launch_bounds__(1024) k_scan_one_block(const uint32_t* __restrict__ in,
                                                         uint32_t* __restrict__ out, int64_t n) {
  __shared__ int tmp[33];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = (int64_t)threadIdx.x * per, hi = min(n, lo + per);
  uint32_t s = 0;
  for (int64_t x = lo; x < hi; ++x) s += in[x];
  int tot;
  uint32_t run = (uint32_t)block_exclusive_sum((int)s, tmp, &tot);
  for (int64_t x = lo; x < hi; ++x) {
    const uint32_t v = in[x];
    out[x] = run;
    run += v;
  }
  if (threadIdx.x == 0) out[n] = (uint32_t)tot;
}

}  // namespace
}  // namespace sedef

extern "C" int sedef_sketch_noalloc(const uint32_t* d_packed, const uint32_t* d_mask,
                                    const uint32_t* d_nbits, const int64_t* h_seq_off,
                                    int32_t nseq, const sedef_params* p, uint64_t* d_rec,
                                    int64_t rec_cap, int64_t* h_nrec, void* stream) {
  using namespace sedef;
  if (!h_nrec) return fail(SEDEF_ERR_INVALID, "h_nrec is NULL");
  *h_nrec = 0;
  Derived D;
  SEDEF_TRY(derive(p, &D));
  if (nseq < 0 || (nseq > 0 && !h_seq_off)) return fail(SEDEF_ERR_INVALID, "bad offsets");
  if (nseq == 0) return SEDEF_OK;
  if (h_seq_off[0] != 0) return fail(SEDEF_ERR_INVALID, "offsets must start at 0");
  for (int s = 0; s < nseq; ++s)
    if (h_seq_off[s + 1] < h_seq_off[s]) return fail(SEDEF_ERR_INVALID, "offsets decrease");
  const int64_t N = h_seq_off[nseq];
  if (N == 0) return SEDEF_OK;
  if (N > kNoallocMaxBases || nseq > kNoallocMaxSeqs)
    return fail(SEDEF_ERR_UNSUPPORTED,
                "sedef_sketch_noalloc: at most 268435456 bases in at most 4096 sequences "
                "(the fixed scratch array); use sedef_sketch for larger inputs");
  if (!d_packed || !d_mask || !d_nbits || (rec_cap > 0 && !d_rec))
    return fail(SEDEF_ERR_INVALID, "NULL buffer");
  int dev = 0;
  SEDEF_CUDA(cudaGetDevice(&dev));
  // The array's device address on the current device.  Looked up on every
  // call (a table lookup once the module is loaded; the first call on a
  // device loads it), so it stays right after a cudaDeviceReset and needs no
  // lock between host threads.  In host code the array's name is only a
  // host-side stand-in, never a device address.
  void* ptr = nullptr;
  {
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  }
  unsigned char* base = (unsigned char*)ptr;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base);
  uint32_t* toff = reinterpret_cast<uint32_t*>(base + kNoallocCountBytes);
  int64_t* d_off = reinterpret_cast<int64_t*>(base + 2 * kNoallocCountBytes);
  cudaStream_t st = (cudaStream_t)stream;
  SEDEF_CUDA(cudaMemcpyAsync(d_off, h_seq_off, (size_t)(nseq + 1) * 8, cudaMemcpyHostToDevice, st));
  SketchArgs a;
  a.packed = d_packed;
  a.mask = d_mask;
  a.nbits = d_nbits;
  a.off = d_off;
  a.nseq = nseq;
  a.N = N;
  a.k = D.k;
  a.w = D.w;
  a.min_unmasked = D.min_unmasked;
  a.kmask = D.kmask;
  a.ntiles = (N + kSkTile - 1) / kSkTile;
  int sms = 0;
  SEDEF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int64_t grid = a.ntiles < (int64_t)sms * 8 ? a.ntiles : (int64_t)sms * 8;
  if (narrow_keys(D))
    k_sketch<0, true><<<(int)grid, kSkThreads, 0, st>>>(a, cnt, nullptr, nullptr, 0, LookBack{});
  else
    k_sketch<0, false><<<(int)grid, kSkThreads, 0, st>>>(a, cnt, nullptr, nullptr, 0, LookBack{});
  count_launch();
  SEDEF_LAUNCHED("k_sketch_count");
  k_scan_one_block<<<1, 1024, 0, st>>>(cnt, toff, a.ntiles);
  count_launch();
  SEDEF_LAUNCHED("k_scan_one_block");
  uint32_t total = 0;
  SEDEF_CUDA(cudaMemcpyAsync(&total, toff + a.ntiles, 4, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  *h_nrec = total;
  if ((int64_t)total > rec_cap) return fail(SEDEF_ERR_CAPACITY, "record buffer too small");
  if (narrow_keys(D))
    k_sketch<1, true><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, toff, d_rec, rec_cap, LookBack{});
  else
    k_sketch<1, false><<<(int)grid, kSkThreads, 0, st>>>(a, nullptr, toff, d_rec, rec_cap, LookBack{});
  count_launch();
  SEDEF_LAUNCHED("k_sketch_write");
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}
