// f2: two-tier local chaining inside the potential SD regions (Section 3.3).
//
// For every region (query [qa, qb), target [ta, tb), strand o from
// sedef_extend) the query is X = G[qa, qb) and the target Y = G[ta, tb),
// reverse-complemented when o = 1, both read from the 2-bit packed genome
// (case does not matter; a base flagged in the N bit-vector matches
// nothing).
//   Seeds: maximal exact matches (x, y, L) of at least k2 = 11 bases.
//   Initial chains: seed b may follow a when it starts later on both axes
//   and the gaps from a's end to b's start are at most g1 = ceil(1000 *
//   delta_G) on both axes (negative where an indel makes them overlap); the
//   link adds the bases new on both axes, min(L_b, end_b - end_a on x,
//   end_b - end_a on y), and must add at least one; f(b) = max(L_b, best
//   f(a) + gain), the later seed on ties.  Chains are taken greedily by
//   decreasing f (earlier seed on ties), each back along its predecessors
//   to the first seed a chain already holds.
//   Final chains: initial chains (sorted by start) chained with gaps of at
//   most g2 = 10,000 on both axes and an affine penalty 25 + g / 50 for the
//   larger gap g; F(d) = S(d) + max(0, best F(c) - pen), a link only when it
//   raises the score, the later chain on ties; the same greedy extraction.
//   A final chain spanning at least 1,000 bases on both axes is an SD.
//
// Regions run in batches (at most 2^26 target k-mers).  Per batch:
//   k_c2_keys     one thread per target position: (region, 11-mer, y) keys
//   radix sort    by (region, 11-mer); y stays ascending
//   k_c2_mems     one thread per query position: the matching target range
//                 by binary search, left-maximal matches extended to the
//                 right (count pass, then write pass at scanned offsets), so
//                 a region's seeds come out sorted by (x, y)
//   k_c2_dp       one warp per region: the chaining DP, predecessors scanned
//                 back from each item, 32 per step, only as far as an item
//                 can still reach (its start at least the current start
//                 minus the gap bound minus the region's longest item)
//   radix sort    by (region, -score, index), then k_c2_take: one thread per
//                 region walks that order and takes the chains greedily
// (once for the seeds and once for the initial chains), and k_c2_emit
// compacts the final chains.
#include <cstring>

#include "common.cuh"

namespace sedef {
namespace {

constexpr int kK2 = 11;                  // seed length (Section 3.3)
constexpr int64_t kG2 = 10000;           // largest gap between initial chains (Section 3.3)
constexpr int64_t kGapOpen = 25;         // affine gap penalty: open
constexpr int64_t kGapDiv = 50;          // one more per kGapDiv gap bases
constexpr int64_t kMinSD = 1000;         // SD length (Section 3)
constexpr int64_t kMaxRegion = int64_t(1) << 20;
constexpr int kDPWarps = 4;

// A region of the batch: query and target starts, lengths, strand.
struct Reg {
  int64_t qa, ta, tb;
  int32_t nx, ny, o, pad;
};

__device__ __forceinline__ uint32_t base2(const uint32_t* packed, int64_t p) {
  return (packed[p >> 4] >> (2 * (p & 15))) & 3u;
}
__device__ __forceinline__ bool isn(const uint32_t* nbits, int64_t p) {
  return (nbits[p >> 5] >> (p & 31)) & 1u;
}

// Base of X (q) or Y (t) at offset u: 0-3, or 4 for a base that matches
// nothing.
__device__ __forceinline__ uint32_t xbase(const uint32_t* packed, const uint32_t* nbits,
                                          const Reg& R, int64_t u) {
  const int64_t p = R.qa + u;
  return isn(nbits, p) ? 4u : base2(packed, p);
}
__device__ __forceinline__ uint32_t ybase(const uint32_t* packed, const uint32_t* nbits,
                                          const Reg& R, int64_t u) {
  if (R.o == 0) {
    const int64_t p = R.ta + u;
    return isn(nbits, p) ? 4u : base2(packed, p);
  }
  const int64_t p = R.tb - 1 - u;
  return isn(nbits, p) ? 4u : (3u - base2(packed, p));
}

__device__ __forceinline__ int region_of(const int64_t* base, int nreg, int64_t g) {
  int lo = 0, hi = nreg;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Keys (region << 42 | code << 20 | y) of every target 11-mer of A, C, G, T.
__global__ void k_c2_keys(const uint32_t* packed, const uint32_t* nbits, const Reg* regs,
                          const int64_t* ybase_of, int nreg, int64_t total, uint64_t* keys) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int r = region_of(ybase_of, nreg, g);
  const Reg R = regs[r];
  const int64_t y = g - ybase_of[r];
  uint64_t key = ~0ull;
  if (y + kK2 <= R.ny) {
    uint64_t code = 0;
    bool ok = true;
    for (int u = 0; u < kK2; ++u) {
      const uint32_t b = ybase(packed, nbits, R, y + u);
      ok = ok && b < 4u;
      code = (code << 2) | (b & 3u);
    }
    if (ok) key = ((uint64_t)r << 42) | (code << 20) | (uint64_t)y;
  }
  keys[g] = key;
}

// Maximal exact matches per query position: counts (write = false) or
// seeds written at out[off[g] ..] (write = true) as x << 40 | y << 20 | L.
template <bool kWrite>
__global__ void k_c2_mems(const uint32_t* packed, const uint32_t* nbits, const Reg* regs,
                          const int64_t* xbase_of, int nreg, int64_t total, const uint64_t* skeys,
                          int64_t nkeys, uint32_t* count, const uint64_t* off, uint64_t* out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int r = region_of(xbase_of, nreg, g);
  const Reg R = regs[r];
  const int64_t x = g - xbase_of[r];
  uint32_t n = 0;
  if (x + kK2 <= R.nx) {
    uint64_t code = 0;
    bool ok = true;
    for (int u = 0; u < kK2; ++u) {
      const uint32_t b = xbase(packed, nbits, R, x + u);
      ok = ok && b < 4u;
      code = (code << 2) | (b & 3u);
    }
    if (ok) {
      const uint64_t want = ((uint64_t)r << 42) | (code << 20);
      int64_t lo = 0, hi = nkeys;  // first key >= want
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (skeys[mid] < want) lo = mid + 1; else hi = mid;
      }
      const uint32_t xprev = x > 0 ? xbase(packed, nbits, R, x - 1) : 4u;
      uint64_t at = kWrite ? off[g] : 0;
      for (int64_t k = lo; k < nkeys && (skeys[k] >> 20) == (want >> 20); ++k) {
        const int64_t y = (int64_t)(skeys[k] & 0xFFFFFull);
        if (x > 0 && y > 0 && xprev < 4u && xprev == ybase(packed, nbits, R, y - 1)) continue;
        int64_t L = kK2;
        while (x + L < R.nx && y + L < R.ny) {
          const uint32_t b = xbase(packed, nbits, R, x + L);
          if (b >= 4u || b != ybase(packed, nbits, R, y + L)) break;
          ++L;
        }
        if (kWrite) out[at++] = ((uint64_t)x << 40) | ((uint64_t)y << 20) | (uint64_t)L;
        ++n;
      }
    }
  }
  if (!kWrite) count[g] = n;
}

// An item of a chaining tier: its box and its own score.
struct Item {
  int32_t x0, x1, y0, y1, score, seeds;
};

__device__ __forceinline__ Item seed_item(uint64_t s) {
  Item it;
  it.x0 = (int32_t)(s >> 40);
  it.y0 = (int32_t)((s >> 20) & 0xFFFFF);
  const int32_t L = (int32_t)(s & 0xFFFFF);
  it.x1 = it.x0 + L;
  it.y1 = it.y0 + L;
  it.score = L;
  it.seeds = 1;
  return it;
}

// Score a link c -> d adds, or INT_MIN when d cannot follow c.
__device__ __forceinline__ int32_t link_gain(const Item& c, const Item& d, int tier, int32_t g1) {
  if (tier == 1) {
    if (c.x0 >= d.x0 || c.y0 >= d.y0) return INT32_MIN;
    if (d.x0 - c.x1 > g1 || d.y0 - c.y1 > g1) return INT32_MIN;
    const int32_t g = min(d.score, min(d.x1 - c.x1, d.y1 - c.y1));
    return g > 0 ? g : INT32_MIN;
  }
  const int32_t gq = d.x0 - c.x1, gt = d.y0 - c.y1;
  if (gq < 0 || gt < 0 || gq > (int32_t)kG2 || gt > (int32_t)kG2) return INT32_MIN;
  return d.score - (int32_t)(kGapOpen + max(gq, gt) / kGapDiv);
}

// The chaining DP of one tier: one warp per region, items of region r at
// [ib[r], ib[r] + n[r]) in start order.  best[] and pred[] (region-local
// index, -1 for none) per item.
__global__ void __launch_bounds__(32 * kDPWarps) k_c2_dp(const Item* items, const int64_t* ib,
                                                        const uint32_t* n_of, int nreg, int tier,
                                                        int32_t g1, int32_t* best, int32_t* pred) {
  const int lane = lane_id();
  const int r = blockIdx.x * kDPWarps + (threadIdx.x >> 5);
  if (r >= nreg) return;
  const int64_t b0 = ib[r];
  const int32_t n = (int32_t)n_of[r];
  // the longest item bounds how far back a predecessor can start
  int32_t span = 0;
  for (int32_t u = lane; u < n; u += 32) span = max(span, items[b0 + u].x1 - items[b0 + u].x0);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) span = max(span, __shfl_xor_sync(0xffffffffu, span, d));
  const int32_t reach = (tier == 1 ? g1 : (int32_t)kG2) + span;
  for (int32_t b = 0; b < n; ++b) {
    const Item d = items[b0 + b];
    int32_t bv = INT32_MIN, ba = -1;  // best value through a predecessor, its index
    for (int32_t top = b - 1; top >= 0; top -= 32) {
      const int32_t a = top - lane;
      bool more = false;
      if (a >= 0) {
        const Item c = items[b0 + a];
        more = c.x0 >= d.x0 - reach;
        if (more) {
          const int32_t g = link_gain(c, d, tier, g1);
          if (g != INT32_MIN) {
            const int32_t v = best[b0 + a] + g;
            if (v > bv || (v == bv && a > ba)) {
              bv = v;
              ba = a;
            }
          }
        }
      }
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const int32_t ov = __shfl_xor_sync(0xffffffffu, bv, s);
        const int32_t oa = __shfl_xor_sync(0xffffffffu, ba, s);
        if (ov > bv || (ov == bv && oa > ba)) {
          bv = ov;
          ba = oa;
        }
      }
      // items are in start order: once every lane is out of reach, so is
      // everything earlier
      if (!__any_sync(0xffffffffu, more)) break;
    }
    // tier 1: f = max(L, best link); tier 2: F = S + max(0, best link - S)
    const int32_t own = d.score;
    int32_t f = own, pr = -1;
    if (bv != INT32_MIN && bv > own) {
      f = bv;
      pr = ba;
    }
    if (lane == 0) {
      best[b0 + b] = f;
      pred[b0 + b] = pr;
    }
    __syncwarp();
  }
}

// Sort keys of the greedy extraction: (region, -score, index).
__global__ void k_c2_order_keys(const int32_t* best, const int64_t* ib, const uint32_t* n_of,
                                int nreg, int64_t total, uint64_t* keys) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int r = region_of(ib, nreg, g);
  const int64_t u = g - ib[r];
  uint64_t key = ~0ull;
  if (u < (int64_t)n_of[r])
    key = ((uint64_t)r << 42) | ((uint64_t)(0xFFFFF - best[g]) << 22) | (uint64_t)u;
  keys[g] = key;
}

// Greedy extraction (one thread per region): chains in the order of
// `order` (sorted keys), each back along pred to the first item already
// taken.  Writes one Item per chain to out[ib[r] + j], its number of items
// to parts[ib[r] + j], and the count.  A chain's box starts at its first
// item; it ends at the furthest item end (tier 1) or at its last item's end
// (tier 2); its score is the first item's plus every link's gain.
__global__ void k_c2_take(const Item* items, const int32_t* pred, const int64_t* ib,
                          const uint32_t* n_of, int nreg, int tier, int32_t g1,
                          const uint64_t* order, uint8_t* used, int32_t* path, Item* out,
                          int32_t* parts, uint32_t* nout) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nreg) return;
  const int64_t b0 = ib[r];
  const int32_t n = (int32_t)n_of[r];
  uint32_t m = 0;
  for (int32_t k = 0; k < n; ++k) {
    const int32_t b = (int32_t)(order[b0 + k] & 0x3FFFFF);
    if (used[b0 + b]) continue;
    int32_t len = 0;
    for (int32_t c = b; c >= 0 && !used[b0 + c]; c = pred[b0 + c]) {
      used[b0 + c] = 1;
      path[b0 + len++] = c;
    }
    // path[b0 .. b0 + len) holds the chain from its end back to its start
    Item ch = items[b0 + path[b0 + len - 1]];
    for (int32_t u = len - 2; u >= 0; --u) {
      const Item prev = items[b0 + path[b0 + u + 1]];
      const Item cur = items[b0 + path[b0 + u]];
      ch.x1 = tier == 1 ? max(ch.x1, cur.x1) : cur.x1;
      ch.y1 = tier == 1 ? max(ch.y1, cur.y1) : cur.y1;
      ch.seeds += cur.seeds;
      ch.score += link_gain(prev, cur, tier, g1);
    }
    out[b0 + m] = ch;
    parts[b0 + m] = len;
    ++m;
  }
  nout[r] = m;
}

// Seeds (x << 40 | y << 20 | L) as chaining items.
__global__ void k_c2_items(const uint64_t* seeds, int64_t n, Item* items) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) items[g] = seed_item(seeds[g]);
}

// Start-order keys of the initial chains: (region, x0, y0) -> slot.
__global__ void k_c2_start_keys(const Item* ch, const int64_t* ib, const uint32_t* n_of, int nreg,
                                int64_t total, uint64_t* keys) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int r = region_of(ib, nreg, g);
  const int64_t u = g - ib[r];
  uint64_t key = ~0ull;
  if (u < (int64_t)n_of[r])
    key = ((uint64_t)r << 42) | ((uint64_t)ch[g].x0 << 21) | (uint64_t)ch[g].y0;
  keys[g] = key;
}

// Gathers the initial chains of each region into start order at the same
// region base (the sort kept regions apart and in order).
__global__ void k_c2_gather(const Item* in, const uint32_t* perm, const uint64_t* skeys,
                            int64_t total, Item* out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  if (skeys[g] != ~0ull) out[g] = in[perm[g]];
}

// Final chains of at least kMinSD bases on both axes, per region, sorted by
// (q0, q1, t0, t1, score) in genome coordinates, written at out[ob[r] ..].
__global__ void k_c2_emit(const Item* fin, const int32_t* parts, const int64_t* ib,
                          const uint32_t* n_of, const Reg* regs, const int64_t* reg_index,
                          int nreg, const int64_t* ob, sedef_sd_t* out, uint32_t* nkept,
                          int count_only) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nreg) return;
  const Reg R = regs[r];
  const int64_t b0 = ib[r];
  uint32_t m = 0;
  for (uint32_t u = 0; u < n_of[r]; ++u) {
    const Item c = fin[b0 + u];
    if (c.x1 - c.x0 < kMinSD || c.y1 - c.y0 < kMinSD) continue;
    if (!count_only) {
      sedef_sd_t s;
      s.region = (uint32_t)reg_index[r];
      s.o = (uint32_t)R.o;
      s.q0 = (uint32_t)(R.qa + c.x0);
      s.q1 = (uint32_t)(R.qa + c.x1);
      s.t0 = (uint32_t)(R.o ? R.tb - c.y1 : R.ta + c.y0);
      s.t1 = (uint32_t)(R.o ? R.tb - c.y0 : R.ta + c.y1);
      s.score = (uint32_t)c.score;
      s.seeds = (uint32_t)c.seeds;
      s.parts = (uint32_t)parts[b0 + u];
      s.reserved = 0;
      // insertion into this region's sorted rows
      sedef_sd_t* row = out + ob[r];
      uint32_t at = m;
      auto less = [](const sedef_sd_t& a, const sedef_sd_t& b) {
        if (a.q0 != b.q0) return a.q0 < b.q0;
        if (a.q1 != b.q1) return a.q1 < b.q1;
        if (a.t0 != b.t0) return a.t0 < b.t0;
        if (a.t1 != b.t1) return a.t1 < b.t1;
        if (a.score != b.score) return a.score < b.score;
        if (a.seeds != b.seeds) return a.seeds < b.seeds;
        return a.parts < b.parts;
      };
      while (at > 0 && less(s, row[at - 1])) {
        row[at] = row[at - 1];
        --at;
      }
      row[at] = s;
    }
    ++m;
  }
  nkept[r] = m;
}

}  // namespace

int run_chain2(sedef_ctx* ctx, const uint32_t* packed, const uint32_t* nbits, int64_t nbases,
               const sedef_region_t* d_regions, int64_t nregions, const Derived& D,
               sedef_sd_t* out, int64_t cap, int64_t* nout) {
  cudaStream_t st = ctx_stream(ctx);
  *nout = 0;
  if (nregions == 0) return SEDEF_OK;
  std::vector<sedef_region_t> hr((size_t)nregions);
  SEDEF_CUDA(cudaMemcpyAsync(hr.data(), d_regions, (size_t)nregions * sizeof(sedef_region_t),
                             cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  for (auto& R : hr) {
    if (R.qb < R.qa || R.tb < R.ta || (int64_t)R.qb > nbases || (int64_t)R.tb > nbases)
      return fail(SEDEF_ERR_INVALID, "sedef_chain2: region outside the sequence");
    if ((int64_t)(R.qb - R.qa) >= kMaxRegion || (int64_t)(R.tb - R.ta) >= kMaxRegion)
      return fail(SEDEF_ERR_UNSUPPORTED, "sedef_chain2: a region of 2^20 bases or more");
  }
  const int32_t g1 = (int32_t)std::ceil(1000.0 * D.delta_g - 1e-9);
  std::vector<sedef_sd_t> all;
  int64_t r0 = 0;
  const int64_t kBatchBases = int64_t(1) << 26;
  while (r0 < nregions) {
    // a batch: regions while their target bases fit the key budget
    int64_t r1 = r0, ysum = 0, xsum = 0;
    while (r1 < nregions && (r1 == r0 || ysum + (hr[r1].tb - hr[r1].ta) <= kBatchBases) &&
           r1 - r0 < (int64_t(1) << 21)) {
      ysum += hr[r1].tb - hr[r1].ta;
      xsum += hr[r1].qb - hr[r1].qa;
      ++r1;
    }
    const int nb = (int)(r1 - r0);
    const std::vector<char> used_before = ctx_pool_snapshot(ctx);
    // uploads: regions, y bases, x bases, region indices
    std::vector<Reg> regs(nb);
    std::vector<int64_t> yb(nb + 1, 0), xb(nb + 1, 0), rid(nb);
    for (int k = 0; k < nb; ++k) {
      const sedef_region_t& R = hr[r0 + k];
      regs[k] = {R.qa, R.ta, R.tb, (int32_t)(R.qb - R.qa), (int32_t)(R.tb - R.ta), (int32_t)R.o, 0};
      yb[k + 1] = yb[k] + regs[k].ny;
      xb[k + 1] = xb[k] + regs[k].nx;
      rid[k] = r0 + k;
    }
    const size_t up = sizeof(Reg) * nb + 8 * (size_t)(nb + 1) * 2 + 8 * (size_t)nb;
    char* d_up = (char*)ctx_alloc(ctx, up);
    if (!d_up) return SEDEF_ERR_OOM;
    Reg* d_regs = (Reg*)d_up;
    int64_t* d_yb = (int64_t*)(d_up + sizeof(Reg) * nb);
    int64_t* d_xb = d_yb + (nb + 1);
    int64_t* d_rid = d_xb + (nb + 1);
    SEDEF_CUDA(cudaMemcpyAsync(d_regs, regs.data(), sizeof(Reg) * nb, cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaMemcpyAsync(d_yb, yb.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaMemcpyAsync(d_xb, xb.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaMemcpyAsync(d_rid, rid.data(), 8 * (size_t)nb, cudaMemcpyHostToDevice, st));
    // target k-mer keys, sorted
    const int64_t ny = ysum > 0 ? ysum : 1;
    uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)ny * 8);
    uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)ny * 8);
    if (!keys || !skeys) return SEDEF_ERR_OOM;
    if (ysum > 0) {
      SEDEF_KERNEL(ctx, "k_c2_keys", k_c2_keys<<<(int)((ysum + 255) / 256), 256, 0, st>>>(
                                         packed, nbits, d_regs, d_yb, nb, ysum, keys));
      SEDEF_TRY(radix_sort_u64(ctx, keys, nullptr, skeys, nullptr, ysum, 20, 64));
    }
    // seeds: count, scan, write
    const int64_t nx = xsum > 0 ? xsum : 1;
    uint32_t* cnt = (uint32_t*)ctx_alloc(ctx, (size_t)(nx + 1) * 4);
    uint64_t* off = (uint64_t*)ctx_alloc(ctx, (size_t)(nx + 1) * 8);
    if (!cnt || !off) return SEDEF_ERR_OOM;
    std::vector<uint32_t> hc((size_t)nx + 1, 0);
    if (xsum > 0 && ysum > 0) {
      SEDEF_KERNEL(ctx, "k_c2_mems", (k_c2_mems<false><<<(int)((xsum + 255) / 256), 256, 0, st>>>(
                                         packed, nbits, d_regs, d_xb, nb, xsum, skeys, ysum, cnt,
                                         nullptr, nullptr)));
      SEDEF_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)xsum * 4, cudaMemcpyDeviceToHost, st));
      SEDEF_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<uint64_t> ho((size_t)nx + 1, 0);
    for (int64_t g = 0; g < xsum; ++g) ho[g + 1] = ho[g] + hc[g];
    const int64_t na = (int64_t)ho[xsum > 0 ? xsum : 0];
    // per-region seed ranges and counts
    std::vector<int64_t> ib(nb + 1, 0);
    std::vector<uint32_t> ncount(nb, 0);
    for (int k = 0; k < nb; ++k) {
      ib[k] = (int64_t)ho[xb[k]];
      ncount[k] = (uint32_t)(ho[xb[k + 1]] - ho[xb[k]]);
      if ((int64_t)ncount[k] >= (int64_t(1) << 22))
        return fail(SEDEF_ERR_UNSUPPORTED, "sedef_chain2: more than 2^22 seeds in a region");
    }
    ib[nb] = na;
    std::vector<sedef_sd_t> rows;
    if (na > 0) {
      uint64_t* seeds = (uint64_t*)ctx_alloc(ctx, (size_t)na * 8);
      Item* items = (Item*)ctx_alloc(ctx, (size_t)na * sizeof(Item));
      Item* init = (Item*)ctx_alloc(ctx, (size_t)na * sizeof(Item));
      Item* sorted = (Item*)ctx_alloc(ctx, (size_t)na * sizeof(Item));
      Item* fin = (Item*)ctx_alloc(ctx, (size_t)na * sizeof(Item));
      int32_t* best = (int32_t*)ctx_alloc(ctx, (size_t)na * 4);
      int32_t* pred = (int32_t*)ctx_alloc(ctx, (size_t)na * 4);
      int32_t* path = (int32_t*)ctx_alloc(ctx, (size_t)na * 4);
      int32_t* parts = (int32_t*)ctx_alloc(ctx, (size_t)na * 4);
      uint8_t* used = (uint8_t*)ctx_alloc(ctx, (size_t)na);
      uint64_t* okeys = (uint64_t*)ctx_alloc(ctx, (size_t)na * 8);
      uint64_t* osorted = (uint64_t*)ctx_alloc(ctx, (size_t)na * 8);
      uint32_t* perm = (uint32_t*)ctx_alloc(ctx, (size_t)na * 4);
      char* d_meta = (char*)ctx_alloc(ctx, (size_t)(nb + 1) * 8 * 2 + (size_t)nb * 4 * 4);
      if (!seeds || !items || !init || !sorted || !fin || !best || !pred || !path || !parts || !used ||
          !okeys || !osorted || !perm || !d_meta)
        return SEDEF_ERR_OOM;
      int64_t* d_ib = (int64_t*)d_meta;
      int64_t* d_ob = d_ib + (nb + 1);
      uint32_t* d_n1 = (uint32_t*)(d_ob + (nb + 1));
      uint32_t* d_n2 = d_n1 + nb;
      uint32_t* d_n3 = d_n2 + nb;
      uint32_t* d_keep = d_n3 + nb;
      uint64_t* d_off = off;
      SEDEF_CUDA(cudaMemcpyAsync(d_off, ho.data(), (size_t)(xsum + 1) * 8, cudaMemcpyHostToDevice, st));
      SEDEF_CUDA(cudaMemcpyAsync(d_ib, ib.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, st));
      SEDEF_CUDA(cudaMemcpyAsync(d_n1, ncount.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, st));
      SEDEF_KERNEL(ctx, "k_c2_mems", (k_c2_mems<true><<<(int)((xsum + 255) / 256), 256, 0, st>>>(
                                         packed, nbits, d_regs, d_xb, nb, xsum, skeys, ysum,
                                         nullptr, d_off, seeds)));
      const int tb = (int)((na + 255) / 256);
      const int rb = (nb + 127) / 128;
      const int wb = (nb + kDPWarps - 1) / kDPWarps;
      SEDEF_KERNEL(ctx, "k_c2_items", k_c2_items<<<tb, 256, 0, st>>>(seeds, na, items));
      // tier 1: DP, greedy extraction into initial chains
      SEDEF_KERNEL(ctx, "k_c2_dp", k_c2_dp<<<wb, 32 * kDPWarps, 0, st>>>(items, d_ib, d_n1, nb, 1, g1,
                                                                       best, pred));
      SEDEF_KERNEL(ctx, "k_c2_order_keys", k_c2_order_keys<<<tb, 256, 0, st>>>(best, d_ib, d_n1, nb,
                                                                              na, okeys));
      SEDEF_TRY(radix_sort_u64(ctx, okeys, nullptr, osorted, nullptr, na, 0, 64));
      SEDEF_CUDA(cudaMemsetAsync(used, 0, (size_t)na, st));
      SEDEF_KERNEL(ctx, "k_c2_take", k_c2_take<<<rb, 128, 0, st>>>(items, pred, d_ib, d_n1, nb, 1, g1,
                                                                  osorted, used, path, init, parts,
                                                                  d_n2));
      // initial chains into start order
      SEDEF_KERNEL(ctx, "k_c2_start_keys", k_c2_start_keys<<<tb, 256, 0, st>>>(init, d_ib, d_n2, nb,
                                                                              na, okeys));
      SEDEF_TRY(radix_sort_u64(ctx, okeys, nullptr, osorted, perm, na, 0, 64));
      // sorted chains of region r now start at the region's first sorted
      // slot: bases from the counts
      std::vector<uint32_t> n2(nb);
      SEDEF_CUDA(cudaMemcpyAsync(n2.data(), d_n2, (size_t)nb * 4, cudaMemcpyDeviceToHost, st));
      SEDEF_CUDA(cudaStreamSynchronize(st));
      std::vector<int64_t> cb(nb + 1, 0);
      for (int k = 0; k < nb; ++k) cb[k + 1] = cb[k] + n2[k];
      int64_t* d_cb = d_ob;
      SEDEF_CUDA(cudaMemcpyAsync(d_cb, cb.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, st));
      SEDEF_KERNEL(ctx, "k_c2_gather", k_c2_gather<<<tb, 256, 0, st>>>(init, perm, osorted, na, sorted));
      // tier 2 over the initial chains (region r at [cb[r], cb[r] + n2[r]))
      SEDEF_KERNEL(ctx, "k_c2_dp", k_c2_dp<<<wb, 32 * kDPWarps, 0, st>>>(sorted, d_cb, d_n2, nb, 2, g1,
                                                                       best, pred));
      const int64_t nc = cb[nb] > 0 ? cb[nb] : 1;
      const int tc = (int)((nc + 255) / 256);
      SEDEF_KERNEL(ctx, "k_c2_order_keys", k_c2_order_keys<<<tc, 256, 0, st>>>(best, d_cb, d_n2, nb,
                                                                              cb[nb], okeys));
      SEDEF_TRY(radix_sort_u64(ctx, okeys, nullptr, osorted, nullptr, cb[nb], 0, 64));
      SEDEF_CUDA(cudaMemsetAsync(used, 0, (size_t)na, st));
      SEDEF_KERNEL(ctx, "k_c2_take", k_c2_take<<<rb, 128, 0, st>>>(sorted, pred, d_cb, d_n2, nb, 2,
                                                                  g1, osorted, used, path, fin,
                                                                  parts, d_n3));
      // final chains of SD size: count, then rows per region
      SEDEF_KERNEL(ctx, "k_c2_emit", k_c2_emit<<<rb, 128, 0, st>>>(fin, parts, d_cb, d_n3, d_regs,
                                                                  d_rid, nb, d_cb, nullptr, d_keep, 1));
      std::vector<uint32_t> keep(nb);
      SEDEF_CUDA(cudaMemcpyAsync(keep.data(), d_keep, (size_t)nb * 4, cudaMemcpyDeviceToHost, st));
      SEDEF_CUDA(cudaStreamSynchronize(st));
      std::vector<int64_t> kb(nb + 1, 0);
      for (int k = 0; k < nb; ++k) kb[k + 1] = kb[k] + keep[k];
      if (kb[nb] > 0) {
        int64_t* d_kb = (int64_t*)ctx_alloc(ctx, (size_t)(nb + 1) * 8);
        sedef_sd_t* d_rows = (sedef_sd_t*)ctx_alloc(ctx, (size_t)kb[nb] * sizeof(sedef_sd_t));
        if (!d_kb || !d_rows) return SEDEF_ERR_OOM;
        SEDEF_CUDA(cudaMemcpyAsync(d_kb, kb.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, st));
        SEDEF_KERNEL(ctx, "k_c2_emit", k_c2_emit<<<rb, 128, 0, st>>>(fin, parts, d_cb, d_n3, d_regs,
                                                                    d_rid, nb, d_kb, d_rows, d_keep,
                                                                    0));
        rows.resize((size_t)kb[nb]);
        SEDEF_CUDA(cudaMemcpyAsync(rows.data(), d_rows, (size_t)kb[nb] * sizeof(sedef_sd_t),
                                   cudaMemcpyDeviceToHost, st));
        SEDEF_CUDA(cudaStreamSynchronize(st));
      }
    }
    all.insert(all.end(), rows.begin(), rows.end());
    ctx_pool_restore(ctx, used_before);
    r0 = r1;
  }
  *nout = (int64_t)all.size();
  if ((int64_t)all.size() > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_chain2: output buffer too small");
  if (!all.empty())
    SEDEF_CUDA(cudaMemcpyAsync(out, all.data(), all.size() * sizeof(sedef_sd_t), cudaMemcpyHostToDevice,
                               st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // namespace sedef
