// a4-a6: candidate lookup, sliding count of shared minimizers against m(s),
// and the winnowed MinHash refine (Sections 2.2 and 3.1).
//
// Shared-memory tiers (one CTA per query window, persistent CTAs):
//   1. the window's query minimizers are sorted by hash in shared memory and
//      deduplicated into W_Q (s hashes, each with its strand set);
//   2. every posting of every hash of W_Q is a hit (t, hid, o).  Hits are
//      counted into direct-mapped 16-bit counters keyed by (t >> 10, o):
//      a target window [j, j+n-k] lies inside bins j>>10 and (j>>10)+1, so a
//      j can only pass when those two counters sum to m or more (aliasing
//      only adds false candidates).  The table has the smallest power of two
//      >= 4 H slots (H = the window's hits), at least 2,048 and at most the
//      tier's size, so the prefilter stays selective when posting lists are
//      long (a large target);
//   3. hits whose bin pair can pass are collected and sorted by (o, t); the
//      exact sweep (one thread, per-hash counters) runs only over j ranges
//      where m consecutive hits fit in n-k bases.  Any j whose true count
//      reaches m has all of its hits collected, and a count computed from a
//      subset never exceeds the true one, so the runs are exact.
// The tiers differ only in their shared-memory budget: an optional warp tier
// (one warp per small window), tier 1 (autotuned shape), tier 2 (more
// collected hits) and the wide tier (32,768 counters) for windows with more
// than 4,096 hits, which tiers 1 and 2 hand over before enumerating them.
// Windows no tier can hold go to a global path that writes their hits to
// global memory, radix-sorts them by (window, o, t) and runs the same sweep.
//
// Refine (k_refine_batch): each run's domain, W_Q u (target minimizers of the
// run's span that can change the estimate), is sorted by a warp into a
// per-warp slot; then one lane per run rolls the target window over the
// run's breakpoints, keeping presence and sharedness counters and the s-th
// present hash, so the estimate |S(W_Q u W_T) n W_Q n W_T| is exact at every
// breakpoint.  Runs whose domain exceeds the batched kernel's slots go to
// k_refine (one warp per run, bitsets over the sorted domain).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>

#include "common.cuh"

namespace sedef {

namespace {

constexpr int kQCap = 256;        // query records per window (fast path)
constexpr int kBinShift = 10;     // 1024-base bins (>= n - k + 1)
constexpr int kSlots = 2048;      // (bin, o) counters (16-bit)
constexpr int kHMax = 65535;      // hits per window (fast path; 16-bit counters)
constexpr uint32_t kNone = 0xFFFFFFFFu;

struct FArgs {
  const uint64_t* qrec;
  const uint64_t* trec;
  const uint64_t* tsorted;
  const uint32_t* toff;
  const int64_t* tseq;   // target sequence offsets (ntseq + 1)
  const int64_t* qseq;   // query sequence offsets (nqseq + 1)
  const int32_t* mtab;
  const uint32_t* win_i;   // window start (global)
  const uint32_t* win_qa;  // first query record of the window
  const uint32_t* win_qb;  // one past the last
  const int32_t* win_seq;  // query sequence of the window
  // per query record: its hash's posting range narrowed to the record's own
  // genome (batch self-search), or (kNone, 0) when the list passes max_occ;
  // nullptr when the tiers look postings up themselves
  const uint2* qpost;
  const uint32_t* tsamp;  // positions of every kSampleStride-th index entry, or nullptr
  int64_t nwin;
  int ntseq, nqseq;
  int64_t ttotal;  // target total length
  int k, n, span, max_occ, self_mode, overlap;
  sedef_run_t* runs;
  unsigned long long* nruns;
  int64_t run_cap;
  uint32_t* ov_list;
  unsigned int* nov;
  unsigned int* next_window;
  unsigned long long* stats;  // [0] hits enumerated, [1] hits collected (fast path)
};

// ----------------------------------------------------------- run emission --

struct RunState {
  bool open;
  int64_t ja, jb, jmx;
  int mx;
  // the target sequence that held the last position looked up
  int64_t seq_lo = 0, seq_hi = -1;
  int seq = 0;
};

struct WinInfo {
  int64_t i;
  int qseq;
  int s, m, o;
};

__device__ __forceinline__ void emit_run(const FArgs& a, const WinInfo& w, RunState& r) {
  if (!r.open) return;
  r.open = false;
  const unsigned long long slot = atomicAdd(a.nruns, 1ull);
  if ((int64_t)slot < a.run_cap) {
    sedef_run_t out;
    out.i = (uint32_t)w.i;
    out.j_a = (uint32_t)r.ja;
    out.j_b = (uint32_t)r.jb;
    out.j_at_max = (uint32_t)r.jmx;
    out.j_star = 0;
    out.s = (uint16_t)w.s;
    out.m = (uint16_t)w.m;
    out.max_shared = (uint16_t)r.mx;
    out.est = 0;
    out.den = 0;
    out.o = (uint8_t)w.o;
    out.keep = 0;
    a.runs[slot] = out;
  }
}

// The shared count is `shared` on every j of [j0, j1]; split by target
// sequence and the validity rules, and extend / open / close runs.
__device__ void segment(const FArgs& a, const WinInfo& w, RunState& r, int64_t j0, int64_t j1,
                        int shared) {
  if (shared < w.m) {
    emit_run(a, w, r);
    return;
  }
  int64_t x = j0 < 0 ? 0 : j0;
  while (x <= j1 && x < a.ttotal) {
    if (x < r.seq_lo || x >= r.seq_hi) {
      r.seq = seq_of(a.tseq, a.ntseq, x);
      r.seq_lo = a.tseq[r.seq];
      r.seq_hi = a.tseq[r.seq + 1];
    }
    const int u = r.seq;
    const int64_t st = r.seq_lo, en = r.seq_hi;
    int64_t lo = st, hi = en - a.n;
    bool ok = true;
    if (a.self_mode) {
      if (u < w.qseq) ok = false;
      else if (u == w.qseq) lo = max(lo, w.i + a.n - a.overlap);
      else if (a.self_mode == 2) ok = false;  // independent genomes
    }
    const int64_t pend = min(j1, en - 1);
    const int64_t vlo = max(x, lo), vhi = min(pend, hi);
    if (ok && vlo <= vhi) {
      if (r.open && vlo == r.jb + 1) {
        r.jb = vhi;
      } else {
        emit_run(a, w, r);
        r.open = true;
        r.ja = vlo;
        r.jb = vhi;
        r.mx = -1;
      }
      if (shared > r.mx) {
        r.mx = shared;
        r.jmx = vlo;
      }
    }
    x = pend + 1;
  }
}

// Exact sweep of one dense group [Jlo, Jhi] over one strand's hits (sorted
// by t; get(x) returns (t, hid)).  cnt[] holds one zeroed counter per hash
// id and is zero again on return.  A group never shares a run with another
// (they are separated by target starts that cannot pass), so the run state
// starts empty and every run is emitted before returning.  Single thread.
template <typename Get>
__device__ void sweep_group(const FArgs& a, const WinInfo& w, Get get, int64_t L, uint16_t* cnt,
                            int64_t Jlo, int64_t Jhi) {
  const int span = a.span;
  RunState r;
  r.open = false;
  int64_t lo = 0, hi = L;  // first hit with t >= Jlo
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)get(mid).x < Jlo) lo = mid + 1; else hi = mid;
  }
  int64_t e = lo, l = lo;
  int shared = 0;
  int64_t j = Jlo;
  while (e < L && (int64_t)get(e).x <= j + span) {
    if (cnt[get(e).y]++ == 0) ++shared;
    ++e;
  }
  while (true) {
    const int64_t ne = e < L ? (int64_t)get(e).x - span : INT64_MAX;
    const int64_t nl = l < e ? (int64_t)get(l).x + 1 : INT64_MAX;
    int64_t nx = min(ne, nl);
    if (nx > Jhi + 1) nx = Jhi + 1;
    segment(a, w, r, j, nx - 1, shared);
    if (nx > Jhi) break;
    j = nx;
    while (l < e && (int64_t)get(l).x + 1 <= j) {
      if (--cnt[get(l).y] == 0) --shared;
      ++l;
    }
    while (e < L && (int64_t)get(e).x - span <= j) {
      if (cnt[get(e).y]++ == 0) ++shared;
      ++e;
    }
  }
  for (int64_t x = l; x < e; ++x) cnt[get(x).y] = 0;
  emit_run(a, w, r);
}

__device__ __forceinline__ int64_t warp_excl_max(int64_t v) {
  const int lane = lane_id();
  int64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d && o > inc) inc = o;
  }
  const int64_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
  return lane == 0 ? INT64_MIN : ex;
}

// Dense groups of one strand's t-sorted hits (warp-cooperative; every lane
// calls).  Hit x is dense when the m hits from x on fit in n-k bases; every
// j whose count reaches m lies in [t(x+m-1) - (n-k), t(x)] for some dense x.
// Overlapping or touching such ranges form a group; emit(Jlo, Jhi) is called
// by every lane, once per group, in increasing order.
template <typename Get, typename Emit>
__device__ void find_groups(Get get, int64_t L, int m, int span, Emit emit) {
  const int lane = lane_id();
  int64_t carry_hi = INT64_MIN;  // largest jhi of the dense hits seen so far
  int64_t cur_lo = 0;
  bool open = false;
  for (int64_t base = 0; base + m - 1 < L; base += 32) {
    const int64_t x = base + lane;
    bool dense = false;
    int64_t jlo = 0, jhi = INT64_MIN;
    if (x + m - 1 < L) {
      const int64_t ta = get(x).x, tb = get(x + m - 1).x;
      if (tb - ta <= span) {
        dense = true;
        jlo = tb - span;
        jhi = ta;
      }
    }
    int64_t before = warp_excl_max(dense ? jhi : INT64_MIN);
    if (carry_hi > before) before = carry_hi;
    const bool start = dense && (before == INT64_MIN || jlo > before + 1);
    unsigned starts = __ballot_sync(0xffffffffu, start);
    while (starts) {
      const int ls = __ffs(starts) - 1;
      starts &= starts - 1;
      const int64_t b_ls = __shfl_sync(0xffffffffu, before, ls);
      const int64_t lo_ls = __shfl_sync(0xffffffffu, jlo, ls);
      if (open) emit(cur_lo, b_ls);
      cur_lo = lo_ls;
      open = true;
    }
    int64_t mx = dense ? jhi : INT64_MIN;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const int64_t o = __shfl_xor_sync(0xffffffffu, mx, d);
      if (o > mx) mx = o;
    }
    if (mx > carry_hi) carry_hi = mx;
  }
  if (open) emit(cur_lo, carry_hi);
}

// ------------------------------------------------------ block bitonic sort --

template <typename T>
__device__ void block_sort(T* v, int n) {  // n a power of two
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        // pair t of this stage: stride is a power of two
        const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const T x = v[lo], y = v[hi];
        if ((x > y) == asc) {
          v[lo] = y;
          v[hi] = x;
        }
      }
      __syncthreads();
    }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Builds W_Q for a window from its query records (already in qkey[0..c) as
// hash<<1|strand), sorted in place.  Writes dh (hash), dm (strand mask),
// pst/plen (posting range) for the kept hashes; returns s.  Uses the whole
// block.  `flag` needs c ints of scratch.
struct QBuild {
  uint32_t* qkey;
  uint32_t* dh;
  uint8_t* dm;
  uint32_t* pst;
  uint32_t* plen;
  int* tmp;
};

// Record positions of every kSampleStride-th entry of the sorted index
// (samp[k] = pos(idx[k * kSampleStride])): a search first brackets its
// answer between two samples, an array small enough to stay in L2, and then
// reads one stretch of kSampleStride index entries (one 128-byte line).
constexpr int kSampleShift = 4, kSampleStride = 1 << kSampleShift;

// pos_lower_bound over the samples, then over the bracketed stretch.
__host__ __device__ __forceinline__ uint32_t pos_lower_bound_sampled(const uint64_t* idx,
                                                                     const uint32_t* samp,
                                                                     uint32_t a0, uint32_t a1,
                                                                     int64_t key) {
  uint32_t lo = a0, hi = a1;  // pos(x) < key below lo; pos(x) >= key from hi (or hi = a1)
  if (a0 < a1) {
    const uint32_t k0 = (a0 + kSampleStride - 1) >> kSampleShift, k1 = (a1 - 1) >> kSampleShift;
    if (k0 <= k1) {  // samples inside the list: the first one at or past key
      uint32_t l = k0, h = k1 + 1;
      while (l < h) {
        const uint32_t m = l + ((h - l) >> 1);
        if ((int64_t)samp[m] >= key) h = m; else l = m + 1;
      }
      if (l <= k1) hi = l << kSampleShift;
      if (l > k0) lo = ((l - 1) << kSampleShift) + 1;
    }
  }
  while (lo < hi) {
    const uint32_t m = lo + ((hi - lo) >> 1);
    if ((int64_t)rec_pos(idx[m]) >= key) hi = m; else lo = m + 1;
  }
  return lo;
}

// Narrows a posting list [*st, *st + *len) to the positions in [lo, hi)
// (one genome of a batch).
__host__ __device__ __forceinline__ void posting_window(const uint64_t* idx, const uint32_t* samp,
                                                        uint32_t* st, uint32_t* len, int64_t lo,
                                                        int64_t hi) {
  const uint32_t a0 = *st, a1 = *st + *len;
  const uint32_t l =
      samp ? pos_lower_bound_sampled(idx, samp, a0, a1, lo) : pos_lower_bound(idx, a0, a1, lo);
  const uint32_t l2 = pos_gallop_forward(idx, l, a1, hi);
  *st = l;
  *len = l2 - l;
}

__global__ void k_sample_pos(const uint64_t* __restrict__ idx, int64_t nt, const uint32_t* dnt,
                             uint32_t* __restrict__ samp) {
  const int64_t n = dnt ? (int64_t)*dnt : nt;
  const int64_t ns = (n + kSampleStride - 1) >> kSampleShift;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ns;
       k += (int64_t)gridDim.x * blockDim.x)
    samp[k] = rec_pos(idx[k << kSampleShift]);
}

// Posting range of every query record of a batch self-search, resolved once
// per record rather than once per window that holds it (a record lies in
// n / step windows), by threads that each follow one record's chain of
// dependent loads.  Records are sorted by position, so neighbouring threads
// share a genome and often a hash.
__global__ void k_qpost(FArgs a, int64_t nq, const uint32_t* dnq, uint2* out) {
  const int64_t n = dnq ? (int64_t)*dnq : nq;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = a.qrec[x];
    const uint32_t h = rec_hash(r);
    uint32_t st = a.toff[h], len = a.toff[h + 1] - st;
    if (a.max_occ > 0 && (int)len > a.max_occ) {
      out[x] = make_uint2(kNone, 0u);
      continue;
    }
    const int sq = seq_of(a.qseq, a.nqseq, (int64_t)rec_pos(r));
    posting_window(a.tsorted, a.tsamp, &st, &len, a.tseq[sq], a.tseq[sq + 1]);
    out[x] = make_uint2(st, len);
  }
}

__device__ int build_wq(const FArgs& a, QBuild q, int c, int64_t seq_lo = 0, int64_t seq_hi = 0) {
  const int np = next_pow2(c < 2 ? 2 : c);
  for (int x = threadIdx.x; x < np; x += blockDim.x)
    if (x >= c) q.qkey[x] = kNone;
  __syncthreads();
  block_sort(q.qkey, np);
  // distinct hashes: first occurrence flags, block-wide compaction
  __shared__ int s_count;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int base = 0; base < c; base += blockDim.x) {
    const int x = base + threadIdx.x;
    int keep = 0;
    uint32_t h = 0, st = 0, len = 0, mask = 0;
    if (x < c) {
      h = q.qkey[x] >> 1;
      if (x == 0 || (q.qkey[x - 1] >> 1) != h) {
        for (int y = x; y < c && (q.qkey[y] >> 1) == h; ++y) mask |= 1u << (q.qkey[y] & 1u);
        st = a.toff[h];
        len = a.toff[h + 1] - st;
        keep = (a.max_occ > 0 && (int)len > a.max_occ) ? 0 : 1;
        // independent genomes: only the query's own sequence can hold targets
        if (keep && a.self_mode == 2)
          posting_window(a.tsorted, a.tsamp, &st, &len, seq_lo, seq_hi);
      }
    }
    int tot;
    const int ex = block_exclusive_sum(keep, q.tmp, &tot);
    if (keep) {
      const int d = s_count + ex;
      q.dh[d] = h;
      q.dm[d] = (uint8_t)mask;
      q.pst[d] = st;
      q.plen[d] = len;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_count += tot;
    __syncthreads();
  }
  return s_count;
}

// Posting ranges in index order (eager batch self-search).  The query
// records of a self-search are the index's own records, and the entries of
// the index with one hash in one genome form a run that is the narrowed
// posting range of each of its records.  So the ranges come from one walk
// over the index: a warp reads 32 consecutive entries, splits them into runs
// by (hash, genome), and searches only for the ends of the runs that leave
// its 32 entries.  Each range goes to its record, found by the rank of the
// record's position among all record positions: a bitmap of the positions
// with the count of set bits before each 32-bit word.
struct RankWord {
  uint32_t before;  // record positions below this word's first position
  uint32_t bits;    // record positions inside it
};

// bits[p >> 5] |= 1 << (p & 31) for every record position p (rec sorted by
// position, so the lanes with one word are consecutive: each run of them is
// OR-ed into its first lane, which alone writes).
__global__ void k_pos_bits(const uint64_t* __restrict__ rec, int64_t n, uint32_t* __restrict__ bits) {
  const int lane = lane_id();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
       base += stride) {
    const int64_t x = base + lane;
    const bool ok = x < n;
    const uint32_t p = ok ? rec_pos(rec[x]) : 0u;
    const uint32_t w = ok ? (p >> 5) : 0xFFFFFFFFu;
    uint32_t v = ok ? (1u << (p & 31)) : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t ov = __shfl_down_sync(0xffffffffu, v, d);
      const uint32_t ow = __shfl_down_sync(0xffffffffu, w, d);
      if (lane + d < 32 && ow == w) v |= ov;
    }
    const uint32_t pw = __shfl_up_sync(0xffffffffu, w, 1);
    if (ok && (lane == 0 || pw != w)) atomicOr(bits + w, v);
  }
}

__global__ void k_pos_popc(const uint32_t* __restrict__ bits, int64_t nw, uint32_t* __restrict__ cnt) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(bits[w]);
}

__global__ void k_rank_words(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ before,
                             int64_t nw, RankWord* __restrict__ rw) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x)
    rw[w] = RankWord{before[w], bits[w]};
}

__global__ void k_qpost_index(FArgs a, int64_t n, const RankWord* __restrict__ rw,
                              uint2* __restrict__ out) {
  const int lane = lane_id();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; e0 < n;
       e0 += stride) {
    const int64_t e = e0 + lane;
    const int L = (int)(n - 1 - e0 < 31 ? n - 1 - e0 : 31);  // last lane with an entry
    const bool ok = lane <= L;
    uint32_t h = 0xFFFFFFFFu, p = 0;
    int g = -1;
    if (ok) {
      const uint64_t r = a.tsorted[e];
      h = rec_hash(r);
      p = rec_pos(r);
      g = seq_of(a.tseq, a.ntseq, (int64_t)p);
    }
    const uint32_t ph = __shfl_up_sync(0xffffffffu, h, 1), nh = __shfl_down_sync(0xffffffffu, h, 1);
    const int pg = __shfl_up_sync(0xffffffffu, g, 1), ng = __shfl_down_sync(0xffffffffu, g, 1);
    const bool st = ok && (lane == 0 || ph != h || pg != g);
    const bool en = ok && (lane == L || nh != h || ng != g);
    const unsigned sb = __ballot_sync(0xffffffffu, st), eb = __ballot_sync(0xffffffffu, en);
    const int fl = 31 - __clz(sb & ((2u << lane) - 1u));  // first lane of my run
    const int ll = __ffs(eb & ~((1u << lane) - 1u)) - 1;  // last lane of my run
    // the run holding the first entry may start before it, the run holding
    // the last one may end after it
    uint32_t s0 = 0, eL = 0;
    if (lane == 0) s0 = pos_lower_bound(a.tsorted, a.toff[h], (uint32_t)e0, a.tseq[g]);
    if (lane == L) eL = pos_gallop_forward(a.tsorted, (uint32_t)e + 1, a.toff[h + 1], a.tseq[g + 1]);
    s0 = __shfl_sync(0xffffffffu, s0, 0);
    eL = __shfl_sync(0xffffffffu, eL, L);
    if (ok) {
      const uint32_t rs = fl == 0 ? s0 : (uint32_t)(e0 + fl);
      const uint32_t re = ll == L ? eL : (uint32_t)(e0 + ll + 1);
      uint2 v = make_uint2(rs, re - rs);
      if (a.max_occ > 0 && (int)(a.toff[h + 1] - a.toff[h]) > a.max_occ) v = make_uint2(kNone, 0u);
      const RankWord q = rw[p >> 5];
      out[q.before + __popc(q.bits & ((1u << (p & 31)) - 1u))] = v;
    }
  }
}

// ------------------------------------------------------------- fast path --

template <int TPB, int LCAP, int GCAP, int SLOTS>
struct FastSmemT {
  uint32_t qkey[kQCap];
  uint32_t dh[kQCap];
  uint32_t pst[kQCap];
  uint32_t plen[kQCap];
  uint32_t pre[kQCap + 1];
  uint8_t dm[kQCap];
  uint32_t slots[SLOTS / 2];  // two 16-bit counters per word
  unsigned long long hits[LCAP];
  uint32_t glo[GCAP];     // dense groups: Jlo (clamped to >= 0), Jhi
  uint32_t ghi[GCAP];
  uint16_t cnt[TPB / 32][kQCap];  // one counter array per warp
  int tmp[33];
  int64_t win;
  int nhit, s, ovf, ng0, ng;
};

// Where a tier of the shared-memory path takes its windows from (all
// windows, or a list) and where it sends the windows it cannot hold.
struct TierIO {
  const uint32_t* in_list;        // nullptr: windows 0..nwin-1
  const unsigned int* in_count;
  uint32_t* out_list;
  unsigned int* out_count;
  unsigned int* next;             // work counter of this tier
  int stats;                      // count hits in the filter statistics
  // windows with more than hlim hits are handed over before their hits are
  // enumerated: to wide_list when set (the wide tier), else to out_list
  uint32_t hlim = 0xFFFFFFFFu;
  uint32_t* wide_list = nullptr;
  unsigned int* wide_count = nullptr;
};

// (bin, o) counter slot of a hit in a direct-mapped table of mask+1 slots
__device__ __forceinline__ uint32_t slot_of(uint32_t t, uint32_t o, uint32_t mask) {
  return (((t >> kBinShift) << 1) | o) & mask;
}

__device__ __forceinline__ uint32_t slot_count(const uint32_t* slots, uint32_t s) {
  return (slots[s >> 1] >> ((s & 1) * 16)) & 0xFFFFu;
}

// Enumerates the window's hits: calls f(t, hid, o) for every posting of every
// kept hash with a compatible relative strand (self positions skipped).
template <typename Smem, typename F>
__device__ __forceinline__ void for_hits(const FArgs& a, const Smem& S, int64_t i, int H, F f) {
  for (int e = threadIdx.x; e < H; e += blockDim.x) {
    int lo = 0, hi = S.s;  // list with pre[l] <= e < pre[l+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((int)S.pre[mid] <= e) lo = mid; else hi = mid;
    }
    const uint64_t r = __ldg(a.tsorted + S.pst[lo] + (uint32_t)(e - (int)S.pre[lo]));
    const uint32_t t = rec_pos(r), st = rec_strand(r);
    if (a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span) continue;
    const uint32_t qm = S.dm[lo];
    if ((qm >> st) & 1u) f(t, (uint32_t)lo, 0u);
    if ((qm >> (st ^ 1u)) & 1u) f(t, (uint32_t)lo, 1u);
  }
}

// One query window through a shared-memory tier: W_Q, the prefilter, the
// collected hits, dense groups and the exact sweep; a window the tier
// cannot hold goes to io.out_list (or io.wide_list).  Every thread of the
// block calls it.
template <int TPB, int LCAP, int GCAP, int SLOTS>
__device__ void fast_window(const FArgs& a, const TierIO& io,
                            FastSmemT<TPB, LCAP, GCAP, SLOTS>& S, int64_t wdx) {
  constexpr int kFThreads = TPB;
  constexpr int kLCap = LCAP;
  constexpr int kGCap = GCAP;
  const int64_t i = __ldcg(a.win_i + wdx);
  const uint32_t qa = __ldcg(a.win_qa + wdx), qb = __ldcg(a.win_qb + wdx);
  const int c = (int)(qb - qa);
  if (c == 0) return;
  if (c > kQCap) {
    if (threadIdx.x == 0) io.out_list[atomicAdd(io.out_count, 1u)] = (uint32_t)wdx;
    return;
  }
  for (int x = threadIdx.x; x < c; x += blockDim.x) {
    const uint64_t r = __ldcg(a.qrec + qa + x);
    S.qkey[x] = (rec_hash(r) << 1) | rec_strand(r);
  }
  __syncthreads();
  QBuild qb_;
  qb_.qkey = S.qkey;
  qb_.dh = S.dh;
  qb_.dm = S.dm;
  qb_.pst = S.pst;
  qb_.plen = S.plen;
  qb_.tmp = S.tmp;
  int64_t seq_lo = 0, seq_hi = 0;
  if (a.self_mode == 2) {
    const int sq = __ldcg(a.win_seq + wdx);
    seq_lo = a.tseq[sq];
    seq_hi = a.tseq[sq + 1];
  }
  const int s = build_wq(a, qb_, c, seq_lo, seq_hi);
  if (s == 0) return;
  // prefix of posting lengths (hit enumeration)
  if (threadIdx.x < 32) {
    uint32_t run = 0;
    for (int base = 0; base < s; base += 32) {
      const int x = base + threadIdx.x;
      const uint32_t v = x < s ? S.plen[x] : 0u;
      const uint32_t inc = warp_inclusive_sum(v);
      if (x < s) S.pre[x] = run + inc - v;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (threadIdx.x == 0) S.pre[s] = run;
  }
  if (threadIdx.x == 0) {
    S.s = s;
    S.nhit = 0;
    S.ovf = 0;
  }
  __syncthreads();
  const uint32_t H = S.pre[s];
  if (H == 0) return;
  if (H > (uint32_t)kHMax || H > io.hlim) {
    if (threadIdx.x == 0) {
      if (H <= (uint32_t)kHMax && io.wide_list)
        io.wide_list[atomicAdd(io.wide_count, 1u)] = (uint32_t)wdx;
      else
        io.out_list[atomicAdd(io.out_count, 1u)] = (uint32_t)wdx;
    }
    return;
  }
  uint32_t nslots = kSlots;
  while (nslots < 4u * H && nslots < (uint32_t)SLOTS) nslots <<= 1;
  const uint32_t smask = nslots - 1;
  for (uint32_t x = threadIdx.x; x < nslots / 2; x += blockDim.x) S.slots[x] = 0;
  __syncthreads();
  const int m = a.mtab[s];
  // pass 1: (bin, o) counts
  for_hits(a, S, i, (int)H, [&](uint32_t t, uint32_t, uint32_t o) {
    const uint32_t sl = slot_of(t, o, smask);
    atomicAdd(&S.slots[sl >> 1], 1u << ((sl & 1) * 16));
  });
  __syncthreads();
  // pass 2: collect the hits of bins whose pair (b, b+1) or (b-1, b) may pass
  for_hits(a, S, i, (int)H, [&](uint32_t t, uint32_t hid, uint32_t o) {
    const uint32_t b = t >> kBinShift;
    const uint32_t c0 = slot_count(S.slots, slot_of(t, o, smask));
    const uint32_t cn = slot_count(S.slots, (((b + 1) << 1) | o) & smask);
    bool need = c0 + cn >= (uint32_t)m;
    if (!need && b > 0) {
      const uint32_t cp = slot_count(S.slots, (((b - 1) << 1) | o) & smask);
      need = cp + c0 >= (uint32_t)m;
    }
    if (need) {
      const int at = atomicAdd(&S.nhit, 1);
      if (at < kLCap)
        S.hits[at] = ((unsigned long long)o << 63) | ((unsigned long long)t << 20) | hid;
    }
  });
  __syncthreads();
  const int L = S.nhit;
  if (L > kLCap) {
    if (threadIdx.x == 0) io.out_list[atomicAdd(io.out_count, 1u)] = (uint32_t)wdx;
    return;
  }
  // statistics count the windows this tier finishes (each window once)
  if (L < m) {
    if (io.stats && threadIdx.x == 0) {
      atomicAdd(a.stats + 0, (unsigned long long)H);
      atomicAdd(a.stats + 1, (unsigned long long)L);
    }
    return;
  }
  const int np = next_pow2(L < 2 ? 2 : L);
  for (int x = L + threadIdx.x; x < np; x += blockDim.x) S.hits[x] = ~0ull;
  __syncthreads();
  block_sort(S.hits, np);
  // dense groups of both strands (warp 0), then one warp per group
  int split = 0;
  {
    // first hit with o = 1
    int lo2 = 0, hi2 = L;
    while (lo2 < hi2) {
      const int mid = (lo2 + hi2) >> 1;
      if ((S.hits[mid] >> 63) == 0) lo2 = mid + 1; else hi2 = mid;
    }
    split = lo2;
  }
  if (threadIdx.x < 32) {
    int ng = 0;
    for (int o = 0; o < 2; ++o) {
      const unsigned long long* base = S.hits + (o ? split : 0);
      const int64_t cnt = o ? L - split : split;
      find_groups(
          [&](int64_t x) {
            const unsigned long long h = base[x];
            return make_uint2((uint32_t)(h >> 20), (uint32_t)(h & 0xFFFFFu));
          },
          cnt, m, a.span, [&](int64_t lo, int64_t hi) {
            if (threadIdx.x == 0 && ng < kGCap) {
              S.glo[ng] = (uint32_t)(lo < 0 ? 0 : lo);
              S.ghi[ng] = (uint32_t)hi;
            }
            ++ng;
          });
      if (o == 0 && threadIdx.x == 0) S.ng0 = ng;
    }
    if (threadIdx.x == 0) S.ng = ng;
  }
  __syncthreads();
  const int ng = S.ng, ng0 = S.ng0;
  if (ng > kGCap) {
    if (threadIdx.x == 0) io.out_list[atomicAdd(io.out_count, 1u)] = (uint32_t)wdx;
    return;
  }
  if (io.stats && threadIdx.x == 0) {
    atomicAdd(a.stats + 0, (unsigned long long)H);
    atomicAdd(a.stats + 1, (unsigned long long)L);
  }
  {
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      WinInfo w;
      w.i = i;
      w.qseq = __ldcg(a.win_seq + wdx);
      w.s = s;
      w.m = m;
      for (int g = warp; g < ng; g += kFThreads / 32) {
        w.o = g < ng0 ? 0 : 1;
        const unsigned long long* base = S.hits + (w.o ? split : 0);
        const int64_t cnt = w.o ? L - split : split;
        sweep_group(a, w,
                    [&](int64_t x) {
                      const unsigned long long h = base[x];
                      return make_uint2((uint32_t)(h >> 20), (uint32_t)(h & 0xFFFFFu));
                    },
                    cnt, S.cnt[warp], (int64_t)S.glo[g], (int64_t)S.ghi[g]);
      }
    }
  }
}

// SLOTS is the largest (bin, o) table; a window uses the smallest power of
// two >= 4 H (at least 2,048 slots), so that aliasing stays rare however
// many hits the window has.
template <int TPB, int LCAP, int GCAP, int SLOTS>
__global__ void __launch_bounds__(TPB) k_filter_fast(FArgs a, TierIO io) {
  using FastSmem = FastSmemT<TPB, LCAP, GCAP, SLOTS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FastSmem& S = *reinterpret_cast<FastSmem*>(smem_raw);
  for (int x = threadIdx.x; x < kQCap * (TPB / 32); x += blockDim.x) (&S.cnt[0][0])[x] = 0;
  const int64_t count = io.in_list ? (int64_t)*io.in_count : a.nwin;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t k = atomicAdd(io.next, 1u);
      S.win = k < count ? (io.in_list ? (int64_t)io.in_list[k] : k) : -1;
    }
    __syncthreads();
    const int64_t wdx = S.win;
    if (wdx < 0) break;
    fast_window<TPB, LCAP, GCAP, SLOTS>(a, io, S, wdx);
  }
}

// ------------------------------------------------------------- warp tier --
//
// Small windows (at most 128 query records, 4,096 hits, 256 collected hits
// and 64 dense groups) take the same steps as k_filter_fast with one warp
// per window and no block barriers: W_Q by insertion into a hash table (no
// sort), hits found 32 at a time by a shuffle search over the posting prefix
// sums, (bin, o) counters as the prefilter (a window with no adjacent bin
// pair reaching m stops there), collected hits sorted per strand, dense
// groups found by the warp and swept exactly by lane 0.  Windows past any
// limit go to the next tier.

constexpr int kWQ = 128;        // query records
static_assert(kWQ <= 128, "a lane holds at most four of a window's query records");
constexpr int kWSlots = 1024;   // (bin, o) 16-bit counters (512 bins)
constexpr int kWL = 256;        // collected hits
constexpr int kWG = 64;         // dense groups
constexpr int kWH = 4096;       // enumerated hits
constexpr int kWWarps = 8;
constexpr int kWTab = 2 * kWL;   // W_Q hash-table slots (u32, over the hit buffer)
static_assert(kWTab >= 2 * kWQ && kWTab <= kWSlots / 2, "the W_Q table and its masks must fit");

struct WarpSmem {
  uint32_t qkey[kWQ];
  uint32_t pst[kWQ];
  uint32_t plen[kWQ];
  uint32_t pre[kWQ + 1];
  uint8_t dm[kWQ];
  uint32_t slots[kWSlots / 2];
  unsigned long long hits[kWL];
  uint32_t glo[kWG];
  uint32_t ghi[kWG];
  uint16_t cnt[kWQ];
  int nhit;
};

template <typename T>
__device__ void warp_sort(T* v, int n) {  // n a power of two
  const int lane = lane_id();
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < (n >> 1); t += 32) {
        const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const T x = v[lo], y = v[hi];
        if ((x > y) == asc) {
          v[lo] = y;
          v[hi] = x;
        }
      }
      __syncwarp();
    }
}

__device__ __forceinline__ uint32_t wslot_of(uint32_t t, uint32_t o) {
  return (((t >> kBinShift) << 1) | o) & (kWSlots - 1);
}

__global__ void __launch_bounds__(32 * kWWarps) k_filter_warp(FArgs a, TierIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
  for (int x = lane; x < kWQ; x += 32) S.cnt[x] = 0;
  const int64_t count = io.in_list ? (int64_t)*io.in_count : a.nwin;
  auto hand_over = [&](int64_t wdx) {
    if (lane == 0) io.out_list[atomicAdd(io.out_count, 1u)] = (uint32_t)wdx;
  };
  while (true) {
    int64_t k = 0;
    if (lane == 0) k = (int64_t)atomicAdd(io.next, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= count) break;
    const int64_t wdx = io.in_list ? (int64_t)io.in_list[k] : k;
    const int64_t i = a.win_i[wdx];
    const uint32_t qa = a.win_qa[wdx], qb = a.win_qb[wdx];
    const int c = (int)(qb - qa);
    if (c == 0) continue;
    if (c > kWQ) {
      hand_over(wdx);
      continue;
    }
    // W_Q: the window's distinct hashes, by insertion into an open-addressing
    // table (key hash + 1, linear probing from the hash's low bits) laid
    // over the hit buffer, with each hash's strand mask beside it in the
    // counter table (both are rebuilt later for the hits).  The order of W_Q
    // plays no part in the counts, so no sort is needed.  A record that
    // inserts its hash first owns it.
    uint32_t* tab = reinterpret_cast<uint32_t*>(S.hits);
    uint32_t* tmask = S.slots;
    for (int x = lane; x < kWTab; x += 32) {
      tab[x] = 0u;
      tmask[x] = 0u;
    }
    __syncwarp();
    const bool packed = a.qpost != nullptr;
    uint32_t own_slot[kWQ / 32], own_h[kWQ / 32];
    unsigned owner = 0;
#pragma unroll
    for (int ch = 0; ch < kWQ / 32; ++ch) {
      const int x = ch * 32 + lane;
      own_slot[ch] = 0;
      own_h[ch] = 0;
      if (x < c) {
        const uint64_t r = __ldg(a.qrec + qa + x);
        const uint32_t h = rec_hash(r);
        uint32_t slot = h & (kWTab - 1);
        while (true) {  // at most kWQ keys in kWTab slots: a free slot is always found
          const uint32_t old = atomicCAS(&tab[slot], 0u, h + 1u);
          if (old == 0u) {
            owner |= 1u << ch;
            break;
          }
          if (old == h + 1u) break;
          slot = (slot + 1u) & (kWTab - 1);
        }
        atomicOr(&tmask[slot], 1u << rec_strand(r));
        own_slot[ch] = slot;
        own_h[ch] = h;
      }
    }
    int64_t seq_lo = 0, seq_hi = 0;
    if (a.self_mode == 2) {
      const int sq = a.win_seq[wdx];
      seq_lo = a.tseq[sq];
      seq_hi = a.tseq[sq + 1];
    }
    __syncwarp();
    int s = 0;
#pragma unroll
    for (int ch = 0; ch < kWQ / 32; ++ch) {
      if (ch * 32 >= c) break;
      const int x = ch * 32 + lane;
      bool keep = false;
      uint32_t st = 0, len = 0, mask = 0;
      if ((owner >> ch) & 1u) {
        const uint32_t h = own_h[ch];
        mask = tmask[own_slot[ch]];
        if (packed) {
          const uint2 pp = a.qpost[qa + x];
          st = pp.x;
          len = pp.y;
          keep = pp.x != kNone;
        } else {
          st = a.toff[h];
          len = a.toff[h + 1] - st;
          keep = !(a.max_occ > 0 && (int)len > a.max_occ);
          if (keep && a.self_mode == 2) posting_window(a.tsorted, a.tsamp, &st, &len, seq_lo, seq_hi);
        }
      }
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int d = s + __popc(km & lanemask_lt());
        S.pst[d] = st;
        S.plen[d] = len;
        S.dm[d] = (uint8_t)mask;
      }
      s += __popc(km);
    }
    __syncwarp();
    if (s == 0) continue;
    // prefix sums of the posting lengths
    uint32_t run = 0;
    for (int base = 0; base < s; base += 32) {
      const int x = base + lane;
      const uint32_t v = x < s ? S.plen[x] : 0u;
      const uint32_t inc = warp_inclusive_sum(v);
      if (x < s) S.pre[x] = run + inc - v;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) S.pre[s] = run;
    const uint32_t H = run;
    if (H == 0) continue;
    if (H > (uint32_t)kWH) {
      hand_over(wdx);
      continue;
    }
    const int m = a.mtab[s];
    for (int x = lane; x < kWSlots / 2; x += 32) S.slots[x] = 0;
    if (lane == 0) S.nhit = 0;
    __syncwarp();
    // Hits in chunks of 32 consecutive ones.  The list holding hit e is the
    // last x with pre[x] <= e: for the chunk at base it is cur (the list
    // holding the previous chunk's last hit) plus the number of lists after
    // cur that start at or before e, found by a 5-step search over the next
    // 32 lists' starts (pre is nondecreasing) instead of a search per hit.
    auto each_hit = [&](auto f) {
      int cur = 0;
      for (int base = 0; base < (int)H; base += 32) {
        const int e = base + lane;
        int lo = cur;
        for (int from = cur + 1;; from += 32) {
          const int x = from + lane;
          const int d = x < s ? (int)S.pre[x] - base : INT_MAX;
          int n = 0;  // lists among from .. from + 30 starting at or before e
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, d, n + step - 1);
            if (v <= lane) n += step;
          }
          const int d31 = __shfl_sync(0xffffffffu, d, 31);
          if (d31 <= lane) n = 32;
          if (n > 0) lo = from + n - 1;
          if (d31 > 31) break;  // no list past these starts inside the chunk
        }
        cur = __shfl_sync(0xffffffffu, lo, 31);
        if (e >= (int)H) continue;
        const uint64_t r = __ldg(a.tsorted + S.pst[lo] + (uint32_t)(e - (int)S.pre[lo]));
        const uint32_t t = rec_pos(r), st = rec_strand(r);
        if (a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span) continue;
        const uint32_t qm = S.dm[lo];
        if ((qm >> st) & 1u) f(t, (uint32_t)lo, 0u);
        if ((qm >> (st ^ 1u)) & 1u) f(t, (uint32_t)lo, 1u);
      }
    };
    each_hit([&](uint32_t t, uint32_t, uint32_t o) {
      const uint32_t sl = wslot_of(t, o);
      atomicAdd(&S.slots[sl >> 1], 1u << ((sl & 1) * 16));
    });
    __syncwarp();
    // A hit is collected only when its bin's counter and a neighbouring
    // bin's (same strand) sum to m or more.  Word x of the table holds bin x
    // (both strands), so when no two cyclically adjacent words reach m on
    // either strand, nothing would be collected: the window ends here.
    {
      bool pass = false;
      for (int x = lane; x < kWSlots / 2; x += 32) {
        const uint32_t c = S.slots[x], d = S.slots[(x + 1) & (kWSlots / 2 - 1)];
        pass |= (c & 0xFFFFu) + (d & 0xFFFFu) >= (uint32_t)m || (c >> 16) + (d >> 16) >= (uint32_t)m;
      }
      if (!__any_sync(0xffffffffu, pass)) {
        if (io.stats && lane == 0) atomicAdd(a.stats + 0, (unsigned long long)H);
        continue;
      }
    }
    each_hit([&](uint32_t t, uint32_t hid, uint32_t o) {
      const uint32_t b = t >> kBinShift;
      const uint32_t c0 = slot_count(S.slots, wslot_of(t, o));
      const uint32_t cn = slot_count(S.slots, (((b + 1) << 1) | o) & (kWSlots - 1));
      bool need = c0 + cn >= (uint32_t)m;
      if (!need && b > 0) {
        const uint32_t cp = slot_count(S.slots, (((b - 1) << 1) | o) & (kWSlots - 1));
        need = cp + c0 >= (uint32_t)m;
      }
      if (need) {
        const int at = atomicAdd(&S.nhit, 1);
        if (at < kWL)
          S.hits[at] = ((unsigned long long)o << 63) | ((unsigned long long)t << 20) | hid;
      }
    });
    __syncwarp();
    const int L = S.nhit;
    if (L > kWL) {
      hand_over(wdx);
      continue;
    }
    if (L < m) {
      if (io.stats && lane == 0) {
        atomicAdd(a.stats + 0, (unsigned long long)H);
        atomicAdd(a.stats + 1, (unsigned long long)L);
      }
      continue;
    }
    const int nh = next_pow2(L < 2 ? 2 : L);
    for (int x = L + lane; x < nh; x += 32) S.hits[x] = ~0ull;
    __syncwarp();
    warp_sort(S.hits, nh);
    int split;
    {
      int lo2 = 0, hi2 = L;  // first hit with o = 1
      while (lo2 < hi2) {
        const int mid = (lo2 + hi2) >> 1;
        if ((S.hits[mid] >> 63) == 0) lo2 = mid + 1; else hi2 = mid;
      }
      split = lo2;
    }
    int ng = 0, ng0 = 0;
    for (int o = 0; o < 2; ++o) {
      const unsigned long long* base = S.hits + (o ? split : 0);
      const int64_t cnt = o ? L - split : split;
      find_groups(
          [&](int64_t x) {
            const unsigned long long h = base[x];
            return make_uint2((uint32_t)(h >> 20), (uint32_t)(h & 0xFFFFFu));
          },
          cnt, m, a.span, [&](int64_t lo, int64_t hi) {
            if (lane == 0 && ng < kWG) {
              S.glo[ng] = (uint32_t)(lo < 0 ? 0 : lo);
              S.ghi[ng] = (uint32_t)hi;
            }
            ++ng;
          });
      if (o == 0) ng0 = ng;
    }
    __syncwarp();
    if (ng > kWG) {
      hand_over(wdx);
      continue;
    }
    if (io.stats && lane == 0) {
      atomicAdd(a.stats + 0, (unsigned long long)H);
      atomicAdd(a.stats + 1, (unsigned long long)L);
    }
    if (lane == 0) {
      WinInfo w;
      w.i = i;
      w.qseq = a.win_seq[wdx];
      w.s = s;
      w.m = m;
      for (int g = 0; g < ng; ++g) {
        w.o = g < ng0 ? 0 : 1;
        const unsigned long long* base = S.hits + (w.o ? split : 0);
        const int64_t cnt = w.o ? L - split : split;
        sweep_group(a, w,
                    [&](int64_t x) {
                      const unsigned long long h = base[x];
                      return make_uint2((uint32_t)(h >> 20), (uint32_t)(h & 0xFFFFFu));
                    },
                    cnt, S.cnt, (int64_t)S.glo[g], (int64_t)S.ghi[g]);
      }
    }
    __syncwarp();
  }
}

int launch_warp_tier(sedef_ctx* ctx, const FArgs& a, const TierIO& io, int64_t max_windows,
                     const char* name) {
  const size_t sm = sizeof(WarpSmem) * kWWarps;
  SEDEF_TRY(ensure_smem_attr((const void*)k_filter_warp, sm));
  int per_sm = 0;
  SEDEF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_warp, 32 * kWWarps, sm));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx_sm_count(ctx) * per_sm;
  const int64_t need = (max_windows + kWWarps - 1) / kWWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  SEDEF_KERNEL(ctx, name, k_filter_warp<<<(int)grid, 32 * kWWarps, sm, ctx_stream(ctx)>>>(a, io));
  return SEDEF_OK;
}

// ------------------------------------------------------------- slow path --

constexpr int kSThreads = 256;

struct SlowSmem {
  uint32_t qkey[kMaxWindowRecs];
  uint32_t dh[kMaxWindowRecs];
  uint32_t pst[kMaxWindowRecs];
  uint32_t plen[kMaxWindowRecs];
  uint8_t dm[kMaxWindowRecs];
  uint16_t cnt[kMaxWindowRecs];
  int tmp[33];
  unsigned long long acc;
};

__device__ int slow_wq(const FArgs& a, SlowSmem& S, int64_t wdx) {
  const uint32_t qa = a.win_qa[wdx], qb = a.win_qb[wdx];
  const int c = (int)(qb - qa);
  for (int x = threadIdx.x; x < c; x += blockDim.x) {
    const uint64_t r = a.qrec[qa + x];
    S.qkey[x] = (rec_hash(r) << 1) | rec_strand(r);
  }
  __syncthreads();
  QBuild q;
  q.qkey = S.qkey;
  q.dh = S.dh;
  q.dm = S.dm;
  q.pst = S.pst;
  q.plen = S.plen;
  q.tmp = S.tmp;
  int64_t seq_lo = 0, seq_hi = 0;
  if (a.self_mode == 2) {
    const int sq = a.win_seq[wdx];
    seq_lo = a.tseq[sq];
    seq_hi = a.tseq[sq + 1];
  }
  return build_wq(a, q, c, seq_lo, seq_hi);
}

// Hits of overflow window v: visits (t, hid, o) for every compatible posting.
template <typename F>
__device__ void slow_hits(const FArgs& a, const SlowSmem& S, int s, int64_t i, F f) {
  for (int l = 0; l < s; ++l) {
    const uint32_t st0 = S.pst[l], len = S.plen[l];
    const uint32_t qm = S.dm[l];
    for (uint32_t x = threadIdx.x; x < len; x += blockDim.x) {
      const uint64_t r = a.tsorted[st0 + x];
      const uint32_t t = rec_pos(r), st = rec_strand(r);
      if (a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span) continue;
      if ((qm >> st) & 1u) f(t, (uint32_t)l, 0u);
      if ((qm >> (st ^ 1u)) & 1u) f(t, (uint32_t)l, 1u);
    }
  }
}

template <typename C>
__global__ void __launch_bounds__(kSThreads) k_slow_count(FArgs a, int64_t nov, C* counts,
                                                          int32_t* s_out, const uint32_t* dnov,
                                                          unsigned long long* total) {
  __shared__ SlowSmem S;
  nov = live_n(nov, dnov);
  for (int64_t v = blockIdx.x; v < nov; v += gridDim.x) {
    __syncthreads();
    const int64_t wdx = a.ov_list[v];
    const int s = slow_wq(a, S, wdx);
    if (threadIdx.x == 0) S.acc = 0;
    __syncthreads();
    unsigned long long mine = 0;
    slow_hits(a, S, s, a.win_i[wdx], [&](uint32_t, uint32_t, uint32_t) { ++mine; });
    atomicAdd(&S.acc, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
      counts[v] = (C)S.acc;
      s_out[v] = s;
      if (total) atomicAdd(total, S.acc);
    }
  }
}

// Writes keys (local window << 33 | o << 32 | t) and hash ids for windows
// [v0, v1) of the overflow list at offsets base[v] - base[v0].
// Windows whose hits would end past `hcap` are skipped (a planned pass
// reports them as an overflow).
__global__ void __launch_bounds__(kSThreads) k_slow_emit(FArgs a, int64_t v0, int64_t v1,
                                                         const unsigned long long* base,
                                                         uint64_t* keys, uint32_t* vals,
                                                         const uint32_t* dnov, int64_t hcap) {
  __shared__ SlowSmem S;
  __shared__ unsigned long long cursor;
  v1 = live_n(v1, dnov);
  for (int64_t v = v0 + blockIdx.x; v < v1; v += gridDim.x) {
    if (base[v + 1] < base[v] || (int64_t)(base[v + 1] - base[v0]) > hcap) continue;
    __syncthreads();
    const int64_t wdx = a.ov_list[v];
    const int s = slow_wq(a, S, wdx);
    if (threadIdx.x == 0) cursor = base[v] - base[v0];
    __syncthreads();
    const uint64_t lw = (uint64_t)(v - v0);
    slow_hits(a, S, s, a.win_i[wdx], [&](uint32_t t, uint32_t hid, uint32_t o) {
      const unsigned long long at = atomicAdd(&cursor, 1ull);
      keys[at] = (lw << 33) | ((uint64_t)o << 32) | t;
      vals[at] = hid;
    });
  }
}

// Dense groups of the overflow windows [v0, v1): one warp per window and
// strand writes one task (window, strand, Jlo, Jhi) per group.
struct SlowTask {
  uint32_t v;   // overflow-list index
  uint32_t o;
  int64_t jlo, jhi;
};

__device__ __forceinline__ void slow_segment(const uint64_t* keys, int64_t lo, int64_t hi,
                                             int64_t* split) {
  int64_t l = lo, h = hi;  // first key with o = 1
  while (l < h) {
    const int64_t mid = (l + h) >> 1;
    if (((keys[mid] >> 32) & 1u) == 0) l = mid + 1; else h = mid;
  }
  *split = l;
}

__global__ void k_slow_groups(FArgs a, int64_t v0, int64_t v1, const unsigned long long* base,
                              const int32_t* s_of, const uint64_t* keys, SlowTask* tasks,
                              unsigned long long* ntask, int64_t task_cap, const uint32_t* dnov,
                              int64_t hcap) {
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  v1 = live_n(v1, dnov);
  for (int64_t v = v0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < v1;
       v += nw) {
    const int s = s_of[v];
    if (s == 0 || base[v + 1] < base[v] || (int64_t)(base[v + 1] - base[v0]) > hcap) continue;
    const int m = a.mtab[s];
    const int64_t lo = (int64_t)(base[v] - base[v0]), hi = (int64_t)(base[v + 1] - base[v0]);
    int64_t split;
    slow_segment(keys, lo, hi, &split);
    for (int o = 0; o < 2; ++o) {
      const int64_t b = o ? split : lo, e = o ? hi : split;
      find_groups([&](int64_t x) { return make_uint2((uint32_t)keys[b + x], 0u); }, e - b, m,
                  a.span, [&](int64_t jlo, int64_t jhi) {
                    if (lane_id() == 0) {
                      const unsigned long long at = atomicAdd(ntask, 1ull);
                      if ((int64_t)at < task_cap) {
                        SlowTask t;
                        t.v = (uint32_t)v;
                        t.o = (uint32_t)o;
                        t.jlo = jlo < 0 ? 0 : jlo;
                        t.jhi = jhi;
                        tasks[at] = t;
                      }
                    }
                  });
    }
  }
}

// One warp per task; lane 0 sweeps the group with the warp's counters.
constexpr int kTaskWarps = 8;

__global__ void __launch_bounds__(32 * kTaskWarps) k_slow_tasks(
    FArgs a, int64_t v0, const unsigned long long* base, const int32_t* s_of,
    const uint64_t* keys, const uint32_t* vals, const SlowTask* tasks,
    const unsigned long long* ntask, int64_t task_cap) {
  __shared__ uint16_t cnt[kTaskWarps][kMaxWindowRecs];
  const int warp = threadIdx.x >> 5;
  for (int x = threadIdx.x & 31; x < kMaxWindowRecs; x += 32) cnt[warp][x] = 0;
  __syncwarp();
  if ((threadIdx.x & 31) != 0) return;
  const int64_t nt = min((int64_t)*ntask, task_cap);
  for (int64_t t = (int64_t)blockIdx.x * kTaskWarps + warp; t < nt;
       t += (int64_t)gridDim.x * kTaskWarps) {
    const SlowTask task = tasks[t];
    const int64_t v = task.v;
    const int64_t wdx = a.ov_list[v];
    const int s = s_of[v];
    WinInfo w;
    w.i = a.win_i[wdx];
    w.qseq = a.win_seq[wdx];
    w.s = s;
    w.m = a.mtab[s];
    w.o = (int)task.o;
    const int64_t lo = (int64_t)(base[v] - base[v0]), hi = (int64_t)(base[v + 1] - base[v0]);
    int64_t split;
    slow_segment(keys, lo, hi, &split);
    const int64_t b = task.o ? split : lo, e = task.o ? hi : split;
    sweep_group(a, w, [&](int64_t x) { return make_uint2((uint32_t)keys[b + x], vals[b + x]); },
                e - b, cnt[warp], task.jlo, task.jhi);
  }
}

// ---------------------------------------------------------- window table --

__global__ void k_windows(const uint64_t* __restrict__ qrec, int64_t nq,
                          const int64_t* __restrict__ qseq, int nqseq,
                          const int64_t* __restrict__ wbase, int64_t nwin, int step, int span,
                          uint32_t* wi, uint32_t* wqa, uint32_t* wqb, int32_t* wseq,
                          const uint32_t* dnq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwin) return;
  nq = live_n(nq, dnq);
  int lo = 0, hi = nqseq;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (wbase[mid] <= w) lo = mid; else hi = mid;
  }
  const int64_t i = qseq[lo] + (w - wbase[lo]) * step;
  auto pos = [](uint64_t r) { return (uint64_t)((r >> 1) & 0xFFFFFFFFull); };
  const int64_t a = lower_bound_by(qrec, 0, nq, (uint64_t)i, pos);
  const int64_t b = lower_bound_by(qrec, a, nq, (uint64_t)(i + span + 1), pos);
  wi[w] = (uint32_t)i;
  wqa[w] = (uint32_t)a;
  wqb[w] = (uint32_t)b;
  wseq[w] = lo;
}

// Sort keys of the runs: (window index, o, j_a).  part 0: the whole key
// when it fits 64 bits; part 1: j_a alone and part 2: (window, o), for a
// two-pass stable sort otherwise.
__global__ void k_run_keys(const sedef_run_t* runs, int64_t n, const int64_t* qseq, int nqseq,
                           const int64_t* wbase, int step, int part, uint64_t* keys,
                           const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= live_n(n, dn)) return;
  const sedef_run_t r = runs[x];
  const int sq = seq_of(qseq, nqseq, r.i);
  const uint64_t widx = (uint64_t)(wbase[sq] + ((int64_t)r.i - qseq[sq]) / step);
  if (part == 0) keys[x] = (widx << 33) | ((uint64_t)r.o << 32) | r.j_a;
  else if (part == 1) keys[x] = r.j_a;
  else keys[x] = (widx << 1) | r.o;
}

__global__ void k_permute_u64(const uint64_t* in, const uint32_t* perm, int64_t n, uint64_t* out,
                              const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < live_n(n, dn)) out[x] = in[perm[x]];
}

__global__ void k_compose_perm(const uint32_t* first, const uint32_t* second, int64_t n,
                               uint32_t* out, const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < live_n(n, dn)) out[x] = first[second[x]];
}

__global__ void k_widen_u32(const uint32_t* in, int64_t n, unsigned long long* out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) out[x] = in[x];
}

__global__ void k_gather_runs(const sedef_run_t* in, const uint32_t* perm, int64_t n, sedef_run_t* out,
                              const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < live_n(n, dn)) out[x] = in[perm[x]];
}

// ----------------------------------------------------------------- refine --
//
// Two instantiations of one kernel: a lean one (at most 256 query records
// and 512 span records per run, one piece, ~12 KB of shared memory per warp
// so that 16 warps per SM hide the latency of the sequential roll) and a
// large one (any run, in pieces of at most 1024 span records) for the runs
// the lean one hands over.
//
// The estimate at j never exceeds the number of W_Q hashes shared with the
// window (the filter's shared_o(j)), so it is evaluated only where that
// count exceeds the best estimate so far, and the run is finished as soon
// as the best estimate reaches the run's max_shared.

constexpr int kRWarps = 8;     // lean kernel: warps per CTA
constexpr int kRWarpsBig = 4;  // large kernel

template <int QC, int RC>
struct RefineWarpT {
  static constexpr int DC = QC + RC;  // domain: W_Q u span hashes
  static_assert((DC & (DC - 1)) == 0, "the sort pads the domain to a power of two");
  uint32_t dom[DC];      // sorted distinct hashes
  uint16_t cntT[DC];     // records of this hash in the target window
  uint16_t cntS[DC];     // shared-compatible records of this hash in the window
  uint8_t qm[DC];        // strand mask for W_Q members (0 = not in W_Q)
  uint32_t pb[DC / 32];  // present: in W_Q or cntT > 0
  uint32_t sb[DC / 32];  // shared: cntS > 0
  uint32_t tpos[RC];     // span record positions (sorted)
  uint16_t tdx[RC];      // domain index of each span record
  uint8_t tsh[RC];       // record is shared-compatible
  uint32_t wq_h[QC];     // W_Q hashes (sorted)
  uint8_t wq_m[QC];      // W_Q strand masks
};

__device__ __forceinline__ void warp_sort_u32(uint32_t* v, int n) {  // n power of two
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane_id(); t < (n >> 1); t += 32) {
        const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const uint32_t x = v[lo], y = v[hi];
        if ((x > y) == asc) {
          v[lo] = y;
          v[hi] = x;
        }
      }
      __syncwarp();
    }
}

__device__ __forceinline__ int dom_find(const uint32_t* dom, int D, uint32_t h) {
  int lo = 0, hi = D;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (dom[mid] < h) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// theta = domain index of the s-th present bit, est = shared bits at or
// below it (warp-wide; same word layout as estimate()).
__device__ __forceinline__ void theta_est(const uint32_t* pb, const uint32_t* sb, int nwords,
                                          int s, int* theta, int* est) {
  const int lane = lane_id();
  const uint32_t p0 = (2 * lane < nwords) ? pb[2 * lane] : 0u;
  const uint32_t p1 = (2 * lane + 1 < nwords) ? pb[2 * lane + 1] : 0u;
  const uint32_t s0 = (2 * lane < nwords) ? sb[2 * lane] : 0u;
  const uint32_t s1 = (2 * lane + 1 < nwords) ? sb[2 * lane + 1] : 0u;
  const int pc = __popc(p0) + __popc(p1);
  const int inc = warp_inclusive_sum(pc);
  const int before = inc - pc;
  const unsigned owner = __ballot_sync(0xffffffffu, before < s && inc >= s);
  const int ol = __ffs(owner) - 1;
  int cnt = (inc < s) ? (__popc(s0) + __popc(s1)) : 0;  // lanes wholly below theta
  int th = 0;
  if (lane == ol) {
    int need = s - before;
    const uint32_t wp[2] = {p0, p1}, ws[2] = {s0, s1};
    cnt = 0;
    for (int x = 0; x < 2; ++x) {
      const int c = __popc(wp[x]);
      if (c < need) {
        cnt += __popc(ws[x]);
        need -= c;
        continue;
      }
      uint32_t v = wp[x];
      for (int y = 1; y < need; ++y) v &= v - 1u;
      const int b = __ffs(v) - 1;
      const uint32_t below = (b >= 31) ? 0xFFFFFFFFu : ((2u << b) - 1u);
      cnt += __popc(ws[x] & below);
      th = (2 * lane + x) * 32 + b;
      break;
    }
  }
  *est = warp_sum(cnt);
  *theta = __shfl_sync(0xffffffffu, th, ol);
}

struct RefineArgs {
  sedef_run_t* runs;
  int64_t nruns;
  const uint64_t* qrec;
  int64_t nq;
  const uint64_t* trec;
  int64_t nt;
  const uint32_t* dnruns = nullptr;  // live counts of a planned pass
  const uint32_t* dnt = nullptr;
  const uint32_t* toff;
  const int32_t* mtab;
  int span, max_occ, self_mode;
  uint32_t* big;        // runs handed to the large kernel
  unsigned int* nbig;
  const uint4* ranges;  // per run: query records [x, y), span records [z, w)
  unsigned long long* next;  // chunk counters of the two kernels
};

template <int QC, int RC, bool kLean>
__global__ void __launch_bounds__(32 * (kLean ? kRWarps : kRWarpsBig)) k_refine(RefineArgs a) {
  a.nruns = live_n(a.nruns, a.dnruns);
  a.nt = live_n(a.nt, a.dnt);
  using RW = RefineWarpT<QC, RC>;
  constexpr int DC = RW::DC;
  constexpr int NW = kLean ? kRWarps : kRWarpsBig;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  RW& R = reinterpret_cast<RW*>(smem_raw)[warp];
  auto pos_of = [](uint64_t r) { return (uint64_t)((r >> 1) & 0xFFFFFFFFull); };
  const int64_t count = kLean ? a.nruns : (int64_t)*a.nbig;
  // contiguous chunks of runs per warp (runs of one window are adjacent, so
  // W_Q is built once per window and chunk), handed out dynamically
  constexpr int kChunk = 16;
  int64_t prev_qa = -1, prev_qb = -1;
  int s = 0;
  while (true) {
    int64_t c0 = 0;
    if (lane == 0) c0 = (int64_t)atomicAdd(kLean ? a.next : a.next + 1, (unsigned long long)kChunk);
    c0 = __shfl_sync(0xffffffffu, c0, 0);
    if (c0 >= count) break;
    const int64_t c1 = min(count, c0 + kChunk);
  for (int64_t t = c0; t < c1; ++t) {
    const int64_t ri = kLean ? t : (int64_t)a.big[t];
    const sedef_run_t run = a.runs[ri];
    const int64_t i = run.i, ja = run.j_a, jb = run.j_b;
    const int o = run.o;
    const uint4 rg = a.ranges[ri];  // query records [qa, qb), span records [rlo, rend)
    const int64_t qa = rg.x, qb = rg.y;
    int64_t rlo = rg.z;
    const int64_t rend = rg.w;
    const int c = (int)(qb - qa);
    if (kLean) {
      if (c > QC || rend - rlo > RC) {
        if (lane == 0) a.big[atomicAdd(a.nbig, 1u)] = (uint32_t)ri;
        continue;
      }
    }
    if (qa != prev_qa || qb != prev_qb) {
    prev_qa = qa;
    prev_qb = qb;
    // ---- W_Q: sorted hashes with strand masks (capped hashes dropped)
    const int npq = next_pow2(c < 2 ? 2 : c);
    for (int x = lane; x < npq; x += 32) {
      uint32_t key = kNone;
      if (x < c) {
        const uint64_t r = a.qrec[qa + x];
        key = (rec_hash(r) << 1) | rec_strand(r);
      }
      R.dom[x] = key;  // the domain array doubles as the sort buffer
    }
    __syncwarp();
    warp_sort_u32(R.dom, npq);
    s = 0;
    for (int base = 0; base < c; base += 32) {
      const int x = base + lane;
      uint32_t h = 0, mask = 0;
      bool first = false;
      if (x < c) {
        h = R.dom[x] >> 1;
        first = (x == 0) || ((R.dom[x - 1] >> 1) != h);
        if (first) {
          for (int y = x; y < c && (R.dom[y] >> 1) == h; ++y) mask |= 1u << (R.dom[y] & 1u);
          if (a.max_occ > 0 && (int)(a.toff[h + 1] - a.toff[h]) > a.max_occ) first = false;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, first);
      if (first) {
        const int d = s + __popc(bal & lanemask_lt());
        R.wq_h[d] = h;
        R.wq_m[d] = (uint8_t)mask;
      }
      s += __popc(bal);
    }
    __syncwarp();
    }
    const int mx = run.max_shared;
    int best = -1;
    int64_t jstar = ja;
    int64_t plo = ja;
    bool finished = false;
    while (plo <= jb && !finished) {
      // ---- the piece [plo, phi]: span records [rlo, rhi), at most RC
      int64_t phi = jb, rhi = 0;
      if (lane == 0) {
        const int64_t rcap_end = rlo + RC < a.nt ? rlo + RC : a.nt;
        rhi = lower_bound_by(a.trec, rlo, a.nt, (uint64_t)(jb + a.span + 1), pos_of);
        if (rhi > rcap_end) {
          const int64_t lim = (int64_t)pos_of(a.trec[rcap_end]);  // first record that does not fit
          phi = lim - a.span - 1;
          rhi = rcap_end;
        }
      }
      phi = __shfl_sync(0xffffffffu, phi, 0);
      rhi = __shfl_sync(0xffffffffu, rhi, 0);
      const int nr = (int)(rhi - rlo);
      // ---- relevant span records.  Only W_Q hashes with a compatible,
      // non-self occurrence in the span (the candidates C) can ever count,
      // and a candidate's rank among W_Q u W_T depends only on the hashes
      // below it.  So the roll needs the candidates' compatible occurrences
      // and the non-W_Q records whose hash is below max(C); every other
      // record leaves the estimate unchanged.  W_Q itself stays in the
      // domain, so at least s hashes are always present.  cntT/cntS double
      // as a scratch array of the kept records' hashes until the domain is
      // built.
      uint32_t* tmp_h = reinterpret_cast<uint32_t*>(R.cntT);  // DC u32 (cntT then cntS)
      auto wq_find = [&](uint32_t h) {  // index in W_Q or -1
        int lo2 = 0, hi2 = s;
        while (lo2 < hi2) {
          const int mid = (lo2 + hi2) >> 1;
          if (R.wq_h[mid] < h) lo2 = mid + 1; else hi2 = mid;
        }
        return (lo2 < s && R.wq_h[lo2] == h) ? lo2 : -1;
      };
      uint32_t cmax = 0;
      bool have_c = false;
      for (int base = 0; base < nr; base += 32) {
        const int x = base + lane;
        bool cand = false;
        uint32_t h = 0;
        if (x < nr) {
          const uint64_t r = a.trec[rlo + x];
          h = rec_hash(r);
          const uint32_t t = rec_pos(r), st = rec_strand(r);
          const int q = wq_find(h);
          const bool self = a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span;
          cand = q >= 0 && !self && ((R.wq_m[q] >> (st ^ (uint32_t)o)) & 1u);
        }
        uint32_t hm = cand ? h : 0u;
        const bool any = __any_sync(0xffffffffu, cand);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, d));
        if (any) {
          cmax = have_c ? max(cmax, hm) : hm;
          have_c = true;
        }
      }
      int nrel = 0;
      for (int base = 0; base < nr && have_c; base += 32) {
        const int x = base + lane;
        bool keep = false;
        uint32_t h = 0, t = 0, st = 0;
        if (x < nr) {
          const uint64_t r = a.trec[rlo + x];
          h = rec_hash(r);
          t = rec_pos(r);
          st = rec_strand(r);
          const int q = wq_find(h);
          if (q >= 0) {
            const bool self = a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span;
            keep = !self && ((R.wq_m[q] >> (st ^ (uint32_t)o)) & 1u);
          } else {
            keep = h < cmax;
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int y = nrel + __popc(bal & lanemask_lt());
          R.tpos[y] = t;
          tmp_h[y] = h;
          R.tsh[y] = (uint8_t)st;  // strand for now
        }
        nrel += __popc(bal);
      }
      __syncwarp();
      // ---- domain: sorted distinct hashes of W_Q u kept records
      const int nd0 = s + nrel;
      const int npd = next_pow2(nd0 < 2 ? 2 : nd0);
      for (int x = lane; x < npd; x += 32) {
        uint32_t v = kNone;
        if (x < s) v = R.wq_h[x];
        else if (x < nd0) v = tmp_h[x - s];
        R.dom[x] = v;
      }
      __syncwarp();
      warp_sort_u32(R.dom, npd);
      int D = 0;
      for (int base = 0; base < nd0; base += 32) {
        const int x = base + lane;
        const uint32_t v = x < nd0 ? R.dom[x] : kNone;
        const bool first = x < nd0 && (x == 0 || R.dom[x - 1] != v);
        const unsigned bal = __ballot_sync(0xffffffffu, first);
        __syncwarp();
        if (first) R.dom[D + __popc(bal & lanemask_lt())] = v;
        __syncwarp();
        D += __popc(bal);
      }
      for (int x = lane; x < nrel; x += 32) R.tdx[x] = (uint16_t)dom_find(R.dom, D, tmp_h[x]);
      __syncwarp();
      const int nwords = (D + 31) >> 5;
      for (int x = lane; x < D; x += 32) {
        R.cntT[x] = 0;
        R.cntS[x] = 0;
        R.qm[x] = 0;
      }
      for (int x = lane; x < DC / 32; x += 32) {
        R.pb[x] = 0;
        R.sb[x] = 0;
      }
      __syncwarp();
      for (int x = lane; x < s; x += 32) {
        const int d = dom_find(R.dom, D, R.wq_h[x]);
        R.qm[d] = R.wq_m[x];
        atomicOr(&R.pb[d >> 5], 1u << (d & 31));
      }
      __syncwarp();
      for (int x = lane; x < nrel; x += 32) {
        const uint32_t t = R.tpos[x], st = R.tsh[x];
        const int d = R.tdx[x];
        const bool self = a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span;
        R.tsh[x] = (!self && ((R.qm[d] >> (st ^ (uint32_t)o)) & 1u)) ? 1 : 0;
      }
      __syncwarp();
      // ---- roll the target window over [plo, phi].  theta is the domain
      // index of the s-th present hash (the largest member of U) and est the
      // number of shared hashes at or below it.  After the first breakpoint
      // lane 0 keeps both exact through every enter and leave, one record at
      // a time: a hash joining below theta pushes theta down to its
      // predecessor, one leaving at or below theta pulls theta up to its
      // successor, and a W_Q hash at or below theta changes est when it
      // becomes or stops being shared.
      int e = 0, l = 0;
      int64_t j = plo;
      if (lane == 0) {
        while (e < nrel && (int64_t)R.tpos[e] <= j + a.span) {
          const int d = R.tdx[e];
          if (R.cntT[d]++ == 0) R.pb[d >> 5] |= 1u << (d & 31);
          if (R.tsh[e] && R.cntS[d]++ == 0) R.sb[d >> 5] |= 1u << (d & 31);
          ++e;
        }
      }
      __syncwarp();
      int theta = 0, est = 0;
      theta_est(R.pb, R.sb, nwords, s, &theta, &est);
      int fin = 0;
      if (lane == 0) {
        auto bit = [&](const uint32_t* bs, int d) { return (int)((bs[d >> 5] >> (d & 31)) & 1u); };
        auto pred = [&](int d) {  // largest present index below d
          int w = d >> 5;
          uint32_t bits = R.pb[w] & ((1u << (d & 31)) - 1u);
          while (bits == 0 && w > 0) bits = R.pb[--w];
          return bits ? w * 32 + 31 - __clz(bits) : 0;
        };
        auto succ = [&](int d) {  // smallest present index above d
          int w = d >> 5;
          uint32_t bits = ((d & 31) == 31) ? 0u : (R.pb[w] & ~((2u << (d & 31)) - 1u));
          while (bits == 0 && w + 1 < nwords) bits = R.pb[++w];
          return bits ? w * 32 + __ffs(bits) - 1 : d;
        };
        auto enter = [&](int x) {
          const int d = R.tdx[x];
          if (R.cntT[d]++ == 0 && R.qm[d] == 0) {
            R.pb[d >> 5] |= 1u << (d & 31);
            if (d < theta) {
              const int old = theta;
              theta = pred(theta);
              est -= bit(R.sb, old);
            }
          }
          if (R.tsh[x] && R.cntS[d]++ == 0) {
            R.sb[d >> 5] |= 1u << (d & 31);
            if (d <= theta) ++est;
          }
        };
        auto leave = [&](int x) {
          const int d = R.tdx[x];
          if (--R.cntT[d] == 0 && R.qm[d] == 0) {
            R.pb[d >> 5] &= ~(1u << (d & 31));
            if (d <= theta) {
              theta = succ(theta);
              est += bit(R.sb, theta);
            }
          }
          if (R.tsh[x] && --R.cntS[d] == 0) {
            R.sb[d >> 5] &= ~(1u << (d & 31));
            if (d <= theta) --est;
          }
        };
        while (true) {
          if (est > best) {
            best = est;
            jstar = j;
            if (best >= mx) {
              fin = 1;
              break;
            }
          }
          const int64_t ne = e < nrel ? (int64_t)R.tpos[e] - a.span : INT64_MAX;
          const int64_t nl = l < e ? (int64_t)R.tpos[l] + 1 : INT64_MAX;
          const int64_t nx = min(ne, nl);
          if (nx > phi) break;
          j = nx;
          while (l < e && (int64_t)R.tpos[l] + 1 <= j) leave(l++);
          while (e < nrel && (int64_t)R.tpos[e] - a.span <= j) enter(e++);
        }
      }
      jstar = __shfl_sync(0xffffffffu, jstar, 0);
      finished = __shfl_sync(0xffffffffu, fin, 0) != 0;
      best = __shfl_sync(0xffffffffu, best, 0);
      plo = phi + 1;
      if (plo <= jb && !finished) {
        if (lane == 0) rlo = lower_bound_by(a.trec, rlo, a.nt, (uint64_t)plo, pos_of);
        rlo = __shfl_sync(0xffffffffu, rlo, 0);
      }
      __syncwarp();
    }
    if (lane == 0) {
      sedef_run_t& out = a.runs[ri];
      out.est = (uint16_t)(best < 0 ? 0 : best);
      out.den = (uint16_t)s;
      out.j_star = (uint32_t)jstar;
      out.keep = (best >= a.mtab[s]) ? 1 : 0;
    }
    __syncwarp();
  }
  }
}

// ------------------------------------------------- batched lean refine ----
//
// A warp sets up runs one at a time (cooperatively) into slots of a per-warp
// arena, then every lane rolls its own run through its slot, so many rolls
// proceed side by side.  Setup per run: the span records are read once
// (hash, rank among W_Q, W_Q membership, candidate flag); the domain is W_Q
// (already sorted) merged by rank with the sorted distinct non-W_Q kept
// hashes, so a kept record's domain index is its rank among W_Q plus its
// rank among those hashes.  A slot holds one 32-bit event per kept record
// (offset of its position from j_a, domain index, W_Q flag) and one counter
// per domain hash (presence for non-W_Q hashes, sharedness for W_Q hashes).
// Transient setup data (the span records' hashes, sort buffers) lives at the
// top of the arena, slots grow from the bottom.  Runs beyond the lean limits
// (more than 256 query records, 512 span records or a span of 65,536 bases)
// go to the large kernel.

constexpr int kBWarps = 4;
constexpr int kBQC = 256, kBRC = 512;
constexpr int kArenaWords = 2816;  // 11 KB per warp

struct BatchWarp {
  uint32_t arena[kArenaWords];
  uint32_t wq_h[kBQC];
  uint8_t wq_m[kBQC];
  // span record: bit0 strand, bit1 in W_Q, bit2 candidate, bit3 kept,
  // bits 4.. its hash's rank among W_Q (lower bound)
  uint16_t rinfo[kBRC];
  uint32_t h_off[32];     // slot start (words)
  uint32_t h_run[32];     // run index
  uint16_t h_nrel[32], h_D[32], h_dmax[32], h_s[32];
};

struct Slot {
  uint32_t* ev;    // per kept record: position - j_a (bits 0-15), domain index (16-25), W_Q (31)
  uint16_t* cnt;   // per domain hash: occurrences in the window
  uint32_t* pb;    // present
  uint32_t* sb;    // shared
};

__device__ __forceinline__ int slot_words(int nrel, int dmax) {
  return nrel + (dmax + 1) / 2 + 2 * ((dmax + 31) / 32);
}

__device__ __forceinline__ Slot slot_at(uint32_t* base, int nrel, int dmax) {
  Slot sl;
  sl.ev = base;
  sl.cnt = reinterpret_cast<uint16_t*>(base + nrel);
  sl.pb = base + nrel + (dmax + 1) / 2;
  sl.sb = sl.pb + (dmax + 31) / 32;
  return sl;
}

// Rolls one run (single lane) over target starts j_a + [0, jend]: enters the
// first window's records, finds theta (s-th present hash) and est by
// scanning the bitsets, then keeps both exact through every enter/leave (as
// in the large kernel).  Offsets from j_a fit in 16 bits, so the roll runs
// in 32-bit arithmetic.
__device__ void roll_run(const Slot& sl, int nrel, int D, int s, int mx, int jend, int span,
                         int* best_out, int* jstar_out) {
  const int nwords = (D + 31) >> 5;
  auto pos = [&](int x) { return (int)(sl.ev[x] & 0xFFFFu); };
  int e = 0, l = 0, j = 0;
  while (e < nrel && pos(e) <= j + span) {
    const uint32_t v = sl.ev[e];
    const int d = (int)((v >> 16) & 0x3FFu);
    if (sl.cnt[d]++ == 0) {
      if (v >> 31) sl.sb[d >> 5] |= 1u << (d & 31);
      else sl.pb[d >> 5] |= 1u << (d & 31);
    }
    ++e;
  }
  int theta = 0, est = 0;
  {
    int acc = 0;
    for (int w = 0; w < nwords; ++w) {
      const int c = __popc(sl.pb[w]);
      if (acc + c >= s) {
        uint32_t v = sl.pb[w];
        for (int y = 1; y < s - acc; ++y) v &= v - 1u;
        const int b = __ffs(v) - 1;
        theta = w * 32 + b;
        const uint32_t below = (b >= 31) ? 0xFFFFFFFFu : ((2u << b) - 1u);
        est += __popc(sl.sb[w] & below);
        break;
      }
      acc += c;
      est += __popc(sl.sb[w]);
    }
  }
  auto bit = [&](const uint32_t* bs, int d) { return (int)((bs[d >> 5] >> (d & 31)) & 1u); };
  auto pred = [&](int d) {
    int w = d >> 5;
    uint32_t bits = sl.pb[w] & ((1u << (d & 31)) - 1u);
    while (bits == 0 && w > 0) bits = sl.pb[--w];
    return bits ? w * 32 + 31 - __clz(bits) : 0;
  };
  auto succ = [&](int d) {
    int w = d >> 5;
    uint32_t bits = ((d & 31) == 31) ? 0u : (sl.pb[w] & ~((2u << (d & 31)) - 1u));
    while (bits == 0 && w + 1 < nwords) bits = sl.pb[++w];
    return bits ? w * 32 + __ffs(bits) - 1 : d;
  };
  int best = -1, jstar = 0;
  while (true) {
    if (est > best) {
      best = est;
      jstar = j;
      if (best >= mx) break;
    }
    const int ne = e < nrel ? pos(e) - span : INT_MAX;
    const int nl = l < e ? pos(l) + 1 : INT_MAX;
    const int nx = min(ne, nl);
    if (nx > jend) break;
    j = nx;
    while (l < e && pos(l) + 1 <= j) {
      const uint32_t v = sl.ev[l];
      const int d = (int)((v >> 16) & 0x3FFu);
      if (--sl.cnt[d] == 0) {
        if (v >> 31) {
          sl.sb[d >> 5] &= ~(1u << (d & 31));
          if (d <= theta) --est;
        } else {
          sl.pb[d >> 5] &= ~(1u << (d & 31));
          if (d <= theta) {
            theta = succ(theta);
            est += bit(sl.sb, theta);
          }
        }
      }
      ++l;
    }
    while (e < nrel && pos(e) - span <= j) {
      const uint32_t v = sl.ev[e];
      const int d = (int)((v >> 16) & 0x3FFu);
      if (sl.cnt[d]++ == 0) {
        if (v >> 31) {
          sl.sb[d >> 5] |= 1u << (d & 31);
          if (d <= theta) ++est;
        } else {
          sl.pb[d >> 5] |= 1u << (d & 31);
          if (d < theta) {
            const int old = theta;
            theta = pred(theta);
            est -= bit(sl.sb, old);
          }
        }
      }
      ++e;
    }
  }
  *best_out = best;
  *jstar_out = jstar;
}

__device__ __forceinline__ int lb_u32(const uint32_t* v, int n, uint32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(32 * kBWarps) k_refine_batch(RefineArgs a) {
  a.nruns = live_n(a.nruns, a.dnruns);
  a.nt = live_n(a.nt, a.dnt);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  BatchWarp& B = reinterpret_cast<BatchWarp*>(smem_raw)[warp];
  constexpr int kChunk = 32;
  int64_t prev_qa = -1, prev_qb = -1;
  int s = 0;
  int nslots = 0, used = 0;

  auto flush = [&]() {
    __syncwarp();
    if (lane < nslots) {
      const int64_t ri = B.h_run[lane];
      const sedef_run_t run = a.runs[ri];
      const int nrel = B.h_nrel[lane], D = B.h_D[lane], sq = B.h_s[lane];
      const Slot sl = slot_at(B.arena + B.h_off[lane], nrel, B.h_dmax[lane]);
      int best, jstar;
      roll_run(sl, nrel, D, sq, run.max_shared, (int)(run.j_b - run.j_a), a.span, &best, &jstar);
      sedef_run_t& out = a.runs[ri];
      out.est = (uint16_t)(best < 0 ? 0 : best);
      out.den = (uint16_t)sq;
      out.j_star = run.j_a + (uint32_t)jstar;
      out.keep = (best >= a.mtab[sq]) ? 1 : 0;
    }
    __syncwarp();
    nslots = 0;
    used = 0;
  };

  while (true) {
    int64_t c0 = 0;
    if (lane == 0) c0 = (int64_t)atomicAdd(a.next, (unsigned long long)kChunk);
    c0 = __shfl_sync(0xffffffffu, c0, 0);
    if (c0 >= a.nruns) break;
    const int64_t c1 = min(a.nruns, c0 + kChunk);
    for (int64_t ri = c0; ri < c1; ++ri) {
      const sedef_run_t run = a.runs[ri];
      const int64_t i = run.i;
      const int o = run.o;
      const uint4 rg = a.ranges[ri];
      const int64_t qa = rg.x, qb = rg.y, rlo = rg.z, rend = rg.w;
      const int c = (int)(qb - qa);
      const int nr = (int)(rend - rlo);
      if (c > kBQC || nr > kBRC || (int64_t)run.j_b + a.span - run.j_a >= 65536) {
        if (lane == 0) a.big[atomicAdd(a.nbig, 1u)] = (uint32_t)ri;
        continue;
      }
      // ---- W_Q (kept from the previous run of the same window); sorted in
      // a transient buffer at the top of the arena
      if (qa != prev_qa || qb != prev_qb) {
        prev_qa = qa;
        prev_qb = qb;
        const int npq = next_pow2(c < 2 ? 2 : c);
        if (used + npq > kArenaWords) flush();
        uint32_t* buf = B.arena + kArenaWords - npq;
        for (int x = lane; x < npq; x += 32) {
          uint32_t key = kNone;
          if (x < c) {
            const uint64_t r = a.qrec[qa + x];
            key = (rec_hash(r) << 1) | rec_strand(r);
          }
          buf[x] = key;
        }
        __syncwarp();
        warp_sort_u32(buf, npq);
        s = 0;
        for (int base = 0; base < c; base += 32) {
          const int x = base + lane;
          uint32_t h = 0, mask = 0;
          bool first = false;
          if (x < c) {
            h = buf[x] >> 1;
            first = (x == 0) || ((buf[x - 1] >> 1) != h);
            if (first) {
              for (int y = x; y < c && (buf[y] >> 1) == h; ++y) mask |= 1u << (buf[y] & 1u);
              if (a.max_occ > 0 && (int)(a.toff[h + 1] - a.toff[h]) > a.max_occ) first = false;
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, first);
          if (first) {
            const int d = s + __popc(bal & lanemask_lt());
            B.wq_h[d] = h;
            B.wq_m[d] = (uint8_t)mask;
          }
          s += __popc(bal);
        }
        __syncwarp();
      }
      // ---- space: the span records' hashes and the largest sort buffer at
      // the top of the arena (the slot's exact size is checked below)
      const int npr = next_pow2(nr < 2 ? 2 : nr);
      if (nslots == 32 || used + nr + npr > kArenaWords) flush();
      uint32_t* th = B.arena + kArenaWords - nr;  // transient: hashes of the span records
      // ---- pass over the span records: hash, rank among W_Q, flags, max(C)
      uint32_t cmax = 0;
      bool have_c = false;
      for (int base = 0; base < nr; base += 32) {
        const int x = base + lane;
        bool cand = false;
        uint32_t h = 0;
        if (x < nr) {
          const uint64_t r = a.trec[rlo + x];
          h = rec_hash(r);
          const uint32_t t = rec_pos(r), st = rec_strand(r);
          const int q = lb_u32(B.wq_h, s, h);
          const bool member = q < s && B.wq_h[q] == h;
          const bool self = a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span;
          cand = member && !self && ((B.wq_m[q] >> (st ^ (uint32_t)o)) & 1u);
          th[x] = h;
          B.rinfo[x] = (uint16_t)(st | (member ? 2u : 0u) | (cand ? 4u : 0u) | ((uint32_t)q << 4));
        }
        uint32_t hm = cand ? h : 0u;
        const bool any = __any_sync(0xffffffffu, cand);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, d));
        if (any) {
          cmax = have_c ? max(cmax, hm) : hm;
          have_c = true;
        }
      }
      __syncwarp();
      // ---- kept records: candidates' occurrences and non-W_Q hashes below max(C)
      int nrel = 0, n1 = 0;
      for (int base = 0; base < nr && have_c; base += 32) {
        const int x = base + lane;
        bool keep = false, nonq = false;
        if (x < nr) {
          const uint32_t f = B.rinfo[x];
          nonq = !(f & 2u) && th[x] < cmax;
          keep = (f & 4u) || nonq;
          if (keep) B.rinfo[x] = (uint16_t)(f | 8u);
        }
        nrel += __popc(__ballot_sync(0xffffffffu, keep));
        n1 += __popc(__ballot_sync(0xffffffffu, nonq));
      }
      __syncwarp();
      const int dmax = s + n1;
      const int np1 = next_pow2(n1 < 2 ? 2 : n1);
      uint32_t* u1 = th - np1;  // transient sort buffer of the non-W_Q kept hashes
      if (used + slot_words(nrel, dmax) > kArenaWords - nr - np1) flush();
      const Slot sl = slot_at(B.arena + used, nrel, dmax);
      {
        int y = 0, z = 0;
        for (int base = 0; base < nr && nrel > 0; base += 32) {
          const int x = base + lane;
          bool keep = false, nonq = false;
          uint32_t f = 0;
          if (x < nr) {
            f = B.rinfo[x];
            keep = (f & 8u) != 0;
            nonq = keep && !(f & 2u);
          }
          const unsigned bk = __ballot_sync(0xffffffffu, keep);
          const unsigned bn = __ballot_sync(0xffffffffu, nonq);
          if (keep) {
            const int yy = y + __popc(bk & lanemask_lt());
            sl.ev[yy] = (rec_pos(a.trec[rlo + x]) - run.j_a) | ((f & 2u) ? 0x80000000u : 0u);
          }
          if (nonq) u1[z + __popc(bn & lanemask_lt())] = th[x];
          y += __popc(bk);
          z += __popc(bn);
        }
        for (int x = n1 + lane; x < np1; x += 32) u1[x] = kNone;
      }
      __syncwarp();
      warp_sort_u32(u1, np1);
      int u = 0;  // distinct non-W_Q kept hashes, compacted in place
      for (int base = 0; base < n1; base += 32) {
        const int x = base + lane;
        const uint32_t v = x < n1 ? u1[x] : kNone;
        const bool first = x < n1 && (x == 0 || u1[x - 1] != v);
        const unsigned bal = __ballot_sync(0xffffffffu, first);
        __syncwarp();
        if (first) u1[u + __popc(bal & lanemask_lt())] = v;
        __syncwarp();
        u += __popc(bal);
      }
      const int D = s + u;
      // domain index of a kept record: its hash's rank among W_Q plus its
      // rank among the distinct non-W_Q kept hashes
      {
        int y = 0;
        for (int base = 0; base < nr && nrel > 0; base += 32) {
          const int x = base + lane;
          const uint32_t f = x < nr ? B.rinfo[x] : 0u;
          const bool keep = (f & 8u) != 0;
          const unsigned bk = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            const uint32_t d = (f >> 4) + (uint32_t)lb_u32(u1, u, th[x]);
            sl.ev[y + __popc(bk & lanemask_lt())] |= d << 16;
          }
          y += __popc(bk);
        }
      }
      for (int x = lane; x < dmax; x += 32) sl.cnt[x] = 0;
      for (int x = lane; x < (dmax + 31) / 32; x += 32) {
        sl.pb[x] = 0;
        sl.sb[x] = 0;
      }
      __syncwarp();
      for (int k = lane; k < s; k += 32) {
        const int d = k + lb_u32(u1, u, B.wq_h[k]);
        atomicOr(&sl.pb[d >> 5], 1u << (d & 31));
      }
      if (lane == 0) {
        B.h_off[nslots] = (uint32_t)used;
        B.h_run[nslots] = (uint32_t)ri;
        B.h_nrel[nslots] = (uint16_t)nrel;
        B.h_D[nslots] = (uint16_t)D;
        B.h_dmax[nslots] = (uint16_t)dmax;
        B.h_s[nslots] = (uint16_t)s;
      }
      __syncwarp();
      ++nslots;
      used += slot_words(nrel, dmax);
    }
  }
  flush();
}

// Per-run record ranges for the refine: query records of the run's window
// (from the window table) and target records of its span [j_a, j_b+n-k].
__global__ void k_run_ranges(const sedef_run_t* runs, int64_t n, const int64_t* qseq, int nqseq,
                             const int64_t* wbase, int step, const uint32_t* win_qa,
                             const uint32_t* win_qb, const uint64_t* trec, int64_t nt, int span,
                             uint4* ranges, const uint32_t* dn, const uint32_t* dnt) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= live_n(n, dn)) return;
  nt = live_n(nt, dnt);
  const sedef_run_t r = runs[x];
  const int sq = seq_of(qseq, nqseq, r.i);
  const int64_t w = wbase[sq] + ((int64_t)r.i - qseq[sq]) / step;
  auto pos_of = [](uint64_t v) { return (uint64_t)((v >> 1) & 0xFFFFFFFFull); };
  const int64_t lo = lower_bound_by(trec, 0, nt, (uint64_t)r.j_a, pos_of);
  // the span holds few records: gallop from lo
  const uint64_t end_pos = (uint64_t)r.j_b + (uint64_t)span + 1;
  int64_t stepg = 1, hi = lo;
  while (hi < nt && pos_of(trec[hi]) < end_pos) {
    hi = lo + stepg;
    stepg <<= 1;
  }
  if (hi > nt) hi = nt;
  const int64_t b = lower_bound_by(trec, lo + (stepg >> 2), hi, end_pos, pos_of);
  ranges[x] = make_uint4(win_qa[w], win_qb[w], (uint32_t)lo, (uint32_t)b);
}

// ------------------------------------------------------- tier launchers --

template <int TPB, int LCAP, int GCAP, int SLOTS = kSlots>
int launch_fast(sedef_ctx* ctx, const FArgs& a, const TierIO& io_in, int64_t max_windows,
                const char* name) {
  const size_t sm = sizeof(FastSmemT<TPB, LCAP, GCAP, SLOTS>);
  static_assert(sizeof(FastSmemT<TPB, LCAP, GCAP, SLOTS>) <= 227 * 1024,
                "a filter tier must fit one CTA's shared memory");
  SEDEF_TRY(ensure_smem_attr((const void*)k_filter_fast<TPB, LCAP, GCAP, SLOTS>, sm));
  // a table of SLOTS counters keeps its aliasing low up to 2 * SLOTS hits;
  // windows with more go on (to the wide tier when the caller names one)
  TierIO io = io_in;
  io.hlim = (uint32_t)(2 * SLOTS);
  int per_sm = 0;
  SEDEF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                           k_filter_fast<TPB, LCAP, GCAP, SLOTS>,
                                                           TPB, sm));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx_sm_count(ctx) * per_sm;
  if (grid > max_windows) grid = max_windows;
  if (grid < 1) grid = 1;
  SEDEF_KERNEL(ctx, name,
               k_filter_fast<TPB, LCAP, GCAP, SLOTS><<<(int)grid, TPB, sm, ctx_stream(ctx)>>>(a, io));
  return SEDEF_OK;
}

using FastLaunch = int (*)(sedef_ctx*, const FArgs&, const TierIO&, int64_t, const char*);

// First-tier shapes the autotuner chooses from: threads per window, hits and
// dense groups the window may hold in shared memory.
const FastLaunch kTier1[] = {launch_fast<128, 2048, 512>, launch_fast<64, 1024, 256>,
                             launch_fast<256, 2048, 512>, launch_fast<128, 1024, 256>};
constexpr int kNumTier1 = 4;
// Second-tier shapes (windows the first tier could not hold).
const FastLaunch kTier2[] = {launch_fast<256, 8192, 2048>, launch_fast<256, 4096, 1024>,
                             launch_fast<512, 8192, 2048>};
constexpr int kNumTier2 = 3;
// Wide tiers: windows with more hits than a 2,048-slot table can separate
// (long posting lists of a large target), before the global path.  32,768
// (bin, o) slots keep the prefilter selective up to 65,535 hits; the second
// wide tier holds 16,384 collected hits for windows in regions with many
// homologous copies.
constexpr int kWideSlots = 32768;
const FastLaunch kTierWide = launch_fast<512, 2048, 512, kWideSlots>;
const FastLaunch kTierWide2 = launch_fast<512, 16384, 1024, kWideSlots>;
// The second wide tier in the form that fits beside the serving kernel
// (8,192 collected hits instead of 16,384), for a context whose tier cap
// leaves the full one out.
const FastLaunch kTierWideMid = launch_fast<512, 8192, 1024, kWideSlots>;
using WideMidSmem = FastSmemT<512, 8192, 1024, kWideSlots>;
static_assert(sizeof(FastSmemT<512, 8192, 2048, 2048>) <= kTierSmemFloor &&
                  sizeof(FastSmemT<512, 2048, 512, kWideSlots>) <= kTierSmemFloor &&
                  sizeof(WarpSmem) * kWWarps <= kTierSmemFloor,
              "a tier that always runs needs more shared memory than a tier cap may be");
// variant = (warp tier off) * 12 + t1 * kNumTier2 + t2
constexpr int kNumShapes = kNumTier1 * kNumTier2;
constexpr int kNumVariants = 2 * kNumShapes;

}  // namespace

int filter_variant_count() { return kNumVariants; }

int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total);

namespace {

// The global path (eager) over the windows a.ov_list[0..nov): hits counted
// per window, then batches of at most 2^27 hits emitted, radix-sorted by
// (window, o, t) and swept by dense group.  Adds the hits to
// *slow_hits_total.
int global_path_eager(sedef_ctx* ctx, const FArgs& a, int64_t nov, unsigned long long* counters,
                      int64_t* slow_hits_total) {
  cudaStream_t st = ctx_stream(ctx);
  // slow path: count, then batches of emit -> sort -> sweep
  unsigned long long* ocnt = (unsigned long long*)ctx_alloc(ctx, (size_t)(nov + 1) * 8);
  int32_t* os = (int32_t*)ctx_alloc(ctx, (size_t)(nov + 1) * 4);
  if (!ocnt || !os) return SEDEF_ERR_OOM;
  int64_t sgrid = nov < (int64_t)ctx_sm_count(ctx) * 4 ? nov : (int64_t)ctx_sm_count(ctx) * 4;
  SEDEF_KERNEL(ctx, "k_slow_count",
               k_slow_count<unsigned long long><<<(int)sgrid, kSThreads, 0, st>>>(a, nov, ocnt, os,
                                                                                  nullptr, nullptr));
  std::vector<unsigned long long> hc(nov + 1, 0);
  SEDEF_CUDA(cudaMemcpyAsync(hc.data(), ocnt, (size_t)nov * 8, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  std::vector<unsigned long long> base(nov + 1, 0);
  for (int64_t v = 0; v < nov; ++v) base[v + 1] = base[v] + hc[v];
  unsigned long long* d_base = (unsigned long long*)ctx_alloc(ctx, (size_t)(nov + 1) * 8);
  if (!d_base) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemcpyAsync(d_base, base.data(), (size_t)(nov + 1) * 8, cudaMemcpyHostToDevice, st));
  *slow_hits_total += (int64_t)base[nov];
  const unsigned long long budget = 1ull << 27;  // hits per batch
  int64_t v0 = 0;
  while (v0 < nov) {
    int64_t v1 = v0 + 1;
    while (v1 < nov && base[v1 + 1] - base[v0] <= budget && v1 - v0 < (1 << 20)) ++v1;
    const unsigned long long nh = base[v1] - base[v0];
    // a batch's scratch goes back to the pool once the batch has run
    const std::vector<char> used_before = ctx_pool_snapshot(ctx);
    if (nh > 0) {
      uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)nh * 8);
      uint32_t* vals = (uint32_t*)ctx_alloc(ctx, (size_t)nh * 4);
      uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)nh * 8);
      uint32_t* svals = (uint32_t*)ctx_alloc(ctx, (size_t)nh * 4);
      if (!keys || !vals || !skeys || !svals) return SEDEF_ERR_OOM;
      const int64_t nb = v1 - v0;
      int g = (int)(nb < (int64_t)ctx_sm_count(ctx) * 4 ? nb : (int64_t)ctx_sm_count(ctx) * 4);
      SEDEF_KERNEL(ctx, "k_slow_emit",
                   k_slow_emit<<<g, kSThreads, 0, st>>>(a, v0, v1, d_base, keys, vals, nullptr,
                                                        (int64_t)nh));
      int wbits = 0;
      while ((int64_t(1) << wbits) < nb) ++wbits;
      SEDEF_TRY(radix_sort_u64(ctx, keys, vals, skeys, svals, (int64_t)nh, 0, 33 + wbits));
      SlowTask* tasks = (SlowTask*)ctx_alloc(ctx, (size_t)nh * sizeof(SlowTask));
      if (!tasks) return SEDEF_ERR_OOM;
      SEDEF_CUDA(cudaMemsetAsync(counters + 6, 0, 8, st));
      const int64_t gw = (nb + 7) / 8;
      int g2 = (int)(gw < (int64_t)ctx_sm_count(ctx) * 8 ? gw : (int64_t)ctx_sm_count(ctx) * 8);
      SEDEF_KERNEL(ctx, "k_slow_groups",
                   k_slow_groups<<<g2, 256, 0, st>>>(a, v0, v1, d_base, os, skeys, tasks,
                                                     counters + 6, (int64_t)nh, nullptr,
                                                     (int64_t)nh));
      SEDEF_KERNEL(ctx, "k_slow_tasks",
                   k_slow_tasks<<<ctx_sm_count(ctx) * 8, 32 * kTaskWarps, 0, st>>>(
                       a, v0, d_base, os, skeys, svals, tasks, counters + 6, (int64_t)nh));
      SEDEF_CUDA(cudaStreamSynchronize(st));
    }
    ctx_pool_restore(ctx, used_before);
    v0 = v1;
  }
  return SEDEF_OK;
}

// Orders the `total` raw runs by (window, o, j_a) into `runs` and refines
// them (the winnowed MinHash estimate at every breakpoint of each run).
// druns / dnt: live counts of a planned pass (nullptr when eager).
int order_and_refine(sedef_ctx* ctx, const FArgs& a, const Derived& D, int nqseq,
                     const int64_t* d_wbase, int64_t nwin, const uint32_t* wqa, const uint32_t* wqb,
                     const uint64_t* qrec, int64_t nq, const uint64_t* trec, int64_t nt,
                     const uint32_t* toff, unsigned long long* counters, sedef_run_t* raw,
                     int64_t total, sedef_run_t* runs, const uint32_t* druns, const uint32_t* dnt) {
  cudaStream_t st = ctx_stream(ctx);
  SEDEF_TRY(ensure_smem_attr((const void*)k_refine_batch, sizeof(BatchWarp) * kBWarps));
  SEDEF_TRY(ensure_smem_attr((const void*)k_refine<kMaxWindowRecs, 1024, false>,
                             sizeof(RefineWarpT<kMaxWindowRecs, 1024>) * kRWarpsBig));
  // order runs by (i, o); the sweep emits each window's runs in j order
  ctx_set_stage(ctx, "runsort");
  uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)total * 8);
  uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)total * 8);
  uint32_t* perm = (uint32_t*)ctx_alloc(ctx, (size_t)total * 4);
  if (!keys || !skeys || !perm) return SEDEF_ERR_OOM;
  const int tb = (int)((total + 255) / 256);
  int wb = 1;
  while ((int64_t(1) << wb) < nwin) ++wb;
  if (33 + wb <= 64) {
    SEDEF_KERNEL(ctx, "k_run_keys",
                 k_run_keys<<<tb, 256, 0, st>>>(raw, total, a.qseq, nqseq, d_wbase, D.step, 0, keys,
                                                druns));
    SEDEF_TRY(radix_sort_u64(ctx, keys, nullptr, skeys, perm, total, 0, 33 + wb, druns));
  } else {
    // stable two-pass order: by j_a, then by (window, o)
    uint32_t* perm1 = (uint32_t*)ctx_alloc(ctx, (size_t)total * 4);
    uint32_t* perm2 = (uint32_t*)ctx_alloc(ctx, (size_t)total * 4);
    uint64_t* k2 = (uint64_t*)ctx_alloc(ctx, (size_t)total * 8);
    if (!perm1 || !perm2 || !k2) return SEDEF_ERR_OOM;
    SEDEF_KERNEL(ctx, "k_run_keys",
                 k_run_keys<<<tb, 256, 0, st>>>(raw, total, a.qseq, nqseq, d_wbase, D.step, 1, keys,
                                                druns));
    SEDEF_TRY(radix_sort_u64(ctx, keys, nullptr, skeys, perm1, total, 0, 32, druns));
    SEDEF_KERNEL(ctx, "k_run_keys",
                 k_run_keys<<<tb, 256, 0, st>>>(raw, total, a.qseq, nqseq, d_wbase, D.step, 2, keys,
                                                druns));
    SEDEF_KERNEL(ctx, "k_permute_u64",
                 k_permute_u64<<<tb, 256, 0, st>>>(keys, perm1, total, k2, druns));
    SEDEF_TRY(radix_sort_u64(ctx, k2, nullptr, skeys, perm2, total, 0, wb + 1, druns));
    SEDEF_KERNEL(ctx, "k_compose_perm",
                 k_compose_perm<<<tb, 256, 0, st>>>(perm1, perm2, total, perm, druns));
  }
  SEDEF_KERNEL(ctx, "k_gather_runs",
               k_gather_runs<<<tb, 256, 0, st>>>(raw, perm, total, runs, druns));
  // refine: lean kernel over all runs, then the large kernel over the runs
  // it handed over (their count stays on the device)
  ctx_set_stage(ctx, "refine");
  uint32_t* big = (uint32_t*)ctx_alloc(ctx, (size_t)total * 4);
  if (!big) return SEDEF_ERR_OOM;
  RefineArgs ra;
  ra.runs = runs;
  ra.nruns = total;
  ra.qrec = qrec;
  ra.nq = nq;
  ra.trec = trec;
  ra.nt = nt;
  ra.dnruns = druns;
  ra.dnt = dnt;
  ra.toff = toff;
  ra.mtab = a.mtab;
  ra.span = D.span;
  ra.max_occ = D.max_occ;
  ra.self_mode = D.self_mode;
  ra.big = big;
  ra.nbig = (unsigned int*)(counters + 3);
  uint4* ranges = (uint4*)ctx_alloc(ctx, (size_t)total * sizeof(uint4));
  if (!ranges) return SEDEF_ERR_OOM;
  SEDEF_KERNEL(ctx, "k_run_ranges",
               k_run_ranges<<<tb, 256, 0, st>>>(runs, total, a.qseq, nqseq, d_wbase, D.step, wqa, wqb,
                                                trec, nt, D.span, ranges, druns, dnt));
  ra.ranges = ranges;
  ra.next = counters + 6;
  SEDEF_CUDA(cudaMemsetAsync(counters + 6, 0, 16, st));
  using Big = RefineWarpT<kMaxWindowRecs, 1024>;
  const size_t lean_sm = sizeof(BatchWarp) * kBWarps, big_sm = sizeof(Big) * kRWarpsBig;
  int rper = 0;
  SEDEF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, k_refine_batch, 32 * kBWarps,
                                                           lean_sm));
  if (rper < 1) rper = 1;
  int64_t rgrid = (total + kBWarps * 32 - 1) / (kBWarps * 32);
  if (rgrid > (int64_t)ctx_sm_count(ctx) * rper) rgrid = (int64_t)ctx_sm_count(ctx) * rper;
  if (rgrid < 1) rgrid = 1;
  SEDEF_KERNEL(ctx, "k_refine",
               k_refine_batch<<<(int)rgrid, 32 * kBWarps, lean_sm, st>>>(ra));
  SEDEF_KERNEL(ctx, "k_refine_big",
               k_refine<kMaxWindowRecs, 1024, false><<<ctx_sm_count(ctx), 32 * kRWarpsBig, big_sm,
                                                       st>>>(ra));
  return SEDEF_OK;
}

}  // namespace

int run_filter(sedef_ctx* ctx, const uint64_t* qrec, int64_t nq, const int64_t* h_qoff, int nqseq,
               const uint64_t* trec, const uint64_t* tsorted, const uint32_t* toff, int64_t nt,
               const int64_t* h_toff, int ntseq, const Derived& D, const int32_t* h_mtab,
               sedef_run_t* runs, int64_t cap, int64_t* nruns, int tune, Planned* pl) {
  cudaStream_t st = ctx_stream(ctx);
  StageScope stage(ctx, "filter");  // the caller's label comes back on return
  if (pl && tune) return fail(SEDEF_ERR_INVALID, "sedef_filter: no autotuning inside a planned pass");
  // live record counts of a planned pass (query and target are one sketch)
  const uint32_t* dnq = pl ? pl->n_rec : nullptr;
  const uint32_t* dnt = pl ? pl->n_rec : nullptr;
  // windows per query sequence
  std::vector<int64_t> wbase(nqseq + 1, 0);
  for (int s = 0; s < nqseq; ++s) {
    const int64_t len = h_qoff[s + 1] - h_qoff[s];
    const int64_t cnt = len >= D.n ? (len - D.n) / D.step + 1 : 0;
    wbase[s + 1] = wbase[s] + cnt;
  }
  const int64_t nwin = wbase[nqseq];
  *nruns = 0;
  if (nwin == 0 || nq == 0 || nt == 0) return SEDEF_OK;
  // uploads: query offsets, target offsets, window bases, m table
  const size_t up_bytes = (size_t)(nqseq + 1) * 8 * 2 + (size_t)(ntseq + 1) * 8 +
                          (size_t)(kMaxWindowRecs + 1) * 4;
  char* h_up = (char*)host_buf(ctx, pl, up_bytes + 64);
  char* d_up = (char*)ctx_alloc(ctx, up_bytes + 64);
  if (!h_up || !d_up) return SEDEF_ERR_OOM;
  size_t o = 0;
  int64_t* h_q = (int64_t*)(h_up + o);
  const size_t oq = o;
  std::memcpy(h_q, h_qoff, (size_t)(nqseq + 1) * 8);
  o += (size_t)(nqseq + 1) * 8;
  const size_t ot = o;
  std::memcpy(h_up + o, h_toff, (size_t)(ntseq + 1) * 8);
  o += (size_t)(ntseq + 1) * 8;
  const size_t ow = o;
  std::memcpy(h_up + o, wbase.data(), (size_t)(nqseq + 1) * 8);
  o += (size_t)(nqseq + 1) * 8;
  const size_t om = o;
  std::memcpy(h_up + o, h_mtab, (size_t)(kMaxWindowRecs + 1) * 4);
  SEDEF_CUDA(cudaMemcpyAsync(d_up, h_up, up_bytes, cudaMemcpyHostToDevice, st));

  uint32_t* wi = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* wqa = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* wqb = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  int32_t* wseq = (int32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* ovl = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* ovl1 = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* ovl0 = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* ovlw = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  uint32_t* ovlw2 = (uint32_t*)ctx_alloc(ctx, (size_t)nwin * 4);
  if (!ovl0 || !ovlw || !ovlw2) return SEDEF_ERR_OOM;
  // [0] runs, [1] windows for the global path, [2] tier-1 work, [3] large
  // refine runs, [4] hits, [5] collected hits, [6]/[7] task and refine work,
  // [8] tier-2 work, [9] windows tier 1 handed to tier 2, [10] sample size,
  // [11] global-path hits (planned pass), [12]/[13] warp-tier hand-overs and
  // work, [14] windows for the wide tier, [15] wide-tier work, [16]/[17] the
  // same for the second wide tier
  unsigned long long* counters = (unsigned long long*)ctx_alloc(ctx, 256);
  sedef_run_t* raw = (sedef_run_t*)ctx_alloc(ctx, (size_t)(cap > 0 ? cap : 1) * sizeof(sedef_run_t));
  if (!wi || !wqa || !wqb || !wseq || !ovl || !ovl1 || !counters || !raw) return SEDEF_ERR_OOM;

  SEDEF_CUDA(cudaMemsetAsync(counters, 0, 256, st));

  FArgs a;
  a.qrec = qrec;
  a.trec = trec;
  a.tsorted = tsorted;
  a.toff = toff;
  a.qseq = (const int64_t*)(d_up + oq);
  a.tseq = (const int64_t*)(d_up + ot);
  a.mtab = (const int32_t*)(d_up + om);
  a.win_i = wi;
  a.win_qa = wqa;
  a.win_qb = wqb;
  a.win_seq = wseq;
  a.nwin = nwin;
  a.ntseq = ntseq;
  a.nqseq = nqseq;
  a.ttotal = h_toff[ntseq];
  a.k = D.k;
  a.n = D.n;
  a.span = D.span;
  a.max_occ = D.max_occ;
  a.self_mode = D.self_mode;
  a.overlap = D.overlap;
  a.runs = raw;
  a.nruns = counters;
  a.run_cap = cap;
  a.ov_list = ovl;
  a.nov = (unsigned int*)(counters + 1);
  a.next_window = (unsigned int*)(counters + 2);
  a.stats = counters + 4;

  a.qpost = nullptr;
  a.tsamp = nullptr;
  if (D.self_mode == 2) {
    // every posting search of a batch self-search starts from the samples
    const int64_t ns = (nt + kSampleStride - 1) >> kSampleShift;
    uint32_t* samp = (uint32_t*)ctx_alloc(ctx, (size_t)ns * 4);
    if (!samp) return SEDEF_ERR_OOM;
    int64_t g = (ns + 255) / 256;
    if (g > (int64_t)ctx_sm_count(ctx) * 16) g = (int64_t)ctx_sm_count(ctx) * 16;
    SEDEF_KERNEL(ctx, "k_sample_pos", k_sample_pos<<<(int)g, 256, 0, st>>>(tsorted, nt, dnt, samp));
    a.tsamp = samp;
  }
  if (D.self_mode == 2 && 2 * D.k <= 24) {
    // batch self-search: every query record's posting range in its own
    // genome, once (the warp tier reads them by record offset).  An eager
    // pass walks the index (the query records are its records, with the
    // same sequence offsets); a planned pass, whose counts live on the
    // device, searches per record.
    uint2* qp = (uint2*)ctx_alloc(ctx, (size_t)nq * sizeof(uint2));
    if (!qp) return SEDEF_ERR_OOM;
    const int64_t nw = (a.ttotal + 31) >> 5;
    const bool walk = !pl && nqseq == ntseq &&
                      std::memcmp(h_qoff, h_toff, (size_t)(ntseq + 1) * sizeof(int64_t)) == 0;
    uint32_t* pbits = walk ? (uint32_t*)ctx_alloc(ctx, (size_t)(nw + 1) * 4) : nullptr;
    uint32_t* pcnt = walk ? (uint32_t*)ctx_alloc(ctx, (size_t)(nw + 1) * 4) : nullptr;
    uint32_t* pbef = walk ? (uint32_t*)ctx_alloc(ctx, (size_t)(nw + 1) * 4) : nullptr;
    RankWord* rw = walk ? (RankWord*)ctx_alloc(ctx, (size_t)(nw + 1) * sizeof(RankWord)) : nullptr;
    if (walk && (!pbits || !pcnt || !pbef || !rw)) return SEDEF_ERR_OOM;
    int64_t g = (nq + 255) / 256;
    if (g > (int64_t)ctx_sm_count(ctx) * 16) g = (int64_t)ctx_sm_count(ctx) * 16;
    if (g < 1) g = 1;
    if (!walk) {
      SEDEF_KERNEL(ctx, "k_qpost", k_qpost<<<(int)g, 256, 0, st>>>(a, nq, dnq, qp));
    } else {
      int64_t gw = (nw + 255) / 256;
      if (gw > (int64_t)ctx_sm_count(ctx) * 16) gw = (int64_t)ctx_sm_count(ctx) * 16;
      if (gw < 1) gw = 1;
      SEDEF_CUDA(cudaMemsetAsync(pbits, 0, (size_t)(nw + 1) * 4, st));
      SEDEF_KERNEL(ctx, "k_pos_bits", k_pos_bits<<<(int)g, 256, 0, st>>>(qrec, nq, pbits));
      SEDEF_KERNEL(ctx, "k_pos_popc", k_pos_popc<<<(int)gw, 256, 0, st>>>(pbits, nw, pcnt));
      SEDEF_TRY(scan_exclusive_u32(ctx, pcnt, pbef, nw, pbef + nw));
      SEDEF_KERNEL(ctx, "k_rank_words", k_rank_words<<<(int)gw, 256, 0, st>>>(pbits, pbef, nw, rw));
      SEDEF_KERNEL(ctx, "k_qpost", k_qpost_index<<<(int)g, 256, 0, st>>>(a, nt, rw, qp));
    }
    a.qpost = qp;
  }
  SEDEF_KERNEL(ctx, "k_windows",
               k_windows<<<(int)((nwin + 255) / 256), 256, 0, st>>>(
                   qrec, nq, a.qseq, nqseq, (const int64_t*)(d_up + ow), nwin, D.step, D.span, wi,
                   wqa, wqb, wseq, dnq));
  if (tune) {
    // time every first-tier shape on a uniform sample of windows (at least
    // 65,536 or a sixteenth of them, so that a run lasts long enough to
    // time); keep the fastest
    const int64_t want = nwin / 16 > 65536 ? nwin / 16 : 65536;
    const int64_t stride = nwin > want ? nwin / want : 1;
    std::vector<uint32_t> sample;
    for (int64_t w = 0; w < nwin; w += stride) sample.push_back((uint32_t)w);
    const unsigned int ns = (unsigned int)sample.size();
    uint32_t* d_sample = (uint32_t*)ctx_alloc(ctx, (size_t)ns * 4 + 8);
    if (!d_sample) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(d_sample, sample.data(), (size_t)ns * 4, cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaMemcpyAsync(counters + 10, &ns, 4, cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    SEDEF_CUDA(cudaEventCreate(&e0));
    SEDEF_CUDA(cudaEventCreate(&e1));
    int best_v = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < kNumVariants; ++v) {
      float ms = 0.f;
      const int sh = v % kNumShapes;
      const bool warp_tier = v < kNumShapes;
      float best_rep = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {  // the first repetition warms up
        SEDEF_CUDA(cudaMemsetAsync(counters, 0, 80, st));
        SEDEF_CUDA(cudaMemsetAsync(counters + 12, 0, 48, st));
        TierIO io0{d_sample, (const unsigned int*)(counters + 10), ovl0,
                   (unsigned int*)(counters + 12), (unsigned int*)(counters + 13), 0};
        TierIO io{warp_tier ? ovl0 : d_sample,
                  (const unsigned int*)(counters + (warp_tier ? 12 : 10)), ovl1,
                  (unsigned int*)(counters + 9), (unsigned int*)(counters + 2), 0};
        io.wide_list = ovlw;
        io.wide_count = (unsigned int*)(counters + 14);
        TierIO io2{ovl1, (const unsigned int*)(counters + 9), ovlw, (unsigned int*)(counters + 14),
                   (unsigned int*)(counters + 8), 0};
        io2.wide_list = ovlw;
        io2.wide_count = (unsigned int*)(counters + 14);
        TierIO iow{ovlw, (const unsigned int*)(counters + 14), ovlw2,
                   (unsigned int*)(counters + 16), (unsigned int*)(counters + 15), 0};
        TierIO iow2{ovlw2, (const unsigned int*)(counters + 16), ovl,
                    (unsigned int*)(counters + 1), (unsigned int*)(counters + 17), 0};
        SEDEF_CUDA(cudaEventRecord(e0, st));
        if (warp_tier) SEDEF_TRY(launch_warp_tier(ctx, a, io0, ns, "k_filter_tune"));
        SEDEF_TRY(kTier1[sh / kNumTier2](ctx, a, io, ns, "k_filter_tune"));
        SEDEF_TRY(kTier2[sh % kNumTier2](ctx, a, io2, ns, "k_filter_tune"));
        SEDEF_TRY(kTierWide(ctx, a, iow, ns, "k_filter_tune"));
        SEDEF_TRY(kTierWide2(ctx, a, iow2, ns, "k_filter_tune"));
        SEDEF_CUDA(cudaEventRecord(e1, st));
        SEDEF_CUDA(cudaEventSynchronize(e1));
        SEDEF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best_rep) best_rep = ms;
      }
      ms = best_rep;
      if (ms < best_ms) {
        best_ms = ms;
        best_v = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_set_filter_variant(ctx, best_v);
    *nruns = best_v;
    return SEDEF_OK;
  }
  {
    // the warp tier over all windows (unless the autotuned variant leaves it
    // out), tier 1 (autotuned shape) over what it could not hold, tier 2
    // (4,096-8,192 hits in shared memory) after that, the wide tier over the
    // windows with many hits (from tiers 1 and 2) and over what tier 2 could
    // not hold, the global path last
    int v = ctx_filter_variant(ctx);
    if (v < 0 || v >= kNumVariants) v = 0;
    const int sh = v % kNumShapes;
    const bool warp_tier = v < kNumShapes;
    if (warp_tier) {
      TierIO io0{nullptr, nullptr, ovl0, (unsigned int*)(counters + 12),
                 (unsigned int*)(counters + 13), 1};
      SEDEF_TRY(launch_warp_tier(ctx, a, io0, nwin, "k_filter_warp"));
    }
    TierIO io1{warp_tier ? ovl0 : nullptr,
               warp_tier ? (const unsigned int*)(counters + 12) : nullptr, ovl1,
               (unsigned int*)(counters + 9), (unsigned int*)(counters + 2), 1};
    io1.wide_list = ovlw;
    io1.wide_count = (unsigned int*)(counters + 14);
    SEDEF_TRY(kTier1[sh / kNumTier2](ctx, a, io1, nwin, "k_filter_fast"));
    TierIO io2{ovl1, (const unsigned int*)(counters + 9), ovlw, (unsigned int*)(counters + 14),
               (unsigned int*)(counters + 8), 1};
    io2.wide_list = ovlw;
    io2.wide_count = (unsigned int*)(counters + 14);
    SEDEF_TRY(kTier2[sh % kNumTier2](ctx, a, io2, nwin, "k_filter_mid"));
    // where the second wide tier's CTA would pass the context's cap, its
    // 8,192-hit form takes its place, or, where that would pass it too, the
    // wide tier hands its leftovers straight to the global path
    const size_t scap = ctx_tier_smem_cap(ctx);
    const bool wide2 = sizeof(FastSmemT<512, 16384, 1024, kWideSlots>) <= scap;
    const bool mid = !wide2 && sizeof(WideMidSmem) <= scap;
    const bool second = wide2 || mid;
    TierIO iow{ovlw, (const unsigned int*)(counters + 14), second ? ovlw2 : ovl,
               (unsigned int*)(counters + (second ? 16 : 1)), (unsigned int*)(counters + 15), 1};
    SEDEF_TRY(kTierWide(ctx, a, iow, nwin, "k_filter_wide"));
    TierIO iow2{ovlw2, (const unsigned int*)(counters + 16), ovl, (unsigned int*)(counters + 1),
                (unsigned int*)(counters + 17), 1};
    if (wide2) SEDEF_TRY(kTierWide2(ctx, a, iow2, nwin, "k_filter_wide2"));
    if (mid) SEDEF_TRY(kTierWideMid(ctx, a, iow2, nwin, "k_filter_widemid"));
  }

  unsigned long long* h_cnt = nullptr;
  int64_t nov = 0, slow_hits_total = 0;
  if (pl) {
    // planned: the global path over the live overflow list in one batch of
    // at most pl->slow_hits hits
    const uint32_t* dnov = (const uint32_t*)(counters + 1);
    const int64_t H = pl->slow_hits > 0 ? pl->slow_hits : 1;
    uint32_t* cnt32 = (uint32_t*)ctx_alloc(ctx, (size_t)(nwin + 1) * 4);
    uint32_t* base32 = (uint32_t*)ctx_alloc(ctx, (size_t)(nwin + 1) * 4);
    unsigned long long* d_base = (unsigned long long*)ctx_alloc(ctx, (size_t)(nwin + 1) * 8);
    int32_t* os = (int32_t*)ctx_alloc(ctx, (size_t)(nwin + 1) * 4);
    uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)H * 8);
    uint32_t* vals = (uint32_t*)ctx_alloc(ctx, (size_t)H * 4);
    uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)H * 8);
    uint32_t* svals = (uint32_t*)ctx_alloc(ctx, (size_t)H * 4);
    SlowTask* tasks = (SlowTask*)ctx_alloc(ctx, (size_t)H * sizeof(SlowTask));
    if (!cnt32 || !base32 || !d_base || !os || !keys || !vals || !skeys || !svals || !tasks)
      return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemsetAsync(cnt32, 0, (size_t)(nwin + 1) * 4, st));
    const int sgrid = (int)(nwin < (int64_t)ctx_sm_count(ctx) * 4 ? nwin : (int64_t)ctx_sm_count(ctx) * 4);
    SEDEF_KERNEL(ctx, "k_slow_count",
                 k_slow_count<uint32_t><<<sgrid, kSThreads, 0, st>>>(a, nwin, cnt32, os, dnov,
                                                                     counters + 11));
    // 32-bit offsets: a window whose range wraps is skipped; the exact
    // 64-bit total (counters[11]) decides the overflow
    SEDEF_TRY(scan_exclusive_u32(ctx, cnt32, base32, nwin, base32 + nwin));
    SEDEF_KERNEL(ctx, "k_widen_u32",
                 k_widen_u32<<<(int)((nwin + 256) / 256), 256, 0, st>>>(base32, nwin + 1, d_base));
    const uint32_t* dhits = base32 + nwin;
    SEDEF_TRY(plan_check64(ctx, pl, counters + 11, H, 1));
    SEDEF_KERNEL(ctx, "k_slow_emit",
                 k_slow_emit<<<sgrid, kSThreads, 0, st>>>(a, 0, nwin, d_base, keys, vals, dnov, H));
    int wbits = 0;
    while ((int64_t(1) << wbits) < nwin) ++wbits;
    SEDEF_TRY(radix_sort_u64(ctx, keys, vals, skeys, svals, H, 0, 33 + wbits, dhits));
    SEDEF_CUDA(cudaMemsetAsync(counters + 6, 0, 8, st));
    const int64_t gw = (nwin + 7) / 8;
    const int g2 = (int)(gw < (int64_t)ctx_sm_count(ctx) * 8 ? gw : (int64_t)ctx_sm_count(ctx) * 8);
    SEDEF_KERNEL(ctx, "k_slow_groups",
                 k_slow_groups<<<g2, 256, 0, st>>>(a, 0, nwin, d_base, os, skeys, tasks,
                                                   counters + 6, H, dnov, H));
    SEDEF_KERNEL(ctx, "k_slow_tasks",
                 k_slow_tasks<<<ctx_sm_count(ctx) * 8, 32 * kTaskWarps, 0, st>>>(
                     a, 0, d_base, os, skeys, svals, tasks, counters + 6, H));
  } else {
    h_cnt = (unsigned long long*)ctx_host(ctx, 64);
    if (!h_cnt) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(h_cnt, counters, 16, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
    nov = (int64_t)(h_cnt[1] & 0xFFFFFFFFull);
  }

  if (nov > 0) {
    SEDEF_TRY(global_path_eager(ctx, a, nov, counters, &slow_hits_total));
    SEDEF_CUDA(cudaMemcpyAsync(h_cnt, counters, 8, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
  }
  // runs: the exact count (eager) or the planned capacity with the live
  // count on the device (the low word of counters[0])
  const uint32_t* druns = nullptr;
  int64_t total;
  if (pl) {
    total = cap;
    druns = (const uint32_t*)counters;
    pl->n_runs = druns;
    SEDEF_TRY(plan_check(ctx, pl, druns, cap, 2));
    *nruns = cap;
    if (total == 0) return SEDEF_OK;
  } else {
    total = (int64_t)h_cnt[0];
    *nruns = total;
    if (total > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_filter: run buffer too small");
    if (total == 0) return SEDEF_OK;
  }
  SEDEF_TRY(order_and_refine(ctx, a, D, nqseq, (const int64_t*)(d_up + ow), nwin, wqa, wqb, qrec,
                             nq, trec, nt, toff, counters, raw, total, runs, druns, dnt));
  if (pl) return SEDEF_OK;
  SEDEF_CUDA(cudaMemcpyAsync(h_cnt, counters, 64, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  {
    const int64_t stats[7] = {nwin, nov, (int64_t)h_cnt[4], (int64_t)h_cnt[5], total,
                              (int64_t)(h_cnt[3] & 0xFFFFFFFFull), slow_hits_total};
    ctx_set_stats(ctx, stats, 7);
  }
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // namespace sedef

// ===================================================== continuous batching ==
//
// Serving against a resident target index.  A persistent kernel (one small
// CTA per SM, so that every SM keeps room for the kernels of other streams)
// drains a work queue of query windows: a
// ring of (slot, window) items in mapped host memory that the host
// publishes as requests are admitted into free slots.  A slot holds one
// request's query sketch, window table and outputs in device memory that
// the server allocated once.  A CTA claims an item only when the ring holds
// one (compare-and-swap on the device head below the published tail), runs
// the window through the shared-memory tier into its slot's runs (windows
// the tier cannot hold into the slot's overflow list), and the CTA that
// finishes a slot's last window writes the slot's epoch into a mapped
// completion word.  The host then runs the global path for the overflow
// windows, the run ordering, refine, chaining and merging of that slot on
// its own stream while the kernel keeps serving the other slots.  A CTA that
// finds the ring empty sleeps and polls; when nothing arrives for
// idle_timeout (or the host raises the stop word) it leaves, and a CTA that
// left on the idle limit records SEDEF_ERR_TIMEOUT in the control block.
// The host relaunches the kernel when work arrives and no CTA is running.
// Query-side data is read past L1 (a slot's buffers are refilled while the
// kernel runs).
namespace sedef {
namespace {

constexpr int kServeMaxSlots = 64;
// One CTA per SM of 256 threads (16 K registers) and ~62 KB of shared
// memory: the rest of every SM stays free for the admission and finishing
// kernels (the radix sort's scatter alone takes ~39 K registers per CTA),
// which would otherwise wait for the persistent kernel to leave.
constexpr int kServeTPB = 256, kServeLCap = 2048, kServeGCap = 512, kServeSlots = 16384;
using ServeSmem = FastSmemT<kServeTPB, kServeLCap, kServeGCap, kServeSlots>;
// Windows with more hits than this go to the slot's wide list before their
// hits are enumerated; the finishing call runs the wide tier (512 threads,
// 32,768 counters) over them as an ordinary launch beside k_serve, as the
// first tier of a whole-genome pass hands them on.
constexpr uint32_t kServeHlim = 2 * kSlots;
// Finishing calls that may run at once (each on its own stream and context).
constexpr int kServeFinishers = 5;

struct ServeItem {
  uint32_t slot, window;
};

// Control block in mapped host memory (both sides read and write it).
struct ServeCtl {
  unsigned long long tail;                   // items published (host)
  int stop;                                  // host: leave now
  int status;                                // device: SEDEF_ERR_TIMEOUT after an idle exit
  long long nwin[kServeMaxSlots];            // host: windows of the slot's request
  unsigned int epoch[kServeMaxSlots];        // host: admission number of the slot
  unsigned int done_epoch[kServeMaxSlots];   // device: epoch whose last window finished
};

// Per-slot constants in device memory (written once, at creation).
struct SlotDev {
  FArgs a;              // the slot's query, windows and outputs
  unsigned int* done;   // windows finished (reset at admission)
  uint32_t* wide_list;  // windows with more hits than k_serve keeps (for the wide tier)
  unsigned int* wide_count;
  uint32_t* mid_list;   // windows k_serve could not hold (for the 8,192-hit tier)
  unsigned int* mid_count;
};

struct ServeArgs {
  const SlotDev* slots;
  const ServeItem* ring;     // mapped host memory (device view)
  unsigned long long ring_cap;
  ServeCtl* ctl;             // mapped host memory (device view)
  unsigned long long* head;  // device memory
  unsigned long long idle_ns;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kServeTPB) k_serve(ServeArgs sv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ServeSmem& S = *reinterpret_cast<ServeSmem*>(smem_raw);
  __shared__ long long s_item;
  __shared__ unsigned int s_slot, s_window;
  for (int x = threadIdx.x; x < kQCap * (kServeTPB / 32); x += blockDim.x) (&S.cnt[0][0])[x] = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      // claim the next published item; sleep while there is none, at most
      // idle_ns in a row
      long long got = -1;
      const unsigned long long idle_from = global_ns();
      unsigned int nap = 256;
      while (true) {
        const unsigned long long t = ld_acquire_sys(&sv.ctl->tail);
        const unsigned long long h = *(volatile unsigned long long*)sv.head;
        if (h < t) {
          if (atomicCAS(sv.head, h, h + 1) == h) {
            got = (long long)h;
            break;
          }
          continue;
        }
        if (*(volatile int*)&sv.ctl->stop) break;
        if (global_ns() - idle_from > sv.idle_ns) {
          *(volatile int*)&sv.ctl->status = SEDEF_ERR_TIMEOUT;
          __threadfence_system();
          break;
        }
        __nanosleep(nap);
        if (nap < 8192) nap <<= 1;
      }
      s_item = got;
      if (got >= 0) {
        const volatile ServeItem* it = sv.ring + (unsigned long long)got % sv.ring_cap;
        s_slot = it->slot;
        s_window = it->window;
      }
    }
    __syncthreads();
    if (s_item < 0) break;
    const unsigned int slot = s_slot;
    const SlotDev& sd = sv.slots[slot];
    TierIO io;
    io.in_list = nullptr;
    io.in_count = nullptr;
    io.out_list = sd.mid_list;
    io.out_count = sd.mid_count;
    io.next = nullptr;
    io.stats = 1;
    io.hlim = kServeHlim;
    io.wide_list = sd.wide_list;
    io.wide_count = sd.wide_count;
    fast_window<kServeTPB, kServeLCap, kServeGCap, kServeSlots>(sd.a, io, S, (int64_t)s_window);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this window's runs and hand-overs before its count
      const unsigned int d = atomicAdd(sd.done, 1u) + 1u;
      if ((long long)d == *(volatile long long*)&sv.ctl->nwin[slot]) {
        __threadfence_system();
        *(volatile unsigned int*)&sv.ctl->done_epoch[slot] =
            *(volatile unsigned int*)&sv.ctl->epoch[slot];
        __threadfence_system();
      }
    }
  }
}

}  // namespace

// Host side of one server.
struct Server {
  int device = 0;
  int nslots = 0;
  int64_t slot_bases = 0;
  Derived D;
  sedef_params P;
  std::vector<int32_t> mtab;
  // the resident target (owned by the caller)
  const uint64_t* trec = nullptr;
  const uint64_t* tsorted = nullptr;
  const uint32_t* toff = nullptr;
  int64_t nt = 0;
  std::vector<int64_t> h_toff;
  // streams and contexts: admission, the persistent kernel, finishing (one
  // stream and context per concurrent sedef_server_finish call)
  cudaStream_t s_prep = nullptr, s_kern = nullptr;
  sedef_ctx* c_prep = nullptr;
  struct Finisher {
    cudaStream_t stream = nullptr;
    sedef_ctx* ctx = nullptr;
    bool busy = false;
  };
  std::vector<Finisher> fins;
  std::condition_variable fin_cv;
  cudaEvent_t kern_done = nullptr;
  bool kern_launched = false;
  char* d_shared = nullptr;  // target offsets and the m table
  // mapped host memory: host views and device views
  ServeCtl* ctl = nullptr;
  ServeCtl* d_ctl = nullptr;
  ServeItem* ring = nullptr;
  ServeItem* d_ring = nullptr;
  unsigned long long ring_cap = 0;
  unsigned long long tail = 0;
  unsigned long long* d_head = nullptr;
  SlotDev* d_slots = nullptr;
  double idle_s = 1.0;
  struct Slot {
    uint8_t* seq = nullptr;
    uint32_t *packed = nullptr, *mask = nullptr, *nbits = nullptr;
    uint64_t* qrec = nullptr;
    int64_t rec_cap = 0;
    uint32_t *wi = nullptr, *wqa = nullptr, *wqb = nullptr, *ov = nullptr, *wl = nullptr,
             *ml = nullptr;
    int32_t* wseq = nullptr;
    int64_t win_cap = 0;
    sedef_run_t* raw = nullptr;
    int64_t run_cap = 0;
    unsigned long long* counters = nullptr;  // 32 words, as in the filter
    unsigned int* done = nullptr;
    char* d_up = nullptr;                    // query offsets (2) and window bases (2)
    int state = 0;                           // 0 free, 1 admitted, 2 queued, 3 filtered
    unsigned int epoch = 0;
    int64_t len = 0, nrec = 0, nwin = 0;
    FArgs a;
    // candidates of a finished slot kept until the caller's buffer holds them
    std::vector<sedef_cand_t> fin;
    bool fin_ready = false;
  };
  std::vector<Slot> slots;
  std::vector<void*> dev_allocs;
  std::mutex mu;
};

namespace {

// Shared memory per CTA that other kernels find on an SM beside one k_serve
// CTA: the largest split (228 KB) less k_serve's block and the 1 KB the SM
// reserves for each of the two CTAs.
int64_t server_smem_left() { return 228 * 1024 - (int64_t)sizeof(ServeSmem) - 2 * 1024; }
static_assert(228 * 1024 - sizeof(ServeSmem) - 2 * 1024 >= kTierSmemFloor &&
                  228 * 1024 - sizeof(ServeSmem) - 2 * 1024 >= sizeof(WideMidSmem),
              "the finishing tiers must fit beside k_serve");

int server_alloc(Server* s, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 256) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(SEDEF_ERR_OOM, "server: device allocation failed");
  }
  s->dev_allocs.push_back(*p);
  return SEDEF_OK;
}

// Launches the persistent kernel unless a launch is still running.  Caller
// holds mu.
int server_kick(Server* s) {
  if (s->kern_launched) {
    const cudaError_t q = cudaEventQuery(s->kern_done);
    if (q == cudaErrorNotReady) return SEDEF_OK;
    if (q != cudaSuccess) return cuda_fail(q, "server: kernel event");
  }
  __atomic_store_n(&s->ctl->status, 0, __ATOMIC_RELEASE);
  ServeArgs sv;
  sv.slots = s->d_slots;
  sv.ring = s->d_ring;
  sv.ring_cap = s->ring_cap;
  sv.ctl = s->d_ctl;
  sv.head = s->d_head;
  sv.idle_ns = (unsigned long long)(s->idle_s * 1e9);
  k_serve<<<ctx_sm_count(s->c_prep), kServeTPB, sizeof(ServeSmem), s->s_kern>>>(sv);
  count_launch();
  SEDEF_LAUNCHED("k_serve");
  SEDEF_CUDA(cudaEventRecord(s->kern_done, s->s_kern));
  s->kern_launched = true;
  return SEDEF_OK;
}

// Admission work of one slot on the prep stream: query upload, pack,
// sketch, window table, counters; synchronizes.
int server_prepare(Server* s, Server::Slot& L, const uint8_t* h_query, int64_t len) {
  sedef_ctx* c = s->c_prep;
  cudaStream_t st = s->s_prep;
  ctx_pool_reset(c);
  if (len == 0) {
    L.len = L.nrec = L.nwin = 0;
    return SEDEF_OK;
  }
  SEDEF_CUDA(cudaMemcpyAsync(L.seq, h_query, (size_t)len, cudaMemcpyHostToDevice, st));
  SEDEF_TRY(launch_pack(c, L.seq, len, L.packed, L.mask, L.nbits));
  const int64_t qoff[2] = {0, len};
  int64_t nrec = 0;
  SEDEF_TRY(run_sketch(c, L.packed, L.mask, L.nbits, qoff, 1, s->D, L.qrec, L.rec_cap, &nrec));
  if (nrec > L.rec_cap) return fail(SEDEF_ERR_CAPACITY, "server: sketch exceeds the slot");
  const int64_t nwin = len >= s->D.n ? (len - s->D.n) / s->D.step + 1 : 0;
  const int64_t up[4] = {0, len, 0, nwin};  // query offsets, window bases
  int64_t* h_up = (int64_t*)ctx_host(c, 64);
  if (!h_up) return SEDEF_ERR_OOM;
  std::memcpy(h_up, up, sizeof(up));
  SEDEF_CUDA(cudaMemcpyAsync(L.d_up, h_up, sizeof(up), cudaMemcpyHostToDevice, st));
  SEDEF_CUDA(cudaMemsetAsync(L.counters, 0, 256 + 64, st));
  if (nwin > 0 && nrec > 0)
    SEDEF_KERNEL(c, "k_windows",
                 k_windows<<<(int)((nwin + 255) / 256), 256, 0, st>>>(
                     L.qrec, nrec, (const int64_t*)L.d_up, 1, (const int64_t*)L.d_up + 2, nwin,
                     s->D.step, s->D.span, L.wi, L.wqa, L.wqb, L.wseq, nullptr));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  L.len = len;
  L.nrec = nrec;
  L.nwin = (nrec > 0) ? nwin : 0;
  L.a.qrec = L.qrec;
  L.a.nwin = L.nwin;
  return SEDEF_OK;
}

}  // namespace
}  // namespace sedef

extern "C" {

using sedef::Server;

int sedef_server_destroy(sedef_server* srv) {
  using namespace sedef;
  Server* s = (Server*)srv;
  if (!s) return SEDEF_OK;
  cudaSetDevice(s->device);
  if (s->ctl) {
    __atomic_store_n(&s->ctl->stop, 1, __ATOMIC_RELEASE);
    if (s->kern_launched) cudaEventSynchronize(s->kern_done);
  }
  if (s->s_prep) cudaStreamSynchronize(s->s_prep);
  for (auto& F : s->fins)
    if (F.stream) cudaStreamSynchronize(F.stream);
  if (s->c_prep) sedef_destroy(s->c_prep);
  for (auto& F : s->fins)
    if (F.ctx) sedef_destroy(F.ctx);
  for (void* p : s->dev_allocs) cudaFree(p);
  if (s->ctl) cudaFreeHost(s->ctl);
  if (s->ring) cudaFreeHost(s->ring);
  if (s->kern_done) cudaEventDestroy(s->kern_done);
  if (s->s_prep) cudaStreamDestroy(s->s_prep);
  if (s->s_kern) cudaStreamDestroy(s->s_kern);
  for (auto& F : s->fins)
    if (F.stream) cudaStreamDestroy(F.stream);
  delete s;
  return SEDEF_OK;
}

int sedef_server_create(sedef_ctx* ctx, const uint64_t* d_trec, const uint64_t* d_tsorted,
                        const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                        const sedef_params* p, int32_t slots, int64_t slot_bases,
                        double idle_timeout_s, sedef_server** out) {
  using namespace sedef;
  if (!ctx || !out || !p) return fail(SEDEF_ERR_INVALID, "NULL argument");
  *out = nullptr;
  Derived D;
  SEDEF_TRY(derive(p, &D));
  if (D.self_mode != 0) return fail(SEDEF_ERR_INVALID, "sedef_server_create: self_mode must be 0");
  if (slots < 1 || slots > kServeMaxSlots)
    return fail(SEDEF_ERR_INVALID, "sedef_server_create: slots must be in [1, 64]");
  if (slot_bases < D.n || slot_bases >= (int64_t(1) << 31))
    return fail(SEDEF_ERR_INVALID, "sedef_server_create: slot_bases must be in [n, 2^31)");
  if (!(idle_timeout_s > 0 && idle_timeout_s < 3600))
    return fail(SEDEF_ERR_INVALID, "sedef_server_create: idle timeout must be in (0, 3600) s");
  if (ntseq < 1 || !h_toff || h_toff[0] != 0 || nt < 1 || !d_trec || !d_tsorted || !d_toff)
    return fail(SEDEF_ERR_INVALID, "sedef_server_create: bad target index");
  for (int u = 0; u < ntseq; ++u)
    if (h_toff[u + 1] < h_toff[u]) return fail(SEDEF_ERR_INVALID, "target offsets decrease");
  SEDEF_CUDA(cudaSetDevice(ctx_device(ctx)));
  Server* s = new Server();
  auto bail = [&](int st) {
    const std::string msg = sedef_last_error();
    sedef_server_destroy((sedef_server*)s);
    set_error(msg);
    return st;
  };
  s->device = ctx_device(ctx);
  s->nslots = slots;
  s->slot_bases = slot_bases;
  s->D = D;
  s->P = *p;
  s->idle_s = idle_timeout_s;
  s->trec = d_trec;
  s->tsorted = d_tsorted;
  s->toff = d_toff;
  s->nt = nt;
  s->h_toff.assign(h_toff, h_toff + ntseq + 1);
  s->mtab.resize(kMaxWindowRecs + 1);
  mtable(p, s->mtab.data(), kMaxWindowRecs, nullptr);
  s->fins.resize(kServeFinishers);
  bool made = cudaStreamCreateWithFlags(&s->s_prep, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->s_kern, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->kern_done, cudaEventDisableTiming) == cudaSuccess;
  for (auto& F : s->fins)
    made = made && cudaStreamCreateWithFlags(&F.stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!made) {
    cudaGetLastError();
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: stream or event creation failed"));
  }
  int st = sedef_create(s->device, s->s_prep, &s->c_prep);
  if (st == SEDEF_OK) st = sedef_set_scratch_limit(s->c_prep, ctx_scratch_limit(ctx));
  // admission and finishing run beside the persistent kernel: nothing they
  // allocate may wait for it
  if (st == SEDEF_OK) st = ctx_use_stream_ordered_alloc(s->c_prep);
  for (auto& F : s->fins) {
    if (st == SEDEF_OK) st = sedef_create(s->device, F.stream, &F.ctx);
    if (st == SEDEF_OK) st = sedef_set_scratch_limit(F.ctx, ctx_scratch_limit(ctx));
    if (st == SEDEF_OK) st = ctx_use_stream_ordered_alloc(F.ctx);
    if (st != SEDEF_OK) break;
    ctx_set_filter_variant(F.ctx, ctx_filter_variant(ctx));
    // the finishing tiers keep to the shared memory left beside k_serve
    ctx_set_tier_smem_cap(F.ctx, (size_t)server_smem_left());
  }
  if (st != SEDEF_OK) return bail(st);
  // An SM splits its unified L1 / shared memory when a CTA arrives on an
  // idle SM and keeps the split while any CTA stays.  The persistent kernel
  // stays, so it asks for the largest shared-memory split: the other
  // streams' kernels then find 228 - 63 KB per SM (the large refine kernel
  // takes 125 KB) instead of waiting for the persistent kernel to leave.
  if (cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(ServeSmem)) != cudaSuccess ||
      cudaFuncSetAttribute(k_serve, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: kernel attributes refused"));
  }
  const size_t up = (size_t)(ntseq + 1) * 8 + (size_t)(kMaxWindowRecs + 1) * 4;
  if ((st = server_alloc(s, (void**)&s->d_shared, up)) != SEDEF_OK) return bail(st);
  if (cudaMemcpy(s->d_shared, h_toff, (size_t)(ntseq + 1) * 8, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(s->d_shared + (ntseq + 1) * 8, s->mtab.data(), (size_t)(kMaxWindowRecs + 1) * 4,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: upload failed"));
  s->slots.resize(slots);
  const int64_t win_cap = (slot_bases - D.n) / D.step + 1;
  s->ring_cap = (unsigned long long)(win_cap * slots);
  if (cudaHostAlloc((void**)&s->ctl, sizeof(ServeCtl), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void**)&s->ring, s->ring_cap * sizeof(ServeItem), cudaHostAllocMapped) !=
          cudaSuccess) {
    cudaGetLastError();
    return bail(fail(SEDEF_ERR_OOM, "sedef_server_create: mapped host allocation failed"));
  }
  std::memset(s->ctl, 0, sizeof(ServeCtl));
  if (cudaHostGetDevicePointer((void**)&s->d_ctl, s->ctl, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_ring, s->ring, 0) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: no device view of mapped memory"));
  }
  if ((st = server_alloc(s, (void**)&s->d_head, 8)) != SEDEF_OK) return bail(st);
  if ((st = server_alloc(s, (void**)&s->d_slots, sizeof(SlotDev) * slots)) != SEDEF_OK)
    return bail(st);
  if (cudaMemset(s->d_head, 0, 8) != cudaSuccess)
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: memset failed"));
  std::vector<SlotDev> sdev(slots);
  for (int k = 0; k < slots; ++k) {
    Server::Slot& L = s->slots[k];
    L.rec_cap = slot_bases;
    L.win_cap = win_cap;
    L.run_cap = win_cap * 64 + 4096;
    void* v = nullptr;
#define SALLOC(field, type, bytes)                                   \
  do {                                                               \
    if ((st = server_alloc(s, &v, (size_t)(bytes))) != SEDEF_OK) return bail(st); \
    L.field = (type)v;                                               \
  } while (0)
    SALLOC(seq, uint8_t*, slot_bases);
    SALLOC(packed, uint32_t*, ((slot_bases + 15) / 16) * 4);
    SALLOC(mask, uint32_t*, ((slot_bases + 31) / 32) * 4);
    SALLOC(nbits, uint32_t*, ((slot_bases + 31) / 32) * 4);
    SALLOC(qrec, uint64_t*, L.rec_cap * 8);
    SALLOC(wi, uint32_t*, win_cap * 4 * 7);
    SALLOC(raw, sedef_run_t*, L.run_cap * (int64_t)sizeof(sedef_run_t));
    SALLOC(counters, unsigned long long*, 256 + 64 + 64);
#undef SALLOC
    L.wqa = L.wi + win_cap;
    L.wqb = L.wqa + win_cap;
    L.ov = L.wqb + win_cap;
    L.wl = L.ov + win_cap;
    L.ml = L.wl + win_cap;
    L.wseq = (int32_t*)(L.ml + win_cap);
    L.done = (unsigned int*)((char*)L.counters + 256);
    L.d_up = (char*)L.counters + 256 + 64;
    FArgs& a = L.a;
    std::memset(&a, 0, sizeof(a));
    a.qrec = L.qrec;
    a.trec = d_trec;
    a.tsorted = d_tsorted;
    a.toff = d_toff;
    a.tseq = (const int64_t*)s->d_shared;
    a.qseq = (const int64_t*)L.d_up;
    a.mtab = (const int32_t*)(s->d_shared + (ntseq + 1) * 8);
    a.win_i = L.wi;
    a.win_qa = L.wqa;
    a.win_qb = L.wqb;
    a.win_seq = L.wseq;
    a.ntseq = ntseq;
    a.nqseq = 1;
    a.ttotal = h_toff[ntseq];
    a.k = D.k;
    a.n = D.n;
    a.span = D.span;
    a.max_occ = D.max_occ;
    a.self_mode = 0;
    a.overlap = D.overlap;
    a.runs = L.raw;
    a.nruns = L.counters;
    a.run_cap = L.run_cap;
    a.ov_list = L.ov;
    a.nov = (unsigned int*)(L.counters + 1);
    a.next_window = (unsigned int*)(L.counters + 2);
    a.stats = L.counters + 4;
    sdev[k].a = a;
    sdev[k].done = L.done;
    sdev[k].wide_list = L.wl;
    sdev[k].wide_count = (unsigned int*)(L.counters + 14);
    sdev[k].mid_list = L.ml;
    sdev[k].mid_count = (unsigned int*)(L.counters + 16);
  }
  if (cudaMemcpy(s->d_slots, sdev.data(), sizeof(SlotDev) * slots, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bail(fail(SEDEF_ERR_CUDA, "sedef_server_create: slot table upload failed"));
  *out = (sedef_server*)s;
  return SEDEF_OK;
}

int sedef_server_submit(sedef_server* srv, const uint8_t* h_query, int64_t len, int32_t* slot_out) {
  using namespace sedef;
  Server* s = (Server*)srv;
  if (!s || !slot_out || (len > 0 && !h_query)) return fail(SEDEF_ERR_INVALID, "NULL argument");
  *slot_out = -1;
  if (len < 0 || len > s->slot_bases)
    return fail(SEDEF_ERR_UNSUPPORTED, "sedef_server_submit: query longer than a slot holds");
  SEDEF_CUDA(cudaSetDevice(s->device));
  int k = -1;
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (int x = 0; x < s->nslots && k < 0; ++x)
      if (s->slots[x].state == 0) k = x;
    if (k < 0) return fail(SEDEF_ERR_CAPACITY, "sedef_server_submit: no free slot");
    s->slots[k].state = 1;
  }
  Server::Slot& L = s->slots[k];
  const int st = server_prepare(s, L, h_query, len);
  std::lock_guard<std::mutex> g(s->mu);
  if (st != SEDEF_OK) {
    L.state = 0;
    return st;
  }
  L.epoch += 1;
  *slot_out = k;
  if (L.nwin == 0) {  // nothing to filter: the slot is done at once
    L.state = 3;
    return SEDEF_OK;
  }
  __atomic_store_n(&s->ctl->nwin[k], (long long)L.nwin, __ATOMIC_RELAXED);
  __atomic_store_n(&s->ctl->epoch[k], L.epoch, __ATOMIC_RELAXED);
  for (int64_t w = 0; w < L.nwin; ++w) {
    ServeItem& it = s->ring[(s->tail + (unsigned long long)w) % s->ring_cap];
    it.slot = (uint32_t)k;
    it.window = (uint32_t)w;
  }
  s->tail += (unsigned long long)L.nwin;
  L.state = 2;
  __atomic_store_n(&s->ctl->tail, s->tail, __ATOMIC_RELEASE);  // items before the tail
  return server_kick(s);
}

int sedef_server_poll(sedef_server* srv, double wait_s, int32_t* slot_out) {
  using namespace sedef;
  Server* s = (Server*)srv;
  if (!s || !slot_out) return fail(SEDEF_ERR_INVALID, "NULL argument");
  *slot_out = -1;
  SEDEF_CUDA(cudaSetDevice(s->device));
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      bool queued = false;
      for (int k = 0; k < s->nslots; ++k) {
        Server::Slot& L = s->slots[k];
        if (L.state == 2 &&
            __atomic_load_n(&s->ctl->done_epoch[k], __ATOMIC_ACQUIRE) == L.epoch)
          L.state = 3;
        if (L.state == 3) {
          L.state = 4;  // handed to the caller for sedef_server_finish
          *slot_out = k;
          return SEDEF_OK;
        }
        queued |= L.state == 2;
      }
      // items left behind by a kernel that went idle are served by a new one
      if (queued) SEDEF_TRY(server_kick(s));
    }
    const double el =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= wait_s) return SEDEF_OK;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int sedef_server_finish(sedef_server* srv, int32_t slot, sedef_cand_t* h_cands, int64_t cap,
                        int64_t* h_ncands) {
  using namespace sedef;
  Server* s = (Server*)srv;
  if (!s || !h_ncands || slot < 0 || slot >= (s ? s->nslots : 0))
    return fail(SEDEF_ERR_INVALID, "bad argument");
  *h_ncands = 0;
  Server::Slot& L = s->slots[slot];
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (L.state != 4) return fail(SEDEF_ERR_INVALID, "sedef_server_finish: slot not polled");
  }
  if (L.fin_ready) {  // a second call after SEDEF_ERR_CAPACITY
    *h_ncands = (int64_t)L.fin.size();
    if ((int64_t)L.fin.size() > cap)
      return fail(SEDEF_ERR_CAPACITY, "sedef_server_finish: candidate buffer too small");
    if (!L.fin.empty()) std::memcpy(h_cands, L.fin.data(), L.fin.size() * sizeof(sedef_cand_t));
    L.fin_ready = false;
    std::lock_guard<std::mutex> g(s->mu);
    L.state = 0;
    return SEDEF_OK;
  }
  SEDEF_CUDA(cudaSetDevice(s->device));
  // a free finishing stream and context, held for the whole call
  struct FinLease {
    Server* s;
    Server::Finisher* f = nullptr;
    explicit FinLease(Server* sv) : s(sv) {
      std::unique_lock<std::mutex> g(s->mu);
      s->fin_cv.wait(g, [&] {
        for (auto& F : s->fins)
          if (!F.busy) {
            F.busy = true;
            f = &F;
            return true;
          }
        return false;
      });
    }
    ~FinLease() {
      {
        std::lock_guard<std::mutex> g(s->mu);
        f->busy = false;
      }
      s->fin_cv.notify_one();
    }
  } lease(s);
  sedef_ctx* c = lease.f->ctx;
  cudaStream_t st = lease.f->stream;
  ctx_pool_reset(c);
  auto release = [&](int status) {
    std::lock_guard<std::mutex> g(s->mu);
    L.state = 0;
    return status;
  };
  const int64_t qoff[2] = {0, L.len};
  int64_t nc = 0;
  if (L.nwin > 0) {
    {
      // the windows k_serve handed on for their many hits: the wide tier,
      // as an ordinary launch beside k_serve; what it cannot hold, and what
      // k_serve could not hold, goes through the 8,192-hit wide tier, and
      // what that cannot hold joins the slot's overflow list
      StageScope stage(c, "filter");
      TierIO iow{L.wl, (const unsigned int*)(L.counters + 14), L.ml,
                 (unsigned int*)(L.counters + 16), (unsigned int*)(L.counters + 15), 1};
      int wst = kTierWide(c, L.a, iow, L.nwin, "k_filter_wide");
      TierIO iom{L.ml, (const unsigned int*)(L.counters + 16), L.ov,
                 (unsigned int*)(L.counters + 1), (unsigned int*)(L.counters + 17), 1};
      if (wst == SEDEF_OK) wst = kTierWideMid(c, L.a, iom, L.nwin, "k_filter_widemid");
      if (wst != SEDEF_OK) return release(wst);
    }
    unsigned long long* h_cnt = (unsigned long long*)ctx_host(c, 64);
    if (!h_cnt) return release(SEDEF_ERR_OOM);
    if (cudaMemcpyAsync(h_cnt, L.counters, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return release(fail(SEDEF_ERR_CUDA, "sedef_server_finish: counter copy failed"));
    const int64_t nov = (int64_t)(h_cnt[1] & 0xFFFFFFFFull);
    int64_t slow = 0;
    int status = SEDEF_OK;
    if (nov > 0) status = global_path_eager(c, L.a, nov, L.counters, &slow);
    if (status == SEDEF_OK &&
        (cudaMemcpyAsync(h_cnt, L.counters, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
      status = fail(SEDEF_ERR_CUDA, "sedef_server_finish: counter copy failed");
    if (status != SEDEF_OK) return release(status);
    const int64_t total = (int64_t)h_cnt[0];
    sedef_run_t* runs = nullptr;
    if (total > L.run_cap) {
      // more runs than the slot holds: the whole filter again, sized exactly
      runs = (sedef_run_t*)ctx_alloc(c, (size_t)total * sizeof(sedef_run_t));
      if (!runs) return release(SEDEF_ERR_OOM);
      int64_t got = 0;
      status = run_filter(c, L.qrec, L.nrec, qoff, 1, s->trec, s->tsorted, s->toff, s->nt,
                          s->h_toff.data(), (int)s->h_toff.size() - 1, s->D, s->mtab.data(), runs,
                          total, &got, 0);
      if (status != SEDEF_OK) return release(status);
    } else if (total > 0) {
      runs = (sedef_run_t*)ctx_alloc(c, (size_t)total * sizeof(sedef_run_t));
      if (!runs) return release(SEDEF_ERR_OOM);
      {
        StageScope stage(c, "runsort");
        status = order_and_refine(c, L.a, s->D, 1, (const int64_t*)L.d_up + 2, L.nwin, L.wqa, L.wqb,
                                  L.qrec, L.nrec, s->trec, s->nt, s->toff, L.counters, L.raw, total,
                                  runs, nullptr, nullptr);
      }
      if (status != SEDEF_OK) return release(status);
    }
    if (total > 0) {
      sedef_chain_t* chains = (sedef_chain_t*)ctx_alloc(c, (size_t)total * sizeof(sedef_chain_t));
      if (!chains) return release(SEDEF_ERR_OOM);
      int64_t nch = 0;
      {
        StageScope stage(c, "chain");
        status = run_chain(c, runs, total, L.qrec, L.nrec, qoff, 1, s->tsorted, s->nt, s->toff,
                           s->h_toff.data(), (int)s->h_toff.size() - 1, s->D, s->mtab.data(),
                           chains, total, &nch);
      }
      if (status != SEDEF_OK) return release(status);
      if (nch > 0) {
        sedef_cand_t* cands = (sedef_cand_t*)ctx_alloc(c, (size_t)nch * sizeof(sedef_cand_t));
        if (!cands) return release(SEDEF_ERR_OOM);
        {
          StageScope stage(c, "merge");
          status = run_merge(c, chains, nch, qoff, 1, s->h_toff.data(),
                             (int)s->h_toff.size() - 1, s->D, cands, nch, &nc);
        }
        if (status != SEDEF_OK) return release(status);
        if (nc > cap) {  // keep them for the next call; the slot stays handed out
          L.fin.resize((size_t)nc);
          if (cudaMemcpyAsync(L.fin.data(), cands, (size_t)nc * sizeof(sedef_cand_t),
                              cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaStreamSynchronize(st) != cudaSuccess)
            return release(fail(SEDEF_ERR_CUDA, "sedef_server_finish: copy failed"));
          L.fin_ready = true;
          *h_ncands = nc;
          return fail(SEDEF_ERR_CAPACITY, "sedef_server_finish: candidate buffer too small");
        }
        if (nc > 0 &&
            cudaMemcpyAsync(h_cands, cands, (size_t)nc * sizeof(sedef_cand_t),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return release(fail(SEDEF_ERR_CUDA, "sedef_server_finish: copy failed"));
      }
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess)
    return release(fail(SEDEF_ERR_CUDA, "sedef_server_finish: stream failed"));
  *h_ncands = nc;
  return release(SEDEF_OK);
}

int sedef_server_smem_left(sedef_server* srv, int64_t* bytes) {
  if (!srv || !bytes) return sedef::fail(SEDEF_ERR_INVALID, "NULL argument");
  *bytes = sedef::server_smem_left();
  return SEDEF_OK;
}

int sedef_server_status(sedef_server* srv, int32_t* running, int32_t* timed_out) {
  using namespace sedef;
  Server* s = (Server*)srv;
  if (!s) return fail(SEDEF_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  int run = 0;
  if (s->kern_launched) {
    const cudaError_t q = cudaEventQuery(s->kern_done);
    if (q == cudaErrorNotReady) run = 1;
    else if (q != cudaSuccess) return cuda_fail(q, "server: kernel event");
  }
  const int tmo = __atomic_load_n(&s->ctl->status, __ATOMIC_ACQUIRE) == SEDEF_ERR_TIMEOUT;
  if (running) *running = run;
  if (timed_out) *timed_out = tmo;
  return (!run && tmo) ? SEDEF_ERR_TIMEOUT : SEDEF_OK;
}

}  // extern "C"
