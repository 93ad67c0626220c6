// a4-a6: candidate lookup, sliding shared-minimizer count against m(s), and
// the winnowed MinHash refine (Sections 2.2 and 3.1).
//
// Fast path (one CTA of 128 threads per query window, persistent CTAs):
//   1. the window's query minimizers are sorted by hash in shared memory and
//      deduplicated into W_Q (s hashes, each with its strand set);
//   2. every posting of every hash of W_Q is a hit (t, hid, o).  Hits are
//      counted into direct-mapped 16-bit counters keyed by (t >> 10, o):
//      a target window [j, j+n-k] lies inside bins j>>10 and (j>>10)+1, so a
//      j can only pass when those two counters sum to m or more (aliasing
//      only adds false candidates);
//   3. hits whose bin pair can pass are collected and sorted by (o, t); the
//      exact sweep (one thread, per-hash counters) runs only over j ranges
//      where m consecutive hits fit in n-k bases.  Any j whose true count
//      reaches m has all of its hits collected, and a count computed from a
//      subset never exceeds the true one, so the runs are exact.
// Windows that exceed the fast path's shared-memory budget go to a slow path
// that writes their hits to global memory, radix-sorts them by
// (window, o, t) and runs the same sweep.
//
// Refine (one warp per run): the domain W_Q u (target minimizers of the
// run's span) is sorted; presence and sharedness are kept as counters and
// bitsets while the target window rolls over the run's breakpoints, and the
// estimate |S(W_Q u W_T) n W_Q n W_T| is read off the first s set bits.
#include <cstring>

#include "common.cuh"

namespace sedef {

namespace {

constexpr int kFThreads = 128;
constexpr int kQCap = 256;        // query records per window (fast path)
constexpr int kBinShift = 10;     // 1024-base bins (>= n - k + 1)
constexpr int kSlots = 2048;      // (bin, o) counters (16-bit)
constexpr int kLCap = 1024;       // collected hits (fast path)
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
};

// ----------------------------------------------------------- run emission --

struct RunState {
  bool open;
  int64_t ja, jb, jmx;
  int mx;
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
    const int u = seq_of(a.tseq, a.ntseq, x);
    const int64_t st = a.tseq[u], en = a.tseq[u + 1];
    int64_t lo = st, hi = en - a.n;
    bool ok = true;
    if (a.self_mode) {
      if (u < w.qseq) ok = false;
      else if (u == w.qseq) lo = max(lo, w.i + a.n - a.overlap);
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

// Exact sweep over one strand's hits, sorted by t.  get(x) returns the hit's
// (t, hid).  cnt[] holds one zeroed counter per hash id and is zero again on
// return.
template <typename Get>
__device__ void sweep(const FArgs& a, WinInfo w, Get get, int64_t L, uint16_t* cnt) {
  const int m = w.m, span = a.span;
  RunState r;
  r.open = false;
  int64_t gl = 0, gh = -1;
  bool have = false;
  auto process = [&](int64_t Jlo, int64_t Jhi) {
    // first hit with t >= Jlo
    int64_t lo = 0, hi = L;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
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
    // a count below m ends any run at the group's end (the next group is
    // separated by j values that cannot pass)
    segment(a, w, r, Jhi + 1, Jhi + 1, 0);
  };
  for (int64_t x = 0; x + m - 1 < L; ++x) {
    const int64_t ta = get(x).x, tb = get(x + m - 1).x;
    if (tb - ta > span) continue;
    const int64_t jlo = tb - span, jhi = ta;
    if (have && jlo <= gh + 1) {
      if (jhi > gh) gh = jhi;
    } else {
      if (have) process(gl, gh);
      have = true;
      gl = jlo;
      gh = jhi;
    }
  }
  if (have) process(gl, gh);
  emit_run(a, w, r);
}

// ------------------------------------------------------ block bitonic sort --

template <typename T>
__device__ void block_sort(T* v, int n) {  // n a power of two
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int lo = 2 * stride * (t / stride) + (t % stride);
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

__device__ int build_wq(const FArgs& a, QBuild q, int c) {
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

// ------------------------------------------------------------- fast path --

struct FastSmem {
  uint32_t qkey[kQCap];
  uint32_t dh[kQCap];
  uint32_t pst[kQCap];
  uint32_t plen[kQCap];
  uint32_t pre[kQCap + 1];
  uint8_t dm[kQCap];
  uint32_t slots[kSlots / 2];  // two 16-bit counters per word
  unsigned long long hits[kLCap];
  uint16_t cnt[kQCap];
  int tmp[33];
  int64_t win;
  int nhit, s, ovf;
};

__device__ __forceinline__ uint32_t slot_of(uint32_t t, uint32_t o) {
  return (((t >> kBinShift) << 1) | o) & (kSlots - 1);
}

__device__ __forceinline__ uint32_t slot_count(const uint32_t* slots, uint32_t s) {
  return (slots[s >> 1] >> ((s & 1) * 16)) & 0xFFFFu;
}

// Enumerates the window's hits: calls f(t, hid, o) for every posting of every
// kept hash with a compatible relative strand (self positions skipped).
template <typename F>
__device__ __forceinline__ void for_hits(const FArgs& a, const FastSmem& S, int64_t i, int H, F f) {
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

__global__ void __launch_bounds__(kFThreads) k_filter_fast(FArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FastSmem& S = *reinterpret_cast<FastSmem*>(smem_raw);
  for (int x = threadIdx.x; x < kQCap; x += blockDim.x) S.cnt[x] = 0;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) S.win = atomicAdd(a.next_window, 1u);
    __syncthreads();
    const int64_t wdx = S.win;
    if (wdx >= a.nwin) break;
    const int64_t i = a.win_i[wdx];
    const uint32_t qa = a.win_qa[wdx], qb = a.win_qb[wdx];
    const int c = (int)(qb - qa);
    if (c == 0) continue;
    if (c > kQCap) {
      if (threadIdx.x == 0) a.ov_list[atomicAdd(a.nov, 1u)] = (uint32_t)wdx;
      continue;
    }
    for (int x = threadIdx.x; x < c; x += blockDim.x) {
      const uint64_t r = __ldg(a.qrec + qa + x);
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
    const int s = build_wq(a, qb_, c);
    if (s == 0) continue;
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
    for (int x = threadIdx.x; x < kSlots / 2; x += blockDim.x) S.slots[x] = 0;
    if (threadIdx.x == 0) {
      S.s = s;
      S.nhit = 0;
      S.ovf = 0;
    }
    __syncthreads();
    const uint32_t H = S.pre[s];
    if (H == 0) continue;
    if (H > (uint32_t)kHMax) {
      if (threadIdx.x == 0) a.ov_list[atomicAdd(a.nov, 1u)] = (uint32_t)wdx;
      continue;
    }
    const int m = a.mtab[s];
    // pass 1: (bin, o) counts
    for_hits(a, S, i, (int)H, [&](uint32_t t, uint32_t, uint32_t o) {
      const uint32_t sl = slot_of(t, o);
      atomicAdd(&S.slots[sl >> 1], 1u << ((sl & 1) * 16));
    });
    __syncthreads();
    // pass 2: collect the hits of bins whose pair (b, b+1) or (b-1, b) may pass
    for_hits(a, S, i, (int)H, [&](uint32_t t, uint32_t hid, uint32_t o) {
      const uint32_t b = t >> kBinShift;
      const uint32_t c0 = slot_count(S.slots, slot_of(t, o));
      const uint32_t cn = slot_count(S.slots, (((b + 1) << 1) | o) & (kSlots - 1));
      bool need = c0 + cn >= (uint32_t)m;
      if (!need && b > 0) {
        const uint32_t cp = slot_count(S.slots, (((b - 1) << 1) | o) & (kSlots - 1));
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
      if (threadIdx.x == 0) a.ov_list[atomicAdd(a.nov, 1u)] = (uint32_t)wdx;
      continue;
    }
    if (L < m) continue;
    const int np = next_pow2(L < 2 ? 2 : L);
    for (int x = L + threadIdx.x; x < np; x += blockDim.x) S.hits[x] = ~0ull;
    __syncthreads();
    block_sort(S.hits, np);
    if (threadIdx.x == 0) {
      WinInfo w;
      w.i = i;
      w.qseq = a.win_seq[wdx];
      w.s = s;
      w.m = m;
      int split = 0;
      while (split < L && (S.hits[split] >> 63) == 0) ++split;
      for (int o = 0; o < 2; ++o) {
        w.o = o;
        const unsigned long long* base = S.hits + (o ? split : 0);
        const int64_t cnt = o ? L - split : split;
        sweep(a, w,
              [&](int64_t x) {
                const unsigned long long h = base[x];
                return make_uint2((uint32_t)(h >> 20), (uint32_t)(h & 0xFFFFFu));
              },
              cnt, S.cnt);
      }
    }
  }
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
  return build_wq(a, q, c);
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

__global__ void __launch_bounds__(kSThreads) k_slow_count(FArgs a, int64_t nov,
                                                          unsigned long long* counts, int32_t* s_out) {
  __shared__ SlowSmem S;
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
      counts[v] = S.acc;
      s_out[v] = s;
    }
  }
}

// Writes keys (local window << 33 | o << 32 | t) and hash ids for windows
// [v0, v1) of the overflow list at offsets base[v] - base[v0].
__global__ void __launch_bounds__(kSThreads) k_slow_emit(FArgs a, int64_t v0, int64_t v1,
                                                         const unsigned long long* base,
                                                         uint64_t* keys, uint32_t* vals) {
  __shared__ SlowSmem S;
  __shared__ unsigned long long cursor;
  for (int64_t v = v0 + blockIdx.x; v < v1; v += gridDim.x) {
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

__global__ void __launch_bounds__(32) k_slow_sweep(FArgs a, int64_t v0, int64_t v1,
                                                   const unsigned long long* base,
                                                   const int32_t* s_of, const uint64_t* keys,
                                                   const uint32_t* vals) {
  __shared__ uint16_t cnt[kMaxWindowRecs];
  for (int x = threadIdx.x; x < kMaxWindowRecs; x += blockDim.x) cnt[x] = 0;
  __syncwarp();
  if (threadIdx.x != 0) return;
  for (int64_t v = v0 + blockIdx.x; v < v1; v += gridDim.x) {
    const int64_t wdx = a.ov_list[v];
    const int s = s_of[v];
    if (s == 0) continue;
    WinInfo w;
    w.i = a.win_i[wdx];
    w.qseq = a.win_seq[wdx];
    w.s = s;
    w.m = a.mtab[s];
    const int64_t lo = (int64_t)(base[v] - base[v0]), hi = (int64_t)(base[v + 1] - base[v0]);
    int64_t split = lo;
    {
      int64_t l = lo, h = hi;
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (((keys[mid] >> 32) & 1u) == 0) l = mid + 1; else h = mid;
      }
      split = l;
    }
    for (int o = 0; o < 2; ++o) {
      w.o = o;
      const int64_t b = o ? split : lo, e = o ? hi : split;
      sweep(a, w,
            [&](int64_t x) { return make_uint2((uint32_t)keys[b + x], vals[b + x]); },
            e - b, cnt);
    }
  }
}

// ---------------------------------------------------------- window table --

__global__ void k_windows(const uint64_t* __restrict__ qrec, int64_t nq,
                          const int64_t* __restrict__ qseq, int nqseq,
                          const int64_t* __restrict__ wbase, int64_t nwin, int step, int span,
                          uint32_t* wi, uint32_t* wqa, uint32_t* wqb, int32_t* wseq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwin) return;
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

__global__ void k_run_keys(const sedef_run_t* runs, int64_t n, uint64_t* keys) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) keys[x] = ((uint64_t)runs[x].i << 1) | runs[x].o;
}

__global__ void k_gather_runs(const sedef_run_t* in, const uint32_t* perm, int64_t n, sedef_run_t* out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) out[x] = in[perm[x]];
}

// ----------------------------------------------------------------- refine --

constexpr int kRWarps = 4;
constexpr int kDCap = 2048;   // domain: |W_Q| + span records of one piece
constexpr int kRCap = 1024;   // span records per piece

struct RefineWarp {
  uint32_t dom[kDCap];       // sorted distinct hashes (W_Q u span)
  uint16_t cntT[kDCap];      // records of this hash in the target window
  uint16_t cntS[kDCap];      // shared-compatible records of this hash in the window
  uint32_t pb[kDCap / 32];   // present: in W_Q or cntT > 0
  uint32_t sb[kDCap / 32];   // shared: cntS > 0
  uint32_t tpos[kRCap];      // span record positions (sorted)
  uint16_t tdx[kRCap];       // domain index of each span record
  uint8_t tsh[kRCap];        // record is shared-compatible
  uint8_t qm[kDCap];         // strand mask for W_Q members (0 = not in W_Q)
};

__device__ __forceinline__ void warp_sort_u32(uint32_t* v, int n) {  // n power of two
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane_id(); t < (n >> 1); t += 32) {
        const int lo = 2 * stride * (t / stride) + (t % stride);
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

// Estimate from the bitsets: shared bits among the first s present bits.
__device__ __forceinline__ int estimate(const RefineWarp& R, int nwords, int s) {
  const int lane = lane_id();
  const uint32_t p0 = (2 * lane < nwords) ? R.pb[2 * lane] : 0u;
  const uint32_t p1 = (2 * lane + 1 < nwords) ? R.pb[2 * lane + 1] : 0u;
  const uint32_t s0 = (2 * lane < nwords) ? R.sb[2 * lane] : 0u;
  const uint32_t s1 = (2 * lane + 1 < nwords) ? R.sb[2 * lane + 1] : 0u;
  const int pc = __popc(p0) + __popc(p1);
  const int inc = warp_inclusive_sum(pc);
  const int before = inc - pc;
  // lane holding the s-th present bit
  const unsigned owner = __ballot_sync(0xffffffffu, before < s && inc >= s);
  const int ol = __ffs(owner) - 1;
  int est_full = (inc <= s) ? (__popc(s0) + __popc(s1)) : 0;  // lanes entirely inside
  int part = 0;
  if (lane == ol) {
    int need = s - before;  // present bits to take from this lane's 64
    uint32_t words_p[2] = {p0, p1}, words_s[2] = {s0, s1};
    for (int x = 0; x < 2 && need > 0; ++x) {
      const int c = __popc(words_p[x]);
      if (c <= need) {
        part += __popc(words_s[x]);
        need -= c;
      } else {
        // position of the need-th set bit (1-based) of words_p[x]
        uint32_t wv = words_p[x];
        for (int y = 1; y < need; ++y) wv &= wv - 1u;
        const int b = __ffs(wv) - 1;
        const uint32_t below = (b >= 31) ? 0xFFFFFFFFu : ((2u << b) - 1u);
        part += __popc(words_s[x] & below);
        need = 0;
      }
    }
    est_full = 0;
  }
  return warp_sum(est_full + part);
}

struct RefineArgs {
  sedef_run_t* runs;
  int64_t nruns;
  const uint64_t* qrec;
  int64_t nq;
  const uint64_t* trec;
  int64_t nt;
  const uint32_t* toff;
  const int32_t* mtab;
  int span, max_occ, self_mode;
};

__global__ void __launch_bounds__(32 * kRWarps) k_refine(RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  RefineWarp& R = reinterpret_cast<RefineWarp*>(smem_raw)[warp];
  auto pos_of = [](uint64_t r) { return (uint64_t)((r >> 1) & 0xFFFFFFFFull); };
  for (int64_t ri = (int64_t)blockIdx.x * kRWarps + warp; ri < a.nruns;
       ri += (int64_t)gridDim.x * kRWarps) {
    sedef_run_t run = a.runs[ri];
    const int64_t i = run.i, ja = run.j_a, jb = run.j_b;
    const int o = run.o;
    // ---- W_Q: sorted hashes with strand masks (capped hashes dropped)
    int64_t qa = 0, qb = 0;
    if (lane == 0) {
      qa = lower_bound_by(a.qrec, 0, a.nq, (uint64_t)i, pos_of);
      qb = lower_bound_by(a.qrec, qa, a.nq, (uint64_t)(i + a.span + 1), pos_of);
    }
    qa = __shfl_sync(0xffffffffu, qa, 0);
    qb = __shfl_sync(0xffffffffu, qb, 0);
    const int c = (int)(qb - qa);
    const int npq = next_pow2(c < 2 ? 2 : c);
    for (int x = lane; x < npq; x += 32) {
      uint32_t key = kNone;
      if (x < c) {
        const uint64_t r = a.qrec[qa + x];
        key = (rec_hash(r) << 1) | rec_strand(r);
      }
      R.dom[x] = key;  // temporary use of dom as the sort buffer
    }
    __syncwarp();
    warp_sort_u32(R.dom, npq);
    // compact to distinct kept hashes in tpos (temporary) with masks in tsh
    int s = 0;
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
        R.tpos[d] = h;
        R.tsh[d] = (uint8_t)mask;
      }
      s += __popc(bal);
    }
    __syncwarp();
    // ---- pieces of the run: span records [P_lo, P_hi + span] <= kRCap
    int best = -1, den = 0;
    int64_t jstar = ja;
    // keep W_Q (hash, mask) in registers-by-stride: copy to the tail of dom later
    // (W_Q has s <= 1024 entries, stored in tpos/tsh until the domain is built)
    __shared__ uint32_t wq_h[kRWarps][kMaxWindowRecs];
    __shared__ uint8_t wq_m[kRWarps][kMaxWindowRecs];
    for (int x = lane; x < s; x += 32) {
      wq_h[warp][x] = R.tpos[x];
      wq_m[warp][x] = R.tsh[x];
    }
    __syncwarp();
    int64_t plo = ja;
    int64_t rlo = 0;
    if (lane == 0) rlo = lower_bound_by(a.trec, 0, a.nt, (uint64_t)ja, pos_of);
    rlo = __shfl_sync(0xffffffffu, rlo, 0);
    while (plo <= jb) {
      // records of the piece: [rlo, rhi) with pos <= P_hi + span, at most kRCap
      int64_t rcap_end = rlo + kRCap < a.nt ? rlo + kRCap : a.nt;
      int64_t phi = jb;
      int64_t rhi = 0;
      if (lane == 0) {
        rhi = lower_bound_by(a.trec, rlo, a.nt, (uint64_t)(jb + a.span + 1), pos_of);
        if (rhi > rcap_end) {
          // shrink the piece so that its records fit: P_hi + span < pos of
          // the first record that does not fit
          const int64_t lim = (int64_t)pos_of(a.trec[rcap_end]);
          phi = lim - a.span - 1;
          rhi = lower_bound_by(a.trec, rlo, a.nt, (uint64_t)(phi + a.span + 1), pos_of);
        }
      }
      phi = __shfl_sync(0xffffffffu, phi, 0);
      rhi = __shfl_sync(0xffffffffu, rhi, 0);
      const int nr = (int)(rhi - rlo);
      // ---- domain: sort W_Q hashes u record hashes
      const int nd0 = s + nr;
      const int npd = next_pow2(nd0 < 2 ? 2 : nd0);
      for (int x = lane; x < npd; x += 32) {
        uint32_t v = kNone;
        if (x < s) v = wq_h[warp][x];
        else if (x < nd0) v = rec_hash(a.trec[rlo + (x - s)]);
        R.dom[x] = v;
      }
      __syncwarp();
      warp_sort_u32(R.dom, npd);
      // dedup in place (warp compaction in order)
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
      const int nwords = (D + 31) >> 5;
      for (int x = lane; x < D; x += 32) {
        R.cntT[x] = 0;
        R.cntS[x] = 0;
        R.qm[x] = 0;
      }
      for (int x = lane; x < kDCap / 32; x += 32) {
        R.pb[x] = 0;
        R.sb[x] = 0;
      }
      __syncwarp();
      for (int x = lane; x < s; x += 32) {
        const int d = dom_find(R.dom, D, wq_h[warp][x]);
        R.qm[d] = wq_m[warp][x];
        atomicOr(&R.pb[d >> 5], 1u << (d & 31));
      }
      __syncwarp();
      for (int x = lane; x < nr; x += 32) {
        const uint64_t r = a.trec[rlo + x];
        const uint32_t t = rec_pos(r), st = rec_strand(r);
        const int d = dom_find(R.dom, D, rec_hash(r));
        R.tpos[x] = t;
        R.tdx[x] = (uint16_t)d;
        const bool self = a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span;
        R.tsh[x] = (!self && ((R.qm[d] >> (st ^ (uint32_t)o)) & 1u)) ? 1 : 0;
      }
      __syncwarp();
      // ---- roll the target window over [plo, phi]
      int e = 0, l = 0;
      int64_t j = plo;
      auto enter = [&](int x) {
        const int d = R.tdx[x];
        if (R.cntT[d]++ == 0) atomicOr(&R.pb[d >> 5], 1u << (d & 31));
        if (R.tsh[x] && R.cntS[d]++ == 0) atomicOr(&R.sb[d >> 5], 1u << (d & 31));
      };
      auto leave = [&](int x) {
        const int d = R.tdx[x];
        if (--R.cntT[d] == 0 && R.qm[d] == 0) atomicAnd(&R.pb[d >> 5], ~(1u << (d & 31)));
        if (R.tsh[x] && --R.cntS[d] == 0) atomicAnd(&R.sb[d >> 5], ~(1u << (d & 31)));
      };
      if (lane == 0) {
        while (l < nr && (int64_t)R.tpos[l] < j) ++l;
        e = l;
        while (e < nr && (int64_t)R.tpos[e] <= j + a.span) enter(e++);
      }
      __syncwarp();
      while (true) {
        const int est = estimate(R, nwords, s);
        if (est > best) {
          best = est;
          jstar = j;
          den = s;
        }
        int64_t nx = 0;
        if (lane == 0) {
          const int64_t ne = e < nr ? (int64_t)R.tpos[e] - a.span : INT64_MAX;
          const int64_t nl = l < e ? (int64_t)R.tpos[l] + 1 : INT64_MAX;
          nx = min(ne, nl);
          if (nx <= phi) {
            while (l < e && (int64_t)R.tpos[l] + 1 <= nx) leave(l++);
            while (e < nr && (int64_t)R.tpos[e] - a.span <= nx) enter(e++);
          }
        }
        nx = __shfl_sync(0xffffffffu, nx, 0);
        __syncwarp();
        if (nx > phi) break;
        j = nx;
      }
      plo = phi + 1;
      if (plo <= jb) {
        if (lane == 0) rlo = lower_bound_by(a.trec, rlo, a.nt, (uint64_t)plo, pos_of);
        rlo = __shfl_sync(0xffffffffu, rlo, 0);
      }
    }
    if (lane == 0) {
      sedef_run_t& out = a.runs[ri];
      out.est = (uint16_t)best;
      out.den = (uint16_t)den;
      out.j_star = (uint32_t)jstar;
      out.keep = (best >= a.mtab[den]) ? 1 : 0;
    }
    __syncwarp();
  }
}

}  // namespace

int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total);

int run_filter(sedef_ctx* ctx, const uint64_t* qrec, int64_t nq, const int64_t* h_qoff, int nqseq,
               const uint64_t* trec, const uint64_t* tsorted, const uint32_t* toff, int64_t nt,
               const int64_t* h_toff, int ntseq, const Derived& D, const int32_t* h_mtab,
               sedef_run_t* runs, int64_t cap, int64_t* nruns) {
  cudaStream_t st = ctx_stream(ctx);
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
  char* h_up = (char*)ctx_host(ctx, up_bytes + 64);
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
  unsigned long long* counters = (unsigned long long*)ctx_alloc(ctx, 64);
  sedef_run_t* raw = (sedef_run_t*)ctx_alloc(ctx, (size_t)(cap > 0 ? cap : 1) * sizeof(sedef_run_t));
  if (!wi || !wqa || !wqb || !wseq || !ovl || !counters || !raw) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemsetAsync(counters, 0, 64, st));

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

  SEDEF_KERNEL(ctx, "k_windows",
               k_windows<<<(int)((nwin + 255) / 256), 256, 0, st>>>(
                   qrec, nq, a.qseq, nqseq, (const int64_t*)(d_up + ow), nwin, D.step, D.span, wi,
                   wqa, wqb, wseq));
  static bool attr = false;
  const size_t fsm = sizeof(FastSmem);
  if (!attr) {
    SEDEF_CUDA(cudaFuncSetAttribute(k_filter_fast, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)fsm));
    SEDEF_CUDA(cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(RefineWarp) * kRWarps)));
    attr = true;
  }
  int per_sm = 0;
  SEDEF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_fast, kFThreads, fsm));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx_sm_count(ctx) * per_sm;
  if (grid > nwin) grid = nwin;
  SEDEF_KERNEL(ctx, "k_filter_fast", k_filter_fast<<<(int)grid, kFThreads, fsm, st>>>(a));

  unsigned long long* h_cnt = (unsigned long long*)ctx_host(ctx, 64);
  if (!h_cnt) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemcpyAsync(h_cnt, counters, 16, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  const int64_t nov = (int64_t)(h_cnt[1] & 0xFFFFFFFFull);

  if (nov > 0) {
    // slow path: count, then batches of emit -> sort -> sweep
    unsigned long long* ocnt = (unsigned long long*)ctx_alloc(ctx, (size_t)(nov + 1) * 8);
    int32_t* os = (int32_t*)ctx_alloc(ctx, (size_t)(nov + 1) * 4);
    if (!ocnt || !os) return SEDEF_ERR_OOM;
    int64_t sgrid = nov < (int64_t)ctx_sm_count(ctx) * 4 ? nov : (int64_t)ctx_sm_count(ctx) * 4;
    SEDEF_KERNEL(ctx, "k_slow_count", k_slow_count<<<(int)sgrid, kSThreads, 0, st>>>(a, nov, ocnt, os));
    std::vector<unsigned long long> hc(nov + 1, 0);
    SEDEF_CUDA(cudaMemcpyAsync(hc.data(), ocnt, (size_t)nov * 8, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
    std::vector<unsigned long long> base(nov + 1, 0);
    for (int64_t v = 0; v < nov; ++v) base[v + 1] = base[v] + hc[v];
    unsigned long long* d_base = (unsigned long long*)ctx_alloc(ctx, (size_t)(nov + 1) * 8);
    if (!d_base) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(d_base, base.data(), (size_t)(nov + 1) * 8, cudaMemcpyHostToDevice, st));
    const unsigned long long budget = 1ull << 27;  // hits per batch
    int64_t v0 = 0;
    while (v0 < nov) {
      int64_t v1 = v0 + 1;
      while (v1 < nov && base[v1 + 1] - base[v0] <= budget && v1 - v0 < (1 << 20)) ++v1;
      const unsigned long long nh = base[v1] - base[v0];
      if (nh > 0) {
        uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)nh * 8);
        uint32_t* vals = (uint32_t*)ctx_alloc(ctx, (size_t)nh * 4);
        uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)nh * 8);
        uint32_t* svals = (uint32_t*)ctx_alloc(ctx, (size_t)nh * 4);
        if (!keys || !vals || !skeys || !svals) return SEDEF_ERR_OOM;
        const int64_t nb = v1 - v0;
        int g = (int)(nb < (int64_t)ctx_sm_count(ctx) * 4 ? nb : (int64_t)ctx_sm_count(ctx) * 4);
        SEDEF_KERNEL(ctx, "k_slow_emit",
                     k_slow_emit<<<g, kSThreads, 0, st>>>(a, v0, v1, d_base, keys, vals));
        int wbits = 0;
        while ((int64_t(1) << wbits) < nb) ++wbits;
        SEDEF_TRY(radix_sort_u64(ctx, keys, vals, skeys, svals, (int64_t)nh, 0, 33 + wbits));
        int g2 = (int)(nb < (int64_t)ctx_sm_count(ctx) * 16 ? nb : (int64_t)ctx_sm_count(ctx) * 16);
        SEDEF_KERNEL(ctx, "k_slow_sweep",
                     k_slow_sweep<<<g2, 32, 0, st>>>(a, v0, v1, d_base, os, skeys, svals));
        SEDEF_CUDA(cudaStreamSynchronize(st));
      }
      v0 = v1;
    }
    SEDEF_CUDA(cudaMemcpyAsync(h_cnt, counters, 8, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
  }
  const int64_t total = (int64_t)h_cnt[0];
  *nruns = total;
  if (total > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_filter: run buffer too small");
  if (total == 0) return SEDEF_OK;
  // order runs by (i, o); the sweep emits each window's runs in j order
  uint64_t* keys = (uint64_t*)ctx_alloc(ctx, (size_t)total * 8);
  uint64_t* skeys = (uint64_t*)ctx_alloc(ctx, (size_t)total * 8);
  uint32_t* perm = (uint32_t*)ctx_alloc(ctx, (size_t)total * 4);
  if (!keys || !skeys || !perm) return SEDEF_ERR_OOM;
  const int tb = (int)((total + 255) / 256);
  SEDEF_KERNEL(ctx, "k_run_keys", k_run_keys<<<tb, 256, 0, st>>>(raw, total, keys));
  int hb = 1;
  while ((int64_t(1) << hb) <= (a.ttotal > h_qoff[nqseq] ? a.ttotal : h_qoff[nqseq])) ++hb;
  SEDEF_TRY(radix_sort_u64(ctx, keys, nullptr, skeys, perm, total, 0, hb + 1));
  SEDEF_KERNEL(ctx, "k_gather_runs", k_gather_runs<<<tb, 256, 0, st>>>(raw, perm, total, runs));
  // refine
  RefineArgs ra;
  ra.runs = runs;
  ra.nruns = total;
  ra.qrec = qrec;
  ra.nq = nq;
  ra.trec = trec;
  ra.nt = nt;
  ra.toff = toff;
  ra.mtab = a.mtab;
  ra.span = D.span;
  ra.max_occ = D.max_occ;
  ra.self_mode = D.self_mode;
  int rper = 0;
  SEDEF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, k_refine, 32 * kRWarps,
                                                           sizeof(RefineWarp) * kRWarps));
  if (rper < 1) rper = 1;
  int64_t rgrid = (total + kRWarps - 1) / kRWarps;
  if (rgrid > (int64_t)ctx_sm_count(ctx) * rper) rgrid = (int64_t)ctx_sm_count(ctx) * rper;
  SEDEF_KERNEL(ctx, "k_refine",
               k_refine<<<(int)rgrid, 32 * kRWarps, sizeof(RefineWarp) * kRWarps, st>>>(ra));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // namespace sedef
