// f1: SD extension -- seeds grown into potential SD regions (Section 3.2).
//
// Every kept seed (i, j*, o) starts as the query region [i, i+n) and the
// target region [j*, j*+n).  Both grow by one base per step (the target at
// the opposite end when o = 1), forward first and then backward, while the
// winnowed MinHash estimate of the two regions stays >= tau: W_Q and W_T are
// the minimizers of the extension sketch (all k-mers, masked ones included)
// whose k-mer lies in the region, s = |W_Q|, U = the s smallest hashes of
// W_Q u W_T, est = the hashes of U that occur in both with relative strand o,
// and a step is kept while est >= m(s).  Growth also stops at a sequence
// end, at max_len bases, and (a self search on one sequence) where the two
// regions would overlap more than before.  In a self search a target
// minimizer inside the query region's k-mer span is the same position, not a
// copy: it is never shared (its hash is in W_Q already, so the union does
// not change).
//
// One warp per seed (persistent, work counter over the kept seeds).  The
// union lives in a per-warp table of 4-bit states, one per hash: bits 0-1
// the query strands, bits 2-3 the shareable target strands; a hash is in the
// union when its state is non-zero.  A shared-memory summary marks the
// 256-hash blocks that hold a member.  The warp keeps theta (the s-th
// smallest member), the number of members <= theta and est exactly as
// minimizers join, so each step costs O(1) table accesses plus the scans
// that move theta to the neighbouring member.  Between two steps that add a
// minimizer the estimate cannot change, so the walk jumps from one such
// step to the next.  A step whose estimate falls below m(s) is taken back.
#include <cstring>

#include "common.cuh"

namespace sedef {
namespace {

constexpr int kExtWarps = 4;        // warps per CTA
constexpr int kExtInit = 2048;      // initial union bound: 2 (n - k + 1) <= 2048

struct ExtArgs {
  const sedef_run_t* runs;
  const uint32_t* kept;   // run index of each kept seed
  int64_t nkept;
  const uint64_t* qrec;   // extension sketch of the query, by position
  int64_t nq;
  const uint64_t* trec;   // extension sketch of the target, by position
  int64_t nt;
  const int64_t* qoff;
  int nqseq;
  const int64_t* toff;
  int ntseq;
  const int32_t* mtab;    // m(s) for s in [0, smax]
  int64_t smax;
  int k, n, self_mode;
  int64_t max_len;
  uint32_t* nib;          // per warp: nib_words words of 4-bit states
  int64_t nib_words;
  int sum_words;          // per warp: summary words (one bit per 256 hashes)
  int64_t nblocks;
  unsigned int* next;     // work counter
  sedef_region_t* out;
};

struct ExtSmem {
  uint32_t init[kExtInit];
};

__device__ __forceinline__ bool shareable(uint32_t v, int o) {
  const uint32_t q = v & 3u, t = (v >> 2) & 3u;
  const uint32_t to = o ? (((t & 1u) << 1) | (t >> 1)) : t;
  return (q & to) != 0u;
}

// One warp's view of its tables.  All lanes hold the same scalars.
struct Ext {
  const ExtArgs* a;
  uint32_t* nib;
  uint32_t* sum;
  int o;
  int64_t s, cnt, est, theta;  // theta = -1: no member counted yet

  __device__ uint32_t state(int64_t h) const {
    return (nib[h >> 3] >> ((h & 7) * 4)) & 0xFu;
  }

  // First member >= lo inside block b (or -1).
  __device__ int64_t block_first(int64_t b, int lo) const {
    const int lane = lane_id();
    const int64_t wi = b * 32 + lane;
    uint32_t w = wi < a->nib_words ? nib[wi] : 0u;
    const int base = lane * 8;
    if (base + 8 <= lo) w = 0u;
    else if (base < lo) w &= ~0u << ((lo - base) * 4);
    const unsigned nz = __ballot_sync(0xffffffffu, w != 0u);
    if (!nz) return -1;
    const int l = __ffs(nz) - 1;
    const uint32_t wl = __shfl_sync(0xffffffffu, w, l);
    return b * 256 + l * 8 + (__ffs(wl) - 1) / 4;
  }

  // Last member <= hi inside block b (or -1).
  __device__ int64_t block_last(int64_t b, int hi) const {
    const int lane = lane_id();
    const int64_t wi = b * 32 + lane;
    uint32_t w = wi < a->nib_words ? nib[wi] : 0u;
    const int base = lane * 8;
    if (base > hi) w = 0u;
    else if (base + 7 > hi) w &= (hi - base == 7) ? ~0u : ((1u << ((hi - base + 1) * 4)) - 1u);
    const unsigned nz = __ballot_sync(0xffffffffu, w != 0u);
    if (!nz) return -1;
    const int l = 31 - __clz(nz);
    const uint32_t wl = __shfl_sync(0xffffffffu, w, l);
    return b * 256 + l * 8 + (31 - __clz(wl)) / 4;
  }

  // Smallest member > x (x >= -1); -1 when there is none.
  __device__ int64_t next_member(int64_t x) const {
    const int64_t start = x + 1;
    int64_t b = start >> 8;
    if (b >= a->nblocks) return -1;
    int64_t r = block_first(b, (int)(start & 255));
    if (r >= 0) return r;
    const int lane = lane_id();
    for (int64_t bb = b + 1; bb < a->nblocks;) {
      const int64_t sw = bb >> 5;
      uint32_t w = 0u;
      const int64_t wl = sw + lane;
      if (wl < a->sum_words) w = sum[wl];
      if (lane == 0) w &= ~0u << (bb & 31);
      const unsigned nz = __ballot_sync(0xffffffffu, w != 0u);
      if (nz) {
        const int l = __ffs(nz) - 1;
        const uint32_t ww = __shfl_sync(0xffffffffu, w, l);
        const int64_t blk = (sw + l) * 32 + (__ffs(ww) - 1);
        return block_first(blk, 0);
      }
      bb = (sw + 32) * 32;
    }
    return -1;
  }

  // Largest member < x; -1 when there is none.
  __device__ int64_t prev_member(int64_t x) const {
    const int64_t end = x - 1;
    if (end < 0) return -1;
    int64_t b = end >> 8;
    int64_t r = block_last(b, (int)(end & 255));
    if (r >= 0) return r;
    const int lane = lane_id();
    for (int64_t bb = b - 1; bb >= 0;) {
      const int64_t sw = bb >> 5;
      uint32_t w = 0u;
      const int64_t wl = sw - lane;
      if (wl >= 0) w = sum[wl];
      if (lane == 0) w &= ((bb & 31) == 31) ? ~0u : ((1u << ((bb & 31) + 1)) - 1u);
      const unsigned nz = __ballot_sync(0xffffffffu, w != 0u);
      if (nz) {
        const int l = __ffs(nz) - 1;  // the lowest lane is the highest word
        const uint32_t ww = __shfl_sync(0xffffffffu, w, l);
        const int64_t blk = (sw - l) * 32 + (31 - __clz(ww));
        return block_last(blk, 255);
      }
      bb = sw * 32 - 32 * 32 + 31;
      if (sw - 32 < 0) break;
    }
    return -1;
  }

  // Adds strand bits (query bits 0-1 or target bits 2-3) for hash h and
  // updates s, the count below theta and est; returns the old state.
  __device__ uint32_t add(int64_t h, uint32_t bits) {
    uint32_t* wp = nib + (h >> 3);
    const int sh = (int)(h & 7) * 4;
    const uint32_t word = *wp;
    const uint32_t old = (word >> sh) & 0xFu, nw = old | bits;
    if (old != nw) {
      __syncwarp();
      if (lane_id() == 0) {
        *wp = (word & ~(0xFu << sh)) | (nw << sh);
        if (old == 0u) sum[h >> 13] |= 1u << ((h >> 8) & 31);
      }
      __syncwarp();
      if (old == 0u && h < theta) ++cnt;
      if ((old & 3u) == 0u && (nw & 3u) != 0u) ++s;
      if (h <= theta) est += (int64_t)shareable(nw, o) - (int64_t)shareable(old, o);
    }
    return old;
  }

  // Puts back the old state of hash h (a step taken back).
  __device__ void restore(int64_t h, uint32_t old) {
    uint32_t* wp = nib + (h >> 3);
    const int sh = (int)(h & 7) * 4;
    const uint32_t word = *wp;
    __syncwarp();
    if (lane_id() == 0) *wp = (word & ~(0xFu << sh)) | (old << sh);
    __syncwarp();
    if (old == 0u && block_first(h >> 8, 0) < 0) {
      if (lane_id() == 0) sum[h >> 13] &= ~(1u << ((h >> 8) & 31));
      __syncwarp();
    }
  }

  // Moves theta until exactly s members are <= theta.
  __device__ void rebalance() {
    while (cnt > s) {
      if (shareable(state(theta), o)) --est;
      --cnt;
      theta = prev_member(theta);
    }
    while (cnt < s) {
      const int64_t x = next_member(theta);
      if (x < 0) break;  // cannot happen: W_Q is inside the union
      theta = x;
      ++cnt;
      if (shareable(state(theta), o)) ++est;
    }
  }
};

__device__ __forceinline__ int64_t first_pos_gt(const uint64_t* r, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rec_pos(r[mid]) <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t overlap_len(int64_t a0, int64_t a1, int64_t b0, int64_t b1) {
  const int64_t lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
  return hi > lo ? hi - lo : 0;
}

__global__ void __launch_bounds__(32 * kExtWarps) k_extend(ExtArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  uint32_t* sum = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)warp * a.sum_words;
  ExtSmem& S = reinterpret_cast<ExtSmem*>(
      smem_raw + (size_t)kExtWarps * a.sum_words * 4)[warp];
  const int64_t gw = (int64_t)blockIdx.x * kExtWarps + warp;
  uint32_t* nib = a.nib + gw * a.nib_words;
  for (int x = lane; x < a.sum_words; x += 32) sum[x] = 0u;
  __syncwarp();
  const int k = a.k;
  while (true) {
    int64_t x = 0;
    if (lane == 0) x = (int64_t)atomicAdd(a.next, 1u);
    x = __shfl_sync(0xffffffffu, x, 0);
    if (x >= a.nkept) break;
    const sedef_run_t run = a.runs[a.kept[x]];
    const int o = run.o;
    const int64_t i = run.i, js = run.j_star;
    const int qs = seq_of(a.qoff, a.nqseq, i), ts = seq_of(a.toff, a.ntseq, js);
    const int64_t qlo = a.qoff[qs], qhi = a.qoff[qs + 1], tlo = a.toff[ts], thi = a.toff[ts + 1];
    const bool same = a.self_mode && qs == ts;
    int64_t qa = i, qb = i + a.n, ta = js, tb = js + a.n;
    Ext E;
    E.a = &a;
    E.nib = nib;
    E.sum = sum;
    E.o = o;
    // ---- the seed: every record of both regions, inserted by all lanes
    // (atomics), then theta, the count below it and est from the sorted union
    const int64_t q0 = first_pos_gt(a.qrec, a.nq, qa - 1), q1 = first_pos_gt(a.qrec, a.nq, qb - k);
    const int64_t t0 = first_pos_gt(a.trec, a.nt, ta - 1), t1 = first_pos_gt(a.trec, a.nt, tb - k);
    int ninit = 0;
    int64_t s0 = 0;
    for (int64_t y = q0 + lane; y < q1; y += 32) {
      const uint64_t r = a.qrec[y];
      const uint32_t h = rec_hash(r);
      const uint32_t old = atomicOr(nib + (h >> 3), (1u << rec_strand(r)) << ((h & 7) * 4));
      if (((old >> ((h & 7) * 4)) & 0xFu) == 0u) atomicOr(sum + (h >> 13), 1u << ((h >> 8) & 31));
      if (((old >> ((h & 7) * 4)) & 3u) == 0u) ++s0;  // first query occurrence
      S.init[(y - q0) < kExtInit ? (y - q0) : 0] = h;
    }
    ninit = (int)(q1 - q0);
    for (int64_t y = t0 + lane; y < t1; y += 32) {
      const uint64_t r = a.trec[y];
      const int64_t pos = rec_pos(r);
      const uint32_t h = rec_hash(r);
      if (!(a.self_mode && pos >= qa && pos <= qb - k)) {
        const uint32_t old = atomicOr(nib + (h >> 3), (4u << rec_strand(r)) << ((h & 7) * 4));
        if (((old >> ((h & 7) * 4)) & 0xFu) == 0u)
          atomicOr(sum + (h >> 13), 1u << ((h >> 8) & 31));
      }
      const int64_t at = ninit + (y - t0);
      S.init[at < kExtInit ? at : 0] = h;
    }
    ninit += (int)(t1 - t0);
    __syncwarp();
    E.s = warp_sum(s0);
    // sort the inserted hashes; theta = the s-th distinct one
    int np = 1;
    while (np < ninit) np <<= 1;
    for (int y = ninit + lane; y < np; y += 32) S.init[y] = 0xFFFFFFFFu;
    __syncwarp();
    for (int size = 2; size <= np; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = lane; t < (np >> 1); t += 32) {
          const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
          const int hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const uint32_t u = S.init[lo], v = S.init[hi];
          if ((u > v) == asc) {
            S.init[lo] = v;
            S.init[hi] = u;
          }
        }
        __syncwarp();
      }
    {
      // members in sorted order: a hash counts once, and only if it is a
      // member (an excluded target record's hash is a member through W_Q)
      int64_t taken = 0, e = 0, th = -1;
      for (int base = 0; base < ninit && taken < E.s; base += 32) {
        const int y = base + lane;
        bool first = false;
        uint32_t h = 0;
        if (y < ninit) {
          h = S.init[y];
          first = (y == 0 || S.init[y - 1] != h) && E.state(h) != 0u;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, first);
        const int rank = (int)taken + __popc(fm & lanemask_lt());
        const bool in_u = first && rank < E.s;
        const unsigned um = __ballot_sync(0xffffffffu, in_u);
        const unsigned shm = __ballot_sync(0xffffffffu, in_u && shareable(E.state(h), o));
        e += __popc(shm);
        if (um) {
          const int last = 31 - __clz(um);
          th = __shfl_sync(0xffffffffu, (int64_t)h, last);
        }
        taken += __popc(um);
      }
      E.theta = th;
      E.cnt = taken;
      E.est = e;
    }
    __syncwarp();
    const int32_t* mt = a.mtab;
    auto m_of = [&](int64_t s) -> int64_t { return s <= a.smax ? mt[s] : mt[a.smax]; };
    int64_t est = E.est, den = E.s;
    if (E.est >= m_of(E.s)) {
      for (int dir = 0; dir < 2; ++dir) {
        // pointers to the next record to enter on each side
        const bool t_right = (dir == 0) == (o == 0);
        int64_t qp = dir == 0 ? first_pos_gt(a.qrec, a.nq, qb - k) : first_pos_gt(a.qrec, a.nq, qa - 1) - 1;
        int64_t tp = t_right ? first_pos_gt(a.trec, a.nt, tb - k) : first_pos_gt(a.trec, a.nt, ta - 1) - 1;
        while (true) {
          // steps until the next record fits in each region
          const int64_t INF = INT64_MAX / 4;
          int64_t dq = INF, dt = INF;
          if (dir == 0) {
            if (qp < a.nq) dq = (int64_t)rec_pos(a.qrec[qp]) + k - qb;
          } else if (qp >= 0) {
            dq = qa - (int64_t)rec_pos(a.qrec[qp]);
          }
          if (t_right) {
            if (tp < a.nt) dt = (int64_t)rec_pos(a.trec[tp]) + k - tb;
          } else if (tp >= 0) {
            dt = ta - (int64_t)rec_pos(a.trec[tp]);
          }
          // steps the limits allow
          int64_t lim = dir == 0 ? qhi - qb : qa - qlo;
          const int64_t lt = t_right ? thi - tb : ta - tlo;
          if (lt < lim) lim = lt;
          const int64_t ll = a.max_len - (qb - qa);
          if (ll < lim) lim = ll;
          if (lim < 0) lim = 0;
          auto grown = [&](int64_t d, int64_t* na, int64_t* nb, int64_t* ma, int64_t* mb) {
            *na = dir == 0 ? qa : qa - d;
            *nb = dir == 0 ? qb + d : qb;
            *ma = t_right ? ta : ta - d;
            *mb = t_right ? tb + d : tb;
          };
          if (same && lim > 0) {
            // the overlap never shrinks as the regions grow: the largest d
            // whose overlap is still the current one
            const int64_t ov0 = overlap_len(qa, qb, ta, tb);
            int64_t lo = 0, hi = lim;
            while (lo < hi) {
              const int64_t mid = (lo + hi + 1) >> 1;
              int64_t na, nb, ma, mb;
              grown(mid, &na, &nb, &ma, &mb);
              if (overlap_len(na, nb, ma, mb) <= ov0) lo = mid; else hi = mid - 1;
            }
            lim = lo;
          }
          const int64_t d = dq < dt ? dq : dt;
          if (d > lim) {  // no minimizer joins before the limit: grow to it
            int64_t na, nb, ma, mb;
            grown(lim, &na, &nb, &ma, &mb);
            qa = na, qb = nb, ta = ma, tb = mb;
            break;
          }
          int64_t na, nb, ma, mb;
          grown(d, &na, &nb, &ma, &mb);
          const int64_t c_s = E.s, c_cnt = E.cnt, c_est = E.est, c_th = E.theta;
          int64_t hq = -1, ht = -1;
          uint32_t oq = 0, ot = 0;
          if (dq == d) {
            const uint64_t r = a.qrec[qp];
            hq = rec_hash(r);
            oq = E.add(hq, 1u << rec_strand(r));
          }
          if (dt == d) {
            const uint64_t r = a.trec[tp];
            const int64_t pos = rec_pos(r);
            if (!(a.self_mode && pos >= na && pos <= nb - k)) {
              ht = rec_hash(r);
              ot = E.add(ht, 4u << rec_strand(r));
            }
          }
          E.rebalance();
          if (E.est < m_of(E.s)) {  // take the step back; grow to just before it
            if (ht >= 0) E.restore(ht, ot);
            if (hq >= 0) E.restore(hq, oq);
            E.s = c_s, E.cnt = c_cnt, E.est = c_est, E.theta = c_th;
            grown(d - 1, &na, &nb, &ma, &mb);
            qa = na, qb = nb, ta = ma, tb = mb;
            break;
          }
          qa = na, qb = nb, ta = ma, tb = mb;
          if (dq == d) qp += dir == 0 ? 1 : -1;
          if (dt == d) tp += t_right ? 1 : -1;
        }
      }
      est = E.est;
      den = E.s;
    }
    if (lane == 0) {
      sedef_region_t R;
      R.i = (uint32_t)i;
      R.j_star = (uint32_t)js;
      R.qa = (uint32_t)qa;
      R.qb = (uint32_t)qb;
      R.ta = (uint32_t)ta;
      R.tb = (uint32_t)tb;
      R.est = (uint32_t)est;
      R.den = (uint32_t)den;
      R.o = (uint32_t)o;
      R.reserved = 0;
      a.out[x] = R;
    }
    // clear the tables: every member comes from a record of the final regions
    __syncwarp();
    {
      const int64_t c0 = first_pos_gt(a.qrec, a.nq, qa - 1), c1 = first_pos_gt(a.qrec, a.nq, qb - k);
      for (int64_t y = c0 + lane; y < c1; y += 32) nib[rec_hash(a.qrec[y]) >> 3] = 0u;
      const int64_t d0 = first_pos_gt(a.trec, a.nt, ta - 1), d1 = first_pos_gt(a.trec, a.nt, tb - k);
      for (int64_t y = d0 + lane; y < d1; y += 32) nib[rec_hash(a.trec[y]) >> 3] = 0u;
      for (int y = lane; y < a.sum_words; y += 32) sum[y] = 0u;
    }
    __syncwarp();
  }
}

__global__ void k_keep_flags(const sedef_run_t* runs, int64_t n, uint32_t* flags) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) flags[r] = runs[r].keep ? 1u : 0u;
}

__global__ void k_keep_list(const sedef_run_t* runs, int64_t n, const uint32_t* pos, uint32_t* kept) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && runs[r].keep) kept[pos[r]] = (uint32_t)r;
}

}  // namespace

int run_extend(sedef_ctx* ctx, const sedef_run_t* runs, int64_t nruns, const uint64_t* qrec,
               int64_t nq, const int64_t* h_qoff, int nqseq, const uint64_t* trec, int64_t nt,
               const int64_t* h_toff, int ntseq, const Derived& D, const sedef_params* p,
               int64_t max_len, sedef_region_t* out, int64_t cap, int64_t* nout) {
  cudaStream_t st = ctx_stream(ctx);
  *nout = 0;
  if (nruns == 0) return SEDEF_OK;
  // kept seeds in run order
  uint32_t* flags = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  uint32_t* pos = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  uint32_t* kept = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  if (!flags || !pos || !kept) return SEDEF_ERR_OOM;
  const int tb = (int)((nruns + 255) / 256);
  SEDEF_KERNEL(ctx, "k_keep_flags", k_keep_flags<<<tb, 256, 0, st>>>(runs, nruns, flags));
  SEDEF_TRY(scan_exclusive_u32(ctx, flags, pos, nruns, pos + nruns));
  SEDEF_KERNEL(ctx, "k_keep_list", k_keep_list<<<tb, 256, 0, st>>>(runs, nruns, pos, kept));
  uint32_t* h_n = (uint32_t*)ctx_host(ctx, 8);
  if (!h_n) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemcpyAsync(h_n, pos + nruns, 4, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  const int64_t nk = *h_n;
  *nout = nk;
  if (nk > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_extend: region buffer too small");
  if (nk == 0) return SEDEF_OK;
  // uploads: offsets and m(s) for every s a region of max_len bases can have
  const int64_t smax = max_len + 1;
  const size_t up = (size_t)(nqseq + 1) * 8 + (size_t)(ntseq + 1) * 8 + (size_t)(smax + 1) * 4;
  char* h_up = (char*)ctx_host(ctx, up + 64);
  char* d_up = (char*)ctx_alloc(ctx, up + 64);
  if (!h_up || !d_up) return SEDEF_ERR_OOM;
  std::memcpy(h_up, h_qoff, (size_t)(nqseq + 1) * 8);
  std::memcpy(h_up + (nqseq + 1) * 8, h_toff, (size_t)(ntseq + 1) * 8);
  int32_t* h_m = (int32_t*)(h_up + (nqseq + 1) * 8 + (ntseq + 1) * 8);
  mtable(p, h_m, (int)smax, nullptr);
  SEDEF_CUDA(cudaMemcpyAsync(d_up, h_up, up, cudaMemcpyHostToDevice, st));
  // per-warp tables: 4 bits per hash, one summary bit per 256 hashes
  const int64_t nhash = int64_t(1) << (2 * D.k);
  ExtArgs a;
  a.runs = runs;
  a.kept = kept;
  a.nkept = nk;
  a.qrec = qrec;
  a.nq = nq;
  a.trec = trec;
  a.nt = nt;
  a.qoff = (const int64_t*)d_up;
  a.nqseq = nqseq;
  a.toff = (const int64_t*)(d_up + (nqseq + 1) * 8);
  a.ntseq = ntseq;
  a.mtab = (const int32_t*)(d_up + (nqseq + 1) * 8 + (ntseq + 1) * 8);
  a.smax = smax;
  a.k = D.k;
  a.n = D.n;
  a.self_mode = D.self_mode;
  a.max_len = max_len;
  a.nib_words = (nhash + 7) / 8;
  a.nblocks = (nhash + 255) / 256;
  a.sum_words = (int)((a.nblocks + 31) / 32);
  int64_t ctas = (nk + kExtWarps - 1) / kExtWarps;
  const int64_t most = (int64_t)ctx_sm_count(ctx) * 2;
  if (ctas > most) ctas = most;
  const size_t tab = (size_t)a.nib_words * 4;
  uint32_t* nib = (uint32_t*)ctx_alloc(ctx, tab * (size_t)(ctas * kExtWarps));
  unsigned int* next = (unsigned int*)ctx_alloc(ctx, 8);
  if (!nib || !next) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemsetAsync(nib, 0, tab * (size_t)(ctas * kExtWarps), st));
  SEDEF_CUDA(cudaMemsetAsync(next, 0, 8, st));
  a.nib = nib;
  a.next = next;
  a.out = out;
  const size_t sm = (size_t)kExtWarps * (a.sum_words * 4 + sizeof(ExtSmem));
  SEDEF_TRY(ensure_smem_attr((const void*)k_extend, sm));
  SEDEF_KERNEL(ctx, "k_extend", k_extend<<<(int)ctas, 32 * kExtWarps, sm, st>>>(a));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // namespace sedef
