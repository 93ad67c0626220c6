// a7: chaining of each kept seed's minimizer anchors (Section 3.3) and the
// merge of chains into SD candidates.
//
// Chain: one warp per kept run.  Anchors are enumerated straight from the
// index: each query minimizer of the window searches its posting list for
// the run's target span (an interpolated search, then a short gallop), so
// anchors come out sorted by (p, t') without a sort (t' = t for o = 0; for
// o = 1 the posting list is walked backwards).
// The DP visits anchors in order; for anchor a the 32 lanes scan the
// predecessors b (only those with p_b >= p_a - gap_max) and a warp max-reduce
// over (f_b + 1, b) picks the predecessor with the larger count, then the
// later index.
//
// Merge: chains sorted by (o, q0); every chain links to the following chains
// whose query interval starts before its own ends; links are united with a
// lock-free union-find that always hooks the larger root under the smaller,
// so every component's root is its smallest member.
#include <cstring>
#include <string>

#include "common.cuh"

namespace sedef {

namespace {

struct ChainArgs {
  const sedef_run_t* runs;
  int64_t nruns;
  const uint64_t* qrec;
  int64_t nq;
  const uint64_t* tidx;     // hash-sorted target records (index)
  int64_t nt;
  const uint32_t* toff;
  const int64_t* qseq;
  int nqseq;
  const int64_t* tseq;
  int ntseq;
  const int32_t* mtab;
  int k, span, max_occ, self_mode, gap_max, diag_max;
  // live counts of a planned pass, the anchor capacity and its overflow flags
  const uint32_t* dnruns = nullptr;
  const uint32_t* dnq = nullptr;
  const uint32_t* dnt = nullptr;
  int64_t acap = 0;
  uint32_t* flags = nullptr;
  unsigned long long* atotal = nullptr;  // exact anchor total (planned pass)
};

// The chain DP is quadratic in a seed's anchors; a seed inside an unmasked
// low-complexity run can have millions.  Such seeds are refused.
constexpr int kMaxChainAnchors = 1 << 16;

__device__ __forceinline__ void resolve(ChainArgs& a) {
  a.nruns = live_n(a.nruns, a.dnruns);
  a.nq = live_n(a.nq, a.dnq);
  a.nt = live_n(a.nt, a.dnt);
}

// Postings of query record q's hash inside run `run`'s target span
// [j_a, j_b + n - k]: [*b0, *b1) of the index (empty when the list passes
// max_occ).  The start comes from an interpolated search of the posting
// list, the end from a gallop forward from it (the span is short).
__device__ __forceinline__ void record_postings(const ChainArgs& a, const sedef_run_t& run,
                                                uint64_t q, uint32_t* b0, uint32_t* b1) {
  const uint32_t h = rec_hash(q);
  const uint32_t st = a.toff[h], en = a.toff[h + 1];
  if (a.max_occ > 0 && (int)(en - st) > a.max_occ) {
    *b0 = *b1 = st;
    return;
  }
  const uint32_t tlo = run.j_a, thi = run.j_b + (uint32_t)a.span;
  *b0 = pos_lower_bound(a.tidx, st, en, (int64_t)tlo);
  *b1 = pos_gallop_forward(a.tidx, *b0, en, (int64_t)thi + 1);
}

// Visits the anchors of run `run` contributed by query record q among the
// postings [b0, b1): calls f(rank, p, t) for each, rank counting this
// record's anchors in (p, t') order.  Returns the number of anchors.
template <typename F>
__device__ int record_anchors(const ChainArgs& a, const sedef_run_t& run, uint64_t q, uint32_t b0,
                              uint32_t b1, F f) {
  const uint32_t p = rec_pos(q), sq = rec_strand(q);
  int cnt = 0;
  const int64_t i = run.i;
  auto visit = [&](int64_t y) {
    const uint64_t r = a.tidx[y];
    const uint32_t t = rec_pos(r);
    if ((sq ^ rec_strand(r)) != run.o) return;
    if (a.self_mode && (int64_t)t >= i && (int64_t)t <= i + a.span) return;
    f(cnt, p, t);
    ++cnt;
  };
  if (run.o == 0)
    for (int64_t y = b0; y < b1; ++y) visit(y);
  else
    for (int64_t y = (int64_t)b1 - 1; y >= (int64_t)b0; --y) visit(y);
  return cnt;
}

__device__ __forceinline__ void window_range(const ChainArgs& a, int64_t i, int64_t* qa, int64_t* qb) {
  auto pos_of = [](uint64_t r) { return (uint64_t)((r >> 1) & 0xFFFFFFFFull); };
  *qa = lower_bound_by(a.qrec, 0, a.nq, (uint64_t)i, pos_of);
  *qb = lower_bound_by(a.qrec, *qa, a.nq, (uint64_t)(i + a.span + 1), pos_of);
}

// Anchors per kept run (0 for runs that are not kept).
__global__ void k_anchor_count(ChainArgs a, uint32_t* count) {
  resolve(a);
  const int lane = lane_id();
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= a.nruns) return;
  const sedef_run_t run = a.runs[r];
  int total = 0;
  if (run.keep) {
    int64_t qa = 0, qb = 0;
    if (lane == 0) window_range(a, run.i, &qa, &qb);
    qa = __shfl_sync(0xffffffffu, qa, 0);
    qb = __shfl_sync(0xffffffffu, qb, 0);
    for (int64_t x = qa + lane; x < qb; x += 32) {
      const uint64_t q = a.qrec[x];
      uint32_t b0, b1;
      record_postings(a, run, q, &b0, &b1);
      total += record_anchors(a, run, q, b0, b1, [](int, uint32_t, uint32_t) {});
    }
    total = warp_sum(total);
  }
  if (lane == 0) {
    count[r] = (uint32_t)total;
    if (a.atotal && total) atomicAdd(a.atotal, (unsigned long long)total);
  }
}

// Writes anchors as (p << 32 | t') at the run's offset, in (p, t') order.
__global__ void k_anchor_fill(ChainArgs a, const uint32_t* aoff, uint64_t* anchors) {
  resolve(a);
  const int lane = lane_id();
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= a.nruns) return;
  const sedef_run_t run = a.runs[r];
  if (!run.keep) return;
  // 32-bit offsets: a range that wraps or ends past the capacity is skipped
  if (aoff[r + 1] < aoff[r] || (int64_t)aoff[r + 1] > a.acap ||
      aoff[r + 1] - aoff[r] > (uint32_t)kMaxChainAnchors)
    return;
  int64_t qa = 0, qb = 0;
  if (lane == 0) window_range(a, run.i, &qa, &qb);
  qa = __shfl_sync(0xffffffffu, qa, 0);
  qb = __shfl_sync(0xffffffffu, qb, 0);
  const uint32_t tref = run.j_b + (uint32_t)a.span;
  uint32_t base = aoff[r];
  for (int64_t x0 = qa; x0 < qb; x0 += 32) {
    const int64_t x = x0 + lane;
    int c = 0;
    uint64_t q = 0;
    uint32_t b0 = 0, b1 = 0;
    if (x < qb) {
      q = a.qrec[x];
      record_postings(a, run, q, &b0, &b1);
      c = record_anchors(a, run, q, b0, b1, [](int, uint32_t, uint32_t) {});
    }
    const int inc = warp_inclusive_sum(c);
    const uint32_t my = base + (uint32_t)(inc - c);
    if (x < qb && c > 0)
      record_anchors(a, run, q, b0, b1, [&](int rank, uint32_t p, uint32_t t) {
        const uint32_t tp = run.o ? tref - t : t;
        anchors[my + rank] = ((uint64_t)p << 32) | tp;
      });
    base += (uint32_t)__shfl_sync(0xffffffffu, inc, 31);
  }
}

// DP over each kept run's anchors; writes the run's chain (score 0 = none).
__global__ void k_chain_dp(ChainArgs a, const uint32_t* aoff, const uint64_t* anchors, int32_t* f,
                           int32_t* pred, sedef_chain_t* out) {
  resolve(a);
  const int lane = lane_id();
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= a.nruns) return;
  const sedef_run_t run = a.runs[r];
  sedef_chain_t c;
  c.i = run.i;
  c.o = run.o;
  c.s = run.s;
  c.score = 0;
  c.reserved = 0;
  const uint32_t A0 = aoff[r], A = aoff[r + 1] - A0;
  const bool wrapped = aoff[r + 1] < A0;
  const bool over = wrapped || (int64_t)aoff[r + 1] > a.acap;
  const bool big = !wrapped && A > (uint32_t)kMaxChainAnchors;
  if (run.keep && (over || big) && a.flags && lane == 0)
    atomicOr(a.flags, (over ? (uint32_t)kOverAnchors : 0u) | (big ? (uint32_t)kAnchorLimit : 0u));
  if (!run.keep || A == 0 || over || big) {
    if (lane == 0) {
      c.qseq = c.q0 = c.q1 = c.tseq = c.t0 = c.t1 = 0;
      out[r] = c;
    }
    return;
  }
  const uint64_t* an = anchors + A0;
  int32_t* F = f + A0;
  int32_t* P = pred + A0;
  uint32_t blo = 0;  // first predecessor with p >= p_a - gap_max
  for (uint32_t x = 0; x < A; ++x) {
    const uint64_t ax = an[x];
    const int64_t pa = (int64_t)(ax >> 32), ta = (int64_t)(uint32_t)ax;
    while (blo < x && (int64_t)(an[blo] >> 32) < pa - a.gap_max) ++blo;
    unsigned long long best = 0;  // (f + 1) << 32 | b
    for (uint32_t b = blo + lane; b < x; b += 32) {
      const uint64_t bx = an[b];
      const int64_t dp = pa - (int64_t)(bx >> 32), dt = ta - (int64_t)(uint32_t)bx;
      if (dp <= 0 || dt <= 0 || dp > a.gap_max || dt > a.gap_max) continue;
      const int64_t dd = dp - dt;
      if (dd > a.diag_max || -dd > a.diag_max) continue;
      const unsigned long long cand = ((unsigned long long)(F[b] + 1) << 32) | b;
      if (cand > best) best = cand;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, d);
      if (o > best) best = o;
    }
    if (lane == 0) {
      if (best) {
        F[x] = (int32_t)(best >> 32);
        P[x] = (int32_t)(uint32_t)best;
      } else {
        F[x] = 1;
        P[x] = -1;
      }
    }
    __syncwarp();
  }
  // best end: largest f, then smallest index
  unsigned long long be = 0;  // f << 32 | (~index)
  for (uint32_t x = lane; x < A; x += 32) {
    const unsigned long long v = ((unsigned long long)F[x] << 32) | (0xFFFFFFFFu - x);
    if (v > be) be = v;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, be, d);
    if (o > be) be = o;
  }
  if (lane != 0) return;
  const int score = (int)(be >> 32);
  const int end = (int)(0xFFFFFFFFu - (uint32_t)be);
  const uint32_t tref = run.j_b + (uint32_t)a.span;
  uint32_t q0 = 0xFFFFFFFFu, q1 = 0, t0 = 0xFFFFFFFFu, t1 = 0;
  for (int x = end; x >= 0; x = P[x]) {
    const uint64_t ax = an[x];
    const uint32_t p = (uint32_t)(ax >> 32), tp = (uint32_t)ax;
    const uint32_t t = run.o ? tref - tp : tp;
    q0 = min(q0, p);
    q1 = max(q1, p + (uint32_t)a.k);
    t0 = min(t0, t);
    t1 = max(t1, t + (uint32_t)a.k);
  }
  c.qseq = (uint32_t)seq_of(a.qseq, a.nqseq, run.i);
  c.tseq = (uint32_t)seq_of(a.tseq, a.ntseq, run.j_a);
  c.q0 = q0;
  c.q1 = q1;
  c.t0 = t0;
  c.t1 = t1;
  c.score = (score >= a.mtab[run.s]) ? (uint16_t)score : 0;
  out[r] = c;
}

__global__ void k_max_u32(const uint32_t* v, int64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    m = max(m, v[x]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
  if (lane_id() == 0) atomicMax(out, m);
}

// Flags over all n slots (zero past the live count, so that a scan over n
// counts the live chains only).
__global__ void k_chain_flags(const sedef_chain_t* c, int64_t n, uint32_t* flag,
                              const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) flag[x] = (x < live_n(n, dn) && c[x].score > 0) ? 1u : 0u;
}

__global__ void k_chain_compact(const sedef_chain_t* c, int64_t n, const uint32_t* pos,
                                sedef_chain_t* out, int64_t cap, const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < live_n(n, dn) && c[x].score > 0 && (int64_t)pos[x] < cap) out[pos[x]] = c[x];
}

// ----------------------------------------------------------------- merge --

struct MergeArgs {
  const sedef_chain_t* ch;
  int64_t n;
  const uint32_t* perm;  // sorted position -> chain index
  int32_t* parent;       // over sorted positions
  int diag_max;
  double delta_g;
  const uint32_t* dn = nullptr;  // live chain count of a planned pass
};

__device__ __forceinline__ int uf_find(int32_t* parent, int x) {
  while (true) {
    const int p = parent[x];
    if (p == x) return x;
    const int g = parent[p];
    if (g != p) parent[x] = g;
    x = p;
  }
}

__device__ __forceinline__ void uf_union(int32_t* parent, int x, int y) {
  while (true) {
    x = uf_find(parent, x);
    y = uf_find(parent, y);
    if (x == y) return;
    if (x < y) {
      const int t = x;
      x = y;
      y = t;
    }
    if (atomicCAS(&parent[x], x, y) == x) return;  // hook the larger root under the smaller
  }
}

__device__ __forceinline__ int64_t diag_of(const sedef_chain_t& c) {
  return c.o == 0 ? (int64_t)c.t0 - (int64_t)c.q0 : (int64_t)c.t1 + (int64_t)c.q0;
}

__device__ __forceinline__ bool linked(const MergeArgs& a, const sedef_chain_t& A, const sedef_chain_t& B) {
  if (A.o != B.o || A.qseq != B.qseq || A.tseq != B.tseq) return false;
  if (B.q0 > A.q1 || A.q0 > B.q1) return false;
  if (B.t0 > A.t1 || A.t0 > B.t1) return false;
  const int64_t len = max((int64_t)A.q1 - A.q0, (int64_t)B.q1 - B.q0);
  const int64_t slack = a.diag_max + (int64_t)ceil(a.delta_g * (double)len);
  const int64_t dd = diag_of(A) - diag_of(B);
  return dd <= slack && -dd <= slack;
}

__global__ void k_merge_init(int32_t* parent, int64_t n) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) parent[x] = (int32_t)x;
}

__global__ void k_merge_link(MergeArgs a) {
  a.n = live_n(a.n, a.dn);
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.n) return;
  const sedef_chain_t A = a.ch[a.perm[x]];
  for (int64_t y = x + 1; y < a.n; ++y) {
    const sedef_chain_t B = a.ch[a.perm[y]];
    if (B.o != A.o || B.q0 > A.q1) break;
    if (linked(a, A, B)) uf_union(a.parent, (int)x, (int)y);
  }
}

struct Agg {
  uint32_t q0, q1, t0, t1, score, count;
};

__global__ void k_merge_agg(MergeArgs a, Agg* agg) {
  a.n = live_n(a.n, a.dn);
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.n) return;
  const int root = uf_find(a.parent, (int)x);
  const sedef_chain_t c = a.ch[a.perm[x]];
  atomicMin(&agg[root].q0, c.q0);
  atomicMax(&agg[root].q1, c.q1);
  atomicMin(&agg[root].t0, c.t0);
  atomicMax(&agg[root].t1, c.t1);
  atomicAdd(&agg[root].score, (uint32_t)c.score);
  atomicAdd(&agg[root].count, 1u);
}

__global__ void k_agg_init(Agg* agg, int64_t n) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) {
    agg[x].q0 = 0xFFFFFFFFu;
    agg[x].q1 = 0;
    agg[x].t0 = 0xFFFFFFFFu;
    agg[x].t1 = 0;
    agg[x].score = 0;
    agg[x].count = 0;
  }
}

__global__ void k_root_flags(const int32_t* parent, int64_t n, uint32_t* flag, const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) flag[x] = (x < live_n(n, dn) && parent[x] == (int32_t)x) ? 1u : 0u;
}

// Candidate keys: primary (q0 << 32 | t0); the tie order (o, q1, t1) is
// applied by k_fix_ties after the primary sort.
__global__ void k_cand_emit(MergeArgs a, const Agg* agg, const uint32_t* pos, sedef_cand_t* tmp,
                            uint64_t* key, int64_t ccap) {
  a.n = live_n(a.n, a.dn);
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.n || a.parent[x] != (int32_t)x || (int64_t)pos[x] >= ccap) return;
  const sedef_chain_t c = a.ch[a.perm[x]];
  const Agg g = agg[x];
  sedef_cand_t d;
  d.qseq = c.qseq;
  d.q0 = g.q0;
  d.q1 = g.q1;
  d.tseq = c.tseq;
  d.t0 = g.t0;
  d.t1 = g.t1;
  d.o = c.o;
  d.score = g.score;
  d.nchains = g.count;
  d.reserved = 0;
  tmp[pos[x]] = d;
  key[pos[x]] = ((uint64_t)g.q0 << 32) | g.t0;
}

__device__ __forceinline__ bool cand_less(const sedef_cand_t& x, const sedef_cand_t& y) {
  if (x.q0 != y.q0) return x.q0 < y.q0;
  if (x.t0 != y.t0) return x.t0 < y.t0;
  if (x.o != y.o) return x.o < y.o;
  if (x.q1 != y.q1) return x.q1 < y.q1;
  if (x.t1 != y.t1) return x.t1 < y.t1;
  if (x.qseq != y.qseq) return x.qseq < y.qseq;
  if (x.tseq != y.tseq) return x.tseq < y.tseq;
  if (x.score != y.score) return x.score < y.score;
  return x.nchains < y.nchains;
}

// Gathers candidates in primary-key order, orders equal-key groups by the
// full comparator (groups are tiny) and converts to per-sequence coordinates.
__global__ void k_cand_final(const sedef_cand_t* tmp, const uint32_t* perm, const uint64_t* skey,
                             int64_t n, const int64_t* qseq, const int64_t* tseq, sedef_cand_t* out,
                             const uint32_t* dn) {
  n = live_n(n, dn);
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  if (x > 0 && skey[x - 1] == skey[x]) return;  // group leader handles the group
  int64_t e = x + 1;
  while (e < n && skey[e] == skey[x]) ++e;
  for (int64_t y = x; y < e; ++y) {
    // selection of the y-th smallest in the group (groups are tiny)
    sedef_cand_t best = tmp[perm[x]];
    bool set = false;
    for (int64_t z = x; z < e; ++z) {
      const sedef_cand_t c = tmp[perm[z]];
      int64_t rank = 0;
      for (int64_t u = x; u < e; ++u) {
        const sedef_cand_t d = tmp[perm[u]];
        if (cand_less(d, c) || (!cand_less(c, d) && u < z)) ++rank;
      }
      if (rank == y - x) {
        best = c;
        set = true;
        break;
      }
    }
    if (!set) best = tmp[perm[y]];
    sedef_cand_t o = best;
    o.q0 -= (uint32_t)qseq[best.qseq];
    o.q1 -= (uint32_t)qseq[best.qseq];
    o.t0 -= (uint32_t)tseq[best.tseq];
    o.t1 -= (uint32_t)tseq[best.tseq];
    out[y] = o;
  }
}

__global__ void k_chain_keys(const sedef_chain_t* c, int64_t n, uint64_t* key, const uint32_t* dn) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < live_n(n, dn)) key[x] = ((uint64_t)c[x].o << 32) | c[x].q0;
}

int grid_of(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total);

static int upload_offsets(sedef_ctx* ctx, Planned* pl, const int64_t* h_q, int nq,
                          const int64_t* h_t, int nt, int64_t** d_q, int64_t** d_t) {
  cudaStream_t st = ctx_stream(ctx);
  const size_t bytes = (size_t)(nq + 1 + nt + 1) * 8;
  int64_t* h = (int64_t*)host_buf(ctx, pl, bytes);
  int64_t* d = (int64_t*)ctx_alloc(ctx, bytes);
  if (!h || !d) return SEDEF_ERR_OOM;
  std::memcpy(h, h_q, (size_t)(nq + 1) * 8);
  std::memcpy(h + nq + 1, h_t, (size_t)(nt + 1) * 8);
  SEDEF_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
  *d_q = d;
  *d_t = d + nq + 1;
  return SEDEF_OK;
}

int run_chain(sedef_ctx* ctx, const sedef_run_t* runs, int64_t nruns, const uint64_t* qrec, int64_t nq,
              const int64_t* h_qoff, int nqseq, const uint64_t* tsorted, int64_t nt,
              const uint32_t* toff, const int64_t* h_toff, int ntseq, const Derived& D,
              const int32_t* h_mtab, sedef_chain_t* chains, int64_t cap, int64_t* nchains,
              Planned* pl) {
  cudaStream_t st = ctx_stream(ctx);
  int64_t *dq = nullptr, *dt = nullptr;
  SEDEF_TRY(upload_offsets(ctx, pl, h_qoff, nqseq, h_toff, ntseq, &dq, &dt));
  int32_t* dm = (int32_t*)ctx_alloc(ctx, (size_t)(kMaxWindowRecs + 1) * 4);
  if (!dm) return SEDEF_ERR_OOM;
  if (pl) {
    int32_t* hm = (int32_t*)host_buf(ctx, pl, (size_t)(kMaxWindowRecs + 1) * 4);
    if (!hm) return SEDEF_ERR_OOM;
    std::memcpy(hm, h_mtab, (size_t)(kMaxWindowRecs + 1) * 4);
    SEDEF_CUDA(cudaMemcpyAsync(dm, hm, (size_t)(kMaxWindowRecs + 1) * 4, cudaMemcpyHostToDevice, st));
  } else {
    SEDEF_CUDA(cudaMemcpyAsync(dm, h_mtab, (size_t)(kMaxWindowRecs + 1) * 4, cudaMemcpyHostToDevice, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));  // the mtab upload reads caller memory
  }

  ChainArgs a;
  a.runs = runs;
  a.nruns = nruns;
  a.qrec = qrec;
  a.nq = nq;
  a.tidx = tsorted;
  a.nt = nt;
  a.toff = toff;
  a.qseq = dq;
  a.nqseq = nqseq;
  a.tseq = dt;
  a.ntseq = ntseq;
  a.mtab = dm;
  a.k = D.k;
  a.span = D.span;
  a.max_occ = D.max_occ;
  a.self_mode = D.self_mode;
  a.gap_max = D.gap_max;
  a.diag_max = D.diag_max;
  unsigned long long* atotal = nullptr;
  if (pl) {
    a.dnruns = pl->n_runs;
    a.dnq = pl->n_rec;
    a.dnt = pl->n_rec;
    a.flags = pl->flags;
    atotal = (unsigned long long*)ctx_alloc(ctx, 8);
    if (!atotal) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemsetAsync(atotal, 0, 8, st));
    a.atotal = atotal;
  }

  uint32_t* cnt = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  uint32_t* aoff = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  sedef_chain_t* tmp = (sedef_chain_t*)ctx_alloc(ctx, (size_t)nruns * sizeof(sedef_chain_t));
  if (!cnt || !aoff || !tmp) return SEDEF_ERR_OOM;
  const int wb = grid_of(nruns * 32, 256);
  if (pl) SEDEF_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(nruns + 1) * 4, st));
  SEDEF_KERNEL(ctx, "k_anchor_count", k_anchor_count<<<wb, 256, 0, st>>>(a, cnt));
  uint32_t* amax = (uint32_t*)ctx_alloc(ctx, 8);
  if (!amax) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemsetAsync(amax, 0, 4, st));
  SEDEF_KERNEL(ctx, "k_max_u32",
               k_max_u32<<<grid_of(nruns < 65536 ? nruns : 65536, 256), 256, 0, st>>>(cnt, nruns, amax));
  SEDEF_TRY(scan_exclusive_u32(ctx, cnt, aoff, nruns, aoff + nruns));
  int64_t A;
  if (pl) {
    // anchors: planned capacity; seeds past it or over the limit are
    // skipped and flagged by the DP
    A = pl->anchors;
    SEDEF_TRY(plan_check64(ctx, pl, atotal, A, 3));
  } else {
    uint32_t* h_tot = (uint32_t*)ctx_host(ctx, 8);
    if (!h_tot) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(h_tot, aoff + nruns, 4, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaMemcpyAsync(h_tot + 1, amax, 4, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
    A = *h_tot;
    ctx_set_anchor_total(ctx, A);
    // refuse instead of running for hours
    if (h_tot[1] > (uint32_t)kMaxChainAnchors)
      return fail(SEDEF_ERR_UNSUPPORTED,
                  "sedef_chain: a seed has " + std::to_string(h_tot[1]) +
                      " anchors (limit 65536); soft-mask low-complexity repeats or set max_occ");
  }
  a.acap = A;
  uint64_t* anchors = (uint64_t*)ctx_alloc(ctx, (size_t)(A ? A : 1) * 8);
  int32_t* f = (int32_t*)ctx_alloc(ctx, (size_t)(A ? A : 1) * 4);
  int32_t* pred = (int32_t*)ctx_alloc(ctx, (size_t)(A ? A : 1) * 4);
  if (!anchors || !f || !pred) return SEDEF_ERR_OOM;
  SEDEF_KERNEL(ctx, "k_anchor_fill", k_anchor_fill<<<wb, 256, 0, st>>>(a, aoff, anchors));
  SEDEF_KERNEL(ctx, "k_chain_dp", k_chain_dp<<<wb, 256, 0, st>>>(a, aoff, anchors, f, pred, tmp));
  uint32_t* flag = cnt;  // reuse
  uint32_t* pos = (uint32_t*)ctx_alloc(ctx, (size_t)(nruns + 1) * 4);
  if (!pos) return SEDEF_ERR_OOM;
  const uint32_t* dn = pl ? pl->n_runs : nullptr;
  SEDEF_KERNEL(ctx, "k_chain_flags",
               k_chain_flags<<<grid_of(nruns, 256), 256, 0, st>>>(tmp, nruns, flag, dn));
  SEDEF_TRY(scan_exclusive_u32(ctx, flag, pos, nruns, pos + nruns));
  if (pl) {
    pl->n_chains = pos + nruns;
    SEDEF_TRY(plan_check(ctx, pl, pos + nruns, cap, 4));
    *nchains = cap;
    SEDEF_KERNEL(ctx, "k_chain_compact",
                 k_chain_compact<<<grid_of(nruns, 256), 256, 0, st>>>(tmp, nruns, pos, chains, cap, dn));
    return SEDEF_OK;
  }
  uint32_t* h_tot = (uint32_t*)ctx_host(ctx, 8);
  if (!h_tot) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemcpyAsync(h_tot, pos + nruns, 4, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  *nchains = *h_tot;
  if (*nchains > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_chain: chain buffer too small");
  SEDEF_KERNEL(ctx, "k_chain_compact",
               k_chain_compact<<<grid_of(nruns, 256), 256, 0, st>>>(tmp, nruns, pos, chains, cap,
                                                                    nullptr));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

int run_merge(sedef_ctx* ctx, const sedef_chain_t* chains, int64_t n, const int64_t* h_qoff,
              int nqseq, const int64_t* h_toff, int ntseq, const Derived& D, sedef_cand_t* cands,
              int64_t cap, int64_t* ncands, Planned* pl) {
  cudaStream_t st = ctx_stream(ctx);
  if (n >= (int64_t(1) << 31)) return fail(SEDEF_ERR_UNSUPPORTED, "too many chains");
  const uint32_t* dn = pl ? pl->n_chains : nullptr;
  int64_t *dq = nullptr, *dt = nullptr;
  SEDEF_TRY(upload_offsets(ctx, pl, h_qoff, nqseq, h_toff, ntseq, &dq, &dt));
  uint64_t* key = (uint64_t*)ctx_alloc(ctx, (size_t)n * 8);
  uint64_t* skey = (uint64_t*)ctx_alloc(ctx, (size_t)n * 8);
  uint32_t* perm = (uint32_t*)ctx_alloc(ctx, (size_t)n * 4);
  int32_t* parent = (int32_t*)ctx_alloc(ctx, (size_t)n * 4);
  Agg* agg = (Agg*)ctx_alloc(ctx, (size_t)n * sizeof(Agg));
  uint32_t* flag = (uint32_t*)ctx_alloc(ctx, (size_t)(n + 1) * 4);
  uint32_t* pos = (uint32_t*)ctx_alloc(ctx, (size_t)(n + 1) * 4);
  if (!key || !skey || !perm || !parent || !agg || !flag || !pos) return SEDEF_ERR_OOM;
  const int g = grid_of(n, 256);
  SEDEF_KERNEL(ctx, "k_chain_keys", k_chain_keys<<<g, 256, 0, st>>>(chains, n, key, dn));
  SEDEF_TRY(radix_sort_u64(ctx, key, nullptr, skey, perm, n, 0, 33, dn));
  MergeArgs a;
  a.ch = chains;
  a.n = n;
  a.perm = perm;
  a.parent = parent;
  a.diag_max = D.diag_max;
  a.delta_g = D.delta_g;
  a.dn = dn;
  SEDEF_KERNEL(ctx, "k_merge_init", k_merge_init<<<g, 256, 0, st>>>(parent, n));
  SEDEF_KERNEL(ctx, "k_merge_link", k_merge_link<<<g, 256, 0, st>>>(a));
  SEDEF_KERNEL(ctx, "k_agg_init", k_agg_init<<<g, 256, 0, st>>>(agg, n));
  SEDEF_KERNEL(ctx, "k_merge_agg", k_merge_agg<<<g, 256, 0, st>>>(a, agg));
  SEDEF_KERNEL(ctx, "k_root_flags", k_root_flags<<<g, 256, 0, st>>>(parent, n, flag, dn));
  SEDEF_TRY(scan_exclusive_u32(ctx, flag, pos, n, pos + n));
  int64_t nc;
  const uint32_t* dnc = nullptr;
  if (pl) {
    nc = cap;
    dnc = pos + n;
    pl->n_cands = dnc;
    SEDEF_TRY(plan_check(ctx, pl, dnc, cap, 5));
    *ncands = cap;
  } else {
    uint32_t* h_tot = (uint32_t*)ctx_host(ctx, 8);
    if (!h_tot) return SEDEF_ERR_OOM;
    SEDEF_CUDA(cudaMemcpyAsync(h_tot, pos + n, 4, cudaMemcpyDeviceToHost, st));
    SEDEF_CUDA(cudaStreamSynchronize(st));
    nc = *h_tot;
    *ncands = nc;
    if (nc > cap) return fail(SEDEF_ERR_CAPACITY, "sedef_merge: candidate buffer too small");
  }
  if (nc == 0) return SEDEF_OK;
  sedef_cand_t* tmp = (sedef_cand_t*)ctx_alloc(ctx, (size_t)nc * sizeof(sedef_cand_t));
  uint64_t* ckey = (uint64_t*)ctx_alloc(ctx, (size_t)nc * 8);
  uint64_t* cskey = (uint64_t*)ctx_alloc(ctx, (size_t)nc * 8);
  uint32_t* cperm = (uint32_t*)ctx_alloc(ctx, (size_t)nc * 4);
  if (!tmp || !ckey || !cskey || !cperm) return SEDEF_ERR_OOM;
  SEDEF_KERNEL(ctx, "k_cand_emit", k_cand_emit<<<g, 256, 0, st>>>(a, agg, pos, tmp, ckey, nc));
  SEDEF_TRY(radix_sort_u64(ctx, ckey, nullptr, cskey, cperm, nc, 0, 64, dnc));
  SEDEF_KERNEL(ctx, "k_cand_final",
               k_cand_final<<<grid_of(nc, 256), 256, 0, st>>>(tmp, cperm, cskey, nc, dq, dt, cands,
                                                              dnc));
  if (pl) return SEDEF_OK;
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // namespace sedef
