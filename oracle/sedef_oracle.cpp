// SEDEF seeding-filter oracle: TEST INFRASTRUCTURE, not product code.
//
// A plain, slow, single-threaded CPU restatement of what the seeding filter
// computes, written from the paper (Numanagic et al., "Fast Characterization
// of Segmental Duplications in Genome Assemblies").  Only the tests, the
// smoke check and the benchmark's CPU-baseline leg may call it.  It shares no
// code, header, table or constant generator with the CUDA library: every
// definition below is written out again from the paper's text.
//
// Steps (each function cites the passage it restates):
//   pack      Section 2 (alphabet {A,C,G,T}), Section 3.2 (soft-masked bases)
//   hash      Section 2.2 (MinHash needs a random permutation of k-mers)
//   sketch    Section 2.2 (winnowing, rightmost k-mer on ties), Section 3.2
//             (seeding uses only k-mers with at least one unmasked base)
//   index     Section 3.1 (I_G: sorted unique (i, x); reverse index x -> [i])
//   filter    Section 2.2 (|W(X_i) ∩ W(X_j)| >= s*tau), Section 3.1 (rolling
//             over the candidate list C sorted by position), Section 2
//             (overlap of the two mates at most delta*n)
//   refine    Section 2.2 (winnowed MinHash estimate), Section 3.1 (keep the j
//             whose estimate is maximal and above tau)
//   chain     Section 3.3 (local chaining by sparse DP, gaps limited by l*delta_G)
//   merge     Section 3 (seeds grown into larger regions while similar),
//             restated at chain granularity
//   tau       Section 3.1 closed form tau >= (1-dG)/(1+dG) / (2 e^{k dM} - 1)
//   extend    Section 3.2 (seeds grown into potential SD regions while the
//             winnowed MinHash estimate stays >= tau; all k-mers)
//   chain2    Section 3.3 (two-tier local chaining of exact seeds of at
//             least 11 bases inside the potential SD regions)
//
// Readings where the paper is silent are listed in the design notes; the code
// below states each one where it is used.
//
// Results are returned as flat int64 row tables (opaque handle + length +
// copy + free) so that the Python test harness can read them with ctypes.

#include <algorithm>
#include <cctype>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

namespace {

const uint64_t kInf = ~0ull;  // hash of an ineligible k-mer (never selected)

// Parameters, passed from Python as a flat int64 array (doubles bit-cast).
struct Par {
  int64_t k, w, n, step, max_occ, self_mode, gap_max, diag_max, min_unmasked;
  double delta_m, delta_g;
};

Par read_par(const int64_t* p) {
  Par r;
  r.k = p[0];
  r.w = p[1];
  r.n = p[2];
  r.step = p[3];
  r.max_occ = p[4];
  r.self_mode = p[5];
  r.gap_max = p[6];
  r.diag_max = p[7];
  r.min_unmasked = p[8];
  std::memcpy(&r.delta_m, &p[9], 8);
  std::memcpy(&r.delta_g, &p[10], 8);
  return r;
}

struct Table {
  int64_t ncols = 0;
  std::vector<int64_t> v;
  void row(std::initializer_list<int64_t> xs) { v.insert(v.end(), xs); }
};

// One sketch record: the minimizer's hash, its start position (global
// coordinate in the concatenated input) and its strand (1 when the reverse
// complement is the canonical form).
struct Rec {
  uint64_t h;
  int64_t pos;
  int sigma;
};

// ---- Section 2: alphabet; Section 3.2: soft-masking ------------------------
// A/a=0, C/c=1, G/g=2, T/t=3; any other byte is N.  A base is masked when it
// is a lowercase letter.
bool decode(uint8_t b, int* code, bool* masked) {
  *masked = (b >= 'a' && b <= 'z');
  switch (b) {
    case 'A': case 'a': *code = 0; return true;
    case 'C': case 'c': *code = 1; return true;
    case 'G': case 'g': *code = 2; return true;
    case 'T': case 't': *code = 3; return true;
    default: *code = 0; return false;
  }
}

// ---- Section 2.2: a collision-free hash, i.e. a permutation of the 4^k codes.
// Reading: a composition of invertible steps on 2k-bit integers -- xor with a
// right shift (shift >= 1) and multiplication by an odd constant, both taken
// modulo 2^(2k).  Each step is a bijection, so the composition is one.
uint64_t hash_code(uint64_t x, int k) {
  const uint64_t M = (k >= 32) ? ~0ull : ((1ull << (2 * k)) - 1);
  x &= M;
  x ^= x >> k;
  x = (x * 0x9E3779B97F4A7C15ull) & M;
  x ^= x >> (k - 1);
  x = (x * 0xD6E8FEB86659FD93ull) & M;
  x ^= x >> k;
  return x;
}

// Seq boundaries as a list of [start, end) in the concatenated coordinates.
std::vector<std::pair<int64_t, int64_t>> seq_ranges(const int64_t* off, int nseq) {
  std::vector<std::pair<int64_t, int64_t>> r;
  for (int s = 0; s < nseq; ++s) r.push_back({off[s], off[s + 1]});
  return r;
}

int seq_of(const std::vector<std::pair<int64_t, int64_t>>& rs, int64_t pos) {
  for (size_t s = 0; s < rs.size(); ++s)
    if (pos >= rs[s].first && pos < rs[s].second) return (int)s;
  return -1;
}

// ---- Section 3.1: threshold tau from the SD error model --------------------
double tau_of(int64_t k, double dm, double dg) {
  return (1.0 - dg) / (1.0 + dg) * (1.0 / (2.0 * std::exp((double)k * dm) - 1.0));
}

// m[s]: the least integer m with m >= tau*s - 1e-9 (shared minimizers needed
// for a sketch of s distinct hashes; Section 2.2, |W ∩ W'| >= s*tau).
int64_t min_shared(double tau, int64_t s) {
  int64_t m = 0;
  while ((double)m < tau * (double)s - 1e-9) ++m;
  return m;
}

// Records are sorted by position; [first, last) indexes those with pos in [lo, hi].
std::pair<size_t, size_t> pos_range(const std::vector<Rec>& recs, int64_t lo, int64_t hi) {
  auto cmp = [](const Rec& r, int64_t p) { return r.pos < p; };
  size_t a = std::lower_bound(recs.begin(), recs.end(), lo, cmp) - recs.begin();
  size_t b = std::lower_bound(recs.begin(), recs.end(), hi + 1, cmp) - recs.begin();
  return {a, std::max(a, b)};
}

// Window k-mer content: distinct hashes of the minimizers with start in
// [lo, hi], each with the set of strands it occurs with (bit sigma).
std::map<uint64_t, int> window_hashes(const std::vector<Rec>& recs, int64_t lo, int64_t hi) {
  std::map<uint64_t, int> w;
  auto r = pos_range(recs, lo, hi);
  for (size_t a = r.first; a < r.second; ++a) w[recs[a].h] |= 1 << recs[a].sigma;
  return w;
}

// Valid target window starts j for query window i (Section 2 overlap rule in
// self mode; windows lie inside one sequence).  In self mode only pairs with
// the target after the query are searched (each unordered pair once), and
// the mates may overlap by at most floor(delta*n) bases.  self_mode 2 treats
// every sequence as an independent genome: targets only on the query's own
// sequence.
std::vector<std::pair<int64_t, int64_t>> valid_targets(
    const std::vector<std::pair<int64_t, int64_t>>& tr, int qseq, int64_t i, const Par& P) {
  std::vector<std::pair<int64_t, int64_t>> v;
  const int64_t overlap = (int64_t)std::floor((P.delta_m + P.delta_g) * (double)P.n);
  for (size_t u = 0; u < tr.size(); ++u) {
    int64_t lo = tr[u].first, hi = tr[u].second - P.n;
    if (hi < lo) continue;
    if (P.self_mode) {
      if ((int)u < qseq) continue;
      if ((int)u == qseq) lo = std::max(lo, i + P.n - overlap);
      if (P.self_mode == 2 && (int)u != qseq) continue;  // each sequence on its own
    }
    if (lo <= hi) v.push_back({lo, hi});
  }
  return v;
}

std::vector<Rec> rows_to_recs(const int64_t* rows, int64_t nrec) {
  std::vector<Rec> v(nrec);
  for (int64_t a = 0; a < nrec; ++a) v[a] = {(uint64_t)rows[3 * a], rows[3 * a + 1], (int)rows[3 * a + 2]};
  return v;
}

// Target postings: hash -> positions with strands (the reverse index).  With
// `only`, postings are kept for those hashes alone (a caller that looks up
// no other hash gets the same answers with less memory).
std::map<uint64_t, std::vector<std::pair<int64_t, int>>> postings_of(
    const std::vector<Rec>& t, const std::set<uint64_t>* only = nullptr) {
  std::map<uint64_t, std::vector<std::pair<int64_t, int>>> m;
  for (const Rec& r : t)
    if (!only || only->count(r.h)) m[r.h].push_back({r.pos, r.sigma});
  for (auto& kv : m) std::sort(kv.second.begin(), kv.second.end());
  return m;
}

// Winnowed MinHash estimate (Section 2.2) for query window content wq (s
// distinct hashes) against the current target window content wt: hash ->
// (records in the window, records that are shared-compatible).  U = the s
// smallest hashes of W_Q u W_T; est = |{h in U : h in W_Q and shared}|;
// den = |U|.
void estimate(const std::map<uint64_t, int>& wq,
              const std::map<uint64_t, std::pair<int64_t, int64_t>>& wt, int64_t* est,
              int64_t* den) {
  const int64_t s = (int64_t)wq.size();
  auto a = wq.begin();
  auto b = wt.begin();
  int64_t taken = 0, e = 0;
  while (taken < s && (a != wq.end() || b != wt.end())) {
    uint64_t h;
    if (b == wt.end() || (a != wq.end() && a->first <= b->first)) h = a->first;
    else h = b->first;
    const bool in_q = (a != wq.end() && a->first == h);
    const bool shared = in_q && b != wt.end() && b->first == h && b->second.second > 0;
    if (shared) ++e;
    ++taken;
    if (a != wq.end() && a->first == h) ++a;
    if (b != wt.end() && b->first == h) ++b;
  }
  *est = e;
  *den = taken;
}

// Colinear chaining DP of Section 3.3 over anchors (p, t') sorted ascending.
// f[a] = 1 + max f[b] over predecessors b < a with both gaps in (0, gap_max]
// and |gap_p - gap_t| <= diag_max; pred[a] = that b (the largest f, then
// the largest index), -1 when a starts its chain.  Returns the chain end:
// the largest f, then the smallest index.  A >= 1.
int64_t chain_dp(const std::vector<std::pair<int64_t, int64_t>>& anc, int64_t gap_max,
                 int64_t diag_max, std::vector<int64_t>* f_out, std::vector<int64_t>* pred_out) {
  const int64_t A = (int64_t)anc.size();
  std::vector<int64_t>& f = *f_out;
  std::vector<int64_t>& pred = *pred_out;
  f.assign(A, 1);
  pred.assign(A, -1);
  for (int64_t a = 0; a < A; ++a)
    for (int64_t b = 0; b < a; ++b) {
      const int64_t dp = anc[a].first - anc[b].first, dt = anc[a].second - anc[b].second;
      if (dp <= 0 || dt <= 0 || dp > gap_max || dt > gap_max) continue;
      if (std::llabs(dp - dt) > diag_max) continue;
      if (pred[a] < 0 || f[b] + 1 > f[a] || (f[b] + 1 == f[a] && b > pred[a])) {
        f[a] = f[b] + 1;
        pred[a] = b;
      }
    }
  int64_t end = 0;
  for (int64_t a = 1; a < A; ++a)
    if (f[a] > f[end]) end = a;
  return end;
}

}  // namespace

extern "C" {

void* orc_table_new() { return new Table(); }
int64_t orc_table_rows(void* t) {
  Table* T = (Table*)t;
  return T->ncols ? (int64_t)T->v.size() / T->ncols : 0;
}
int64_t orc_table_cols(void* t) { return ((Table*)t)->ncols; }
void orc_table_copy(void* t, int64_t* dst) {
  Table* T = (Table*)t;
  if (!T->v.empty()) std::memcpy(dst, T->v.data(), T->v.size() * 8);
}
void orc_table_free(void* t) { delete (Table*)t; }

// ---- a1 pack (Section 2 alphabet, Section 3.2 masking) ---------------------
// Base p goes to bits 2*(p%16) of packed[p/16]; mask bit p%32 of mask[p/32]
// is set for a lowercase base; nbits likewise for a non-ACGT byte.
void orc_pack(const uint8_t* seq, int64_t n, uint32_t* packed, uint32_t* mask, uint32_t* nbits) {
  for (int64_t w = 0; w < (n + 15) / 16; ++w) packed[w] = 0;
  for (int64_t w = 0; w < (n + 31) / 32; ++w) mask[w] = nbits[w] = 0;
  for (int64_t p = 0; p < n; ++p) {
    int code;
    bool masked;
    bool ok = decode(seq[p], &code, &masked);
    packed[p / 16] |= (uint32_t)code << (2 * (p % 16));
    if (masked) mask[p / 32] |= 1u << (p % 32);
    if (!ok) nbits[p / 32] |= 1u << (p % 32);
  }
}

uint64_t orc_hash(uint64_t code, int k) { return hash_code(code, k); }

void orc_hash_all(int k, uint64_t* out) {
  const uint64_t N = 1ull << (2 * k);
  for (uint64_t x = 0; x < N; ++x) out[x] = hash_code(x, k);
}

double orc_tau(int64_t k, double dm, double dg) { return tau_of(k, dm, dg); }

void orc_mtable(int64_t k, double dm, double dg, int64_t smax, int64_t* out) {
  double tau = tau_of(k, dm, dg);
  for (int64_t s = 0; s <= smax; ++s) out[s] = min_shared(tau, s);
}

// ---- a2 sketch: canonical k-mers + winnowing (Section 2.2, Section 3.2) -----
// Output rows (hash, pos, strand) sorted by pos.
// Sequences are independent (windows never cross a boundary), so with
// nthreads > 1 they are shared out to threads and their rows joined in
// sequence order; the result does not depend on nthreads.
static void sketch_one(const uint8_t* seq, int64_t st, int64_t en, const Par& P, Table* T);

void* orc_sketch(const uint8_t* seq, const int64_t* off, int nseq, const int64_t* par,
                 int nthreads) {
  Par P = read_par(par);
  Table* T = new Table();
  T->ncols = 3;
  if (nthreads < 1) nthreads = 1;
  std::vector<Table> part(nseq);
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int s; (s = next.fetch_add(1)) < nseq;) {
      part[s].ncols = 3;
      sketch_one(seq, off[s], off[s + 1], P, &part[s]);
    }
  };
  std::vector<std::thread> th;
  for (int x = 1; x < nthreads; ++x) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  for (auto& p : part) {
    T->v.insert(T->v.end(), p.v.begin(), p.v.end());
    std::vector<int64_t>().swap(p.v);
  }
  return T;
}

static void sketch_one(const uint8_t* seq, int64_t st, int64_t en, const Par& P, Table* T) {
  {
    const int64_t nk = en - st - P.k + 1;  // k-mer starts inside the sequence
    if (nk <= 0) return;
    std::vector<uint64_t> h(nk);
    std::vector<int> sig(nk);
    for (int64_t a = 0; a < nk; ++a) {
      uint64_t f = 0, r = 0;
      bool ok = true;
      int64_t unmasked = 0;
      for (int64_t x = 0; x < P.k; ++x) {
        int code;
        bool masked;
        if (!decode(seq[st + a + x], &code, &masked)) ok = false;
        if (!masked) ++unmasked;
        f = f * 4 + (uint64_t)code;                       // first base most significant
        r = r + ((uint64_t)(3 - code) << (2 * x));        // complement, reversed order
      }
      // eligible: no N, at least min_unmasked unmasked bases, strand defined
      if (!ok || unmasked < P.min_unmasked || f == r) {
        h[a] = kInf;
        sig[a] = 0;
      } else {
        h[a] = hash_code(std::min(f, r), (int)P.k);
        sig[a] = (r < f) ? 1 : 0;
      }
    }
    std::set<int64_t> chosen;
    for (int64_t q = 0; q + P.w <= nk; ++q) {  // every full window of w k-mer starts
      uint64_t best = kInf;
      int64_t arg = -1;
      for (int64_t x = q; x < q + P.w; ++x)
        if (h[x] != kInf && h[x] <= best) {  // '<=' keeps the rightmost minimum
          best = h[x];
          arg = x;
        }
      if (arg >= 0) chosen.insert(arg);
    }
    for (int64_t a : chosen) T->row({(int64_t)h[a], st + a, sig[a]});
  }
}

// ---- a3 index: I_G sorted by (hash, position) plus offsets (Section 3.1) ----
// off_out has 4^k + 1 entries: off[x] = number of records with hash < x.
void* orc_index(const int64_t* rows, int64_t nrec, int k, uint32_t* off_out) {
  std::vector<Rec> v = rows_to_recs(rows, nrec);
  std::sort(v.begin(), v.end(), [](const Rec& a, const Rec& b) {
    return std::tie(a.h, a.pos) < std::tie(b.h, b.pos);
  });
  const uint64_t N = 1ull << (2 * k);
  std::vector<int64_t> cnt(N + 1, 0);
  for (const Rec& r : v) cnt[r.h + 1]++;
  for (uint64_t x = 0; x < N; ++x) cnt[x + 1] += cnt[x];
  for (uint64_t x = 0; x <= N; ++x) off_out[x] = (uint32_t)cnt[x];
  Table* T = new Table();
  T->ncols = 3;
  for (const Rec& r : v) T->row({(int64_t)r.h, r.pos, r.sigma});
  return T;
}

// ---- a4/a5/a6 filter + refine (Section 2.2, Section 3.1, Section 2) ---------
// For every query window i (start of each sequence, then every `step` bases,
// while i + n <= sequence end) and each relative strand o:
//   shared_o(j) = number of distinct hashes h of W(G_i) that occur in the
//   target window [j, j+n-k] with relative strand o;
//   j passes when it is a valid target window and shared_o(j) >= m[s];
//   each maximal run of passing j is one output row, with its refined seed.
// The rolling follows Section 3.1: the candidates C are sorted by position and
// the window slides right; every hit at position t enters at j = t-(n-k) and
// leaves at j = t+1, and the shared count is constant between such events.
//
// Rows: i, o, j_a, j_b, max_shared, j_at_max, s, m, est, j_star, den, keep.
// `windows` (optional, nwin >= 0) restricts the query windows to that list of
// starts; nwin < 0 means all windows.  dense != 0 evaluates the refine
// estimate at every j of the run instead of at its breakpoints.
// Windows are independent: with nthreads > 1 contiguous blocks of windows
// go to threads and their rows are joined in window order (the result does
// not depend on nthreads).
void* orc_filter(const int64_t* qrows, int64_t nq, const int64_t* qoff, int nqseq,
                 const int64_t* trows, int64_t nt, const int64_t* toff, int ntseq,
                 const int64_t* par, const int64_t* windows, int64_t nwin, int dense,
                 int nthreads) {
  Par P = read_par(par);
  std::vector<Rec> qrecs = rows_to_recs(qrows, nq);
  std::vector<Rec> trecs = rows_to_recs(trows, nt);
  auto qr = seq_ranges(qoff, nqseq);
  auto tr = seq_ranges(toff, ntseq);
  const double tau = tau_of(P.k, P.delta_m, P.delta_g);
  const int64_t span = P.n - P.k;  // a window's k-mer starts are [j, j+span]

  std::vector<int64_t> starts;
  if (nwin >= 0) {
    starts.assign(windows, windows + nwin);
  } else {
    for (auto& r : qr)
      for (int64_t i = r.first; i + P.n <= r.second; i += P.step) starts.push_back(i);
  }
  // postings of the hashes the windows hold (the only ones looked up)
  std::set<uint64_t> needed;
  for (int64_t i : starts)
    for (auto& kv : window_hashes(qrecs, i, i + span)) needed.insert(kv.first);
  auto post = postings_of(trecs, &needed);

  auto one = [&](int64_t i, Table* T) {
    const int qseq = seq_of(qr, i);
    std::map<uint64_t, int> wq = window_hashes(qrecs, i, i + span);
    if (P.max_occ > 0) {  // optional occurrence cap (off by default)
      for (auto it = wq.begin(); it != wq.end();) {
        auto p = post.find(it->first);
        int64_t occ = (p == post.end()) ? 0 : (int64_t)p->second.size();
        if (occ > P.max_occ) it = wq.erase(it); else ++it;
      }
    }
    const int64_t s = (int64_t)wq.size();
    if (s == 0) return;
    const int64_t m = min_shared(tau, s);
    auto valid = valid_targets(tr, qseq, i, P);

    for (int o = 0; o < 2; ++o) {
      // candidate list C for this strand: (j, +1/-1, hash) events
      std::vector<std::tuple<int64_t, int, uint64_t>> ev;
      for (auto& kv : wq) {
        auto p = post.find(kv.first);
        if (p == post.end()) continue;
        for (auto& ts : p->second) {
          // self mode: the query window's own positions are not copies
          if (P.self_mode && ts.first >= i && ts.first <= i + span) continue;
          if (kv.second >> (ts.second ^ o) & 1) {  // some query strand sq with sq^st == o
            ev.push_back({ts.first - span, +1, kv.first});
            ev.push_back({ts.first + 1, -1, kv.first});
          }
        }
      }
      std::sort(ev.begin(), ev.end());
      std::map<uint64_t, int64_t> cnt;
      int64_t shared = 0;
      bool in_run = false;
      int64_t ja = 0, jb = 0, mx = 0, jmx = 0;
      auto close_run = [&]() {
        if (!in_run) return;
        // refine (Section 3.1): roll the target window over the run, keeping
        // its minimizers in an ordered map (the paper's set L), and evaluate
        // the estimate at j_a and at every j in (j_a, j_b] where a target
        // minimizer enters or leaves the window -- the estimate only changes
        // there -- or at every j when dense.  In self mode a target record
        // inside the query window's own span is not shared-compatible.
        std::map<uint64_t, std::pair<int64_t, int64_t>> wt;
        auto rg = pos_range(trecs, ja, jb + span);
        auto compatible = [&](const Rec& r) {
          if (P.self_mode && r.pos >= i && r.pos <= i + span) return false;
          auto q = wq.find(r.h);
          return q != wq.end() && ((q->second >> (r.sigma ^ o)) & 1);
        };
        auto enter = [&](const Rec& r) {
          auto& c = wt[r.h];
          c.first += 1;
          if (compatible(r)) c.second += 1;
        };
        auto leave = [&](const Rec& r) {
          auto it = wt.find(r.h);
          it->second.first -= 1;
          if (compatible(r)) it->second.second -= 1;
          if (it->second.first == 0) wt.erase(it);
        };
        size_t in = rg.first, out = rg.first;  // next record to enter / to leave
        int64_t j = ja;
        while (in < rg.second && trecs[in].pos <= j + span) enter(trecs[in++]);
        int64_t best = -1, jstar = ja, dstar = 0;
        while (true) {
          int64_t e, d;
          estimate(wq, wt, &e, &d);
          if (e > best) {
            best = e;
            jstar = j;
            dstar = d;
          }
          int64_t nx;
          if (dense) {
            nx = j + 1;
          } else {
            nx = INT64_MAX;
            if (in < rg.second) nx = std::min(nx, trecs[in].pos - span);
            if (out < in) nx = std::min(nx, trecs[out].pos + 1);
          }
          if (nx > jb) break;
          j = nx;
          while (out < in && trecs[out].pos < j) leave(trecs[out++]);
          while (in < rg.second && trecs[in].pos <= j + span) enter(trecs[in++]);
        }
        const int64_t keep = (best >= min_shared(tau, dstar)) ? 1 : 0;
        T->row({i, o, ja, jb, mx, jmx, s, m, best, jstar, dstar, keep});
        in_run = false;
      };
      size_t a = 0;
      while (a < ev.size()) {
        const int64_t j = std::get<0>(ev[a]);
        while (a < ev.size() && std::get<0>(ev[a]) == j) {
          auto& e = ev[a];
          int64_t& c = cnt[std::get<2>(e)];
          if (std::get<1>(e) > 0) {
            if (c++ == 0) ++shared;
          } else {
            if (--c == 0) --shared;
          }
          ++a;
        }
        const int64_t jend = (a < ev.size()) ? std::get<0>(ev[a]) - 1 : j;  // constant on [j, jend]
        if (a >= ev.size()) break;  // after the last event nothing is covered
        for (auto& vr : valid) {
          int64_t lo = std::max(j, vr.first), hi = std::min(jend, vr.second);
          if (lo > hi) continue;
          if (shared >= m) {
            if (in_run && lo == jb + 1) {
              jb = hi;
            } else {
              close_run();
              in_run = true;
              ja = lo;
              jb = hi;
              mx = -1;
            }
            if (shared > mx) {
              mx = shared;
              jmx = lo;
            }
          } else {
            close_run();
          }
        }
      }
      close_run();
    }
  };
  Table* T = new Table();
  T->ncols = 12;
  if (nthreads < 1) nthreads = 1;
  const int64_t nw = (int64_t)starts.size();
  std::vector<Table> part(nthreads);
  std::vector<std::thread> th;
  for (int x = 0; x < nthreads; ++x) {
    part[x].ncols = 12;
    auto work = [&, x]() {
      const int64_t lo = nw * x / nthreads, hi = nw * (x + 1) / nthreads;
      for (int64_t w = lo; w < hi; ++w) one(starts[w], &part[x]);
    };
    if (x + 1 < nthreads) th.emplace_back(work); else work();
  }
  for (auto& t : th) t.join();
  for (auto& pt : part) T->v.insert(T->v.end(), pt.v.begin(), pt.v.end());
  return T;
}

// ---- a7 chain: colinear chaining of seed anchors (Section 3.3) -------------
// For every kept run row (i, o, j_a, j_b, ..., s) the anchors are the pairs
// (p, t) of a query-window minimizer p in [i, i+n-k] and a target minimizer t
// in [j_a, j_b+n-k] with equal hash and strands differing by o.  For o = 1
// the target axis is reversed (t' = j_b+n-k - t) so that a chain is increasing
// on both axes.  f(a) = 1 + max f(b) over predecessors b with p_b < p_a,
// t'_b < t'_a, both gaps <= gap_max and |gap_p - gap_t| <= diag_max.
// Ties: the predecessor with the largest f, then the largest sorted index; the
// chain end with the largest f, then the smallest sorted index.  A chain is
// kept when f >= m[s].
// Rows: i, o, qseq, q0, q1, tseq, t0, t1, score, s  (q/t in global coordinates).
void* orc_chain(const int64_t* runs, int64_t nruns, int64_t run_cols,
                const int64_t* qrows, int64_t nq, const int64_t* qoff, int nqseq,
                const int64_t* trows, int64_t nt, const int64_t* toff, int ntseq,
                const int64_t* par) {
  Par P = read_par(par);
  std::vector<Rec> qrecs = rows_to_recs(qrows, nq);
  std::vector<Rec> trecs = rows_to_recs(trows, nt);
  // postings are needed only for the optional occurrence cap
  std::map<uint64_t, std::vector<std::pair<int64_t, int>>> post;
  if (P.max_occ > 0) post = postings_of(trecs);
  auto qr = seq_ranges(qoff, nqseq);
  auto tr = seq_ranges(toff, ntseq);
  const double tau = tau_of(P.k, P.delta_m, P.delta_g);
  const int64_t span = P.n - P.k;
  Table* T = new Table();
  T->ncols = 10;
  for (int64_t r = 0; r < nruns; ++r) {
    const int64_t* R = runs + r * run_cols;
    const int64_t i = R[0], o = R[1], ja = R[2], jb = R[3], s = R[6], keep = R[11];
    if (!keep) continue;
    std::map<uint64_t, int> wq = window_hashes(qrecs, i, i + span);
    const int64_t tref = jb + span;
    std::vector<std::tuple<int64_t, int64_t, int64_t>> anc;  // (p, t', t)
    auto qrg = pos_range(qrecs, i, i + span);
    auto trg = pos_range(trecs, ja, tref);
    for (size_t x = qrg.first; x < qrg.second; ++x) {
      const Rec& q = qrecs[x];
      if (P.max_occ > 0) {
        auto p = post.find(q.h);
        if (p != post.end() && (int64_t)p->second.size() > P.max_occ) continue;
      }
      for (size_t y = trg.first; y < trg.second; ++y) {
        const Rec& t = trecs[y];
        if (t.h != q.h || (q.sigma ^ t.sigma) != o) continue;
        if (P.self_mode && t.pos >= i && t.pos <= i + span) continue;  // same position
        anc.push_back({q.pos, o ? tref - t.pos : t.pos, t.pos});
      }
    }
    std::sort(anc.begin(), anc.end());
    const int64_t A = (int64_t)anc.size();
    if (A == 0) continue;
    std::vector<std::pair<int64_t, int64_t>> pt(A);
    for (int64_t a = 0; a < A; ++a) pt[a] = {std::get<0>(anc[a]), std::get<1>(anc[a])};
    std::vector<int64_t> f, pred;
    const int64_t end = chain_dp(pt, P.gap_max, P.diag_max, &f, &pred);
    const int64_t score = f[end];
    if (score < min_shared(tau, s)) continue;
    int64_t q0 = INT64_MAX, q1 = -1, t0 = INT64_MAX, t1 = -1;
    for (int64_t a = end; a >= 0; a = pred[a]) {
      q0 = std::min(q0, std::get<0>(anc[a]));
      q1 = std::max(q1, std::get<0>(anc[a]) + P.k);
      t0 = std::min(t0, std::get<2>(anc[a]));
      t1 = std::max(t1, std::get<2>(anc[a]) + P.k);
    }
    T->row({i, o, (int64_t)seq_of(qr, i), q0, q1, (int64_t)seq_of(tr, ja), t0, t1, score, s});
  }
  return T;
}

// Chaining of one explicit anchor list (for pin tests): anchors are (p, t')
// rows; returns rows (p, t', f, pred) per anchor in sorted (p, t') order,
// computed by chain_dp, the DP orc_chain runs for every kept seed.
void* orc_chain_anchors(const int64_t* anchors, int64_t A, int64_t gap_max, int64_t diag_max) {
  std::vector<std::pair<int64_t, int64_t>> anc(A);
  for (int64_t a = 0; a < A; ++a) anc[a] = {anchors[2 * a], anchors[2 * a + 1]};
  std::sort(anc.begin(), anc.end());
  std::vector<int64_t> f, pred;
  if (A > 0) chain_dp(anc, gap_max, diag_max, &f, &pred);
  Table* T = new Table();
  T->ncols = 4;
  for (int64_t a = 0; a < A; ++a) T->row({anc[a].first, anc[a].second, f[a], pred[a]});
  return T;
}

// ---- merge chains into SD candidates ---------------------------------------
// Reading of Section 3 ("keep expanding both seed regions while similar") at
// chain granularity: chains a and b are linked when they have the same query
// sequence, target sequence and strand, their query intervals overlap or
// touch, their target intervals overlap or touch, and their diagonals differ
// by at most diag_max + ceil(delta_G * max(len_a, len_b)) (len = query span;
// diagonal t0 - q0 for o = 0, t1 + q0 for o = 1).  Candidates are the
// connected components: bounding boxes, summed scores and chain counts.
// Rows (sorted by q0, t0, o, q1, t1; global coordinates):
//   qseq, q0, q1, tseq, t0, t1, o, score, nchains
void* orc_merge(const int64_t* chains, int64_t nc, int64_t cols, const int64_t* par) {
  Par P = read_par(par);
  std::vector<int64_t> parent(nc);
  for (int64_t a = 0; a < nc; ++a) parent[a] = a;
  auto find = [&](int64_t x) {
    while (parent[x] != x) x = parent[x];
    return x;
  };
  auto diag = [&](const int64_t* c) { return c[1] == 0 ? c[6] - c[3] : c[7] + c[3]; };
  for (int64_t a = 0; a < nc; ++a)
    for (int64_t b = a + 1; b < nc; ++b) {
      const int64_t* A = chains + a * cols;
      const int64_t* B = chains + b * cols;
      if (A[1] != B[1] || A[2] != B[2] || A[5] != B[5]) continue;
      if (B[3] > A[4] || A[3] > B[4]) continue;  // query intervals overlap or touch
      if (B[6] > A[7] || A[6] > B[7]) continue;  // target intervals overlap or touch
      const int64_t len = std::max(A[4] - A[3], B[4] - B[3]);
      const int64_t slack = P.diag_max + (int64_t)std::ceil(P.delta_g * (double)len);
      if (std::llabs(diag(A) - diag(B)) > slack) continue;
      int64_t ra = find(a), rb = find(b);
      if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
    }
  std::map<int64_t, std::vector<int64_t>> comp;
  for (int64_t a = 0; a < nc; ++a) {
    const int64_t* A = chains + a * cols;
    int64_t r = find(a);
    auto it = comp.find(r);
    if (it == comp.end()) {
      comp[r] = {A[2], A[3], A[4], A[5], A[6], A[7], A[1], A[8], 1};
    } else {
      auto& c = it->second;
      c[1] = std::min(c[1], A[3]);
      c[2] = std::max(c[2], A[4]);
      c[4] = std::min(c[4], A[6]);
      c[5] = std::max(c[5], A[7]);
      c[7] += A[8];
      c[8] += 1;
    }
  }
  std::vector<std::vector<int64_t>> out;
  for (auto& kv : comp) out.push_back(kv.second);
  std::sort(out.begin(), out.end(), [](const std::vector<int64_t>& x, const std::vector<int64_t>& y) {
    return std::make_tuple(x[1], x[4], x[6], x[2], x[5], x[0], x[3], x[7], x[8]) <
           std::make_tuple(y[1], y[4], y[6], y[2], y[5], y[0], y[3], y[7], y[8]);
  });
  Table* T = new Table();
  T->ncols = 9;
  for (auto& c : out) T->v.insert(T->v.end(), c.begin(), c.end());
  return T;
}

// Exact k-mer set Jaccard of two substrings (Section 2.2 definition), used to
// pin the closed form J = c / (2t - c) of Section 3.1.
double orc_jaccard(const uint8_t* seq, int64_t i, int64_t j, int64_t n, int k) {
  std::set<std::vector<uint8_t>> X, Y;
  for (int64_t a = 0; a + k <= n; ++a) {
    X.insert(std::vector<uint8_t>(seq + i + a, seq + i + a + k));
    Y.insert(std::vector<uint8_t>(seq + j + a, seq + j + a + k));
  }
  int64_t inter = 0;
  for (auto& x : X) inter += Y.count(x);
  return (double)inter / (double)(X.size() + Y.size() - inter);
}

// ---- f3 q-gram filter (Section 3.2) -------------------------------------------
// Q(X, Y): the q-grams X and Y share, counted with multiplicity (for every
// q-gram the smaller of its two occurrence counts, summed).  Case does not
// matter; a q-gram holding a base other than ACGT is not counted.  For a
// seed (i, j*, o) X = G[i, i+n) and Y = G[j*, j*+n), reverse-complemented
// when o = 1.  Section 3.2's adapted q-gram lemma: a pair within the SD error
// model shares at least B = n (1 - delta_G - q delta_M) - (n p_G + 1)(q - 1)
// q-grams (n <= m); the pair passes when Q >= the least integer >= B - 1e-9.
// Rows per run: Q, pass (0, 0 for runs that are not kept seeds).
double orc_qgram_bound(int64_t n, int q, double delta_g, double delta_m, double p_gap) {
  return (double)n * (1.0 - delta_g - (double)q * delta_m) -
         ((double)n * p_gap + 1.0) * (double)(q - 1);
}

static std::string upper_window(const uint8_t* seq, int64_t a, int64_t n, bool revcomp) {
  std::string x(seq + a, seq + a + n);
  for (char& c : x) c = (char)std::toupper((unsigned char)c);
  if (revcomp) {
    std::reverse(x.begin(), x.end());
    for (char& c : x) {
      switch (c) {
        case 'A': c = 'T'; break;
        case 'C': c = 'G'; break;
        case 'G': c = 'C'; break;
        case 'T': c = 'A'; break;
        default: c = 'N';
      }
    }
  }
  return x;
}

static std::map<std::string, int64_t> qgram_counts(const std::string& x, int q) {
  std::map<std::string, int64_t> c;
  for (size_t a = 0; a + q <= x.size(); ++a) {
    std::string g = x.substr(a, q);
    if (g.find_first_not_of("ACGT") != std::string::npos) continue;
    c[g] += 1;
  }
  return c;
}

int64_t orc_qgram_shared(const uint8_t* seq, int64_t i, int64_t j, int64_t n, int o, int q) {
  auto cx = qgram_counts(upper_window(seq, i, n, false), q);
  auto cy = qgram_counts(upper_window(seq, j, n, o != 0), q);
  int64_t shared = 0;
  for (auto& kv : cx) {
    auto it = cy.find(kv.first);
    if (it != cy.end()) shared += std::min(kv.second, it->second);
  }
  return shared;
}

void* orc_qgram(const uint8_t* seq, const int64_t* runs, int64_t nruns, int64_t run_cols,
                const int64_t* par, int q, double p_gap) {
  Par P = read_par(par);
  const double B = orc_qgram_bound(P.n, q, P.delta_g, P.delta_m, p_gap);
  int64_t need = (int64_t)std::ceil(B - 1e-9);
  while ((double)need < B - 1e-9) ++need;
  while ((double)(need - 1) >= B - 1e-9) --need;
  if (need < 0) need = 0;
  Table* T = new Table();
  T->ncols = 2;
  for (int64_t r = 0; r < nruns; ++r) {
    const int64_t* R = runs + r * run_cols;
    const int64_t i = R[0], o = R[1], jstar = R[9], keep = R[11];
    if (!keep) {
      T->row({0, 0});
      continue;
    }
    const int64_t Q = orc_qgram_shared(seq, i, jstar, P.n, (int)o, q);
    T->row({Q, Q >= need ? 1 : 0});
  }
  return T;
}

}  // extern "C"

// ---- f1 SD extension: seeds grown into potential SD regions (Section 3.2) --
// For every kept seed (i, j*, o) the query region starts as [i, i+n) and the
// target region as [j*, j*+n).  W_Q and W_T are the minimizers of the
// extension sketch (all k-mers, masked ones included: Section 3.2, last
// paragraph) whose k-mer span lies inside the region.  The regions grow by
// one base per step on each side (n and m increase together); for o = 1 the
// target grows at the opposite end, since its copy is reverse-complemented.
// After every step the winnowed MinHash estimate is taken as in Section 2.2,
// with s = |W_Q| (distinct hashes): U = the s smallest hashes of W_Q u W_T,
// est = hashes of U in W_Q and in W_T with relative strand o; the step is
// kept while est >= m(s) = the least integer >= tau*s - 1e-9.  Growth stops
// at the first step whose estimate falls below, that would leave a
// sequence, that would make a region longer than max_len, or (query and
// target on one sequence of a self search) that would make the two regions
// overlap more than they already do.  Forward growth (right ends) runs first,
// then backward growth (left ends) from its result.  In a self search a
// target minimizer inside the query region's own k-mer span is the same
// genome position, so it joins the union but is never shared.
// Rows per kept run (global coordinates):
//   i, o, j_star, qa, qb, ta, tb, est, den
namespace {

struct ExtState {
  std::map<uint64_t, int> q;                    // hash -> query strand mask
  std::map<uint64_t, std::pair<int, int>> t;    // hash -> (target records, shareable strand mask)
};

// est and den of the current regions (Section 2.2 estimator, s = |W_Q|).
void ext_estimate(const ExtState& S, int o, int64_t* est, int64_t* den) {
  const int64_t s = (int64_t)S.q.size();
  auto a = S.q.begin();
  auto b = S.t.begin();
  int64_t taken = 0, e = 0;
  while (taken < s && (a != S.q.end() || b != S.t.end())) {
    uint64_t h;
    if (b == S.t.end() || (a != S.q.end() && a->first <= b->first)) h = a->first;
    else h = b->first;
    const bool in_q = a != S.q.end() && a->first == h;
    const bool in_t = b != S.t.end() && b->first == h;
    if (in_q && in_t) {
      const int qm = a->second, tm = b->second.second;
      // some query strand sq and target strand st with sq ^ st == o
      const int tm_o = o ? (((tm & 1) << 1) | ((tm >> 1) & 1)) : tm;
      if (qm & tm_o) ++e;
    }
    ++taken;
    if (in_q) ++a;
    if (in_t) ++b;
  }
  *est = e;
  *den = taken;
}

// The record starting at `pos`, if the extension sketch has one there.
const Rec* rec_at(const std::vector<Rec>& recs, int64_t pos) {
  auto it = std::lower_bound(recs.begin(), recs.end(), pos,
                             [](const Rec& r, int64_t p) { return r.pos < p; });
  return (it != recs.end() && it->pos == pos) ? &*it : nullptr;
}

}  // namespace

extern "C" {

void* orc_extend(const int64_t* runs, int64_t nruns, int64_t run_cols, const int64_t* qrows,
                 int64_t nq, const int64_t* qoff, int nqseq, const int64_t* trows, int64_t nt,
                 const int64_t* toff, int ntseq, const int64_t* par, int64_t max_len,
                 int nthreads) {
  Par P = read_par(par);
  std::vector<Rec> qrecs = rows_to_recs(qrows, nq);
  std::vector<Rec> trecs = rows_to_recs(trows, nt);
  auto qr = seq_ranges(qoff, nqseq);
  auto tr = seq_ranges(toff, ntseq);
  const double tau = tau_of(P.k, P.delta_m, P.delta_g);
  const int64_t k = P.k;
  std::vector<int64_t> kept;
  for (int64_t r = 0; r < nruns; ++r)
    if (runs[r * run_cols + 11]) kept.push_back(r);
  const int64_t nk = (int64_t)kept.size();
  std::vector<std::vector<int64_t>> out(nk);

  auto one = [&](int64_t x) {
    const int64_t* R = runs + kept[x] * run_cols;
    const int64_t i = R[0], o = R[1], js = R[9];
    const int qs = seq_of(qr, i), ts = seq_of(tr, js);
    const int64_t qlo = qr[qs].first, qhi = qr[qs].second;
    const int64_t tlo = tr[ts].first, thi = tr[ts].second;
    const bool same = P.self_mode && qs == ts;
    int64_t qa = i, qb = i + P.n, ta = js, tb = js + P.n;
    ExtState S;
    // a target record is shareable unless, in a self search, it lies in the
    // query region's own k-mer span
    auto add_q = [&](const Rec& r) { S.q[r.h] |= 1 << r.sigma; };
    auto add_t = [&](const Rec& r, int64_t qa_, int64_t qb_) {
      auto& c = S.t[r.h];
      c.first += 1;
      if (!(P.self_mode && r.pos >= qa_ && r.pos <= qb_ - k)) c.second |= 1 << r.sigma;
    };
    auto overlap = [&](int64_t a0, int64_t a1, int64_t b0, int64_t b1) -> int64_t {
      return std::max<int64_t>(0, std::min(a1, b1) - std::max(a0, b0));
    };
    {
      auto rq = pos_range(qrecs, qa, qb - k);
      for (size_t y = rq.first; y < rq.second; ++y) add_q(qrecs[y]);
      auto rt = pos_range(trecs, ta, tb - k);
      for (size_t y = rt.first; y < rt.second; ++y) add_t(trecs[y], qa, qb);
    }
    int64_t est = 0, den = 0;
    ext_estimate(S, (int)o, &est, &den);
    const bool start_ok = est >= min_shared(tau, den);
    for (int dir = 0; dir < 2 && start_ok; ++dir) {  // 0: right ends, 1: left ends
      while (true) {
        int64_t nqa = qa, nqb = qb, nta = ta, ntb = tb;
        if (dir == 0) {
          nqb = qb + 1;
          if (o == 0) ntb = tb + 1; else nta = ta - 1;
        } else {
          nqa = qa - 1;
          if (o == 0) nta = ta - 1; else ntb = tb + 1;
        }
        if (nqa < qlo || nqb > qhi || nta < tlo || ntb > thi) break;
        if (nqb - nqa > max_len || ntb - nta > max_len) break;
        if (same && overlap(nqa, nqb, nta, ntb) > overlap(qa, qb, ta, tb)) break;
        // the k-mers that now fit in each region; their old entries are kept
        // so that a failed step can be taken back
        const Rec* nqr = dir == 0 ? rec_at(qrecs, nqb - k) : rec_at(qrecs, nqa);
        if (!(nqr && nqr->pos >= nqa && nqr->pos <= nqb - k)) nqr = nullptr;
        const Rec* ntr = (ntb != tb) ? rec_at(trecs, ntb - k) : rec_at(trecs, nta);
        if (!(ntr && ntr->pos >= nta && ntr->pos <= ntb - k)) ntr = nullptr;
        const bool q_had = nqr && S.q.count(nqr->h);
        const int q_old = q_had ? S.q[nqr->h] : 0;
        const bool t_had = ntr && S.t.count(ntr->h);
        const std::pair<int, int> t_old = t_had ? S.t[ntr->h] : std::pair<int, int>(0, 0);
        if (nqr) add_q(*nqr);
        if (ntr) add_t(*ntr, nqa, nqb);
        // the estimate changes only when a minimizer joined a region
        int64_t e2 = est, d2 = den;
        if (nqr || ntr) ext_estimate(S, (int)o, &e2, &d2);
        if (e2 < min_shared(tau, d2)) {  // back to the last good state
          if (nqr) {
            if (q_had) S.q[nqr->h] = q_old; else S.q.erase(nqr->h);
          }
          if (ntr) {
            if (t_had) S.t[ntr->h] = t_old; else S.t.erase(ntr->h);
          }
          break;
        }
        qa = nqa, qb = nqb, ta = nta, tb = ntb;
        est = e2, den = d2;
      }
    }
    out[x] = {i, o, js, qa, qb, ta, tb, est, den};
  };
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (int64_t x; (x = next.fetch_add(1)) < nk;) one(x);
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  Table* T = new Table();
  T->ncols = 9;
  for (auto& row : out) T->v.insert(T->v.end(), row.begin(), row.end());
  return T;
}

}  // extern "C"

// ---- f2 two-tier local chaining inside potential SD regions (Section 3.3) --
// For every region row (i, o, j*, qa, qb, ta, tb, ...) the query is
// X = G[qa, qb) and the target Y = G[ta, tb) (reverse-complemented when
// o = 1), both read case-insensitively.
//   Seeds: maximal exact matches (x, y, L) of at least k2 bases of A, C, G,
//   T between X and Y (Section 3.3: matching seeds of size 11 and higher).
//   Initial chains: a seed b may follow a if it starts later on both axes
//   and the gaps from a's end to b's start are at most g1 on both axes (the
//   maximum gap l * delta_G with l the 1,000 bp SD length; a gap may be
//   negative where an indel makes the seeds overlap); the link adds the
//   bases of b that are new on both axes, gain = min(L_b, end_b - end_a on
//   x, end_b - end_a on y), and must add at least one.  f(b) = the larger of
//   L_b and the best f(a) + gain (ties: the later seed in (x, y) order).
//   Chains are taken greedily: the seed of largest f (then the earlier seed)
//   that no chain holds yet, and its predecessors back to the first one a
//   chain already holds; score = L of the first seed plus the gains.
//   Final chains: initial chains chained again with gaps of at most g2
//   (10,000 bp) on both axes and an affine penalty go + g / gdiv for a gap
//   of g = the larger of the two gaps (Section 3.3 leaves the penalty's
//   values open); F(d) = S(d) + max(0, max F(c) - pen(c, d)), and the same
//   greedy extraction (score = the summed initial-chain scores less the
//   penalties of the links taken).  A final chain spanning at least min_len
//   bases on both axes is an SD (l >= 1,000).
// Rows (region index, o, q0, q1, t0, t1, score, seeds, initial chains) in
// genome coordinates, sorted by (region, q0, q1, t0, t1, score).
namespace {

struct Mem {
  int64_t x, y, L;
};

std::string region_text(const uint8_t* seq, int64_t a, int64_t b, bool revcomp) {
  return upper_window(seq, a, b - a, revcomp);
}

bool acgt(char c) { return c == 'A' || c == 'C' || c == 'G' || c == 'T'; }

// Maximal exact matches of at least k2 ACGT bases (x, y ascending).
std::vector<Mem> find_mems(const std::string& X, const std::string& Y, int64_t k2) {
  std::map<std::string, std::vector<int64_t>> at;
  for (int64_t y = 0; y + k2 <= (int64_t)Y.size(); ++y) {
    std::string w = Y.substr(y, k2);
    bool ok = true;
    for (char c : w) ok = ok && acgt(c);
    if (ok) at[w].push_back(y);
  }
  std::vector<Mem> out;
  for (int64_t x = 0; x + k2 <= (int64_t)X.size(); ++x) {
    auto it = at.find(X.substr(x, k2));
    if (it == at.end()) continue;
    for (int64_t y : it->second) {
      // left-maximal: the bases before do not extend the match
      if (x > 0 && y > 0 && X[x - 1] == Y[y - 1] && acgt(X[x - 1])) continue;
      int64_t L = k2;
      while (x + L < (int64_t)X.size() && y + L < (int64_t)Y.size() && X[x + L] == Y[y + L] &&
             acgt(X[x + L]))
        ++L;
      out.push_back({x, y, L});
    }
  }
  std::sort(out.begin(), out.end(), [](const Mem& a, const Mem& b) {
    return std::tie(a.x, a.y) < std::tie(b.x, b.y);
  });
  return out;
}

struct Box {
  int64_t x0, x1, y0, y1, score, seeds, parts;
};

// Greedy extraction of disjoint chains from a DP (f, pred over items in
// their sort order): repeatedly the item of largest f (then smallest index)
// not yet taken, with its predecessors back to the first one already taken.
std::vector<std::vector<int64_t>> extract_chains(const std::vector<int64_t>& f,
                                                 const std::vector<int64_t>& pred) {
  const int64_t A = (int64_t)f.size();
  std::vector<int64_t> order(A);
  for (int64_t a = 0; a < A; ++a) order[a] = a;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return f[a] != f[b] ? f[a] > f[b] : a < b;
  });
  std::vector<char> used(A, 0);
  std::vector<std::vector<int64_t>> chains;
  for (int64_t b : order) {
    if (used[b]) continue;
    std::vector<int64_t> path;
    for (int64_t c = b; c >= 0 && !used[c]; c = pred[c]) {
      used[c] = 1;
      path.push_back(c);
    }
    std::reverse(path.begin(), path.end());
    chains.push_back(path);
  }
  return chains;
}

std::vector<Box> chain_two_tiers(const std::vector<Mem>& mems, int64_t g1, int64_t g2,
                                 int64_t gap_open, int64_t gap_div) {
  // tier 1 over the seeds
  const int64_t A = (int64_t)mems.size();
  auto gain = [&](int64_t a, int64_t b) -> int64_t {  // <= 0: b cannot follow a
    const Mem &P = mems[a], &Q = mems[b];
    if (P.x >= Q.x || P.y >= Q.y) return 0;
    if (Q.x - (P.x + P.L) > g1 || Q.y - (P.y + P.L) > g1) return 0;
    return std::min(Q.L, std::min(Q.x + Q.L - (P.x + P.L), Q.y + Q.L - (P.y + P.L)));
  };
  std::vector<int64_t> f(A), pred(A, -1);
  for (int64_t b = 0; b < A; ++b) {
    f[b] = mems[b].L;
    for (int64_t a = 0; a < b; ++a) {
      const int64_t g = gain(a, b);
      if (g <= 0) continue;
      const int64_t v = f[a] + g;
      if (v > f[b] || (v == f[b] && pred[b] >= 0)) {
        f[b] = v;
        pred[b] = a;
      }
    }
  }
  std::vector<Box> init;
  for (auto& ch : extract_chains(f, pred)) {
    Box B{mems[ch.front()].x, 0, mems[ch.front()].y, 0, mems[ch.front()].L, (int64_t)ch.size(), 1};
    for (size_t u = 0; u < ch.size(); ++u) {
      B.x1 = std::max(B.x1, mems[ch[u]].x + mems[ch[u]].L);
      B.y1 = std::max(B.y1, mems[ch[u]].y + mems[ch[u]].L);
      if (u > 0) B.score += gain(ch[u - 1], ch[u]);
    }
    init.push_back(B);
  }
  std::sort(init.begin(), init.end(), [](const Box& a, const Box& b) {
    return std::tie(a.x0, a.y0, a.x1, a.y1, a.score) < std::tie(b.x0, b.y0, b.x1, b.y1, b.score);
  });
  // tier 2 over the initial chains (affine gap penalty)
  const int64_t C = (int64_t)init.size();
  auto pen = [&](const Box& c, const Box& d, int64_t* ok) {
    const int64_t gq = d.x0 - c.x1, gt = d.y0 - c.y1;
    *ok = gq >= 0 && gt >= 0 && gq <= g2 && gt <= g2;
    return gap_open + std::max(gq, gt) / gap_div;
  };
  std::vector<int64_t> F(C), P(C, -1);
  for (int64_t d = 0; d < C; ++d) {
    int64_t best = 0, arg = -1;
    for (int64_t c = 0; c < d; ++c) {
      int64_t ok = 0;
      const int64_t v = F[c] - pen(init[c], init[d], &ok);
      if (!ok) continue;
      if (v > best || (v == best && arg >= 0)) {
        best = v;
        arg = c;
      }
    }
    F[d] = init[d].score + best;
    P[d] = arg;
  }
  std::vector<Box> fin;
  for (auto& ch : extract_chains(F, P)) {
    const Box& a = init[ch.front()];
    const Box& z = init[ch.back()];
    Box B{a.x0, z.x1, a.y0, z.y1, 0, 0, (int64_t)ch.size()};
    for (size_t u = 0; u < ch.size(); ++u) {
      B.score += init[ch[u]].score;
      B.seeds += init[ch[u]].seeds;
      if (u > 0) {
        int64_t ok = 0;
        B.score -= pen(init[ch[u - 1]], init[ch[u]], &ok);
      }
    }
    fin.push_back(B);
  }
  return fin;
}

}  // namespace

extern "C" {

// Seeds of one pair of substrings (pins): rows (x, y, L).
void* orc_mems(const uint8_t* x, int64_t nx, const uint8_t* y, int64_t ny, int64_t k2) {
  std::string X((const char*)x, nx), Y((const char*)y, ny);
  Table* T = new Table();
  T->ncols = 3;
  for (auto& m : find_mems(X, Y, k2)) T->row({m.x, m.y, m.L});
  return T;
}

// Both tiers on explicit seed rows (x, y, L) (pins): final chain rows
// (x0, x1, y0, y1, score, seeds, parts) in extraction order.
void* orc_chain_tiers(const int64_t* seeds, int64_t A, int64_t g1, int64_t g2, int64_t gap_open,
                      int64_t gap_div) {
  std::vector<Mem> m(A);
  for (int64_t a = 0; a < A; ++a) m[a] = {seeds[3 * a], seeds[3 * a + 1], seeds[3 * a + 2]};
  std::sort(m.begin(), m.end(),
            [](const Mem& a, const Mem& b) { return std::tie(a.x, a.y) < std::tie(b.x, b.y); });
  Table* T = new Table();
  T->ncols = 7;
  for (auto& b : chain_two_tiers(m, g1, g2, gap_open, gap_div))
    T->row({b.x0, b.x1, b.y0, b.y1, b.score, b.seeds, b.parts});
  return T;
}

void* orc_chain2(const uint8_t* seq, const int64_t* regions, int64_t nreg, int64_t reg_cols,
                 int64_t k2, int64_t g1, int64_t g2, int64_t gap_open, int64_t gap_div,
                 int64_t min_len, int nthreads) {
  std::vector<std::vector<std::vector<int64_t>>> out(nreg);
  auto one = [&](int64_t r) {
    const int64_t* R = regions + r * reg_cols;
    const int64_t o = R[1], qa = R[3], qb = R[4], ta = R[5], tb = R[6];
    const std::string X = region_text(seq, qa, qb, false);
    const std::string Y = region_text(seq, ta, tb, o != 0);
    for (auto& b : chain_two_tiers(find_mems(X, Y, k2), g1, g2, gap_open, gap_div)) {
      if (b.x1 - b.x0 < min_len || b.y1 - b.y0 < min_len) continue;
      const int64_t t0 = o ? tb - b.y1 : ta + b.y0, t1 = o ? tb - b.y0 : ta + b.y1;
      out[r].push_back({r, o, qa + b.x0, qa + b.x1, t0, t1, b.score, b.seeds, b.parts});
    }
    std::sort(out[r].begin(), out[r].end());
  };
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (int64_t r; (r = next.fetch_add(1)) < nreg;) one(r);
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  Table* T = new Table();
  T->ncols = 9;
  for (auto& v : out)
    for (auto& row : v) T->v.insert(T->v.end(), row.begin(), row.end());
  return T;
}

}  // extern "C"
