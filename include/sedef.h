/*
 * sedef.h -- C ABI of the GB300 seeding filter for segmental-duplication
 * detection (SEDEF: Numanagic et al., "Fast Characterization of Segmental
 * Duplications in Genome Assemblies").
 *
 * The library computes the seed stage of the method on one GPU:
 *   sedef_pack    2-bit codes plus soft-mask and N bit-vectors (Section 2
 *                 alphabet; Section 3.2 soft-masked repeats)
 *   sedef_sketch  canonical k-mer hashes and winnowing minimizers (Section
 *                 2.2; Section 3.2 eligibility: at least one unmasked base)
 *   sedef_index   I_G sorted by (hash, position) and the reverse index as an
 *                 offset table over all 4^k hashes (Section 3.1)
 *   sedef_filter  per query window: candidate lookup, sliding count of shared
 *                 minimizers tested against tau, and the winnowed MinHash
 *                 estimate that picks each run's seed (Sections 2.2 and 3.1)
 *   sedef_chain   colinear chaining of the seed's minimizer anchors (Section
 *                 3.3, sparse DP with gaps bounded via delta_G)
 *   sedef_merge   chains joined into SD candidates (Section 3: seeds grown
 *                 while similar, at chain granularity)
 *
 * Conventions
 *   - Every call returns SEDEF_OK (0) or a negative sedef_status.  On error
 *     sedef_last_error() holds a message for the calling thread.
 *   - Pointers named d_* are device pointers (cudaMalloc or torch); h_* are
 *     host pointers.  The caller owns every buffer it passes; the library
 *     owns only its context (and the scratch memory the context allocates).
 *   - All work is enqueued on the context's stream.  Calls that return a
 *     count synchronize that stream before returning; the others do not.
 *   - Sequences are concatenated into one byte array; sequence s covers
 *     [seq_off[s], seq_off[s+1]) of it.  Positions inside the library are
 *     global coordinates in that array (uint32: total length < 2^32).
 *     sedef_cand_t reports per-sequence coordinates.  Intervals are 0-based
 *     and half-open unless stated.
 *   - Outputs are deterministic and sorted, so runs compare bit for bit.
 *   - Outputs with a data-dependent size take a capacity.  When the true
 *     size exceeds it the call returns SEDEF_ERR_CAPACITY, stores the
 *     needed size in the count argument and leaves the output undefined;
 *     call again with a larger buffer.
 */
#ifndef SEDEF_H
#define SEDEF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sedef_status {
  SEDEF_OK = 0,
  SEDEF_ERR_INVALID = -1,     /* bad argument or parameter */
  SEDEF_ERR_OOM = -2,         /* device or pinned-host allocation failed */
  SEDEF_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  SEDEF_ERR_TIMEOUT = -4,     /* a bounded device wait gave up */
  SEDEF_ERR_UNSUPPORTED = -5, /* parameters outside the supported range */
  SEDEF_ERR_CAPACITY = -6     /* output buffer too small; count holds the need */
} sedef_status;

/*
 * Parameters.  Defaults (sedef_default_params):
 *   k = 12          k-mer length for seeding (Section 3.3)
 *   w = 16          winnowing window, in consecutive k-mer start positions
 *                   (Section 2.2 leaves w open)
 *   n = 750         seed window length, n >= 1000 * (1 - delta) (Section 3)
 *   query_step = 250  distance between query window starts (the paper slides
 *                   over every locus; 250 = 1000 - n keeps a whole window
 *                   inside every SD of at least 1 kbp)
 *   max_occ = 0     0: no cap; otherwise hashes with more than max_occ
 *                   index entries are dropped from every query window
 *   self_mode = 1   query and target are the same genome: only pairs with
 *                   the target after the query are reported, the mates may
 *                   overlap by at most floor(delta * n) bases (Section 2),
 *                   and a target occurrence inside the query window's own
 *                   k-mer span is not a shared k-mer.  self_mode = 2: the
 *                   same, but every sequence is an independent genome
 *                   (targets only on the query's own sequence), so one call
 *                   self-searches a whole batch of genomes.  0: query
 *                   windows against a separate target, every target window
 *   gap_max = 750   largest gap between chained anchors on either axis
 *   diag_max = 75   largest drift |gap_q - gap_t| between chained anchors,
 *                   ceil(n * delta_G) (Section 3.3: gaps bounded by l*delta_G)
 *   min_unmasked = 1  unmasked bases a seeding k-mer needs (Section 3.2)
 *   delta_m = 0.15, delta_g = 0.10  error split (Section 2.1); tau from the
 *                   Section 3.1 bound
 * Supported: 2 <= k <= 15, 1 <= w <= 256, k < n, n - k + 1 <= 1024,
 * query_step >= 1.
 */
typedef struct sedef_params {
  int32_t k;
  int32_t w;
  int32_t n;
  int32_t query_step;
  int32_t max_occ;
  int32_t self_mode;
  int32_t gap_max;
  int32_t diag_max;
  int32_t min_unmasked;
  int32_t reserved;
  double delta_m;
  double delta_g;
} sedef_params;

/*
 * Sketch record (sedef_sketch, sedef_index): one uint64 per minimizer,
 *   bits 33..62  hash H(c) of the canonical code c (2k significant bits)
 *   bits  1..32  start position p (global coordinate)
 *   bit   0      strand: 1 when the reverse complement is the canonical form
 */
#define SEDEF_REC_HASH(r) ((uint64_t)(r) >> 33)
#define SEDEF_REC_POS(r) ((uint32_t)((uint64_t)(r) >> 1))
#define SEDEF_REC_STRAND(r) ((uint32_t)((r)&1u))

/*
 * One maximal run of passing target windows for one query window and one
 * relative strand (Section 3.1 rolling), with its refined seed.
 *   i         query window start (global); the window is [i, i+n)
 *   j_a, j_b  first and last passing target window start (global, inclusive)
 *   j_at_max  smallest j in the run where the shared count is max_shared
 *   j_star    smallest j in the run where the winnowed MinHash estimate
 *             (Section 2.2) is largest; the seed is (i, j_star, o)
 *   s         distinct minimizer hashes of the query window
 *   m         shared hashes needed, the least integer >= tau*s - 1e-9
 *   max_shared  largest shared count in the run
 *   est, den  estimate numerator and denominator at j_star
 *   o         relative strand (0 same, 1 reverse complement)
 *   keep      1 when est >= m(den) (the seed is kept)
 */
typedef struct sedef_run_t {
  uint32_t i, j_a, j_b, j_at_max, j_star;
  uint16_t s, m, max_shared, est, den;
  uint8_t o, keep;
} sedef_run_t;

/*
 * Best chain of one kept seed (Section 3.3), global coordinates:
 * query [q0, q1) and target [t0, t1) bounding boxes of the chained anchors,
 * score = number of anchors, s = the query window's sketch size.
 */
typedef struct sedef_chain_t {
  uint32_t i, qseq, q0, q1, tseq, t0, t1;
  uint16_t score, s;
  uint32_t o;
  uint32_t reserved;
} sedef_chain_t;

/*
 * Potential SD region (f1, Section 3.2): a kept seed (i, j_star, o) grown
 * into query [qa, qb) and target [ta, tb), global coordinates; est / den is
 * the winnowed MinHash estimate of the grown regions (den = s = |W_Q|).
 */
typedef struct sedef_region_t {
  uint32_t i, j_star, qa, qb, ta, tb;
  uint32_t est, den, o, reserved;
} sedef_region_t;

/*
 * An SD found by the two-tier chaining of Section 3.3 inside a potential
 * SD region: query [q0, q1) and target [t0, t1), global coordinates, with
 * the strand o, the chain score (aligned bases less the gap penalties), the
 * exact seeds it holds and the initial chains it joins; region = the index
 * of its potential SD region in the sedef_chain2 input.
 */
typedef struct sedef_sd_t {
  uint32_t region, o, q0, q1, t0, t1;
  uint32_t score, seeds, parts, reserved;
} sedef_sd_t;

/* SD candidate: one connected group of chains, per-sequence coordinates. */
typedef struct sedef_cand_t {
  uint32_t qseq, q0, q1, tseq, t0, t1;
  uint32_t o, score, nchains, reserved;
} sedef_cand_t;

typedef struct sedef_ctx sedef_ctx;

/* Fills *p with the defaults listed above. */
void sedef_default_params(sedef_params* p);

/* Message of the last failed call on this thread ("" if none). */
const char* sedef_last_error(void);

/*
 * Creates a context on `device` that enqueues work on `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  The
 * context owns a growable device scratch buffer and a pinned host buffer;
 * sedef_destroy frees both.  A context is not thread-safe.
 */
int sedef_create(int device, void* stream, sedef_ctx** out);
int sedef_destroy(sedef_ctx* ctx);
int sedef_set_stream(sedef_ctx* ctx, void* stream);

/*
 * Caps the device scratch memory the context may hold (its pool and the
 * buffers of sedef_selfsearch*) at `bytes` (< 0: no cap, the default).  A
 * call whose scratch would pass the cap fails with SEDEF_ERR_OOM as if
 * cudaMalloc had failed, and the context stays usable.  Lowering the cap
 * below what the context holds gives its blocks back first.  Synchronizes.
 */
int sedef_set_scratch_limit(sedef_ctx* ctx, int64_t bytes);

/*
 * Caps the shared memory per CTA that the filter's shared-memory tiers of
 * this context may ask for (< 0: no cap, the default).  When the second
 * wide tier (16,384 collected hits, about 213 KB per CTA) is above the cap,
 * a form of it that holds 8,192 collected hits (about 150 KB) takes its
 * place, and when that is above the cap too the wide tier hands the windows
 * it cannot hold straight to the global path; the windows a smaller tier
 * cannot hold go to the global path, so the results do not change.  The
 * other tiers need at most 100 KB per CTA
 * and always run: a cap below 100 KB (102,400 bytes) is refused with
 * SEDEF_ERR_UNSUPPORTED.  For a context whose
 * kernels run beside a persistent kernel (sedef_server_create): an SM keeps
 * its L1 / shared-memory split while any CTA stays on it, so a kernel that
 * needs more shared memory than the persistent kernel leaves waits until
 * that kernel exits.  No GPU work.
 */
int sedef_set_tier_smem_limit(sedef_ctx* ctx, int64_t bytes);

/*
 * Tracing.  While enabled, every kernel the context launches is bracketed by
 * CUDA events on the context's stream.  sedef_trace_report synchronizes the
 * stream and writes one line per kernel name, "name launches total_ms", in
 * first-launch order, into buf (NUL-terminated, truncated to cap bytes); it
 * returns the full text length (or a negative status) and, with reset != 0,
 * forgets the recorded launches.
 */
int sedef_trace_enable(sedef_ctx* ctx, int on);
int sedef_trace_report(sedef_ctx* ctx, char* buf, int64_t cap, int reset);

/* Kernels launched by this process through the library so far. */
uint64_t sedef_launch_count(void);

/*
 * Counters of the context's last sedef_filter call, out[0..n): query
 * windows, windows sent to the global-memory path, hits enumerated and hits
 * collected by the shared-memory path, runs, runs refined by the large
 * refine kernel, hits of the global-memory path; out[7] = anchors of the
 * context's last sedef_chain call (at most 8 values).  out[6] and out[7]
 * are the totals a captured pass needs as capacities.
 */
int sedef_filter_stats(sedef_ctx* ctx, int64_t* out, int32_t n);

/*
 * tau from the Section 3.1 bound, tau = (1-dG)/(1+dG) / (2 e^{k dM} - 1),
 * and m_out[s] = the least integer m with m >= tau*s - 1e-9 for s in
 * [0, smax].  m_out may be NULL.  Host only.
 */
int sedef_threshold_table(const sedef_params* p, int32_t* m_out, int32_t smax, double* tau_out);

/*
 * a1: d_seq holds n ASCII bytes.  Writes d_packed[ceil(n/16)] (base p in
 * bits 2*(p%16) of word p/16; A/a=0 C/c=1 G/g=2 T/t=3, other bytes 0),
 * d_mask[ceil(n/32)] (bit p%32 of word p/32 set for a lowercase letter) and
 * d_nbits[ceil(n/32)] (bit set for a byte that is not ACGTacgt).  n may be 0.
 */
int sedef_pack(sedef_ctx* ctx, const uint8_t* d_seq, int64_t n, uint32_t* d_packed,
               uint32_t* d_mask, uint32_t* d_nbits);

/*
 * a2: winnowing sketch of the packed input.  For each k-mer start p whose k
 * bases lie in one sequence: forward code f (first base most significant),
 * reverse-complement code r, canonical c = min(f, r), strand (r < f).  The
 * k-mer is eligible when it has no N, at least min_unmasked unmasked bases
 * and f != r; its hash is H(c), a bijection of [0, 4^k).  For every window
 * of w consecutive k-mer starts inside one sequence, the eligible k-mer of
 * least hash (the rightmost on ties) is selected.  Writes the distinct
 * selected k-mers as records (layout above) sorted by position into
 * d_rec[0..rec_cap) and their number to *h_nrec.  Synchronizes.
 */
int sedef_sketch(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_mask,
                 const uint32_t* d_nbits, const int64_t* h_seq_off, int32_t nseq,
                 const sedef_params* p, uint64_t* d_rec, int64_t rec_cap, int64_t* h_nrec);

/*
 * sedef_sketch without any allocation (no counterpart in the paper: this is
 * an interface for callers, not part of the method).  Same inputs, outputs,
 * results and return codes as sedef_sketch, with no context: the work is
 * enqueued on `stream` (a cudaStream_t as void*).  For callers that cannot
 * allocate device memory themselves or through the library -- for example a
 * host framework that owns the whole device heap through its own pool, or
 * a latency-critical path that must avoid cudaMalloc's implicit device
 * synchronization.  Its scratch is one fixed static device array of about
 * 1 MB (per-tile counts and offsets for at most 268,435,456 bases and the
 * offsets of at most 4096 sequences); larger inputs are rejected with
 * SEDEF_ERR_UNSUPPORTED.  The array stays allocated on every device that
 * loads the library until the process exits.  Every call looks up the
 * array's device address on the current device (cudaGetSymbolAddress); the
 * first call on a device also loads the array there, so make that first
 * call before any stream capture.  All calls share the one array, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialize them.  Synchronizes `stream`.
 */
int sedef_sketch_noalloc(const uint32_t* d_packed, const uint32_t* d_mask,
                         const uint32_t* d_nbits, const int64_t* h_seq_off, int32_t nseq,
                         const sedef_params* p, uint64_t* d_rec, int64_t rec_cap,
                         int64_t* h_nrec, void* stream);

/*
 * a3: sorts the nrec records of d_rec by (hash, position) into d_sorted and
 * writes d_off[0..4^k] with d_off[x] = number of records whose hash is < x,
 * so the postings of hash x are d_sorted[d_off[x] .. d_off[x+1]).
 * d_rec and d_sorted must not overlap.
 */
int sedef_index(sedef_ctx* ctx, const uint64_t* d_rec, int64_t nrec, const sedef_params* p,
                uint64_t* d_sorted, uint32_t* d_off);

/*
 * a4-a6: for every query window i (each query sequence start, then every
 * query_step bases while i + n <= the sequence end) with W_Q = the distinct
 * hashes of the query minimizers starting in [i, i+n-k] (s = |W_Q|, m = m(s))
 * and each relative strand o, shared_o(j) counts the hashes of W_Q that occur
 * in the target window [j, j+n-k] with relative strand o.  A target start j
 * is valid when [j, j+n) lies in one target sequence (self mode: see
 * sedef_params).  Each maximal run of valid j with shared_o(j) >= m is one
 * sedef_run_t, refined with the winnowed MinHash estimate at every j of the run
 * where the target window's minimizers change.
 *
 * Query: d_qrec (nq records sorted by position) over sequences h_qoff.
 * Target: d_trec (nt records sorted by position), its index d_tsorted/d_toff
 * (sedef_index), over sequences h_toff.  In self mode query and target are
 * the same arrays.  Runs are sorted by (i, o, j_a).  Synchronizes.
 */
int sedef_filter(sedef_ctx* ctx, const uint64_t* d_qrec, int64_t nq, const int64_t* h_qoff,
                 int32_t nqseq, const uint64_t* d_trec, const uint64_t* d_tsorted,
                 const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                 const sedef_params* p, sedef_run_t* d_runs, int64_t run_cap, int64_t* h_nruns);

/*
 * Autotuner of the filter's first shared-memory tier: times each compiled
 * shape (threads per query window; hits and dense groups a window may keep
 * in shared memory) on a uniform sample of the query windows (at least
 * 65,536 or one in sixteen; best of two timed runs each) with the same
 * arguments as sedef_filter, and keeps the fastest for later
 * sedef_filter calls on this context; *variant_out receives its number.
 * Results never depend on the shape: windows a shape cannot hold move to
 * the next tier.  Synchronizes.
 */
int sedef_filter_autotune(sedef_ctx* ctx, const uint64_t* d_qrec, int64_t nq,
                          const int64_t* h_qoff, int32_t nqseq, const uint64_t* d_trec,
                          const uint64_t* d_tsorted, const uint32_t* d_toff, int64_t nt,
                          const int64_t* h_toff, int32_t ntseq, const sedef_params* p,
                          int32_t* variant_out);

/* Sets the first-tier filter shape when set >= 0; returns the current one
 * and the number of shapes (either pointer may be NULL). */
int sedef_filter_variant(sedef_ctx* ctx, int32_t set, int32_t* current, int32_t* count);

/*
 * Index persistence (checkpoint and restart of a serving process).  A blob
 * holds the sequence offsets, the records by position (sedef_sketch), the
 * records by hash (sedef_index), the 4^k + 1 offsets and a checksum.
 * sedef_index_blob_size gives its size; sedef_index_save fills a host
 * buffer of at least that size (synchronizes); sedef_index_blob_info checks
 * the header, size and checksum and reports k, nrec and nseq;
 * sedef_index_load copies the blob back to caller-allocated device arrays
 * and host offsets (SEDEF_ERR_INVALID on a damaged or mismatched blob).
 */
int64_t sedef_index_blob_size(int32_t k, int64_t nrec, int32_t nseq);
int sedef_index_save(sedef_ctx* ctx, const uint64_t* d_rec, const uint64_t* d_sorted,
                     const uint32_t* d_off, int64_t nrec, int32_t k, const int64_t* h_seq_off,
                     int32_t nseq, void* h_blob, int64_t cap);
int sedef_index_blob_info(const void* h_blob, int64_t size, int32_t* k, int64_t* nrec,
                          int32_t* nseq);
int sedef_index_load(sedef_ctx* ctx, const void* h_blob, int64_t size, int64_t* h_seq_off,
                     int32_t nseq_cap, uint64_t* d_rec, uint64_t* d_sorted, uint32_t* d_off,
                     int64_t rec_cap);

/*
 * a7 (chaining): for each kept run, the anchors are the pairs (p, t) of a
 * query-window minimizer and a target minimizer starting in [j_a, j_b+n-k]
 * with equal hash and strands differing by o (self mode: t outside the query
 * window's span).  For o = 1 the target axis is reversed.  The best chain
 * maximizes the number of anchors; consecutive anchors advance on both axes
 * by at most gap_max with |gap_q - gap_t| <= diag_max.  Ties: predecessor
 * with the larger count then the later anchor in (p, t') order; chain end
 * with the larger count then the earlier anchor.  Chains with fewer than
 * m(s) anchors are dropped.  Query records as in sedef_filter; the target
 * is given by its index (d_tsorted, d_toff from sedef_index).  Writes chains
 * in run order.  Synchronizes.
 */
int sedef_chain(sedef_ctx* ctx, const sedef_run_t* d_runs, int64_t nruns, const uint64_t* d_qrec,
                int64_t nq, const int64_t* h_qoff, int32_t nqseq, const uint64_t* d_tsorted,
                const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                const sedef_params* p, sedef_chain_t* d_chains, int64_t cap, int64_t* h_nchains);

/*
 * a7 (merge): chains with the same query sequence, target sequence and
 * strand are linked when their query intervals overlap or touch, their
 * target intervals overlap or touch, and their diagonals (t0 - q0 for o = 0,
 * t1 + q0 for o = 1) differ by at most diag_max + ceil(delta_g * L), L the
 * longer query span.  Each connected component becomes one candidate: the
 * bounding boxes, the summed scores and the chain count, in per-sequence
 * coordinates, sorted by global (q0, t0, o, q1, t1).  Synchronizes.
 */
int sedef_merge(sedef_ctx* ctx, const sedef_chain_t* d_chains, int64_t nchains,
                const int64_t* h_qoff, int32_t nqseq, const int64_t* h_toff, int32_t ntseq,
                const sedef_params* p, sedef_cand_t* d_cands, int64_t cap, int64_t* h_ncands);

/*
 * f3 (the q-gram filter of Section 3.2), applied to kept seeds: for run r
 * with keep = 1, X = G[i, i+n) and Y = G[j_star, j_star+n) (reverse
 * complement when o = 1); d_shared[r] = the q-grams X and Y share, counted
 * with multiplicity (sum over q-grams of the smaller occurrence count;
 * q-grams over a non-ACGT base are not counted); d_pass[r] = 1 when
 * d_shared[r] >= the least integer >= B - 1e-9, where
 * B = n (1 - delta_G - q delta_M) - (n p_gap + 1)(q - 1) is the paper's
 * adapted q-gram lemma bound (p_gap: expected gaps per base).  Runs with
 * keep = 0 get 0 and 0.  d_packed / d_nbits are sedef_pack's outputs for
 * the nbases bases the runs refer to (global coordinates).  q in [1, 5].
 * *h_npass = passing seeds.  Synchronizes.
 */
int sedef_qgram(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_nbits, int64_t nbases,
                const sedef_run_t* d_runs, int64_t nruns, const sedef_params* p, int32_t q,
                double p_gap, uint32_t* d_shared, uint8_t* d_pass, int64_t* h_npass);

/*
 * f1 (Section 3.2, SD extension): every kept run's seed (i, j_star, o) is
 * grown into a potential SD region.  The query region starts as [i, i+n)
 * and the target region as [j_star, j_star+n); both grow by one base per
 * step -- right ends first, then left ends; for o = 1 the target grows at
 * the opposite end -- while the winnowed MinHash estimate of the two
 * regions (Section 2.2: s = |W_Q|, U = the s smallest hashes of W_Q u W_T,
 * est = hashes of U in both with relative strand o) stays >= m(s).  Growth
 * also stops at a sequence end, at max_len bases (Section 3.2 limits
 * potential SDs to 1 Mbp), and, in a self search with both regions on one
 * sequence, where the regions would overlap more than before.  W_Q and W_T
 * come from the extension sketches d_qext / d_text: sedef_sketch of the
 * same sequences with min_unmasked = 0 (the extension uses every k-mer,
 * masked ones included), sorted by position.  In a self search (self_mode 1
 * or 2) d_qext and d_text are the same array and a target minimizer inside
 * the query region's k-mer span is not shared.  Writes one region per kept
 * run, in run order, to d_regions[0..cap) and their number to *h_nregions
 * (SEDEF_ERR_CAPACITY when cap is too small).  Needs k <= 12 (a 4-bit state
 * per hash, 2^(2k) / 2 bytes of scratch per resident warp).  Synchronizes.
 */
int sedef_extend(sedef_ctx* ctx, const sedef_run_t* d_runs, int64_t nruns, const uint64_t* d_qext,
                 int64_t nq, const int64_t* h_qoff, int32_t nqseq, const uint64_t* d_text,
                 int64_t nt, const int64_t* h_toff, int32_t ntseq, const sedef_params* p,
                 int64_t max_len, sedef_region_t* d_regions, int64_t cap, int64_t* h_nregions);

/*
 * f2 (Section 3.3, detecting the final SDs inside potential SD regions):
 * for every region of d_regions (sedef_extend's output) the query
 * X = G[qa, qb) and the target Y = G[ta, tb) (reverse complement when
 * o = 1), read from sedef_pack's d_packed / d_nbits over nbases bases (case
 * does not matter; non-ACGT bases match nothing).  Seeds are the maximal
 * exact matches of at least 11 bases.  Tier 1: colinear seeds whose gaps
 * on both axes are at most ceil(1000 * delta_G) (seeds may overlap where an
 * indel shifts the diagonal; a link scores the bases new on both axes),
 * best chains by DP (ties: the later seed), taken greedily by decreasing
 * score as disjoint initial chains.  Tier 2: initial chains chained with
 * gaps of at most 10,000 on both axes and an affine gap penalty of
 * 25 + g / 50 for the larger gap g (the paper leaves its values open), a
 * link only when it raises the score, the same greedy extraction.  Every
 * final chain spanning at least 1,000 bases on both axes is one sedef_sd_t,
 * sorted by (region, q0, q1, t0, t1, score).  Regions must be shorter than
 * 2^20 bases (SEDEF_ERR_UNSUPPORTED otherwise).  Writes d_out[0..cap) and
 * *h_nout (SEDEF_ERR_CAPACITY when cap is too small).  Synchronizes.
 */
int sedef_chain2(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_nbits, int64_t nbases,
                 const sedef_region_t* d_regions, int64_t nregions, const sedef_params* p,
                 sedef_sd_t* d_out, int64_t cap, int64_t* h_nout);

/*
 * Whole self-search of a device-resident input (Sections 2.2-3.3 in one
 * call): pack, sketch, index, filter (with refine), chain and merge of
 * d_seq (total bytes h_seq_off[nseq]) on the context's stream, with
 * self_mode 1 (one genome) or 2 (a batch of independent genomes, one per
 * sequence).  Writes the candidates to the caller's device buffer
 * d_cands[0..cap) and their number to *h_ncands (SEDEF_ERR_CAPACITY when
 * cap is too small).  Scratch comes from the context and is reused by the
 * next call; the run buffer starts at the previous call's run count, so a
 * repeated search runs the filter once.  Synchronizes.
 */
int sedef_selfsearch(sedef_ctx* ctx, const uint8_t* d_seq, const int64_t* h_seq_off,
                     int32_t nseq, const sedef_params* p, sedef_cand_t* d_cands, int64_t cap,
                     int64_t* h_ncands);

/*
 * Whole self-search through host buffers: brings h_seq (total bytes
 * h_seq_off[nseq]) to the device, runs sedef_selfsearch's stages on the
 * context's stream, and copies the candidates back to h_cands.  Page-locked
 * h_seq (cudaHostAlloc / cudaHostRegister) is read once by the packing
 * kernel through its device mapping; pageable h_seq is copied to device
 * memory first.  Either way h_seq must stay unchanged until the call
 * returns.  Device memory comes from the context.  Synchronizes.
 */
int sedef_selfsearch_host(sedef_ctx* ctx, const uint8_t* h_seq, const int64_t* h_seq_off,
                          int32_t nseq, const sedef_params* p, sedef_cand_t* h_cands, int64_t cap,
                          int64_t* h_ncands);

/*
 * Captured self-search pass (one CUDA graph).  The paper has no counterpart:
 * this is the batched driver's launch form.  sedef_graph_create records
 * pack, sketch, index, filter, refine, chain and merge for the device
 * sequence d_seq (sequences at h_seq_off; self_mode from p: 1 for one
 * genome, 2 for a batch of independent genomes) into a graph whose every
 * data-dependent size is a capacity from `caps`: no stage synchronizes with
 * the host, exact counts stay on the device, and work past a capacity is
 * skipped and flagged.  Capacities below 1 are taken as 1; each must be
 * below 2^32 (chains below 2^31).
 *
 * The graph reads d_seq and writes the caller's buffers at every launch:
 * d_rec and d_sorted (caps->records entries each), d_off (4^k + 1),
 * d_runs (caps->runs), d_chains (caps->chains), d_cands (caps->cands).
 * They must stay allocated, and d_seq keep its layout, until
 * sedef_graph_destroy.  Scratch memory and the pinned copies of uploads
 * belong to the graph (a private context on `ctx`'s device, with the filter
 * shape `ctx` was autotuned to).
 *
 * sedef_graph_launch enqueues one replay on `stream` (NULL: the graph's own
 * stream).  sedef_graph_wait synchronizes that stream and fills
 * h_need[0..5] with the exact totals (records, global-path hits, runs,
 * anchors, chains, candidates); each output holds min(total, capacity)
 * entries.  It returns SEDEF_ERR_CAPACITY when a total exceeded its
 * capacity (outputs are then incomplete: create a graph with the reported
 * totals as capacities) and SEDEF_ERR_UNSUPPORTED when a seed exceeded the
 * 65,536-anchor limit.  sedef_graph_nodes gives the number of kernel nodes
 * one launch runs.
 */
typedef struct sedef_graph sedef_graph;
typedef struct sedef_graph_caps {
  int64_t records, slow_hits, runs, anchors, chains, cands;
} sedef_graph_caps;

int sedef_graph_create(sedef_ctx* ctx, const uint8_t* d_seq, const int64_t* h_seq_off,
                       int32_t nseq, const sedef_params* p, const sedef_graph_caps* caps,
                       uint64_t* d_rec, uint64_t* d_sorted, uint32_t* d_off, sedef_run_t* d_runs,
                       sedef_chain_t* d_chains, sedef_cand_t* d_cands, sedef_graph** out);
int sedef_graph_launch(sedef_graph* g, void* stream);
int sedef_graph_wait(sedef_graph* g, int64_t* h_need);
int64_t sedef_graph_nodes(sedef_graph* g);
int sedef_graph_destroy(sedef_graph* g);

/*
 * Serving with continuous batching (no counterpart in the paper: this is the
 * serving form of the seed stage, non-self search against a resident
 * target index).  sedef_server_create keeps the target index (d_trec,
 * d_tsorted, d_toff from sedef_sketch / sedef_index, owned by the caller;
 * they must stay allocated) and allocates `slots` request slots of up to
 * slot_bases query bases each.  A persistent filter kernel (one CTA per SM)
 * drains a work queue of query windows in mapped host memory; the host adds
 * a request's windows when sedef_server_submit admits it into a free slot,
 * so requests that arrive while others are on the GPU join the running
 * kernel.  sedef_server_submit copies the query (h_query, len bases) to the
 * device, sketches it, builds its window table and publishes its windows;
 * it returns SEDEF_ERR_CAPACITY when no slot is free.  sedef_server_poll
 * waits up to wait_s seconds for a request whose windows are all filtered
 * (*slot_out = its slot, or -1); sedef_server_finish then runs the rest of
 * the path for that slot (windows the kernel's shared-memory tier could not
 * hold, run ordering and refine, chaining, merging) and copies its
 * candidates (query coordinates within the request, target coordinates per
 * target sequence) to h_cands; the slot is free again afterwards (when cap
 * is too small it returns SEDEF_ERR_CAPACITY with the count in *h_ncands
 * and keeps the candidates: call it again with a larger buffer).  A CTA of
 * the persistent kernel that finds no work for idle_timeout_s seconds
 * leaves; when all have left that way sedef_server_status returns
 * SEDEF_ERR_TIMEOUT (running = 0, timed_out = 1), and the next submit or
 * poll launches the kernel again.  submit may run on one host thread while
 * poll runs on another; submit and poll are not reentrant.  finish may run
 * on several threads at once for different slots: up to five calls work at
 * the same time, each on its own stream, and further calls wait for one of
 * them to return.  The kernel keeps a window with more than 4,096 hits for
 * finish, which runs the wide shared-memory tier over such windows.
 * sedef_server_destroy stops the kernel and frees the server.
 * The persistent kernel asks for the largest L1 / shared-memory split and
 * keeps 62 KB of shared memory on every SM while it runs; a kernel of
 * another stream that needs more than what is left waits for it to leave.
 * sedef_server_smem_left gives that bound (bytes per CTA); finish keeps its
 * own filter tiers within it, and a context that runs beside the server
 * should do the same (sedef_set_tier_smem_limit).
 */
typedef struct sedef_server sedef_server;
int sedef_server_create(sedef_ctx* ctx, const uint64_t* d_trec, const uint64_t* d_tsorted,
                        const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                        const sedef_params* p, int32_t slots, int64_t slot_bases,
                        double idle_timeout_s, sedef_server** out);
int sedef_server_submit(sedef_server* s, const uint8_t* h_query, int64_t len, int32_t* slot_out);
int sedef_server_poll(sedef_server* s, double wait_s, int32_t* slot_out);
int sedef_server_finish(sedef_server* s, int32_t slot, sedef_cand_t* h_cands, int64_t cap,
                        int64_t* h_ncands);
int sedef_server_status(sedef_server* s, int32_t* running, int32_t* timed_out);
int sedef_server_smem_left(sedef_server* s, int64_t* bytes);
int sedef_server_destroy(sedef_server* s);

#ifdef __cplusplus
}
#endif

#endif /* SEDEF_H */
