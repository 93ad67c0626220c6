// Shared device/host helpers of the GB300 seeding-filter library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sedef.h"

namespace sedef {

constexpr uint32_t kInfHash = 0xFFFFFFFFu;  // ineligible k-mer: never selected
constexpr int kMaxWindowRecs = 1024;        // n - k + 1 bound (records per window)

// Host-side error reporting (thread-local message, negative status).
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SEDEF_CUDA(call)                                   \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return ::sedef::cuda_fail(_e, #call); \
  } while (0)

#define SEDEF_LAUNCHED(name)                               \
  do {                                                     \
    cudaError_t _e = cudaGetLastError();                   \
    if (_e != cudaSuccess) return ::sedef::cuda_fail(_e, name); \
  } while (0)

// Every kernel launch goes through SEDEF_KERNEL: it counts the launch,
// brackets it with CUDA events when the context traces, and turns a launch
// error into a status.
#define SEDEF_KERNEL(ctx, name, ...)                                        \
  do {                                                                      \
    ::sedef::TraceScope _ts((ctx), (name));                                 \
    __VA_ARGS__;                                                            \
    ::sedef::count_launch();                                                \
    cudaError_t _e = cudaGetLastError();                                    \
    if (_e != cudaSuccess) return ::sedef::cuda_fail(_e, name);             \
  } while (0)

#define SEDEF_TRY(call)            \
  do {                             \
    int _s = (call);               \
    if (_s != SEDEF_OK) return _s; \
  } while (0)

// Device scratch pool owned by a context.  Blocks are cudaMalloc'ed on
// demand and reused; reset() releases every block for the next call (the
// stream orders the next call's kernels after the previous ones).
struct Pool {
  struct Block {
    void* ptr;
    size_t size;
    bool used;
  };
  std::vector<Block> blocks;
  int device = 0;
  // device bytes the pool may hold in all (sedef_set_scratch_limit); an
  // allocation past it fails as cudaMalloc would
  const size_t* limit = nullptr;
  size_t* held = nullptr;
  // stream-ordered blocks (cudaMallocAsync / cudaFreeAsync on *ordered):
  // they do not synchronize with the work of other streams
  const cudaStream_t* ordered = nullptr;
  void* alloc(size_t bytes);
  void reset();
  void release();
  // Blocks in use now; restore() hands back every block taken since (the
  // stream orders later kernels after the ones that used them).
  std::vector<char> snapshot() const;
  void restore(const std::vector<char>& used_before);
};

// Launch-time derived parameters shared by the kernels (computed on the host
// from sedef_params).
struct Derived {
  int k, w, n, span;        // span = n - k: a window's k-mer starts are [j, j+span]
  int step, max_occ, self_mode, gap_max, diag_max, min_unmasked;
  int overlap;              // floor((delta_m + delta_g) * n)
  uint32_t kmask;           // 4^k - 1
  double delta_g;
};

int derive(const sedef_params* p, Derived* d);

// ---------------------------------------------------------------- device ---

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Inclusive warp scan (add).
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, v, d);
    if ((int)lane_id() >= d) v += o;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x multiple of
// 32, at most 1024).  `tmp` holds 33 ints of shared memory.  Returns the
// exclusive prefix; *total receives the block sum.
__device__ __forceinline__ int block_exclusive_sum(int v, int* tmp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = warp_inclusive_sum(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int x = lane < nw ? tmp[lane] : 0;
    int xi = warp_inclusive_sum(x);
    if (lane < nw) tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  int r = tmp[warp] + inc - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

// First index in [lo, hi) of a sorted uint64 array whose value is >= key
// under the projection proj.
template <typename F>
__device__ __forceinline__ int64_t lower_bound_by(const uint64_t* a, int64_t lo, int64_t hi,
                                                  uint64_t key, F proj) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (proj(a[mid]) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// A data-dependent count inside a captured pass.  Host code sizes grids and
// buffers by a planned capacity `n`; the exact count stays on the device at
// `d` (nullptr in an eager call, where `n` is exact).  Kernels read it here.
__device__ __forceinline__ int64_t live_n(int64_t n, const uint32_t* d) {
  if (!d) return n;
  const int64_t v = (int64_t)*d;
  return v < n ? v : n;
}

// Record field access (layout in sedef.h).
__host__ __device__ __forceinline__ uint32_t rec_hash(uint64_t r) { return (uint32_t)(r >> 33); }
__host__ __device__ __forceinline__ uint32_t rec_pos(uint64_t r) { return (uint32_t)(r >> 1); }
__host__ __device__ __forceinline__ uint32_t rec_strand(uint64_t r) { return (uint32_t)(r & 1u); }

// First x in [a0, a1) whose record position is >= key (a1 when none): the
// same answer as a binary search, found with fewer dependent loads.  A
// posting list of a batch spans every genome with positions spread over the
// whole target, so one interpolation probe lands near the answer; a gallop
// from it brackets the answer and a binary search finishes inside the
// bracket.  Invariant: pos(lo) < key <= pos(hi).
__host__ __device__ __forceinline__ uint32_t pos_lower_bound(const uint64_t* idx, uint32_t a0,
                                                             uint32_t a1, int64_t key) {
  if (a0 >= a1) return a0;
  const int64_t pf = rec_pos(idx[a0]), pl = rec_pos(idx[a1 - 1]);
  if (pf >= key) return a0;
  if (pl < key) return a1;
  uint32_t lo = a0, hi = a1 - 1;
  if (hi - lo > 1) {
    // (key - pf) / (pl - pf) is in (0, 1]; any probe strictly inside the
    // bracket is correct, so a single-precision estimate clamped into it
    // will do (an integer division here costs more than a search step)
    const float f = (float)(key - pf) / (float)(pl - pf) * (float)(hi - lo - 1);
    const uint32_t g = lo + 1 + (f < (float)(hi - lo - 2) ? (uint32_t)f : hi - lo - 2);
    uint32_t step = 1;
    if ((int64_t)rec_pos(idx[g]) >= key) {
      hi = g;
      while (hi - lo > 1) {  // gallop down
        const uint32_t c = hi - lo > step ? hi - step : lo;
        if (c == lo) break;
        if ((int64_t)rec_pos(idx[c]) >= key) {
          hi = c;
          step <<= 1;
        } else {
          lo = c;
          break;
        }
      }
    } else {
      lo = g;
      while (hi - lo > 1) {  // gallop up
        const uint32_t c = hi - lo > step ? lo + step : hi;
        if (c == hi) break;
        if ((int64_t)rec_pos(idx[c]) < key) {
          lo = c;
          step <<= 1;
        } else {
          hi = c;
          break;
        }
      }
    }
  }
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((int64_t)rec_pos(idx[mid]) >= key) hi = mid; else lo = mid;
  }
  return hi;
}

// First x in [a0, a1) whose record position is >= key, galloping forward
// from a0: the answer is expected a few entries on (the postings of one
// genome of a batch).
__host__ __device__ __forceinline__ uint32_t pos_gallop_forward(const uint64_t* idx, uint32_t a0,
                                                                uint32_t a1, int64_t key) {
  if (a0 >= a1 || (int64_t)rec_pos(idx[a0]) >= key) return a0;
  uint32_t lo = a0, hi = a1;  // pos(lo) < key; pos(hi) >= key, or hi = a1
  uint32_t step = 1;
  while (hi - lo > 1) {
    const uint32_t c = hi - lo > step ? lo + step : hi;
    if (c == hi) break;
    if ((int64_t)rec_pos(idx[c]) < key) {
      lo = c;
      step <<= 1;
    } else {
      hi = c;
      break;
    }
  }
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((int64_t)rec_pos(idx[mid]) >= key) hi = mid; else lo = mid;
  }
  return hi;
}

// Index of the sequence containing global position pos (offsets has nseq+1
// entries, offsets[0] = 0).
__device__ __forceinline__ int seq_of(const int64_t* off, int nseq, int64_t pos) {
  int lo = 0, hi = nseq;  // answer in [0, nseq)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= pos) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace sedef

// Launchers implemented in the kernel translation units.
namespace sedef {
struct Ctx;

// A pass without host synchronization (one CUDA graph): every stage sizes
// its buffers and grids by these capacities, leaves its exact counts on the
// device and records overflow in `flags` instead of returning.  The counts
// in `need` (device, u64) are the exact totals, so that a caller whose
// capacities were too small learns the sizes to plan for.
struct Planned {
  int64_t rec = 0, slow_hits = 0, runs = 0, anchors = 0, chains = 0, cands = 0;
  const uint32_t* n_rec = nullptr;     // set by the sketch
  const uint32_t* n_runs = nullptr;    // set by the filter
  const uint32_t* n_chains = nullptr;  // set by the chain
  const uint32_t* n_cands = nullptr;   // set by the merge
  // device words: [0] flags (bit 0 records, 1 slow hits, 2 runs, 3 anchors,
  // 4 chains, 5 candidates over capacity; bit 6 a seed over the anchor
  // limit), [1..7] reserved; need[0..5] exact totals in the order above
  uint32_t* flags = nullptr;
  unsigned long long* need = nullptr;
  std::vector<void*> host_keep;  // pinned uploads the graph reads at replay
};
enum PlanFlag : uint32_t {
  kOverRec = 1u, kOverSlowHits = 2u, kOverRuns = 4u, kOverAnchors = 8u, kOverChains = 16u,
  kOverCands = 32u, kAnchorLimit = 64u
};
// Pinned host memory for an upload: the context's reusable buffer in an
// eager call (drains the stream first), a buffer kept for the graph's
// lifetime in a planned pass.
void* host_buf(sedef_ctx* ctx, Planned* pl, size_t bytes);
// Enqueues: need[which] = *d_count; flags |= 1 << which when it exceeds cap.
int plan_check(sedef_ctx* ctx, Planned* pl, const uint32_t* d_count, int64_t cap, int which);
int plan_check64(sedef_ctx* ctx, Planned* pl, const unsigned long long* d_count, int64_t cap,
                 int which);
// m(s) for s in [0, smax] from the parameters' tau (Section 3.1).
void mtable(const sedef_params* p, int32_t* m, int smax, double* tau_out);
int launch_pack(sedef_ctx* ctx, const uint8_t* seq, int64_t n, uint32_t* packed, uint32_t* mask,
                uint32_t* nbits);
int run_sketch(sedef_ctx* ctx, const uint32_t* packed, const uint32_t* mask, const uint32_t* nbits,
               const int64_t* h_off, int nseq, const Derived& D, uint64_t* rec, int64_t cap,
               int64_t* nrec, Planned* pl = nullptr);
int radix_sort_u64(sedef_ctx* ctx, const uint64_t* keys_in, const uint32_t* vals_in,
                   uint64_t* keys_out, uint32_t* vals_out, int64_t n, int bit_lo, int bit_hi,
                   const uint32_t* dn = nullptr);
int build_offsets(sedef_ctx* ctx, const uint64_t* sorted, int64_t n, int k, uint32_t* off,
                  const uint32_t* dn = nullptr);
int run_filter(sedef_ctx* ctx, const uint64_t* qrec, int64_t nq, const int64_t* h_qoff, int nqseq,
               const uint64_t* trec, const uint64_t* tsorted, const uint32_t* toff, int64_t nt,
               const int64_t* h_toff, int ntseq, const Derived& D, const int32_t* h_mtab,
               sedef_run_t* runs, int64_t cap, int64_t* nruns, int tune, Planned* pl = nullptr);
int filter_variant_count();
int run_chain2(sedef_ctx* ctx, const uint32_t* packed, const uint32_t* nbits, int64_t nbases,
               const sedef_region_t* d_regions, int64_t nregions, const Derived& D,
               sedef_sd_t* out, int64_t cap, int64_t* nout);
int run_extend(sedef_ctx* ctx, const sedef_run_t* runs, int64_t nruns, const uint64_t* qrec,
               int64_t nq, const int64_t* h_qoff, int nqseq, const uint64_t* trec, int64_t nt,
               const int64_t* h_toff, int ntseq, const Derived& D, const sedef_params* p,
               int64_t max_len, sedef_region_t* out, int64_t cap, int64_t* nout);
int run_chain(sedef_ctx* ctx, const sedef_run_t* runs, int64_t nruns, const uint64_t* qrec, int64_t nq,
              const int64_t* h_qoff, int nqseq, const uint64_t* tsorted, int64_t nt,
              const uint32_t* toff, const int64_t* h_toff, int ntseq, const Derived& D,
              const int32_t* h_mtab, sedef_chain_t* chains, int64_t cap, int64_t* nchains,
              Planned* pl = nullptr);
int run_merge(sedef_ctx* ctx, const sedef_chain_t* chains, int64_t nchains, const int64_t* h_qoff,
              int nqseq, const int64_t* h_toff, int ntseq, const Derived& D, sedef_cand_t* cands,
              int64_t cap, int64_t* ncands, Planned* pl = nullptr);
int scan_exclusive_u32(sedef_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       uint32_t* d_total);
// Tracing (per-kernel CUDA events on the context's stream) and launch count.
void count_launch();
void count_launches(unsigned long long n);  // kernel nodes of a graph replay
struct TraceScope {
  sedef_ctx* ctx;
  int slot;
  TraceScope(sedef_ctx* c, const char* name);
  ~TraceScope();
};
// Stage label of the traced launches (reported as "stage:kernel"); the
// previous label comes back when the scope ends.
const char* ctx_set_stage(sedef_ctx* ctx, const char* stage);
struct StageScope {
  sedef_ctx* ctx;
  const char* prev;
  StageScope(sedef_ctx* c, const char* stage) : ctx(c), prev(ctx_set_stage(c, stage)) {}
  ~StageScope() { ctx_set_stage(ctx, prev); }
};
// Context accessors for the kernel translation units.
cudaStream_t ctx_stream(sedef_ctx* ctx);
void* ctx_alloc(sedef_ctx* ctx, size_t bytes);
std::vector<char> ctx_pool_snapshot(sedef_ctx* ctx);
void ctx_pool_reset(sedef_ctx* ctx);  // every pool block free for the next call
// The context allocates its scratch in stream order and keeps a 1 MB pinned
// buffer, so that its calls never synchronize with other streams' kernels
// (a persistent kernel on another stream would hold them up).
int ctx_use_stream_ordered_alloc(sedef_ctx* ctx);
int64_t ctx_scratch_limit(sedef_ctx* ctx);  // sedef_set_scratch_limit's cap (-1: none)
void ctx_pool_restore(sedef_ctx* ctx, const std::vector<char>& used_before);
void* ctx_host(sedef_ctx* ctx, size_t bytes);  // pinned host scratch
int ctx_device(sedef_ctx* ctx);
int ctx_sm_count(sedef_ctx* ctx);
void ctx_set_stats(sedef_ctx* ctx, const int64_t* v, int n);  // last sedef_filter call
void ctx_set_anchor_total(sedef_ctx* ctx, int64_t a);         // last sedef_chain call
int ctx_filter_variant(sedef_ctx* ctx);
void ctx_set_filter_variant(sedef_ctx* ctx, int v);
// Largest shared memory per CTA that run_filter's tiers may use (default:
// no limit); a tier above it is left out and its windows go on to the next.
// Sets a kernel's dynamic shared-memory limit on the current device the
// first time it is asked for there (thread-safe; the attribute belongs to
// the device's context, so each device is set once).
int ensure_smem_attr(const void* kernel, size_t bytes);
size_t ctx_tier_smem_cap(sedef_ctx* ctx);
// Every tier but the second wide one fits in this much shared memory per CTA
// (checked where the tiers are defined).
constexpr int64_t kTierSmemFloor = 100 * 1024;
void ctx_set_tier_smem_cap(sedef_ctx* ctx, size_t bytes);
}  // namespace sedef
