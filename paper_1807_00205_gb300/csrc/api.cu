// C ABI entry points, context, scratch pool and parameter checks.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <mutex>
#include <set>
#include <tuple>

#include "common.cuh"

#include <atomic>
#include <map>

struct sedef_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  sedef::Pool pool;
  sedef::Pool io;  // buffers of sedef_selfsearch_host, kept across calls
  void* pinned = nullptr;
  size_t pinned_cap = 0;
  // tracing: one (name, start, stop) per traced launch since the last report
  bool trace = false;
  struct Mark {
    const char* stage;
    const char* name;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> spare;  // recycled events
  int64_t filter_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int filter_variant = 0;  // first-tier filter shape (sedef_filter_autotune)
  // shared memory a filter tier's CTA may ask for (a context whose kernels
  // run beside a persistent kernel leaves out the tiers that cannot fit)
  size_t tier_smem_cap = SIZE_MAX;
  // run count of the last whole self-search (its run buffer's first size
  // next time, so that a repeated search does not rerun the filter)
  int64_t last_runs = 0;
  const char* stage = "";  // label of traced launches (sedef::StageScope)
  size_t scratch_limit = SIZE_MAX;  // device bytes both pools may hold
  size_t scratch_held = 0;
};

namespace sedef {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SEDEF_ERR_OOM : SEDEF_ERR_CUDA;
}

void* Pool::alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  int best = -1;
  for (size_t b = 0; b < blocks.size(); ++b)
    if (!blocks[b].used && blocks[b].size >= bytes &&
        (best < 0 || blocks[b].size < blocks[best].size))
      best = (int)b;
  if (best >= 0) {
    blocks[best].used = true;
    return blocks[best].ptr;
  }
  if (limit && held && *held + bytes > *limit) return nullptr;
  void* p = nullptr;
  const cudaError_t e = ordered ? cudaMallocAsync(&p, bytes, *ordered) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (held) *held += bytes;
  blocks.push_back({p, bytes, true});
  return p;
}

void Pool::reset() {
  for (auto& b : blocks) b.used = false;
}

std::vector<char> Pool::snapshot() const {
  std::vector<char> u(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) u[b] = blocks[b].used ? 1 : 0;
  return u;
}

void Pool::restore(const std::vector<char>& used_before) {
  for (size_t b = 0; b < blocks.size(); ++b)
    if (b >= used_before.size() || !used_before[b]) blocks[b].used = false;
}

void Pool::release() {
  for (auto& b : blocks) {
    if (ordered) cudaFreeAsync(b.ptr, *ordered); else cudaFree(b.ptr);
    if (held) *held -= b.size;
  }
  blocks.clear();
}

int ensure_smem_attr(const void* kernel, size_t bytes) {
  // The attribute is one maximum per kernel and device: it is only ever
  // raised, so a launch with fewer bytes after a larger one stays valid.
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> raised;
  int dev = 0;
  SEDEF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  size_t& cur = raised[std::make_pair(dev, kernel)];
  if (bytes <= cur) return SEDEF_OK;
  SEDEF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return SEDEF_OK;
}

static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static cudaEvent_t take_event(sedef_ctx* c) {
  if (!c->spare.empty()) {
    cudaEvent_t e = c->spare.back();
    c->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

TraceScope::TraceScope(sedef_ctx* c, const char* name) : ctx(c), slot(-1) {
  if (!c || !c->trace) return;
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return;
  cudaEventRecord(a, c->stream);
  c->marks.push_back({c->stage, name, a, b});
  slot = (int)c->marks.size() - 1;
}

TraceScope::~TraceScope() {
  if (slot >= 0) cudaEventRecord(ctx->marks[slot].stop, ctx->stream);
}

cudaStream_t ctx_stream(sedef_ctx* ctx) { return ctx->stream; }
void ctx_pool_reset(sedef_ctx* ctx) { ctx->pool.reset(); }
int ctx_use_stream_ordered_alloc(sedef_ctx* ctx) {
  ctx->pool.ordered = ctx->io.ordered = &ctx->stream;
  if (!ctx_host(ctx, 1 << 20)) return SEDEF_ERR_OOM;
  return SEDEF_OK;
}
int64_t ctx_scratch_limit(sedef_ctx* ctx) {
  return ctx->scratch_limit == SIZE_MAX ? -1 : (int64_t)ctx->scratch_limit;
}

const char* ctx_set_stage(sedef_ctx* ctx, const char* stage) {
  if (!ctx) return "";
  const char* prev = ctx->stage;
  ctx->stage = stage ? stage : "";
  return prev;
}

int ctx_filter_variant(sedef_ctx* ctx) { return ctx->filter_variant; }
void ctx_set_filter_variant(sedef_ctx* ctx, int v) { ctx->filter_variant = v; }
size_t ctx_tier_smem_cap(sedef_ctx* ctx) { return ctx->tier_smem_cap; }
void ctx_set_tier_smem_cap(sedef_ctx* ctx, size_t bytes) { ctx->tier_smem_cap = bytes; }

void ctx_set_stats(sedef_ctx* ctx, const int64_t* v, int n) {
  for (int x = 0; x < 7; ++x) ctx->filter_stats[x] = x < n ? v[x] : 0;
}
void ctx_set_anchor_total(sedef_ctx* ctx, int64_t a) { ctx->filter_stats[7] = a; }
int ctx_device(sedef_ctx* ctx) { return ctx->device; }
int ctx_sm_count(sedef_ctx* ctx) { return ctx->sm_count; }

void* host_buf(sedef_ctx* ctx, Planned* pl, size_t bytes) {
  if (!pl) return ctx_host(ctx, bytes);
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes < 64 ? 64 : bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned host allocation failed");
    return nullptr;
  }
  pl->host_keep.push_back(p);
  return p;
}

namespace {
__global__ void k_plan_check(const uint32_t* count, int64_t cap, int which, uint32_t* flags,
                             unsigned long long* need) {
  const uint32_t v = *count;
  need[which] = v;
  if ((int64_t)v > cap) atomicOr(flags, 1u << which);
}
}  // namespace

__global__ void k_plan_check64(const unsigned long long* count, int64_t cap, int which,
                               uint32_t* flags, unsigned long long* need) {
  const unsigned long long v = *count;
  need[which] = v;
  if (v > (unsigned long long)cap) atomicOr(flags, 1u << which);
}

int plan_check64(sedef_ctx* ctx, Planned* pl, const unsigned long long* d_count, int64_t cap,
                 int which) {
  SEDEF_KERNEL(ctx, "k_plan_check",
               k_plan_check64<<<1, 1, 0, ctx->stream>>>(d_count, cap, which, pl->flags, pl->need));
  return SEDEF_OK;
}

int plan_check(sedef_ctx* ctx, Planned* pl, const uint32_t* d_count, int64_t cap, int which) {
  SEDEF_KERNEL(ctx, "k_plan_check",
               k_plan_check<<<1, 1, 0, ctx->stream>>>(d_count, cap, which, pl->flags, pl->need));
  return SEDEF_OK;
}

std::vector<char> ctx_pool_snapshot(sedef_ctx* ctx) { return ctx->pool.snapshot(); }
void ctx_pool_restore(sedef_ctx* ctx, const std::vector<char>& used_before) {
  ctx->pool.restore(used_before);
}

void* ctx_alloc(sedef_ctx* ctx, size_t bytes) {
  void* p = ctx->pool.alloc(bytes);
  if (!p) set_error("device scratch allocation of " + std::to_string(bytes) + " bytes failed");
  return p;
}

// Pinned staging for small uploads and counters.  The stream is drained
// before the buffer is handed out again, so an earlier async copy from it
// has completed.
void* ctx_host(sedef_ctx* ctx, size_t bytes) {
  cudaStreamSynchronize(ctx->stream);
  if (bytes > ctx->pinned_cap) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    size_t cap = bytes < 65536 ? 65536 : bytes * 2;
    if (cudaMallocHost(&ctx->pinned, cap) != cudaSuccess) {
      cudaGetLastError();
      ctx->pinned_cap = 0;
      set_error("pinned host allocation failed");
      return nullptr;
    }
    ctx->pinned_cap = cap;
  }
  return ctx->pinned;
}

int derive(const sedef_params* p, Derived* d) {
  if (!p) return fail(SEDEF_ERR_INVALID, "params is NULL");
  if (p->k < 2 || p->k > 15) return fail(SEDEF_ERR_UNSUPPORTED, "k must be in [2, 15]");
  if (p->w < 1 || p->w > 256) return fail(SEDEF_ERR_UNSUPPORTED, "w must be in [1, 256]");
  if (p->n <= p->k) return fail(SEDEF_ERR_UNSUPPORTED, "n must exceed k");
  if (p->n - p->k + 1 > kMaxWindowRecs)
    return fail(SEDEF_ERR_UNSUPPORTED, "n - k + 1 must be at most 1024");
  if (p->query_step < 1) return fail(SEDEF_ERR_INVALID, "query_step must be >= 1");
  if (p->max_occ < 0 || p->gap_max < 0 || p->diag_max < 0 || p->min_unmasked < 0)
    return fail(SEDEF_ERR_INVALID, "negative limit");
  if (!(p->delta_m >= 0 && p->delta_g >= 0 && p->delta_g < 1))
    return fail(SEDEF_ERR_INVALID, "delta_m, delta_g out of range");
  d->k = p->k;
  d->w = p->w;
  d->n = p->n;
  d->span = p->n - p->k;
  d->step = p->query_step;
  d->max_occ = p->max_occ;
  if (p->self_mode < 0 || p->self_mode > 2) return fail(SEDEF_ERR_INVALID, "self_mode must be 0, 1 or 2");
  d->self_mode = p->self_mode;
  d->gap_max = p->gap_max;
  d->diag_max = p->diag_max;
  d->min_unmasked = p->min_unmasked;
  d->overlap = (int)std::floor((p->delta_m + p->delta_g) * (double)p->n);
  d->kmask = (uint32_t)((1ull << (2 * p->k)) - 1);
  d->delta_g = p->delta_g;
  return SEDEF_OK;
}

// m(s) table for s in [0, smax] (Section 3.1 tau; Section 2.2 count test).
void mtable(const sedef_params* p, int32_t* m, int smax, double* tau_out) {
  const double tau = (1.0 - p->delta_g) / (1.0 + p->delta_g) *
                     (1.0 / (2.0 * std::exp((double)p->k * p->delta_m) - 1.0));
  if (tau_out) *tau_out = tau;
  if (!m) return;
  for (int s = 0; s <= smax; ++s) {
    double need = tau * (double)s - 1e-9;
    int32_t v = (int32_t)std::ceil(need);
    if (v < 0) v = 0;
    // least integer >= need
    while ((double)(v - 1) >= need && v > 0) --v;
    while ((double)v < need) ++v;
    m[s] = v;
  }
}

static int check_offsets(const int64_t* off, int nseq, const char* what) {
  if (nseq < 0 || (nseq > 0 && !off)) return fail(SEDEF_ERR_INVALID, std::string(what) + ": bad offsets");
  if (nseq == 0) return SEDEF_OK;
  if (off[0] != 0) return fail(SEDEF_ERR_INVALID, std::string(what) + ": offsets must start at 0");
  for (int s = 0; s < nseq; ++s)
    if (off[s + 1] < off[s]) return fail(SEDEF_ERR_INVALID, std::string(what) + ": offsets decrease");
  if (off[nseq] >= (int64_t(1) << 32))
    return fail(SEDEF_ERR_UNSUPPORTED, std::string(what) + ": total length must be < 2^32");
  return SEDEF_OK;
}

}  // namespace sedef

using namespace sedef;

extern "C" {

void sedef_default_params(sedef_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->k = 12;
  p->w = 16;
  p->n = 750;
  p->query_step = 250;
  p->max_occ = 0;
  p->self_mode = 1;
  p->gap_max = 750;
  p->diag_max = 75;
  p->min_unmasked = 1;
  p->delta_m = 0.15;
  p->delta_g = 0.10;
}

const char* sedef_last_error(void) { return g_last_error.c_str(); }

int sedef_create(int device, void* stream, sedef_ctx** out) {
  if (!out) return fail(SEDEF_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  SEDEF_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(SEDEF_ERR_INVALID, "no such device");
  SEDEF_CUDA(cudaSetDevice(device));
  sedef_ctx* c = new sedef_ctx();
  c->device = device;
  c->pool.device = device;
  c->io.device = device;
  c->stream = (cudaStream_t)stream;
  c->pool.limit = c->io.limit = &c->scratch_limit;
  c->pool.held = c->io.held = &c->scratch_held;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return SEDEF_OK;
}

int sedef_destroy(sedef_ctx* ctx) {
  if (!ctx) return SEDEF_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& m : ctx->marks) {
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  for (auto e : ctx->spare) cudaEventDestroy(e);
  ctx->pool.release();
  ctx->io.release();
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
  return SEDEF_OK;
}

int sedef_set_scratch_limit(sedef_ctx* ctx, int64_t bytes) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  SEDEF_CUDA(cudaStreamSynchronize(ctx->stream));
  // blocks above the new limit are given back first
  if (bytes >= 0 && ctx->scratch_held > (size_t)bytes) {
    ctx->pool.release();
    ctx->io.release();
  }
  ctx->scratch_limit = bytes < 0 ? SIZE_MAX : (size_t)bytes;
  return SEDEF_OK;
}

int sedef_set_tier_smem_limit(sedef_ctx* ctx, int64_t bytes) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  if (bytes >= 0 && bytes < kTierSmemFloor)
    return fail(SEDEF_ERR_UNSUPPORTED,
                "sedef_set_tier_smem_limit: the filter tiers other than the second wide tier "
                "need up to 100 KB per CTA");
  ctx->tier_smem_cap = bytes < 0 ? SIZE_MAX : (size_t)bytes;
  return SEDEF_OK;
}

int sedef_set_stream(sedef_ctx* ctx, void* stream) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = (cudaStream_t)stream;
  return SEDEF_OK;
}

int sedef_trace_enable(sedef_ctx* ctx, int on) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  ctx->trace = on != 0;
  return SEDEF_OK;
}

int sedef_trace_report(sedef_ctx* ctx, char* buf, int64_t cap, int reset) {
  if (!ctx || (cap > 0 && !buf)) return fail(SEDEF_ERR_INVALID, "bad arguments");
  SEDEF_CUDA(cudaStreamSynchronize(ctx->stream));
  std::map<std::string, std::pair<long, double>> agg;
  std::vector<std::string> order;
  for (auto& m : ctx->marks) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m.start, m.stop);
    const std::string key = m.stage[0] ? std::string(m.stage) + ":" + m.name : std::string(m.name);
    auto it = agg.find(key);
    if (it == agg.end()) {
      order.push_back(key);
      agg[key] = {1, ms};
    } else {
      it->second.first += 1;
      it->second.second += ms;
    }
  }
  std::string out;
  char line[256];
  for (auto& n : order) {
    std::snprintf(line, sizeof(line), "%s %ld %.6f\n", n.c_str(), agg[n].first, agg[n].second);
    out += line;
  }
  if (reset) {
    for (auto& m : ctx->marks) {
      ctx->spare.push_back(m.start);
      ctx->spare.push_back(m.stop);
    }
    ctx->marks.clear();
  }
  if (cap > 0) {
    const size_t n = out.size() < (size_t)(cap - 1) ? out.size() : (size_t)(cap - 1);
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return (int)out.size();
}

uint64_t sedef_launch_count(void) { return g_launches.load(); }

int sedef_filter_stats(sedef_ctx* ctx, int64_t* out, int32_t n) {
  if (!ctx || (n > 0 && !out)) return fail(SEDEF_ERR_INVALID, "bad arguments");
  for (int x = 0; x < n && x < 8; ++x) out[x] = ctx->filter_stats[x];
  return SEDEF_OK;
}

int sedef_threshold_table(const sedef_params* p, int32_t* m_out, int32_t smax, double* tau_out) {
  Derived d;
  SEDEF_TRY(derive(p, &d));
  if (smax < 0) return fail(SEDEF_ERR_INVALID, "smax < 0");
  mtable(p, m_out, smax, tau_out);
  return SEDEF_OK;
}

int sedef_pack(sedef_ctx* ctx, const uint8_t* d_seq, int64_t n, uint32_t* d_packed,
               uint32_t* d_mask, uint32_t* d_nbits) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  if (n < 0) return fail(SEDEF_ERR_INVALID, "n < 0");
  if (n == 0) return SEDEF_OK;
  if (!d_seq || !d_packed || !d_mask || !d_nbits) return fail(SEDEF_ERR_INVALID, "NULL buffer");
  if (n >= (int64_t(1) << 32)) return fail(SEDEF_ERR_UNSUPPORTED, "n must be < 2^32");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  StageScope stage(ctx, "pack");
  return launch_pack(ctx, d_seq, n, d_packed, d_mask, d_nbits);
}

int sedef_sketch(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_mask,
                 const uint32_t* d_nbits, const int64_t* h_seq_off, int32_t nseq,
                 const sedef_params* p, uint64_t* d_rec, int64_t rec_cap, int64_t* h_nrec) {
  if (!ctx || !h_nrec) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_seq_off, nseq, "sedef_sketch"));
  *h_nrec = 0;
  if (nseq == 0 || h_seq_off[nseq] == 0) return SEDEF_OK;
  if (!d_packed || !d_mask || !d_nbits) return fail(SEDEF_ERR_INVALID, "NULL input buffer");
  if (rec_cap > 0 && !d_rec) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  StageScope stage(ctx, "sketch");
  return run_sketch(ctx, d_packed, d_mask, d_nbits, h_seq_off, nseq, D, d_rec, rec_cap, h_nrec);
}

int sedef_index(sedef_ctx* ctx, const uint64_t* d_rec, int64_t nrec, const sedef_params* p,
                uint64_t* d_sorted, uint32_t* d_off) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  if (nrec < 0 || nrec >= (int64_t(1) << 32)) return fail(SEDEF_ERR_INVALID, "bad nrec");
  if (!d_off || (nrec > 0 && (!d_rec || !d_sorted))) return fail(SEDEF_ERR_INVALID, "NULL buffer");
  if (nrec > 0 && d_rec == d_sorted) return fail(SEDEF_ERR_INVALID, "d_rec and d_sorted overlap");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  StageScope stage(ctx, "index");
  if (nrec > 0)
    SEDEF_TRY(radix_sort_u64(ctx, d_rec, nullptr, d_sorted, nullptr, nrec, 33, 33 + 2 * D.k));
  return build_offsets(ctx, d_sorted, nrec, D.k, d_off);
}

int sedef_filter(sedef_ctx* ctx, const uint64_t* d_qrec, int64_t nq, const int64_t* h_qoff,
                 int32_t nqseq, const uint64_t* d_trec, const uint64_t* d_tsorted,
                 const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                 const sedef_params* p, sedef_run_t* d_runs, int64_t run_cap, int64_t* h_nruns) {
  if (!ctx || !h_nruns) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_qoff, nqseq, "query"));
  SEDEF_TRY(check_offsets(h_toff, ntseq, "target"));
  if (D.self_mode && (nqseq != ntseq || d_qrec != d_trec || nq != nt))
    return fail(SEDEF_ERR_INVALID, "self mode needs identical query and target");
  if (D.self_mode)
    for (int s = 0; s <= nqseq; ++s)
      if (h_qoff[s] != h_toff[s]) return fail(SEDEF_ERR_INVALID, "self mode offsets differ");
  if (nq < 0 || nt < 0 || (nq > 0 && !d_qrec) || (nt > 0 && (!d_trec || !d_tsorted)) || !d_toff)
    return fail(SEDEF_ERR_INVALID, "bad record arrays");
  if (run_cap > 0 && !d_runs) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  std::vector<int32_t> mt(kMaxWindowRecs + 1);
  mtable(p, mt.data(), kMaxWindowRecs, nullptr);
  *h_nruns = 0;
  StageScope stage(ctx, "filter");
  return run_filter(ctx, d_qrec, nq, h_qoff, nqseq, d_trec, d_tsorted, d_toff, nt, h_toff, ntseq,
                    D, mt.data(), d_runs, run_cap, h_nruns, 0);
}

int sedef_filter_autotune(sedef_ctx* ctx, const uint64_t* d_qrec, int64_t nq, const int64_t* h_qoff,
                          int32_t nqseq, const uint64_t* d_trec, const uint64_t* d_tsorted,
                          const uint32_t* d_toff, int64_t nt, const int64_t* h_toff,
                          int32_t ntseq, const sedef_params* p, int32_t* variant_out) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_qoff, nqseq, "query"));
  SEDEF_TRY(check_offsets(h_toff, ntseq, "target"));
  if (nq < 0 || nt < 0 || (nq > 0 && !d_qrec) || (nt > 0 && (!d_trec || !d_tsorted)) || !d_toff)
    return fail(SEDEF_ERR_INVALID, "bad record arrays");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  std::vector<int32_t> mt(kMaxWindowRecs + 1);
  mtable(p, mt.data(), kMaxWindowRecs, nullptr);
  int64_t chosen = 0;
  // runs from the timing passes are discarded (capacity 1)
  sedef_run_t* scratch = (sedef_run_t*)ctx_alloc(ctx, sizeof(sedef_run_t));
  if (!scratch) return SEDEF_ERR_OOM;
  SEDEF_TRY(run_filter(ctx, d_qrec, nq, h_qoff, nqseq, d_trec, d_tsorted, d_toff, nt, h_toff, ntseq,
                       D, mt.data(), scratch, 1, &chosen, 1));
  SEDEF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (variant_out) *variant_out = (int32_t)ctx->filter_variant;
  return SEDEF_OK;
}

int sedef_filter_variant(sedef_ctx* ctx, int32_t set, int32_t* current, int32_t* count) {
  if (!ctx) return fail(SEDEF_ERR_INVALID, "ctx is NULL");
  if (set >= filter_variant_count()) return fail(SEDEF_ERR_INVALID, "no such variant");
  if (set >= 0) ctx->filter_variant = set;
  if (current) *current = ctx->filter_variant;
  if (count) *count = filter_variant_count();
  return SEDEF_OK;
}

int sedef_chain(sedef_ctx* ctx, const sedef_run_t* d_runs, int64_t nruns, const uint64_t* d_qrec,
                int64_t nq, const int64_t* h_qoff, int32_t nqseq, const uint64_t* d_tsorted,
                const uint32_t* d_toff, int64_t nt, const int64_t* h_toff, int32_t ntseq,
                const sedef_params* p, sedef_chain_t* d_chains, int64_t cap, int64_t* h_nchains) {
  if (!ctx || !h_nchains) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_qoff, nqseq, "query"));
  SEDEF_TRY(check_offsets(h_toff, ntseq, "target"));
  if (nruns < 0 || (nruns > 0 && !d_runs)) return fail(SEDEF_ERR_INVALID, "bad runs");
  if (cap > 0 && !d_chains) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  std::vector<int32_t> mt(kMaxWindowRecs + 1);
  mtable(p, mt.data(), kMaxWindowRecs, nullptr);
  *h_nchains = 0;
  if (nruns == 0) return SEDEF_OK;
  if ((nq > 0 && !d_qrec) || (nt > 0 && !d_tsorted) || !d_toff)
    return fail(SEDEF_ERR_INVALID, "bad record arrays");
  StageScope stage(ctx, "chain");
  return run_chain(ctx, d_runs, nruns, d_qrec, nq, h_qoff, nqseq, d_tsorted, nt, d_toff, h_toff,
                   ntseq, D, mt.data(), d_chains, cap, h_nchains);
}

int sedef_extend(sedef_ctx* ctx, const sedef_run_t* d_runs, int64_t nruns, const uint64_t* d_qext,
                 int64_t nq, const int64_t* h_qoff, int32_t nqseq, const uint64_t* d_text,
                 int64_t nt, const int64_t* h_toff, int32_t ntseq, const sedef_params* p,
                 int64_t max_len, sedef_region_t* d_regions, int64_t cap, int64_t* h_nregions) {
  if (!ctx || !h_nregions) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_qoff, nqseq, "query"));
  SEDEF_TRY(check_offsets(h_toff, ntseq, "target"));
  *h_nregions = 0;
  if (D.k > 12) return fail(SEDEF_ERR_UNSUPPORTED, "sedef_extend: k must be at most 12");
  if (max_len < D.n || max_len >= (int64_t(1) << 31))
    return fail(SEDEF_ERR_INVALID, "sedef_extend: max_len must be in [n, 2^31)");
  if (nruns < 0 || (nruns > 0 && !d_runs)) return fail(SEDEF_ERR_INVALID, "bad runs");
  if (nq < 0 || nt < 0 || (nq > 0 && !d_qext) || (nt > 0 && !d_text))
    return fail(SEDEF_ERR_INVALID, "bad record arrays");
  if (D.self_mode && (nqseq != ntseq || d_qext != d_text || nq != nt))
    return fail(SEDEF_ERR_INVALID, "self mode needs identical query and target");
  if (cap > 0 && !d_regions) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  if (nruns == 0) return SEDEF_OK;
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  StageScope stage(ctx, "extend");
  return run_extend(ctx, d_runs, nruns, d_qext, nq, h_qoff, nqseq, d_text, nt, h_toff, ntseq, D,
                    p, max_len, d_regions, cap, h_nregions);
}

int sedef_chain2(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_nbits, int64_t nbases,
                 const sedef_region_t* d_regions, int64_t nregions, const sedef_params* p,
                 sedef_sd_t* d_out, int64_t cap, int64_t* h_nout) {
  if (!ctx || !h_nout) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  *h_nout = 0;
  if (nregions < 0 || (nregions > 0 && !d_regions)) return fail(SEDEF_ERR_INVALID, "bad regions");
  if (nbases < 0 || (nbases > 0 && (!d_packed || !d_nbits)))
    return fail(SEDEF_ERR_INVALID, "bad packed sequence");
  if (cap > 0 && !d_out) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  if (nregions == 0) return SEDEF_OK;
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  StageScope stage(ctx, "chain2");
  return run_chain2(ctx, d_packed, d_nbits, nbases, d_regions, nregions, D, d_out, cap, h_nout);
}

int sedef_merge(sedef_ctx* ctx, const sedef_chain_t* d_chains, int64_t nchains,
                const int64_t* h_qoff, int32_t nqseq, const int64_t* h_toff, int32_t ntseq,
                const sedef_params* p, sedef_cand_t* d_cands, int64_t cap, int64_t* h_ncands) {
  if (!ctx || !h_ncands) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_qoff, nqseq, "query"));
  SEDEF_TRY(check_offsets(h_toff, ntseq, "target"));
  if (nchains < 0 || (nchains > 0 && !d_chains)) return fail(SEDEF_ERR_INVALID, "bad chains");
  if (cap > 0 && !d_cands) return fail(SEDEF_ERR_INVALID, "NULL output buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  ctx->pool.reset();
  *h_ncands = 0;
  if (nchains == 0) return SEDEF_OK;
  StageScope stage(ctx, "merge");
  return run_merge(ctx, d_chains, nchains, h_qoff, nqseq, h_toff, ntseq, D, d_cands, cap, h_ncands);
}

}  // extern "C"

namespace {

// The whole self-search on a device-resident sequence: pack, sketch, index,
// filter (with refine), chain and merge on the context's stream.  Device
// buffers come from the context's I/O pool (reused by the next call,
// released by sedef_destroy); *cands points into it on return.
int selfsearch_device(sedef_ctx* ctx, const uint8_t* seq, const int64_t* h_seq_off, int32_t nseq,
                      const sedef_params* p, const sedef::Derived& D, sedef_cand_t** cands_out,
                      int64_t* nc_out) {
  using namespace sedef;
  const int64_t N = h_seq_off[nseq];
  uint32_t *packed = nullptr, *mask = nullptr, *nbits = nullptr, *off = nullptr;
  uint64_t *rec = nullptr, *sorted = nullptr;
  sedef_run_t* runs = nullptr;
  sedef_chain_t* chains = nullptr;
  sedef_cand_t* cands = nullptr;
  int status = SEDEF_OK;
  int64_t nrec = 0, nruns = 0, nch = 0, nc = 0;
  const size_t nwords16 = (size_t)((N + 15) / 16), nwords32 = (size_t)((N + 31) / 32);
#define DALLOC(ptr, bytes)                                                 \
  do {                                                                     \
    ptr = (decltype(ptr))ctx->io.alloc((bytes) ? (bytes) : 256);           \
    if (!ptr) return fail(SEDEF_ERR_OOM, "selfsearch: device allocation failed"); \
  } while (0)
  DALLOC(packed, nwords16 * 4);
  DALLOC(mask, nwords32 * 4);
  DALLOC(nbits, nwords32 * 4);
  SEDEF_TRY(sedef_pack(ctx, seq, N, packed, mask, nbits));
  // sketch: start from the expected density and grow once if needed
  int64_t rcap = N / 4 + 1024;
  DALLOC(rec, (size_t)rcap * 8);
  status = sedef_sketch(ctx, packed, mask, nbits, h_seq_off, nseq, p, rec, rcap, &nrec);
  if (status == SEDEF_ERR_CAPACITY) {
    rcap = nrec;
    DALLOC(rec, (size_t)rcap * 8);
    status = sedef_sketch(ctx, packed, mask, nbits, h_seq_off, nseq, p, rec, rcap, &nrec);
  }
  SEDEF_TRY(status);
  DALLOC(sorted, (size_t)(nrec ? nrec : 1) * 8);
  DALLOC(off, ((size_t(1) << (2 * D.k)) + 1) * 4);
  SEDEF_TRY(sedef_index(ctx, rec, nrec, p, sorted, off));
  // runs: the larger of a density guess and the last search's count
  int64_t fcap = N / 32 + 4096;
  if (ctx->last_runs + ctx->last_runs / 8 > fcap) fcap = ctx->last_runs + ctx->last_runs / 8;
  DALLOC(runs, (size_t)fcap * sizeof(sedef_run_t));
  status = sedef_filter(ctx, rec, nrec, h_seq_off, nseq, rec, sorted, off, nrec, h_seq_off, nseq, p,
                        runs, fcap, &nruns);
  if (status == SEDEF_ERR_CAPACITY) {
    fcap = nruns;
    DALLOC(runs, (size_t)fcap * sizeof(sedef_run_t));
    status = sedef_filter(ctx, rec, nrec, h_seq_off, nseq, rec, sorted, off, nrec, h_seq_off, nseq,
                          p, runs, fcap, &nruns);
  }
  SEDEF_TRY(status);
  ctx->last_runs = nruns;
  DALLOC(chains, (size_t)(nruns ? nruns : 1) * sizeof(sedef_chain_t));
  SEDEF_TRY(sedef_chain(ctx, runs, nruns, rec, nrec, h_seq_off, nseq, sorted, off, nrec, h_seq_off,
                        nseq, p, chains, nruns, &nch));
  DALLOC(cands, (size_t)(nch ? nch : 1) * sizeof(sedef_cand_t));
  SEDEF_TRY(sedef_merge(ctx, chains, nch, h_seq_off, nseq, h_seq_off, nseq, p, cands, nch, &nc));
#undef DALLOC
  *cands_out = cands;
  *nc_out = nc;
  return SEDEF_OK;
}

}  // namespace

extern "C" {

int sedef_selfsearch(sedef_ctx* ctx, const uint8_t* d_seq, const int64_t* h_seq_off, int32_t nseq,
                     const sedef_params* p, sedef_cand_t* d_cands, int64_t cap,
                     int64_t* h_ncands) {
  if (!ctx || !h_ncands) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_seq_off, nseq, "sedef_selfsearch"));
  if (!D.self_mode) return fail(SEDEF_ERR_INVALID, "self search needs self_mode 1 or 2");
  *h_ncands = 0;
  if (nseq == 0 || h_seq_off[nseq] == 0) return SEDEF_OK;
  if (!d_seq || (cap > 0 && !d_cands)) return fail(SEDEF_ERR_INVALID, "NULL buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ctx->io.reset();
  sedef_cand_t* cands = nullptr;
  int64_t nc = 0;
  const int status = selfsearch_device(ctx, d_seq, h_seq_off, nseq, p, D, &cands, &nc);
  if (status != SEDEF_OK) {
    cudaStreamSynchronize(st);
    return status;
  }
  *h_ncands = nc;
  if (nc > cap) {
    cudaStreamSynchronize(st);
    return fail(SEDEF_ERR_CAPACITY, "selfsearch: candidate buffer too small");
  }
  if (nc > 0)
    SEDEF_CUDA(cudaMemcpyAsync(d_cands, cands, (size_t)nc * sizeof(sedef_cand_t),
                               cudaMemcpyDeviceToDevice, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

int sedef_selfsearch_host(sedef_ctx* ctx, const uint8_t* h_seq, const int64_t* h_seq_off,
                          int32_t nseq, const sedef_params* p, sedef_cand_t* h_cands, int64_t cap,
                          int64_t* h_ncands) {
  if (!ctx || !h_ncands) return fail(SEDEF_ERR_INVALID, "NULL argument");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  SEDEF_TRY(check_offsets(h_seq_off, nseq, "sedef_selfsearch_host"));
  if (!D.self_mode) return fail(SEDEF_ERR_INVALID, "self search needs self_mode 1 or 2");
  *h_ncands = 0;
  if (nseq == 0 || h_seq_off[nseq] == 0) return SEDEF_OK;
  if (!h_seq || (cap > 0 && !h_cands)) return fail(SEDEF_ERR_INVALID, "NULL buffer");
  SEDEF_CUDA(cudaSetDevice(ctx->device));
  const int64_t N = h_seq_off[nseq];
  cudaStream_t st = ctx->stream;
  ctx->io.reset();
  // Page-locked input is read by the pack kernel in place, through its
  // device mapping (one pass over the host link, no staging copy); any other
  // host memory is copied to the device first.
  const uint8_t* seq = nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, h_seq) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr) {
    seq = (const uint8_t*)at.devicePointer;
  } else {
    cudaGetLastError();
    uint8_t* d = (uint8_t*)ctx->io.alloc((size_t)N);
    if (!d) return fail(SEDEF_ERR_OOM, "selfsearch: device allocation failed");
    if (cudaMemcpyAsync(d, h_seq, (size_t)N, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaStreamSynchronize(st);
      return fail(SEDEF_ERR_CUDA, "selfsearch: H2D copy failed");
    }
    seq = d;
  }
  sedef_cand_t* cands = nullptr;
  int64_t nc = 0;
  const int status = selfsearch_device(ctx, seq, h_seq_off, nseq, p, D, &cands, &nc);
  if (status != SEDEF_OK) {
    cudaStreamSynchronize(st);
    return status;
  }
  *h_ncands = nc;
  if (nc > cap) {
    cudaStreamSynchronize(st);
    return fail(SEDEF_ERR_CAPACITY, "selfsearch: candidate buffer too small");
  }
  if (nc > 0 &&
      cudaMemcpyAsync(h_cands, cands, (size_t)nc * sizeof(sedef_cand_t), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess) {
    cudaStreamSynchronize(st);
    return fail(SEDEF_ERR_CUDA, "selfsearch: D2H copy failed");
  }
  SEDEF_CUDA(cudaStreamSynchronize(st));
  return SEDEF_OK;
}

}  // extern "C"
