// Captured self-search pass: the whole path as one CUDA graph.
//
// Every stage runs in its planned form (no host synchronization; buffers and
// grids sized by capacities; exact counts left on the device; overflow
// recorded in a flag word), so the pass can be recorded by stream capture
// once and replayed with a single cudaGraphLaunch.  The graph owns a private
// context (its stream, scratch pool and the pinned copies of the uploads
// its memcpy nodes read), so nothing it references is reused elsewhere; the
// input and output buffers are the caller's.
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

struct sedef_graph {
  sedef_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t last = nullptr;  // stream of the last launch
  sedef::Planned pl;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  sedef_graph_caps caps{};
  uint64_t* rec = nullptr;
  uint64_t* srt = nullptr;
  uint32_t* off = nullptr;
  sedef_run_t* runs = nullptr;
  sedef_chain_t* chains = nullptr;
  sedef_cand_t* cands = nullptr;
  unsigned char* d_block = nullptr;  // flags (32 B) then need[8] (u64)
  unsigned char* h_block = nullptr;  // pinned copy written by the last node
};

namespace sedef {
namespace {

constexpr size_t kBlockBytes = 32 + 8 * 8;

int record_pass(sedef_graph* g, const uint8_t* d_seq, const int64_t* h_off, int nseq,
                const Derived& D, const int32_t* mt) {
  sedef_ctx* c = g->ctx;
  cudaStream_t st = ctx_stream(c);
  const int64_t N = h_off[nseq];
  const sedef_graph_caps& cp = g->caps;
  const size_t nw16 = (size_t)((N + 15) / 16), nw32 = (size_t)((N + 31) / 32);
  uint32_t* packed = (uint32_t*)ctx_alloc(c, (nw16 ? nw16 : 1) * 4);
  uint32_t* mask = (uint32_t*)ctx_alloc(c, (nw32 ? nw32 : 1) * 4);
  uint32_t* nbits = (uint32_t*)ctx_alloc(c, (nw32 ? nw32 : 1) * 4);
  if (!packed || !mask || !nbits) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemsetAsync(g->d_block, 0, kBlockBytes, st));
  SEDEF_TRY(launch_pack(c, d_seq, N, packed, mask, nbits));
  int64_t nrec = 0, nruns = 0, nch = 0, nc = 0;
  SEDEF_TRY(run_sketch(c, packed, mask, nbits, h_off, nseq, D, g->rec, cp.records, &nrec, &g->pl));
  SEDEF_TRY(radix_sort_u64(c, g->rec, nullptr, g->srt, nullptr, cp.records, 33, 33 + 2 * D.k,
                           g->pl.n_rec));
  SEDEF_TRY(build_offsets(c, g->srt, cp.records, D.k, g->off, g->pl.n_rec));
  SEDEF_TRY(run_filter(c, g->rec, cp.records, h_off, nseq, g->rec, g->srt, g->off, cp.records,
                       h_off, nseq, D, mt, g->runs, cp.runs, &nruns, 0, &g->pl));
  SEDEF_TRY(run_chain(c, g->runs, cp.runs, g->rec, cp.records, h_off, nseq, g->srt, cp.records,
                      g->off, h_off, nseq, D, mt, g->chains, cp.chains, &nch, &g->pl));
  SEDEF_TRY(run_merge(c, g->chains, cp.chains, h_off, nseq, h_off, nseq, D, g->cands, cp.cands,
                      &nc, &g->pl));
  SEDEF_CUDA(cudaMemcpyAsync(g->h_block, g->d_block, kBlockBytes, cudaMemcpyDeviceToHost, st));
  return SEDEF_OK;
}

void free_graph(sedef_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->ctx) sedef_destroy(g->ctx);
  for (void* p : g->pl.host_keep) cudaFreeHost(p);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

}  // namespace
}  // namespace sedef

using namespace sedef;

extern "C" {

int sedef_graph_create(sedef_ctx* ctx, const uint8_t* d_seq, const int64_t* h_off, int32_t nseq,
                       const sedef_params* p, const sedef_graph_caps* caps, uint64_t* d_rec,
                       uint64_t* d_sorted, uint32_t* d_off, sedef_run_t* d_runs,
                       sedef_chain_t* d_chains, sedef_cand_t* d_cands, sedef_graph** out) {
  if (!out) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: out is NULL");
  *out = nullptr;
  if (!ctx || !p || !caps || !h_off || nseq < 1)
    return fail(SEDEF_ERR_INVALID, "sedef_graph_create: bad arguments");
  if (!d_rec || !d_sorted || !d_off || !d_runs || !d_chains || !d_cands)
    return fail(SEDEF_ERR_INVALID, "sedef_graph_create: NULL output buffer");
  if (d_rec == d_sorted) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: d_rec and d_sorted overlap");
  Derived D;
  SEDEF_TRY(derive(p, &D));
  if (h_off[0] != 0) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: offsets must start at 0");
  int64_t nwin = 0;
  for (int s = 0; s < nseq; ++s) {
    const int64_t len = h_off[s + 1] - h_off[s];
    if (len < 0) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: offsets decrease");
    if (len >= D.n) nwin += (len - D.n) / D.step + 1;
  }
  const int64_t N = h_off[nseq];
  if (N >= (int64_t(1) << 32))
    return fail(SEDEF_ERR_UNSUPPORTED, "sedef_graph_create: total length must be < 2^32");
  if (nwin == 0) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: no query window fits");
  if (!d_seq) return fail(SEDEF_ERR_INVALID, "sedef_graph_create: d_seq is NULL");
  SEDEF_CUDA(cudaSetDevice(ctx_device(ctx)));
  sedef_graph* g = new sedef_graph();
  auto bail = [&](int status) {
    free_graph(g);
    return status;
  };
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    g->stream = nullptr;
    return bail(cuda_fail(cudaGetLastError(), "sedef_graph_create: stream"));
  }
  int rc = sedef_create(ctx_device(ctx), g->stream, &g->ctx);
  if (rc != SEDEF_OK) return bail(rc);
  ctx_set_filter_variant(g->ctx, ctx_filter_variant(ctx));
  // the graph's scratch counts against the caller's cap
  if ((rc = sedef_set_scratch_limit(g->ctx, ctx_scratch_limit(ctx))) != SEDEF_OK) return bail(rc);
  auto at_least_1 = [](int64_t v) { return v < 1 ? (int64_t)1 : v; };
  g->caps.records = at_least_1(caps->records);
  g->caps.slow_hits = at_least_1(caps->slow_hits);
  g->caps.runs = at_least_1(caps->runs);
  g->caps.anchors = at_least_1(caps->anchors);
  g->caps.chains = at_least_1(caps->chains);
  g->caps.cands = at_least_1(caps->cands);
  if (g->caps.records >= (int64_t(1) << 32) || g->caps.runs >= (int64_t(1) << 32) ||
      g->caps.chains >= (int64_t(1) << 31) || g->caps.anchors >= (int64_t(1) << 32) ||
      g->caps.slow_hits >= (int64_t(1) << 32) || g->caps.cands >= (int64_t(1) << 32))
    return bail(fail(SEDEF_ERR_INVALID, "sedef_graph_create: capacities must be below 2^32"));
  g->pl.rec = g->caps.records;
  g->pl.slow_hits = g->caps.slow_hits;
  g->pl.runs = g->caps.runs;
  g->pl.anchors = g->caps.anchors;
  g->pl.chains = g->caps.chains;
  g->pl.cands = g->caps.cands;
  sedef_ctx* c = g->ctx;
  g->rec = d_rec;
  g->srt = d_sorted;
  g->off = d_off;
  g->runs = d_runs;
  g->chains = d_chains;
  g->cands = d_cands;
  g->d_block = (unsigned char*)ctx_alloc(c, kBlockBytes);
  g->h_block = (unsigned char*)host_buf(c, &g->pl, kBlockBytes);
  if (!g->d_block || !g->h_block) return bail(SEDEF_ERR_OOM);
  std::memset(g->h_block, 0, kBlockBytes);
  g->pl.flags = (uint32_t*)g->d_block;
  g->pl.need = (unsigned long long*)(g->d_block + 32);
  std::vector<int32_t> mt(kMaxWindowRecs + 1);
  mtable(p, mt.data(), kMaxWindowRecs, nullptr);

  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "sedef_graph_create: begin capture"));
  rc = record_pass(g, d_seq, h_off, nseq, D, mt.data());
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(g->stream, &graph);
  g->graph = graph;
  if (rc != SEDEF_OK) return bail(rc);
  if (ec != cudaSuccess || !graph) return bail(cuda_fail(ec, "sedef_graph_create: end capture"));
  const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
  if (ei != cudaSuccess) {
    g->exec = nullptr;
    return bail(cuda_fail(ei, "sedef_graph_create: instantiate"));
  }
  size_t nn = 0;
  SEDEF_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) SEDEF_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++g->kernels;
  }
  *out = g;
  return SEDEF_OK;
}

int sedef_graph_launch(sedef_graph* g, void* stream) {
  if (!g || !g->exec) return fail(SEDEF_ERR_INVALID, "sedef_graph_launch: no graph");
  SEDEF_CUDA(cudaSetDevice(ctx_device(g->ctx)));
  cudaStream_t st = stream ? (cudaStream_t)stream : g->stream;
  SEDEF_CUDA(cudaGraphLaunch(g->exec, st));
  g->last = st;
  count_launches((unsigned long long)g->kernels);
  return SEDEF_OK;
}

int sedef_graph_wait(sedef_graph* g, int64_t* h_need) {
  if (!g) return fail(SEDEF_ERR_INVALID, "sedef_graph_wait: no graph");
  SEDEF_CUDA(cudaSetDevice(ctx_device(g->ctx)));
  SEDEF_CUDA(cudaStreamSynchronize(g->last ? g->last : g->stream));
  uint32_t flags = 0;
  std::memcpy(&flags, g->h_block, 4);
  unsigned long long need[8];
  std::memcpy(need, g->h_block + 32, sizeof(need));
  if (h_need)
    for (int x = 0; x < 6; ++x) h_need[x] = (int64_t)need[x];
  if (flags & kAnchorLimit)
    return fail(SEDEF_ERR_UNSUPPORTED,
                "sedef_graph: a seed has more than 65536 anchors; soft-mask low-complexity "
                "repeats or set max_occ");
  if (flags & 63u) {
    static const char* names[6] = {"records", "slow_hits", "runs", "anchors", "chains", "cands"};
    std::string m = "sedef_graph: capacity exceeded:";
    for (int x = 0; x < 6; ++x)
      if (flags & (1u << x)) m += std::string(" ") + names[x] + "=" + std::to_string(need[x]);
    return fail(SEDEF_ERR_CAPACITY, m);
  }
  return SEDEF_OK;
}

int64_t sedef_graph_nodes(sedef_graph* g) { return g ? g->kernels : -1; }

int sedef_graph_destroy(sedef_graph* g) {
  if (!g) return SEDEF_OK;
  cudaSetDevice(ctx_device(g->ctx));
  if (g->last) cudaStreamSynchronize(g->last);
  free_graph(g);
  return SEDEF_OK;
}

}  // extern "C"
