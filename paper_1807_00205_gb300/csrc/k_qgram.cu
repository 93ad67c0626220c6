// f3: the q-gram filter of Section 3.2 on kept seeds.
//
// For a seed (i, j*, o) the two windows X = G[i, i+n) and Y = G[j*, j*+n)
// (Y reverse-complemented when o = 1) share Q q-grams, counted with
// multiplicity: for every q-gram, the smaller of its occurrence counts in X
// and in Y; q-grams over a non-ACGT base are not counted.  Section 3.2's
// adapted q-gram lemma bounds Q from below for any pair within the SD error
// model by B = n (1 - delta_G - q delta_M) - (n p_G + 1)(q - 1); a seed
// passes when Q >= the least integer >= B (with a 1e-9 margin, in double on
// the host).
//
// One warp per run: the warp histograms the q-grams of X and of Y (4^q
// 32-bit bins each, q <= 5, in shared memory), then sums the bin-wise
// minima.  The reverse complement of Y's q-gram at G[a, a+q) is formed
// directly from the bases (complement = 3 - code, order reversed).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sedef {
namespace {

constexpr int kQgWarps = 8;
constexpr int kMaxQ = 5;
constexpr int kMaxBins = 1 << (2 * kMaxQ);

struct QgArgs {
  const uint32_t* packed;
  const uint32_t* nbits;
  const sedef_run_t* runs;
  int64_t nruns;
  int n, q, need;
  uint32_t* shared;
  uint8_t* pass;
  unsigned long long* npass;
};

__device__ __forceinline__ uint32_t base_at(const uint32_t* packed, int64_t p) {
  return (packed[p >> 4] >> (2 * (p & 15))) & 3u;
}

__device__ __forceinline__ bool is_n(const uint32_t* nbits, int64_t p) {
  return (nbits[p >> 5] >> (p & 31)) & 1u;
}

// Adds every valid q-gram of G[a, a+n) to h (reverse complements when rc).
__device__ void histogram(const QgArgs& A, int64_t a, bool rc, uint32_t* h) {
  const int lane = lane_id();
  for (int64_t x = a + lane; x + A.q <= a + A.n; x += 32) {
    uint32_t g = 0;
    bool ok = true;
    for (int t = 0; t < A.q; ++t) {
      const int64_t p = x + t;
      if (is_n(A.nbits, p)) {
        ok = false;
        break;
      }
      const uint32_t b = base_at(A.packed, p);
      g = rc ? (g | ((3u - b) << (2 * t))) : ((g << 2) | b);
    }
    if (ok) atomicAdd(&h[g], 1u);
  }
}

__global__ void __launch_bounds__(32 * kQgWarps) k_qgram(QgArgs A) {
  extern __shared__ uint32_t qg_smem[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int bins = 1 << (2 * A.q);
  uint32_t* hx = qg_smem + (size_t)warp * 2 * bins;
  uint32_t* hy = hx + bins;
  const int64_t stride = (int64_t)gridDim.x * kQgWarps;
  for (int64_t r = (int64_t)blockIdx.x * kQgWarps + warp; r < A.nruns; r += stride) {
    const sedef_run_t run = A.runs[r];
    if (!run.keep) {
      if (lane == 0) {
        A.shared[r] = 0;
        A.pass[r] = 0;
      }
      continue;
    }
    for (int b = lane; b < 2 * bins; b += 32) hx[b] = 0;
    __syncwarp();
    histogram(A, run.i, false, hx);
    histogram(A, run.j_star, run.o != 0, hy);
    __syncwarp();
    uint32_t s = 0;
    for (int b = lane; b < bins; b += 32) s += min(hx[b], hy[b]);
    s = warp_sum(s);
    if (lane == 0) {
      const bool ok = (int64_t)s >= (int64_t)A.need;
      A.shared[r] = s;
      A.pass[r] = ok ? 1 : 0;
      if (ok) atomicAdd(A.npass, 1ull);
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace sedef

using namespace sedef;

extern "C" int sedef_qgram(sedef_ctx* ctx, const uint32_t* d_packed, const uint32_t* d_nbits,
                           int64_t nbases, const sedef_run_t* d_runs, int64_t nruns,
                           const sedef_params* p, int32_t q, double p_gap, uint32_t* d_shared,
                           uint8_t* d_pass, int64_t* h_npass) {
  if (!ctx || !p || !h_npass) return fail(SEDEF_ERR_INVALID, "sedef_qgram: bad arguments");
  *h_npass = 0;
  Derived D;
  SEDEF_TRY(derive(p, &D));
  if (q < 1 || q > kMaxQ) return fail(SEDEF_ERR_INVALID, "sedef_qgram: q must be in [1, 5]");
  if (!(p_gap >= 0.0)) return fail(SEDEF_ERR_INVALID, "sedef_qgram: p_gap must be >= 0");
  if (nruns < 0 || nbases < 0) return fail(SEDEF_ERR_INVALID, "sedef_qgram: negative size");
  if (nruns == 0) return SEDEF_OK;
  if (!d_packed || !d_nbits || !d_runs || !d_shared || !d_pass)
    return fail(SEDEF_ERR_INVALID, "sedef_qgram: NULL buffer");
  SEDEF_CUDA(cudaSetDevice(ctx_device(ctx)));
  StageScope stage(ctx, "qgram");
  cudaStream_t st = ctx_stream(ctx);
  // least integer >= B - 1e-9 (Section 3.2 bound), in double
  const double B = (double)D.n * (1.0 - p->delta_g - (double)q * p->delta_m) -
                   ((double)D.n * p_gap + 1.0) * (double)(q - 1);
  double need = std::ceil(B - 1e-9);
  if (need - 1.0 >= B - 1e-9) need -= 1.0;
  if (need < 0.0) need = 0.0;
  QgArgs A;
  A.packed = d_packed;
  A.nbits = d_nbits;
  A.runs = d_runs;
  A.nruns = nruns;
  A.n = D.n;
  A.q = q;
  A.need = (int)need;
  A.shared = d_shared;
  A.pass = d_pass;
  unsigned long long* cnt = (unsigned long long*)ctx_alloc(ctx, 8);
  if (!cnt) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemsetAsync(cnt, 0, 8, st));
  A.npass = cnt;
  const size_t smem = (size_t)kQgWarps * 2 * (size_t(1) << (2 * q)) * 4;
  SEDEF_TRY(ensure_smem_attr((const void*)k_qgram, (size_t)kQgWarps * 2 * kMaxBins * 4));
  int64_t grid = (nruns + kQgWarps - 1) / kQgWarps;
  if (grid > (int64_t)ctx_sm_count(ctx) * 8) grid = (int64_t)ctx_sm_count(ctx) * 8;
  SEDEF_KERNEL(ctx, "k_qgram", k_qgram<<<(int)grid, 32 * kQgWarps, smem, st>>>(A));
  unsigned long long* h = (unsigned long long*)ctx_host(ctx, 8);
  if (!h) return SEDEF_ERR_OOM;
  SEDEF_CUDA(cudaMemcpyAsync(h, cnt, 8, cudaMemcpyDeviceToHost, st));
  SEDEF_CUDA(cudaStreamSynchronize(st));
  *h_npass = (int64_t)*h;
  return SEDEF_OK;
}
