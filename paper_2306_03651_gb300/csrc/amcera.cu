// AMCERA numerators (Sec. 4.1; Alg. 1 lines computing r_j^u, r_j and the average).
//
// R_q^u = sum over samples j holding u of sigma_{q,j} = 2 P_q^u - c_u, where
// P_q^u counts u's samples whose sign bit q is set.  The sup over |S| <= k of
// sum_{u in S} R_q^u is the sum of the <= k largest positive R_q^u (the
// objective is additive in S), found per row by an exact MSB-first radix
// select; the same select over c_u gives the wimpy-variance numerator.
#include <mutex>

#include "job.cuh"

namespace cen {

// Warp per node u with c_u > 0: lanes take 32 incident samples at a time; for
// each sign word the warp ballots bit q across the 32 samples (the word's
// rows only) and lane q adds the popcount.  The block sums its scanned
// incidences before one atomic.
__global__ void __launch_bounds__(256) k_rade(int32_t n, int t, int nw, const int64_t *__restrict__ noff,
                                              const int32_t *__restrict__ nsamp, const uint32_t *__restrict__ sign,
                                              int32_t *R, unsigned long long *units) {
  __shared__ unsigned long long s_scanned;
  if (threadIdx.x == 0) s_scanned = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nwarps) {
    const int64_t r0 = noff[u], r1 = noff[u + 1];
    const int32_t cu = (int32_t)(r1 - r0);
    if (cu == 0) continue;  // R rows are zero-filled
    for (int w = 0; w < nw; ++w) {
      const int qn = min(32, t - 32 * w);  // rows of this word
      int32_t P = 0;
      for (int64_t base = r0; base < r1; base += 32) {
        const int64_t i = base + lane;
        const uint32_t x = i < r1 ? sign[(int64_t)nsamp[i] * nw + w] : 0u;
#pragma unroll 8
        for (int q = 0; q < qn; ++q) {
          const int c = __popc(__ballot_sync(0xffffffffu, (x >> q) & 1u));
          if (lane == q) P += c;
        }
      }
      const int q = 32 * w + lane;
      if (q < t) R[(int64_t)q * n + u] = 2 * P - cu;
    }
    scanned += (unsigned long long)cu;
  }
  if (lane == 0 && scanned) atomicAdd(&s_scanned, scanned);
  __syncthreads();
  if (threadIdx.x == 0 && s_scanned) atomicAdd(units, s_scanned);
}

// ------------------------------------------------------------ radix select
// Per row: prefix/mask of the k-th largest positive value found so far, the
// count still to take (krem) and the sum of values already known to be in.
struct SelRow {
  uint32_t prefix, mask;
  int32_t krem;
  int32_t done;
  long long sum;
};

__global__ void k_sel_init(SelRow *rows, int nrows, int32_t k) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x)
    rows[r] = SelRow{0u, 0u, k, 0, 0ll};
}

// Histogram of digit `shift` over positive values matching the row's prefix.
__global__ void __launch_bounds__(256) k_sel_hist(const int32_t *__restrict__ vals, int64_t n, int nrows, int shift,
                                                  const SelRow *__restrict__ rows, unsigned int *hcnt,
                                                  unsigned long long *hsum) {
  __shared__ unsigned int sc[256];
  __shared__ unsigned long long ss[256];
  const int r = blockIdx.y;
  const SelRow row = rows[r];
  if (row.done) return;
  sc[threadIdx.x] = 0;
  ss[threadIdx.x] = 0;
  __syncthreads();
  const int32_t *v = vals + (int64_t)r * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = v[i];
    if (x > 0 && ((uint32_t)x & row.mask) == row.prefix) {
      const uint32_t d = ((uint32_t)x >> shift) & 255u;
      atomicAdd(&sc[d], 1u);
      atomicAdd(&ss[d], (unsigned long long)x);
    }
  }
  __syncthreads();
  if (sc[threadIdx.x]) {
    atomicAdd(&hcnt[r * 256 + threadIdx.x], sc[threadIdx.x]);
    atomicAdd(&hsum[r * 256 + threadIdx.x], ss[threadIdx.x]);
  }
}

// One block of 256 threads per row, thread i on digit 255 - i: scans of the
// bucket counts and sums from the top digit down give, for each digit, what
// the buckets above it hold.  Whole buckets are taken while their running
// count stays below krem; the first bucket whose running count reaches krem
// is descended into (its digit joins the prefix).  If every matching value
// fits in krem, all are taken.  Clears the row's buckets for the next digit.
__global__ void __launch_bounds__(256) k_sel_step(int nrows, int shift, SelRow *rows, unsigned int *hcnt,
                                                  unsigned long long *hsum) {
  __shared__ long long wc[8], ws[8];
  const int r = blockIdx.x, i = threadIdx.x, lane = i & 31, w = i >> 5;
  if (r >= nrows) return;
  const SelRow row = rows[r];  // every thread reads it before thread 0 may rewrite it
  if (row.done) return;        // the histogram pass skipped the row: its buckets are zero
  const int d = 255 - i;
  const long long c = (long long)hcnt[r * 256 + d];
  const long long sv = (long long)hsum[r * 256 + d];
  long long ci = c, si = sv;  // inclusive scans over digits 255 .. d
  for (int o = 1; o < 32; o <<= 1) {
    const long long yc = __shfl_up_sync(0xffffffffu, ci, o), ys = __shfl_up_sync(0xffffffffu, si, o);
    if (lane >= o) {
      ci += yc;
      si += ys;
    }
  }
  if (lane == 31) {
    wc[w] = ci;
    ws[w] = si;
  }
  __syncthreads();
  long long total = 0, stotal = 0;
  for (int q = 0; q < 8; ++q) {
    if (q < w) {
      ci += wc[q];
      si += ws[q];
    }
    total += wc[q];
    stotal += ws[q];
  }
  hcnt[r * 256 + d] = 0;
  hsum[r * 256 + d] = 0;
  SelRow out = row;
  if (total <= row.krem) {  // every matching value is in
    if (i != 0) return;
    out.sum += stotal;
    out.krem = 0;
    out.done = 1;
  } else {
    const long long ce = ci - c, se = si - sv;  // the buckets above digit d
    if (!(ci >= row.krem && ce < row.krem)) return;  // not the bucket that reaches krem
    out.krem = row.krem - (int32_t)ce;
    out.sum += se;
    out.prefix |= (uint32_t)d << shift;
    out.mask |= 255u << shift;
    if (shift == 0) {  // prefix is now the exact k-th value; krem copies of it remain
      out.sum += (long long)out.krem * (long long)out.prefix;
      out.krem = 0;
      out.done = 1;
    }
  }
  rows[r] = out;
}

// Enqueues on `run` the sums of the <= k largest positive entries of each of
// `nrows` rows of length n (select state sized beforehand, see mcera_prepare);
// the per-row results reach hdst (pinned, nrows SelRow) once `run` drains.
static void topk_enqueue(cen_job *job, const int32_t *vals, int64_t n, int nrows, int32_t k, cudaStream_t run,
                         SelRow *hdst, int64_t vmax = INT32_MAX) {
  Stats *S = &job->stats;
  SelRow *rows = job->selst.as<SelRow>();
  unsigned int *hcnt = job->selh.as<unsigned int>();
  unsigned long long *hsum = (unsigned long long *)(hcnt + (size_t)nrows * 256);
  CEN_CK(cudaMemsetAsync(job->selh.p, 0, (size_t)nrows * 256 * 12, run));
  launch(S, K_SELECT, run, [&] { k_sel_init<<<grid_for(nrows, 128), 128, 0, run>>>(rows, nrows, k); });
  const int bx = grid_for((size_t)n, 256 * 8, 512);
  // digits above the highest one a value <= vmax can have are 0 for every
  // value, so their passes would only descend into digit 0
  int top = 24;
  while (top > 0 && (vmax >> top) == 0) top -= 8;
  for (int shift = top; shift >= 0; shift -= 8) {
    launch(S, K_SELECT, run, [&] {
      k_sel_hist<<<dim3(bx, nrows), 256, 0, run>>>(vals, n, nrows, shift, rows, hcnt, hsum);
    });
    launch(S, K_SELECT, run, [&] { k_sel_step<<<nrows, 256, 0, run>>>(nrows, shift, rows, hcnt, hsum); });
  }
  CEN_CK(cudaMemcpyAsync(hdst, rows, sizeof(SelRow) * (size_t)nrows, cudaMemcpyDeviceToHost, run));
}

// Host bytes mcera_enqueue copies into: t + 1 select rows, then b_H.
size_t mcera_result_bytes(const cen_job *job) { return sizeof(SelRow) * (size_t)(job->t + 1) + 8; }

// Sizes the AMCERA workspace (allocations ordered on the job's stream).  The
// incidence must be current.
void mcera_prepare(cen_job *job, int32_t k) {
  CEN_REQUIRE(k >= 1, CEN_EINVAL, "cen_mcera: k must be >= 1");
  cudaStream_t st = job->st;
  const int nrows = job->t + 1;
  job->R.ensure(4 * (size_t)job->g->n * nrows, st);
  job->selst.ensure(sizeof(SelRow) * (size_t)nrows, st);
  job->selh.ensure((size_t)nrows * 256 * (4 + 8), st);
}

// Enqueues the AMCERA of Alg. 1 on stream `run` (after mcera_prepare): rows
// 0 .. t-1 of R are R_q^u, row t is c_u, so one selection gives every Rnum and
// Wnum.  Results reach hdst (pinned, mcera_result_bytes) once `run` drains.
void mcera_enqueue(cen_job *job, int32_t k, cudaStream_t run, void *hdst) {
  Stats *S = &job->stats;
  const int32_t n = job->g->n;
  const int t = job->t;
  CEN_CK(cudaMemsetAsync(job->R.p, 0, 4 * (size_t)n * t, run));
  launch(S, K_RADE, run, [&] {
    k_rade<<<grid_for((size_t)n * 32, 256, sm_count() * 64), 256, 0, run>>>(n, t, job->nw, job->noff.as<int64_t>(),
                                                                       job->nsamp.as<int32_t>(),
                                                                       job->sign.as<uint32_t>(), job->R.as<int32_t>(),
                                                                       (unsigned long long *)(job->stats.d_units + K_RADE));
  });
  CEN_CK(cudaMemcpyAsync(job->R.as<int32_t>() + (size_t)n * t, job->c.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice,
                         run));
  SelRow *hrows = (SelRow *)hdst;
  // |R_q^u| <= c_u <= m: every value the select ranks is at most m
  topk_enqueue(job, job->R.as<int32_t>(), n, t + 1, k, run, hrows, (int64_t)job->m);
  if (job->m) CEN_CK(cudaMemcpyAsync(hrows + t + 1, job->bmax.p, 4, cudaMemcpyDeviceToHost, run));  // b_H = 0 if m = 0
}

// Rnum[t], Wnum and b_H from the copied result.
void mcera_result(cen_job *job, int32_t k, const void *h, int64_t *Rnum, int64_t *Wnum, int32_t *b) {
  const SelRow *hrows = (const SelRow *)h;
  const int t = job->t;
  for (int q = 0; q < t; ++q) Rnum[q] = hrows[q].sum;
  *Wnum = hrows[t].sum;  // the c_u are positive, so this is the sum of the k largest
  int hb = 0;
  memcpy(&hb, hrows + t + 1, 4);
  *b = job->m ? hb : 0;
  job->rade_valid_k = k;
}

// greedyCover on the job's stream and the AMCERA on its second stream at the
// same time: the two read the same incidence and write disjoint buffers, so
// the results are those of greedy_cover followed by mcera.
void cover_and_mcera(cen_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered, int64_t *Rnum,
                     int64_t *Wnum, int32_t *b) {
  CEN_REQUIRE(k >= 1, CEN_EINVAL, "cen_cover_and_mcera: k must be >= 1");
  Range range("cen_cover_and_mcera");
  build_incidence(job);
  greedy_prepare(job, k);
  mcera_prepare(job, k);
  const size_t gb = (greedy_result_bytes(k) + 15) & ~(size_t)15;
  char *h = (char *)host_staging(job, gb + mcera_result_bytes(job));
  job->aux.ensure();
  CEN_CK(cudaEventRecord(job->aux.fork, job->st));
  CEN_CK(cudaStreamWaitEvent(job->aux.st, job->aux.fork, 0));
  greedy_enqueue(job, k, job->st, h);
  try {
    mcera_enqueue(job, k, job->aux.st, h + gb);
  } catch (...) {  // still join, so that nothing on the job's stream outruns the second stream
    cudaEventRecord(job->aux.join, job->aux.st);
    cudaStreamWaitEvent(job->st, job->aux.join, 0);
    throw;
  }
  CEN_CK(cudaEventRecord(job->aux.join, job->aux.st));
  CEN_CK(cudaStreamWaitEvent(job->st, job->aux.join, 0));
  CEN_CK(cudaStreamSynchronize(job->st));
  greedy_result(h, S, S_size, covered);
  mcera_result(job, k, h + gb, Rnum, Wnum, b);
}

// ----------------------------------------------- AMCERA of a split sample
// A shard's R (rows 0 .. t-1) and c (row t) over its own samples, into a
// caller's device matrix, and its b_H; the caller sums the shards' matrices
// (R and c are sums over samples) and takes shard_topk of the sum.
void shard_rade(cen_job *job, int32_t *R_out, int32_t *b) {
  build_incidence(job);
  mcera_prepare(job, 1);
  cudaStream_t st = job->st;
  const int32_t n = job->g->n;
  const int t = job->t;
  CEN_CK(cudaMemsetAsync(job->R.p, 0, 4 * (size_t)n * t, st));
  launch(&job->stats, K_RADE, st, [&] {
    k_rade<<<grid_for((size_t)n * 32, 256, sm_count() * 64), 256, 0, st>>>(
        n, t, job->nw, job->noff.as<int64_t>(), job->nsamp.as<int32_t>(), job->sign.as<uint32_t>(),
        job->R.as<int32_t>(), (unsigned long long *)(job->stats.d_units + K_RADE));
  });
  CEN_CK(cudaMemcpyAsync(job->R.as<int32_t>() + (size_t)n * t, job->c.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
  CEN_CK(cudaMemcpyAsync(R_out, job->R.p, 4 * (size_t)n * (t + 1), cudaMemcpyDeviceToDevice, st));
  int32_t *h = (int32_t *)host_staging(job, 4);
  *h = 0;
  if (job->m) CEN_CK(cudaMemcpyAsync(h, job->bmax.p, 4, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  *b = job->m ? *h : 0;
}

// Sums of the <= k largest positive entries of each of nrows rows of length n
// (the job's graph's n) of a device matrix, with the job's select workspace.
void shard_topk(cen_job *job, const int32_t *vals, int32_t nrows, int32_t k, int64_t *out) {
  CEN_REQUIRE(nrows >= 1 && k >= 1, CEN_EINVAL, "cen_shard_topk: need nrows >= 1 and k >= 1");
  cudaStream_t st = job->st;
  job->selst.ensure(sizeof(SelRow) * (size_t)nrows, st);
  job->selh.ensure((size_t)nrows * 256 * (4 + 8), st);
  SelRow *h = (SelRow *)host_staging(job, sizeof(SelRow) * (size_t)nrows);
  topk_enqueue(job, vals, job->g->n, nrows, k, st, h);
  CEN_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < nrows; ++r) out[r] = h[r].sum;
}

void mcera(cen_job *job, int32_t k, int64_t *Rnum, int64_t *Wnum, int32_t *b) {
  CEN_REQUIRE(k >= 1, CEN_EINVAL, "cen_mcera: k must be >= 1");
  Range range("cen_mcera");
  build_incidence(job);
  mcera_prepare(job, k);
  void *h = host_staging(job, mcera_result_bytes(job));
  mcera_enqueue(job, k, job->st, h);
  CEN_CK(cudaStreamSynchronize(job->st));
  mcera_result(job, k, h, Rnum, Wnum, b);
}

}  // namespace cen

// ---------------------------------------------------------------------------
// Allocation-free top-k positive sums (no counterpart in the paper).
//
// Same kernels as the select inside cen_mcera, but the scratch (per-row
// select state and the 256-bucket count/sum histograms) lives in one
// file-scope __device__ array, so a call allocates no device memory.  Every
// call on a device shares that array; calls that overlap on the GPU race.
namespace cen {

constexpr int kNoAllocMaxRows = 128;
struct NoAllocScratch {
  SelRow rows[kNoAllocMaxRows];
  unsigned int hcnt[kNoAllocMaxRows * 256];
  unsigned long long hsum[kNoAllocMaxRows * 256];
};
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device.  The host-side name is only a stand-in for the symbol.
static NoAllocScratch *noalloc_scratch() {
  int dev = -1;
  CEN_CK(cudaGetDevice(&dev));
  CEN_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, CEN_EINVAL, "cen_topk_positive_sum_noalloc: device id too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      fail(CEN_ECUDA, std::string("cen_topk_positive_sum_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  return static_cast<NoAllocScratch *>(g_noalloc_addr[dev]);
}

}  // namespace cen

extern "C" int cen_topk_positive_sum_noalloc(const int32_t *vals, int64_t n, int32_t nrows, int32_t k, int64_t *out,
                                             void *stream) {
  using namespace cen;
  try {
    CEN_REQUIRE(vals && out, CEN_EINVAL, "cen_topk_positive_sum_noalloc: null argument");
    CEN_REQUIRE(nrows >= 1 && nrows <= kNoAllocMaxRows, CEN_EINVAL,
                "cen_topk_positive_sum_noalloc: nrows must be in [1, 128] (size of the static scratch)");
    CEN_REQUIRE(n >= 0 && k >= 1, CEN_EINVAL, "cen_topk_positive_sum_noalloc: need n >= 0 and k >= 1");
    // the select's bucket counts are 32-bit
    CEN_REQUIRE(n <= INT32_MAX, CEN_EINVAL, "cen_topk_positive_sum_noalloc: rows longer than 2^31 - 1 entries");
    cudaStream_t st = (cudaStream_t)stream;
    NoAllocScratch *sc = noalloc_scratch();
    // the histograms must start at zero; the row states are written by k_sel_init
    CEN_CK(cudaMemsetAsync(sc->hcnt, 0, sizeof(sc->hcnt) + sizeof(sc->hsum), st));
    launch(nullptr, K_SELECT, st, [&] { k_sel_init<<<grid_for(nrows, 128), 128, 0, st>>>(sc->rows, nrows, k); });
    const int bx = grid_for((size_t)(n > 0 ? n : 1), 256 * 8, 512);
    for (int shift = 24; shift >= 0; shift -= 8) {
      launch(nullptr, K_SELECT, st, [&] {
        k_sel_hist<<<dim3(bx, nrows), 256, 0, st>>>(vals, n, nrows, shift, sc->rows, sc->hcnt, sc->hsum);
      });
      launch(nullptr, K_SELECT, st,
             [&] { k_sel_step<<<nrows, 256, 0, st>>>(nrows, shift, sc->rows, sc->hcnt, sc->hsum); });
    }
    SelRow h[kNoAllocMaxRows];
    CEN_CK(cudaMemcpyAsync(h, sc->rows, sizeof(SelRow) * (size_t)nrows, cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    for (int r = 0; r < nrows; ++r) out[r] = h[r].sum;
    return CEN_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (...) {
    set_last_error("cen_topk_positive_sum_noalloc: unexpected internal error");
    return CEN_ECUDA;
  }
}
