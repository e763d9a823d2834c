// Node -> sample incidence and greedyCover(k, H) (Sec. 3.1; Alg. 1 line "greedyCover").
#include <cooperative_groups.h>

#include <cstdlib>
#include <mutex>

#include "job.cuh"

namespace cg = cooperative_groups;

namespace cen {

// ------------------------------------------------------- incidence
__global__ void k_count_members(const int32_t *__restrict__ hmem, int64_t total, int32_t *c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&c[hmem[i]], 1);
}

// Thread per sample: each member u gets j appended to row u (order within a
// row follows atomic arrival; every consumer of the rows is order-free).
__global__ void k_scatter_members(const int64_t *__restrict__ hoff, const int32_t *__restrict__ hmem, uint64_t m,
                                  const int64_t *__restrict__ noff, int32_t *cursor, int32_t *nsamp) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
    for (int64_t e = hoff[j]; e < hoff[j + 1]; ++e) {
      const int32_t u = hmem[e];
      const int32_t pos = atomicAdd(&cursor[u], 1);
      nsamp[noff[u] + pos] = (int32_t)j;
    }
  }
}

void build_incidence(cen_job *job) {
  if (job->inc_m == job->m) return;
  cudaStream_t st = job->st;
  Stats *S = &job->stats;
  const int32_t n = job->g->n;
  job->c.ensure(4 * (size_t)n, st);
  job->cursor.ensure(4 * (size_t)n, st);
  job->noff.ensure(8 * ((size_t)n + 1), st);
  job->nsamp.ensure(4 * (size_t)(job->members + 1), st);
  CEN_CK(cudaMemsetAsync(job->c.p, 0, 4 * (size_t)n, st));
  CEN_CK(cudaMemsetAsync(job->cursor.p, 0, 4 * (size_t)n, st));
  if (job->members)
    launch(S, K_TRANSPOSE, st, [&] {
      k_count_members<<<grid_for((size_t)job->members, 256), 256, 0, st>>>(job->hmem.as<int32_t>(), job->members,
                                                                         job->c.as<int32_t>());
    });
  counts_to_offsets(job->c.as<int32_t>(), job->noff.as<int64_t>(), (size_t)n, job->scan_tmp, st, S);
  if (job->m)
    launch(S, K_TRANSPOSE, st, [&] {
      k_scatter_members<<<grid_for(job->m, 256), 256, 0, st>>>(job->hoff.as<int64_t>(), job->hmem.as<int32_t>(),
                                                               job->m, job->noff.as<int64_t>(),
                                                               job->cursor.as<int32_t>(), job->nsamp.as<int32_t>());
    });
  job->inc_m = job->m;
}

// ---------------------------------------------------------------- greedy
// Control words: key[2] (ping-pong argmax keys), covered count, picks, done.
struct GreedyCtl {
  unsigned long long key[2];
  unsigned long long covered;
  int size;
  int done;
  int S[1];  // k entries follow
};

__global__ void k_gain_init(const int32_t *__restrict__ c, int32_t *gain, int32_t n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) gain[i] = c[i];
}

// argmax over nodes of key = gain << 32 | (2^32 - 1 - u): the max key has the
// largest gain and, among equal gains, the lowest id.
__global__ void __launch_bounds__(256) k_greedy_argmax(const int32_t *__restrict__ gain, int32_t n, GreedyCtl *ctl,
                                                       int slot) {
  if (ctl->done) return;
  unsigned long long best = 0;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const unsigned long long k = ((unsigned long long)(uint32_t)gain[u] << 32) | (0xFFFFFFFFu - (uint32_t)u);
    best = k > best ? k : best;
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
    best = y > best ? y : best;
  }
  __shared__ unsigned long long wb[8];
  if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wb[w] > best ? wb[w] : best;
    if (best) atomicMax(&ctl->key[slot], best);
  }
}

// Warp per incident sample of the pick u*: a still-uncovered sample becomes
// covered and every member's gain drops by one.
__global__ void __launch_bounds__(256) k_greedy_update(const int64_t *__restrict__ noff,
                                                       const int32_t *__restrict__ nsamp,
                                                       const int64_t *__restrict__ hoff,
                                                       const int32_t *__restrict__ hmem, int32_t *gain,
                                                       uint32_t *covered, GreedyCtl *ctl, int slot, int it) {
  if (ctl->done) return;
  const unsigned long long key = ctl->key[slot];
  const uint32_t g = (uint32_t)(key >> 32);
  if (g == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->done = 1;
    return;
  }
  const int32_t u = (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->S[it] = u;
    ctl->size = it + 1;
    ctl->covered += g;
    ctl->key[slot ^ 1] = 0;  // reset the other slot for the next argmax
  }
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t r0 = noff[u], r1 = noff[u + 1];
  for (int64_t q = r0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < r1; q += nwarps) {
    const int32_t j = nsamp[q];
    const uint32_t mask = 1u << (j & 31);
    if (covered[j >> 5] & mask) continue;  // j occurs once in row u: only this warp can set its bit now
    if (lane == 0) atomicOr(&covered[j >> 5], mask);
    for (int64_t e = hoff[j] + lane; e < hoff[j + 1]; e += 32) atomicSub(&gain[hmem[e]], 1);
  }
}

// All k iterations in one cooperative launch: each iteration is the argmax
// (block maxima, one atomicMax per block), a grid barrier, the update of the
// picked node's samples, and another barrier.  The picks, ties and counts
// are those of k_greedy_argmax / k_greedy_update.  A cooperative launch runs
// only when every block is resident at once, so the barriers always complete.
__global__ void __launch_bounds__(256) k_greedy_all(const int64_t *__restrict__ noff, const int32_t *__restrict__ nsamp,
                                                    const int64_t *__restrict__ hoff, const int32_t *__restrict__ hmem,
                                                    int32_t *gain, int32_t n, uint32_t *covered, GreedyCtl *ctl,
                                                    int k) {
  cg::grid_group grid = cg::this_grid();
  __shared__ unsigned long long wb[8];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int it = 0; it < k; ++it) {
    const int slot = it & 1;
    unsigned long long best = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
      const unsigned long long key = ((unsigned long long)(uint32_t)gain[u] << 32) | (0xFFFFFFFFu - (uint32_t)u);
      best = key > best ? key : best;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
      best = y > best ? y : best;
    }
    if (lane == 0) wb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = wb[w] > best ? wb[w] : best;
      if (best) atomicMax(&ctl->key[slot], best);
    }
    grid.sync();
    const unsigned long long key = ((volatile unsigned long long *)ctl->key)[slot];
    const uint32_t g = (uint32_t)(key >> 32);
    if (g == 0) break;  // every block sees the same key: all leave together
    const int32_t u = (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->S[it] = u;
      ctl->size = it + 1;
      ctl->covered += g;
      ctl->key[slot ^ 1] = 0;
    }
    const int64_t r0 = noff[u], r1 = noff[u + 1];
    for (int64_t q = r0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < r1; q += nwarps) {
      const int32_t j = nsamp[q];
      const uint32_t mask = 1u << (j & 31);
      if (covered[j >> 5] & mask) continue;
      if (lane == 0) atomicOr(&covered[j >> 5], mask);
      for (int64_t e = hoff[j] + lane; e < hoff[j + 1]; e += 32) atomicSub(&gain[hmem[e]], 1);
    }
    grid.sync();
  }
}

// All k iterations in one thread-block cluster of C CTAs (16 where the device
// allows clusters that large, else 8), the gains held in the CTAs' shared
// memory (CTA r owns nodes [r per, (r+1) per)).
// Per iteration: each CTA takes the largest key of its nodes (the same key as
// k_greedy_all: largest gain, lowest id), a cluster barrier, every CTA reads
// the others' keys through distributed shared memory and so picks the same
// u*; then a thread per incident sample of u* sets the sample's covered bit
// and, if it was not set, decrements the gains of the sample's members in
// their owners' shared memory; another cluster barrier.  The picks and counts
// are those of k_greedy_all.  A cluster is launched only when all of its CTAs
// are resident at once, so the barriers always complete.
constexpr int kGreedyClusterMax = 16;  // non-portable; 8 is the portable size
// 512 threads: cheaper barriers per pick than 1,024 (measured 0.215 vs 0.23 ms per R-MAT 18
// round with 16 CTAs; 0.24 vs 0.25 ms with 8)
constexpr int kGreedyThreads = 512;

__global__ void __launch_bounds__(kGreedyThreads, 1)
    k_greedy_cluster(const int32_t *__restrict__ c, const int64_t *__restrict__ noff,
                     const int32_t *__restrict__ nsamp, const int64_t *__restrict__ hoff,
                     const int32_t *__restrict__ hmem, int32_t n, int32_t per, uint32_t *covered, GreedyCtl *ctl,
                     int k) {
  extern __shared__ int32_t s_gain[];
  __shared__ unsigned long long s_wbest[kGreedyThreads / 32];
  __shared__ unsigned long long s_best, s_key;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int32_t u0 = rank * per, u1 = min(n, u0 + per);
  for (int32_t u = u0 + tid; u < u1; u += kGreedyThreads) s_gain[u - u0] = c[u];
  cl.sync();
  const int64_t gt = (int64_t)rank * kGreedyThreads + tid;
  const int C = (int)cl.num_blocks();
  const int64_t nthreads = (int64_t)C * kGreedyThreads;
  for (int it = 0; it < k; ++it) {
    unsigned long long best = 0;
    for (int32_t u = u0 + tid; u < u1; u += kGreedyThreads) {
      const unsigned long long key = ((unsigned long long)(uint32_t)s_gain[u - u0] << 32) | (0xFFFFFFFFu - (uint32_t)u);
      best = key > best ? key : best;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
      best = y > best ? y : best;
    }
    if (lane == 0) s_wbest[wid] = best;
    __syncthreads();
    if (wid == 0) {
      best = lane < kGreedyThreads / 32 ? s_wbest[lane] : 0ull;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
      }
      if (lane == 0) s_best = best;
    }
    cl.sync();  // every CTA's key is in place
    if (wid == 0) {
      unsigned long long key = lane < C ? *cl.map_shared_rank(&s_best, lane) : 0ull;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
        key = y > key ? y : key;
      }
      if (lane == 0) s_key = key;
    }
    __syncthreads();
    const unsigned long long key = s_key;
    const uint32_t g = (uint32_t)(key >> 32);
    if (g == 0) break;  // every CTA holds the same key: all leave together
    const int32_t u = (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
    if (rank == 0 && tid == 0) {
      ctl->S[it] = u;
      ctl->size = it + 1;
      ctl->covered += g;
    }
    const int64_t r0 = noff[u], r1 = noff[u + 1];
    for (int64_t q = r0 + gt; q < r1; q += nthreads) {
      const int32_t j = nsamp[q];
      const uint32_t mask = 1u << (j & 31);
      const int64_t e0 = hoff[j], e1 = hoff[j + 1];  // loaded alongside the covered bit
      if (atomicOr(&covered[j >> 5], mask) & mask) continue;  // covered by an earlier pick
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t w = hmem[e];
        const int owner = w / per;
        atomicSub(cl.map_shared_rank(s_gain + (w - owner * per), owner), 1);
      }
    }
    cl.sync();  // every gain update has landed before the next argmax
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Nodes per CTA the cluster form can hold (the rest of the shared memory is
// the kernel's own).
constexpr int64_t kGreedyClusterMaxPer = (227 * 1024 - 2048) / 4;

size_t greedy_result_bytes(int32_t k) { return sizeof(GreedyCtl) + 4 * (size_t)k; }

// Whether a cluster of C CTAs of k_greedy_cluster with `smem` bytes of gains
// can be resident on this device (the kernel's shared-memory limit is raised,
// and clusters over 8 allowed, once per process).
static bool greedy_cluster_ready(int C, size_t smem) {
  static std::mutex mu;
  static int attr_ok = -1, big_ok = -1;
  std::lock_guard<std::mutex> lk(mu);
  if (attr_ok < 0) {
    attr_ok = cudaFuncSetAttribute(k_greedy_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kGreedyClusterMaxPer * 4)) == cudaSuccess;
    cudaGetLastError();
    big_ok = cudaFuncSetAttribute(k_greedy_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    cudaGetLastError();
  }
  if (!attr_ok || (C > 8 && !big_ok)) return false;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kGreedyThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&clusters, k_greedy_cluster, &cfg) == cudaSuccess && clusters >= 1;
  cudaGetLastError();
  return ok;
}

// Sizes the greedy workspace for k picks (allocations ordered on the job's
// stream).  The incidence must be current.
void greedy_prepare(cen_job *job, int32_t k) {
  CEN_REQUIRE(k >= 1, CEN_EINVAL, "cen_greedy_cover: k must be >= 1");
  cudaStream_t st = job->st;
  job->gain.ensure(4 * (size_t)job->g->n, st);
  job->covered.ensure(4 * ((job->m + 31) / 32 + 1), st);
  job->gctl.ensure(greedy_result_bytes(k), st);
}

// Enqueues greedyCover(k) on stream `run` (after greedy_prepare); the result
// reaches hdst (pinned, greedy_result_bytes(k)) once `run` has drained.
void greedy_enqueue(cen_job *job, int32_t k, cudaStream_t run, void *hdst) {
  Stats *St = &job->stats;
  const int32_t n = job->g->n;
  const size_t cbytes = greedy_result_bytes(k);
  CEN_CK(cudaMemsetAsync(job->covered.p, 0, 4 * ((job->m + 31) / 32 + 1), run));
  CEN_CK(cudaMemsetAsync(job->gctl.p, 0, cbytes, run));
  GreedyCtl *ctl = job->gctl.as<GreedyCtl>();
  // diagnostics: CEN_GREEDY_GRID=1 keeps the cooperative grid form, CEN_GREEDY_CLUSTER=8 the
  // portable cluster size
  const char *grid_env = getenv("CEN_GREEDY_GRID");
  const char *size_env = getenv("CEN_GREEDY_CLUSTER");
  const bool grid_form = grid_env && grid_env[0] == '1';
  int C = 0;
  for (int c : {kGreedyClusterMax, 8}) {
    if (grid_form || C || (c > 8 && size_env && atoi(size_env) == 8)) continue;
    const int64_t per_c = ((int64_t)n + c - 1) / c;
    if (per_c <= kGreedyClusterMaxPer && greedy_cluster_ready(c, (size_t)per_c * 4)) C = c;
  }
  if (C) {
    const int64_t per = ((int64_t)n + C - 1) / C;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kGreedyThreads);
    cfg.dynamicSmemBytes = (size_t)per * 4;
    cfg.stream = run;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    launch(St, K_GREEDY, run, [&] {
      CEN_CK(cudaLaunchKernelEx(&cfg, k_greedy_cluster, (const int32_t *)job->c.as<int32_t>(),
                                (const int64_t *)job->noff.as<int64_t>(), (const int32_t *)job->nsamp.as<int32_t>(),
                                (const int64_t *)job->hoff.as<int64_t>(), (const int32_t *)job->hmem.as<int32_t>(), n,
                                (int32_t)per, job->covered.as<uint32_t>(), ctl, (int)k));
    });
    CEN_CK(cudaMemcpyAsync(hdst, ctl, cbytes, cudaMemcpyDeviceToHost, run));
    return;
  }
  launch(St, K_GREEDY, run,
         [&] { k_gain_init<<<grid_for(n, 256), 256, 0, run>>>(job->c.as<int32_t>(), job->gain.as<int32_t>(), n); });
  const int coop = cooperative_grid((const void *)k_greedy_all, 256);
  if (coop > 0) {
    const int64_t *a_noff = job->noff.as<int64_t>();
    const int32_t *a_nsamp = job->nsamp.as<int32_t>();
    const int64_t *a_hoff = job->hoff.as<int64_t>();
    const int32_t *a_hmem = job->hmem.as<int32_t>();
    int32_t *a_gain = job->gain.as<int32_t>();
    int32_t a_n = n;
    uint32_t *a_cov = job->covered.as<uint32_t>();
    int a_k = k;
    void *args[] = {&a_noff, &a_nsamp, &a_hoff, &a_hmem, &a_gain, &a_n, &a_cov, &ctl, &a_k};
    launch(St, K_GREEDY, run, [&] {
      CEN_CK(cudaLaunchCooperativeKernel((const void *)k_greedy_all, dim3(coop), dim3(256), args, 0, run));
    });
  } else {
    const int gblocks = grid_for((size_t)n, 256, sm_count() * 4);
    for (int it = 0; it < k; ++it) {
      const int slot = it & 1;
      launch(St, K_GREEDY, run,
             [&] { k_greedy_argmax<<<gblocks, 256, 0, run>>>(job->gain.as<int32_t>(), n, ctl, slot); });
      launch(St, K_GREEDY, run, [&] {
        k_greedy_update<<<sm_count() * 4, 256, 0, run>>>(job->noff.as<int64_t>(), job->nsamp.as<int32_t>(),
                                                   job->hoff.as<int64_t>(), job->hmem.as<int32_t>(),
                                                   job->gain.as<int32_t>(), job->covered.as<uint32_t>(), ctl, slot,
                                                   it);
      });
    }
  }
  CEN_CK(cudaMemcpyAsync(hdst, ctl, cbytes, cudaMemcpyDeviceToHost, run));
}

// S, |S| and the covered count from the copied result.
void greedy_result(const void *h, int32_t *S, int32_t *S_size, uint64_t *covered) {
  const GreedyCtl *hc = (const GreedyCtl *)h;
  *S_size = hc->size;
  *covered = hc->covered;
  for (int i = 0; i < hc->size; ++i) S[i] = hc->S[i];
}

// ------------------------------------------- greedyCover one pick at a time
// For a sample split over several GPUs (shards): every shard keeps its own
// gains and covered bits; the caller sums the shards' gains, takes the pick
// (shard_pick, the same key as k_greedy_all: largest gain, lowest id) and
// applies it to every shard.  A shard's newly covered samples are exactly its
// part of the pick's summed gain.

// Warp per incident sample of u, as k_greedy_update; counts the samples it
// newly covers.
__global__ void __launch_bounds__(256) k_shard_apply(const int64_t *__restrict__ noff,
                                                     const int32_t *__restrict__ nsamp,
                                                     const int64_t *__restrict__ hoff,
                                                     const int32_t *__restrict__ hmem, int32_t *gain,
                                                     uint32_t *covered, int32_t u, unsigned long long *newly) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t r0 = noff[u], r1 = noff[u + 1];
  unsigned long long mine = 0;
  for (int64_t q = r0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < r1; q += nwarps) {
    const int32_t j = nsamp[q];
    const uint32_t mask = 1u << (j & 31);
    if (covered[j >> 5] & mask) continue;  // j occurs once in row u: only this warp can set its bit now
    if (lane == 0) {
      atomicOr(&covered[j >> 5], mask);
      ++mine;
    }
    for (int64_t e = hoff[j] + lane; e < hoff[j + 1]; e += 32) atomicSub(&gain[hmem[e]], 1);
  }
  if (lane == 0 && mine) atomicAdd(newly, mine);
}

void shard_greedy_begin(cen_job *job) {
  build_incidence(job);
  greedy_prepare(job, 1);
  cudaStream_t st = job->st;
  const int32_t n = job->g->n;
  CEN_CK(cudaMemsetAsync(job->covered.p, 0, 4 * ((job->m + 31) / 32 + 1), st));
  launch(&job->stats, K_GREEDY, st,
         [&] { k_gain_init<<<grid_for(n, 256), 256, 0, st>>>(job->c.as<int32_t>(), job->gain.as<int32_t>(), n); });
  CEN_CK(cudaStreamSynchronize(st));
  job->shard_greedy_m = (int64_t)job->m;
}

static void require_shard_greedy(const cen_job *job, const char *what) {
  CEN_REQUIRE(job->shard_greedy_m == (int64_t)job->m, CEN_EINVAL,
              std::string(what) + ": call cen_shard_greedy_begin after the last cen_sample");
}

void shard_gains(const cen_job *job, int32_t *dst) {
  require_shard_greedy(job, "cen_shard_gains");
  CEN_CK(cudaMemcpyAsync(dst, job->gain.p, 4 * (size_t)job->g->n, cudaMemcpyDeviceToDevice, job->st));
  CEN_CK(cudaStreamSynchronize(job->st));
}

void shard_pick(cen_job *job, const int32_t *gains, int32_t *u, int32_t *gain) {
  cudaStream_t st = job->st;
  const int32_t n = job->g->n;
  job->gctl.ensure(greedy_result_bytes(1), st);
  GreedyCtl *ctl = job->gctl.as<GreedyCtl>();
  CEN_CK(cudaMemsetAsync(ctl, 0, sizeof(GreedyCtl), st));
  launch(&job->stats, K_GREEDY, st, [&] {
    k_greedy_argmax<<<grid_for((size_t)n, 256, sm_count() * 4), 256, 0, st>>>(gains, n, ctl, 0);
  });
  unsigned long long *h = (unsigned long long *)host_staging(job, 8);
  CEN_CK(cudaMemcpyAsync(h, &ctl->key[0], 8, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  const unsigned long long key = *h;
  *gain = (int32_t)(uint32_t)(key >> 32);
  *u = key ? (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu)) : -1;
}

void shard_apply(cen_job *job, int32_t u, uint64_t *newly) {
  require_shard_greedy(job, "cen_shard_apply");
  CEN_REQUIRE(u >= 0 && u < job->g->n, CEN_EINVAL, "cen_shard_apply: node out of range");
  cudaStream_t st = job->st;
  GreedyCtl *ctl = job->gctl.as<GreedyCtl>();
  CEN_CK(cudaMemsetAsync(&ctl->covered, 0, 8, st));
  launch(&job->stats, K_GREEDY, st, [&] {
    k_shard_apply<<<sm_count() * 4, 256, 0, st>>>(job->noff.as<int64_t>(), job->nsamp.as<int32_t>(),
                                                  job->hoff.as<int64_t>(), job->hmem.as<int32_t>(),
                                                  job->gain.as<int32_t>(), job->covered.as<uint32_t>(), u,
                                                  &ctl->covered);
  });
  unsigned long long *h = (unsigned long long *)host_staging(job, 8);
  CEN_CK(cudaMemcpyAsync(h, &ctl->covered, 8, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  *newly = *h;
}

void greedy_cover(cen_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered) {
  CEN_REQUIRE(k >= 1, CEN_EINVAL, "cen_greedy_cover: k must be >= 1");
  Range range("cen_greedy_cover");
  build_incidence(job);
  greedy_prepare(job, k);
  void *h = host_staging(job, greedy_result_bytes(k));
  greedy_enqueue(job, k, job->st, h);
  CEN_CK(cudaStreamSynchronize(job->st));
  greedy_result(h, S, S_size, covered);
}

}  // namespace cen
