// Hyper-edge spaces other than set betweenness (Sec. 2): kappa-path and
// triangle centralities.  CentRA is oblivious to sampleHEs (Sec. 4.2), so only
// the sampler changes; greedyCover, AMCERA and the bounds run as they are.
//
// kappa-path: s uniform (purpose 0), a length l uniform in 1..kappa (purpose
// 1), then a random simple walk of up to l steps: step i moves to the r-th
// (ascending id) out-neighbour of the current node that is not yet on the
// walk, r uniform below their number (purpose 2 + i); the walk stops early
// when there is none.  The hyper-edge is the nodes after s in walk order.
//
// Triangle: on an undirected graph, triangles {u < v < w} are ranked in
// (u, v, w) order: tri_off[e] (an exclusive prefix over arcs e = (u, v) in CSR
// order of the number of common neighbours w > v of u and v, counted only when
// v > u) ranks the first triangle on arc e, and within the arc the common
// neighbours ascend.  A rank r uniform below the total (purpose 0) is unranked
// and the three nodes, ascending, are the hyper-edge.
#include "job.cuh"

namespace cen {

namespace {

constexpr int kWalkWarps = 8;      // warps (samples) per block of the walk kernel
constexpr int kMaxKappa = 1024;

// Warp per sample.  The walk (at most kappa nodes after s) sits in shared
// memory; each step counts the current node's out-neighbours that are not on
// it, 32 arcs at a time, and takes the r-th of them.
__global__ void __launch_bounds__(32 * kWalkWarps) k_kpath(uint64_t j0, uint64_t count, int32_t n, int kappa,
                                                           const int64_t *__restrict__ off,
                                                           const int32_t *__restrict__ col, SampleKey key,
                                                           int32_t *ps, int32_t *pt, int32_t *pd, int32_t *out,
                                                           const int64_t *__restrict__ hoff, int *bmax,
                                                           unsigned long long *units) {
  extern __shared__ int32_t walk_sh[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t *walk = walk_sh + (size_t)wib * kappa;
  const uint64_t nw = (uint64_t)gridDim.x * kWalkWarps;
  unsigned long long arcs = 0;
  int mymax = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kWalkWarps + wib; i < count; i += nw) {
    const uint64_t j = j0 + i;
    const int32_t s = (int32_t)uniform_below64(key.seed, key.id(j), kPurposeS, (uint64_t)n);
    const int32_t l = 1 + (int32_t)uniform_below64(key.seed, key.id(j), kPurposeT, (uint64_t)kappa);
    int32_t cur = s, len = 0;
    for (int32_t step = 0; step < l; ++step) {
      const int64_t e0 = off[cur], e1 = off[cur + 1];
      // free out-neighbours: not s and not on the walk
      unsigned long long nfree = 0;
      for (int64_t b = e0; b < e1; b += 32) {
        const int64_t e = b + lane;
        bool fr = false;
        if (e < e1) {
          const int32_t w = col[e];
          fr = w != s;
          for (int q = 0; q < len && fr; ++q) fr = walk[q] != w;
        }
        nfree += __popc(__ballot_sync(0xffffffffu, fr));
      }
      arcs += (unsigned long long)(e1 - e0);
      if (nfree == 0) break;
      unsigned long long r = uniform_below64(key.seed, key.id(j), kPurposeWalk0 + (uint32_t)step, nfree);
      int32_t next = -1;
      for (int64_t b = e0; b < e1 && next < 0; b += 32) {
        const int64_t e = b + lane;
        bool fr = false;
        int32_t w = -1;
        if (e < e1) {
          w = col[e];
          fr = w != s;
          for (int q = 0; q < len && fr; ++q) fr = walk[q] != w;
        }
        const unsigned m = __ballot_sync(0xffffffffu, fr);
        const unsigned c = (unsigned)__popc(m);
        if (r < c) {  // the r-th free arc of this chunk
          unsigned mm = m;
          for (unsigned q = 0; q < (unsigned)r; ++q) mm &= mm - 1;
          next = __shfl_sync(0xffffffffu, w, __ffs(mm) - 1);
        } else {
          r -= c;
        }
      }
      __syncwarp();
      if (lane == 0) walk[len] = next;
      __syncwarp();
      ++len;
      cur = next;
    }
    if (out) {  // members at stride kappa, or at their place in the store when hoff is given
      int32_t *dst = hoff ? out + hoff[j] : out + (size_t)i * kappa;
      for (int q = lane; q < len; q += 32) dst[q] = walk[q];
    }
    if (lane == 0) {
      ps[j] = s;
      pt[j] = l;
      pd[j] = len;
    }
    mymax = max(mymax, len);
    __syncwarp();
  }
  if (lane == 0) {
    if (mymax) atomicMax(bmax, mymax);
    if (arcs) atomicAdd(units, arcs * 4ull);
  }
}

// Common neighbours w > v of u and v, ascending: the shorter row's entries
// above v are looked up in the longer row by binary search (both rows are
// sorted, so either order of the two rows gives the same ascending w).
// Returns how many there are; with want >= 0, stops at the one of that rank
// and returns it in *w_out.
__device__ int64_t common_above(const int64_t *__restrict__ off, const int32_t *__restrict__ col, int32_t u, int32_t v,
                                int64_t want, int32_t *w_out) {
  int64_t a0 = off[u], a1 = off[u + 1], b0 = off[v], b1 = off[v + 1];
  if (a1 - a0 > b1 - b0) {
    const int64_t t0 = a0, t1 = a1;
    a0 = b0;
    a1 = b1;
    b0 = t0;
    b1 = t1;
  }
  {  // first entry of the shorter row above v
    int64_t lo = a0, hi = a1;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (col[mid] <= v)
        lo = mid + 1;
      else
        hi = mid;
    }
    a0 = lo;
  }
  int64_t c = 0;
  for (int64_t a = a0; a < a1; ++a) {
    const int32_t w = col[a];
    int64_t lo = b0, hi = b1;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (col[mid] < w)
        lo = mid + 1;
      else
        hi = mid;
    }
    b0 = lo;  // w ascends, so the search range only shrinks
    if (lo < b1 && col[lo] == w) {
      if (c == want) {
        *w_out = w;
        return c;
      }
      ++c;
    }
  }
  return c;
}

// Thread per arc: its triangle count (0 unless col > row).
__global__ void k_tri_count(int32_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                            int64_t *cnt) {
  for (int32_t u = blockIdx.x * blockDim.y + threadIdx.y; u < n; u += gridDim.x * blockDim.y)
    for (int64_t e = off[u] + threadIdx.x; e < off[u + 1]; e += blockDim.x) {
      const int32_t v = col[e];
      cnt[e] = v > u ? common_above(off, col, u, v, -1, nullptr) : 0;
    }
}

// Thread per sample: rank r -> arc e (the last with tri_off[e] <= r) -> (u, v)
// -> the common neighbour of rank r - tri_off[e].
__global__ void k_tri_sample(uint64_t j0, uint64_t count, int32_t n, int64_t nnz, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ col, const int64_t *__restrict__ tri_off, SampleKey key,
                             int32_t *ps, int32_t *pt, int32_t *pd, const int64_t *__restrict__ hoff, int32_t *hmem) {
  const uint64_t T = (uint64_t)tri_off[nnz];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = j0 + i;
    const int64_t r = (int64_t)uniform_below64(key.seed, key.id(j), kPurposeS, T);
    int64_t lo = 0, hi = nnz + 1;  // upper bound of r in tri_off[0 .. nnz], minus one
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (tri_off[mid] <= r)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t e = lo - 1;
    int32_t a = 0, b = n;  // the row holding arc e
    while (b - a > 1) {
      const int32_t mid = a + ((b - a) >> 1);
      if (off[mid] <= e)
        a = mid;
      else
        b = mid;
    }
    const int32_t u = a, v = col[e];
    int32_t w = -1;
    common_above(off, col, u, v, r - tri_off[e], &w);
    ps[j] = u;
    pt[j] = v;
    pd[j] = w;
    const int64_t h = hoff[j];
    hmem[h] = u;
    hmem[h + 1] = v;
    hmem[h + 2] = w;
  }
}

}  // namespace

// Writes ps/pt/pd of the new samples and their members: to `out` at stride
// kappa, or, with hoff, into the store at hoff[j]; none when out is null.
void kpath_sample(cen_job *job, uint64_t j0, uint64_t count, int32_t *out, const int64_t *hoff) {
  const cen_graph *g = job->g;
  cudaStream_t st = job->st;
  const size_t smem = sizeof(int32_t) * (size_t)job->kappa * kWalkWarps;
  launch(&job->stats, K_SPACE, st, [&] {
    k_kpath<<<grid_for(count, kWalkWarps, sm_count() * 16), 32 * kWalkWarps, smem, st>>>(
        j0, count, g->n, job->kappa, g->off.as<int64_t>(), g->col.as<int32_t>(), job->key(), job->ps.as<int32_t>(),
        job->pt.as<int32_t>(), job->pd.as<int32_t>(), out, hoff, job->bmax.as<int>(),
        (unsigned long long *)(job->stats.d_units + K_SPACE));
  });
}

// Triangle ranks of the graph (kept on the graph), and their total.
int64_t triangle_index(cen_job *job) {
  cen_graph *g = const_cast<cen_graph *>(job->g);
  std::lock_guard<std::mutex> lk(g->tri_mu);
  if (g->tri_total < 0) {
    cudaStream_t st = job->st;
    DevBuf cnt;
    cnt.ensure(8 * (size_t)(g->nnz + 1), st);
    g->tri_off.ensure(8 * (size_t)(g->nnz + 1), st);
    launch(&job->stats, K_SPACE, st, [&] {
      k_tri_count<<<grid_for((size_t)g->n, 8, sm_count() * 64), dim3(32, 8), 0, st>>>(g->n, g->off.as<int64_t>(),
                                                                              g->col.as<int32_t>(), cnt.as<int64_t>());
    });
    exclusive_scan_i64(cnt.as<int64_t>(), g->tri_off.as<int64_t>(), (size_t)g->nnz, g->tri_off.as<int64_t>() + g->nnz,
                       job->scan_tmp, st, &job->stats);
    int64_t *h = (int64_t *)host_staging(job, 8);
    CEN_CK(cudaMemcpyAsync(h, g->tri_off.as<int64_t>() + g->nnz, 8, cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    cnt.release();
    CEN_CK(cudaStreamSynchronize(st));
    g->tri_total = *h;
  }
  return g->tri_total;
}

// Members of samples j0 .. j0+count-1 straight into the store (3 each; hoff set).
void triangle_sample(cen_job *job, uint64_t j0, uint64_t count) {
  const cen_graph *g = job->g;
  cudaStream_t st = job->st;
  launch(&job->stats, K_SPACE, st, [&] {
    k_tri_sample<<<grid_for(count, 256), 256, 0, st>>>(j0, count, g->n, g->nnz, g->off.as<int64_t>(),
                                                         g->col.as<int32_t>(), g->tri_off.as<int64_t>(), job->key(),
                                                         job->ps.as<int32_t>(), job->pt.as<int32_t>(),
                                                         job->pd.as<int32_t>(), job->hoff.as<int64_t>(),
                                                         job->hmem.as<int32_t>());
  });
}

int max_kappa() { return kMaxKappa; }

}  // namespace cen
