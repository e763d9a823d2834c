// Graph upload: canonical-CSR validation on the GPU and, for directed graphs,
// the in-arc CSR (a stable sort of arcs by head keeps each row ascending).
#include <algorithm>

#include "job.cuh"

namespace cen {

// Canonical-CSR validation in three passes (each *bad |= 1 on a violation):
// offsets that rise from 0 to nnz, with the first arc of every non-empty row
// marked; every head in [0, n) and above the arc before it unless it starts
// its row (so rows are strictly ascending: no repeats); and no row that holds
// its own node (a binary search, exact once the rows are ascending).
__global__ void k_mark_starts(const int64_t *__restrict__ off, int32_t n, int64_t nnz, uint8_t *start, int *bad) {
  if (blockIdx.x == 0 && threadIdx.x == 0)
    if (off[0] != 0 || off[n] != nnz) atomicOr(bad, 1);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[v], e = off[v + 1];
    if (b > e || b < 0 || e > nnz)
      atomicOr(bad, 1);
    else if (b < e)
      start[b] = 1;
  }
}

__global__ void k_check_arcs(const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                             const uint8_t *__restrict__ start, int *bad) {
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = col[i];
    ok &= c >= 0 && c < n;
    if (i > 0 && !start[i]) ok &= col[i - 1] < c;
  }
  if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

__global__ void k_check_loops(const int64_t *__restrict__ off, const int32_t *__restrict__ col, int32_t n,
                              int64_t nnz, int *bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = off[v], hi = off[v + 1];
    if (lo < 0 || hi > nnz || lo >= hi) continue;  // bad offsets are flagged by k_mark_starts
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      const int32_t c = col[mid];
      if (c == (int32_t)v) {
        atomicOr(bad, 1);
        break;
      }
      if (c < (int32_t)v)
        lo = mid + 1;
      else
        hi = mid;
    }
  }
}

// Arc list in CSR order: key = head, value = tail.
__global__ void k_arcs_by_tail(const int64_t *off, const int32_t *col, int32_t n, uint32_t *key, uint32_t *val) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
    for (int64_t i = off[v] + lane; i < off[v + 1]; i += 32) {
      key[i] = (uint32_t)col[i];
      val[i] = (uint32_t)v;
    }
  }
}

// In-CSR offsets from the heads sorted ascending (nnz >= 1): roff[w] is the
// first position whose head is >= w.  Position i sets it for the heads w in
// (key[i-1], key[i]], with key[-1] = -1 and key[nnz] = n, so every w in
// [0, n] is set exactly once (roff[n] = nnz).
__global__ void k_in_offsets(const uint32_t *__restrict__ key, int64_t nnz, int32_t n, int64_t *roff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nnz; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = i == 0 ? -1 : (int64_t)key[i - 1];
    const int64_t hi = i == nnz ? (int64_t)n : (int64_t)key[i];
    for (int64_t w = lo + 1; w <= hi; ++w) roff[w] = i;
  }
}

// Chunk table of the rows longer than kHeavyRow: row v contributes
// ceil(deg/kChunk) chunks starting at off[v], off[v]+kChunk, ...
__global__ void k_chunk_count(const int64_t *off, int32_t n, int32_t *cnt) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int64_t d = off[v + 1] - off[v];
    cnt[v] = d > kHeavyRow ? (int32_t)((d + kChunk - 1) / kChunk) : 0;
  }
}
__global__ void k_chunk_fill(const int64_t *off, int32_t n, const int64_t *coff, int32_t *cw, int64_t *cbeg) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    for (int64_t c = coff[v]; c < coff[v + 1]; ++c) {
      cw[c] = v;
      cbeg[c] = off[v] + (c - coff[v]) * kChunk;
    }
  }
}

static void build_chunks(const int64_t *off, int32_t n, ChunkTable &T, cudaStream_t st, Stats *S) {
  DevBuf cnt, coff, tmp;
  cnt.ensure(4 * (size_t)n, st);
  coff.ensure(8 * ((size_t)n + 1), st);
  launch(S, K_GRAPH, st, [&] { k_chunk_count<<<grid_for(n, 256), 256, 0, st>>>(off, n, cnt.as<int32_t>()); });
  counts_to_offsets(cnt.as<int32_t>(), coff.as<int64_t>(), (size_t)n, tmp, st, S);
  int64_t total = 0;
  CEN_CK(cudaMemcpyAsync(&total, coff.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  T.count = total;
  T.w.ensure(4 * (size_t)(total + 1), st);
  T.beg.ensure(8 * (size_t)(total + 1), st);
  if (total)
    launch(S, K_GRAPH, st, [&] {
      k_chunk_fill<<<grid_for(n, 256), 256, 0, st>>>(off, n, coff.as<int64_t>(), T.w.as<int32_t>(),
                                                     T.beg.as<int64_t>());
    });
  CEN_CK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------- canonical form
// Offsets non-decreasing from 0 to nnz and every id in [0, n): else *bad = 1.
__global__ void k_check_ids(const int64_t *__restrict__ off, const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                            int *bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= (int64_t)n; i += (int64_t)gridDim.x * blockDim.x)
    if ((i == 0 && off[0] != 0) || (i == n && off[n] != nnz) || (i > 0 && off[i] < off[i - 1])) *bad = 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    if (col[e] < 0 || col[e] >= n) *bad = 1;
}

// Arc list of the input rows (u, v), and with `both` also (v, u).
__global__ void k_arc_list(const int64_t *__restrict__ off, const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                           bool both, uint32_t *tail, uint32_t *head) {
  for (int32_t u = blockIdx.x * blockDim.y + threadIdx.y; u < n; u += gridDim.x * blockDim.y)
    for (int64_t e = off[u] + threadIdx.x; e < off[u + 1]; e += blockDim.x) {
      tail[e] = (uint32_t)u;
      head[e] = (uint32_t)col[e];
      if (both) {
        tail[nnz + e] = (uint32_t)col[e];
        head[nnz + e] = (uint32_t)u;
      }
    }
}

// keep[i] = arc i (of the list sorted by (tail, head)) is not a self-loop and
// not a repeat of arc i - 1; cnt[tail] counts the kept arcs of each row.
__global__ void k_keep_arcs(const uint32_t *__restrict__ tail, const uint32_t *__restrict__ head, int64_t A,
                            int64_t *keep, int32_t *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A; i += (int64_t)gridDim.x * blockDim.x) {
    const bool k = tail[i] != head[i] && (i == 0 || tail[i] != tail[i - 1] || head[i] != head[i - 1]);
    keep[i] = k;
    if (k) atomicAdd(&cnt[tail[i]], 1);
  }
}

__global__ void k_pack_arcs(const uint32_t *__restrict__ head, const int64_t *__restrict__ keep,
                            const int64_t *__restrict__ pos, int64_t A, int32_t *col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A; i += (int64_t)gridDim.x * blockDim.x)
    if (keep[i]) col[pos[i]] = (int32_t)head[i];
}

// Canonical CSR of the input rows on the device: rows sorted, repeated arcs and
// self-loops dropped, and with `symmetrize` the reverse of every arc added
// first.  Sets g->off, g->col and g->nnz.  Ids out of [0, n) or malformed
// offsets give CEN_EINVAL.
void graph_canonicalize(cen_graph *g, const int64_t *off, const int32_t *col, int64_t nnz, bool on_device,
                        bool symmetrize, Stats *S) {
  cudaStream_t st = g->st;
  const int32_t n = g->n;
  DevBuf ioff, icol, bad;
  ioff.ensure(8 * ((size_t)n + 1), st);
  icol.ensure(4 * (size_t)(nnz > 0 ? nnz : 1), st);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CEN_CK(cudaMemcpyAsync(ioff.p, off, 8 * ((size_t)n + 1), kind, st));
  if (nnz) CEN_CK(cudaMemcpyAsync(icol.p, col, 4 * (size_t)nnz, kind, st));
  bad.ensure(4, st);
  CEN_CK(cudaMemsetAsync(bad.p, 0, 4, st));
  launch(S, K_GRAPH, st, [&] {
    k_check_ids<<<grid_for((size_t)std::max<int64_t>(nnz, n + 1), 256), 256, 0, st>>>(
        ioff.as<int64_t>(), icol.as<int32_t>(), n, nnz, bad.as<int>());
  });
  int hbad = 0;
  CEN_CK(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_REQUIRE(hbad == 0, CEN_EINVAL, "cen_graph_load: offsets must rise from 0 to nnz and ids lie in [0, n)");
  const int64_t A = symmetrize ? 2 * nnz : nnz;
  CEN_REQUIRE(A < ((int64_t)1 << 32), CEN_EINVAL, "cen_graph_load: too many arcs to canonicalize");
  g->off.ensure(8 * ((size_t)n + 1), st);
  g->col.ensure(4 * (size_t)(A > 0 ? A : 1), st);
  if (A == 0) {
    CEN_CK(cudaMemsetAsync(g->off.p, 0, 8 * ((size_t)n + 1), st));
    g->nnz = 0;
    return;
  }
  DevBuf tail, head, k2, v2, hist, tmp, keep, pos, cnt;
  tail.ensure(4 * (size_t)A, st);
  head.ensure(4 * (size_t)A, st);
  launch(S, K_GRAPH, st, [&] {
    k_arc_list<<<grid_for((size_t)n, 8, sm_count() * 64), dim3(32, 8), 0, st>>>(ioff.as<int64_t>(), icol.as<int32_t>(), n,
                                                                        nnz, symmetrize, tail.as<uint32_t>(),
                                                                        head.as<uint32_t>());
  });
  int bits = 1;
  while (bits < 31 && (1u << bits) < (uint32_t)n) ++bits;
  // by head, then (stably) by tail: the arcs end up sorted by (tail, head)
  radix_sort_pairs(head.as<uint32_t>(), tail.as<uint32_t>(), (size_t)A, bits, k2, v2, hist, tmp, st, S);
  radix_sort_pairs(tail.as<uint32_t>(), head.as<uint32_t>(), (size_t)A, bits, k2, v2, hist, tmp, st, S);
  keep.ensure(8 * (size_t)A, st);
  pos.ensure(8 * (size_t)(A + 1), st);
  cnt.ensure(4 * (size_t)n, st);
  CEN_CK(cudaMemsetAsync(cnt.p, 0, 4 * (size_t)n, st));
  launch(S, K_GRAPH, st, [&] {
    k_keep_arcs<<<grid_for((size_t)A, 256), 256, 0, st>>>(tail.as<uint32_t>(), head.as<uint32_t>(), A,
                                                           keep.as<int64_t>(), cnt.as<int32_t>());
  });
  exclusive_scan_i64(keep.as<int64_t>(), pos.as<int64_t>(), (size_t)A, pos.as<int64_t>() + A, tmp, st, S);
  launch(S, K_GRAPH, st, [&] {
    k_pack_arcs<<<grid_for((size_t)A, 256), 256, 0, st>>>(head.as<uint32_t>(), keep.as<int64_t>(), pos.as<int64_t>(),
                                                           A, g->col.as<int32_t>());
  });
  counts_to_offsets(cnt.as<int32_t>(), g->off.as<int64_t>(), (size_t)n, tmp, st, S);
  int64_t kept = 0;
  CEN_CK(cudaMemcpyAsync(&kept, pos.as<int64_t>() + A, 8, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  g->nnz = kept;
}

// Sums of d and d^2 over the rows of off (one pass, double sums).
__global__ void k_degree_moments(const int64_t *__restrict__ off, int32_t n, double *sums) {
  double a = 0.0, b = 0.0;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double d = (double)(off[v + 1] - off[v]);
    a += d;
    b += d * d;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

// The chunk tables of the bit-parallel sampler's long rows, built on their
// first use (on `st`, synchronized; released later on the graph's stream).
static void graph_chunks_ready(const cen_graph *g, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g->chunks_mu);
  if (g->chunks_built) return;
  build_chunks(g->off.as<int64_t>(), g->n, g->out_chunks, st, nullptr);
  if (g->directed) build_chunks(g->roff.as<int64_t>(), g->n, g->in_chunks_own, st, nullptr);
  for (DevBuf *b : {&g->out_chunks.w, &g->out_chunks.beg, &g->in_chunks_own.w, &g->in_chunks_own.beg}) b->st = g->st;
  g->chunks_built = true;
}

const ChunkTable &graph_out_chunks(const cen_graph *g, cudaStream_t st) {
  graph_chunks_ready(g, st);
  return g->out_chunks;
}

const ChunkTable &graph_in_chunks(const cen_graph *g, cudaStream_t st) {
  graph_chunks_ready(g, st);
  return g->directed ? g->in_chunks_own : g->out_chunks;
}

double graph_branching(const cen_graph *g, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g->branching_mu);
  if (g->branching >= 0.0) return g->branching;
  DevBuf sums;
  sums.ensure(4 * sizeof(double), st);
  CEN_CK(cudaMemsetAsync(sums.p, 0, 4 * sizeof(double), st));
  const int blocks = grid_for((size_t)g->n, 256, sm_count() * 4);
  k_degree_moments<<<blocks, 256, 0, st>>>(g->off.as<int64_t>(), g->n, sums.as<double>());
  if (g->directed) k_degree_moments<<<blocks, 256, 0, st>>>(g->in_off(), g->n, sums.as<double>() + 2);
  CEN_CK(cudaGetLastError());
  double h[4] = {0, 0, 0, 0};
  CEN_CK(cudaMemcpyAsync(h, sums.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  const double out = h[0] > 0 ? h[1] / h[0] : 0.0, in = h[2] > 0 ? h[3] / h[2] : 0.0;
  g->branching = out > in ? out : in;
  return g->branching;
}

void graph_build(cen_graph *g, const int64_t *off, const int32_t *col, bool on_device, Stats *S) {
  cudaStream_t st = g->st;
  const int32_t n = g->n;
  const int64_t nnz = g->nnz;
  if (off) {  // null: g->off / g->col already hold the graph (see graph_canonicalize)
    g->off.ensure(sizeof(int64_t) * ((size_t)n + 1), st);
    g->col.ensure(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), st);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CEN_CK(cudaMemcpyAsync(g->off.p, off, sizeof(int64_t) * ((size_t)n + 1), kind, st));
    if (nnz) CEN_CK(cudaMemcpyAsync(g->col.p, col, sizeof(int32_t) * (size_t)nnz, kind, st));
  }
  // the validation flag and the degree moments (sums of d and d^2 over the
  // out-rows, then the in-rows) come back in one copy
  struct Check {
    double sums[4];
    int bad;
  };
  DevBuf chk;
  chk.ensure(sizeof(Check), st);
  CEN_CK(cudaMemsetAsync(chk.p, 0, sizeof(Check), st));
  Check *dchk = chk.as<Check>();
  DevBuf start;
  start.ensure((size_t)(nnz > 0 ? nnz : 1), st);
  CEN_CK(cudaMemsetAsync(start.p, 0, (size_t)(nnz > 0 ? nnz : 1), st));
  launch(S, K_GRAPH, st, [&] {
    k_mark_starts<<<grid_for((size_t)n, 256), 256, 0, st>>>(g->off.as<int64_t>(), n, nnz, start.as<uint8_t>(),
                                                           &dchk->bad);
  });
  if (nnz)
    launch(S, K_GRAPH, st, [&] {
      k_check_arcs<<<grid_for((size_t)nnz, 256), 256, 0, st>>>(g->col.as<int32_t>(), n, nnz, start.as<uint8_t>(),
                                                                &dchk->bad);
    });
  launch(S, K_GRAPH, st, [&] {
    k_check_loops<<<grid_for((size_t)n, 256), 256, 0, st>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), n, nnz,
                                                           &dchk->bad);
  });
  const int mblocks = grid_for((size_t)n, 256, sm_count() * 4);
  launch(S, K_GRAPH, st,
         [&] { k_degree_moments<<<mblocks, 256, 0, st>>>(g->off.as<int64_t>(), n, dchk->sums); });
  Check h{};
  CEN_CK(cudaMemcpyAsync(&h, chk.p, sizeof(Check), cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_REQUIRE(h.bad == 0, CEN_EINVAL,
              "cen_graph_load: CSR is not canonical (offsets, ids in [0,n), no self-loops, rows strictly ascending)");
  const double bout = h.sums[0] > 0 ? h.sums[1] / h.sums[0] : 0.0;
  if (!g->directed || nnz == 0) {
    if (g->directed) {  // no arcs: in-CSR is all zeros
      g->roff.ensure(sizeof(int64_t) * ((size_t)n + 1), st);
      CEN_CK(cudaMemsetAsync(g->roff.p, 0, sizeof(int64_t) * ((size_t)n + 1), st));
      g->rcol.ensure(4, st);
      CEN_CK(cudaStreamSynchronize(st));
    }
    g->branching = bout;
    return;
  }
  // arcs (head, tail) in CSR order, stably sorted by head: the tails of each
  // head stay ascending, so rcol rows are ascending; the tails are sorted in
  // place in rcol
  DevBuf key, k2, v2, hist, tmp;
  key.ensure(4 * (size_t)nnz, st);
  g->rcol.ensure(4 * (size_t)nnz, st);
  launch(S, K_GRAPH, st, [&] {
    k_arcs_by_tail<<<grid_for((size_t)n, 8), 256, 0, st>>>(g->off.as<int64_t>(), g->col.as<int32_t>(), n,
                                                           key.as<uint32_t>(), g->rcol.as<uint32_t>());
  });
  int bits = 1;
  while (bits < 31 && (1u << bits) < (uint32_t)n) ++bits;
  radix_sort_pairs(key.as<uint32_t>(), g->rcol.as<uint32_t>(), (size_t)nnz, bits, k2, v2, hist, tmp, st, S);
  g->roff.ensure(sizeof(int64_t) * ((size_t)n + 1), st);
  launch(S, K_GRAPH, st, [&] {
    k_in_offsets<<<grid_for((size_t)nnz + 1, 256), 256, 0, st>>>(key.as<uint32_t>(), nnz, n, g->roff.as<int64_t>());
  });
  launch(S, K_GRAPH, st,
         [&] { k_degree_moments<<<mblocks, 256, 0, st>>>(g->roff.as<int64_t>(), n, dchk->sums + 2); });
  CEN_CK(cudaMemcpyAsync(&h, chk.p, sizeof(Check), cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  const double bin = h.sums[2] > 0 ? h.sums[3] / h.sums[2] : 0.0;
  g->branching = bout > bin ? bout : bin;
}

}  // namespace cen
