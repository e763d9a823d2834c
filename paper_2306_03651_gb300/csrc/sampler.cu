// Bit-parallel hyper-edge sampler for set betweenness (Sec. 3.1, Sec. 5 sampleHEs).
//
// A wave handles W = 64 G samples ("slots").  Each slot b draws its pair
// (s_b, t_b); all W searches then advance together, one BFS level per step,
// with every per-vertex set stored as G 64-bit words (bit b%64 of word b/64):
//   1. discovery: lev[L][v] = slots whose BFS reaches v at distance exactly L.
//      Before expanding level L, slot b stops if some in-neighbour of t_b is in
//      lev[L] (then d(s,t) = L+1); the last level is never expanded.
//   2. cone: walking levels downwards, lev[L] is cut to the nodes that lie on
//      some shortest s_b -> t_b path (in-neighbours of t_b at level d-1, then
//      in-neighbours of cone nodes one level lower).
//   3. path counts sigma_b[v] (number of shortest s_b -> v paths) on the cone
//      only, pulled from cone in-neighbours one level lower; every
//      predecessor of a cone node is itself a cone node, so these equal the
//      counts of a full BFS, and they are all the backward walk reads.
//   4. backward walk from t_b: at v on level L draw r uniform below sigma_v
//      (Philox purpose 2 + (d - L)), scan v's in-neighbours in ascending id,
//      add sigma of those on level L-1, take the first whose running sum
//      exceeds r.  The interior nodes are written to the hyper-edge in s->t
//      order.  A slot whose sigma_t reaches 2^64 is re-run with 128-bit counts.
#include <algorithm>
#include <cstring>

#include "job.cuh"

namespace cen {

struct Ctl {
  unsigned long long active[32];  // slots still searching
  unsigned long long alive[32];   // slots whose newest level is non-empty
  unsigned long long farcs;       // out-arcs of the frontier list
  long long total;                // members appended by this wave
  int fcount;                     // frontier list length
  int nflag;                      // slots flagged for 128-bit counts
  int err;                        // CEN_* code from device
  int pad;
  int flagged[2048];
};
constexpr int kMaxG = 32;
constexpr int kMaxW = 64 * kMaxG;

// --------------------------------------------------------------- init
template <class T>
__global__ void k_wave_init(int count, uint64_t jbase, const uint64_t *__restrict__ jlist, int32_t n, uint64_t seed,
                            int G, int W, uint64_t *slot_j, int32_t *slot_s, int32_t *slot_t, int32_t *slot_d,
                            uint64_t *lev0, uint64_t *vis, T *sig, const int64_t *__restrict__ off, int32_t *flist,
                            Ctl *ctl) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < W; b += gridDim.x * blockDim.x) {
    if (b >= count) {
      slot_d[b] = -3;
      continue;
    }
    const uint64_t j = jlist ? jlist[b] : jbase + (uint64_t)b;
    // Sec. 5: s uniform over V; t uniform over V \ {s} (Sec. 3.1 pairs u != v)
    const int32_t s = (int32_t)uniform_below64(seed, j, kPurposeS, (uint64_t)n);
    const int32_t tt = (int32_t)uniform_below64(seed, j, kPurposeT, (uint64_t)(n - 1));
    const int32_t t = tt + (tt >= s);
    slot_j[b] = j;
    slot_s[b] = s;
    slot_t[b] = t;
    slot_d[b] = -2;
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    atomicOr((unsigned long long *)&lev0[(int64_t)s * G + g], bit);
    atomicOr((unsigned long long *)&vis[(int64_t)s * G + g], bit);
    sig[(int64_t)s * W + b] = (T)1;
    atomicOr(&ctl->active[g], bit);
    const int pos = atomicAdd(&ctl->fcount, 1);
    flist[pos] = s;
    atomicAdd(&ctl->farcs, (unsigned long long)(off[s + 1] - off[s]));
  }
}

// ------------------------------------------------------- target check
// Warp per slot: before level L is expanded, slot b finishes when t_b has an
// in-neighbour at distance L (d = L+1), or when its level L is empty (t_b is
// unreachable: Sec. 5 returns the empty set).
__global__ void k_tcheck(int W, int G, int L, const int32_t *__restrict__ slot_t, int32_t *slot_d,
                         const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                         const uint64_t *__restrict__ lev, Ctl *ctl, int use_alive, unsigned long long *units) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < W; b += nwarps) {
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    if (!(((volatile unsigned long long *)ctl->active)[g] & bit)) continue;
    if (use_alive && !(ctl->alive[g] & bit)) {
      if (lane == 0) {
        slot_d[b] = -1;
        atomicAnd(&ctl->active[g], ~bit);
      }
      continue;
    }
    const int32_t t = slot_t[b];
    const int64_t e0 = roff[t], e1 = roff[t + 1];
    bool found = false;
    for (int64_t base = e0; base < e1 && !found; base += 32) {
      const int64_t i = base + lane;
      bool hit = false;
      if (i < e1) hit = (lev[(int64_t)rcol[i] * G + g] & bit) != 0;
      found = __any_sync(0xffffffffu, hit);
      scanned += 32;
    }
    if (found && lane == 0) {
      slot_d[b] = L + 1;
      atomicAnd(&ctl->active[g], ~bit);
    }
  }
  if (lane == 0 && scanned) atomicAdd(units, scanned / 32);
}

// ----------------------------------------------------------- expansion
// Lane layout for per-vertex word work: g = lane % G (word), a = lane / G
// (which of the A = 32/G arcs handled in parallel).

// Bottom-up: every node w with an unreached active slot ORs the level-L words
// of its in-neighbours (stopping once every unreached slot is found).
__global__ void __launch_bounds__(256) k_expand_pull(const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                                                     int32_t n, int G, int gshift, const uint64_t *__restrict__ lev,
                                                     uint64_t *__restrict__ nxt, const uint64_t *__restrict__ vis,
                                                     const Ctl *__restrict__ ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0, verts = 0, opened = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nwarps) {
    ++verts;
    const uint64_t unv = act & ~vis[w * G + g];
    if (!__any_sync(0xffffffffu, unv != 0)) {
      if (a == 0) nxt[w * G + g] = 0;
      continue;
    }
    ++opened;
    const int64_t e0 = roff[w], e1 = roff[w + 1];
    if (e1 - e0 > kHeavyRow) {  // long rows: k_expand_pull_heavy ORs their chunks in
      if (a == 0) nxt[w * G + g] = 0;
      continue;
    }
    uint64_t acc = 0;
    for (int64_t base = e0; base < e1; base += (int64_t)A * 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1) acc |= lev[(int64_t)rcol[i] * G + g];
      }
      if (e1 - e0 > (int64_t)A * 8) {  // long rows: stop once every unreached slot is found
        uint64_t r = acc;
        for (int o = G; o < 32; o <<= 1) r |= __shfl_xor_sync(0xffffffffu, r, o);
        if (__all_sync(0xffffffffu, (r & unv) == unv)) {
          scanned += (uint64_t)(base + (int64_t)A * 8 - e0);
          goto reduced;
        }
      }
    }
    scanned += (uint64_t)(e1 - e0);
  reduced:
    for (int o = G; o < 32; o <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    if (a == 0) nxt[w * G + g] = acc & unv;
  }
  // algorithmic bytes: every node reads its reached word and writes its next
  // word (16 G); an opened node reads its two offsets (16) and, per scanned
  // in-arc, the arc (4) and the tail's level words (8 G)
  if (lane == 0 && verts)
    atomicAdd(units, verts * 16ull * G + opened * 16ull + scanned * (4ull + 8ull * G));
}

// Bottom-up over the chunks of long rows: warp per chunk, OR of the chunk's
// in-neighbour level words, merged into the node's next word.
__global__ void __launch_bounds__(256) k_expand_pull_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                           const int64_t *__restrict__ cbeg,
                                                           const int64_t *__restrict__ roff,
                                                           const int32_t *__restrict__ rcol, int G, int gshift,
                                                           const uint64_t *__restrict__ lev, uint64_t *nxt,
                                                           const uint64_t *__restrict__ vis,
                                                           const Ctl *__restrict__ ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int32_t w = cw[q];
    const uint64_t unv = act & ~vis[(int64_t)w * G + g];
    bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, unv != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, roff[w + 1]);
    uint64_t acc = 0;
    for (int64_t base = e0; base < e1; base += (int64_t)A * 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1) acc |= lev[(int64_t)rcol[i] * G + g];
      }
    }
    for (int o = G; o < 32; o <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    const uint64_t nb = acc & unv;
    if (a == 0 && nb) atomicOr((unsigned long long *)&nxt[(int64_t)w * G + g], (unsigned long long)nb);
    bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 8ull * G) + 16ull * G;
  }
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// Top-down: every frontier node v ORs its active level-L words into the
// next-level words of its out-neighbours.
__global__ void __launch_bounds__(256) k_expand_push(const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                     const int32_t *__restrict__ flist, int G, int gshift,
                                                     const uint64_t *__restrict__ lev, uint64_t *nxt,
                                                     const Ctl *__restrict__ ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int fcount = ctl->fcount;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < fcount; q += nwarps) {
    const int32_t v = flist[q];
    const int64_t e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 > kHeavyRow) continue;  // long rows: k_expand_push_heavy
    const uint64_t f = lev[(int64_t)v * G + g] & act;
    if (!__any_sync(0xffffffffu, f != 0)) continue;
    for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1 && f) atomicOr((unsigned long long *)&nxt[(int64_t)col[i] * G + g], (unsigned long long)f);
      }
    }
    // bytes: offsets (16) and level words (8 G) of v; per out-arc the arc (4)
    // and an 8-byte read-modify-write per non-empty word
    const int nzw = __popc(__ballot_sync(0xffffffffu, f != 0 && a == 0));
    scanned += 16ull + 8ull * G + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  if (lane == 0 && scanned) atomicAdd(units, scanned);
}

// Top-down over the chunks of long out-rows: a chunk of a frontier node pushes
// its active level words to the chunk's out-neighbours.
__global__ void __launch_bounds__(256) k_expand_push_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                           const int64_t *__restrict__ cbeg,
                                                           const int64_t *__restrict__ off,
                                                           const int32_t *__restrict__ col, int G, int gshift,
                                                           const uint64_t *__restrict__ lev, uint64_t *nxt,
                                                           const Ctl *__restrict__ ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int32_t v = cw[q];
    const uint64_t f = lev[(int64_t)v * G + g] & act;
    bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, f != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, off[v + 1]);
    for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1 && f) atomicOr((unsigned long long *)&nxt[(int64_t)col[i] * G + g], (unsigned long long)f);
      }
    }
    const int nzw = __popc(__ballot_sync(0xffffffffu, f != 0 && a == 0));
    bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// Thread per word: keep only newly reached active slots, mark them reached,
// collect the non-empty nodes into the frontier list and OR the per-word
// "level not empty" masks.
__global__ void __launch_bounds__(256) k_level_finalize(int32_t n, int G, int gshift, uint64_t *__restrict__ nxt,
                                                        uint64_t *__restrict__ vis, const int64_t *__restrict__ off,
                                                        int32_t *flist, Ctl *ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31;
  const int g = lane & (G - 1);
  const uint64_t act = ctl->active[g];
  const int64_t words = (int64_t)n * G;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint64_t alive = 0;
  unsigned long long arcs = 0;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < words; base += nwarps * 32) {
    const int64_t idx = base + lane;
    uint64_t nb = 0;
    if (idx < words) {
      nb = nxt[idx] & ~vis[idx] & act;
      nxt[idx] = nb;
      if (nb) vis[idx] |= nb;
    }
    alive |= nb;
    uint64_t any = nb;
    for (int o = 1; o < G; o <<= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
    const bool head = (g == 0) && idx < words && any != 0;
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    if (hm) {
      int basepos = 0;
      if (lane == __ffs(hm) - 1) basepos = atomicAdd(&ctl->fcount, __popc(hm));
      basepos = __shfl_sync(0xffffffffu, basepos, __ffs(hm) - 1);
      if (head) {
        const int32_t w = (int32_t)(idx >> gshift);
        flist[basepos + __popc(hm & ((1u << lane) - 1u))] = w;
        arcs += (unsigned long long)(off[w + 1] - off[w]);
      }
    }
  }
  for (int o = G; o < 32; o <<= 1) alive |= __shfl_xor_sync(0xffffffffu, alive, o);
  if (lane < G && alive) atomicOr(&ctl->alive[g], (unsigned long long)alive);
  arcs = warp_sum(arcs);
  if (lane == 0 && arcs) atomicAdd(&ctl->farcs, arcs);
  // bytes: each word is read twice (next, reached) and written twice
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(units, (unsigned long long)words * 32ull);
}

// ------------------------------------------------------ offsets + store
// One block: slot lengths max(d-1, 0) -> hoff of the wave's samples, per-sample
// s, t, d, and the running max |h|.
__global__ void __launch_bounds__(1024) k_wave_append(int count, uint64_t jbase, const int32_t *slot_s,
                                                      const int32_t *slot_t, const int32_t *slot_d, int64_t *hoff,
                                                      int32_t *ps, int32_t *pt, int32_t *pd, int *bmax, Ctl *ctl) {
  __shared__ long long wsum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const long long base = hoff[jbase];
  int mymax = 0;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int b = c0 + threadIdx.x;
    int len = 0;
    if (b < count) {
      const int d = slot_d[b];
      len = d >= 2 ? d - 1 : 0;
      ps[jbase + b] = slot_s[b];
      pt[jbase + b] = slot_t[b];
      pd[jbase + b] = d;
      mymax = max(mymax, len);
    }
    long long x = len;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long v = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;
    }
    __syncthreads();
    const long long incl = carry + (warp ? wsum[warp - 1] : 0) + x;
    if (b < count) hoff[jbase + b + 1] = base + incl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  for (int o = 16; o; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
  if ((threadIdx.x & 31) == 0 && mymax) atomicMax(bmax, mymax);
  if (threadIdx.x == 0) ctl->total = carry;
}

// ------------------------------------------------------------------ cone
// Warp per slot with d-1 == L: in-neighbours of t_b at level L seed the cone.
__global__ void k_cone_seed(int W, int G, int L, const int32_t *__restrict__ slot_t, const int32_t *__restrict__ slot_d,
                            const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                            const uint64_t *__restrict__ lev, uint64_t *tmp) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < W; b += nwarps) {
    const int d = slot_d[b];
    if (d < 2 || d - 1 != L) continue;
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    const int32_t t = slot_t[b];
    for (int64_t i = roff[t] + lane; i < roff[t + 1]; i += 32) {
      const int32_t x = rcol[i];
      if (lev[(int64_t)x * G + g] & bit) atomicOr((unsigned long long *)&tmp[(int64_t)x * G + g], bit);
    }
  }
}

// Warp per node x: cone words of x at level L+1 go to x's in-neighbours.
__global__ void __launch_bounds__(256) k_cone_push(int32_t n, int G, int gshift, const int64_t *__restrict__ roff,
                                                   const int32_t *__restrict__ rcol, const uint64_t *__restrict__ up,
                                                   uint64_t *tmp, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0, verts = 0;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
    ++verts;
    const uint64_t c = up[x * G + g];
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    const int64_t e0 = roff[x], e1 = roff[x + 1];
    if (e1 - e0 > kHeavyRow) continue;  // long rows: k_cone_push_heavy
    for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1 && c) atomicOr((unsigned long long *)&tmp[(int64_t)rcol[i] * G + g], (unsigned long long)c);
      }
    }
    const int nzw = __popc(__ballot_sync(0xffffffffu, c != 0 && a == 0));
    scanned += 16ull + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  // bytes: every node's cone words (8 G); a non-empty node's offsets, arcs and
  // one read-modify-write per non-empty word and arc
  if (lane == 0) atomicAdd(units, scanned + verts * 8ull * G);
}

// Chunks of long rows: cone words of x at level L+1 go to the chunk's in-neighbours.
__global__ void __launch_bounds__(256) k_cone_push_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                         const int64_t *__restrict__ cbeg,
                                                         const int64_t *__restrict__ roff,
                                                         const int32_t *__restrict__ rcol, int G, int gshift,
                                                         const uint64_t *__restrict__ up, uint64_t *tmp,
                                                         unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int32_t x = cw[q];
    const uint64_t c = up[(int64_t)x * G + g];
    bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, roff[x + 1]);
    for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1 && c) atomicOr((unsigned long long *)&tmp[(int64_t)rcol[i] * G + g], (unsigned long long)c);
      }
    }
    const int nzw = __popc(__ballot_sync(0xffffffffu, c != 0 && a == 0));
    bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// Thread per word: lev[L] &= tmp; tmp = 0.
__global__ void k_cone_fin(int64_t words, uint64_t *__restrict__ lev, uint64_t *__restrict__ tmp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = tmp[i];
    const uint64_t l = lev[i];
    if (l) lev[i] = l & c;
    if (c) tmp[i] = 0;
  }
}

// ------------------------------------------------------------- counts
// Path counts on the cone, level L from level L-1.  Lane layout (g, a) as in
// the expansion.  Warp per node w with cone slots c (word g): the counts of
// those slots are zeroed, then every in-neighbour v with cone slots f = c &
// levP[v] adds its counts with 64-bit atomics; a wrap-around (true sum >=
// 2^64) or an overflowed predecessor sets the slot's overflow flag.  Long
// rows only get zeroed here; k_cone_sigma64_heavy adds their chunks.
__device__ __forceinline__ unsigned long long sigma_arcs(int64_t e0, int64_t e1, int A, int a, int G, int g, int W,
                                                         int64_t w, uint64_t c, const int32_t *__restrict__ rcol,
                                                         const uint64_t *__restrict__ levP,
                                                         uint64_t *__restrict__ sig,
                                                         const uint64_t *__restrict__ ovf, uint64_t &myovf) {
  unsigned long long bytes = 0;
  for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = base + (int64_t)u * A + a;
      if (i >= e1) continue;
      const int32_t v = rcol[i];
      uint64_t f = levP[(int64_t)v * G + g] & c;
      if (!f) continue;
      myovf |= ovf[(int64_t)v * G + g] & f;
      bytes += 8ull;
      while (f) {
        const int b = __ffsll((long long)f) - 1;
        f &= f - 1;
        const unsigned long long x = sig[(int64_t)v * W + 64 * g + b];
        const unsigned long long old = atomicAdd((unsigned long long *)&sig[w * W + 64 * g + b], x);
        if (old + x < old) myovf |= 1ull << b;
        bytes += 24ull;
      }
    }
  }
  return bytes;
}

__global__ void __launch_bounds__(256) k_cone_sigma64(int32_t n, int G, int gshift, int W,
                                                      const int64_t *__restrict__ roff,
                                                      const int32_t *__restrict__ rcol,
                                                      const uint64_t *__restrict__ levL,
                                                      const uint64_t *__restrict__ levP, uint64_t *__restrict__ sig,
                                                      uint64_t *__restrict__ ovf, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0, verts = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nwarps) {
    ++verts;
    const uint64_t c = levL[w * G + g];
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    for (uint64_t z = c; z; z &= z - 1) {
      const int b = __ffsll((long long)z) - 1;
      if ((b & (A - 1)) == a) sig[w * W + 64 * g + b] = 0;
    }
    __syncwarp();
    const int64_t e0 = roff[w], e1 = roff[w + 1];
    if (e1 - e0 > kHeavyRow) continue;
    uint64_t myovf = 0;
    bytes += sigma_arcs(e0, e1, A, a, G, g, W, w, c, rcol, levP, sig, ovf, myovf);
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 8ull * G);
    for (int o = G; o < 32; o <<= 1) myovf |= __shfl_xor_sync(0xffffffffu, myovf, o);
    if (a == 0 && myovf) atomicOr((unsigned long long *)&ovf[w * G + g], (unsigned long long)myovf);
  }
  // bytes: every node's cone words (8 G); per opened node its offsets and,
  // per in-arc, the arc (4) and the tail's cone words (8 G); per contributing
  // (arc, slot) the tail's overflow word share, its count and the atomic add
  bytes = warp_sum(bytes);
  if (lane == 0) atomicAdd(units, bytes + verts * 8ull * G);
}

__global__ void __launch_bounds__(256) k_cone_sigma64_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                            const int64_t *__restrict__ cbeg, int G, int gshift,
                                                            int W, const int64_t *__restrict__ roff,
                                                            const int32_t *__restrict__ rcol,
                                                            const uint64_t *__restrict__ levL,
                                                            const uint64_t *__restrict__ levP,
                                                            uint64_t *__restrict__ sig, uint64_t *__restrict__ ovf,
                                                            unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int64_t w = cw[q];
    const uint64_t c = levL[w * G + g];
    if (lane == 0) bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, roff[w + 1]);
    uint64_t myovf = 0;
    bytes += sigma_arcs(e0, e1, A, a, G, g, W, w, c, rcol, levP, sig, ovf, myovf);
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 8ull * G);
    for (int o = G; o < 32; o <<= 1) myovf |= __shfl_xor_sync(0xffffffffu, myovf, o);
    if (a == 0 && myovf) atomicOr((unsigned long long *)&ovf[w * G + g], (unsigned long long)myovf);
  }
  bytes = warp_sum(bytes);
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// 128-bit counts for a re-run wave (G = 1): lane handles slots lane and
// lane + 32, each summing its cone in-neighbours' counts serially.
__global__ void __launch_bounds__(256) k_cone_sigma128(int32_t n, const int64_t *__restrict__ roff,
                                                       const int32_t *__restrict__ rcol,
                                                       const uint64_t *__restrict__ levL,
                                                       const uint64_t *__restrict__ levP, u128 *__restrict__ sig,
                                                       uint64_t *__restrict__ ovf) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nwarps) {
    const uint64_t c = levL[w];
    if (!c) continue;
    uint64_t myovf = 0;
    for (int h = 0; h < 2; ++h) {
      const int b = lane + 32 * h;
      if (!((c >> b) & 1)) continue;
      u128 acc = 0;
      bool of = false;
      for (int64_t i = roff[w]; i < roff[w + 1]; ++i) {
        const int32_t v = rcol[i];
        if (!((levP[v] >> b) & 1)) continue;
        if ((ovf[v] >> b) & 1) of = true;
        const u128 x = sig[(int64_t)v * 64 + b];
        const u128 r = acc + x;
        if (r < acc) of = true;
        acc = r;
      }
      sig[w * 64 + b] = acc;
      if (of) myovf |= 1ull << b;
    }
    for (int o = 16; o; o >>= 1) myovf |= __shfl_xor_sync(0xffffffffu, myovf, o);
    if (lane == 0 && myovf) ovf[w] |= myovf;
  }
}

// ----------------------------------------------------------------- walk
__device__ __forceinline__ uint64_t shfl_up_T(uint64_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ u128 shfl_up_T(u128 v, int o) {
  const uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)v, o);
  const uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ uint64_t shfl_xor_T(uint64_t v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ u128 shfl_xor_T(u128 v, int o) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, o);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_T(u128 v, int src) {
  const uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)v, src);
  const uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(v >> 64), src);
  return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ uint64_t shfl_T(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ uint64_t draw_below(uint64_t seed, uint64_t j, uint32_t p, uint64_t B) {
  return uniform_below64(seed, j, p, B);
}
__device__ __forceinline__ u128 draw_below(uint64_t seed, uint64_t j, uint32_t p, u128 B) {
  return uniform_below128(seed, j, p, B);
}

// Warp per slot (see the file header, step 4).  T = uint64_t: a slot whose
// sigma_t does not fit is appended to ctl->flagged.  T = u128: such a slot
// sets ctl->err = CEN_EOVERFLOW.
template <class T>
__global__ void k_walk(int count, int G, int Wst, const uint64_t *__restrict__ slot_j,
                       const int32_t *__restrict__ slot_t, const int32_t *__restrict__ slot_d,
                       const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                       const uint64_t *const *__restrict__ levs, const T *__restrict__ sig,
                       const uint64_t *__restrict__ ovf, const int64_t *__restrict__ hoff, int32_t *hmem,
                       uint64_t seed, Ctl *ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < count; b += nwarps) {
    const int d = slot_d[b];
    if (d < 2) continue;
    const int g = b >> 6;
    const uint64_t bit = 1ull << (b & 63);
    const uint64_t j = slot_j[b];
    int32_t v = slot_t[b];
    int L = d;
    // sigma_t = sum over in-neighbours on level d-1 (all of them are cone nodes)
    T acc = 0;
    bool of = false;
    {
      const uint64_t *lp = levs[L - 1];
      for (int64_t i = roff[v] + lane; i < roff[v + 1]; i += 32) {
        const int32_t x = rcol[i];
        if (lp[(int64_t)x * G + g] & bit) {
          if (ovf[(int64_t)x * G + g] & bit) of = true;
          const T y = sig[(int64_t)x * Wst + b];
          const T r = acc + y;
          if (r < acc) of = true;
          acc = r;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const T y = shfl_xor_T(acc, o);
        const bool oy = __shfl_xor_sync(0xffffffffu, (int)of, o) != 0;
        const T r = acc + y;
        of = of || oy || (r < acc);
        acc = r;
      }
      scanned += (uint64_t)(roff[v + 1] - roff[v]);
    }
    if (of) {
      if (lane == 0) {
        if (sizeof(T) == 8) {
          const int pos = atomicAdd(&ctl->nflag, 1);
          ctl->flagged[pos] = b;
        } else {
          atomicExch(&ctl->err, CEN_EOVERFLOW);
        }
      }
      continue;
    }
    T sv = acc;
    const int64_t hbase = hoff[j];
    uint32_t step = 0;
    while (L >= 2) {
      const T r = draw_below(seed, j, kPurposeWalk0 + step, sv);
      const uint64_t *lp = levs[L - 1];
      T cum = 0;
      int32_t pick = -1;
      const int64_t e0 = roff[v], e1 = roff[v + 1];
      for (int64_t base = e0; base < e1; base += 32) {
        const int64_t i = base + lane;
        int32_t x = -1;
        T val = 0;
        if (i < e1) {
          x = rcol[i];
          if (lp[(int64_t)x * G + g] & bit) val = sig[(int64_t)x * Wst + b];
        }
        T pre = val;
        for (int o = 1; o < 32; o <<= 1) {
          const T y = shfl_up_T(pre, o);
          if (lane >= o) pre += y;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, (cum + pre) > r);
        scanned += 1;
        if (hit) {
          pick = __shfl_sync(0xffffffffu, x, __ffs(hit) - 1);
          break;
        }
        cum += shfl_T(pre, 31);
      }
      if (pick < 0) {  // cannot happen with consistent counts
        if (lane == 0) atomicExch(&ctl->err, CEN_EINVAL);
        break;
      }
      if (lane == 0) hmem[hbase + (L - 2)] = pick;
      sv = sig[(int64_t)pick * Wst + b];
      v = pick;
      --L;
      ++step;
    }
  }
  if (lane == 0 && scanned) atomicAdd(units, scanned);
}

// --------------------------------------------------------------- sign words
// Alg. 1 "sampleRadeVars", extended by the new columns j: word w of sample j
// is word w%4 of Philox block (j, SIGN, w/4); bits >= t are cleared.
__global__ void k_sign(uint64_t j0, uint64_t count, int t, int nw, uint64_t seed, uint32_t *sign) {
  const int nblk = (nw + 3) / 4;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count * nblk;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = j0 + idx / nblk;
    const int blk = (int)(idx % nblk);
    const uint4 x = philox_block(seed, j, kPurposeSign, (uint32_t)blk);
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int w = blk * 4 + q;
      if (w >= nw) break;
      uint32_t v = xs[q];
      const int hi = t - 32 * w;
      if (hi < 32) v &= (1u << hi) - 1u;
      sign[j * nw + w] = v;
    }
  }
}

// ------------------------------------------------------------------ host
namespace {

struct Sampler {
  cen_job *job;
  const cen_graph *g;
  cudaStream_t st;
  Stats *S;
  int32_t n;
  int G = 1, gshift = 0, W = 64;
  Ctl *ctl = nullptr;
  Ctl *hctl = nullptr;  // pinned mirror (header part)
  uint64_t *slot_j = nullptr;
  int32_t *slot_s = nullptr, *slot_t = nullptr, *slot_d = nullptr;

  unsigned long long *units(int cls) { return (unsigned long long *)(job->stats.d_units + cls); }

  void setup(int Gwant) {
    G = Gwant;
    gshift = 0;
    while ((1 << gshift) < G) ++gshift;
    W = 64 * G;
    WaveWS &ws = job->ws;
    ws.G = G;
    const size_t words = (size_t)n * G;
    ws.vis.ensure(words * 8, st);
    ws.tmp.ensure(words * 8, st);
    ws.ovf.ensure(words * 8, st);
    ws.ctl.ensure(sizeof(Ctl), st);
    ws.slots.ensure((size_t)kMaxW * (8 + 4 * 3), st);
    ws.flist.ensure((size_t)std::max<int64_t>(n, kMaxW) * 4, st);  // init lists one source per slot
    ctl = ws.ctl.as<Ctl>();
    slot_j = ws.slots.as<uint64_t>();
    slot_s = (int32_t *)(slot_j + kMaxW);
    slot_t = slot_s + kMaxW;
    slot_d = slot_t + kMaxW;
    hctl = (Ctl *)host_staging(job, sizeof(Ctl));
  }

  uint64_t *level(int L) {
    WaveWS &ws = job->ws;
    const size_t bytes = (size_t)n * G * 8;
    while ((int)ws.lev.size() <= L) ws.lev.emplace_back(new DevBuf());
    ws.lev[L]->ensure(bytes, st);
    return ws.lev[L]->as<uint64_t>();
  }

  void publish_levels(int Lmax) {
    WaveWS &ws = job->ws;
    std::vector<uint64_t *> ptrs(Lmax + 1);
    for (int L = 0; L <= Lmax; ++L) ptrs[L] = ws.lev[L]->as<uint64_t>();
    ws.lev_ptrs.ensure(sizeof(uint64_t *) * (Lmax + 1), st);
    uint64_t **h = (uint64_t **)host_staging(job, sizeof(uint64_t *) * (Lmax + 1) + sizeof(Ctl));
    memcpy(h, ptrs.data(), sizeof(uint64_t *) * (Lmax + 1));
    CEN_CK(cudaMemcpyAsync(ws.lev_ptrs.p, h, sizeof(uint64_t *) * (Lmax + 1), cudaMemcpyHostToDevice, st));
    CEN_CK(cudaStreamSynchronize(st));
    hctl = (Ctl *)host_staging(job, sizeof(Ctl));
  }

  void fetch_ctl_head() {
    CEN_CK(cudaMemcpyAsync(hctl, ctl, offsetof(Ctl, flagged), cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
  }

  bool any_active() const {
    for (int g = 0; g < G; ++g)
      if (hctl->active[g]) return true;
    return false;
  }

  // Discovery for slots [0, count): returns the highest level materialised.
  template <class T>
  int discover(int count, uint64_t jbase, const uint64_t *jlist, T *sig) {
    const size_t words = (size_t)n * G;
    uint64_t *vis = job->ws.vis.as<uint64_t>();
    int32_t *flist = job->ws.flist.as<int32_t>();
    CEN_CK(cudaMemsetAsync(vis, 0, words * 8, st));
    CEN_CK(cudaMemsetAsync(job->ws.ovf.p, 0, words * 8, st));
    CEN_CK(cudaMemsetAsync(ctl, 0, offsetof(Ctl, flagged), st));
    uint64_t *lev0 = level(0);
    CEN_CK(cudaMemsetAsync(lev0, 0, words * 8, st));
    const int64_t *off = g->off.as<int64_t>();
    const int32_t *col = g->col.as<int32_t>();
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    launch(S, K_PAIRS, st, [&] {
      k_wave_init<T><<<grid_for(W, 256), 256, 0, st>>>(count, jbase, jlist, n, job->seed, G, W, slot_j, slot_s,
                                                       slot_t, slot_d, lev0, vis, sig, off, flist, ctl);
    });
    launch(S, K_TCHECK, st, [&] {
      k_tcheck<<<grid_for((size_t)W * 32, 256), 256, 0, st>>>(W, G, 0, slot_t, slot_d, roff, rcol, lev0, ctl, 0,
                                                              units(K_TCHECK));
    });
    fetch_ctl_head();
    int L = 0;
    while (any_active()) {
      uint64_t *cur = level(L);
      uint64_t *nxt = level(L + 1);
      const bool push = (double)hctl->farcs * 4.0 < (double)g->nnz;
      const long long fcount = hctl->fcount;
      if (push) {
        CEN_CK(cudaMemsetAsync(nxt, 0, words * 8, st));
        launch(S, K_PUSH, st, [&] {
          k_expand_push<<<grid_for((size_t)fcount * 32, 256, 152 * 64), 256, 0, st>>>(
              off, col, flist, G, gshift, cur, nxt, ctl, units(K_PUSH));
        });
        const ChunkTable &oc = g->out_chunks;
        if (oc.count)
          launch(S, K_PUSH, st, [&] {
            k_expand_push_heavy<<<grid_for((size_t)oc.count * 32, 256, 152 * 64), 256, 0, st>>>(
                oc.count, oc.rows(), oc.begins(), off, col, G, gshift, cur, nxt, ctl, units(K_PUSH));
          });
      } else {
        launch(S, K_PULL, st, [&] {
          k_expand_pull<<<grid_for((size_t)n * 32, 256, 152 * 64), 256, 0, st>>>(
              roff, rcol, n, G, gshift, cur, nxt, vis, ctl, units(K_PULL));
        });
        const ChunkTable &ic = g->in_chunks();
        if (ic.count)
          launch(S, K_PULL, st, [&] {
            k_expand_pull_heavy<<<grid_for((size_t)ic.count * 32, 256, 152 * 64), 256, 0, st>>>(
                ic.count, ic.rows(), ic.begins(), roff, rcol, G, gshift, cur, nxt, vis, ctl, units(K_PULL));
          });
      }
      CEN_CK(cudaMemsetAsync(&ctl->alive, 0, sizeof(ctl->alive) + sizeof(ctl->farcs) + sizeof(ctl->total) +
                                                 sizeof(ctl->fcount), st));
      launch(S, K_LEVEL_FIN, st, [&] {
        k_level_finalize<<<grid_for(words, 256, 152 * 32), 256, 0, st>>>(n, G, gshift, nxt, vis, off, flist, ctl,
                                                                         units(K_LEVEL_FIN));
      });
      launch(S, K_TCHECK, st, [&] {
        k_tcheck<<<grid_for((size_t)W * 32, 256), 256, 0, st>>>(W, G, L + 1, slot_t, slot_d, roff, rcol, nxt, ctl,
                                                                1, units(K_TCHECK));
      });
      fetch_ctl_head();
      ++L;
      CEN_REQUIRE(L <= n, CEN_ECUDA, "cen_sample: level loop exceeded n levels");
    }
    return L;
  }

  void cone(int Lmax) {
    const size_t words = (size_t)n * G;
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    uint64_t *tmp = job->ws.tmp.as<uint64_t>();
    for (int L = Lmax; L >= 0; --L) {
      uint64_t *lev = level(L);
      launch(S, K_CONE, st, [&] {
        k_cone_seed<<<grid_for((size_t)W * 32, 256), 256, 0, st>>>(W, G, L, slot_t, slot_d, roff, rcol, lev, tmp);
      });
      if (L < Lmax) {
        uint64_t *up = level(L + 1);
        launch(S, K_CONE, st, [&] {
          k_cone_push<<<grid_for((size_t)n * 32, 256, 152 * 64), 256, 0, st>>>(n, G, gshift, roff, rcol, up, tmp,
                                                                               units(K_CONE));
        });
        const ChunkTable &ic = g->in_chunks();
        if (ic.count)
          launch(S, K_CONE, st, [&] {
            k_cone_push_heavy<<<grid_for((size_t)ic.count * 32, 256, 152 * 64), 256, 0, st>>>(
                ic.count, ic.rows(), ic.begins(), roff, rcol, G, gshift, up, tmp, units(K_CONE));
          });
      }
      launch(S, K_CONE, st, [&] { k_cone_fin<<<grid_for(words, 256, 152 * 16), 256, 0, st>>>((int64_t)words, lev, tmp); });
    }
  }

  template <class T>
  void sigma_and_walk(int count, int Lmax, T *sig) {
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    uint64_t *ovf = job->ws.ovf.as<uint64_t>();
    for (int L = 1; L <= Lmax; ++L) {
      uint64_t *lv = level(L), *lp = level(L - 1);
      if constexpr (sizeof(T) == 8) {
        launch(S, K_SIGMA, st, [&] {
          k_cone_sigma64<<<grid_for((size_t)n * 32, 256, 152 * 64), 256, 0, st>>>(
              n, G, gshift, W, roff, rcol, lv, lp, (uint64_t *)sig, ovf, units(K_SIGMA));
        });
        const ChunkTable &ic = g->in_chunks();
        if (ic.count)
          launch(S, K_SIGMA, st, [&] {
            k_cone_sigma64_heavy<<<grid_for((size_t)ic.count * 32, 256, 152 * 64), 256, 0, st>>>(
                ic.count, ic.rows(), ic.begins(), G, gshift, W, roff, rcol, lv, lp, (uint64_t *)sig, ovf,
                units(K_SIGMA));
          });
      } else {
        launch(S, K_SIGMA, st, [&] {
          k_cone_sigma128<<<grid_for((size_t)n * 32, 256, 152 * 64), 256, 0, st>>>(n, roff, rcol, lv, lp,
                                                                                   (u128 *)sig, ovf);
        });
      }
    }
    publish_levels(Lmax);
    launch(S, K_WALK, st, [&] {
      k_walk<T><<<grid_for((size_t)count * 32, 256), 256, 0, st>>>(
          count, G, W, slot_j, slot_t, slot_d, roff, rcol, job->ws.lev_ptrs.as<const uint64_t *>(), sig, ovf,
          job->hoff.as<int64_t>(), job->hmem.as<int32_t>(), job->seed, ctl, units(K_WALK));
    });
  }
};

}  // namespace

static int pick_G(uint64_t remaining, int32_t n, size_t budget) {
  int G = 1;
  while (G < kMaxG && (uint64_t)64 * G < remaining) G <<= 1;
  while (G > 1 && (size_t)n * 64 * G * 8 > budget) G >>= 1;
  return G;
}

void sample_append(cen_job *job, uint64_t m_new) {
  if (m_new == 0) return;
  const cen_graph *g = job->g;
  cudaStream_t st = job->st;
  Sampler sp;
  sp.job = job;
  sp.g = g;
  sp.st = st;
  sp.S = &job->stats;
  sp.n = g->n;
  const uint64_t m0 = job->m;
  const uint64_t m1 = m0 + m_new;
  job->hoff.ensure(sizeof(int64_t) * (m1 + 1), st, sizeof(int64_t) * (m0 + 1));
  if (m0 == 0) CEN_CK(cudaMemsetAsync(job->hoff.p, 0, sizeof(int64_t), st));
  job->ps.ensure(4 * m1, st, 4 * m0);
  job->pt.ensure(4 * m1, st, 4 * m0);
  job->pd.ensure(4 * m1, st, 4 * m0);
  job->sign.ensure(4 * (size_t)job->nw * m1, st, 4 * (size_t)job->nw * m0);
  job->bmax.ensure(4, st, 4);
  if (m0 == 0) CEN_CK(cudaMemsetAsync(job->bmax.p, 0, 4, st));
  int64_t members = job->members;
  std::vector<uint64_t> flagged_js;
  for (uint64_t j0 = m0; j0 < m1;) {
    const int G = pick_G(m1 - j0, g->n, job->sigma_budget);
    sp.setup(G);
    const int count = (int)std::min<uint64_t>((uint64_t)sp.W, m1 - j0);
    job->ws.sig64.ensure((size_t)g->n * sp.W * 8, st);
    uint64_t *sig = job->ws.sig64.as<uint64_t>();
    const int Lmax = sp.discover<uint64_t>(count, j0, nullptr, sig);
    launch(sp.S, K_APPEND, st, [&] {
      k_wave_append<<<1, 1024, 0, st>>>(count, j0, sp.slot_s, sp.slot_t, sp.slot_d, job->hoff.as<int64_t>(),
                                        job->ps.as<int32_t>(), job->pt.as<int32_t>(), job->pd.as<int32_t>(),
                                        job->bmax.as<int>(), sp.ctl);
    });
    sp.fetch_ctl_head();
    const int64_t wave_total = sp.hctl->total;
    job->hmem.ensure(4 * (size_t)(members + wave_total + 1), st, 4 * (size_t)members);
    sp.cone(Lmax);
    sp.sigma_and_walk<uint64_t>(count, Lmax, sig);
    CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent path counts in the backward walk");
    if (sp.hctl->nflag > 0) {
      std::vector<uint64_t> js(sp.hctl->nflag);
      std::vector<uint64_t> slot_js(count);
      CEN_CK(cudaMemcpyAsync(slot_js.data(), sp.slot_j, 8 * (size_t)count, cudaMemcpyDeviceToHost, st));
      CEN_CK(cudaStreamSynchronize(st));
      for (int q = 0; q < sp.hctl->nflag; ++q) flagged_js.push_back(slot_js[sp.hctl->flagged[q]]);
    }
    members += wave_total;
    j0 += (uint64_t)count;
  }
  // 128-bit re-run of the slots whose path count reached 2^64 (offsets already known)
  if (!flagged_js.empty()) {
    std::sort(flagged_js.begin(), flagged_js.end());
    sp.setup(1);
    job->ws.sig128.ensure((size_t)g->n * 64 * 16, st);
    job->ws.jlist.ensure(8 * 64, st);
    for (size_t q0 = 0; q0 < flagged_js.size(); q0 += 64) {
      const int count = (int)std::min<size_t>(64, flagged_js.size() - q0);
      uint64_t *h = (uint64_t *)host_staging(job, 8 * 64);
      memcpy(h, flagged_js.data() + q0, 8 * (size_t)count);
      CEN_CK(cudaMemcpyAsync(job->ws.jlist.p, h, 8 * (size_t)count, cudaMemcpyHostToDevice, st));
      CEN_CK(cudaStreamSynchronize(st));
      sp.hctl = (Ctl *)host_staging(job, sizeof(Ctl));
      u128 *sig = job->ws.sig128.as<u128>();
      const int Lmax = sp.discover<u128>(count, 0, job->ws.jlist.as<uint64_t>(), sig);
      sp.cone(Lmax);
      sp.sigma_and_walk<u128>(count, Lmax, sig);
      CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, offsetof(Ctl, flagged), cudaMemcpyDeviceToHost, st));
      CEN_CK(cudaStreamSynchronize(st));
      CEN_REQUIRE(sp.hctl->err != CEN_EOVERFLOW, CEN_EOVERFLOW,
                  "cen_sample: a sampled pair has >= 2^128 shortest paths");
      CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent 128-bit path counts");
    }
  }
  // sign columns of the new samples
  {
    const int nblk = (job->nw + 3) / 4;
    launch(sp.S, K_SIGN, st, [&] {
      k_sign<<<grid_for(m_new * nblk, 256), 256, 0, st>>>(m0, m_new, job->t, job->nw, job->seed,
                                                          job->sign.as<uint32_t>());
    });
  }
  CEN_CK(cudaStreamSynchronize(st));
  job->m = m1;
  job->members = members;
}

}  // namespace cen
