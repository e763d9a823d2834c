// Bit-parallel hyper-edge sampler for set betweenness (Sec. 3.1, Sec. 5 sampleHEs).
//
// A wave handles W = 64 G samples ("slots").  Each slot b draws its pair
// (s_b, t_b); all W searches then advance together, one BFS level per step,
// with every per-vertex set stored as G 64-bit words (bit b%64 of word b/64):
//   1. discovery: lev[L][v] = slots whose BFS reaches v at distance exactly L.
//      After level L+1 is built, slot b stops when t_b is in it (d = L+1), or
//      when it is empty (t_b unreachable: Sec. 5 returns the empty set).
//   2. cone: walking levels downwards, lev[L] is cut to the nodes on some
//      shortest s_b -> t_b path: t_b on level d, then the in-neighbours on level
//      L of cone nodes on level L+1.
//   3. path counts sigma_b[v] (number of shortest s_b -> v paths) on the cone
//      only, pulled from cone in-neighbours one level lower; every
//      predecessor of a cone node is itself a cone node, so these equal the
//      counts of a full BFS, and they are all the backward walk reads.
//   4. backward walk from t_b: at v on level L draw r uniform below sigma_v
//      (Philox purpose 2 + (d - L)), scan v's in-neighbours in ascending id,
//      add sigma of those on level L-1, take the first whose running sum
//      exceeds r.  The interior nodes are written to the hyper-edge in s->t
//      order.  A slot whose sigma_t reaches 2^64 is re-run with 128-bit counts.
//
// Rows longer than kHeavyRow arcs are handled a second time by *_heavy
// kernels, one warp per kChunk-arc chunk, merging with atomics; the light
// kernels skip them.  Lane layout for per-vertex work: g = lane % G (word),
// a = lane / G (one of A = 32/G arcs handled side by side).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>

#include "job.cuh"

namespace cen {

struct Ctl {
  unsigned long long active[32];  // slots still searching
  unsigned long long alive[32];   // slots whose newest level is non-empty
  unsigned long long farcs;       // out-arcs of the newest level (push/pull choice)
  long long total;                // members appended by this wave
  unsigned long long arcs;        // cone arcs logged by the cone pass
  int nflag;                      // slots flagged for 128-bit counts
  int err;                        // CEN_* code from device
  int flagged[2048];
};
constexpr int kMaxG = 32;
constexpr int kMaxW = 64 * kMaxG;
constexpr int kLevelBlocksPerSM = 8;  // grid of the per-level node sweeps, per SM
constexpr int kWalkUnroll = 8;          // 32-arc chunks in flight per walk step
constexpr size_t kArcLogCap = (size_t)1 << 24;  // cone arcs logged per wave (24 B each)

// Compact path-count store: only (node, slot) pairs on some cone get a count.
// any[v*G+g] holds every cone slot of node v (over all levels; a node is on
// at most one level per slot); base[v*G+g] is the exclusive prefix sum of
// their popcounts, so slot b of word g of v is entry base + rank of b.
struct SigIdx {
  const uint64_t *any;
  const int64_t *base;
  __device__ __forceinline__ int64_t operator()(int64_t vg, int b) const {
    return base[vg] + __popcll(any[vg] & ((1ull << b) - 1ull));
  }
};

// Block-level OR of per-word masks and sum of arc counts, then one global
// atomic per word and block.
__device__ __forceinline__ void block_publish(uint64_t alive, unsigned long long arcs, int G, Ctl *ctl) {
  __shared__ unsigned long long s_alive[32];
  __shared__ unsigned long long s_arcs;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) s_alive[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_arcs = 0;
  __syncthreads();
  for (int o = G; o < 32; o <<= 1) alive |= __shfl_xor_sync(0xffffffffu, alive, o);
  arcs = warp_sum(arcs);
  if (lane < G && alive) atomicOr(&s_alive[lane], (unsigned long long)alive);
  if (lane == 0 && arcs) atomicAdd(&s_arcs, arcs);
  __syncthreads();
  if ((int)threadIdx.x < G && s_alive[threadIdx.x]) atomicOr(&ctl->alive[threadIdx.x], s_alive[threadIdx.x]);
  if (threadIdx.x == 0 && s_arcs) atomicAdd(&ctl->farcs, s_arcs);
}

// --------------------------------------------------------------- init
__global__ void k_wave_init(int count, uint64_t jbase, const uint64_t *__restrict__ jlist, int32_t n, SampleKey key,
                            int G, int W, uint64_t *slot_j, int32_t *slot_s, int32_t *slot_t, int32_t *slot_d,
                            uint64_t *lev0, uint64_t *vis, const int64_t *__restrict__ off, Ctl *ctl) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < W; b += gridDim.x * blockDim.x) {
    if (b >= count) {
      slot_d[b] = -3;
      continue;
    }
    const uint64_t j = jlist ? jlist[b] : jbase + (uint64_t)b;
    // Sec. 5: s uniform over V; t uniform over V \ {s} (Sec. 3.1 pairs u != v)
    const int32_t s = (int32_t)uniform_below64(key.seed, key.id(j), kPurposeS, (uint64_t)n);
    const int32_t tt = (int32_t)uniform_below64(key.seed, key.id(j), kPurposeT, (uint64_t)(n - 1));
    const int32_t t = tt + (tt >= s);
    slot_j[b] = j;
    slot_s[b] = s;
    slot_t[b] = t;
    slot_d[b] = -2;
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    atomicOr((unsigned long long *)&lev0[(int64_t)s * G + g], bit);
    atomicOr((unsigned long long *)&vis[(int64_t)s * G + g], bit);
    atomicOr(&ctl->active[g], bit);
    atomicAdd(&ctl->farcs, (unsigned long long)(off[s + 1] - off[s]));
  }
}

// ------------------------------------------------------- target check
// Thread per slot, after level L was built: t_b on level L ends the search
// with d = L; an empty level L means t_b is unreachable (d = -1).
__global__ void k_tcheck(int W, int G, int L, const int32_t *__restrict__ slot_t, int32_t *slot_d,
                         int32_t *slot_kind, const uint64_t *__restrict__ lev, Ctl *ctl) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < W; b += gridDim.x * blockDim.x) {
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    if (!(ctl->active[g] & bit)) continue;
    if (lev[(int64_t)slot_t[b] * G + g] & bit) {
      slot_d[b] = L;
      slot_kind[b] = 0;
      atomicAnd(&ctl->active[g], ~bit);
    } else if (!(ctl->alive[g] & bit)) {
      slot_d[b] = -1;
      atomicAnd(&ctl->active[g], ~bit);
    }
  }
}

// Warp per active slot whose target has at most kHeavyRow in-arcs, before
// level L is expanded: an in-neighbour of t_b on level L gives d = L+1 and the
// slot is not expanded further (kind 1: its cone is seeded from those
// in-neighbours).  Slots with long-row targets are found after the expansion.
__global__ void k_tcheck_before(int W, int G, int L, const int32_t *__restrict__ slot_t, int32_t *slot_d,
                                int32_t *slot_kind, const int64_t *__restrict__ roff,
                                const int32_t *__restrict__ rcol, const uint64_t *__restrict__ lev, Ctl *ctl) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < W; b += nwarps) {
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    if (!(((volatile unsigned long long *)ctl->active)[g] & bit)) continue;
    const int32_t t = slot_t[b];
    const int64_t e0 = roff[t], e1 = roff[t + 1];
    if (e1 - e0 > kHeavyRow) continue;
    bool hit = false;
    for (int64_t i = e0 + lane; i < e1; i += 32) hit |= (lev[(int64_t)rcol[i] * G + g] & bit) != 0;
    if (__any_sync(0xffffffffu, hit) && lane == 0) {
      slot_d[b] = L + 1;
      slot_kind[b] = 1;
      atomicAnd(&ctl->active[g], ~bit);
    }
  }
}


// OR of the level-L words (word g) of the tails of arcs [e0, e1): 32 arc ids
// are loaded at once (coalesced) and handed out by shuffles, so the level
// rows of up to 8 arcs per lane are in flight together.  Lanes with
// need == 0 skip their loads.  With early exit, the scan stops after a
// 32-arc chunk once every bit of `need` is found (across the warp).
template <bool kEarlyExit>
__device__ __forceinline__ uint64_t or_tail_words(int64_t e0, int64_t e1, int G, int gshift, int g, int a, int A,
                                                  uint64_t need, const int32_t *__restrict__ rcol,
                                                  const uint64_t *__restrict__ lev, unsigned long long &scanned) {
  const int lane = threadIdx.x & 31;
  uint64_t acc = 0;
  for (int64_t base = e0; base < e1; base += 32) {
    const int32_t myv = base + lane < e1 ? rcol[base + lane] : -1;
    const int cnt = (int)min((int64_t)32, e1 - base);
    for (int r0 = 0; r0 < G; r0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int src = ((r0 + u) << (5 - gshift)) + a;  // arc (r0+u)*A + a of this chunk
        const int32_t v = __shfl_sync(0xffffffffu, myv, src & 31);
        if (r0 + u < G && src < cnt && need) acc |= lev[(int64_t)v * G + g];
      }
    }
    scanned += (unsigned long long)cnt;
    if (kEarlyExit) {
      uint64_t r = acc;
      for (int o = G; o < 32; o <<= 1) r |= __shfl_xor_sync(0xffffffffu, r, o);
      if (__all_sync(0xffffffffu, (r & need) == need)) break;
    }
  }
  (void)A;
  return acc;
}
// ----------------------------------------------------------- expansion
// Bottom-up: every node w with an unreached active slot ORs the level-L words
// of its in-neighbours (stopping once every unreached slot is found), and
// records the new bits: next level, reached set, level-not-empty masks.
__global__ void __launch_bounds__(256) k_expand_pull(const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                                                     const int64_t *__restrict__ off, int32_t n, int G, int gshift,
                                                     const uint64_t *__restrict__ lev, uint64_t *__restrict__ nxt,
                                                     uint64_t *__restrict__ vis, Ctl *ctl,
                                                     unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0, verts = 0, opened = 0, arcs = 0;
  uint64_t alive = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nwarps) {
    ++verts;
    const uint64_t vw = vis[w * G + g];
    const uint64_t unv = act & ~vw;
    if (!__any_sync(0xffffffffu, unv != 0)) {
      if (a == 0) nxt[w * G + g] = 0;
      continue;
    }
    const int64_t e0 = roff[w], e1 = roff[w + 1];
    if (e1 - e0 > kHeavyRow) {  // long rows: k_expand_pull_heavy ORs their chunks in
      if (a == 0) nxt[w * G + g] = 0;
      continue;
    }
    ++opened;
    uint64_t acc = or_tail_words<true>(e0, e1, G, gshift, g, a, A, unv, rcol, lev, scanned);
    for (int o = G; o < 32; o <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    {
      const uint64_t nb = acc & unv;
      if (a == 0) {
        nxt[w * G + g] = nb;
        if (nb) vis[w * G + g] = vw | nb;
      }
      alive |= nb;
      if (__any_sync(0xffffffffu, nb != 0) && lane == 0) arcs += (unsigned long long)(off[w + 1] - off[w]);
    }
  }
  block_publish(alive, arcs, G, ctl);
  // algorithmic bytes: every node reads its reached word and writes its next
  // word (16 G); an opened node reads its offsets (16) and, per scanned
  // in-arc, the arc (4) and the tail's level words (8 G)
  if (lane == 0 && verts)
    atomicAdd(units, verts * 16ull * G + opened * 16ull + scanned * (4ull + 8ull * G));
}

// Bottom-up over the chunks of long rows: OR of the chunk's in-neighbour level
// words, merged into the node's next word and reached set.  Chunks of one
// node may see each other's new bits in its reached word; the union of what
// they add is still exactly the node's new bits.
__global__ void __launch_bounds__(256) k_expand_pull_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                           const int64_t *__restrict__ cbeg,
                                                           const int64_t *__restrict__ roff,
                                                           const int32_t *__restrict__ rcol, int G, int gshift,
                                                           const uint64_t *__restrict__ lev, uint64_t *nxt,
                                                           uint64_t *vis, Ctl *ctl, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0, arcs = 0;
  uint64_t alive = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int32_t w = cw[q];
    const uint64_t unv = act & ~*(volatile uint64_t *)&vis[(int64_t)w * G + g];
    if (lane == 0) bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, unv != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, roff[w + 1]);
    unsigned long long sc = 0;
    uint64_t acc = or_tail_words<true>(e0, e1, G, gshift, g, a, A, unv, rcol, lev, sc);
    for (int o = G; o < 32; o <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    const uint64_t nb = acc & unv;
    uint64_t fresh = 0;
    if (a == 0 && nb) {
      const uint64_t old = atomicOr((unsigned long long *)&nxt[(int64_t)w * G + g], (unsigned long long)nb);
      fresh = nb & ~old;
      if (fresh) atomicOr((unsigned long long *)&vis[(int64_t)w * G + g], (unsigned long long)fresh);
    }
    alive |= fresh;
    if (__any_sync(0xffffffffu, fresh != 0) && lane == 0) arcs += (unsigned long long)(e1 - e0);
    if (lane == 0) bytes += 16ull + sc * (4ull + 8ull * G) + 16ull * G;
  }
  block_publish(alive, arcs, G, ctl);
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// Top-down: every node v on level L ORs its active level words into the
// next-level words of its out-neighbours (next must start zeroed).
__global__ void __launch_bounds__(256) k_expand_push(const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                     int32_t n, int G, int gshift, const uint64_t *__restrict__ lev,
                                                     uint64_t *nxt, const Ctl *__restrict__ ctl,
                                                     unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift, A = 32 >> gshift;
  const uint64_t act = ctl->active[g];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
    const uint64_t f = lev[v * G + g] & act;
    if (lane == 0) bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, f != 0)) continue;
    const int64_t e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 > kHeavyRow) continue;  // long rows: k_expand_push_heavy
    for (int64_t base = e0; base < e1; base += (int64_t)A * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = base + (int64_t)u * A + a;
        if (i < e1 && f) atomicOr((unsigned long long *)&nxt[(int64_t)col[i] * G + g], (unsigned long long)f);
      }
    }
    // bytes: offsets of v; per out-arc the arc (4) and an 8-byte
    // read-modify-write per non-empty word
    const int nzw = __popc(__ballot_sync(0xffffffffu, f != 0 && a == 0));
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

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
    if (lane == 0) bytes += 8ull * G;
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
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 16ull * nzw);
  }
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// After a push: keep only newly reached active slots, mark them reached and
// publish the level masks and out-arc count.
__global__ void __launch_bounds__(256) k_level_finalize(int32_t n, int G, int gshift, uint64_t *__restrict__ nxt,
                                                        uint64_t *__restrict__ vis, const int64_t *__restrict__ off,
                                                        Ctl *ctl, unsigned long long *units) {
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
      const uint64_t x = nxt[idx];
      if (x) {
        const uint64_t v = vis[idx];
        nb = x & ~v & act;
        nxt[idx] = nb;
        if (nb) vis[idx] = v | nb;
      }
    }
    alive |= nb;
    uint64_t any = nb;
    for (int o = 1; o < G; o <<= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
    if (g == 0 && idx < words && any) {
      const int64_t w = idx >> gshift;
      arcs += (unsigned long long)(off[w + 1] - off[w]);
    }
  }
  block_publish(alive, arcs, G, ctl);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(units, (unsigned long long)words * 16ull);
}

// ------------------------------------------------------ offsets + store
// One block: per-sample s, t, d of the wave, wave-local member offsets
// woff[b] (exclusive prefix of max(d-1, 0)), the wave's member total and the
// running max |h|.
__global__ void __launch_bounds__(1024) k_wave_lengths(int count, uint64_t jbase, const uint64_t *__restrict__ jlist,
                                                       const int32_t *slot_s, const int32_t *slot_t,
                                                       const int32_t *slot_d, int64_t *woff, int32_t *ps, int32_t *pt,
                                                       int32_t *pd, int *bmax, Ctl *ctl) {
  __shared__ long long wsum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int mymax = 0;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int b = c0 + threadIdx.x;
    int len = 0;
    if (b < count) {
      const int d = slot_d[b];
      len = d >= 2 ? d - 1 : 0;
      const uint64_t j = jlist ? jlist[b] : jbase + b;
      ps[j] = slot_s[b];
      pt[j] = slot_t[b];
      pd[j] = d;
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
    if (b < count) woff[b] = incl - len;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  for (int o = 16; o; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
  if ((threadIdx.x & 31) == 0 && mymax) atomicMax(bmax, mymax);
  if (threadIdx.x == 0) ctl->total = carry;
}

// Member counts of samples j0 .. j0+count-1 from their third field: set
// betweenness max(d - 1, 0) (the interior of a d-arc path), kappa-path the
// steps taken, triangle 3.
__global__ void k_lengths_of(const int32_t *__restrict__ pd, uint64_t j0, uint64_t count, int space, int32_t *lens) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const int d = pd[j0 + i];
    lens[i] = space == CEN_SPACE_KPATH ? d : space == CEN_SPACE_TRIANGLE ? 3 : (d >= 2 ? d - 1 : 0);
  }
}

// Warp per new sample: lens[i] members from src[i * stride] to the store.
__global__ void k_gather_strided(uint64_t count, uint64_t j0, int stride, const int32_t *__restrict__ lens,
                                 const int64_t *__restrict__ hoff, const int32_t *__restrict__ src, int32_t *hmem) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nwarps) {
    const int64_t h = hoff[j0 + i];
    for (int q = lane; q < lens[i]; q += 32) hmem[h + q] = src[i * (uint64_t)stride + q];
  }
}

// hoff[j0 + i] = hoff[j0] + ex[i] for i = 1 .. count.
__global__ void k_hoff_add(int64_t *hoff, uint64_t j0, uint64_t count, const int64_t *__restrict__ ex) {
  const int64_t base = hoff[j0];
  for (uint64_t i = 1 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= count;
       i += (uint64_t)gridDim.x * blockDim.x)
    hoff[j0 + i] = base + ex[i];
}

// aoff[jlist[b] - j0] = base + woff[b] for the slots of a wave whose members
// went to the arena at base (slots with d < 2 have none).
__global__ void k_set_aoff(int count, const uint64_t *__restrict__ jlist, uint64_t j0, const int64_t *__restrict__ woff,
                           const int32_t *__restrict__ slot_d, int64_t base, int64_t *aoff) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x)
    aoff[jlist[b] - j0] = slot_d[b] >= 2 ? base + woff[b] : -1;
}

// Warp per new sample: its members move from the arena (at aoff) to the store.
__global__ void k_gather_arena(uint64_t count, uint64_t j0, const int64_t *__restrict__ aoff,
                               const int32_t *__restrict__ pd, const int64_t *__restrict__ hoff,
                               const int32_t *__restrict__ arena, int32_t *hmem) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nwarps) {
    const int64_t a = aoff[i];
    const int d = pd[j0 + i];
    if (a < 0 || d < 2) continue;
    const int64_t h = hoff[j0 + i];
    for (int q = lane; q < d - 1; q += 32) hmem[h + q] = arena[a + q];
  }
}

// ------------------------------------------------------------------ cone
// The cone pass also records the cone's arcs: (w on level L, x on level L+1,
// word g, slots f) meaning sigma_b[x] += sigma_b[w] for every b in f.  The
// path-count pass then only visits these arcs.
struct ConeArc {
  int32_t w, x;
  int32_t g, pad;
  uint64_t f;
};
struct ArcLog {
  ConeArc *arcs;
  unsigned long long *count;  // total appended (may exceed cap: then the log is unusable)
  unsigned long long cap;
};

// Thread per kind-0 slot with d == L >= 2: t_b is the cone on its own level.
__global__ void k_cone_seed(int W, int G, int L, const int32_t *__restrict__ slot_t, const int32_t *__restrict__ slot_d,
                            const int32_t *__restrict__ slot_kind, uint64_t *cone, uint64_t *any) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < W; b += gridDim.x * blockDim.x) {
    if (slot_d[b] != L || L < 2 || slot_kind[b] != 0) continue;
    const int64_t tg = (int64_t)slot_t[b] * G + (b >> 6);
    atomicOr((unsigned long long *)&cone[tg], 1ull << (b & 63));
    atomicOr((unsigned long long *)&any[tg], 1ull << (b & 63));
  }
}

// Warp per kind-1 slot with d - 1 == L >= 1: t_b gets a count slot, and its
// in-neighbours on level L seed the cone, each arc logged.
__global__ void k_cone_seed_pred(int W, int G, int L, const int32_t *__restrict__ slot_t,
                                 const int32_t *__restrict__ slot_d, const int32_t *__restrict__ slot_kind,
                                 const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                                 const uint64_t *__restrict__ lev, uint64_t *cone, uint64_t *any, ArcLog log) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < W; b += nwarps) {
    if (slot_d[b] - 1 != L || slot_d[b] < 2 || slot_kind[b] != 1) continue;
    const int g = b >> 6;
    const unsigned long long bit = 1ull << (b & 63);
    const int32_t t = slot_t[b];
    if (lane == 0) atomicOr((unsigned long long *)&any[(int64_t)t * G + g], bit);
    const int64_t e0 = roff[t], e1 = roff[t + 1];
    for (int64_t base = e0; base < e1; base += 32) {
      const int64_t i = base + lane;
      int32_t w = -1;
      bool hit = false;
      if (i < e1) {
        w = rcol[i];
        hit = (lev[(int64_t)w * G + g] & bit) != 0;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (!m) continue;
      unsigned long long pos = 0;
      if (lane == __ffs(m) - 1) pos = atomicAdd(log.count, (unsigned long long)__popc(m));
      pos = __shfl_sync(0xffffffffu, pos, __ffs(m) - 1) + __popc(m & ((1u << lane) - 1u));
      if (hit) {
        atomicOr((unsigned long long *)&cone[(int64_t)w * G + g], bit);
        atomicOr((unsigned long long *)&any[(int64_t)w * G + g], bit);
        if (pos < log.cap) log.arcs[pos] = ConeArc{w, t, g, 0, (uint64_t)bit};
      }
    }
  }
}

// Level 1 of the cone: the only predecessor is s_b (count 1), so every cone
// node on level 1 has count 1 and nothing needs logging.
template <class T>
__global__ void k_cone_level1(int64_t words, const uint64_t *__restrict__ lev1, SigIdx ix, T *sig) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = lev1[i];
    if (!c) continue;
    for (uint64_t z = c; z; z &= z - 1) sig[ix(i, __ffsll((long long)z) - 1)] = (T)1;
  }
}

// Popcount of every cone word (input of the compact index scan).
__global__ void k_popc_words(int64_t words, const uint64_t *__restrict__ any, int32_t *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = __popcll(any[i]);
}

// Arc records are staged per warp in shared memory and appended to the log
// in batches (one global atomic per batch).
constexpr int kWarpArcBuf = 64;
struct WarpArcBuf {
  ConeArc rec[kWarpArcBuf];
  int n;
};

__device__ __forceinline__ void arcbuf_flush(WarpArcBuf &B, const ArcLog &log) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const int nrec = B.n;
  if (nrec == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(log.count, (unsigned long long)nrec);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int k = lane; k < nrec; k += 32)
    if (base + k < log.cap) log.arcs[base + k] = B.rec[k];
  __syncwarp();
  if (lane == 0) B.n = 0;
  __syncwarp();
}

__device__ __forceinline__ void arcbuf_put(WarpArcBuf &B, const ArcLog &log, bool have, const ConeArc &r) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, have);
  if (!m) return;
  if (B.n + __popc(m) > kWarpArcBuf) arcbuf_flush(B, log);
  const int pos = B.n + __popc(m & ((1u << lane) - 1u));
  if (have) B.rec[pos] = r;
  __syncwarp();
  if (lane == 0) B.n += __popc(m);
  __syncwarp();
}

// Cone slots c of node x on level L+1 mark x's in-neighbours that are on
// level L for those slots (read first, then one atomic OR if any), and log
// each such arc.  Arc ids are loaded 32 at a time and shuffled out.
__device__ __forceinline__ unsigned long long cone_arcs(int64_t e0, int64_t e1, int G, int gshift, int g, int a,
                                                        uint64_t c, int32_t x, const int32_t *__restrict__ rcol,
                                                        const uint64_t *__restrict__ lev, uint64_t *cone,
                                                        uint64_t *any, WarpArcBuf &B, const ArcLog &log) {
  const int lane = threadIdx.x & 31;
  unsigned long long hits = 0;
  for (int64_t base = e0; base < e1; base += 32) {
    const int32_t myv = base + lane < e1 ? rcol[base + lane] : -1;
    const int cnt = (int)min((int64_t)32, e1 - base);
    for (int r0 = 0; r0 < G; r0 += 4) {
      int32_t w[4];
      uint64_t f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int src = ((r0 + u) << (5 - gshift)) + a;
        w[u] = __shfl_sync(0xffffffffu, myv, src & 31);
        f[u] = 0;
        if (r0 + u < G && src < cnt && c) f[u] = lev[(int64_t)w[u] * G + g] & c;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (f[u]) {
          atomicOr((unsigned long long *)&cone[(int64_t)w[u] * G + g], (unsigned long long)f[u]);
          atomicOr((unsigned long long *)&any[(int64_t)w[u] * G + g], (unsigned long long)f[u]);
          ++hits;
        }
        arcbuf_put(B, log, f[u] != 0, ConeArc{w[u], x, g, 0, f[u]});
      }
    }
  }
  return hits;
}

// Warp per node x on level L+1 with cone slots c: mark and log its cone
// in-arcs (long rows: k_cone_push_heavy).
__global__ void __launch_bounds__(256) k_cone_push(int32_t n, int G, int gshift, const int64_t *__restrict__ roff,
                                                   const int32_t *__restrict__ rcol, const uint64_t *__restrict__ up,
                                                   const uint64_t *__restrict__ lev, uint64_t *cone, uint64_t *any,
                                                   ArcLog log, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift;
  __shared__ WarpArcBuf s_buf[8];
  WarpArcBuf &B = s_buf[threadIdx.x >> 5];
  if (lane == 0) B.n = 0;
  __syncwarp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
    const uint64_t c = up[x * G + g];
    if (lane == 0) bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    const int64_t e0 = roff[x], e1 = roff[x + 1];
    if (e1 - e0 > kHeavyRow) continue;
    const unsigned long long hits = cone_arcs(e0, e1, G, gshift, g, a, c, (int32_t)x, rcol, lev, cone, any, B, log);
    const int nzw = __popc(__ballot_sync(0xffffffffu, c != 0 && a == 0));
    bytes += 56ull * hits;
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 8ull * nzw);
  }
  arcbuf_flush(B, log);
  // bytes: every node's cone words (8 G); per non-empty node its offsets and,
  // per in-arc, the arc (4) and the level word of each non-empty cone word
  // (8); per hit two 16-byte atomic read-modify-writes and a 24-byte record
  bytes = warp_sum(bytes);
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

__global__ void __launch_bounds__(256) k_cone_push_heavy(int64_t nchunks, const int32_t *__restrict__ cw,
                                                         const int64_t *__restrict__ cbeg,
                                                         const int64_t *__restrict__ roff,
                                                         const int32_t *__restrict__ rcol, int G, int gshift,
                                                         const uint64_t *__restrict__ up,
                                                         const uint64_t *__restrict__ lev, uint64_t *cone,
                                                         uint64_t *any, ArcLog log, unsigned long long *units) {
  const int lane = threadIdx.x & 31, g = lane & (G - 1), a = lane >> gshift;
  __shared__ WarpArcBuf s_buf[8];
  WarpArcBuf &B = s_buf[threadIdx.x >> 5];
  if (lane == 0) B.n = 0;
  __syncwarp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchunks; q += nwarps) {
    const int32_t x = cw[q];
    const uint64_t c = up[(int64_t)x * G + g];
    if (lane == 0) bytes += 8ull * G;
    if (!__any_sync(0xffffffffu, c != 0)) continue;
    const int64_t e0 = cbeg[q], e1 = min(e0 + (int64_t)kChunk, roff[x + 1]);
    const unsigned long long hits = cone_arcs(e0, e1, G, gshift, g, a, c, x, rcol, lev, cone, any, B, log);
    const int nzw = __popc(__ballot_sync(0xffffffffu, c != 0 && a == 0));
    bytes += 56ull * hits;
    if (lane == 0) bytes += 16ull + (uint64_t)(e1 - e0) * (4ull + 8ull * nzw);
  }
  arcbuf_flush(B, log);
  bytes = warp_sum(bytes);
  if (lane == 0 && bytes) atomicAdd(units, bytes);
}

// Path counts over the logged cone arcs of one level: thread per arc (w, x,
// g, f): sigma_b[x] += sigma_b[w] for each slot b in f, with 64-bit atomics;
// a wrap-around (true sum >= 2^64) or an overflowed sigma_b[w] flags slot b
// of x.  The arcs of a level are read from [range[0], range[1]).
__global__ void __launch_bounds__(256) k_sigma_arcs64(const ConeArc *__restrict__ arcs,
                                                      const unsigned long long *__restrict__ range, int G,
                                                      SigIdx ix, uint64_t *__restrict__ sig,
                                                      uint64_t *__restrict__ ovf, unsigned long long *units) {
  const unsigned long long r0 = range[0], r1 = range[1];
  unsigned long long bytes = 0;
  for (unsigned long long i = r0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const ConeArc e = arcs[i];
    const int64_t wg = (int64_t)e.w * G + e.g, xg = (int64_t)e.x * G + e.g;
    uint64_t f = e.f;
    uint64_t of = ovf[wg] & f;
    bytes += 64ull;
    while (f) {
      const int b = __ffsll((long long)f) - 1;
      f &= f - 1;
      const unsigned long long v = sig[ix(wg, b)];
      const unsigned long long old = atomicAdd((unsigned long long *)&sig[ix(xg, b)], v);
      if (old + v < old) of |= 1ull << b;
      bytes += 24ull;
    }
    if (of) atomicOr((unsigned long long *)&ovf[xg], (unsigned long long)of);
  }
  // bytes: per arc the 24-byte record, the tail's overflow word and the cone
  // words and bases of both ends; per slot the tail's count and a 16-byte
  // atomic read-modify-write
  bytes = warp_sum(bytes);
  if ((threadIdx.x & 31) == 0 && bytes) atomicAdd(units, bytes);
}

// 128-bit variant for a re-run wave: the 128-bit add is two 64-bit atomics
// (low word, then high word plus carry); all terms are non-negative, so the
// high word wraps exactly when the true sum reaches 2^128.
__global__ void __launch_bounds__(256) k_sigma_arcs128(const ConeArc *__restrict__ arcs,
                                                       const unsigned long long *__restrict__ range, int G, SigIdx ix,
                                                       u128 *__restrict__ sig, uint64_t *__restrict__ ovf) {
  const unsigned long long r0 = range[0], r1 = range[1];
  for (unsigned long long i = r0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const ConeArc e = arcs[i];
    const int64_t wg = (int64_t)e.w * G + e.g, xg = (int64_t)e.x * G + e.g;
    uint64_t f = e.f;
    uint64_t of = ovf[wg] & f;
    while (f) {
      const int b = __ffsll((long long)f) - 1;
      f &= f - 1;
      const u128 v = sig[ix(wg, b)];
      unsigned long long *dst = (unsigned long long *)&sig[ix(xg, b)];
      const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
      const unsigned long long olo = atomicAdd(dst, lo);
      const unsigned long long add_hi = hi + (olo + lo < olo ? 1ull : 0ull);
      if (add_hi < hi) of |= 1ull << b;  // hi + carry wrapped
      if (add_hi) {
        const unsigned long long ohi = atomicAdd(dst + 1, add_hi);
        if (ohi + add_hi < ohi) of |= 1ull << b;
      }
    }
    if (of) atomicOr((unsigned long long *)&ovf[xg], (unsigned long long)of);
  }
}

// ----------------------------------------------------------------- walk
__device__ __forceinline__ uint64_t shfl_up_T(uint64_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ u128 shfl_up_T(u128 v, int o) {
  const uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)v, o);
  const uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(v >> 64), o);
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

// Warp per slot (see the file header, step 4).  Arcs are scanned 256 at a time
// (8 chunks of 32 loaded together).  T = uint64_t: a slot whose sigma_t
// overflowed is appended to ctl->flagged.  T = u128: it sets ctl->err.
// Members of slot b go to out[slot_off[b] ...] when slot_off is given (a
// wave-local buffer), else to out[hoff[j] ...] (the job's store).
template <class T>
__global__ void k_walk(int count, int G, SigIdx ix, const uint64_t *__restrict__ slot_j,
                       const int32_t *__restrict__ slot_t, const int32_t *__restrict__ slot_d,
                       const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol,
                       const uint64_t *const *__restrict__ levs, const T *__restrict__ sig,
                       const uint64_t *__restrict__ ovf, const int64_t *__restrict__ slot_off,
                       const int64_t *__restrict__ hoff, int32_t *out, SampleKey key, Ctl *ctl,
                       unsigned long long *units) {
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
    if (ovf[(int64_t)v * G + g] & bit) {
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
    T sv = sig[ix((int64_t)v * G + g, b & 63)];
    const int64_t hbase = slot_off ? slot_off[b] : hoff[j];
    uint32_t step = 0;
    int L = d;
    while (L >= 2) {
      const T r = draw_below(key.seed, key.id(j), kPurposeWalk0 + step, sv);
      const uint64_t *lp = levs[L - 1];
      T cum = 0;
      int32_t pick = -1;
      const int64_t e0 = roff[v], e1 = roff[v + 1];
      for (int64_t base = e0; base < e1 && pick < 0; base += 32 * kWalkUnroll) {
        int32_t x[kWalkUnroll];
        T val[kWalkUnroll];
#pragma unroll
        for (int u = 0; u < kWalkUnroll; ++u) {
          const int64_t i = base + 32 * u + lane;
          x[u] = i < e1 ? rcol[i] : -1;
        }
        uint64_t hit_bits = 0;
#pragma unroll
        for (int u = 0; u < kWalkUnroll; ++u)
          if (x[u] >= 0 && (lp[(int64_t)x[u] * G + g] & bit)) hit_bits |= 1ull << u;
#pragma unroll
        for (int u = 0; u < kWalkUnroll; ++u)
          val[u] = ((hit_bits >> u) & 1) ? sig[ix((int64_t)x[u] * G + g, b & 63)] : (T)0;
#pragma unroll
        for (int u = 0; u < kWalkUnroll; ++u) {
          if (pick >= 0) break;
          T pre = val[u];
          for (int o = 1; o < 32; o <<= 1) {
            const T y = shfl_up_T(pre, o);
            if (lane >= o) pre += y;
          }
          const unsigned hit = __ballot_sync(0xffffffffu, (cum + pre) > r);
          if (hit) {
            pick = __shfl_sync(0xffffffffu, x[u], __ffs(hit) - 1);
          } else {
            cum += shfl_T(pre, 31);
          }
        }
        scanned += 32 * kWalkUnroll;
      }
      if (pick < 0) {  // cannot happen with consistent counts
        if (lane == 0) atomicExch(&ctl->err, CEN_EINVAL);
        break;
      }
      if (lane == 0) out[hbase + (L - 2)] = pick;
      sv = sig[ix((int64_t)pick * G + g, b & 63)];
      v = pick;
      --L;
      ++step;
    }
  }
  if (lane == 0 && scanned) atomicAdd(units, scanned * 12ull);
}

// --------------------------------------------------------------- sign words
// Alg. 1 "sampleRadeVars", extended by the new columns j: word w of sample j
// is word w%4 of Philox block (j, SIGN, w/4); bits >= t are cleared.
__global__ void k_sign(uint64_t j0, uint64_t count, int t, int nw, SampleKey key, uint32_t *sign) {
  const int nblk = (nw + 3) / 4;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count * nblk;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = j0 + idx / nblk;
    const int blk = (int)(idx % nblk);
    const uint4 x = philox_block(key.seed, key.id(j), kPurposeSign, (uint32_t)blk);
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

void *ws_staging(WaveWS &ws, size_t bytes) {
  if (bytes > ws.host_bytes) {
    if (ws.host) cudaFreeHost(ws.host);  // synchronizes: no copy may still use it
    ws.host = nullptr;
    ws.host_bytes = 0;
    size_t cap = 0;
    ws.host = pinned_take(bytes, &cap);
    ws.host_bytes = cap;
  }
  return ws.host;
}

// One wave pipeline on one stream with its own workspace.
struct Sampler {
  cen_job *job;
  WaveWS *wsp;
  const cen_graph *g;
  cudaStream_t st;
  Stats *S;
  int32_t n;
  int G = 1, gshift = 0, W = 64;
  Ctl *ctl = nullptr;
  Ctl *hctl = nullptr;  // pinned mirror (header part)
  uint64_t *slot_j = nullptr;
  int32_t *slot_s = nullptr, *slot_t = nullptr, *slot_d = nullptr, *slot_kind = nullptr;

  WaveWS &ws() { return *wsp; }
  unsigned long long *units(int cls) { return (unsigned long long *)(job->stats.d_units + cls); }

  void setup(int Gwant) {
    G = Gwant;
    gshift = 0;
    while ((1 << gshift) < G) ++gshift;
    W = 64 * G;
    WaveWS &w = ws();
    const size_t words = (size_t)n * G;
    w.vis.ensure(words * 8, st);
    w.ovf.ensure(words * 8, st);
    w.any.ensure(words * 8, st);
    w.base.ensure((words + 1) * 8, st);
    w.cnt.ensure(words * 4, st);
    if (w.G != G || !w.tmp.p) {  // the cone scratch is kept zero between waves of one width
      w.tmp.ensure(words * 8, st);
      CEN_CK(cudaMemsetAsync(w.tmp.p, 0, words * 8, st));
    }
    w.G = G;
    w.ctl.ensure(sizeof(Ctl), st);
    w.slots.ensure((size_t)kMaxW * (8 + 4 * 4), st);
    w.woff.ensure((size_t)kMaxW * 8, st);
    if (w.arc_cap == 0)  // grows (and the wave is redone) when a wave logs more arcs
      w.arc_cap = std::min<size_t>(kArcLogCap, std::max<size_t>((size_t)1 << 16, 2 * words));
    w.arcs.ensure(sizeof(ConeArc) * w.arc_cap, st);
    ctl = w.ctl.as<Ctl>();
    slot_j = w.slots.as<uint64_t>();
    slot_s = (int32_t *)(slot_j + kMaxW);
    slot_t = slot_s + kMaxW;
    slot_d = slot_t + kMaxW;
    slot_kind = slot_d + kMaxW;
    hctl = (Ctl *)ws_staging(w, sizeof(Ctl));
  }

  uint64_t *level(int L) {
    WaveWS &w = ws();
    const size_t bytes = (size_t)n * G * 8;
    while ((int)w.lev.size() <= L) w.lev.emplace_back(new DevBuf());
    w.lev[L]->ensure(bytes, st);
    return w.lev[L]->as<uint64_t>();
  }

  void publish_levels(int Lmax) {
    WaveWS &w = ws();
    std::vector<uint64_t *> ptrs(Lmax + 1);
    for (int L = 0; L <= Lmax; ++L) ptrs[L] = w.lev[L]->as<uint64_t>();
    w.lev_ptrs.ensure(sizeof(uint64_t *) * (Lmax + 1), st);
    uint64_t **h = (uint64_t **)ws_staging(w, sizeof(uint64_t *) * (Lmax + 1) + sizeof(Ctl));
    memcpy(h, ptrs.data(), sizeof(uint64_t *) * (Lmax + 1));
    CEN_CK(cudaMemcpyAsync(w.lev_ptrs.p, h, sizeof(uint64_t *) * (Lmax + 1), cudaMemcpyHostToDevice, st));
    CEN_CK(cudaStreamSynchronize(st));
    hctl = (Ctl *)ws_staging(w, sizeof(Ctl));
  }

  void fetch_ctl_head() {
    CEN_CK(cudaMemcpyAsync(hctl, ctl, offsetof(Ctl, flagged), cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
  }

  bool any_active() const {
    for (int gg = 0; gg < G; ++gg)
      if (hctl->active[gg]) return true;
    return false;
  }

  // Discovery for slots [0, count): returns the highest level materialised.
  int discover(int count, uint64_t jbase, const uint64_t *jlist) {
    const size_t words = (size_t)n * G;
    uint64_t *vis = ws().vis.as<uint64_t>();
    CEN_CK(cudaMemsetAsync(vis, 0, words * 8, st));
    CEN_CK(cudaMemsetAsync(ws().ovf.p, 0, words * 8, st));
    CEN_CK(cudaMemsetAsync(ctl, 0, offsetof(Ctl, flagged), st));
    uint64_t *lev0 = level(0);
    CEN_CK(cudaMemsetAsync(lev0, 0, words * 8, st));
    const int64_t *off = g->off.as<int64_t>();
    const int32_t *col = g->col.as<int32_t>();
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    launch(S, K_PAIRS, st, [&] {
      k_wave_init<<<grid_for(W, 256), 256, 0, st>>>(count, jbase, jlist, n, job->key(), G, W, slot_j, slot_s, slot_t,
                                                    slot_d, lev0, vis, off, ctl);
    });
    fetch_ctl_head();
    int L = 0;
    while (any_active()) {
      uint64_t *cur = level(L);
      uint64_t *nxt = level(L + 1);
      launch(S, K_TCHECK, st, [&] {
        k_tcheck_before<<<grid_for((size_t)W * 32, 256), 256, 0, st>>>(W, G, L, slot_t, slot_d, slot_kind, roff,
                                                                       rcol, cur, ctl);
      });
      const bool push = (double)hctl->farcs * job->push_ratio < (double)g->nnz;
      CEN_CK(cudaMemsetAsync(&ctl->alive, 0, sizeof(ctl->alive) + sizeof(ctl->farcs), st));
      if (push) {
        CEN_CK(cudaMemsetAsync(nxt, 0, words * 8, st));
        launch(S, K_PUSH, st, [&] {
          k_expand_push<<<resident_grid((const void *)k_expand_push, 256), 256, 0, st>>>(off, col, n, G, gshift, cur,
                                                                                         nxt, ctl, units(K_PUSH));
        });
        const ChunkTable &oc = graph_out_chunks(g, st);
        if (oc.count)
          launch(S, K_PUSH, st, [&] {
            k_expand_push_heavy<<<grid_for((size_t)oc.count * 32, 256, sm_count() * 64), 256, 0, st>>>(
                oc.count, oc.rows(), oc.begins(), off, col, G, gshift, cur, nxt, ctl, units(K_PUSH));
          });
        launch(S, K_LEVEL_FIN, st, [&] {
          k_level_finalize<<<resident_grid((const void *)k_level_finalize, 256), 256, 0, st>>>(
              n, G, gshift, nxt, vis, off, ctl, units(K_LEVEL_FIN));
        });
      } else {
        launch(S, K_PULL, st, [&] {
          k_expand_pull<<<resident_grid((const void *)k_expand_pull, 256), 256, 0, st>>>(
              roff, rcol, off, n, G, gshift, cur, nxt, vis, ctl, units(K_PULL));
        });
        const ChunkTable &ic = graph_in_chunks(g, st);
        if (ic.count)
          launch(S, K_PULL, st, [&] {
            k_expand_pull_heavy<<<resident_grid((const void *)k_expand_pull_heavy, 256), 256, 0, st>>>(
                ic.count, ic.rows(), ic.begins(), roff, rcol, G, gshift, cur, nxt, vis, ctl, units(K_PULL));
          });
      }
      launch(S, K_TCHECK, st, [&] {
        k_tcheck<<<grid_for(W, 256), 256, 0, st>>>(W, G, L + 1, slot_t, slot_d, slot_kind, nxt, ctl);
      });
      fetch_ctl_head();
      ++L;
      CEN_REQUIRE(L <= n, CEN_ECUDA, "cen_sample: level loop exceeded n levels");
    }
    return L;
  }

  // Cut every level >= 1 to the cone (lev[L] and the zeroed scratch swap
  // roles), record every node's cone slots in `any` and log the cone arcs
  // above level 1; range[2U], range[2U+1] bound the arcs into level U.
  // Returns the number of logged arcs (the log is usable iff <= its capacity).
  unsigned long long cone(int Lmax) {
    const size_t words = (size_t)n * G;
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    WaveWS &w = ws();
    w.arc_range.ensure(sizeof(unsigned long long) * 2 * (size_t)(Lmax + 3), st);
    unsigned long long *range = w.arc_range.as<unsigned long long>();
    CEN_CK(cudaMemsetAsync(range, 0, sizeof(unsigned long long) * 2 * (size_t)(Lmax + 3), st));
    unsigned long long *count = &ctl->arcs;
    CEN_CK(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st));
    uint64_t *any = w.any.as<uint64_t>();
    CEN_CK(cudaMemsetAsync(any, 0, words * 8, st));
    const ArcLog log{w.arcs.as<ConeArc>(), count, (unsigned long long)w.arc_cap};
    const ChunkTable &ic = graph_in_chunks(g, st);
    for (int L = Lmax; L >= 1; --L) {
      uint64_t *lev = level(L);
      uint64_t *cone = w.tmp.as<uint64_t>();
      launch(S, K_CONE, st, [&] {
        k_cone_seed<<<grid_for(W, 256), 256, 0, st>>>(W, G, L, slot_t, slot_d, slot_kind, cone, any);
      });
      CEN_CK(cudaMemcpyAsync(range + 2 * (L + 1), count, 8, cudaMemcpyDeviceToDevice, st));
      if (L < Lmax) {
        const uint64_t *up = level(L + 1);
        launch(S, K_CONE, st, [&] {
          k_cone_push<<<resident_grid((const void *)k_cone_push, 256), 256, 0, st>>>(n, G, gshift, roff, rcol, up, lev,
                                                                                     cone, any, log, units(K_CONE));
        });
        if (ic.count)
          launch(S, K_CONE, st, [&] {
            k_cone_push_heavy<<<resident_grid((const void *)k_cone_push_heavy, 256), 256, 0, st>>>(
                ic.count, ic.rows(), ic.begins(), roff, rcol, G, gshift, up, lev, cone, any, log, units(K_CONE));
          });
      }
      launch(S, K_CONE, st, [&] {
        k_cone_seed_pred<<<grid_for((size_t)W * 32, 256), 256, 0, st>>>(W, G, L, slot_t, slot_d, slot_kind, roff, rcol,
                                                                         lev, cone, any, log);
      });
      CEN_CK(cudaMemcpyAsync(range + 2 * (L + 1) + 1, count, 8, cudaMemcpyDeviceToDevice, st));
      w.lev[L]->swap(w.tmp);  // the cone becomes level L
      CEN_CK(cudaMemsetAsync(w.tmp.p, 0, words * 8, st));
    }
    fetch_ctl_head();
    return hctl->arcs;
  }

  // Discovery + cone, redone with a larger arc log when a wave overflows it.
  int discover_and_cone(int count, uint64_t jbase, const uint64_t *jlist, int64_t *wave_total) {
    for (;;) {
      const int Lmax = discover(count, jbase, jlist);
      if (wave_total) {
        launch(S, K_APPEND, st, [&] {
          k_wave_lengths<<<1, 1024, 0, st>>>(count, jbase, jlist, slot_s, slot_t, slot_d, ws().woff.as<int64_t>(),
                                             job->ps.as<int32_t>(), job->pt.as<int32_t>(), job->pd.as<int32_t>(),
                                             job->bmax.as<int>(), ctl);
        });
        fetch_ctl_head();
        *wave_total = hctl->total;
      }
      const unsigned long long narcs = cone(Lmax);
      if (narcs <= ws().arc_cap) return Lmax;
      ws().arc_cap = (size_t)(narcs + narcs / 4);
      ws().arcs.release();
      setup(G);
    }
  }

  // Compact count store for the cone pairs: bases by an exclusive scan of the
  // popcounts of `any`; counts zeroed, level 1 set to 1.  Returns the index.
  template <class T>
  SigIdx sigma_store(T **sig_out) {
    const size_t words = (size_t)n * G;
    WaveWS &w = ws();
    const uint64_t *any = w.any.as<uint64_t>();
    int64_t *base = w.base.as<int64_t>();
    launch(S, K_SIGMA, st, [&] {
      k_popc_words<<<grid_for(words, 256, sm_count() * kLevelBlocksPerSM), 256, 0, st>>>((int64_t)words, any, w.cnt.as<int32_t>());
    });
    counts_to_offsets(w.cnt.as<int32_t>(), base, words, w.scan_tmp, st, S);
    int64_t *h = (int64_t *)ws_staging(w, sizeof(Ctl) + 8);
    CEN_CK(cudaMemcpyAsync(h, base + words, 8, cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    const int64_t pairs = *h;
    hctl = (Ctl *)ws_staging(w, sizeof(Ctl));
    w.sigc.ensure(sizeof(T) * (size_t)(pairs + 1), st);
    CEN_CK(cudaMemsetAsync(w.sigc.p, 0, sizeof(T) * (size_t)(pairs + 1), st));
    const SigIdx ix{any, base};
    T *sig = w.sigc.as<T>();
    launch(S, K_SIGMA, st, [&] {
      k_cone_level1<T><<<grid_for(words, 256, sm_count() * kLevelBlocksPerSM), 256, 0, st>>>((int64_t)words, level(1), ix, sig);
    });
    *sig_out = sig;
    return ix;
  }

  // Path counts level by level over the logged arcs (levels 2 .. Lmax+1;
  // Lmax+1 holds only targets found before their last expansion), then the
  // walk, writing members to out (at slot_off[b], or at hoff[j] if null).
  template <class T>
  void sigma_and_walk(int count, int Lmax, const int64_t *slot_off, int32_t *out) {
    const int64_t *roff = g->in_off();
    const int32_t *rcol = g->in_col();
    uint64_t *ovf = ws().ovf.as<uint64_t>();
    const ConeArc *arcs = ws().arcs.as<ConeArc>();
    T *sig = nullptr;
    const SigIdx ix = sigma_store<T>(&sig);
    for (int L = 2; L <= Lmax + 1; ++L) {
      const unsigned long long *range = ws().arc_range.as<unsigned long long>() + 2 * L;
      launch(S, K_SIGMA, st, [&] {
        if constexpr (sizeof(T) == 8)
          k_sigma_arcs64<<<resident_grid((const void *)k_sigma_arcs64, 256), 256, 0, st>>>(
              arcs, range, G, ix, (uint64_t *)sig, ovf, units(K_SIGMA));
        else
          k_sigma_arcs128<<<resident_grid((const void *)k_sigma_arcs128, 256), 256, 0, st>>>(arcs, range, G, ix,
                                                                                             (u128 *)sig, ovf);
      });
    }
    publish_levels(Lmax);
    launch(S, K_WALK, st, [&] {
      k_walk<T><<<grid_for((size_t)count * 32, 256), 256, 0, st>>>(
          count, G, ix, slot_j, slot_t, slot_d, roff, rcol, ws().lev_ptrs.as<const uint64_t *>(), sig, ovf, slot_off,
          job->hoff.as<int64_t>(), out, job->key(), ctl, units(K_WALK));
    });
  }
};

// Wave width: up to gmax words, no wider than the samples left need, and with
// one level array ([n][G] words) within `budget` bytes.
int pick_G(uint64_t remaining, int32_t n, size_t budget, int gmax) {
  int G = 1;
  while (G < kMaxG && G < gmax && (uint64_t)64 * G < remaining) G <<= 1;
  while (G > 1 && (size_t)n * G * 8 > budget) G >>= 1;
  return G;
}

struct WaveOut {
  uint64_t j0 = 0;
  int count = 0, G = 0;
  int64_t total = 0;
  DevBuf mem;  // the wave's members, samples in order
  std::vector<uint64_t> flagged;
};

}  // namespace

namespace {

Sampler make_sampler(cen_job *job, WaveWS &w, cudaStream_t st) {
  Sampler sp;
  sp.job = job;
  sp.wsp = &w;
  sp.g = job->g;
  sp.st = st;
  sp.S = &job->stats;
  sp.n = job->g->n;
  return sp;
}

WaveWS &wave_ws0(cen_job *job) {
  if (job->wws.empty()) job->wws.emplace_back(new WaveWS());
  return *job->wws[0];
}

// Uploads ids to the workspace's jlist through its pinned staging.
void upload_jlist(WaveWS &w, const uint64_t *ids, int count, cudaStream_t st) {
  w.jlist.ensure(8 * (size_t)kMaxW, st);
  uint64_t *h = (uint64_t *)ws_staging(w, 8 * (size_t)kMaxW + sizeof(Ctl));
  memcpy(h, ids, 8 * (size_t)count);
  CEN_CK(cudaMemcpyAsync(w.jlist.p, h, 8 * (size_t)count, cudaMemcpyHostToDevice, st));
  CEN_CK(cudaStreamSynchronize(st));
}

// Members of the listed samples (offsets already in hoff) written in place
// by the bit-parallel sampler: 64-bit counts first, then 128-bit counts for
// the pairs whose count reached 2^64.
void rerun_in_place(cen_job *job, std::vector<uint64_t> ids) {
  if (ids.empty()) return;
  std::sort(ids.begin(), ids.end());
  cudaStream_t st = job->st;
  WaveWS &w0 = wave_ws0(job);
  Sampler sp = make_sampler(job, w0, st);
  std::vector<uint64_t> wide;
  for (size_t q0 = 0; q0 < ids.size();) {
    const int G = pick_G(ids.size() - q0, job->g->n, job->level_budget, job->max_wave_words);
    const int count = (int)std::min<size_t>((size_t)64 * G, ids.size() - q0);
    upload_jlist(w0, ids.data() + q0, count, st);
    sp.setup(G);
    const int Lmax = sp.discover_and_cone(count, 0, w0.jlist.as<uint64_t>(), nullptr);
    sp.sigma_and_walk<uint64_t>(count, Lmax, nullptr, job->hmem.as<int32_t>());
    CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent path counts in the backward walk");
    for (int f = 0; f < sp.hctl->nflag; ++f) wide.push_back(ids[q0 + sp.hctl->flagged[f]]);
    q0 += (size_t)count;
  }
  if (wide.empty()) return;
  std::sort(wide.begin(), wide.end());
  sp.setup(1);
  for (size_t q0 = 0; q0 < wide.size(); q0 += 64) {
    const int count = (int)std::min<size_t>(64, wide.size() - q0);
    upload_jlist(w0, wide.data() + q0, count, st);
    sp.hctl = (Ctl *)ws_staging(w0, sizeof(Ctl));
    const int Lmax = sp.discover_and_cone(count, 0, w0.jlist.as<uint64_t>(), nullptr);
    sp.sigma_and_walk<u128>(count, Lmax, nullptr, job->hmem.as<int32_t>());
    CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, offsetof(Ctl, flagged), cudaMemcpyDeviceToHost, st));
    CEN_CK(cudaStreamSynchronize(st));
    CEN_REQUIRE(sp.hctl->err != CEN_EOVERFLOW, CEN_EOVERFLOW, "cen_sample: a sampled pair has >= 2^128 shortest paths");
    CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent 128-bit path counts");
  }
}

// hoff of the new samples from their distances; returns their member total
// (known_total, when the caller has counted it, saves reading it back).
int64_t offsets_from_distances(cen_job *job, uint64_t m0, uint64_t m_new, int64_t known_total = -1) {
  cudaStream_t st = job->st;
  Stats *S = &job->stats;
  WaveWS &w0 = wave_ws0(job);
  w0.lens.ensure(4 * (size_t)m_new, st);
  w0.exoff.ensure(8 * ((size_t)m_new + 1), st);
  launch(S, K_APPEND, st, [&] {
    k_lengths_of<<<grid_for(m_new, 256), 256, 0, st>>>(job->pd.as<int32_t>(), m0, m_new, job->space,
                                                        w0.lens.as<int32_t>());
  });
  counts_to_offsets(w0.lens.as<int32_t>(), w0.exoff.as<int64_t>(), (size_t)m_new, w0.scan_tmp, st, S);
  launch(S, K_APPEND, st, [&] {
    k_hoff_add<<<grid_for(m_new, 256), 256, 0, st>>>(job->hoff.as<int64_t>(), m0, m_new, w0.exoff.as<int64_t>());
  });
  if (known_total >= 0) return known_total;  // the caller counted the members already
  int64_t *h = (int64_t *)host_staging(job, 8);
  CEN_CK(cudaMemcpyAsync(h, w0.exoff.as<int64_t>() + m_new, 8, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  return *h;
}

// Workspace for as many resident CTAs as the byte budget allows (at least
// one).  The small tables are sized so that all of them take about kTableL2
// bytes (they stay in L2), unless a size was set.
constexpr size_t kTableL2 = (size_t)80 << 20;
// Measured: warp searches are 1.3-1.75x faster than whole-CTA searches on BA graphs and small
// R-MATs (E[d^2]/E[d] from 19 to 126) and slower on R-MAT 16, 18 and directed 22 (684 to 2,244).
constexpr double kWarpBranching = 256.0;

void bidir_setup(cen_job *job, uint64_t m_new) {
  const int32_t n = job->g->n;
  cudaStream_t st = job->st;
  const int64_t QC = std::max<int64_t>(16, std::min<int64_t>(n, job->bidir_queue));
  int64_t H2 = 1024;
  while (H2 < 4 * QC) H2 *= 2;
  // by default, warp searches only where frontiers grow slowly (E[d^2] / E[d], the mean degree at
  // the far end of an arc, at most kWarpBranching), and until a call hands too many on
  const bool warps = job->bidir_warps > 0 ||
                     (job->bidir_warps < 0 && !job->g->bidir_warps_off.load() &&
                      graph_branching(job->g, st) <= kWarpBranching);
  const int64_t WQ = warps ? bidir_warp_queue(QC) : 0;
  auto per_slot = [&](int64_t h1) {
    return 8 * (size_t)h1 + 16 * (size_t)H2 + 7 * 4 * (size_t)QC + (WQ ? bidir_warp_bytes_per_slot() : 0);
  };
  const size_t res = (size_t)bidir_resident_slots();
  int slots = (int)std::min<size_t>(res, std::max<size_t>(1, job->bidir_budget / per_slot(0)));
  int64_t H1 = 0;
  if (job->bidir_table < 0 && !job->g->bidir_table_off.load()) {
    H1 = 1024;
    while ((size_t)(2 * H1) * 8 * (size_t)slots <= kTableL2 && 2 * H1 < H2) H1 *= 2;
  } else if (job->bidir_table > 0) {
    H1 = std::min<int64_t>(job->bidir_table, H2 / 2);
  }
  if (H1) slots = (int)std::min<size_t>(res, std::max<size_t>(1, job->bidir_budget / per_slot(H1)));
  int dev = 0;
  CEN_CK(cudaGetDevice(&dev));
  BiWS *cur = job->bws.get();
  if (!(cur && cur->QC == QC && cur->H1 == H1 && cur->nslots == slots && cur->WQ == WQ && cur->dev == dev)) {
    if (cur && cur->nslots) {  // another shape: keep this one for later jobs, once idle
      CEN_CK(cudaStreamSynchronize(st));
      bidir_give(std::move(job->bws));
    }
    job->bws = bidir_take(dev, QC, H1, slots, WQ);
    if (!job->bws) job->bws.reset(new BiWS());
  }
  BiWS &wk = *job->bws;
  if (wk.nslots == 0) {
    keep_pool_memory();
    if (H1) wk.tab1.ensure_exact(8 * (size_t)H1 * slots, st);
    wk.tab2.ensure_exact(8 * (size_t)H2 * slots, st);
    wk.lists.ensure_exact(4 * 7 * (size_t)QC * slots, st);
    wk.sig.ensure_exact(8 * (size_t)H2 * slots, st);
    wk.epochs.ensure(8 * (size_t)slots, st);
    if (H1) CEN_CK(cudaMemsetAsync(wk.tab1.p, 0, 8 * (size_t)H1 * slots, st));
    CEN_CK(cudaMemsetAsync(wk.tab2.p, 0, 8 * (size_t)H2 * slots, st));
    CEN_CK(cudaMemsetAsync(wk.epochs.p, 0, 8 * (size_t)slots, st));
    if (WQ) {
      const size_t tb = bidir_warp_table_bytes_per_slot() * (size_t)slots;
      const size_t eb = bidir_warp_epoch_bytes_per_slot() * (size_t)slots;
      wk.tabw.ensure_exact(tb, st);
      wk.epw.ensure_exact(eb, st);
      CEN_CK(cudaMemsetAsync(wk.tabw.p, 0, tb, st));
      CEN_CK(cudaMemsetAsync(wk.epw.p, 0, eb, st));
    }
    wk.QC = QC;
    wk.WQ = WQ;
    wk.H1 = H1;
    wk.H2 = H2;
    wk.nslots = slots;
    wk.dev = dev;
  }
  for (DevBuf *b : {&wk.tab1, &wk.tab2, &wk.lists, &wk.sig, &wk.epochs, &wk.tabw, &wk.epw}) b->st = st;
  wk.ctl.ensure(sizeof(BiCtl), st);
  wk.big.ensure(8 * (size_t)m_new, st);
  wk.aoff.ensure(8 * (size_t)m_new, st);
  wk.dsearch.ensure(8 * (size_t)m_new, st);
  wk.dwalk.ensure(8 * (size_t)m_new, st);
}

// The control block of the last bidir_launch.
static BiCtl bidir_finish(cen_job *job) {
  BiWS &bw = *job->bws;
  cudaStream_t st = job->st;
  CEN_CK(cudaMemcpyAsync(host_staging(job, sizeof(BiCtl)), bw.ctl.p, sizeof(BiCtl), cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  const BiCtl h = *(const BiCtl *)host_staging(job, sizeof(BiCtl));
  CEN_REQUIRE(h.err == 0, h.err, "cen_sample: inconsistent path counts in the bidirectional walk");
  return h;
}

// Bidirectional form: one CTA per sample writes its members to an arena;
// what it defers runs on the bit-parallel sampler (see bidir.cu).  Returns
// the new members.
int64_t append_bidir(cen_job *job, uint64_t m0, uint64_t m_new) {
  cudaStream_t st = job->st;
  bidir_setup(job, m_new);
  BiWS &bw = *job->bws;
  const double mean = job->m ? (double)job->members / (double)job->m : 4.0;
  int64_t cap = (int64_t)((double)m_new * std::max(8.0, 2.0 * mean)) + ((int64_t)1 << 20);
  bw.arena.ensure(4 * (size_t)cap, st);
  bidir_launch(job, m0, m_new, cap);
  BiCtl h = bidir_finish(job);
  if ((int64_t)h.cursor > cap) {
    // The arena was short (long paths in a job's first round, where no mean
    // is known yet): the cursor has counted every walk's members, so size the
    // arena to it and run the samples again (they are functions of their ids)
    // instead of leaving those walks to the bit-parallel sampler.
    cap = (int64_t)h.cursor + ((int64_t)1 << 20);
    bw.arena.ensure(4 * (size_t)cap, st);
    bidir_launch(job, m0, m_new, cap);
    h = bidir_finish(job);
  }
  if (job->bidir_table < 0 && m_new >= 1024 && 2 * h.nmigrate > m_new) job->g->bidir_table_off.store(true);
  // warp searches pay off when few outgrow a warp; each one handed on is searched twice
  if (job->bidir_warps < 0 && bw.WQ && m_new >= 1024 && 10 * h.nbig > 3 * m_new) job->g->bidir_warps_off.store(true);
  std::vector<uint64_t> search(h.nsearch), walk(h.nwalk);
  if (h.nsearch)
    CEN_CK(cudaMemcpyAsync(search.data(), bw.dsearch.p, 8 * h.nsearch, cudaMemcpyDeviceToHost, st));
  if (h.nwalk) CEN_CK(cudaMemcpyAsync(walk.data(), bw.dwalk.p, 8 * h.nwalk, cudaMemcpyDeviceToHost, st));
  if (h.nsearch || h.nwalk) CEN_CK(cudaStreamSynchronize(st));
  std::sort(search.begin(), search.end());

  // whole samples the CTAs could not search: bit-parallel, members into the arena
  int64_t cursor = std::min<int64_t>((int64_t)h.cursor, cap);
  if (!search.empty()) {
    WaveWS &w0 = wave_ws0(job);
    Sampler sp = make_sampler(job, w0, st);
    for (size_t q0 = 0; q0 < search.size();) {
      const int G = pick_G(search.size() - q0, job->g->n, job->level_budget, job->max_wave_words);
      const int count = (int)std::min<size_t>((size_t)64 * G, search.size() - q0);
      upload_jlist(w0, search.data() + q0, count, st);
      sp.setup(G);
      int64_t total = 0;
      const int Lmax = sp.discover_and_cone(count, 0, w0.jlist.as<uint64_t>(), &total);
      bw.arena.ensure(4 * (size_t)(cursor + total + 1), st, 4 * (size_t)cursor);
      sp.sigma_and_walk<uint64_t>(count, Lmax, w0.woff.as<int64_t>(), bw.arena.as<int32_t>() + cursor);
      launch(&job->stats, K_APPEND, st, [&] {
        k_set_aoff<<<grid_for(count, 256), 256, 0, st>>>(count, w0.jlist.as<uint64_t>(), m0, w0.woff.as<int64_t>(),
                                                          sp.slot_d, cursor, bw.aoff.as<int64_t>());
      });
      CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      CEN_CK(cudaStreamSynchronize(st));
      CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent path counts in the backward walk");
      for (int f = 0; f < sp.hctl->nflag; ++f) walk.push_back(search[q0 + sp.hctl->flagged[f]]);
      cursor += total;
      q0 += (size_t)count;
    }
  }
  // Without searches on the bit-parallel sampler, every sample with d >= 2
  // reserved its d - 1 members in the arena (walked or deferred), so the
  // cursor is the new members' total and the offsets need no read-back.
  const int64_t total = offsets_from_distances(job, m0, m_new, search.empty() ? (int64_t)h.cursor : -1);
  job->hmem.ensure(4 * (size_t)(job->members + total + 1), st, 4 * (size_t)job->members);
  launch(&job->stats, K_APPEND, st, [&] {
    k_gather_arena<<<grid_for(m_new * 32, 256), 256, 0, st>>>(m_new, m0, bw.aoff.as<int64_t>(),
                                                              job->pd.as<int32_t>(), job->hoff.as<int64_t>(),
                                                              bw.arena.as<int32_t>(), job->hmem.as<int32_t>());
  });
  // walks the CTAs left (cone or counts too large, arena full) and the pairs
  // whose count reached 2^64 in the waves above: written in place
  rerun_in_place(job, walk);
  job->bidir_deferred_search += h.nsearch;
  job->bidir_deferred_walk += walk.size();
  job->bidir_migrated += h.nmigrate;
  job->bidir_escalated += h.nbig;
  return total;
}

// kappa-path space: a warp per walk into a strided buffer, then packed.  When
// that buffer would exceed kKpathBuffer bytes, the walks run twice instead
// (they are functions of the sample ids): once for their lengths, then again
// writing members straight into the store.
constexpr size_t kKpathBuffer = (size_t)1 << 30;

int64_t append_kpath(cen_job *job, uint64_t m0, uint64_t m_new) {
  cudaStream_t st = job->st;
  const bool staged = 4 * (size_t)m_new * (size_t)job->kappa <= kKpathBuffer;
  if (staged) {
    job->space_buf.ensure(4 * (size_t)m_new * (size_t)job->kappa, st);
    kpath_sample(job, m0, m_new, job->space_buf.as<int32_t>(), nullptr);
  } else {
    kpath_sample(job, m0, m_new, nullptr, nullptr);
  }
  const int64_t total = offsets_from_distances(job, m0, m_new);
  job->hmem.ensure(4 * (size_t)(job->members + total + 1), st, 4 * (size_t)job->members);
  if (!staged) {
    kpath_sample(job, m0, m_new, job->hmem.as<int32_t>(), job->hoff.as<int64_t>());
    return total;
  }
  WaveWS &w0 = wave_ws0(job);
  launch(&job->stats, K_APPEND, st, [&] {
    k_gather_strided<<<grid_for(m_new * 32, 256), 256, 0, st>>>(m_new, m0, job->kappa, w0.lens.as<int32_t>(),
                                                                job->hoff.as<int64_t>(), job->space_buf.as<int32_t>(),
                                                                job->hmem.as<int32_t>());
  });
  return total;
}

// Triangle space: three members each, written in place.
int64_t append_triangle(cen_job *job, uint64_t m0, uint64_t m_new) {
  cudaStream_t st = job->st;
  const int64_t total = offsets_from_distances(job, m0, m_new);
  job->hmem.ensure(4 * (size_t)(job->members + total + 1), st, 4 * (size_t)job->members);
  triangle_sample(job, m0, m_new);
  int *h = (int *)host_staging(job, 4);  // |h| = 3 for every sample
  *h = 3;
  CEN_CK(cudaMemcpyAsync(job->bmax.p, h, 4, cudaMemcpyHostToDevice, st));
  CEN_CK(cudaStreamSynchronize(st));
  return total;
}

// Bit-parallel form: the new samples are cut into waves; up to
// job->wave_streams waves run at once, each on its own stream and workspace,
// writing members to a wave buffer.  Then the offsets of all new samples come
// from one scan of their lengths and the wave buffers are copied in order, so
// the store is the same whatever the concurrency.  Pairs whose path count
// reached 2^64 are re-run with 128-bit counts at the end.  Returns the new
// members.
int64_t append_waves(cen_job *job, uint64_t m0, uint64_t m_new) {
  const cen_graph *g = job->g;
  cudaStream_t st = job->st;
  const uint64_t m1 = m0 + m_new;
  std::vector<std::unique_ptr<WaveOut>> waves;
  for (uint64_t j0 = m0; j0 < m1;) {
    const int G = pick_G(m1 - j0, g->n, job->level_budget, job->max_wave_words);
    const int count = (int)std::min<uint64_t>((uint64_t)64 * G, m1 - j0);
    waves.emplace_back(new WaveOut());
    waves.back()->j0 = j0;
    waves.back()->count = count;
    waves.back()->G = G;
    j0 += (uint64_t)count;
  }
  int K = std::max(1, std::min<int>(job->wave_streams, (int)waves.size()));
  if ((size_t)g->n * 8 * waves[0]->G > ((size_t)256 << 20)) K = 1;  // large graphs: one wave at a time
  while ((int)job->wws.size() < K) {
    job->wws.emplace_back(new WaveWS());
    if (job->wws.size() > 1) CEN_CK(cudaStreamCreateWithFlags(&job->wws.back()->own_stream, cudaStreamNonBlocking));
  }
  cudaEvent_t ready;
  CEN_CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  CEN_CK(cudaEventRecord(ready, st));

  std::atomic<size_t> next{0};
  std::mutex err_mu;
  Error first_err{CEN_OK, ""};
  auto work = [&](int w) {
    try {
      WaveWS &wsw = *job->wws[w];
      Sampler sp = make_sampler(job, wsw, w == 0 ? st : wsw.own_stream);
      if (w > 0) CEN_CK(cudaStreamWaitEvent(sp.st, ready, 0));
      for (;;) {
        {
          std::lock_guard<std::mutex> lk(err_mu);
          if (first_err.code != CEN_OK) return;
        }
        const size_t q = next.fetch_add(1);
        if (q >= waves.size()) break;
        WaveOut &wo = *waves[q];
        Range wave_range("wave");
        sp.setup(wo.G);
        const int Lmax = sp.discover_and_cone(wo.count, wo.j0, nullptr, &wo.total);
        wo.mem.ensure(4 * (size_t)(wo.total + 1), sp.st);
        sp.sigma_and_walk<uint64_t>(wo.count, Lmax, wsw.woff.as<int64_t>(), wo.mem.as<int32_t>());
        CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sp.st));
        CEN_CK(cudaStreamSynchronize(sp.st));
        CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent path counts in the backward walk");
        for (int f = 0; f < sp.hctl->nflag; ++f) wo.flagged.push_back(wo.j0 + (uint64_t)sp.hctl->flagged[f]);
      }
      CEN_CK(cudaStreamSynchronize(sp.st));
    } catch (const Error &e) {
      std::lock_guard<std::mutex> lk(err_mu);
      if (first_err.code == CEN_OK) first_err = e;
    } catch (...) {
      std::lock_guard<std::mutex> lk(err_mu);
      if (first_err.code == CEN_OK) first_err = Error{CEN_ECUDA, "cen_sample: unexpected error in a wave worker"};
    }
  };
  int dev = 0;
  CEN_CK(cudaGetDevice(&dev));
  std::vector<std::thread> pool;
  for (int w = 1; w < K; ++w)
    pool.emplace_back([&, w] {
      if (cudaSetDevice(dev) != cudaSuccess) return;
      work(w);
    });
  work(0);
  for (auto &th : pool) th.join();
  cudaEventDestroy(ready);
  if (first_err.code != CEN_OK) throw first_err;

  // offsets of the new samples, then the wave buffers in order
  const int64_t total = offsets_from_distances(job, m0, m_new);
  const int64_t members = job->members;
  job->hmem.ensure(4 * (size_t)(members + total + 1), st, 4 * (size_t)members);
  int64_t pos = members;
  std::vector<uint64_t> flagged_js;
  for (auto &wo : waves) {
    if (wo->total)
      CEN_CK(cudaMemcpyAsync(job->hmem.as<int32_t>() + pos, wo->mem.p, 4 * (size_t)wo->total,
                             cudaMemcpyDeviceToDevice, st));
    pos += wo->total;
    flagged_js.insert(flagged_js.end(), wo->flagged.begin(), wo->flagged.end());
  }
  // 128-bit re-run of the slots whose path count reached 2^64 (offsets known)
  if (!flagged_js.empty()) {
    std::sort(flagged_js.begin(), flagged_js.end());
    WaveWS &w0 = *job->wws[0];
    Sampler sp = make_sampler(job, w0, st);
    sp.setup(1);
    for (size_t q0 = 0; q0 < flagged_js.size(); q0 += 64) {
      const int count = (int)std::min<size_t>(64, flagged_js.size() - q0);
      upload_jlist(w0, flagged_js.data() + q0, count, st);
      sp.hctl = (Ctl *)ws_staging(w0, sizeof(Ctl));
      const int Lmax = sp.discover_and_cone(count, 0, w0.jlist.as<uint64_t>(), nullptr);
      sp.sigma_and_walk<u128>(count, Lmax, nullptr, job->hmem.as<int32_t>());
      CEN_CK(cudaMemcpyAsync(sp.hctl, sp.ctl, offsetof(Ctl, flagged), cudaMemcpyDeviceToHost, st));
      CEN_CK(cudaStreamSynchronize(st));
      CEN_REQUIRE(sp.hctl->err != CEN_EOVERFLOW, CEN_EOVERFLOW,
                  "cen_sample: a sampled pair has >= 2^128 shortest paths");
      CEN_REQUIRE(sp.hctl->err == 0, sp.hctl->err, "cen_sample: inconsistent 128-bit path counts");
    }
  }
  for (auto &wo : waves) wo->mem.release();  // stream-ordered after the copies above
  return total;
}

}  // namespace

// Alg. 1 "sampleHEs": appends samples m .. m + m_new - 1 (pairs, distances,
// hyper-edges, sign columns).
void sample_append(cen_job *job, uint64_t m_new) {
  if (m_new == 0) return;
  Range range("cen_sample");
  cudaStream_t st = job->st;
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
  int64_t total;
  if (job->space == CEN_SPACE_KPATH)
    total = append_kpath(job, m0, m_new);
  else if (job->space == CEN_SPACE_TRIANGLE)
    total = append_triangle(job, m0, m_new);
  else
    total = job->sampler == 0 ? append_bidir(job, m0, m_new) : append_waves(job, m0, m_new);
  // sign columns of the new samples
  {
    const int nblk = (job->nw + 3) / 4;
    launch(&job->stats, K_SIGN, st, [&] {
      k_sign<<<grid_for(m_new * nblk, 256), 256, 0, st>>>(m0, m_new, job->t, job->nw, job->key(),
                                                          job->sign.as<uint32_t>());
    });
  }
  CEN_CK(cudaStreamSynchronize(st));
  job->m = m1;
  job->members += total;
}

}  // namespace cen
