// Balanced bidirectional sampler for set betweenness (Sec. 5 sampleHEs).
//
// For the pair (s, t) a forward ball grows from s over out-arcs and a backward
// ball from t over in-arcs, one level at a time, always on the side whose
// frontier has fewer arcs to scan (Sec. 5: the balanced bidirectional BFS).
// The first level that touches the other ball fixes d(s, t) = ls + lb + 1,
// where ls and lb are the two frontier levels, and every shortest path crosses
// exactly one arc from the forward frontier into the backward frontier.
//
// The hyper-edge equals the one the forward sampler draws for the same
// sample: the cone (nodes on some shortest s-t path) is cut from the crossing
// arcs down both balls; the path counts sigma_s (shortest s -> v paths) are
// taken over the cone in order of distance from s, through the crossing arcs
// into the backward ball; and the backward walk from t draws the same Philox
// numbers and scans in-neighbours in the same ascending order.  A node one
// step closer to s than a cone node, with an arc into it, is itself a cone
// node, so these counts equal a full BFS's wherever the walk reads them, and
// which side grew when changes only the cost.
//
// Two granularities run in two persistent launches of 128-thread CTAs.  In
// the first, each warp takes sample ids from a counter and searches on its
// own ("warp search"): no CTA barrier, a private node table of kWarpTable
// entries and lists carved from its CTA's.  A warp search that would expand a
// level of more than kWarpLevelArcs arcs, fills half of its table or a list,
// or needs more than kWarpLevels levels on a side stops before writing
// anything but the pair and appends its id to a list; the second launch
// searches the listed samples with whole CTAs ("CTA search") and the CTAs'
// tables.  Which granularity searched a sample changes only the cost: the
// search is the same code at two group sizes.
//
// Node state lives in hash tables (open addressing, linear probing, entries
// stamped with a per-table epoch so nothing is cleared between samples).  A
// CTA search starts in a small table sized so that all CTAs' tables stay in
// L2 and moves, once that is half full, to a large table of 4 QC entries that
// always has room for both balls, redoing the level it was building.  Path
// counts are indexed by table position.
//
// Work a CTA cannot hold is left to the bit-parallel sampler, which gives the
// identical hyper-edge: more than kBiMaxLevels levels on one side or more
// than QC nodes in one ball ("search" deferral, distance unknown); a path
// count reaching 2^64 or a full member arena ("walk" deferral, distance
// known).  A cone side is part of its ball, so it always fits.
#include <algorithm>
#include <mutex>
#include <vector>

#include "job.cuh"

namespace cen {

namespace {

constexpr int kBiThreads = 128;
constexpr int kBiWarps = kBiThreads / 32;
constexpr int kBiMaxLevels = 256;   // levels per side of a CTA search (0 .. kBiMaxLevels - 1)
constexpr int kWarpLevels = 64;     // levels per side of a warp search
constexpr int kBiHeavy = 256;       // rows longer than this are scanned by the whole search group
constexpr uint32_t kEpochMax = (1u << 16) - 1;
constexpr int kWarpLevelArcs = 2048; // a warp search hands on a level with more arcs to expand
constexpr int kBiCtaPerSM = 16;      // resident CTAs per SM (32 registers)
constexpr int kBiWarpCtaPerSM = 12;  // warp-search CTAs per SM (40 registers: fewer spills, measured faster)

// Table entry: node 31 | epoch 16 | cone 1 | side 1 | level 14.
constexpr uint64_t kConeBit = 1ull << 15;
__device__ __forceinline__ int st_level(uint64_t s) { return (int)(s & 0x3FFFu); }
__device__ __forceinline__ int st_side(uint64_t s) { return (int)((s >> 14) & 1u); }
__device__ __forceinline__ bool st_cone(uint64_t s) { return (s & kConeBit) != 0; }
__device__ __forceinline__ uint32_t h_epoch(uint64_t s) { return (uint32_t)((s >> 16) & 0xFFFFu); }
__device__ __forceinline__ uint32_t h_node(uint64_t s) { return (uint32_t)(s >> 32); }
__device__ __forceinline__ uint64_t h_make(uint32_t v, uint32_t epoch, int side, int level) {
  return ((uint64_t)v << 32) | ((uint64_t)epoch << 16) | ((uint64_t)side << 14) | (uint64_t)level;
}
__device__ __forceinline__ uint32_t h_slot(uint32_t v, uint32_t mask) {
  uint32_t h = v * 0x9E3779B1u;
  return (h ^ (h >> 15)) & mask;
}
__device__ __forceinline__ uint64_t ld_vol(const uint64_t *p) { return *(const volatile uint64_t *)p; }
__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// The table the current search uses.  Copied into every thread; changed only
// between barriers.
struct BiMap {
  uint64_t *tab;
  uint32_t mask;  // entries - 1
  uint32_t ep;    // current epoch
};

// State of v in the current search (0 if unvisited); idx receives its table
// position, which also indexes its path count.
__device__ __forceinline__ uint64_t bi_find(const BiMap &M, int v, int64_t &idx) {
  uint32_t p = h_slot((uint32_t)v, M.mask);
  for (uint32_t k = 0; k <= M.mask; ++k) {
    const uint64_t e = ld_vol(&M.tab[p]);
    if (h_epoch(e) != M.ep) return 0;  // a free position ends the probe: v was never inserted
    if (h_node(e) == (uint32_t)v) {
      idx = p;
      return e;
    }
    p = (p + 1) & M.mask;
  }
  return 0;
}

__device__ __forceinline__ uint64_t bi_find(const BiMap &M, int v) {
  int64_t idx;
  return bi_find(M, v, idx);
}

// Claims v for side x on `level`.  Returns 0 when this call claimed it, 1 when
// it was already in the search (its state in *found, 0 if the table is full).
__device__ __forceinline__ int bi_claim(const BiMap &M, int v, int x, int level, uint64_t &found) {
  const uint64_t mine = h_make((uint32_t)v, M.ep, x, level);
  uint32_t p = h_slot((uint32_t)v, M.mask);
  for (uint32_t k = 0; k <= M.mask; ++k) {
    uint64_t e = ld_vol(&M.tab[p]);
    for (;;) {
      if (h_epoch(e) == M.ep) {
        if (h_node(e) == (uint32_t)v) {
          found = e;
          return 1;
        }
        break;  // another node's entry: next position
      }
      const unsigned long long old =
          atomicCAS((unsigned long long *)&M.tab[p], (unsigned long long)e, (unsigned long long)mine);
      if (old == e) return 0;
      e = old;  // taken meanwhile: look at it again
    }
    p = (p + 1) & M.mask;
  }
  found = 0;
  return 1;
}

// One probe for discovery: returns 0 when this call claimed v for side x on
// `level`, 1 when v was already in the search (its state in *found), 2 when
// it was not and `claim` was false (nothing written).
__device__ __forceinline__ int bi_visit(const BiMap &M, int v, int x, int level, bool claim, uint64_t &found) {
  const uint64_t mine = h_make((uint32_t)v, M.ep, x, level);
  uint32_t p = h_slot((uint32_t)v, M.mask);
  for (uint32_t k = 0; k <= M.mask; ++k) {
    uint64_t e = ld_vol(&M.tab[p]);
    for (;;) {
      if (h_epoch(e) == M.ep) {
        if (h_node(e) == (uint32_t)v) {
          found = e;
          return 1;
        }
        break;  // another node's entry: next position
      }
      if (!claim) return 2;
      const unsigned long long old =
          atomicCAS((unsigned long long *)&M.tab[p], (unsigned long long)e, (unsigned long long)mine);
      if (old == e) return 0;
      e = old;  // taken meanwhile: look at it again
    }
    p = (p + 1) & M.mask;
  }
  return 2;
}

// Shared state of one search: LV levels per side, a group of W warps.
template <int LV, int W>
struct BiSh {
  int lo[2][LV + 1];                  // ball queue of side x: level L is lo[x][L] .. lo[x][L+1]
  unsigned long long hcost[2][LV];    // arcs out of level L of side x (out-arcs forward, in-arcs backward)
  int cs[2][LV];                      // cone list of side x: level L is cs[x][L] .. ce[x][L]
  int ce[2][LV];
  unsigned long long red[W], red2[W];
  // arc-balanced scan (warp searches only, W = 1): first arc of each row of a
  // chunk and the total, the rows' nodes and their first arcs in the CSR
  static constexpr int kBal = W == 1 ? 32 : 1;
  long long bpre[kBal + 1];
  int bv[kBal];
  long long be0[kBal];
  unsigned long long sum, sum2, arcs;
  int added, nheavy, ccount[2], ncross;
  int hcount, hfull;  // small-table entries of this search; set once it is half full
  int lvl[2];
  int met, ovf, xovf;
  int status, d;
  int s, t;
  uint32_t ep;        // epoch of the table in use
  int tier;           // 1: small table, 2: large table
  int clear;          // the table in use must be cleared first
  long long abase;
};
using BiShCta = BiSh<kBiMaxLevels, kBiWarps>;
using BiShWarp = BiSh<kWarpLevels, 1>;

// Barrier and thread index of a search group of T threads: a warp (T = 32) or
// the whole CTA (T = 128).  __syncwarp orders memory among the warp's lanes.
template <int T>
__device__ __forceinline__ void gsync() {
  if (T == 32)
    __syncwarp();
  else
    __syncthreads();
}
template <int T>
__device__ __forceinline__ int gtid() {
  return (int)(threadIdx.x & (unsigned)(T - 1));
}

// Sum over the group of one value per thread, returned to every thread.
template <int T, class SH>
__device__ __forceinline__ unsigned long long gsum(unsigned long long a, SH &sh) {
  a = warp_sum(a);  // every lane holds its warp's total
  if (T == 32) return a;
  const int tid = gtid<T>();
  if ((tid & 31) == 0) sh.red[tid >> 5] = a;
  __syncthreads();
  if (tid == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < T / 32; ++w) tot += sh.red[w];
    sh.sum = tot;
  }
  __syncthreads();
  const unsigned long long r = sh.sum;
  __syncthreads();
  return r;
}

// Sets the cone bit of v and, the first time, appends v to the cone list of
// side x (capacity QC).
template <class SH>
__device__ __forceinline__ void bi_mark(const BiMap &M, uint64_t *sg, uint32_t *clist, int x, int64_t QC, SH &sh,
                                        int v) {
  int64_t p = -1;
  if (!bi_find(M, v, p)) {  // cannot happen: every cone node is in its ball
    sh.ovf = 1;
    return;
  }
  const unsigned long long old = atomicOr((unsigned long long *)&M.tab[p], (unsigned long long)kConeBit);
  if (old & kConeBit) return;
  sg[p] = 0;  // its path count starts from zero
  const int pos = atomicAdd(&sh.ccount[x], 1);
  if (pos >= QC) {
    sh.ovf = 1;
    return;
  }
  clist[pos] = (uint32_t)v;
}

// Group size for a list of cnt rows with `arcs` arcs in all: the power of two
// near the mean row length, 1 .. 32.
__device__ __forceinline__ int bi_group(unsigned long long arcs, int cnt) {
  const unsigned long long mean = cnt ? (arcs + cnt - 1) / (unsigned long long)cnt : 1;
  int gs = 1;
  while (gs < 32 && (unsigned long long)gs < mean) gs <<= 1;
  return gs;
}

// Sum over list[0, cnt) of the row lengths in o.  Called by the whole group.
template <int T, class SH>
__device__ unsigned long long bi_row_sum(const uint32_t *list, int cnt, const int64_t *__restrict__ o, SH &sh) {
  const int tid = gtid<T>();
  unsigned long long a = 0;
  for (int i = tid; i < cnt; i += T) {
    const int v = (int)list[i];
    a += (unsigned long long)(o[v + 1] - o[v]);
  }
  const unsigned long long r = gsum<T>(a, sh);
  if (T == 32) __syncwarp();
  return r;
}

// Row-length sums of two lists at once (list1 in o1, list2 in o2), into
// *s1, *s2.  Called by the whole group.
template <int T, class SH>
__device__ void bi_row_sum2(const uint32_t *list1, int cnt1, const int64_t *__restrict__ o1, const uint32_t *list2,
                            int cnt2, const int64_t *__restrict__ o2, SH &sh, unsigned long long *s1,
                            unsigned long long *s2) {
  const int tid = gtid<T>();
  unsigned long long a = 0, b = 0;
  for (int i = tid; i < cnt1; i += T) {
    const int v = (int)list1[i];
    a += (unsigned long long)(o1[v + 1] - o1[v]);
  }
  for (int i = tid; i < cnt2; i += T) {
    const int v = (int)list2[i];
    b += (unsigned long long)(o2[v + 1] - o2[v]);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (T == 32) {
    *s1 = a;
    *s2 = b;
    __syncwarp();
    return;
  }
  if ((tid & 31) == 0) {
    sh.red[tid >> 5] = a;
    sh.red2[tid >> 5] = b;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long ta = 0, tb = 0;
    for (int w = 0; w < T / 32; ++w) {
      ta += sh.red[w];
      tb += sh.red2[w];
    }
    sh.sum = ta;
    sh.sum2 = tb;
  }
  __syncthreads();
  *s1 = sh.sum;
  *s2 = sh.sum2;
  __syncthreads();
}

// For every node v of list[0, cnt) and every arc of v's row in (o, c), calls
// f(v, w).  Rows of at most kBiHeavy arcs are scanned by a subgroup of gs
// lanes; longer rows are queued in `heavy` and scanned by the whole group.
// Called by the whole group.
template <int T, class SH, class F>
__device__ void bi_scan_rows(const uint32_t *list, int cnt, const int64_t *__restrict__ o,
                             const int32_t *__restrict__ c, int gs, uint32_t *heavy, SH &sh, F &&f) {
  const int tid = gtid<T>();
  if (tid == 0) sh.nheavy = 0;
  gsync<T>();
  const int gl = tid & (gs - 1), gi = tid / gs, ng = T / gs;
  unsigned long long arcs = 0;
  for (int i = gi; i < cnt; i += ng) {
    const int v = (int)list[i];
    const int64_t e0 = o[v], e1 = o[v + 1];
    if (e1 - e0 > kBiHeavy) {
      if (gl == 0) heavy[atomicAdd(&sh.nheavy, 1)] = (uint32_t)v;
      continue;
    }
    for (int64_t e = e0 + gl; e < e1; e += gs) f(v, c[e]);
    if (gl == 0) arcs += (unsigned long long)(e1 - e0);
  }
  gsync<T>();
  const int nh = sh.nheavy;
  for (int h = 0; h < nh; ++h) {
    const int v = (int)heavy[h];
    const int64_t e0 = o[v], e1 = o[v + 1];
    for (int64_t e = e0 + tid; e < e1; e += T) f(v, c[e]);
    if (tid == 0) arcs += (unsigned long long)(e1 - e0);
  }
  if (arcs) atomicAdd(&sh.arcs, arcs);
  gsync<T>();
}

// As bi_scan_rows for a warp search, with every row's arcs dealt evenly to
// the warp's lanes: the rows are taken 32 at a time, a scan of their lengths
// gives each row's first arc within the chunk, and lane i takes arcs i,
// i + 32, ... of the chunk, finding each arc's row by binary search, so that
// no lane waits on a long row of its subgroup and a long row needs no pass of
// its own.  Called by the whole warp.
template <int T, class SH, class F>
__device__ void bi_scan_rows_bal(const uint32_t *list, int cnt, const int64_t *__restrict__ o,
                                 const int32_t *__restrict__ c, SH &sh, F &&f) {
  static_assert(T == 32, "the even deal is the warp searches' scan");
  const int lane = gtid<T>();
  unsigned long long arcs = 0;
  for (int c0 = 0; c0 < cnt; c0 += T) {
    int v = 0;
    long long e0 = 0, len = 0;
    if (c0 + lane < cnt) {
      v = (int)list[c0 + lane];
      e0 = o[v];
      len = o[v + 1] - e0;
    }
    arcs += (unsigned long long)len;
    long long x = len;  // inclusive scan of the lengths
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    sh.bpre[lane] = x - len;
    sh.bv[lane] = v;
    sh.be0[lane] = e0;
    if (lane == T - 1) sh.bpre[T] = x;
    __syncwarp();
    const long long total = sh.bpre[T];
    for (long long a = lane; a < total; a += T) {
      int lo = 0, hi = T - 1;  // the last row starting at or before arc a
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sh.bpre[mid] <= a)
          lo = mid;
        else
          hi = mid - 1;
      }
      f(sh.bv[lo], c[sh.be0[lo] + (a - sh.bpre[lo])]);
    }
    __syncwarp();  // the next chunk overwrites the shared rows
  }
  if (arcs) atomicAdd(&sh.arcs, arcs);
  __syncwarp();
}

// The row scan of a search group: a warp deals every row's arcs evenly to its
// lanes (measured faster for warps, 1.1-1.35x on BA graphs); a CTA gives rows
// to lane groups of gs and long rows to the whole CTA (the even deal was no
// faster for CTAs).
template <int T, class SH, class F>
__device__ __forceinline__ void bi_scan(const uint32_t *list, int cnt, const int64_t *__restrict__ o,
                                        const int32_t *__restrict__ c, int gs, uint32_t *heavy, SH &sh, F &&f) {
  if constexpr (T == 32)
    bi_scan_rows_bal<T>(list, cnt, o, c, sh, f);
  else
    bi_scan_rows<T>(list, cnt, o, c, gs, heavy, sh, f);
}

__device__ __forceinline__ void add_carry(unsigned long long &acc, unsigned long long v, int &ovf) {
  acc += v;
  ovf |= acc < v;
}

// Distance from s of a visited node: its level in the forward ball, d minus
// its level in the backward ball.
__device__ __forceinline__ int st_dist(uint64_t s, int d) { return st_side(s) ? d - st_level(s) : st_level(s); }

// Pull form of one path-count level: each cone node of list[0, cnt) (all at
// distance D from s) gets the sum of the counts of its in-neighbours that are
// cone nodes at D - 1.  A sum that wraps 2^64 raises sh.ovf.
template <int T, class SH>
__device__ void bi_sigma_pull(const uint32_t *list, int cnt, int D, int d, const BiMap &M, uint64_t *sg,
                              const int64_t *__restrict__ roff, const int32_t *__restrict__ rcol, int gs,
                              uint32_t *heavy, SH &sh) {
  const int tid = gtid<T>(), lane = tid & 31;
  if (tid == 0) sh.nheavy = 0;
  gsync<T>();
  const int gl = tid & (gs - 1), gi = tid / gs, ng = T / gs;
  const unsigned gmask = gs == 32 ? 0xffffffffu : (((1u << gs) - 1u) << (lane & ~(gs - 1)));
  int ovf = 0;
  unsigned long long arcs = 0;
  for (int i = gi; i < cnt; i += ng) {
    const int v = (int)list[i];
    const int64_t e0 = roff[v], e1 = roff[v + 1];
    if (e1 - e0 > kBiHeavy) {
      if (gl == 0) heavy[atomicAdd(&sh.nheavy, 1)] = (uint32_t)v;
      continue;
    }
    unsigned long long acc = 0;
    for (int64_t e = e0 + gl; e < e1; e += gs) {
      int64_t iu = 0;
      const uint64_t su = bi_find(M, rcol[e], iu);
      if (su && st_cone(su) && st_dist(su, d) == D - 1) add_carry(acc, sg[iu], ovf);
    }
    for (int o2 = gs >> 1; o2; o2 >>= 1) add_carry(acc, __shfl_xor_sync(gmask, acc, o2, gs), ovf);
    if (gl == 0) {
      int64_t iv = 0;
      bi_find(M, v, iv);
      sg[iv] = acc;
      arcs += (unsigned long long)(e1 - e0);
    }
  }
  if (ovf) sh.ovf = 1;
  gsync<T>();
  const int nh = sh.nheavy;
  for (int h = 0; h < nh; ++h) {
    const int v = (int)heavy[h];
    const int64_t e0 = roff[v], e1 = roff[v + 1];
    unsigned long long acc = 0;
    int hovf = 0;
    for (int64_t e = e0 + tid; e < e1; e += T) {
      int64_t iu = 0;
      const uint64_t su = bi_find(M, rcol[e], iu);
      if (su && st_cone(su) && st_dist(su, d) == D - 1) add_carry(acc, sg[iu], hovf);
    }
    for (int o2 = 16; o2; o2 >>= 1) add_carry(acc, __shfl_xor_sync(0xffffffffu, acc, o2), hovf);
    if (hovf) sh.ovf = 1;
    unsigned long long tot = acc;
    int tovf = 0;
    if (T > 32) {
      if (lane == 0) sh.red[tid >> 5] = acc;
      gsync<T>();
      if (tid == 0) {
        tot = 0;
        for (int w = 0; w < T / 32; ++w) add_carry(tot, sh.red[w], tovf);
      }
    }
    if (tid == 0) {
      if (tovf) sh.ovf = 1;
      int64_t iv = 0;
      bi_find(M, v, iv);
      sg[iv] = tot;
      arcs += (unsigned long long)(e1 - e0);
    }
    gsync<T>();
  }
  if (arcs) atomicAdd(&sh.arcs, arcs);
  gsync<T>();
}

// Whether the sorted row c[e0, e1) holds v (binary search).
__device__ __forceinline__ bool row_has(const int32_t *__restrict__ c, int64_t e0, int64_t e1, int32_t v) {
  while (e0 < e1) {
    const int64_t mid = e0 + ((e1 - e0) >> 1);
    const int32_t x = c[mid];
    if (x == v) return true;
    if (x < v)
      e0 = mid + 1;
    else
      e1 = mid;
  }
  return false;
}

}  // namespace

struct BiArgs {
  int32_t n;
  const int64_t *off, *roff;
  const int32_t *col, *rcol;
  SampleKey key;  // Philox key and the map from store positions to sample ids
  uint64_t j0, count;
  uint64_t *tab1;     // [slots][H1] small tables of the CTA searches (H1 = mask1 + 1; none when mask1 = 0)
  uint32_t mask1;
  uint64_t *tab2;     // [slots][H2] large tables
  uint32_t mask2;
  uint32_t *lists;    // [slots][7][QC]: ball queues and cone lists (forward, backward), heavy rows,
                      //                  crossing-arc tails and heads; a warp search uses [7][WQ] of
                      //                  its CTA's, at warp * 7 WQ
  uint64_t *sig;      // [slots][H2]: path counts by table position (a warp search: its CTA's, at
                      //              warp * kWarpTable)
  uint32_t *epochs;   // [slots][2]: epochs of the small and the large table
  int64_t QC;
  uint64_t *tabw;     // [slots][4][kWarpTable] node tables of the warp searches (null: CTA searches only)
  uint32_t *epw;      // [slots][4][2]: their epochs
  int64_t WQ;         // entries of each list of a warp search
  uint64_t *big;      // [count]: relative ids of the searches the warp kernel handed on
  const uint64_t *list;                   // list mode: relative sample ids, one CTA search each
  const unsigned long long *list_count;   // list mode: their number (device)
  int32_t *ps, *pt, *pd;
  int *bmax;
  int32_t *arena;
  int64_t arena_cap;
  int64_t *aoff;      // [count of the main launch]: first member in the arena, or -1
  uint64_t *dsearch;  // search-deferred sample ids
  uint64_t *dwalk;    // walk-deferred sample ids
  BiCtl *ctl;
  unsigned long long *units;
};

namespace {

constexpr int kWarpTable = 1024;  // node-table entries of a warp search (it stops at half)

// One search group's lists and tables.
struct BiWork {
  uint32_t *q[2], *cl[2], *heavy, *xt, *xh;
  int64_t QC;        // entries of each list
  uint64_t *sg;      // path counts by table position
  uint64_t *tab1;    // small table (null when h1 = 0)
  uint32_t h1;
  uint64_t *tab2;    // large table (CTA searches only)
  uint32_t h2;
  uint32_t *epochs;  // [0] small table, [1] large table
};

constexpr int kSearchBig = 3;  // a warp search outgrew its table, levels or lists: nothing was written

// One sample (relative id jr), searched by a group of T threads with LV levels
// per side.  Writes the pair, the distance, the arena offset and the members,
// or queues the sample for the bit-parallel sampler; a warp search (T = 32)
// that outgrows its resources returns kSearchBig before writing anything but
// the pair.  sh.arcs holds the arcs it scanned.  Called by the whole group.
template <int T, int LV>
__device__ __forceinline__ int bi_search(const BiArgs &A, BiSh<LV, T / 32> &sh, const BiWork &W, uint64_t jr) {
  constexpr bool kWarp = T == 32;
  const int tid = gtid<T>(), lane = threadIdx.x & 31;
  const int64_t QC = W.QC;
  uint32_t *heavy = W.heavy, *xt = W.xt, *xh = W.xh;
  uint32_t *q[2] = {W.q[0], W.q[1]};
  uint32_t *cl[2] = {W.cl[0], W.cl[1]};
  uint64_t *sg = W.sg;
  if (tid == 0) {
    sh.tier = W.h1 ? 1 : 2;  // a new epoch of the table the search starts in
    uint32_t e = W.epochs[sh.tier - 1] + 1;
    sh.clear = e > kEpochMax;
    if (sh.clear) e = 1;
    W.epochs[sh.tier - 1] = e;
    sh.ep = e;
    sh.arcs = 0;
  }
  gsync<T>();
  if (sh.clear) {  // the epoch field wrapped: the table starts over
    uint64_t *t0 = sh.tier == 1 ? W.tab1 : W.tab2;
    const uint32_t h0 = sh.tier == 1 ? W.h1 : W.h2;
    for (uint32_t p = tid; p < h0; p += T) t0[p] = 0;
    gsync<T>();
  }
  BiMap M{sh.tier == 1 ? W.tab1 : W.tab2, (sh.tier == 1 ? W.h1 : W.h2) - 1u, sh.ep};
  int tier = sh.tier;
  const uint64_t j = A.j0 + jr;
  if (tid == 0) {
    // Sec. 5: s uniform over V; t uniform over V \ {s} (Sec. 3.1 pairs u != v)
    const int32_t s = (int32_t)uniform_below64(A.key.seed, A.key.id(j), kPurposeS, (uint64_t)A.n);
    const int32_t tt = (int32_t)uniform_below64(A.key.seed, A.key.id(j), kPurposeT, (uint64_t)(A.n - 1));
    const int32_t t = tt + (tt >= s);
    A.ps[j] = s;
    A.pt[j] = t;
    sh.s = s;
    sh.t = t;
    uint64_t f;
    bi_claim(M, s, 0, 0, f);
    bi_claim(M, t, 1, 0, f);
    q[0][0] = (uint32_t)s;
    q[1][0] = (uint32_t)t;
    sh.lo[0][0] = 0;
    sh.lo[0][1] = 1;
    sh.lo[1][0] = 0;
    sh.lo[1][1] = 1;
    sh.lvl[0] = sh.lvl[1] = 0;
    sh.hcost[0][0] = (unsigned long long)(A.off[s + 1] - A.off[s]);
    sh.hcost[1][0] = (unsigned long long)(A.roff[t + 1] - A.roff[t]);
    sh.hcount = 2;
    sh.hfull = 0;
    sh.met = 0;
    sh.ovf = 0;
    sh.xovf = 0;
    sh.ncross = 0;
    sh.status = 0;
    sh.d = -1;
  }
  gsync<T>();

  // ---- discovery: grow the cheaper side until the balls touch.  The level
  // that touches is scanned to its end so that every crossing arc is logged.
  for (;;) {
    // the side with fewer arcs to scan; on a tie the shallower side, so that
    // graphs whose frontiers cost the same (cycles, grids) grow both balls
    const unsigned long long c0 = sh.hcost[0][sh.lvl[0]], c1 = sh.hcost[1][sh.lvl[1]];
    const int x = c0 < c1 || (c0 == c1 && sh.lvl[0] <= sh.lvl[1]) ? 0 : 1;
    const int L = sh.lvl[x];
    const unsigned long long fcost = sh.hcost[x][L];
    if (L + 1 >= LV || (kWarp && fcost > (unsigned long long)kWarpLevelArcs)) {
      // too deep for this group, or a level too wide for one warp: a CTA takes it
      if (tid == 0) sh.status = kWarp && L + 1 < kBiMaxLevels ? kSearchBig : 1;
      break;
    }
    const int f0 = sh.lo[x][L], f1 = sh.lo[x][L + 1];
    gsync<T>();
    if (tid == 0) {
      sh.added = 0;
      sh.ncross = 0;
      sh.xovf = 0;
    }
    uint32_t *qx = q[x];
    const int64_t *o = x ? A.roff : A.off;
    const int32_t *c = x ? A.rcol : A.col;
    const int hlimit = (int)(W.h1 >> 1), hbase = sh.hcount;
    auto visit = [&](int v, int w) {
      uint64_t sw = 0;
      // once the distance is known, or the small table is half full, nothing more is claimed
      const bool claim = !(*(volatile int *)&sh.met || *(volatile int *)&sh.hfull);
      const int r = bi_visit(M, w, x, L + 1, claim, sw);
      if (r == 0) {
        const int pos = atomicAdd(&sh.added, 1);
        if ((int64_t)f1 + pos < QC)
          qx[f1 + pos] = (uint32_t)w;
        else
          sh.ovf = 1;
        if (tier == 1 && hbase + pos + 1 >= hlimit) sh.hfull = 1;
        return;
      }
      if (r == 2 || !sw) return;
      if (st_side(sw) != x) {  // an arc between the balls: (tail, head) in s -> t direction
        sh.met = 1;
        const int pos = atomicAdd(&sh.ncross, 1);
        if (pos < QC) {
          xt[pos] = (uint32_t)(x ? w : v);
          xh[pos] = (uint32_t)(x ? v : w);
        } else {
          sh.xovf = 1;
        }
      }
    };
    bi_scan<T>(qx + f0, f1 - f0, o, c, bi_group(fcost, f1 - f0), heavy, sh, visit);
    if (sh.met) {
      if (tid == 0) sh.d = sh.lvl[0] + sh.lvl[1] + 1;
      break;
    }
    if (sh.hfull) {
      if (kWarp) {  // a warp search does not move to a large table: the CTA takes the sample
        if (tid == 0) sh.status = kSearchBig;
        break;
      }
      // the small table is half full: the search so far moves to the large
      // table (a new epoch of it), without the half-built level, which is redone
      if (tid == 0) {
        uint32_t e = W.epochs[1] + 1;
        sh.clear = e > kEpochMax;
        if (sh.clear) e = 1;
        W.epochs[1] = e;
        sh.ep = e;
      }
      gsync<T>();
      if (sh.clear) {
        for (uint32_t p = tid; p < W.h2; p += T) W.tab2[p] = 0;
        gsync<T>();
      }
      const BiMap M2{W.tab2, W.h2 - 1u, sh.ep};
      for (uint32_t p = tid; p < W.h1; p += T) {
        const uint64_t e = W.tab1[p];
        if (h_epoch(e) == M.ep && !(st_side(e) == x && st_level(e) == L + 1)) {
          uint64_t f;
          bi_claim(M2, (int)h_node(e), st_side(e), st_level(e), f);
        }
      }
      M = M2;
      tier = 2;
      gsync<T>();
      if (tid == 0) {
        sh.tier = 2;
        sh.hfull = 0;
        sh.ovf = 0;
        atomicAdd(&A.ctl->nmigrate, 1ull);
      }
      gsync<T>();
      continue;
    }
    if (sh.ovf) {
      if (tid == 0) sh.status = kWarp ? kSearchBig : 1;
      break;
    }
    if (sh.added == 0) break;  // this side's ball is closed: t is unreachable
    // arcs out of the new level, summed once it is complete (all rows at once)
    const int nadd = sh.added;
    const unsigned long long cost = bi_row_sum<T>(qx + f1, nadd, o, sh);
    if (tid == 0) {
      sh.lo[x][L + 2] = f1 + nadd;
      sh.hcost[x][L + 1] = cost;
      sh.lvl[x] = L + 1;
      sh.hcount += nadd;
    }
    gsync<T>();
  }
  gsync<T>();
  const int d = sh.d;
  if (sh.status == kSearchBig) return kSearchBig;
  if (sh.status == 1) {  // distance unknown: the bit-parallel sampler takes the whole sample
    if (tid == 0) {
      A.pd[j] = -1;
      A.aoff[jr] = -1;
      A.dsearch[atomicAdd(&A.ctl->nsearch, 1ull)] = j;
    }
    gsync<T>();
    return 0;
  }
  if (tid == 0) {
    A.pd[j] = d;
    A.aoff[jr] = -1;
    if (d >= 2) {
      atomicMax(A.bmax, d - 1);
      const unsigned long long base = atomicAdd(&A.ctl->cursor, (unsigned long long)(d - 1));
      if ((long long)(base + (unsigned long long)(d - 1)) > A.arena_cap)
        sh.status = 2;
      else
        sh.abase = (long long)base;
    }
    sh.ccount[0] = sh.ccount[1] = 0;
    sh.ovf = 0;
  }
  gsync<T>();
  if (d < 2) return 0;  // adjacent or unreachable: the empty hyper-edge

  const int ls = sh.lvl[0], lb = sh.lvl[1];
  const int ncross = min(sh.ncross, (int)QC);
  if (sh.status == 0) {
    // ---- crossing arcs: forward level ls -> backward level lb
    if (!sh.xovf) {
      for (int i = tid; i < ncross; i += T) {
        bi_mark(M, sg, cl[0], 0, QC, sh, (int)xt[i]);
        bi_mark(M, sg, cl[1], 1, QC, sh, (int)xh[i]);
      }
      gsync<T>();
    } else {
      const int f0 = sh.lo[0][ls], f1 = sh.lo[0][ls + 1];
      bi_scan<T>(q[0] + f0, f1 - f0, A.off, A.col, bi_group(sh.hcost[0][ls], f1 - f0), heavy, sh,
                      [&](int v, int w) {
                        const uint64_t sw = bi_find(M, w);
                        if (sw && st_side(sw) == 1 && st_level(sw) == lb) {
                          bi_mark(M, sg, cl[0], 0, QC, sh, v);
                          bi_mark(M, sg, cl[1], 1, QC, sh, w);
                        }
                      });
    }
    if (tid == 0) {
      sh.cs[0][ls] = 0;
      sh.ce[0][ls] = min(sh.ccount[0], (int)QC);
      sh.cs[1][lb] = 0;
      sh.ce[1][lb] = min(sh.ccount[1], (int)QC);
    }
    gsync<T>();
    // ---- cone, forward ball, level L -> L-1: scan the cone nodes' in-arcs,
    // or the out-arcs of level L-1 of the ball, whichever is fewer
    for (int L = ls; L >= 1 && !sh.ovf; --L) {
      const int a = sh.cs[0][L], b = sh.ce[0][L];
      const unsigned long long in_cone = bi_row_sum<T>(cl[0] + a, b - a, A.roff, sh);
      if (in_cone <= sh.hcost[0][L - 1]) {
        bi_scan<T>(cl[0] + a, b - a, A.roff, A.rcol, 8, heavy, sh, [&](int, int u) {
          const uint64_t su = bi_find(M, u);
          if (su && st_side(su) == 0 && st_level(su) == L - 1) bi_mark(M, sg, cl[0], 0, QC, sh, u);
        });
      } else {
        const int f0 = sh.lo[0][L - 1], f1 = sh.lo[0][L];
        bi_scan<T>(q[0] + f0, f1 - f0, A.off, A.col, bi_group(sh.hcost[0][L - 1], f1 - f0), heavy, sh,
                        [&](int u, int w) {
                          const uint64_t sw = bi_find(M, w);
                          if (sw && st_cone(sw) && st_side(sw) == 0 && st_level(sw) == L)
                            bi_mark(M, sg, cl[0], 0, QC, sh, u);
                        });
      }
      if (tid == 0) {
        sh.cs[0][L - 1] = b;
        sh.ce[0][L - 1] = min(sh.ccount[0], (int)QC);
      }
      gsync<T>();
    }
    // ---- cone, backward ball, level L -> L-1 (towards t): the cone nodes'
    // out-arcs, or the in-arcs of level L-1 of the ball
    for (int L = lb; L >= 1 && !sh.ovf; --L) {
      const int a = sh.cs[1][L], b = sh.ce[1][L];
      const unsigned long long out_cone = bi_row_sum<T>(cl[1] + a, b - a, A.off, sh);
      if (out_cone <= sh.hcost[1][L - 1]) {
        bi_scan<T>(cl[1] + a, b - a, A.off, A.col, 8, heavy, sh, [&](int, int y) {
          const uint64_t sy = bi_find(M, y);
          if (sy && st_side(sy) == 1 && st_level(sy) == L - 1) bi_mark(M, sg, cl[1], 1, QC, sh, y);
        });
      } else {
        const int f0 = sh.lo[1][L - 1], f1 = sh.lo[1][L];
        bi_scan<T>(q[1] + f0, f1 - f0, A.roff, A.rcol, bi_group(sh.hcost[1][L - 1], f1 - f0), heavy, sh,
                        [&](int y, int xv) {
                          const uint64_t sx = bi_find(M, xv);
                          if (sx && st_cone(sx) && st_side(sx) == 1 && st_level(sx) == L)
                            bi_mark(M, sg, cl[1], 1, QC, sh, y);
                        });
      }
      if (tid == 0) {
        sh.cs[1][L - 1] = b;
        sh.ce[1][L - 1] = min(sh.ccount[1], (int)QC);
      }
      gsync<T>();
    }
    if (sh.ovf) {
      gsync<T>();
      if (tid == 0) sh.status = 2;
    }
    gsync<T>();
  }
  if (sh.status == 0) {
    // ---- path counts over the cone, by distance D from s; each level is
    // pulled over the cone nodes' in-arcs or pushed over the out-arcs of
    // the level below, whichever is fewer; the crossing level adds along
    // the logged crossing arcs
    if (tid == 0) {
      int64_t is = 0;
      bi_find(M, sh.s, is);
      sg[is] = 1;
    }
    gsync<T>();
    for (int D = 1; D <= d && !sh.ovf; ++D) {
      const int x = D <= ls ? 0 : 1;
      const int L = x ? d - D : D;
      const int xp = D - 1 <= ls ? 0 : 1;
      const int Lp = xp ? d - (D - 1) : D - 1;
      const uint32_t *cur = cl[x] + sh.cs[x][L];
      const int ncur = sh.ce[x][L] - sh.cs[x][L];
      const uint32_t *prev = cl[xp] + sh.cs[xp][Lp];
      const int nprev = sh.ce[xp][Lp] - sh.cs[xp][Lp];
      if (D == ls + 1 && !sh.xovf) {
        int ovf = 0;
        for (int i = tid; i < ncross; i += T) {
          int64_t it = 0, ih = 0;
          bi_find(M, (int)xt[i], it);
          bi_find(M, (int)xh[i], ih);
          const unsigned long long add = sg[it];
          const unsigned long long old = atomicAdd((unsigned long long *)&sg[ih], add);
          ovf |= old + add < old;
        }
        if (ovf) sh.ovf = 1;
        gsync<T>();
        continue;
      }
      unsigned long long pull = 0, push = 0;
      bi_row_sum2<T>(cur, ncur, A.roff, prev, nprev, A.off, sh, &pull, &push);
      if (pull <= push) {
        bi_sigma_pull<T>(cur, ncur, D, d, M, sg, A.roff, A.rcol, 8, heavy, sh);
      } else {
        bi_scan<T>(prev, nprev, A.off, A.col, bi_group(push, nprev), heavy, sh, [&](int u, int w) {
          int64_t iw = 0;
          const uint64_t sw = bi_find(M, w, iw);
          if (sw && st_cone(sw) && st_dist(sw, d) == D) {
            int64_t iu = 0;
            bi_find(M, u, iu);
            const unsigned long long add = sg[iu];
            const unsigned long long old = atomicAdd((unsigned long long *)&sg[iw], add);
            if (old + add < old) sh.ovf = 1;
          }
        });
      }
    }
    gsync<T>();
    if (sh.ovf && tid == 0) sh.status = 2;
    gsync<T>();
  }
  if (sh.status == 0) {
    // ---- backward walk from t (one warp), the forward sampler's rule: at v
    // on distance L draw r below sigma_v and take the in-neighbour on L - 1
    // (ascending id) whose running count first exceeds r.  When the cone
    // level L - 1 has at most 32 nodes and v's row is long, the candidates
    // are those cone nodes with an arc into v, ranked by id.
    if (T == 32 || tid < 32) {
      int32_t v = sh.t;
      int64_t it = 0;
      bi_find(M, v, it);
      uint64_t sv = sg[it];
      int32_t *out = A.arena + sh.abase;
      uint32_t step = 0;
      unsigned long long scanned = 0;
      for (int L = d; L >= 2; --L, ++step) {
        const uint64_t r = uniform_below64(A.key.seed, A.key.id(j), kPurposeWalk0 + step, sv);
        const int xp = L - 1 <= ls ? 0 : 1;
        const int Lp = xp ? d - (L - 1) : L - 1;
        const int npc = sh.ce[xp][Lp] - sh.cs[xp][Lp];
        const int64_t e0 = A.roff[v], e1 = A.roff[v + 1];
        int32_t pick = -1;
        uint64_t pick_sig = 0;
        if (npc <= 32 && e1 - e0 > 64) {
          const uint32_t *pc = cl[xp] + sh.cs[xp][Lp];
          int32_t u = -1;
          uint64_t val = 0;
          if (lane < npc) {
            u = (int32_t)pc[lane];
            if (row_has(A.col, A.off[u], A.off[u + 1], v)) {
              int64_t iu = 0;
              bi_find(M, u, iu);
              val = sg[iu];
            }
            scanned += 16;
          }
          uint64_t pre = 0;  // counts of the candidates with smaller ids
          for (int k = 0; k < 32; ++k) {
            const int32_t uk = __shfl_sync(0xffffffffu, u, k);
            const uint64_t vk = __shfl_sync(0xffffffffu, val, k);
            if (vk != 0 && uk < u) pre += vk;
          }
          const unsigned hit = __ballot_sync(0xffffffffu, val != 0 && pre <= r && r - pre < val);
          if (hit) {
            const int src = __ffs(hit) - 1;
            pick = __shfl_sync(0xffffffffu, u, src);
            pick_sig = __shfl_sync(0xffffffffu, val, src);
          }
        } else {
          uint64_t cum = 0;
          for (int64_t base = e0; base < e1 && pick < 0; base += 32) {
            const int64_t i = base + lane;
            const int32_t u = i < e1 ? A.rcol[i] : -1;
            uint64_t val = 0;
            if (u >= 0) {
              int64_t iu = 0;
              const uint64_t su = bi_find(M, u, iu);
              if (su && st_cone(su) && st_dist(su, d) == L - 1) val = sg[iu];
            }
            uint64_t pre = val;
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              const uint64_t y = __shfl_up_sync(0xffffffffu, pre, o2);
              if (lane >= o2) pre += y;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, val != 0 && cum + pre > r);
            if (hit) {
              const int src = __ffs(hit) - 1;
              pick = __shfl_sync(0xffffffffu, u, src);
              pick_sig = __shfl_sync(0xffffffffu, val, src);
            } else {
              cum += __shfl_sync(0xffffffffu, pre, 31);
            }
            scanned += 32;
          }
        }
        if (pick < 0) {  // cannot happen with consistent counts
          if (lane == 0) atomicExch(&A.ctl->err, CEN_EINVAL);
          break;
        }
        if (lane == 0) out[L - 2] = pick;
        v = pick;
        sv = pick_sig;
      }
      if (lane == 0) {
        A.aoff[jr] = sh.abase;
        if (scanned) atomicAdd(&sh.arcs, scanned);
      }
    }
  } else if (tid == 0) {
    A.dwalk[atomicAdd(&A.ctl->nwalk, 1ull)] = j;
  }
  gsync<T>();
  return 0;
}

__device__ __forceinline__ BiWork cta_work(const BiArgs &A) {
  const int64_t QC = A.QC;
  uint32_t *lists = A.lists + (size_t)blockIdx.x * 7 * (size_t)QC;
  const uint32_t H1 = A.mask1 ? A.mask1 + 1 : 0, H2 = A.mask2 + 1;
  BiWork w;
  w.q[0] = lists;
  w.q[1] = lists + QC;
  w.cl[0] = lists + 2 * QC;
  w.cl[1] = lists + 3 * QC;
  w.heavy = lists + 4 * QC;
  w.xt = lists + 5 * QC;
  w.xh = lists + 6 * QC;
  w.QC = QC;
  w.sg = A.sig + (size_t)blockIdx.x * (size_t)H2;
  w.tab1 = H1 ? A.tab1 + (size_t)blockIdx.x * (size_t)H1 : nullptr;
  w.h1 = H1;
  w.tab2 = A.tab2 + (size_t)blockIdx.x * (size_t)H2;
  w.h2 = H2;
  w.epochs = A.epochs + 2 * (size_t)blockIdx.x;
  return w;
}

}  // namespace

// CTA searches, 16 CTAs of 128 threads per SM (32 registers): the kernel is
// bound by the latency of dependent L2 accesses, so samples in flight matter
// more than the few registers spilled.  LIST = false: every sample of the
// launch; LIST = true: the listed relative ids, their number read from
// *list_count when the launch starts (the warp kernel fills the list just
// before, on the same stream).
template <bool LIST>
__global__ void __launch_bounds__(kBiThreads, kBiCtaPerSM) k_bidir(BiArgs A) {
  __shared__ BiShCta sh;
  __shared__ unsigned long long s_item, s_arcs;
  const int tid = threadIdx.x;
  const BiWork cw = cta_work(A);
  const unsigned long long count = LIST ? *(volatile const unsigned long long *)A.list_count : A.count;
  if (tid == 0) s_arcs = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(LIST ? &A.ctl->bignext : &A.ctl->next, 1ull);
    __syncthreads();
    const unsigned long long i = s_item;
    if (i >= count) break;
    bi_search<kBiThreads, kBiMaxLevels>(A, sh, cw, LIST ? A.list[i] : i);
    if (tid == 0) s_arcs += sh.arcs;
  }
  if (tid == 0 && s_arcs) atomicAdd(A.units, s_arcs * 12ull);
}

// Warp searches: each warp of a 128-thread CTA takes sample ids and searches
// them alone in its own node table and lists.  A search that would expand a
// level of more than kWarpLevelArcs arcs, fills half of its table or its
// lists, or needs more than kWarpLevels levels on a side is handed on: its id
// is appended to the list the CTA kernel searches next.  Launched with no
// more CTAs than are resident at once; CTA b works in slot b's workspace.
__global__ void __launch_bounds__(kBiThreads, kBiWarpCtaPerSM) k_bidir_warp(BiArgs A) {
  __shared__ BiShWarp sh[kBiWarps];
  __shared__ unsigned long long s_arcs;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t WQ = A.WQ;
  uint32_t *wl = A.lists + (size_t)blockIdx.x * 7 * (size_t)A.QC + (size_t)wid * 7 * (size_t)WQ;
  BiWork ww;
  ww.q[0] = wl;
  ww.q[1] = wl + WQ;
  ww.cl[0] = wl + 2 * WQ;
  ww.cl[1] = wl + 3 * WQ;
  ww.heavy = wl + 4 * WQ;
  ww.xt = wl + 5 * WQ;
  ww.xh = wl + 6 * WQ;
  ww.QC = WQ;
  ww.sg = A.sig + (size_t)blockIdx.x * (size_t)(A.mask2 + 1) + (size_t)wid * kWarpTable;
  ww.tab1 = A.tabw + ((size_t)blockIdx.x * kBiWarps + wid) * kWarpTable;
  ww.h1 = kWarpTable;
  ww.tab2 = nullptr;
  ww.h2 = 0;
  ww.epochs = A.epw + 2 * ((size_t)blockIdx.x * kBiWarps + wid);
  if (tid == 0) s_arcs = 0;
  __syncthreads();
  unsigned long long arcs = 0;
  for (;;) {
    unsigned long long jr = 0;
    if (lane == 0) jr = atomicAdd(&A.ctl->next, 1ull);
    jr = __shfl_sync(0xffffffffu, jr, 0);
    if (jr >= A.count) break;
    const int r = bi_search<32, kWarpLevels>(A, sh[wid], ww, jr);
    if (lane == 0) {
      if (r == kSearchBig)
        A.big[atomicAdd(&A.ctl->nbig, 1ull)] = jr;
      else
        arcs += sh[wid].arcs;
    }
    __syncwarp();
  }
  if (lane == 0 && arcs) atomicAdd(&s_arcs, arcs);
  __syncthreads();
  if (tid == 0 && s_arcs) atomicAdd(A.units, s_arcs * 12ull);
}

// ------------------------------------------------------------------ host
int bidir_resident_slots() { return resident_grid((const void *)k_bidir<false>, kBiThreads); }

int64_t bidir_warp_queue(int64_t QC) {
  // each warp's seven lists fit a quarter of its CTA's; a warp search never
  // holds more than half of its table, so lists beyond that are not needed
  const int64_t wq = std::min<int64_t>(kWarpTable / 2, QC / kBiWarps);
  return wq >= 256 ? wq : 0;
}

size_t bidir_warp_table_bytes_per_slot() { return (size_t)kBiWarps * 8 * (size_t)kWarpTable; }
size_t bidir_warp_epoch_bytes_per_slot() { return (size_t)kBiWarps * 8; }  // two u32 epochs per warp
size_t bidir_warp_bytes_per_slot() { return bidir_warp_table_bytes_per_slot() + bidir_warp_epoch_bytes_per_slot(); }

namespace {
constexpr size_t kBiCacheMax = 4;
struct BiCache {
  std::mutex mu;
  std::vector<std::unique_ptr<BiWS>> idle;  // oldest first
};
// Never destroyed: nothing is freed after the CUDA runtime has unloaded.
BiCache &bi_cache() {
  static BiCache *c = new BiCache();
  return *c;
}
}  // namespace

std::unique_ptr<BiWS> bidir_take(int dev, int64_t QC, int64_t H1, int slots, int64_t WQ) {
  BiCache &c = bi_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  for (size_t i = c.idle.size(); i-- > 0;) {
    BiWS &w = *c.idle[i];
    if (w.dev == dev && w.QC == QC && w.H1 == H1 && w.nslots == slots && w.WQ == WQ) {
      std::unique_ptr<BiWS> out = std::move(c.idle[i]);
      c.idle.erase(c.idle.begin() + (ptrdiff_t)i);
      return out;
    }
  }
  return nullptr;
}

void bidir_give(std::unique_ptr<BiWS> w) {
  if (!w) return;
  // the job's stream may be gone before these buffers are: free them in order on the legacy stream
  for (DevBuf *b : {&w->tab1, &w->tab2, &w->lists, &w->sig, &w->epochs, &w->ctl, &w->aoff, &w->dsearch, &w->dwalk,
                    &w->arena, &w->tabw, &w->epw, &w->big})
    b->st = nullptr;
  BiCache &c = bi_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  c.idle.push_back(std::move(w));
  if (c.idle.size() > kBiCacheMax) c.idle.erase(c.idle.begin());
}

void bidir_drop_cached() {
  BiCache &c = bi_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  c.idle.clear();
}

namespace {
BiArgs bidir_args(cen_job *job, uint64_t j0, uint64_t count, int64_t arena_cap) {
  const cen_graph *g = job->g;
  BiWS &w = *job->bws;
  BiArgs a;
  a.n = g->n;
  a.off = g->off.as<int64_t>();
  a.col = g->col.as<int32_t>();
  a.roff = g->in_off();
  a.rcol = g->in_col();
  a.key = job->key();
  a.j0 = j0;
  a.count = count;
  a.tab1 = w.H1 ? w.tab1.as<uint64_t>() : nullptr;
  a.mask1 = w.H1 ? (uint32_t)(w.H1 - 1) : 0u;
  a.tab2 = w.tab2.as<uint64_t>();
  a.mask2 = (uint32_t)(w.H2 - 1);
  a.lists = w.lists.as<uint32_t>();
  a.sig = w.sig.as<uint64_t>();
  a.epochs = w.epochs.as<uint32_t>();
  a.QC = w.QC;
  a.tabw = w.WQ ? w.tabw.as<uint64_t>() : nullptr;
  a.epw = w.WQ ? w.epw.as<uint32_t>() : nullptr;
  a.WQ = w.WQ;
  a.big = w.big.as<uint64_t>();
  a.list = nullptr;
  a.list_count = nullptr;
  a.ps = job->ps.as<int32_t>();
  a.pt = job->pt.as<int32_t>();
  a.pd = job->pd.as<int32_t>();
  a.bmax = job->bmax.as<int>();
  a.arena = w.arena.as<int32_t>();
  a.arena_cap = arena_cap;
  a.aoff = w.aoff.as<int64_t>();
  a.dsearch = w.dsearch.as<uint64_t>();
  a.dwalk = w.dwalk.as<uint64_t>();
  a.ctl = w.ctl.as<BiCtl>();
  a.units = (unsigned long long *)(job->stats.d_units + K_BIDIR);
  return a;
}
}  // namespace

void bidir_launch(cen_job *job, uint64_t j0, uint64_t count, int64_t arena_cap) {
  BiWS &w = *job->bws;
  cudaStream_t st = job->st;
  CEN_CK(cudaMemsetAsync(w.ctl.p, 0, sizeof(BiCtl), st));
  BiArgs a = bidir_args(job, j0, count, arena_cap);
  const int grid = (int)std::min<uint64_t>((uint64_t)w.nslots, count);
  if (!w.WQ) {
    launch(&job->stats, K_BIDIR, st, [&] { k_bidir<false><<<grid, kBiThreads, 0, st>>>(a); });
    return;
  }
  // warp searches, then CTA searches of what they handed on (the list's
  // length is read on the device, so no host round trip separates the two)
  const int wgrid = std::max(1, std::min(grid, resident_grid((const void *)k_bidir_warp, kBiThreads)));
  launch(&job->stats, K_BIDIR, st, [&] { k_bidir_warp<<<wgrid, kBiThreads, 0, st>>>(a); });
  a.list = w.big.as<uint64_t>();
  a.list_count = &w.ctl.as<BiCtl>()->nbig;
  launch(&job->stats, K_BIDIR, st, [&] { k_bidir<true><<<grid, kBiThreads, 0, st>>>(a); });
}

}  // namespace cen
