/*
 * Seeded synthetic graph generators (inputs only; no part of the sampling,
 * covering or bounding arithmetic lives here).
 *
 * The paper evaluates on SNAP/KONECT graphs (Table 1, Sec. 5) that
 * are not available offline; these generators produce stand-ins with the same
 * shape: Barabasi-Albert preferential attachment, R-MAT (Chakrabarti et al.),
 * and a 4-neighbour grid with a fraction of its edges rewired.
 *
 * Every generator emits a canonical CSR: rows sorted ascending, no duplicate
 * arcs, no self-loops; undirected graphs store both arcs of every edge.
 * Randomness: splitmix64 (Steele, Lea, Flood 2014), seeded per call.
 * Host-portable C (x86_64 and aarch64 give identical output).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG */
typedef struct { uint64_t s; } gen_rng;

static uint64_t rng_next(gen_rng *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* uniform integer in [0, b), b >= 1, by rejection on the top bits */
static uint64_t rng_below(gen_rng *r, uint64_t b) {
  if (b <= 1) return 0;
  uint64_t lim = UINT64_MAX - (UINT64_MAX % b);
  for (;;) {
    uint64_t x = rng_next(r);
    if (x < lim) return x % b;
  }
}
static double rng_unit(gen_rng *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------ edge list -> CSR */
/* Builds a canonical CSR from arcs (src[i] -> dst[i]).  If undirected, both
 * directions are inserted.  Self-loops and duplicates are dropped.  Writes
 * off[n+1]; returns the arc count and stores a malloc'd col array in *col_out
 * (caller frees with gen_free). */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int64_t build_csr(int32_t n, int64_t ne, const int32_t *src, const int32_t *dst, int undirected,
                         int64_t *off, int32_t **col_out) {
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < ne; ++i) {
    if (src[i] == dst[i]) continue;
    cnt[src[i] + 1]++;
    if (undirected) cnt[dst[i] + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  int64_t total = cnt[n];
  int32_t *tmp = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < ne; ++i) {
    if (src[i] == dst[i]) continue;
    tmp[pos[src[i]]++] = dst[i];
    if (undirected) tmp[pos[dst[i]]++] = src[i];
  }
  free(pos);
  /* sort rows and dedup in place */
  int64_t w = 0;
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t b = cnt[v], e = cnt[v + 1];
    if (e - b > 1) qsort(tmp + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    int32_t last = -1;
    for (int64_t i = b; i < e; ++i) {
      if (tmp[i] == last) continue;
      last = tmp[i];
      tmp[w++] = tmp[i];
    }
    off[v + 1] = w;
  }
  free(cnt);
  *col_out = tmp;
  return w;
}

void gen_free(void *p) { free(p); }

/* -------------------------------------------------- Barabasi-Albert */
/* Start from the complete graph on d+1 nodes; every later node v attaches d
 * distinct targets drawn proportionally to degree (uniform over a list holding
 * each edge's two endpoints), rejecting repeats.  n >= d+1, d >= 1.
 * Returns the arc count (2 x edges); *col_out malloc'd. */
int64_t gen_ba(int32_t n, int32_t d, uint64_t seed, int64_t *off, int32_t **col_out) {
  if (d < 1 || n < d + 1) return -1;
  gen_rng r = {seed};
  int64_t ne_max = (int64_t)d * (d + 1) / 2 + (int64_t)(n - d - 1) * d;
  int32_t *src = (int32_t *)malloc((size_t)ne_max * sizeof(int32_t));
  int32_t *dst = (int32_t *)malloc((size_t)ne_max * sizeof(int32_t));
  int32_t *ends = (int32_t *)malloc((size_t)ne_max * 2 * sizeof(int32_t));
  int32_t *pick = (int32_t *)malloc((size_t)d * sizeof(int32_t));
  int64_t ne = 0, nends = 0;
  for (int32_t a = 0; a <= d; ++a)
    for (int32_t b = a + 1; b <= d; ++b) {
      src[ne] = a; dst[ne] = b; ++ne;
      ends[nends++] = a; ends[nends++] = b;
    }
  for (int32_t v = d + 1; v < n; ++v) {
    int32_t got = 0;
    while (got < d) {
      int32_t c = ends[rng_below(&r, (uint64_t)nends)];
      int dup = 0;
      for (int32_t q = 0; q < got; ++q) dup |= (pick[q] == c);
      if (!dup) pick[got++] = c;
    }
    for (int32_t q = 0; q < d; ++q) {
      src[ne] = v; dst[ne] = pick[q]; ++ne;
      ends[nends++] = v; ends[nends++] = pick[q];
    }
  }
  int64_t nnz = build_csr(n, ne, src, dst, 1, off, col_out);
  free(src); free(dst); free(ends); free(pick);
  return nnz;
}

/* ------------------------------------------------------------ R-MAT */
/* ef * 2^scale edge draws; each draw descends `scale` quadrant choices with
 * probabilities (a, b, c, 1-a-b-c), no noise.  Writes raw (src, dst) arrays of
 * length ef * 2^scale into caller buffers. */
void gen_rmat_edges(int32_t scale, int64_t ne, double a, double b, double c, uint64_t seed, int32_t *src,
                    int32_t *dst) {
  gen_rng r = {seed};
  double ab = a + b, abc = a + b + c;
  for (int64_t i = 0; i < ne; ++i) {
    uint32_t u = 0, v = 0;
    for (int32_t l = 0; l < scale; ++l) {
      double x = rng_unit(&r);
      uint32_t ub, vb;
      if (x < a) { ub = 0; vb = 0; }
      else if (x < ab) { ub = 0; vb = 1; }
      else if (x < abc) { ub = 1; vb = 0; }
      else { ub = 1; vb = 1; }
      u = (u << 1) | ub;
      v = (v << 1) | vb;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}

/* Canonical CSR from raw arcs (exported so Python can build from any list). */
int64_t gen_csr_from_edges(int32_t n, int64_t ne, const int32_t *src, const int32_t *dst, int undirected,
                           int64_t *off, int32_t **col_out) {
  return build_csr(n, ne, src, dst, undirected, off, col_out);
}

/* Largest connected component of an undirected canonical CSR (ties: the
 * component holding the smallest node id).  Writes keep[v] = new id or -1,
 * relabelling kept nodes in ascending original id order; returns its size. */
int32_t gen_lcc(int32_t n, const int64_t *off, const int32_t *col, int32_t *keep) {
  int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int32_t v = 0; v < n; ++v) comp[v] = -1;
  int32_t best = -1, best_size = 0, ncomp = 0;
  for (int32_t r0 = 0; r0 < n; ++r0) {
    if (comp[r0] >= 0) continue;
    int32_t head = 0, tail = 0;
    queue[tail++] = r0;
    comp[r0] = ncomp;
    while (head < tail) {
      int32_t v = queue[head++];
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        int32_t w = col[e];
        if (comp[w] < 0) { comp[w] = ncomp; queue[tail++] = w; }
      }
    }
    if (tail > best_size) { best_size = tail; best = ncomp; }
    ++ncomp;
  }
  int32_t nid = 0;
  for (int32_t v = 0; v < n; ++v) keep[v] = (comp[v] == best) ? nid++ : -1;
  free(comp); free(queue);
  return nid;
}

/* Induced subgraph on keep[] (new ids), canonical CSR.  Returns arc count. */
int64_t gen_induce(int32_t n, const int64_t *off, const int32_t *col, const int32_t *keep, int32_t n_new,
                   int64_t *off_new, int32_t **col_out) {
  int64_t cnt = 0;
  for (int32_t v = 0; v < n; ++v)
    if (keep[v] >= 0)
      for (int64_t e = off[v]; e < off[v + 1]; ++e) cnt += (keep[col[e]] >= 0);
  int32_t *c = (int32_t *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int32_t));
  int64_t w = 0;
  off_new[0] = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (keep[v] < 0) continue;
    for (int64_t e = off[v]; e < off[v + 1]; ++e)
      if (keep[col[e]] >= 0) c[w++] = keep[col[e]]; /* monotone relabel keeps rows sorted */
    off_new[keep[v] + 1] = w;
  }
  (void)n_new;
  *col_out = c;
  return w;
}

/* ------------------------------------------------ rewired 2-D grid */
/* Open-addressing set of undirected edges keyed by (min << 32 | max). */
typedef struct { uint64_t *slot; uint64_t mask; } eset;
#define ESET_EMPTY UINT64_MAX
static uint64_t ekey(uint32_t u, uint32_t v) { return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u; }
static uint64_t ehash(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
  return k;
}
static int eset_has(const eset *s, uint64_t k) {
  for (uint64_t h = ehash(k) & s->mask;; h = (h + 1) & s->mask) {
    if (s->slot[h] == k) return 1;
    if (s->slot[h] == ESET_EMPTY) return 0;
  }
}
static void eset_put(eset *s, uint64_t k) {
  uint64_t h = ehash(k) & s->mask;
  while (s->slot[h] != ESET_EMPTY && s->slot[h] != k) h = (h + 1) & s->mask;
  s->slot[h] = k;
}
/* tombstone-free delete (backward shift) */
static void eset_del(eset *s, uint64_t k) {
  uint64_t h = ehash(k) & s->mask;
  while (s->slot[h] != k) {
    if (s->slot[h] == ESET_EMPTY) return;
    h = (h + 1) & s->mask;
  }
  uint64_t i = h;
  for (;;) {
    s->slot[i] = ESET_EMPTY;
    uint64_t j = i;
    for (;;) {
      j = (j + 1) & s->mask;
      if (s->slot[j] == ESET_EMPTY) return;
      uint64_t home = ehash(s->slot[j]) & s->mask;
      /* can slot j move to i?  yes if home is not cyclically in (i, j] */
      int in_range = (i <= j) ? (home > i && home <= j) : (home > i || home <= j);
      if (!in_range) break;
    }
    s->slot[i] = s->slot[j];
    i = j;
  }
}

/* W x H 4-neighbour grid, node id = y*W + x.  Every edge, independently with
 * probability p, keeps one endpoint (fair coin) and gets the other replaced
 * by a uniform node, redrawn while that would make a self-loop or duplicate. */
int64_t gen_grid_rewired(int32_t W, int32_t H, double p, uint64_t seed, int64_t *off, int32_t **col_out) {
  int64_t n = (int64_t)W * H;
  int64_t ne = (int64_t)(W - 1) * H + (int64_t)W * (H - 1);
  int32_t *src = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
  int32_t *dst = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
  int64_t e = 0;
  for (int32_t y = 0; y < H; ++y)
    for (int32_t x = 0; x < W; ++x) {
      int32_t v = y * W + x;
      if (x + 1 < W) { src[e] = v; dst[e] = v + 1; ++e; }
      if (y + 1 < H) { src[e] = v; dst[e] = v + W; ++e; }
    }
  uint64_t cap = 1;
  while (cap < (uint64_t)ne * 2) cap <<= 1;
  eset s = {(uint64_t *)malloc(cap * sizeof(uint64_t)), cap - 1};
  for (uint64_t i = 0; i < cap; ++i) s.slot[i] = ESET_EMPTY;
  for (int64_t i = 0; i < ne; ++i) eset_put(&s, ekey((uint32_t)src[i], (uint32_t)dst[i]));
  gen_rng r = {seed};
  for (int64_t i = 0; i < ne; ++i) {
    if (rng_unit(&r) >= p) continue;
    int32_t keepv = (rng_next(&r) & 1) ? dst[i] : src[i];
    int32_t nv;
    do {
      nv = (int32_t)rng_below(&r, (uint64_t)n);
    } while (nv == keepv || eset_has(&s, ekey((uint32_t)keepv, (uint32_t)nv)));
    eset_del(&s, ekey((uint32_t)src[i], (uint32_t)dst[i]));
    src[i] = keepv;
    dst[i] = nv;
    eset_put(&s, ekey((uint32_t)keepv, (uint32_t)nv));
  }
  free(s.slot);
  int64_t nnz = build_csr((int32_t)n, ne, src, dst, 1, off, col_out);
  free(src); free(dst);
  return nnz;
}

/* Draw parameters that the batched workload needs (n, attachment, k) from the
 * same generator family so Python and C agree across machines. */
void gen_draw_u64(uint64_t seed, int64_t count, uint64_t *out) {
  gen_rng r = {seed};
  for (int64_t i = 0; i < count; ++i) out[i] = rng_next(&r);
}
