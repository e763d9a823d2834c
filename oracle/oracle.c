/*
 * CentRA oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain single-threaded C: every step is the definition it cites, in the order
 * the paper states it, with no blocking, fusion or reordering.  Path counts are
 * 128-bit with a saturating overflow flag; all other arithmetic on samples is
 * integer; only orc_bounds uses FP64 (compile with -ffp-contract=off).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
#define U128_MAX (~(u128)0)

/* ------------------------------------------------------------------ RNG */
/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words 0
 * and 2 by the round constants, mixes the high halves with words 1 and 3 and
 * the key, and the key is bumped by the Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void block_for(uint64_t seed, uint64_t j, uint32_t purpose, uint32_t word3, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), purpose, word3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* Uniform integer below B by bitmask rejection: mask = 2^ceil(log2 B) - 1;
 * attempt a = 0, 1, ... draws block (j, purpose, a); the candidate is the low
 * 64 bits (128 bits when B > 2^64) of the block under the mask; the first
 * candidate < B is returned.  (The paper only says "uniformly at random".) */
static u128 uniform_below(uint64_t seed, uint64_t j, uint32_t purpose, u128 B, uint32_t *attempts) {
  int bits = 0;
  while (bits < 128 && (((u128)1 << bits) < B)) ++bits; /* smallest bits with 2^bits >= B */
  u128 mask = (bits == 128) ? U128_MAX : (((u128)1 << bits) - 1);
  int wide = B > ((u128)1 << 64);
  for (uint32_t a = 0;; ++a) {
    uint32_t x[4];
    block_for(seed, j, purpose, a, x);
    u128 v = (u128)x[0] | ((u128)x[1] << 32);
    if (wide) v |= ((u128)x[2] << 64) | ((u128)x[3] << 96);
    v &= mask;
    if (v < B) {
      if (attempts) *attempts = a;
      return v;
    }
  }
}

int orc_uniform_below(uint64_t seed, uint64_t j, uint32_t purpose, uint64_t B_lo, uint64_t B_hi, uint64_t *r_lo,
                      uint64_t *r_hi) {
  u128 B = ((u128)B_hi << 64) | B_lo;
  if (B == 0) return ORC_EINVAL;
  uint32_t att = 0;
  u128 r = uniform_below(seed, j, purpose, B, &att);
  *r_lo = (uint64_t)r;
  *r_hi = (uint64_t)(r >> 64);
  return (int)att;
}

#define PURPOSE_S 0u
#define PURPOSE_T 1u
#define PURPOSE_WALK0 2u
#define PURPOSE_SIGN 0xFFFFFFFFu

/* Sec. 5: "a starting node u and final node v uniformly at random"; the
 * hyper-edge space of Sec. 3.1 ranges over u != v, so t is drawn from the
 * n-1 other nodes. */
void orc_pair(uint64_t seed, uint64_t j, int32_t n, int32_t *s, int32_t *t) {
  int32_t a = (int32_t)uniform_below(seed, j, PURPOSE_S, (u128)(uint32_t)n, NULL);
  int32_t b = (int32_t)uniform_below(seed, j, PURPOSE_T, (u128)(uint32_t)(n - 1), NULL);
  *s = a;
  *t = b + (b >= a);
}

/* Alg. 1 "sampleRadeVars": the t entries sigma_{q,j} of column j, one bit each
 * (set = +1), from blocks (j, SIGN, blk) for blk = 0 .. ceil(t/128)-1. */
void orc_sign_words(uint64_t seed, uint64_t j, int32_t t, uint32_t *words) {
  int32_t nw = (t + 31) / 32;
  for (int32_t w = 0; w < nw; ++w) {
    uint32_t x[4];
    block_for(seed, j, PURPOSE_SIGN, (uint32_t)(w / 4), x);
    uint32_t v = x[w % 4];
    int32_t hi = t - 32 * w;
    if (hi < 32) v &= (1u << hi) - 1u;
    words[w] = v;
  }
}

static int sign_bit(const uint32_t *words, int32_t q) { return (words[q >> 5] >> (q & 31)) & 1u; }

/* ---------------------------------------------------------------- graph */
struct orc_graph {
  int32_t n;
  int64_t nnz;
  int directed;
  int64_t *off;  /* out-arcs */
  int32_t *col;
  int64_t *roff; /* in-arcs (== out-arcs when undirected) */
  int32_t *rcol;
};

int orc_graph_new(int32_t n, int64_t nnz, const int64_t *off, const int32_t *col, int directed, orc_graph **out) {
  if (n < 2 || nnz < 0 || off[0] != 0 || off[n] != nnz) return ORC_EINVAL;
  for (int32_t v = 0; v < n; ++v) {
    if (off[v + 1] < off[v]) return ORC_EINVAL;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      if (col[e] < 0 || col[e] >= n || col[e] == v) return ORC_EINVAL;
      if (e > off[v] && col[e] <= col[e - 1]) return ORC_EINVAL;
    }
  }
  orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
  g->n = n;
  g->nnz = nnz;
  g->directed = directed ? 1 : 0;
  g->off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  memcpy(g->off, off, sizeof(int64_t) * ((size_t)n + 1));
  memcpy(g->col, col, sizeof(int32_t) * (size_t)nnz);
  if (!directed) {
    g->roff = g->off;
    g->rcol = g->col;
  } else {
    /* in-CSR: the transpose, rows ascending (scanning sources in order keeps each row sorted) */
    g->roff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->rcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t e = 0; e < nnz; ++e) g->roff[col[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) g->roff[v + 1] += g->roff[v];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(pos, g->roff, sizeof(int64_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v)
      for (int64_t e = off[v]; e < off[v + 1]; ++e) g->rcol[pos[col[e]]++] = v;
    free(pos);
  }
  *out = g;
  return ORC_OK;
}

void orc_graph_free(orc_graph *g) {
  if (!g) return;
  if (g->directed) {
    free(g->roff);
    free(g->rcol);
  }
  free(g->off);
  free(g->col);
  free(g);
}

/* ------------------------------------------------------- sigma-BFS */
/* Level-synchronous BFS from s (Brandes-style path counting): level L+1 is
 * every unreached out-neighbour of level L; then each new node w gets
 * sigma_w = sum of sigma_v over in-neighbours v at level L (pull order,
 * ascending ids).  Stops after the level holding t is complete, or when the
 * frontier is empty (t unreachable: Sec. 5 returns the empty set). */
typedef struct {
  int32_t *dist;
  u128 *sig;
  uint8_t *ovf;
  int32_t *q0, *q1;
  uint64_t reached_lt_d, arcs_expanded; /* work tallies, see orc_job_work */
} bfs_ws;

static int32_t sigma_bfs(const orc_graph *g, int32_t s, int32_t t, bfs_ws *w) {
  int32_t n = g->n;
  for (int32_t v = 0; v < n; ++v) {
    w->dist[v] = -1;
    w->sig[v] = 0;
    w->ovf[v] = 0;
  }
  w->dist[s] = 0;
  w->sig[s] = 1;
  int32_t *cur = w->q0, *nxt = w->q1;
  int32_t ncur = 1, level = 0;
  cur[0] = s;
  /* per-level sizes kept to tally the minimal work after d(s,t) is known */
  uint64_t reached_by_level_sum = 1; /* nodes at levels <= level */
  uint64_t arcs_out_of_levels_lt = 0; /* arcs out of levels < level */
  uint64_t tally_reached = 0, tally_arcs = 0;
  while (ncur > 0 && w->dist[t] < 0) {
    int32_t nnext = 0;
    uint64_t arcs_this = 0;
    for (int32_t i = 0; i < ncur; ++i) {
      int32_t v = cur[i];
      arcs_this += (uint64_t)(g->off[v + 1] - g->off[v]);
      for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
        int32_t x = g->col[e];
        if (w->dist[x] < 0) {
          w->dist[x] = level + 1;
          nxt[nnext++] = x;
        }
      }
    }
    for (int32_t i = 0; i < nnext; ++i) {
      int32_t x = nxt[i];
      u128 acc = 0;
      uint8_t of = 0;
      for (int64_t e = g->roff[x]; e < g->roff[x + 1]; ++e) {
        int32_t v = g->rcol[e];
        if (w->dist[v] != level) continue;
        if (w->ovf[v] || acc > U128_MAX - w->sig[v]) {
          of = 1;
          acc = U128_MAX;
        } else {
          acc += w->sig[v];
        }
      }
      w->sig[x] = acc;
      w->ovf[x] = of;
    }
    /* tallies: when t is found at level+1, the reached set below d is levels
     * 0..level and the arcs that must be scanned are those out of levels < level */
    if (w->dist[t] >= 0) {
      tally_reached = reached_by_level_sum;
      tally_arcs = arcs_out_of_levels_lt;
    }
    reached_by_level_sum += (uint64_t)nnext;
    arcs_out_of_levels_lt += arcs_this;
    int32_t *tmp = cur;
    cur = nxt;
    nxt = tmp;
    ncur = nnext;
    ++level;
  }
  if (w->dist[t] < 0) { /* unreachable: the whole component was explored */
    tally_reached = reached_by_level_sum;
    tally_arcs = arcs_out_of_levels_lt;
  }
  w->reached_lt_d += tally_reached;
  w->arcs_expanded += tally_arcs;
  return w->dist[t];
}

static int bfs_ws_init(bfs_ws *w, int32_t n) {
  memset(w, 0, sizeof(*w));
  w->dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  w->sig = (u128 *)malloc(sizeof(u128) * (size_t)n);
  w->ovf = (uint8_t *)malloc((size_t)n);
  w->q0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  w->q1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  return (w->dist && w->sig && w->ovf && w->q0 && w->q1) ? ORC_OK : ORC_ENOMEM;
}

static void bfs_ws_free(bfs_ws *w) {
  free(w->dist); free(w->sig); free(w->ovf); free(w->q0); free(w->q1);
}

int32_t orc_sigma_bfs(const orc_graph *g, int32_t s, int32_t t, int32_t *dist, uint64_t *sig_lo, uint64_t *sig_hi,
                      uint8_t *ovf) {
  bfs_ws w;
  if (bfs_ws_init(&w, g->n) != ORC_OK) {
    bfs_ws_free(&w);
    return -2;
  }
  int32_t d = sigma_bfs(g, s, t, &w);
  for (int32_t v = 0; v < g->n; ++v) {
    if (dist) dist[v] = w.dist[v];
    if (sig_lo) sig_lo[v] = (uint64_t)w.sig[v];
    if (sig_hi) sig_hi[v] = (uint64_t)(w.sig[v] >> 64);
    if (ovf) ovf[v] = w.ovf[v];
  }
  bfs_ws_free(&w);
  return d;
}

/* ------------------------------------------------------- backward walk */
/* From v = t, step l = 0, 1, ...: r = uniform below sigma_v (purpose 2+l);
 * scan v's in-neighbours w in ascending id with dist_w = dist_v - 1, adding
 * sigma_w, and move to the first w whose running sum exceeds r.  Each
 * predecessor w is taken with probability sigma_w / sigma_v, so the whole walk
 * yields each shortest s->t path with probability 1 / sigma_st.  The interior
 * nodes (all but s and t) form the hyper-edge of Sec. 3.1, in s->t order. */
static int walk_back(const orc_graph *g, uint64_t seed, uint64_t j, int32_t s, int32_t t, const bfs_ws *w,
                     int32_t *path, int32_t *len, uint64_t *arcs_scanned) {
  int32_t d = w->dist[t];
  if (w->ovf[t]) return ORC_EOVERFLOW;
  int32_t v = t, pos = d - 1; /* interior nodes occupy path[0 .. d-2] */
  uint32_t step = 0;
  while (v != s) {
    u128 r = uniform_below(seed, j, PURPOSE_WALK0 + step, w->sig[v], NULL);
    u128 cum = 0;
    int32_t pick = -1;
    for (int64_t e = g->roff[v]; e < g->roff[v + 1]; ++e) {
      int32_t x = g->rcol[e];
      ++*arcs_scanned;
      if (w->dist[x] != w->dist[v] - 1) continue;
      cum += w->sig[x];
      if (cum > r) {
        pick = x;
        break;
      }
    }
    if (pick < 0) return ORC_EINVAL; /* unreachable for a correct sigma */
    if (pick != s) path[--pos] = pick;
    v = pick;
    ++step;
  }
  *len = d - 1;
  return ORC_OK;
}

static int hyperedge_ws(const orc_graph *g, uint64_t seed, uint64_t j, bfs_ws *w, int32_t *s, int32_t *t, int32_t *d,
                        int32_t *len, int32_t *path, uint64_t *walk_arcs) {
  orc_pair(seed, j, g->n, s, t);
  *d = sigma_bfs(g, *s, *t, w);
  *len = 0;
  if (*d < 0) return ORC_OK;
  return walk_back(g, seed, j, *s, *t, w, path, len, walk_arcs);
}

int orc_hyperedge(const orc_graph *g, uint64_t seed, uint64_t j, int32_t *s, int32_t *t, int32_t *d, int32_t *len,
                  int32_t *path) {
  bfs_ws w;
  if (bfs_ws_init(&w, g->n) != ORC_OK) {
    bfs_ws_free(&w);
    return ORC_ENOMEM;
  }
  uint64_t arcs = 0;
  int rc = hyperedge_ws(g, seed, j, &w, s, t, d, len, path, &arcs);
  bfs_ws_free(&w);
  return rc;
}

/* ------------------------------------------------------------------ job */
/* ------------------------------------------------- other hyper-edge spaces */
/* kappa-path centrality (Sec. 2: "sets of nodes traversed by simple paths of
 * length at most kappa").  Reading: s uniform over V (purpose 0), a length
 * l uniform in 1..kappa (purpose 1), then a random simple walk from s of up
 * to l steps: at step i the walk moves to the r-th (ascending id) out-neighbour
 * of the current node not yet on the walk, r uniform below their number
 * (purpose 2 + i), and stops early when there is none.  The hyper-edge is the
 * nodes after s, in walk order (at most kappa of them, the paper's b <= kappa).
 * Writes s, l, the steps taken and the path; returns the path length. */
static int32_t kpath_walk(const orc_graph *g, uint64_t seed, uint64_t j, int32_t kappa, int32_t *s_out,
                          int32_t *l_out, int32_t *path, uint64_t *arcs) {
  const int32_t s = (int32_t)uniform_below(seed, j, PURPOSE_S, (u128)(uint32_t)g->n, NULL);
  const int32_t l = 1 + (int32_t)uniform_below(seed, j, PURPOSE_T, (u128)(uint32_t)kappa, NULL);
  int32_t len = 0, cur = s;
  for (int32_t i = 0; i < l; ++i) {
    int64_t free_nb = 0;
    for (int64_t e = g->off[cur]; e < g->off[cur + 1]; ++e) {
      int32_t w = g->col[e], seen = (w == s);
      for (int32_t q = 0; q < len && !seen; ++q) seen = (path[q] == w);
      free_nb += !seen;
    }
    *arcs += (uint64_t)(g->off[cur + 1] - g->off[cur]);
    if (free_nb == 0) break;
    int64_t r = (int64_t)uniform_below(seed, j, PURPOSE_WALK0 + (uint32_t)i, (u128)(uint64_t)free_nb, NULL);
    int32_t next = -1;
    for (int64_t e = g->off[cur]; e < g->off[cur + 1] && next < 0; ++e) {
      int32_t w = g->col[e], seen = (w == s);
      for (int32_t q = 0; q < len && !seen; ++q) seen = (path[q] == w);
      if (!seen && r-- == 0) next = w;
    }
    path[len++] = next;
    cur = next;
  }
  *s_out = s;
  *l_out = l;
  return len;
}

/* Triangle centrality (Sec. 2: "sets of nodes incident to triangles of G").
 * Reading: a triangle {u, v, w} of the undirected graph drawn uniformly; its
 * three nodes are the hyper-edge, in ascending order.  Triangles are ranked
 * by (u, v, w) with u < v < w: off[e] (the exclusive prefix over arcs e = (u,v)
 * in CSR order of the number of common neighbours w > v when v > u, else 0)
 * ranks the first triangle on arc e, and within the arc the common
 * neighbours ascend.  r uniform below the total (purpose 0) is unranked. */
static int64_t common_above(const orc_graph *g, int32_t u, int32_t v, int32_t *w_out, int64_t rank) {
  int64_t a = g->off[u], ae = g->off[u + 1], b = g->off[v], be = g->off[v + 1], c = 0;
  while (a < ae && b < be) {
    if (g->col[a] < g->col[b]) ++a;
    else if (g->col[a] > g->col[b]) ++b;
    else {
      if (g->col[a] > v) {
        if (w_out && c == rank) {
          *w_out = g->col[a];
          return c;
        }
        ++c;
      }
      ++a;
      ++b;
    }
  }
  return c;
}

static int64_t *triangle_offsets(const orc_graph *g) {
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)g->nnz + 1));
  if (!off) return NULL;
  int64_t acc = 0;
  for (int32_t u = 0; u < g->n; ++u)
    for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
      off[e] = acc;
      if (g->col[e] > u) acc += common_above(g, u, g->col[e], NULL, -1);
    }
  off[g->nnz] = acc;
  return off;
}

/* the triangle of rank r (0 <= r < off[nnz]) */
static void triangle_unrank(const orc_graph *g, const int64_t *off, int64_t r, int32_t *u, int32_t *v, int32_t *w) {
  int64_t lo = 0, hi = g->nnz; /* last arc e with off[e] <= r and a triangle on it */
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (off[mid] <= r) lo = mid; else hi = mid;
  }
  while (off[lo + 1] == off[lo]) ++lo; /* arcs without triangles share the prefix */
  int32_t a = 0, b = g->n; /* the row holding arc lo */
  while (b - a > 1) {
    int32_t mid = a + (b - a) / 2;
    if (g->off[mid] <= lo) a = mid; else b = mid;
  }
  *u = a;
  *v = g->col[lo];
  common_above(g, a, *v, w, r - off[lo]);
}

int64_t orc_triangle_count(const orc_graph *g) {
  if (!g || g->directed) return -1;
  int64_t *off = triangle_offsets(g);
  if (!off) return -1;
  int64_t T = off[g->nnz];
  free(off);
  return T;
}

int orc_triangle_unrank(const orc_graph *g, int64_t r, int32_t *u, int32_t *v, int32_t *w) {
  if (!g || g->directed) return ORC_EINVAL;
  int64_t *off = triangle_offsets(g);
  if (!off) return ORC_ENOMEM;
  int rc = ORC_OK;
  if (r < 0 || r >= off[g->nnz]) rc = ORC_EINVAL;
  else triangle_unrank(g, off, r, u, v, w);
  free(off);
  return rc;
}

struct orc_job {
  const orc_graph *g;
  uint64_t seed;
  int32_t t;
  uint64_t m;
  uint64_t next_id; /* sample id of the next appended sample (= m unless a range was requested) */
  uint64_t *ids;    /* sample id of each stored sample */
  uint64_t cap_m;
  int64_t *hoff;     /* [m+1] */
  int32_t *hmem;     /* [hoff[m]] */
  int64_t cap_mem;
  int32_t *ps, *pt, *pd;
  uint64_t work[4];
  int32_t space, kappa; /* hyper-edge space (ORC_SPACE_*) and the path bound of the kappa-path space */
  int64_t *tri_off;     /* triangle space: exclusive prefix of per-arc triangle counts ([nnz+1]) */
};

int orc_job_new(const orc_graph *g, uint64_t seed, int32_t t, orc_job **out) {
  return orc_job_new_space(g, seed, t, ORC_SPACE_BETWEENNESS, 0, out);
}

int orc_job_new_space(const orc_graph *g, uint64_t seed, int32_t t, int32_t space, int32_t kappa, orc_job **out) {
  if (!g || t < 1) return ORC_EINVAL;
  if (space != ORC_SPACE_BETWEENNESS && space != ORC_SPACE_KPATH && space != ORC_SPACE_TRIANGLE) return ORC_EINVAL;
  if (space == ORC_SPACE_KPATH && (kappa < 1 || kappa > 1024)) return ORC_EINVAL;
  int64_t *tri_off = NULL;
  if (space == ORC_SPACE_TRIANGLE) {
    if (g->directed) return ORC_EINVAL;
    tri_off = triangle_offsets(g);
    if (!tri_off) return ORC_ENOMEM;
    if (tri_off[g->nnz] == 0) { /* no triangle to draw */
      free(tri_off);
      return ORC_EINVAL;
    }
  }
  orc_job *job = (orc_job *)calloc(1, sizeof(orc_job));
  job->g = g;
  job->seed = seed;
  job->t = t;
  job->space = space;
  job->kappa = kappa;
  job->tri_off = tri_off;
  job->cap_m = 1024;
  job->hoff = (int64_t *)calloc(job->cap_m + 1, sizeof(int64_t));
  job->ps = (int32_t *)malloc(sizeof(int32_t) * job->cap_m);
  job->pt = (int32_t *)malloc(sizeof(int32_t) * job->cap_m);
  job->pd = (int32_t *)malloc(sizeof(int32_t) * job->cap_m);
  job->ids = (uint64_t *)malloc(sizeof(uint64_t) * job->cap_m);
  job->cap_mem = 4096;
  job->hmem = (int32_t *)malloc(sizeof(int32_t) * (size_t)job->cap_mem);
  *out = job;
  return ORC_OK;
}

void orc_job_free(orc_job *job) {
  if (!job) return;
  free(job->hoff); free(job->hmem); free(job->ps); free(job->pt); free(job->pd); free(job->ids);
  free(job->tri_off);
  free(job);
}

uint64_t orc_job_m(const orc_job *job) { return job->m; }

/* Shards by sample index: append the samples with ids j_first .. j_first+count-1
 * (the store keeps them in id order after any earlier ones). */
int orc_job_sample_from(orc_job *job, uint64_t j_first, uint64_t count) {
  job->next_id = j_first;
  return orc_job_sample(job, count);
}
int64_t orc_job_members(const orc_job *job) { return job->hoff[job->m]; }

/* Stores `count` samples with ids j_first .. j_first+count-1 that another job
 * of the same graph, seed and space drew (plumbing for computing index ranges
 * in several processes: a sample is a function of its id).  hoff[count+1] is
 * relative to hmem[0]; the work tallies are not carried over. */
int orc_job_append(orc_job *job, uint64_t j_first, uint64_t count, const int64_t *hoff, const int32_t *hmem,
                   const int32_t *s, const int32_t *t, const int32_t *d) {
  if (!hoff || (count && (!s || !t || !d)) || hoff[0] != 0) return ORC_EINVAL;
  int64_t add = hoff[count];
  if (job->m + count > job->cap_m) {
    while (job->m + count > job->cap_m) job->cap_m *= 2;
    job->hoff = (int64_t *)realloc(job->hoff, sizeof(int64_t) * (job->cap_m + 1));
    job->ps = (int32_t *)realloc(job->ps, sizeof(int32_t) * job->cap_m);
    job->pt = (int32_t *)realloc(job->pt, sizeof(int32_t) * job->cap_m);
    job->pd = (int32_t *)realloc(job->pd, sizeof(int32_t) * job->cap_m);
    job->ids = (uint64_t *)realloc(job->ids, sizeof(uint64_t) * job->cap_m);
  }
  int64_t base = job->hoff[job->m];
  if (base + add > job->cap_mem) {
    while (base + add > job->cap_mem) job->cap_mem *= 2;
    job->hmem = (int32_t *)realloc(job->hmem, sizeof(int32_t) * (size_t)job->cap_mem);
  }
  if (!job->hoff || !job->ps || !job->pt || !job->pd || !job->ids || !job->hmem) return ORC_ENOMEM;
  if (add) memcpy(job->hmem + base, hmem, sizeof(int32_t) * (size_t)add);
  for (uint64_t q = 0; q < count; ++q) {
    uint64_t j = job->m + q;
    job->hoff[j + 1] = base + hoff[q + 1];
    job->ps[j] = s[q];
    job->pt[j] = t[q];
    job->pd[j] = d[q];
    job->ids[j] = j_first + q;
  }
  job->m += count;
  job->next_id = j_first + count;
  return ORC_OK;
}

void orc_job_copy(const orc_job *job, int64_t *hoff, int32_t *hmem, int32_t *s, int32_t *t, int32_t *d) {
  if (hoff) memcpy(hoff, job->hoff, sizeof(int64_t) * (size_t)(job->m + 1));
  if (hmem) memcpy(hmem, job->hmem, sizeof(int32_t) * (size_t)job->hoff[job->m]);
  if (s) memcpy(s, job->ps, sizeof(int32_t) * (size_t)job->m);
  if (t) memcpy(t, job->pt, sizeof(int32_t) * (size_t)job->m);
  if (d) memcpy(d, job->pd, sizeof(int32_t) * (size_t)job->m);
}

void orc_job_work(const orc_job *job, uint64_t out[4]) { memcpy(out, job->work, sizeof(job->work)); }

/* Alg. 1 line "sampleHEs(H, m_i - m_{i-1})": append hyper-edges in index order. */
int orc_job_sample(orc_job *job, uint64_t m_new) {
  const orc_graph *g = job->g;
  bfs_ws w;
  int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
  if (bfs_ws_init(&w, g->n) != ORC_OK || !path) {
    bfs_ws_free(&w);
    free(path);
    return ORC_ENOMEM;
  }
  int rc = ORC_OK;
  for (uint64_t q = 0; q < m_new && rc == ORC_OK; ++q) {
    uint64_t j = job->m;
    if (j + 1 > job->cap_m) {
      job->cap_m *= 2;
      job->hoff = (int64_t *)realloc(job->hoff, sizeof(int64_t) * (job->cap_m + 1));
      job->ps = (int32_t *)realloc(job->ps, sizeof(int32_t) * job->cap_m);
      job->pt = (int32_t *)realloc(job->pt, sizeof(int32_t) * job->cap_m);
      job->pd = (int32_t *)realloc(job->pd, sizeof(int32_t) * job->cap_m);
      job->ids = (uint64_t *)realloc(job->ids, sizeof(uint64_t) * job->cap_m);
    }
    int32_t s, t, d, len;
    uint64_t walk_arcs = 0;
    const uint64_t jid = job->next_id;
    w.reached_lt_d = 0;
    w.arcs_expanded = 0;
    if (job->space == ORC_SPACE_KPATH) {
      /* s: start, t: drawn length l, d: steps taken */
      len = kpath_walk(g, job->seed, jid, job->kappa, &s, &t, path, &walk_arcs);
      d = len;
    } else if (job->space == ORC_SPACE_TRIANGLE) {
      /* s, t, d: the triangle's nodes, ascending */
      const int64_t r = (int64_t)uniform_below(job->seed, jid, PURPOSE_S, (u128)(uint64_t)job->tri_off[g->nnz], NULL);
      triangle_unrank(g, job->tri_off, r, &s, &t, &d);
      path[0] = s;
      path[1] = t;
      path[2] = d;
      len = 3;
    } else {
      rc = hyperedge_ws(g, job->seed, jid, &w, &s, &t, &d, &len, path, &walk_arcs);
      if (rc != ORC_OK) break;
    }
    int64_t base = job->hoff[j];
    if (base + len > job->cap_mem) {
      while (base + len > job->cap_mem) job->cap_mem *= 2;
      job->hmem = (int32_t *)realloc(job->hmem, sizeof(int32_t) * (size_t)job->cap_mem);
    }
    memcpy(job->hmem + base, path, sizeof(int32_t) * (size_t)len);
    job->hoff[j + 1] = base + len;
    job->ps[j] = s;
    job->pt[j] = t;
    job->pd[j] = d;
    job->ids[j] = jid;
    job->next_id = jid + 1;
    job->work[0] += w.reached_lt_d;
    job->work[1] += w.arcs_expanded;
    job->work[2] += walk_arcs;
    job->work[3] += (uint64_t)len;
    job->m = j + 1;
  }
  bfs_ws_free(&w);
  free(path);
  return rc;
}

/* --------------------------------------------------------- greedyCover */
/* Sec. 3.1 "greedyCover(k, H)": k times insert u* = argmax_u C_H(S + {u}).
 * C_H(S + {u}) = C_H(S) + (uncovered samples holding u)/m, so the argmax is
 * the node with most uncovered samples; the marginal counts are recomputed
 * from scratch each iteration.  Ties go to the lowest id; an iteration whose
 * best gain is 0 ends the loop (|S| <= k). */
int orc_greedy_cover(const orc_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered) {
  if (k < 1) return ORC_EINVAL;
  int32_t n = job->g->n;
  uint64_t m = job->m;
  uint8_t *cov = (uint8_t *)calloc(m > 0 ? m : 1, 1);
  uint64_t *gain = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  uint64_t ncov = 0;
  int32_t size = 0;
  for (int32_t it = 0; it < k; ++it) {
    memset(gain, 0, sizeof(uint64_t) * (size_t)n);
    for (uint64_t j = 0; j < m; ++j) {
      if (cov[j]) continue;
      for (int64_t e = job->hoff[j]; e < job->hoff[j + 1]; ++e) gain[job->hmem[e]]++;
    }
    int32_t best = 0;
    for (int32_t u = 1; u < n; ++u)
      if (gain[u] > gain[best]) best = u;
    if (gain[best] == 0) break;
    S[size++] = best;
    for (uint64_t j = 0; j < m; ++j) {
      if (cov[j]) continue;
      for (int64_t e = job->hoff[j]; e < job->hoff[j + 1]; ++e)
        if (job->hmem[e] == best) {
          cov[j] = 1;
          ++ncov;
          break;
        }
    }
  }
  free(cov);
  free(gain);
  *S_size = size;
  *covered = ncov;
  return ORC_OK;
}

/* ---------------------------------------------------------------- AMCERA */
/* Alg. 1 lines "r_j^u" and "r_j": with integer numerators R_q^u = m r_q^u =
 * sum over samples s holding u of sigma_{q,s}. */
int orc_rade_matrix(const orc_job *job, int32_t *R, int32_t *c) {
  int32_t n = job->g->n, t = job->t;
  uint32_t *words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)((t + 31) / 32));
  memset(R, 0, sizeof(int32_t) * (size_t)n * (size_t)t);
  memset(c, 0, sizeof(int32_t) * (size_t)n);
  for (uint64_t j = 0; j < job->m; ++j) {
    orc_sign_words(job->seed, job->ids[j], t, words);
    for (int64_t e = job->hoff[j]; e < job->hoff[j + 1]; ++e) {
      int32_t u = job->hmem[e];
      c[u] += 1;
      for (int32_t q = 0; q < t; ++q) R[(size_t)u * t + q] += sign_bit(words, q) ? 1 : -1;
    }
  }
  free(words);
  return ORC_OK;
}

static int cmp_desc_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x < y) - (x > y);
}

/* sup over |S'| <= k of sum_{u in S'} r_q^u is the sum of the <= k largest
 * positive entries (the objective is additive in S', and the empty set gives
 * 0); the wimpy variance's sup (Sec. 4.1, f_u^2 = f_u) is the sum of the k
 * largest c_u, times b_H = max |h|. */
int orc_mcera(const orc_job *job, int32_t k, int64_t *Rnum, int64_t *Wnum, int32_t *b) {
  if (k < 1) return ORC_EINVAL;
  int32_t n = job->g->n, t = job->t;
  int32_t *R = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)t);
  int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *vals = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!R || !c || !vals) {
    free(R); free(c); free(vals);
    return ORC_ENOMEM;
  }
  orc_rade_matrix(job, R, c);
  for (int32_t q = 0; q < t; ++q) {
    int32_t cnt = 0;
    for (int32_t u = 0; u < n; ++u)
      if (R[(size_t)u * t + q] > 0) vals[cnt++] = R[(size_t)u * t + q];
    qsort(vals, (size_t)cnt, sizeof(int64_t), cmp_desc_i64);
    int64_t sum = 0;
    for (int32_t i = 0; i < cnt && i < k; ++i) sum += vals[i];
    Rnum[q] = sum;
  }
  for (int32_t u = 0; u < n; ++u) vals[u] = c[u];
  qsort(vals, (size_t)n, sizeof(int64_t), cmp_desc_i64);
  int64_t w = 0;
  for (int32_t i = 0; i < n && i < k; ++i) w += vals[i];
  *Wnum = w;
  int32_t bmax = 0;
  for (uint64_t j = 0; j < job->m; ++j) {
    int32_t len = (int32_t)(job->hoff[j + 1] - job->hoff[j]);
    if (len > bmax) bmax = len;
  }
  *b = bmax;
  free(R); free(c); free(vals);
  return ORC_OK;
}

/* ---------------------------------------------------------------- bounds */
/* Theorem 4.4 (Eq. 2) with ln(5/delta_i), and Alg. 1's xi and
 * stopping test, in this evaluation order (a = 1 - 1/e, L = ln(5/delta_i),
 * Lm = L/m):
 *   C   = covered / m
 *   A   = Rsum / (t m)                 (AMCERA, Alg. 1 line "r_j" average)
 *   w   = (b Wnum) / m                 (approximate wimpy variance, Sec. 4.1)
 *   xi  = sqrt(Lm Lm + (2 C L) / (a m)) + Lm          (Alg. 1 line "xi")
 *   nu  = C / a + xi                                  (Thm. 4.4)
 *   Rt  = A + sqrt((4 w L) / (t m))
 *   R   = Rt + sqrt(Lm Lm + (2 L Rt) / m) + Lm
 *   eta = 2 R + sqrt((2 L (nu + 4 R)) / m) + L / (3 m)
 *   stop  <=>  a ((a - eps) xi + eta) <= eps C        (Alg. 1 stopping line)
 */
/* Thm. 4.4 from the sample's fractions C, A, w at sample size md and
 * L = ln(5 / delta_i); out[3..7] = nu, xi, Rtilde, R, eta. */
static void bounds_from_fractions(double C, double A, double w, int32_t t, double md, double L, double *out) {
  double a = 1.0 - exp(-1.0);
  double Lm = L / md;
  double xi = sqrt(Lm * Lm + (2.0 * C * L) / (a * md)) + Lm;
  double nu = C / a + xi;
  double Rt = A + sqrt((4.0 * w * L) / ((double)t * md));
  double R = Rt + sqrt(Lm * Lm + (2.0 * L * Rt) / md) + Lm;
  double eta = 2.0 * R + sqrt((2.0 * L * (nu + 4.0 * R)) / md) + L / (3.0 * md);
  out[3] = nu; out[4] = xi; out[5] = Rt; out[6] = R; out[7] = eta;
}

int orc_bounds(uint64_t covered, uint64_t m, int64_t Rsum, int32_t t, int64_t Wnum, int32_t b, double eps,
               double delta, int32_t i, double *out) {
  double a = 1.0 - exp(-1.0);
  double md = (double)m;
  double delta_i = ldexp(delta, -i);
  double L = log(5.0 / delta_i);
  double C = (double)covered / md;
  double A = (double)Rsum / ((double)t * md);
  double w = ((double)b * (double)Wnum) / md;
  out[0] = C; out[1] = A; out[2] = w;
  bounds_from_fractions(C, A, w, t, md, L, out);
  return (a * ((a - eps) * out[4] + out[7]) <= eps * C) ? 1 : 0;
}

/* HEDGE-P (Sec. 6, progressive HEDGE): a union bound over the at most n^k
 * sets of size <= k of a two-sided Bernstein (Chernoff-type) tail for each
 * set's coverage, i.i.d. 0/1 terms of mean C(S) and variance
 * C(S)(1 - C(S)) <= min(C(S*), 1/4).  With L_U = k ln n + ln(2 / delta_i),
 * every set deviates by at most lam(v) = b + sqrt(b^2 + 2 v L_U / m),
 * b = L_U / (3 m), the root of m lam^2 = L_U (2 v + 2 lam / 3).  C(S*) is
 * unknown; on the same event C(S*) <= C_H(S*) + lam(C(S*)) <= C / (1 - 1/e) +
 * lam(C(S*)) (the greedy set keeps a 1 - 1/e share of the sample optimum), so
 * C(S*) is at most the larger root nu_U of u = C / (1 - 1/e) + lam(u).  The SD
 * bound is eta_U = lam(min(nu_U, 1/4)).  HEDGE's sufficient condition is
 * SD <= eps C(S*) / 2; since C(S*) >= C(S) >= C - SD, it holds once
 * eta_U <= eps (C - eta_U) / 2.
 * out[0..3] = C, L_U, nu_U, eta_U; returns stop (0/1). */
/* eta_U and nu_U from the coverage fraction C at sample size md; out[2], out[3] */
static void hedge_from_fraction(double C, double md, double LU, double *out) {
  double a = 1.0 - exp(-1.0);
  double Lm = LU / md;
  double b = LU / (3.0 * md);
  double c0 = C / a + b;
  /* (u - c0)^2 = b^2 + 2 u Lm, larger root */
  double nu = c0 + Lm + sqrt(2.0 * c0 * Lm + Lm * Lm + b * b);
  double v = nu < 0.25 ? nu : 0.25;
  out[2] = nu;
  out[3] = b + sqrt(b * b + 2.0 * v * Lm);
}

static double hedge_L(int32_t n, int32_t k, double delta, int32_t i) {
  return (double)k * log((double)n) + log(2.0 / ldexp(delta, -i));
}

int orc_bounds_hedge(uint64_t covered, uint64_t m, int32_t n, int32_t k, double eps, double delta, int32_t i,
                     double *out) {
  double md = (double)m;
  double C = (double)covered / md;
  out[0] = C;
  out[1] = hedge_L(n, k, delta, i);
  hedge_from_fraction(C, md, out[1], out);
  return (out[3] <= eps * (C - out[3]) / 2.0) ? 1 : 0;
}

/* The prediction of the extrapolating schedule: would round i's stopping test
 * pass at sample size mp if the coverage fraction C and the wimpy-variance
 * fraction w stayed as measured at m and the AMCERA shrank as 1/sqrt(m)?
 * (rule 0; rule 1 keeps C only). */
static int predicted_stop(int32_t rule, double C, double A, double w, int32_t t, int32_t n, int32_t k, uint64_t m,
                          uint64_t mp, double eps, double delta, int32_t i) {
  double a = 1.0 - exp(-1.0);
  double md = (double)mp;
  double o[8];
  if (rule == 0) {
    double Ap = A * sqrt((double)m / md);
    bounds_from_fractions(C, Ap, w, t, md, log(5.0 / ldexp(delta, -i)), o);
    return a * ((a - eps) * o[4] + o[7]) <= eps * C;
  }
  hedge_from_fraction(C, md, hedge_L(n, k, delta, i), o);
  return o[3] <= eps * (C - o[3]) / 2.0;
}

/* Smallest mp > m at which predicted_stop holds (bisection after doubling),
 * or 0 when none up to 2^40 does (then the prediction is not used). */
static uint64_t predict_m(int32_t rule, double C, double A, double w, int32_t t, int32_t n, int32_t k, uint64_t m,
                          double eps, double delta, int32_t i) {
  if (!(C > 0.0)) return 0;
  uint64_t lo = m, hi = 2 * m;
  while (!predicted_stop(rule, C, A, w, t, n, k, m, hi, eps, delta, i)) {
    if (hi >= ((uint64_t)1 << 40)) return 0;
    lo = hi;
    hi = 2 * hi;
  }
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (predicted_stop(rule, C, A, w, t, n, k, m, mid, eps, delta, i)) hi = mid; else lo = mid;
  }
  return hi;
}

/* ------------------------------------------------------------- Alg. 1 */
/* Sec. 4.2 "samplingSchedule", optimistic part: Thm. 4.4 with R = 0
 * and nu = 1 leaves eta(m) = sqrt(2 L / m) + L / (3 m); the smallest m with
 * eta(m) <= eps C / (1 - 1/e) (the stopping test when xi is negligible) solves
 * (L/3) y^2 + sqrt(2 L) y - target = 0 for y = 1/sqrt(m).  Returns 0 when C = 0
 * (no finite guess).  Evaluation order is part of the reading. */
double orc_schedule_guess(double C, double eps, double delta, int32_t i) {
  double a = 1.0 - exp(-1.0);
  double L = log(5.0 / ldexp(delta, -i));
  double target = eps * C / a;
  if (!(target > 0.0)) return 0.0;
  double A3 = L / 3.0;
  double B = sqrt(2.0 * L);
  double y = (sqrt(B * B + 4.0 * A3 * target) - B) / (2.0 * A3);
  return 1.0 / (y * y);
}

/* Next sample size of the schedule for round i.  Schedule 0 doubles from m0.
 * Schedule 1 (Sec. 4.2): round 1 is max(m0, ceil(guess(C = 1))); round i > 1
 * is max(ceil(alpha m_{i-1}), ceil(guess(C_{i-1}))).  Schedule 2 also takes
 * m_pred (> 0), the size at which round i's stopping test is predicted to
 * pass from round i-1's summary (predict_m).  Every schedule grows by at least
 * one sample. */
uint64_t orc_schedule_next(int32_t schedule, double alpha, uint64_t m0, uint64_t m_prev, double C_prev,
                           uint64_t m_pred, double eps, double delta, int32_t i) {
  if (schedule == 0) return i == 1 ? m0 : 2 * m_prev;
  double grow = i == 1 ? (double)m0 : ceil(alpha * (double)m_prev);
  double guess = ceil(orc_schedule_guess(i == 1 ? 1.0 : C_prev, eps, delta, i));
  double m = grow > guess ? grow : guess;
  if (schedule == 2 && i > 1 && m_pred > 0 && (double)m_pred > m) m = (double)m_pred;
  if (i > 1 && m <= (double)m_prev) m = (double)m_prev + 1.0;
  return m >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)m;
}

int orc_run(const orc_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
            uint64_t m_cap, int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final, int32_t *rounds,
            double *log, int32_t max_rounds) {
  return orc_run_ex(g, k, eps, delta, t, seed, m0, m_cap, 0, 2.0, 0, 0, 0, S_out, S_size, covered, m_final, rounds,
                    log, max_rounds);
}

int orc_run_ex(const orc_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
               uint64_t m_cap, int32_t schedule, double alpha, int32_t rule, int32_t space, int32_t kappa,
               int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final, int32_t *rounds, double *log,
               int32_t max_rounds) {
  double a = 1.0 - exp(-1.0);
  if (!g || k < 1 || t < 1 || !(eps > 0.0 && eps < a) || !(delta > 0.0 && delta < 1.0) || m0 < 1 || m_cap < m0 ||
      schedule < 0 || schedule > 2 || (schedule != 0 && !(alpha > 1.0)) || (rule != 0 && rule != 1))
    return ORC_EINVAL;
  orc_job *job;
  int rc = orc_job_new_space(g, seed, t, space, kappa, &job);
  if (rc) return rc;
  int64_t *Rnum = (int64_t *)malloc(sizeof(int64_t) * (size_t)t);
  uint64_t m_prev = 0;
  uint64_t m_i = orc_schedule_next(schedule, alpha, m0, 0, 1.0, 0, eps, delta, 1);
  int32_t i = 0;
  rc = ORC_ENOTCERTIFIED;
  if (m_i > m_cap) m_i = m_cap;
  for (;;) {
    ++i;
    int r = orc_job_sample(job, m_i - m_prev);
    if (r) { rc = r; break; }
    uint64_t cov;
    r = orc_greedy_cover(job, k, S_out, S_size, &cov);
    if (r) { rc = r; break; }
    int64_t Wnum = 0, Rsum = 0;
    int32_t b = 0;
    double bd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int stop;
    if (rule == 0) {
      r = orc_mcera(job, k, Rnum, &Wnum, &b);
      if (r) { rc = r; break; }
      for (int32_t q = 0; q < t; ++q) Rsum += Rnum[q];
      stop = orc_bounds(cov, m_i, Rsum, t, Wnum, b, eps, delta, i, bd);
    } else {
      /* HEDGE-P: no AMCERA; the log keeps C, nu_U and eta_U in the C, nu and eta columns */
      double hb[4];
      stop = orc_bounds_hedge(cov, m_i, g->n, k, eps, delta, i, hb);
      bd[0] = hb[0]; bd[3] = hb[2]; bd[7] = hb[3];
    }
    if (log && i <= max_rounds) {
      double *row = log + (size_t)(i - 1) * 16;
      row[0] = i; row[1] = (double)m_i; row[2] = (double)cov; row[3] = (double)Rsum; row[4] = (double)Wnum;
      row[5] = b;
      for (int q = 0; q < 8; ++q) row[6 + q] = bd[q];
      row[14] = stop; row[15] = *S_size;
    }
    *covered = cov;
    *m_final = m_i;
    *rounds = i;
    if (stop) { rc = ORC_OK; break; }
    uint64_t m_pred = schedule == 2 ? predict_m(rule, bd[0], bd[1], bd[2], t, g->n, k, m_i, eps, delta, i + 1) : 0;
    uint64_t next = orc_schedule_next(schedule, alpha, m0, m_i, bd[0], m_pred, eps, delta, i + 1);
    if (next > m_cap) { rc = ORC_ENOTCERTIFIED; break; } /* next m would exceed m_cap */
    m_prev = m_i;
    m_i = next;
  }
  free(Rnum);
  orc_job_free(job);
  return rc;
}
