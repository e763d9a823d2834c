/*
 * CentRA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what the CUDA path computes
 * for CentRA (Pellegrina, "Efficient Centrality Maximization with Rademacher
 * Averages", KDD'23), Algorithm 1 with the set-betweenness hyper-edge sampler of
 * Sec. 5.  Only the tests, the package's smoke check and the benchmark's CPU
 * baseline may load this library; the product path never does.  It shares no
 * code with the CUDA library.
 *
 * Readings of the paper that fix the free choices (each repeated at its use):
 *   - randomness: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *     (j_lo, j_hi, purpose, attempt) for sample j; integers by bitmask rejection;
 *   - pairs: s uniform in V, t uniform in V \ {s} (Sec. 3.1: u != v);
 *   - path: uniform over the s->t shortest paths, drawn by a backward walk
 *     from t that picks each predecessor w of v with probability
 *     sigma_sw / sigma_sv, scanning in-neighbours in ascending id order;
 *   - greedyCover: ties to the lowest node id; stops early at zero gain;
 *   - sign matrix: extended (never redrawn) across rounds, keyed by sample;
 *   - other spaces (kappa-path, triangle): see orc_job_new_space;
 *   - schedule: m_i = m0 * 2^(i-1) (doubling), or Sec. 4.2's growth by alpha
 *     with the optimistic guess (R = 0, nu = 1, target eta = eps C_{i-1} /
 *     (1 - 1/e), C_0 = 1); delta_i = delta / 2^i.
 *
 * Status codes match the CUDA library's public values.
 */
#ifndef CENTRA_ORACLE_H
#define CENTRA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EOVERFLOW (-4)
#define ORC_ENOTCERTIFIED (-5)

typedef struct orc_graph orc_graph;
typedef struct orc_job orc_job;

/* Philox4x32-10 block: out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Uniform integer in [0, B) for B = B_hi:B_lo >= 1 (128-bit), drawn for
 * sample j and the given purpose; returns the value in *r_hi:*r_lo and the
 * number of rejected attempts. */
int orc_uniform_below(uint64_t seed, uint64_t j, uint32_t purpose, uint64_t B_lo, uint64_t B_hi, uint64_t *r_lo,
                      uint64_t *r_hi);

/* The (s, t) pair of sample j on n >= 2 nodes. */
void orc_pair(uint64_t seed, uint64_t j, int32_t n, int32_t *s, int32_t *t);

/* Sign bits of sample j: t bits, bit q set <=> sigma_{q,j} = +1, packed into
 * ceil(t/32) little-endian 32-bit words. */
void orc_sign_words(uint64_t seed, uint64_t j, int32_t t, uint32_t *words);

/* Graph: canonical CSR (rows ascending, no duplicates, no self-loops). */
int orc_graph_new(int32_t n, int64_t nnz, const int64_t *off, const int32_t *col, int directed, orc_graph **out);
void orc_graph_free(orc_graph *g);

/* Single-source shortest-path counts from s, level-synchronous, stopping once
 * the level of t is complete (or the frontier empties).  dist[v] = -1 when
 * not reached; sigma as 128-bit (lo, hi); ovf[v] = 1 when sigma_sv >= 2^128.
 * Returns d(s,t) or -1. */
int32_t orc_sigma_bfs(const orc_graph *g, int32_t s, int32_t t, int32_t *dist, uint64_t *sig_lo, uint64_t *sig_hi,
                      uint8_t *ovf);

/* One hyper-edge: the interior nodes of a uniform shortest s->t path, s->t
 * order.  Writes s, t, d(s,t) (-1 unreachable), len, path[len] (capacity n).
 * Returns ORC_OK or ORC_EOVERFLOW (sigma_st >= 2^128). */
int orc_hyperedge(const orc_graph *g, uint64_t seed, uint64_t j, int32_t *s, int32_t *t, int32_t *d, int32_t *len,
                  int32_t *path);

/* Job: the growing sample H = (h_0, ..., h_{m-1}) of one CentRA run. */
int orc_job_new(const orc_graph *g, uint64_t seed, int32_t t, orc_job **out);
/* Hyper-edge spaces (Sec. 2): set betweenness (interior nodes of a uniform
 * shortest path between a uniform pair), kappa-path (the nodes after s of a
 * random simple walk of up to l steps, l uniform in 1..kappa), triangle (the
 * three nodes of a uniform triangle; undirected graphs with a triangle only).
 * The copied s, t, d of a sample are (s, t, d(s,t)), (s, l, steps taken) and
 * the triangle's nodes in ascending order.  See oracle.c for the draws. */
#define ORC_SPACE_BETWEENNESS 0
#define ORC_SPACE_KPATH 1
#define ORC_SPACE_TRIANGLE 2
int orc_job_new_space(const orc_graph *g, uint64_t seed, int32_t t, int32_t space, int32_t kappa, orc_job **out);
/* Triangles of an undirected graph: their number, and the one of rank r in
 * (u, v, w) order with u < v < w. */
int64_t orc_triangle_count(const orc_graph *g);
int orc_triangle_unrank(const orc_graph *g, int64_t r, int32_t *u, int32_t *v, int32_t *w);
void orc_job_free(orc_job *job);
int orc_job_sample(orc_job *job, uint64_t m_new);      /* append samples [m, m+m_new) */
/* append the samples with ids j_first .. j_first+count-1 (shards by sample index) */
int orc_job_sample_from(orc_job *job, uint64_t j_first, uint64_t count);
uint64_t orc_job_m(const orc_job *job);
int64_t orc_job_members(const orc_job *job);           /* sum of |h| */
/* copy out hoff[m+1], hmem[members], and per-sample s, t, d (any may be NULL) */
void orc_job_copy(const orc_job *job, int64_t *hoff, int32_t *hmem, int32_t *s, int32_t *t, int32_t *d);
/* Store count samples (ids j_first ..) drawn by another job of the same graph,
 * seed and space, e.g. in another process; hoff[count+1] starts at 0. */
int orc_job_append(orc_job *job, uint64_t j_first, uint64_t count, const int64_t *hoff, const int32_t *hmem,
                   const int32_t *s, const int32_t *t, const int32_t *d);
/* algorithmic-work tallies of all samples drawn so far:
 * [0] nodes reached at levels < d(s,t), [1] arcs scanned out of levels < d(s,t)-1,
 * [2] in-arcs scanned by the backward walks, [3] path members written */
void orc_job_work(const orc_job *job, uint64_t out[4]);

/* greedyCover(k, H): S[<=k] in pick order, |S|, covered sample count. */
int orc_greedy_cover(const orc_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered);

/* AMCERA numerators: Rnum[q] = sum of the <=k largest positive
 * R_q^u = sum_{s: u in h_s} sigma_{q,s} (integer, = m * r_q^u); Wnum = sum of
 * the k largest c_u = |{s: u in h_s}|; b = max |h|. */
int orc_mcera(const orc_job *job, int32_t k, int64_t *Rnum, int64_t *Wnum, int32_t *b);
/* the raw R matrix, R[u * t + q], and c[u] (for element-wise parity) */
int orc_rade_matrix(const orc_job *job, int32_t *R, int32_t *c);

/* Host FP64 bounds of Theorem 4.4 and the stopping test of
 * Algorithm 1 for iteration i >= 1 (delta_i = delta / 2^i).
 * Pinned at generic inputs against the proofs' own steps: nu and R are the
 * largest fixed points of the self-bounding tail inversions, R~ inverts the
 * hypercube tail at the flip-sum bound 4 t m w~ (reached on a tight sample),
 * and eta is Bousquet's inequality at E[Z] = 2R with variance nu.
 * out[0..7] = C, A (AMCERA), w (wimpy), nu, xi, Rtilde, R, eta; returns stop (0/1). */
int orc_bounds(uint64_t covered, uint64_t m, int64_t Rsum, int32_t t, int64_t Wnum, int32_t b, double eps,
               double delta, int32_t i, double *out);

/* Algorithm 1 end to end.  S_out has capacity k; log rows (capacity
 * max_rounds x 16 doubles): i, m_i, covered, Rsum, Wnum, b, C, A, w, nu, xi,
 * Rt, R, eta, stop, |S|.  Returns ORC_OK when certified, ORC_ENOTCERTIFIED when
 * the next m would exceed m_cap, or another error. */
int orc_run(const orc_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
            uint64_t m_cap, int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final, int32_t *rounds,
            double *log, int32_t max_rounds);

/* Sampling schedule (Sec. 4.2): 0 = doubling from m0; 1 = the paper's
 * geometric growth by alpha combined with the optimistic guess; 2 = schedule 1
 * plus m_pred, the smallest size at which the next round's stopping test
 * passes if C and w hold and the AMCERA shrinks as 1/sqrt(m) (see oracle.c). */
double orc_schedule_guess(double C, double eps, double delta, int32_t i);
uint64_t orc_schedule_next(int32_t schedule, double alpha, uint64_t m0, uint64_t m_prev, double C_prev,
                           uint64_t m_pred, double eps, double delta, int32_t i);
/* HEDGE-P bounds (union bound over n^k sets of a Bernstein tail; see oracle.c):
 * out[0..3] = C, L_U, nu_U, eta_U; returns 1 iff eta_U <= eps (C - eta_U) / 2. */
int orc_bounds_hedge(uint64_t covered, uint64_t m, int32_t n, int32_t k, double eps, double delta, int32_t i,
                     double *out);
/* Algorithm 1 with a schedule and a stopping rule: rule 0 = CentRA (AMCERA and
 * Thm. 4.4), rule 1 = HEDGE-P (orc_bounds_hedge; no AMCERA; the log's
 * C, nu and eta columns hold C, nu_U, eta_U and the AMCERA columns are 0). */
int orc_run_ex(const orc_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
               uint64_t m_cap, int32_t schedule, double alpha, int32_t rule, int32_t space, int32_t kappa,
               int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final, int32_t *rounds, double *log,
               int32_t max_rounds);

#ifdef __cplusplus
}
#endif
#endif
