/*
 * cen.h -- C ABI of the GB300 CentRA sample-and-cover library (libcen.so).
 *
 * CentRA (Pellegrina, "Efficient Centrality Maximization with Rademacher
 * Averages", KDD'23) approximates the size-k node set of maximum set
 * betweenness: it draws random shortest paths (hyper-edges), runs greedy
 * max-coverage on them, bounds the supremum deviation with Monte Carlo
 * Rademacher averages, and doubles the sample until its stopping rule certifies
 * a (1 - 1/e - eps)-approximation with probability >= 1 - delta (Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Return value: int status, CEN_OK (0) or a negative CEN_E* code; the
 *     message of the last failure on the calling thread is in cen_last_error().
 *     No C++ exception crosses this boundary.
 *   - Node ids are int32 in [0, n); CSR offsets are int64.
 *   - Pointers documented as "host" must be host memory; "device" must be
 *     device memory of the current CUDA device.  Output arrays are owned by
 *     the caller; every handle is owned by the library until its _free call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     returns only after its GPU work on that stream is complete.
 *   - A job handle is not thread-safe; distinct jobs may be used from distinct
 *     threads.  All device memory is allocated by the library, stream-ordered.
 *   - Randomness is Philox4x32-10 keyed by the job seed with counter
 *     (j_lo, j_hi, purpose, attempt) for sample j: results depend only on
 *     (graph, seed, parameters), never on launch configuration or timing.
 */
#ifndef CEN_H
#define CEN_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CEN_OK 0
#define CEN_EINVAL (-1)        /* bad argument or malformed graph */
#define CEN_ENOMEM (-2)        /* device allocation failed */
#define CEN_ECUDA (-3)         /* a CUDA runtime call or kernel failed */
#define CEN_EOVERFLOW (-4)     /* a sampled pair has >= 2^128 shortest paths */
#define CEN_ENOTCERTIFIED (-5) /* cen_run: the next sample size would exceed m_cap */

#define CEN_LOG_COLS 16 /* per-round log row, see cen_run */

typedef struct cen_graph cen_graph;
typedef struct cen_job cen_job;

/* Device memory (no counterpart in the paper).  The library owns every
 * device buffer it allocates (graph copies, samples, workspaces); arrays the
 * caller passes stay the caller's.  By default buffers come from the device's
 * stream-ordered pool (cudaMallocAsync on the call's stream).
 * cen_set_allocator installs another source for the allocations made after it: alloc(bytes, stream, ctx) returns
 * device memory for use on `stream` (null: the call fails with CEN_ENOMEM),
 * and free(ptr, bytes, stream, ctx) takes back a buffer that alloc made,
 * called only once `stream` has drained, so the memory is idle and may be
 * handed out again at once.  A buffer always goes back to the allocator that
 * made it, so an installed pair (and ctx) must stay valid until every graph
 * and job is freed and cen_release_cached has run.  alloc = free = null
 * restores the pool.  Both must be null or both set (else CEN_EINVAL).  Do not
 * call it while another thread is inside the library. */
typedef void *(*cen_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*cen_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int cen_set_allocator(cen_alloc_fn alloc, cen_free_fn free_fn, void *ctx);

/* Library version (major * 10000 + minor * 100 + patch). */
int cen_version(void);

/* Text of the last failure on the calling thread ("" if none). */
const char *cen_last_error(void);

/* Graph G = (V, E) of Sec. 3.1, as a canonical CSR: off[n+1] (int64, off[0] =
 * 0, nondecreasing, off[n] = nnz), col[nnz] (int32), every row strictly
 * ascending, no self-loops.  Undirected graphs list both arcs of each edge
 * and set directed = 0; directed graphs list out-arcs.  `on_device` says
 * whether off/col are device (1) or host (0) pointers; they are copied, the
 * caller keeps them.  The copy is validated on the GPU; a malformed CSR gives
 * CEN_EINVAL.  n >= 2.  For directed graphs the in-arc CSR is built on the GPU. */
int cen_graph_load(const int64_t *off, const int32_t *col, int32_t n, int64_t nnz, int directed, int on_device,
                   void *stream, cen_graph **out);
/* cen_graph_load from any CSR with ids in [0, n) and offsets rising from 0 to
 * nnz (else CEN_EINVAL).  The paper takes G as given (Sec. 3.1); this builds
 * the canonical form above from raw input.  flags:
 *   CEN_GRAPH_CANONICALIZE  sort each row, drop repeated arcs and self-loops;
 *   CEN_GRAPH_SYMMETRIZE    (undirected only) add the reverse of every arc
 *                           first, then canonicalize.
 * Done on the GPU (two stable radix sorts of the arc list and a compaction);
 * the graph's nnz is the arcs kept (cen_graph_info).  flags = 0 is
 * cen_graph_load.  At most 2^32 - 1 arcs after symmetrizing. */
#define CEN_GRAPH_CANONICALIZE 1
#define CEN_GRAPH_SYMMETRIZE 2
int cen_graph_load_ex(const int64_t *off, const int32_t *col, int32_t n, int64_t nnz, int directed, int on_device,
                      int flags, void *stream, cen_graph **out);
/* The graph's canonical out-CSR, read back (no counterpart in the paper):
 * off[n+1] and col[nnz] (nnz of cen_graph_info), host or device pointers,
 * caller-owned; either may be null.  Synchronous on the graph's stream. */
int cen_graph_copy(const cen_graph *g, int64_t *off, int32_t *col);
int cen_graph_free(cen_graph *g);
int cen_graph_info(const cen_graph *g, int32_t *n, int64_t *nnz, int *directed);

/* A job holds the growing sample H (Alg. 1 "H_i") for one (graph, seed, t).
 * t >= 1 is the number of Rademacher vectors (rows of sigma, Sec. 3.2). */
int cen_job_create(const cen_graph *g, uint64_t seed, int32_t t, void *stream, cen_job **out);

/* Hyper-edge spaces (Sec. 2; CentRA is oblivious to the sampler, Sec. 4.2):
 *   BETWEENNESS  set betweenness: the interior nodes of a uniform shortest
 *                s -> t path, s uniform, t uniform over V \ {s} (the default);
 *   KPATH        kappa-path centrality: s uniform, a length l uniform in
 *                1..kappa, then a random simple walk of up to l steps, each to
 *                a uniform out-neighbour not yet on the walk (stopping early
 *                when there is none); the hyper-edge is the nodes after s;
 *   TRIANGLE     triangle centrality: the three nodes of a uniform triangle of
 *                an undirected graph.
 * The per-sample s, t, d of cen_job_copy_samples are (s, t, d(s,t)),
 * (s, l, steps taken) and the triangle's nodes in ascending order. */
#define CEN_SPACE_BETWEENNESS 0
#define CEN_SPACE_KPATH 1
#define CEN_SPACE_TRIANGLE 2
/* cen_job_create with a space.  kappa (KPATH only) in 1 .. 1024.  TRIANGLE
 * needs an undirected graph with at least one triangle (else CEN_EINVAL); the
 * first such job on a graph ranks its triangles on the GPU and keeps the ranks
 * on the graph. */
int cen_job_create_space(const cen_graph *g, uint64_t seed, int32_t t, int32_t space, int32_t kappa, void *stream,
                         cen_job **out);
int cen_job_free(cen_job *job);
/* m = samples drawn so far; members = sum of |h| over them. */
int cen_job_size(const cen_job *job, uint64_t *m, int64_t *members);

/* Alg. 1 "sampleHEs(H, m_new)" for set betweenness (Sec. 3.1, Sec. 5):
 * appends samples j = m .. m+m_new-1.  Sample j draws s uniform in V and t
 * uniform in V \ {s}; counts shortest paths from s (BFS, exact, to 2^128);
 * draws one shortest s->t path uniformly by a backward walk from t; and
 * appends the path's interior nodes (s->t order) as hyper-edge h_j (empty if
 * t is unreachable or adjacent).  Also extends the sign matrix sigma by the
 * columns j (Alg. 1 "sampleRadeVars", extended rather than redrawn).
 * CEN_EOVERFLOW if some pair has >= 2^128 shortest paths (job unchanged). */
int cen_sample(cen_job *job, uint64_t m_new);

/* Alg. 1 "greedyCover(k, H)" (Sec. 3.1): k times add the node covering the
 * most still-uncovered samples (lowest id on ties); stop early when that
 * count is 0.  S_out[k] (host) receives the picks in order, *S_size their
 * number, *covered = |{j : h_j meets S}| = m * C_H(S).  Runs as one
 * thread-block cluster holding the gains in shared memory when they fit (16
 * CTAs, n <= 921,600, where the device allows such clusters; else 8 CTAs,
 * n <= 460,800), otherwise as one cooperative grid launch.  Diagnostics (the
 * picks are the same): the environment variable CEN_GREEDY_CLUSTER=8 keeps
 * 8-CTA clusters, CEN_GREEDY_GRID=1 the grid form. */
int cen_greedy_cover(cen_job *job, int32_t k, int32_t *S_out, int32_t *S_size, uint64_t *covered);

/* AMCERA numerators (Sec. 4.1, Alg. 1 lines computing r_j^u and r_j), all
 * integers: with R_q^u = sum_{j: u in h_j} sigma_{q,j} (= m r_q^u),
 * Rnum_out[q] (host, t entries) = sum of the <= k largest positive R_q^u,
 * *Wnum_out = sum of the k largest c_u = |{j: u in h_j}|, *b_out = max |h_j|.
 * Then AMCERA = sum_q Rnum_q / (t m) and the wimpy variance w = b Wnum / m. */
int cen_mcera(cen_job *job, int32_t k, int64_t *Rnum_out, int64_t *Wnum_out, int32_t *b_out);

/* cen_greedy_cover and cen_mcera of one Alg. 1 round in one call, with the same
 * outputs: the two read the same sample and write disjoint buffers, so the
 * greedy runs on the job's stream while the AMCERA runs on a second stream
 * of the job (made on first use).  Synchronous at return; host outputs as
 * above.  cen_run uses it for every CentRA round. */
int cen_cover_and_mcera(cen_job *job, int32_t k, int32_t *S_out, int32_t *S_size, uint64_t *covered,
                        int64_t *Rnum_out, int64_t *Wnum_out, int32_t *b_out);

/* ---- one sample split over several GPUs (shards) ----
 * Samples are functions of (seed, sample id) (Sec. 5 sampleHEs; Alg. 1
 * sampleRadeVars), so a round's m_i samples can be drawn as disjoint id sets
 * on several jobs, one per GPU, and the round's greedyCover and AMCERA
 * assembled from per-shard counts that add up (Sec. 3.1 coverage gains,
 * Sec. 4.1 R_q^u and c_u are sums over samples).  The exchange (summing the
 * shards' device vectors) is the caller's: a collective library, or host code
 * for shards in one process.  All calls are synchronous at return.
 *
 * cen_job_set_ids: store position p of the job holds sample id
 * p * stride + offset (stride >= 1; before the first cen_sample, else
 * CEN_EINVAL).  Rank r of N uses (N, r): together the N jobs hold ids 0 .. m-1
 * when job r holds ceil((m - r) / N) samples.  (1, 0) is the default. */
int cen_job_set_ids(cen_job *job, uint64_t stride, uint64_t offset);
/* greedyCover one pick at a time (Sec. 3.1).  cen_shard_greedy_begin: after the
 * round's cen_sample, sets this shard's gains to its c_u and clears its covered
 * bits.  cen_shard_gains: copies the n gains (int32) into the caller's device
 * buffer `gains`.  cen_shard_pick: the pick over a device gain vector [n] (the
 * shards' sum): *u = the largest gain, lowest id on ties, *gain = that gain (0:
 * nothing left to cover, *u = -1 when every gain is 0).  cen_shard_apply: covers
 * this shard's still-uncovered samples holding u and lowers their members'
 * gains; *newly_covered = how many (the shards' counts add up to the pick's
 * summed gain).  Gains and apply before a begin that follows the last
 * cen_sample give CEN_EINVAL. */
int cen_shard_greedy_begin(cen_job *job);
int cen_shard_gains(const cen_job *job, int32_t *gains);
int cen_shard_pick(cen_job *job, const int32_t *gains, int32_t *u, int32_t *gain);
int cen_shard_apply(cen_job *job, int32_t u, uint64_t *newly_covered);
/* AMCERA of a split sample (Sec. 4.1, Alg. 1 r_j^u line): cen_shard_rade writes
 * this shard's R_q^u over its own samples into rows 0 .. t-1 and c_u into row
 * t of the caller's device matrix R [t+1][n] (int32, row-major), and its b_H
 * (max |h| over its samples, 0 without samples) to *b.  Summed over the shards,
 * R and c are the whole sample's; b_H is the maximum.  cen_shard_topk: out[r] =
 * the sum of the <= k largest positive entries of row r of a device matrix
 * vals [nrows][n] (n of the job's graph): over the summed matrix, rows 0 .. t-1
 * give Rnum and row t gives Wnum, as cen_mcera does for one job.  nrows >= 1,
 * k >= 1, else CEN_EINVAL. */
int cen_shard_rade(cen_job *job, int32_t *R, int32_t *b);
int cen_shard_topk(cen_job *job, const int32_t *vals, int32_t nrows, int32_t k, int64_t *out);

/* Host FP64 bounds of Thm. 4.4 (Eq. 2, ln(5/delta_i)) and the
 * stopping test of Alg. 1 at iteration i >= 1 (delta_i = delta / 2^i).
 * out[8] = C, AMCERA, w, nu, xi, R~, R, eta.  *stop = 1 iff
 * (1-1/e)((1-1/e-eps) xi + eta) <= eps C.  Pure host code; no GPU work. */
int cen_bounds(uint64_t covered, uint64_t m, int64_t Rsum, int32_t t, int64_t Wnum, int32_t b, double eps,
               double delta, int32_t i, double *out, int32_t *stop);

/* Algorithm 1 end to end on one graph: m_i = m0 2^(i-1) samples in round i,
 * greedyCover, AMCERA, bounds, stop test.  Requires k >= 1, t >= 1,
 * 0 < eps < 1 - 1/e, 0 < delta < 1, 1 <= m0 <= m_cap.  S_out (host, capacity
 * k), *S_size, *covered, *m_final, *rounds describe the last round; log (host,
 * may be NULL) receives min(rounds, max_rounds) rows of CEN_LOG_COLS doubles:
 * i, m_i, covered, Rsum, Wnum, b, C, AMCERA, w, nu, xi, R~, R, eta, stop, |S|.
 * Returns CEN_OK when certified, CEN_ENOTCERTIFIED when the next sample size
 * would exceed m_cap (outputs then describe the last round), or an error. */
int cen_run(const cen_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
            uint64_t m_cap, void *stream, int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final,
            int32_t *rounds, double *log, int32_t max_rounds);

/* Options of cen_run_ex.  A zeroed struct (or a NULL pointer) is cen_run:
 * doubling schedule, CentRA's stopping rule.
 *
 * Sample-size schedules (Sec. 4.2):
 *   DOUBLING    m_i = m0 2^(i-1).
 *   PAPER       growth by alpha > 1 combined with the optimistic guess:
 *               m_1 = max(m0, ceil(g(1))), m_i = max(ceil(alpha m_{i-1}),
 *               ceil(g(C_{i-1}))), where g(C) is the m at which
 *               sqrt(2L/m) + L/(3m) = eps C / (1 - 1/e), L = ln(5 / delta_i)
 *               (the SD bound with no observed deviation, R = 0, nu = 1) and
 *               C_{i-1} the previous round's coverage fraction (g(0) = 0).
 *   EXTRAPOLATE PAPER plus m_pred: the smallest m > m_{i-1} at which round
 *               i's stopping test passes if the coverage fraction C and the
 *               wimpy-variance fraction w stay as measured in round i-1 and
 *               the AMCERA shrinks as 1/sqrt(m) (HEDGE-P: C only); found by
 *               doubling then bisection, and skipped when C = 0 or no size up
 *               to 2^40 passes.  Not in the paper: a sharper reading of its
 *               "adaptive guess" that certifies in a few rounds.
 * Every schedule grows by at least one sample per round; a first size beyond
 * m_cap is clamped to m_cap.
 *
 * Stopping rules:
 *   CENTRA   Alg. 1: AMCERA, Thm. 4.4, stop iff
 *            (1-1/e)((1-1/e-eps) xi + eta) <= eps C.
 *   HEDGE_P  Sec. 6's progressive HEDGE: no AMCERA; the SD bound eta_U of
 *            cen_bounds_hedge; stop iff eta_U <= eps (C - eta_U) / 2.  The
 *            log row's C, nu and eta columns hold C, nu_U and eta_U and its
 *            AMCERA columns (Rsum, Wnum, b, AMCERA, w, xi, R~, R) are 0. */
#define CEN_SCHEDULE_DOUBLING 0
#define CEN_SCHEDULE_PAPER 1
#define CEN_SCHEDULE_EXTRAPOLATE 2
#define CEN_RULE_CENTRA 0
#define CEN_RULE_HEDGE_P 1
typedef struct cen_run_opts {
  int32_t schedule; /* CEN_SCHEDULE_* */
  int32_t rule;     /* CEN_RULE_* */
  double alpha;     /* growth factor of PAPER and EXTRAPOLATE (> 1) */
  int32_t space;    /* CEN_SPACE_* (zeroed: set betweenness) */
  int32_t kappa;    /* path bound of CEN_SPACE_KPATH */
} cen_run_opts;

/* cen_run with options (NULL = defaults).  Same outputs and status codes. */
int cen_run_ex(const cen_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
               uint64_t m_cap, const cen_run_opts *opts, void *stream, int32_t *S_out, int32_t *S_size,
               uint64_t *covered, uint64_t *m_final, int32_t *rounds, double *log, int32_t max_rounds);

/* HEDGE-P's SD bound (no counterpart formula is printed in the paper; this is a
 * union bound over the <= n^k sets of size <= k of a two-sided Bernstein tail):
 * L_U = k ln n + ln(2 / delta_i), delta_i = delta / 2^i; nu_U the largest u
 * with u = C/(1-1/e) + lam(u); eta_U = lam(min(nu_U, 1/4)), where
 * lam(v) = L_U/(3m) + sqrt((L_U/(3m))^2 + 2 v L_U / m).  out[4] = C, L_U,
 * nu_U, eta_U; *stop = 1 iff eta_U <= eps (C - eta_U) / 2.  Host code only. */
int cen_bounds_hedge(uint64_t covered, uint64_t m, int32_t n, int32_t k, double eps, double delta, int32_t i,
                     double *out, int32_t *stop);

/* Batched Algorithm 1: `njobs` independent runs of cen_run_ex, each described by
 * a spec and answered in the result with the same index.  `nworkers` host
 * threads, each with its own CUDA stream on the caller's current device, take
 * jobs longest-first (by arc count) so that jobs overlap on the GPU.  Each
 * job's outputs equal those of cen_run_ex called alone with the same spec.
 * Caller-owned buffers: results[i].S (capacity specs[i].k) and, optionally,
 * results[i].log (results[i].max_rounds rows of CEN_LOG_COLS doubles).
 * Returns CEN_OK once every job has finished (per-job status in results[i]),
 * CEN_EINVAL for bad arguments, or CEN_ECUDA (text in cen_last_error) when no
 * worker could set up its device and stream, so that some job never ran.
 * start_s/end_s: seconds since the call. */
typedef struct cen_job_spec {
  const cen_graph *graph;
  int32_t k, t;
  double eps, delta;
  uint64_t seed, m0, m_cap;
  cen_run_opts opts; /* zeroed: doubling schedule, CentRA's rule */
} cen_job_spec;
typedef struct cen_job_result {
  int32_t status, S_size, rounds, max_rounds;
  uint64_t covered, m_final;
  int32_t *S;
  double *log;
  double start_s, end_s;
} cen_job_result;
int cen_run_batch(const cen_job_spec *specs, int32_t njobs, int32_t nworkers, cen_job_result *results);
/* One run of Algorithm 1 with its arguments and results in the two structs
 * above: the same as cen_run_ex(spec->graph, spec->k, spec->eps, ..., &spec->opts,
 * stream, out->S, &out->S_size, &out->covered, &out->m_final, &out->rounds,
 * out->log, out->max_rounds), with out->status set to its return value and
 * start_s / end_s to 0 and the run's seconds.  Caller-owned: out->S (capacity
 * spec->k), out->log (optional).  Returns CEN_OK, CEN_ENOTCERTIFIED or an
 * error (CEN_EINVAL for a null spec, out or out->S). */
int cen_run_result(const cen_job_spec *spec, void *stream, cen_job_result *out);

/* Allocation-free sum of the <= k largest positive entries of each row: the
 * per-vector sup that cen_mcera computes (Rnum), for callers that supply their
 * own matrix.  The paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory, e.g. code running while another
 * runtime or pool owns every byte of the device, or host callbacks in which
 * cudaMalloc/cudaFree are not allowed because they would synchronize the
 * device.  It allocates nothing: its scratch is one static device array
 * (about 390 KB, held by every GPU that loads the library until exit) sized
 * for at most 128 rows.
 *   vals  device, int32 [nrows][n] row-major (only entries > 0 count);
 *   0 <= n <= 2^31 - 1, 1 <= nrows <= 128, k >= 1, otherwise CEN_EINVAL;
 *   out   host, int64 [nrows]: out[r] = sum of the min(k, #positive) largest
 *         positive entries of row r (0 for a row without positives).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array, which keeps the last call's contents
 * (each call clears what must start at zero): calls that overlap on the GPU,
 * from any stream or thread, race.  The sums are copied to `out` through host
 * memory, so the call synchronizes `stream` before it returns. */
int cen_topk_positive_sum_noalloc(const int32_t *vals, int64_t n, int32_t nrows, int32_t k, int64_t *out,
                                  void *stream);

/* ---- inspection (copies device state to host; for tests and tooling) ---- */
/* hoff[m+1], hmem[members], s[m], t[m], d[m] (d = -1 when unreachable); any may be NULL. */
int cen_job_copy_samples(const cen_job *job, int64_t *hoff, int32_t *hmem, int32_t *s, int32_t *t, int32_t *d);
/* The node -> samples incidence built by the last greedy/mcera call: noff[n+1],
 * nsamp[members] (each node's sample ids, as a set: order within a row is
 * unspecified).  Either may be NULL. */
int cen_job_copy_incidence(const cen_job *job, int64_t *noff, int32_t *nsamp);
/* R[q * n + u] (int32, t x n) and c[n] from the last cen_mcera call. */
int cen_job_copy_rade(const cen_job *job, int32_t *R, int32_t *c);
/* Packed sign words of samples [0, m): words[j * ceil(t/32) + w], bit q%32 of word q/32 set iff sigma_{q,j} = +1. */
int cen_job_copy_signs(const cen_job *job, uint32_t *words);

/* ---- tuning (results never depend on these; only speed and memory do) ---- */
#define CEN_PARAM_WAVE_WORDS 1   /* max samples per wave / 64, 1..32 (default 32) */
#define CEN_PARAM_WAVE_STREAMS 2 /* waves of one cen_sample call in flight, 1..8 (default 4) */
#define CEN_PARAM_PUSH_RATIO 3   /* expand top-down while frontier out-arcs * ratio < arcs (default 4) */
#define CEN_PARAM_LEVEL_BUDGET 4 /* max bytes of one per-level bit array [n][wave words] (default 2^30) */
#define CEN_PARAM_SAMPLER 5      /* 0: balanced bidirectional search, one CTA per sample, with the
                                    bit-parallel sampler for what exceeds its per-CTA limits (default);
                                    1: bit-parallel waves only.  Hyper-edges are identical. */
#define CEN_PARAM_BIDIR_BUDGET 6 /* device bytes for the bidirectional sampler's per-CTA workspace,
                                    >= 2^20 (default 2^34); fewer CTAs run when it is small.  One CTA
                                    needs 8 h + 16 H + 28 q bytes, plus 32,800 with warp searches
                                    (q = min(n, queue), H = the power of two >= max(4 q, 1024),
                                    h = small-table entries), whatever the graph */
#define CEN_PARAM_BIDIR_QUEUE 7  /* nodes one CTA may hold per ball or cone side, 16 .. 2^27 (default
                                    2^16, at most n); larger searches go to the bit-parallel sampler */
#define CEN_PARAM_BIDIR_TABLE 8  /* entries of each CTA's small node table: a power of two in
                                    2^10 .. 2^24 (at most H / 2), 0 for none (searches use the large
                                    table of H entries only), or -1 (default) to size all CTAs' small
                                    tables to about 80 MiB so that they stay in L2; a search that
                                    fills half of it moves to the large table.  With -1, once a call
                                    of 1,024 or more samples sees most searches move, later jobs on
                                    the graph use no small table */
#define CEN_PARAM_BIDIR_WARPS 9  /* 1: each warp of a CTA searches samples alone with a 1,024-entry
                                    node table, and a second launch searches with whole CTAs those it
                                    hands on (a level of more than 2,048 arcs to expand, more than 512
                                    nodes, or more than 64 levels a side); 0: every sample is searched
                                    by a whole CTA; -1 (default): 0 on graphs whose degrees have
                                    E[d^2]/E[d] > 256 (frontiers that soon outgrow a warp), else 1
                                    until a call of 1,024 or more samples hands more than 30% on,
                                    then 0 for later jobs on the graph.  Queues of fewer than 1,024
                                    nodes use CTA searches only */
int cen_job_set_param(cen_job *job, int32_t param, double value);
/* Releases the device memory the library keeps for reuse once jobs end: idle
 * bidirectional-sampler workspaces (up to four, each as large as
 * CEN_PARAM_BIDIR_BUDGET allows) and the unused part of the current device's
 * stream-ordered memory pool, which the library sets to keep freed memory.
 * Synchronizes the device.  Later jobs allocate again. */
int cen_release_cached(void);
/* How the job's samples were drawn so far: samples the bidirectional search
 * left whole to the bit-parallel sampler (*deferred_search), samples whose walk
 * it left to it (*deferred_walk), searches that outgrew the small node table
 * (*migrated), the CTAs (slots) the bidirectional search runs on (0 before
 * its first use), and the warp searches handed on to whole CTAs because a
 * level, the node count or the depth was too large for one warp (*escalated).
 * Any pointer may be NULL. */
int cen_job_sampler_info(const cen_job *job, uint64_t *deferred_search, uint64_t *deferred_walk, uint64_t *migrated,
                         int32_t *slots, uint64_t *escalated);
/* Defaults for jobs created later on this graph (cen_job_create, cen_run, cen_run_batch);
 * they take precedence over the environment (CEN_WAVE_WORDS, CEN_WAVE_STREAMS). */
int cen_graph_set_param(cen_graph *g, int32_t param, double value);

/* Testing hook (no counterpart in the paper): the n-th device allocation the
 * library makes from now on (n >= 1, any thread) fails with CEN_ENOMEM as if
 * the device were out of memory; n = 0 disarms.  Process-wide.  Lets callers
 * test their handling of a full device without filling one. */
int cen_debug_fail_alloc(int64_t n);

/* ---- instrumentation ---- */
/* Per-kernel-class launch counts, device time and work units since the job
 * was created (or last reset).  Device time is recorded only while
 * timing is enabled (CUDA events around each launch on the job stream). */
#define CEN_NKCLASS 24
typedef struct cen_kstat {
  char name[32];
  uint64_t launches;
  double ms;          /* sum of event-timed durations (timing enabled only) */
  uint64_t timed;     /* launches that were event-timed */
  uint64_t units;     /* work units counted by the kernel (class-specific) */
} cen_kstat;
int cen_job_set_timing(cen_job *job, int enable);
int cen_job_stats(cen_job *job, cen_kstat *out /* [CEN_NKCLASS] */, int32_t *nclasses);
int cen_job_reset_stats(cen_job *job);

#ifdef __cplusplus
}
#endif
#endif
