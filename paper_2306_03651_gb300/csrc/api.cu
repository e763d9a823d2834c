// C ABI of libcen (include/cen.h): argument checks, handle lifetimes,
// Algorithm 1's progressive loop and the FP64 bounds.  Every entry point
// converts internal failures into a status code and a thread-local message.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "job.cuh"

namespace cen {
const std::string &last_error();

void *host_staging(cen_job *job, size_t bytes) {
  if (bytes > job->host_bytes) {
    if (job->host) {
      CEN_CK(cudaStreamSynchronize(job->st));  // no copy may still use the old buffer
      pinned_give(job->host, job->host_bytes);
    }
    job->host = nullptr;
    job->host_bytes = 0;
    size_t cap = 0;
    job->host = pinned_take(bytes, &cap);
    job->host_bytes = cap;
  }
  return job->host;
}

// Thm. 4.4 (Eq. 2) with ln(5/delta_i) and the xi / stopping
// lines of Alg. 1.  Evaluation order (a = 1 - 1/e, L = ln(5/delta_i), Lm = L/m):
//   C = covered/m;  A = Rsum/(t m);  w = (b Wnum)/m
//   xi = sqrt(Lm Lm + (2 C L)/(a m)) + Lm;   nu = C/a + xi
//   Rt = A + sqrt((4 w L)/(t m));   R = Rt + sqrt(Lm Lm + (2 L Rt)/m) + Lm
//   eta = 2 R + sqrt((2 L (nu + 4 R))/m) + L/(3 m)
//   stop <=> a ((a - eps) xi + eta) <= eps C
// Thm. 4.4 from the sample's fractions C, A (AMCERA), w at sample
// size md with L = ln(5 / delta_i); writes out[3..7] = nu, xi, R~, R, eta.
static void bounds_from_fractions(double C, double A, double w, int32_t t, double md, double L, double *out) {
  const double a = 1.0 - exp(-1.0);
  const double Lm = L / md;
  const double xi = sqrt(Lm * Lm + (2.0 * C * L) / (a * md)) + Lm;
  const double nu = C / a + xi;
  const double Rt = A + sqrt((4.0 * w * L) / ((double)t * md));
  const double R = Rt + sqrt(Lm * Lm + (2.0 * L * Rt) / md) + Lm;
  const double eta = 2.0 * R + sqrt((2.0 * L * (nu + 4.0 * R)) / md) + L / (3.0 * md);
  out[3] = nu;
  out[4] = xi;
  out[5] = Rt;
  out[6] = R;
  out[7] = eta;
}

static int bounds_fp64(uint64_t covered, uint64_t m, int64_t Rsum, int32_t t, int64_t Wnum, int32_t b, double eps,
                       double delta, int32_t i, double *out) {
  const double a = 1.0 - exp(-1.0);
  const double md = (double)m;
  const double L = log(5.0 / ldexp(delta, -i));
  const double C = (double)covered / md;
  out[0] = C;
  out[1] = (double)Rsum / ((double)t * md);
  out[2] = ((double)b * (double)Wnum) / md;
  bounds_from_fractions(C, out[1], out[2], t, md, L, out);
  return (a * ((a - eps) * out[4] + out[7]) <= eps * C) ? 1 : 0;
}

// Sample-size schedule of Sec. 4.2.  The optimistic guess is the smallest m
// at which the stopping test could pass if the sample showed no deviation
// (R = 0, nu = 1 in Thm. 4.4): eta(m) = sqrt(2L/m) + L/(3m) must reach
// eps C / (1 - 1/e).  With y = 1/sqrt(m) that is the quadratic
// (L/3) y^2 + sqrt(2L) y = target, solved for its positive root.
static double schedule_guess(double C, double eps, double delta, int32_t i) {
  const double a = 1.0 - exp(-1.0);
  const double L = log(5.0 / ldexp(delta, -i));
  const double target = eps * C / a;
  if (!(target > 0.0)) return 0.0;  // C = 0: no finite guess
  const double A3 = L / 3.0;
  const double B = sqrt(2.0 * L);
  const double y = (sqrt(B * B + 4.0 * A3 * target) - B) / (2.0 * A3);
  return 1.0 / (y * y);
}

// m_i for round i.  Schedule 0 doubles from m0.  Schedule 1 grows by alpha
// and jumps to the guess made from the previous round's coverage C_{i-1}
// (C = 1 before the first round).  Schedule 2 also jumps to m_pred (> 0), the
// size at which round i's stopping test is predicted to pass (predict_m).
// Every schedule grows by at least one sample.
static uint64_t schedule_next(int32_t schedule, double alpha, uint64_t m0, uint64_t m_prev, double C_prev,
                              uint64_t m_pred, double eps, double delta, int32_t i) {
  if (schedule == CEN_SCHEDULE_DOUBLING) return i == 1 ? m0 : 2 * m_prev;
  const double grow = i == 1 ? (double)m0 : ceil(alpha * (double)m_prev);
  const double guess = ceil(schedule_guess(i == 1 ? 1.0 : C_prev, eps, delta, i));
  double m = grow > guess ? grow : guess;
  if (schedule == CEN_SCHEDULE_EXTRAPOLATE && i > 1 && m_pred > 0 && (double)m_pred > m) m = (double)m_pred;
  if (i > 1 && m <= (double)m_prev) m = (double)m_prev + 1.0;
  return m >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)m;
}

// HEDGE-P's SD bound (Sec. 6; HEDGE's union bound of Sec. 2).  For one set S
// the coverage estimate is a mean of m i.i.d. 0/1 terms with variance
// C(S)(1 - C(S)) <= min(C(S*), 1/4); a two-sided Bernstein tail at level
// delta_i / n^k, union-bounded over the <= n^k sets of size <= k, gives every
// set a deviation of at most lam(v) = b + sqrt(b^2 + 2 v L_U / m) with
// L_U = k ln n + ln(2 / delta_i) and b = L_U / (3 m).  On that event
// C(S*) <= C / (1 - 1/e) + lam(C(S*)) (greedy keeps 1 - 1/e of the sample
// optimum), whose largest solution is nu_U; eta_U = lam(min(nu_U, 1/4)).
// HEDGE's sufficient condition SD <= eps C(S*) / 2 then holds once
// eta_U <= eps (C - eta_U) / 2, because C(S*) >= C(S) >= C - SD.
static double hedge_L(int32_t n, int32_t k, double delta, int32_t i) {
  return (double)k * log((double)n) + log(2.0 / ldexp(delta, -i));
}

// writes out[2] = nu_U, out[3] = eta_U for coverage fraction C at size md
static void hedge_from_fraction(double C, double md, double LU, double *out) {
  const double a = 1.0 - exp(-1.0);
  const double Lm = LU / md;
  const double b = LU / (3.0 * md);
  const double c0 = C / a + b;
  const double nu = c0 + Lm + sqrt(2.0 * c0 * Lm + Lm * Lm + b * b);  // larger root of (u - c0)^2 = b^2 + 2 u Lm
  const double v = nu < 0.25 ? nu : 0.25;
  out[2] = nu;
  out[3] = b + sqrt(b * b + 2.0 * v * Lm);
}

static int bounds_hedge_fp64(uint64_t covered, uint64_t m, int32_t n, int32_t k, double eps, double delta,
                             int32_t i, double *out) {
  const double md = (double)m;
  const double C = (double)covered / md;
  out[0] = C;
  out[1] = hedge_L(n, k, delta, i);
  hedge_from_fraction(C, md, out[1], out);
  return (out[3] <= eps * (C - out[3]) / 2.0) ? 1 : 0;
}

// Would round i's stopping test pass at size mp if the coverage fraction C
// and the wimpy-variance fraction w stayed as measured at size m and the
// AMCERA A shrank as 1/sqrt(m), the rate of both SD bounds (Sec. 6)?
// (HEDGE-P keeps C only.)
static bool predicted_stop(int32_t rule, double C, double A, double w, int32_t t, int32_t n, int32_t k, uint64_t m,
                           uint64_t mp, double eps, double delta, int32_t i) {
  const double a = 1.0 - exp(-1.0);
  const double md = (double)mp;
  double o[8];
  if (rule == CEN_RULE_CENTRA) {
    const double Ap = A * sqrt((double)m / md);
    bounds_from_fractions(C, Ap, w, t, md, log(5.0 / ldexp(delta, -i)), o);
    return a * ((a - eps) * o[4] + o[7]) <= eps * C;
  }
  hedge_from_fraction(C, md, hedge_L(n, k, delta, i), o);
  return o[3] <= eps * (C - o[3]) / 2.0;
}

// Smallest mp > m with predicted_stop (doubling, then bisection), or 0 when
// none up to 2^40 passes (the prediction is then not used).
static uint64_t predict_m(int32_t rule, double C, double A, double w, int32_t t, int32_t n, int32_t k, uint64_t m,
                          double eps, double delta, int32_t i) {
  if (!(C > 0.0)) return 0;
  uint64_t lo = m, hi = 2 * m;
  while (!predicted_stop(rule, C, A, w, t, n, k, m, hi, eps, delta, i)) {
    if (hi >= (1ull << 40)) return 0;
    lo = hi;
    hi *= 2;
  }
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (predicted_stop(rule, C, A, w, t, n, k, m, mid, eps, delta, i))
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

}  // namespace cen

using cen::Error;

static void apply_param(cen_job *job, int32_t param, double value) {
  switch (param) {
    case CEN_PARAM_WAVE_WORDS:
      CEN_REQUIRE(value >= 1 && value <= 32, CEN_EINVAL, "cen_job_set_param: wave words must be in [1, 32]");
      job->max_wave_words = (int)value;
      break;
    case CEN_PARAM_WAVE_STREAMS:
      CEN_REQUIRE(value >= 1 && value <= 8, CEN_EINVAL, "cen_job_set_param: wave streams must be in [1, 8]");
      job->wave_streams = (int)value;
      break;
    case CEN_PARAM_PUSH_RATIO:
      CEN_REQUIRE(value > 0 && value <= 1e6, CEN_EINVAL, "cen_job_set_param: push ratio must be in (0, 1e6]");
      job->push_ratio = value;
      break;
    case CEN_PARAM_LEVEL_BUDGET:
      CEN_REQUIRE(value >= (1 << 20), CEN_EINVAL, "cen_job_set_param: level budget must be >= 1 MiB");
      job->level_budget = (size_t)value;
      break;
    case CEN_PARAM_SAMPLER:
      CEN_REQUIRE(value == 0 || value == 1, CEN_EINVAL, "cen_job_set_param: sampler must be 0 or 1");
      job->sampler = (int)value;
      break;
    case CEN_PARAM_BIDIR_BUDGET:
      CEN_REQUIRE(value >= (1 << 20), CEN_EINVAL, "cen_job_set_param: bidirectional budget must be >= 1 MiB");
      job->bidir_budget = (size_t)value;
      break;
    case CEN_PARAM_BIDIR_TABLE: {
      const int64_t h = (int64_t)value;
      CEN_REQUIRE(value == -1 || value == 0 || (h >= 1024 && h <= ((int64_t)1 << 24) && (h & (h - 1)) == 0),
                  CEN_EINVAL, "cen_job_set_param: table entries must be -1, 0 or a power of two in [2^10, 2^24]");
      job->bidir_table = h;
      break;
    }
    case CEN_PARAM_BIDIR_WARPS:
      CEN_REQUIRE(value == -1 || value == 0 || value == 1, CEN_EINVAL,
                  "cen_job_set_param: warp searches must be -1, 0 or 1");
      job->bidir_warps = (int)value;
      break;
    case CEN_PARAM_BIDIR_QUEUE:
      CEN_REQUIRE(value >= 16 && value <= (double)(1 << 27), CEN_EINVAL,
                  "cen_job_set_param: bidirectional queue must be in [16, 2^27]");
      job->bidir_queue = (int64_t)value;
      break;
    default:
      cen::fail(CEN_EINVAL, "cen_job_set_param: unknown parameter");
  }
}


#define CEN_API_BEGIN try {
#define CEN_API_END                                  \
  return CEN_OK;                                     \
  }                                                  \
  catch (const Error &e) {                           \
    cen::set_last_error(e.msg);                      \
    return e.code;                                   \
  }                                                  \
  catch (const std::bad_alloc &) {                   \
    cen::set_last_error("host allocation failed");   \
    return CEN_ENOMEM;                               \
  }                                                  \
  catch (...) {                                      \
    cen::set_last_error("unexpected internal error"); \
    return CEN_ECUDA;                                \
  }

extern "C" {

int cen_version(void) { return 100; }

const char *cen_last_error(void) { return cen::last_error().c_str(); }

int cen_set_allocator(cen_alloc_fn alloc, cen_free_fn free_fn, void *ctx) {
  CEN_API_BEGIN
  CEN_REQUIRE(!alloc == !free_fn, CEN_EINVAL, "cen_set_allocator: give both functions or neither");
  cen::set_allocator(alloc, free_fn, ctx);
  CEN_API_END
}

int cen_graph_load(const int64_t *off, const int32_t *col, int32_t n, int64_t nnz, int directed, int on_device,
                   void *stream, cen_graph **out) {
  CEN_API_BEGIN
  CEN_REQUIRE(out && off && (col || nnz == 0), CEN_EINVAL, "cen_graph_load: null argument");
  CEN_REQUIRE(n >= 2 && nnz >= 0, CEN_EINVAL, "cen_graph_load: need n >= 2 and nnz >= 0");
  *out = nullptr;
  cen_graph *g = new cen_graph();
  g->n = n;
  g->nnz = nnz;
  g->directed = directed ? 1 : 0;
  g->st = (cudaStream_t)stream;
  try {
    cen::graph_build(g, off, col, on_device != 0, nullptr);
  } catch (...) {
    delete g;
    throw;
  }
  *out = g;
  CEN_API_END
}

int cen_graph_load_ex(const int64_t *off, const int32_t *col, int32_t n, int64_t nnz, int directed, int on_device,
                      int flags, void *stream, cen_graph **out) {
  if (flags == 0) return cen_graph_load(off, col, n, nnz, directed, on_device, stream, out);
  CEN_API_BEGIN
  CEN_REQUIRE(!(flags & ~(CEN_GRAPH_CANONICALIZE | CEN_GRAPH_SYMMETRIZE)), CEN_EINVAL, "cen_graph_load: unknown flag");
  CEN_REQUIRE(out && off && (col || nnz == 0), CEN_EINVAL, "cen_graph_load: null argument");
  CEN_REQUIRE(n >= 2 && nnz >= 0, CEN_EINVAL, "cen_graph_load: need n >= 2 and nnz >= 0");
  CEN_REQUIRE(!(directed && (flags & CEN_GRAPH_SYMMETRIZE)), CEN_EINVAL,
              "cen_graph_load: SYMMETRIZE is for undirected graphs");
  *out = nullptr;
  cen_graph *g = new cen_graph();
  g->n = n;
  g->directed = directed ? 1 : 0;
  g->st = (cudaStream_t)stream;
  try {
    cen::graph_canonicalize(g, off, col, nnz, on_device != 0, (flags & CEN_GRAPH_SYMMETRIZE) != 0, nullptr);
    cen::graph_build(g, nullptr, nullptr, true, nullptr);
  } catch (...) {
    delete g;
    throw;
  }
  *out = g;
  CEN_API_END
}

int cen_graph_copy(const cen_graph *g, int64_t *off, int32_t *col) {
  CEN_API_BEGIN
  CEN_REQUIRE(g, CEN_EINVAL, "cen_graph_copy: null graph");
  cudaStream_t st = g->st;
  if (off) CEN_CK(cudaMemcpyAsync(off, g->off.p, sizeof(int64_t) * ((size_t)g->n + 1), cudaMemcpyDefault, st));
  if (col && g->nnz) CEN_CK(cudaMemcpyAsync(col, g->col.p, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_API_END
}

int cen_graph_free(cen_graph *g) {
  CEN_API_BEGIN
  if (g) {
    cudaStream_t st = g->st;
    delete g;
    CEN_CK(cudaStreamSynchronize(st));
  }
  CEN_API_END
}

int cen_graph_info(const cen_graph *g, int32_t *n, int64_t *nnz, int *directed) {
  CEN_API_BEGIN
  CEN_REQUIRE(g, CEN_EINVAL, "cen_graph_info: null graph");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (directed) *directed = g->directed;
  CEN_API_END
}

int cen_job_create(const cen_graph *g, uint64_t seed, int32_t t, void *stream, cen_job **out) {
  return cen_job_create_space(g, seed, t, CEN_SPACE_BETWEENNESS, 0, stream, out);
}

int cen_job_create_space(const cen_graph *g, uint64_t seed, int32_t t, int32_t space, int32_t kappa, void *stream,
                         cen_job **out) {
  CEN_API_BEGIN
  CEN_REQUIRE(g && out, CEN_EINVAL, "cen_job_create: null argument");
  CEN_REQUIRE(t >= 1 && t <= 4096, CEN_EINVAL, "cen_job_create: need 1 <= t <= 4096");
  CEN_REQUIRE(space == CEN_SPACE_BETWEENNESS || space == CEN_SPACE_KPATH || space == CEN_SPACE_TRIANGLE, CEN_EINVAL,
              "cen_job_create: unknown hyper-edge space");
  CEN_REQUIRE(space != CEN_SPACE_KPATH || (kappa >= 1 && kappa <= cen::max_kappa()), CEN_EINVAL,
              "cen_job_create: kappa must be in [1, 1024]");
  CEN_REQUIRE(space != CEN_SPACE_TRIANGLE || !g->directed, CEN_EINVAL,
              "cen_job_create: the triangle space needs an undirected graph");
  *out = nullptr;
  cen_job *job = new cen_job();
  job->g = g;
  job->seed = seed;
  job->t = t;
  job->space = space;
  job->kappa = space == CEN_SPACE_KPATH ? kappa : 0;
  job->nw = (t + 31) / 32;
  job->st = (cudaStream_t)stream;
  if (const char *e = getenv("CEN_WAVE_WORDS")) {  // wave width in 64-slot words (1..32), a tuning knob
    const int w = atoi(e);
    if (w >= 1 && w <= 32) job->max_wave_words = w;
  }
  if (const char *e = getenv("CEN_WAVE_STREAMS")) {  // waves of one cen_sample call in flight (1..8)
    const int w = atoi(e);
    if (w >= 1 && w <= 8) job->wave_streams = w;
  }
  for (int p = 1; p <= 9; ++p)  // the graph's tuned defaults override the environment
    if (g->param_set[p]) apply_param(job, p, g->param[p]);
  try {
    job->stats.init(job->st);
    if (space == CEN_SPACE_TRIANGLE)
      CEN_REQUIRE(cen::triangle_index(job) > 0, CEN_EINVAL, "cen_job_create: the graph has no triangle");
  } catch (...) {
    CEN_CK(cudaStreamSynchronize(job->st));
    delete job;
    throw;
  }
  *out = job;
  CEN_API_END
}

int cen_job_free(cen_job *job) {
  CEN_API_BEGIN
  if (job) {
    cudaStream_t st = job->st;
    cudaStreamSynchronize(st);
    void *h = job->host;
    const size_t hb = job->host_bytes;
    cen::bidir_give(std::move(job->bws));  // idle, since the stream has drained
    delete job;
    CEN_CK(cudaStreamSynchronize(st));
    cen::pinned_give(h, hb);
  }
  CEN_API_END
}

int cen_job_size(const cen_job *job, uint64_t *m, int64_t *members) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_size: null job");
  if (m) *m = job->m;
  if (members) *members = job->members;
  CEN_API_END
}

int cen_sample(cen_job *job, uint64_t m_new) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_sample: null job");
  CEN_REQUIRE(job->m + m_new < (1ull << 31), CEN_EINVAL, "cen_sample: at most 2^31 - 1 samples per job");
  cen::sample_append(job, m_new);
  job->stats.resolve();
  CEN_API_END
}

int cen_greedy_cover(cen_job *job, int32_t k, int32_t *S_out, int32_t *S_size, uint64_t *covered) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && S_out && S_size && covered, CEN_EINVAL, "cen_greedy_cover: null argument");
  cen::greedy_cover(job, k, S_out, S_size, covered);
  job->stats.resolve();
  CEN_API_END
}

int cen_cover_and_mcera(cen_job *job, int32_t k, int32_t *S_out, int32_t *S_size, uint64_t *covered,
                        int64_t *Rnum_out, int64_t *Wnum_out, int32_t *b_out) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && S_out && S_size && covered && Rnum_out && Wnum_out && b_out, CEN_EINVAL,
              "cen_cover_and_mcera: null argument");
  cen::cover_and_mcera(job, k, S_out, S_size, covered, Rnum_out, Wnum_out, b_out);
  CEN_API_END
}

int cen_mcera(cen_job *job, int32_t k, int64_t *Rnum_out, int64_t *Wnum_out, int32_t *b_out) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && Rnum_out && Wnum_out && b_out, CEN_EINVAL, "cen_mcera: null argument");
  cen::mcera(job, k, Rnum_out, Wnum_out, b_out);
  job->stats.resolve();
  CEN_API_END
}

int cen_bounds(uint64_t covered, uint64_t m, int64_t Rsum, int32_t t, int64_t Wnum, int32_t b, double eps,
               double delta, int32_t i, double *out, int32_t *stop) {
  CEN_API_BEGIN
  CEN_REQUIRE(out && stop && m >= 1 && t >= 1 && i >= 1 && delta > 0 && delta < 1, CEN_EINVAL,
              "cen_bounds: need m >= 1, t >= 1, i >= 1, 0 < delta < 1");
  *stop = cen::bounds_fp64(covered, m, Rsum, t, Wnum, b, eps, delta, i, out);
  CEN_API_END
}

int cen_run(const cen_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
            uint64_t m_cap, void *stream, int32_t *S_out, int32_t *S_size, uint64_t *covered, uint64_t *m_final,
            int32_t *rounds, double *log, int32_t max_rounds) {
  return cen_run_ex(g, k, eps, delta, t, seed, m0, m_cap, nullptr, stream, S_out, S_size, covered, m_final, rounds,
                    log, max_rounds);
}

int cen_bounds_hedge(uint64_t covered, uint64_t m, int32_t n, int32_t k, double eps, double delta, int32_t i,
                     double *out, int32_t *stop) {
  CEN_API_BEGIN
  CEN_REQUIRE(out && stop && m >= 1 && n >= 2 && k >= 1 && i >= 1 && delta > 0 && delta < 1, CEN_EINVAL,
              "cen_bounds_hedge: need m >= 1, n >= 2, k >= 1, i >= 1, 0 < delta < 1");
  *stop = cen::bounds_hedge_fp64(covered, m, n, k, eps, delta, i, out);
  CEN_API_END
}

int cen_run_ex(const cen_graph *g, int32_t k, double eps, double delta, int32_t t, uint64_t seed, uint64_t m0,
               uint64_t m_cap, const cen_run_opts *opts, void *stream, int32_t *S_out, int32_t *S_size,
               uint64_t *covered, uint64_t *m_final, int32_t *rounds, double *log, int32_t max_rounds) {
  cen_job *job = nullptr;
  int rc = CEN_OK;
  try {
    const double a = 1.0 - exp(-1.0);
    const cen_run_opts o = opts ? *opts : cen_run_opts{CEN_SCHEDULE_DOUBLING, CEN_RULE_CENTRA, 0.0, 0, 0};
    CEN_REQUIRE(g && S_out && S_size && covered && m_final && rounds, CEN_EINVAL, "cen_run: null argument");
    CEN_REQUIRE(k >= 1 && t >= 1 && eps > 0.0 && eps < a && delta > 0.0 && delta < 1.0 && m0 >= 1 && m_cap >= m0,
                CEN_EINVAL, "cen_run: need k >= 1, t >= 1, 0 < eps < 1-1/e, 0 < delta < 1, 1 <= m0 <= m_cap");
    CEN_REQUIRE(o.schedule >= CEN_SCHEDULE_DOUBLING && o.schedule <= CEN_SCHEDULE_EXTRAPOLATE &&
                    (o.schedule == CEN_SCHEDULE_DOUBLING || o.alpha > 1.0),
                CEN_EINVAL, "cen_run: unknown schedule, or alpha <= 1 for a growing schedule");
    CEN_REQUIRE(o.rule == CEN_RULE_CENTRA || o.rule == CEN_RULE_HEDGE_P, CEN_EINVAL, "cen_run: unknown rule");
    int crc = cen_job_create_space(g, seed, t, o.space, o.kappa, stream, &job);
    if (crc) return crc;
    std::vector<int64_t> Rnum(t);
    uint64_t m_prev = 0;
    uint64_t m_i = cen::schedule_next(o.schedule, o.alpha, m0, 0, 1.0, 0, eps, delta, 1);
    if (m_i > m_cap) m_i = m_cap;  // a first guess beyond the cap runs one round at the cap
    rc = CEN_ENOTCERTIFIED;
    for (int32_t i = 1;; ++i) {
      cen::Range round_range("cen_run round");
      CEN_REQUIRE(m_i < (1ull << 31), CEN_EINVAL, "cen_run: at most 2^31 - 1 samples per job");
      cen::sample_append(job, m_i - m_prev);
      uint64_t cov = 0;
      int64_t Wnum = 0, Rsum = 0;
      int32_t b = 0;
      double bd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int stop;
      if (o.rule == CEN_RULE_CENTRA) {
        cen::cover_and_mcera(job, k, S_out, S_size, &cov, Rnum.data(), &Wnum, &b);
        for (int q = 0; q < t; ++q) Rsum += Rnum[q];
        stop = cen::bounds_fp64(cov, m_i, Rsum, t, Wnum, b, eps, delta, i, bd);
      } else {  // HEDGE-P needs no AMCERA; its C, nu_U, eta_U go to the C, nu, eta columns
        cen::greedy_cover(job, k, S_out, S_size, &cov);
        double hb[4];
        stop = cen::bounds_hedge_fp64(cov, m_i, g->n, k, eps, delta, i, hb);
        bd[0] = hb[0];
        bd[3] = hb[2];
        bd[7] = hb[3];
      }
      if (log && i <= max_rounds) {
        double *row = log + (size_t)(i - 1) * CEN_LOG_COLS;
        row[0] = i;
        row[1] = (double)m_i;
        row[2] = (double)cov;
        row[3] = (double)Rsum;
        row[4] = (double)Wnum;
        row[5] = b;
        for (int q = 0; q < 8; ++q) row[6 + q] = bd[q];
        row[14] = stop;
        row[15] = *S_size;
      }
      *covered = cov;
      *m_final = m_i;
      *rounds = i;
      if (stop) {
        rc = CEN_OK;
        break;
      }
      const uint64_t m_pred =
          o.schedule == CEN_SCHEDULE_EXTRAPOLATE
              ? cen::predict_m(o.rule, bd[0], bd[1], bd[2], t, g->n, k, m_i, eps, delta, i + 1)
              : 0;
      const uint64_t next = cen::schedule_next(o.schedule, o.alpha, m0, m_i, bd[0], m_pred, eps, delta, i + 1);
      if (next > m_cap) {
        rc = CEN_ENOTCERTIFIED;
        cen::set_last_error("cen_run: not certified within m_cap samples");
        break;
      }
      m_prev = m_i;
      m_i = next;
    }
  } catch (const Error &e) {
    cen::set_last_error(e.msg);
    rc = e.code;
  } catch (...) {
    cen::set_last_error("unexpected internal error");
    rc = CEN_ECUDA;
  }
  if (job) cen_job_free(job);
  return rc;
}

int cen_job_copy_samples(const cen_job *job, int64_t *hoff, int32_t *hmem, int32_t *s, int32_t *t, int32_t *d) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_copy_samples: null job");
  cudaStream_t st = job->st;
  if (hoff) {
    if (job->m)
      CEN_CK(cudaMemcpyAsync(hoff, job->hoff.p, 8 * (job->m + 1), cudaMemcpyDeviceToHost, st));
    else
      hoff[0] = 0;
  }
  if (hmem && job->members) CEN_CK(cudaMemcpyAsync(hmem, job->hmem.p, 4 * job->members, cudaMemcpyDeviceToHost, st));
  if (s && job->m) CEN_CK(cudaMemcpyAsync(s, job->ps.p, 4 * job->m, cudaMemcpyDeviceToHost, st));
  if (t && job->m) CEN_CK(cudaMemcpyAsync(t, job->pt.p, 4 * job->m, cudaMemcpyDeviceToHost, st));
  if (d && job->m) CEN_CK(cudaMemcpyAsync(d, job->pd.p, 4 * job->m, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_API_END
}

int cen_job_copy_incidence(const cen_job *job, int64_t *noff, int32_t *nsamp) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && job->inc_m == job->m, CEN_EINVAL,
              "cen_job_copy_incidence: no incidence for the current sample (call cen_greedy_cover or cen_mcera)");
  cudaStream_t st = job->st;
  if (noff) CEN_CK(cudaMemcpyAsync(noff, job->noff.p, 8 * ((size_t)job->g->n + 1), cudaMemcpyDeviceToHost, st));
  if (nsamp && job->members)
    CEN_CK(cudaMemcpyAsync(nsamp, job->nsamp.p, 4 * job->members, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_API_END
}

int cen_job_copy_rade(const cen_job *job, int32_t *R, int32_t *c) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && job->rade_valid_k >= 0 && job->inc_m == job->m, CEN_EINVAL,
              "cen_job_copy_rade: call cen_mcera first");
  cudaStream_t st = job->st;
  if (R) CEN_CK(cudaMemcpyAsync(R, job->R.p, 4 * (size_t)job->g->n * job->t, cudaMemcpyDeviceToHost, st));
  if (c) CEN_CK(cudaMemcpyAsync(c, job->c.p, 4 * (size_t)job->g->n, cudaMemcpyDeviceToHost, st));
  CEN_CK(cudaStreamSynchronize(st));
  CEN_API_END
}

int cen_job_copy_signs(const cen_job *job, uint32_t *words) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && words, CEN_EINVAL, "cen_job_copy_signs: null argument");
  if (job->m)
    CEN_CK(cudaMemcpyAsync(words, job->sign.p, 4 * (size_t)job->nw * job->m, cudaMemcpyDeviceToHost, job->st));
  CEN_CK(cudaStreamSynchronize(job->st));
  CEN_API_END
}

int cen_job_set_timing(cen_job *job, int enable) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_set_timing: null job");
  CEN_CK(cudaStreamSynchronize(job->st));
  job->stats.resolve();
  job->stats.timing = enable != 0;
  CEN_API_END
}

int cen_job_stats(cen_job *job, cen_kstat *out, int32_t *nclasses) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && out && nclasses, CEN_EINVAL, "cen_job_stats: null argument");
  CEN_CK(cudaStreamSynchronize(job->st));
  job->stats.resolve();
  uint64_t units[cen::K_COUNT];
  CEN_CK(cudaMemcpy(units, job->stats.d_units, sizeof(units), cudaMemcpyDeviceToHost));
  for (int c = 0; c < cen::K_COUNT; ++c) {
    out[c] = job->stats.k[c];
    out[c].units = units[c];
  }
  *nclasses = cen::K_COUNT;
  CEN_API_END
}

int cen_job_set_param(cen_job *job, int32_t param, double value) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_set_param: null job");
  apply_param(job, param, value);
  CEN_API_END
}

int cen_release_cached(void) {
  CEN_API_BEGIN
  cen::bidir_drop_cached();
  cen::pinned_drop_cached();
  int dev = 0;
  CEN_CK(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  CEN_CK(cudaDeviceGetDefaultMemPool(&pool, dev));
  CEN_CK(cudaDeviceSynchronize());  // the dropped workspaces are freed in stream order
  CEN_CK(cudaMemPoolTrimTo(pool, 0));
  CEN_API_END
}

int cen_job_set_ids(cen_job *job, uint64_t stride, uint64_t offset) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && stride >= 1, CEN_EINVAL, "cen_job_set_ids: null job or stride 0");
  CEN_REQUIRE(job->m == 0, CEN_EINVAL, "cen_job_set_ids: the job already holds samples");
  job->id_stride = stride;
  job->id_offset = offset;
  CEN_API_END
}

int cen_shard_greedy_begin(cen_job *job) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_shard_greedy_begin: null job");
  cen::shard_greedy_begin(job);
  CEN_API_END
}

int cen_shard_gains(const cen_job *job, int32_t *gains) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && gains, CEN_EINVAL, "cen_shard_gains: null argument");
  cen::shard_gains(job, gains);
  CEN_API_END
}

int cen_shard_pick(cen_job *job, const int32_t *gains, int32_t *u, int32_t *gain) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && gains && u && gain, CEN_EINVAL, "cen_shard_pick: null argument");
  cen::shard_pick(job, gains, u, gain);
  CEN_API_END
}

int cen_shard_apply(cen_job *job, int32_t u, uint64_t *newly_covered) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && newly_covered, CEN_EINVAL, "cen_shard_apply: null argument");
  cen::shard_apply(job, u, newly_covered);
  CEN_API_END
}

int cen_shard_rade(cen_job *job, int32_t *R, int32_t *b) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && R && b, CEN_EINVAL, "cen_shard_rade: null argument");
  cen::shard_rade(job, R, b);
  CEN_API_END
}

int cen_shard_topk(cen_job *job, const int32_t *vals, int32_t nrows, int32_t k, int64_t *out) {
  CEN_API_BEGIN
  CEN_REQUIRE(job && vals && out, CEN_EINVAL, "cen_shard_topk: null argument");
  cen::shard_topk(job, vals, nrows, k, out);
  CEN_API_END
}

int cen_job_sampler_info(const cen_job *job, uint64_t *deferred_search, uint64_t *deferred_walk, uint64_t *migrated,
                         int32_t *slots, uint64_t *escalated) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_sampler_info: null job");
  if (deferred_search) *deferred_search = job->bidir_deferred_search;
  if (deferred_walk) *deferred_walk = job->bidir_deferred_walk;
  if (migrated) *migrated = job->bidir_migrated;
  if (slots) *slots = job->bws ? job->bws->nslots : 0;
  if (escalated) *escalated = job->bidir_escalated;
  CEN_API_END
}

int cen_graph_set_param(cen_graph *g, int32_t param, double value) {
  CEN_API_BEGIN
  CEN_REQUIRE(g, CEN_EINVAL, "cen_graph_set_param: null graph");
  CEN_REQUIRE(param >= 1 && param <= 9, CEN_EINVAL, "cen_graph_set_param: unknown parameter");
  cen_job probe;  // validates the value with the job rules
  apply_param(&probe, param, value);
  g->param[param] = value;
  g->param_set[param] = true;
  CEN_API_END
}

int cen_job_reset_stats(cen_job *job) {
  CEN_API_BEGIN
  CEN_REQUIRE(job, CEN_EINVAL, "cen_job_reset_stats: null job");
  CEN_CK(cudaStreamSynchronize(job->st));
  job->stats.reset(job->st);
  CEN_CK(cudaStreamSynchronize(job->st));
  CEN_API_END
}

}  // extern "C"
