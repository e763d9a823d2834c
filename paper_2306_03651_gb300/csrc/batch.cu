// Batched Algorithm 1: many independent CentRA jobs driven concurrently.
//
// Each worker thread owns one CUDA stream and runs whole jobs (cen_run) on it;
// jobs are handed out longest-first (by arc count).  Kernels of different
// jobs overlap on the GPU, host synchronisation of one job hides behind
// another's kernels, and every job's result is exactly what cen_run gives for
// it alone: samples, signs and picks depend only on (graph, seed, parameters).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <string>
#include <numeric>
#include <thread>
#include <vector>

#include "job.cuh"

extern "C" int cen_run_result(const cen_job_spec *spec, void *stream, cen_job_result *out) {
  if (!spec || !out || !out->S) {
    cen::set_last_error("cen_run_result: null spec, result or S buffer");
    return CEN_EINVAL;
  }
  const auto t0 = std::chrono::steady_clock::now();
  out->start_s = 0.0;
  out->status = cen_run_ex(spec->graph, spec->k, spec->eps, spec->delta, spec->t, spec->seed, spec->m0, spec->m_cap,
                           &spec->opts, stream, out->S, &out->S_size, &out->covered, &out->m_final, &out->rounds,
                           out->log, out->log ? out->max_rounds : 0);
  out->end_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return out->status;
}

extern "C" int cen_run_batch(const cen_job_spec *specs, int32_t njobs, int32_t nworkers, cen_job_result *results) {
  try {
    CEN_REQUIRE(specs && results && njobs >= 0 && nworkers >= 1, CEN_EINVAL, "cen_run_batch: bad arguments");
    for (int32_t i = 0; i < njobs; ++i)
      CEN_REQUIRE(specs[i].graph && results[i].S, CEN_EINVAL, "cen_run_batch: null graph or S buffer");
    int dev = 0;
    CEN_CK(cudaGetDevice(&dev));
    std::vector<int32_t> order(njobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return specs[a].graph->nnz > specs[b].graph->nnz; });
    std::atomic<int32_t> next{0};
    const auto t0 = std::chrono::steady_clock::now();
    auto secs = [&] {
      return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    std::vector<char> ran(njobs, 0);
    std::mutex err_mu;
    std::string setup_err;  // why a worker could not start, if one could not
    auto worker = [&] {
      cudaStream_t st = nullptr;
      cudaError_t e = cudaSetDevice(dev);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e != cudaSuccess) {  // the other workers take the jobs; the call fails only if none could
        std::lock_guard<std::mutex> lk(err_mu);
        setup_err = std::string("cen_run_batch: worker setup failed: ") + cudaGetErrorString(e);
        return;
      }
      for (;;) {
        const int32_t q = next.fetch_add(1);
        if (q >= njobs) break;
        const int32_t i = order[q];
        const cen_job_spec &sp = specs[i];
        cen_job_result &r = results[i];
        r.start_s = secs();
        r.status = cen_run_ex(sp.graph, sp.k, sp.eps, sp.delta, sp.t, sp.seed, sp.m0, sp.m_cap, &sp.opts, st, r.S,
                              &r.S_size, &r.covered, &r.m_final, &r.rounds, r.log, r.log ? r.max_rounds : 0);
        r.end_s = secs();
        ran[i] = 1;
      }
      cudaStreamDestroy(st);
    };
    for (int32_t i = 0; i < njobs; ++i) results[i].status = CEN_ECUDA;  // until a worker runs it
    std::vector<std::thread> pool;
    const int32_t nw = std::min<int32_t>(nworkers, std::max<int32_t>(njobs, 1));
    try {
      for (int32_t w = 0; w < nw; ++w) pool.emplace_back(worker);
    } catch (...) {  // a thread could not be started: the ones that were finish the jobs
      if (pool.empty()) throw;
    }
    for (auto &th : pool) th.join();
    for (int32_t i = 0; i < njobs; ++i)
      if (!ran[i]) cen::fail(CEN_ECUDA, setup_err.empty() ? "cen_run_batch: a job was not run" : setup_err);
    return CEN_OK;
  } catch (const cen::Error &e) {
    cen::set_last_error(e.msg);
    return e.code;
  } catch (...) {
    cen::set_last_error("cen_run_batch: unexpected internal error");
    return CEN_ECUDA;
  }
}
