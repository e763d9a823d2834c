// Generic device primitives of libcen: exclusive scans and a stable LSD radix
// sort of (key, value) pairs; plus error and accounting plumbing.
#include <stdio.h>

#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace cen {

// ------------------------------------------------------------- errors
static thread_local std::string g_last_error;
void set_last_error(const std::string &msg) { g_last_error = msg; }
const std::string &last_error() { return g_last_error; }
[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

// --------------------------------------------------------- accounting
const char *const kClassNames[K_COUNT] = {"pairs", "target_check", "expand_push", "expand_pull", "level_finalize",
                                          "cone", "cone_sigma", "walk", "append", "sign", "transpose", "greedy",
                                          "rade", "select", "graph", "misc", "bidir", "space"};

Stats::Stats() {
  memset(k, 0, sizeof(k));
  for (int c = 0; c < K_COUNT; ++c) snprintf(k[c].name, sizeof(k[c].name), "%s", kClassNames[c]);
}
Stats::~Stats() {
  for (auto &p : pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
  if (d_units) dev_free(d_units, sizeof(uint64_t) * K_COUNT, nullptr, d_units_al);
}
void Stats::init(cudaStream_t st) {
  if (!d_units) {
    d_units = (uint64_t *)dev_alloc(sizeof(uint64_t) * K_COUNT, st, &d_units_al);
    CEN_CK(cudaMemsetAsync(d_units, 0, sizeof(uint64_t) * K_COUNT, st));
  }
}
cudaEvent_t Stats::ev() {  // caller holds mu
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CEN_CK(cudaEventCreate(&e));
  return e;
}
void Stats::begin(int cls, cudaStream_t st, cudaEvent_t *a, cudaEvent_t *b) {
  std::lock_guard<std::mutex> lock(mu);
  k[cls].launches++;
  if (!timing) return;
  *a = ev();
  *b = ev();
  CEN_CK(cudaEventRecord(*a, st));
}
void Stats::end(int cls, cudaStream_t st, cudaEvent_t a, cudaEvent_t b) {
  if (!a) return;
  std::lock_guard<std::mutex> lock(mu);
  CEN_CK(cudaEventRecord(b, st));
  pending.push_back({cls, a, b});
}
void Stats::resolve() {
  std::lock_guard<std::mutex> lock(mu);
  for (auto &p : pending) {
    float ms = 0.f;
    CEN_CK(cudaEventElapsedTime(&ms, p.a, p.b));
    k[p.cls].ms += ms;
    k[p.cls].timed++;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}
void Stats::reset(cudaStream_t st) {
  resolve();
  std::lock_guard<std::mutex> lock(mu);
  for (int c = 0; c < CEN_NKCLASS; ++c) {
    k[c].launches = 0;
    k[c].ms = 0;
    k[c].timed = 0;
    k[c].units = 0;
  }
  if (d_units) CEN_CK(cudaMemsetAsync(d_units, 0, sizeof(uint64_t) * K_COUNT, st));
}

// ------------------------------------------------------ fault hook
static std::atomic<long long> g_fail_alloc{0};
void alloc_fault_tick() {
  if (g_fail_alloc.load(std::memory_order_relaxed) <= 0) return;
  if (g_fail_alloc.fetch_sub(1) == 1) fail(CEN_ENOMEM, "device allocation failed (injected by cen_debug_fail_alloc)");
}

// ------------------------------------------------------ memory source
static std::atomic<const Allocator *> g_allocator{nullptr};

void set_allocator(cen_alloc_fn alloc, cen_free_fn free_fn, void *ctx) {
  static std::mutex mu;
  static std::vector<std::unique_ptr<Allocator>> installed;  // kept for the buffers they made
  std::lock_guard<std::mutex> lk(mu);
  if (!alloc) {
    g_allocator.store(nullptr);
    return;
  }
  installed.emplace_back(new Allocator{alloc, free_fn, ctx});
  g_allocator.store(installed.back().get());
}

void *dev_alloc(size_t bytes, cudaStream_t s, const Allocator **al) {
  alloc_fault_tick();
  const Allocator *a = g_allocator.load();
  void *p = nullptr;
  if (a) {
    p = a->alloc(bytes, (void *)s, a->ctx);
    CEN_REQUIRE(p, CEN_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (installed allocator)");
  } else {
    CEN_CK(cudaMallocAsync(&p, bytes, s));
  }
  *al = a;
  return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s, const Allocator *al) noexcept {
  if (!p) return;
  if (al) {
    cudaStreamSynchronize(s);  // the allocator may hand p out again at once
    al->free(p, bytes, (void *)s, al->ctx);
  } else {
    cudaFreeAsync(p, s);
  }
}

// ------------------------------------------------------ occupancy
int sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  CEN_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  CEN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cache[dev] = sms > 0 ? sms : 1;
  return cache[dev];
}

int resident_grid(const void *kernel, int block) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> cache;
  int dev = 0;
  CEN_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, kernel});
  if (it != cache.end()) return it->second;
  int sms = 0, per = 0;
  CEN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CEN_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0));
  const int g = sms * (per > 0 ? per : 1);
  cache[{dev, kernel}] = g;
  return g;
}

// -------------------------------------------------------------- scans
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *smem_warp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) smem_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  T before = warp ? smem_warp[warp - 1] : T(0);
  *total = smem_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

template <class T>
__global__ void scan_partials(const T *in, size_t n, T *part) {
  __shared__ T sw[32];
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  T tot;
  block_exclusive_scan<T>(s, sw, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_top(T *part, size_t nparts, T *d_total) {
  __shared__ T sw[32];
  T carry = 0;
  for (size_t base = 0; base < nparts; base += blockDim.x) {
    size_t i = base + threadIdx.x;
    T v = i < nparts ? part[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, sw, &tot);
    if (i < nparts) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

template <class T>
__global__ void scan_final(const T *in, T *out, size_t n, const T *part) {
  __shared__ T sw[32];
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    s += v[i];
  }
  T tot;
  T ex = block_exclusive_scan<T>(s, sw, &tot) + part[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

template <class T>
static void exclusive_scan(const T *in, T *out, size_t n, T *d_total, DevBuf &tmp, cudaStream_t st, Stats *S) {
  if (n == 0) {
    if (d_total) CEN_CK(cudaMemsetAsync(d_total, 0, sizeof(T), st));
    return;
  }
  size_t nparts = (n + kScanTile - 1) / kScanTile;
  tmp.ensure(nparts * sizeof(T), st);
  T *part = tmp.as<T>();
  launch(S, K_MISC, st, [&] { scan_partials<T><<<(unsigned)nparts, kScanThreads, 0, st>>>(in, n, part); });
  launch(S, K_MISC, st, [&] { scan_top<T><<<1, kScanThreads, 0, st>>>(part, nparts, d_total); });
  launch(S, K_MISC, st, [&] { scan_final<T><<<(unsigned)nparts, kScanThreads, 0, st>>>(in, out, n, part); });
}

void exclusive_scan_i64(const int64_t *in, int64_t *out, size_t n, int64_t *d_total, DevBuf &tmp, cudaStream_t st,
                        Stats *S) {
  exclusive_scan<int64_t>(in, out, n, d_total, tmp, st, S);
}

__global__ void widen_i32(const int32_t *cnt, int64_t *out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = cnt[i];
}

void counts_to_offsets(const int32_t *cnt, int64_t *out, size_t n, DevBuf &tmp, cudaStream_t st, Stats *S) {
  if (n) launch(S, K_MISC, st, [&] { widen_i32<<<grid_for(n, 256), 256, 0, st>>>(cnt, out, n); });
  exclusive_scan<int64_t>(out, out, n, out + n, tmp, st, S);
}

// --------------------------------------------------------- radix sort
// One 8-bit digit per pass.  Pass: per-tile digit histograms (digit-major),
// one exclusive scan over them gives every (digit, tile) its output base, and
// the scatter ranks equal digits inside a tile in input order (stable).
constexpr int kRsThreads = 256, kRsRounds = 8, kRsTile = kRsThreads * kRsRounds;

__global__ void rs_hist(const uint32_t *keys, size_t n, int shift, uint32_t *hist, int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
    size_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout, size_t n,
                           int shift, const uint32_t *hist, int ntiles) {
  __shared__ uint32_t base_off[256];
  __shared__ uint32_t running[256];
  __shared__ uint32_t wcnt[kRsThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base_off[tid] = hist[(size_t)tid * ntiles + blockIdx.x];
  running[tid] = 0;
  const size_t tile = (size_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
    const size_t idx = tile + (size_t)r * kRsThreads + tid;
    const bool valid = idx < n;
    const uint32_t k = valid ? kin[idx] : 0u, v = valid ? vin[idx] : 0u;
    const uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
    for (int i = tid; i < (kRsThreads / 32) * 256; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned before = peers & ((1u << lane) - 1u);
    if (valid && before == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = running[tid];
#pragma unroll
      for (int w = 0; w < kRsThreads / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      running[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base_off[d] + wcnt[warp][d] + __popc(before);
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
  }
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, size_t n, int key_bits, DevBuf &k2, DevBuf &v2, DevBuf &hist,
                      DevBuf &tmp, cudaStream_t st, Stats *S) {
  if (n <= 1) return;
  CEN_REQUIRE(n < (1ull << 32), CEN_EINVAL, "radix_sort_pairs: too many elements");
  const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  k2.ensure(n * 4, st);
  v2.ensure(n * 4, st);
  hist.ensure((size_t)ntiles * 256 * 4, st);
  uint32_t *ka = keys, *va = vals, *kb = k2.as<uint32_t>(), *vb = v2.as<uint32_t>();
  const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    uint32_t *h = hist.as<uint32_t>();
    launch(S, K_MISC, st, [&] { rs_hist<<<ntiles, kRsThreads, 0, st>>>(ka, n, shift, h, ntiles); });
    exclusive_scan<uint32_t>(h, h, (size_t)ntiles * 256, nullptr, tmp, st, S);
    launch(S, K_MISC, st,
           [&] { rs_scatter<<<ntiles, kRsThreads, 0, st>>>(ka, va, kb, vb, n, shift, h, ntiles); });
    uint32_t *t;
    t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    CEN_CK(cudaMemcpyAsync(keys, ka, n * 4, cudaMemcpyDeviceToDevice, st));
    CEN_CK(cudaMemcpyAsync(vals, va, n * 4, cudaMemcpyDeviceToDevice, st));
  }
}

}  // namespace cen

extern "C" int cen_debug_fail_alloc(int64_t n) {
  if (n < 0) {
    cen::set_last_error("cen_debug_fail_alloc: n must be >= 0");
    return CEN_EINVAL;
  }
  cen::g_fail_alloc.store(n);
  return CEN_OK;
}

namespace cen {
// Stream-ordered frees return memory to the device's default pool; with the
// release threshold at its maximum the pool keeps it mapped for the next
// allocation instead of handing it back at every synchronisation.  Once per
// device; cen_release_cached trims the pool.
void keep_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}
}  // namespace cen

namespace cen {
int cooperative_grid(const void *kernel, int block) {
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) return 0;
  return sms * std::min(per_sm, 2);
}
}  // namespace cen

namespace cen {
// Pinned host buffers of finished jobs, kept for the next ones: allocating and
// freeing page-locked memory costs far more than a round's small copies.
namespace {
constexpr size_t kPinnedKeep = 16;
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<void *, size_t>> idle;
};
PinnedPool &pinned_pool() {
  static PinnedPool *p = new PinnedPool();  // never destroyed: nothing is freed after the runtime unloads
  return *p;
}
}  // namespace

void *pinned_take(size_t bytes, size_t *cap) {
  {
    PinnedPool &pp = pinned_pool();
    std::lock_guard<std::mutex> lk(pp.mu);
    size_t best = pp.idle.size();
    for (size_t i = 0; i < pp.idle.size(); ++i)
      if (pp.idle[i].second >= bytes && (best == pp.idle.size() || pp.idle[i].second < pp.idle[best].second)) best = i;
    if (best < pp.idle.size()) {
      void *p = pp.idle[best].first;
      *cap = pp.idle[best].second;
      pp.idle.erase(pp.idle.begin() + (ptrdiff_t)best);
      return p;
    }
  }
  size_t c = 4096;
  while (c < bytes) c *= 2;
  void *p = nullptr;
  CEN_CK(cudaMallocHost(&p, c));
  *cap = c;
  return p;
}

void pinned_give(void *p, size_t cap) {
  if (!p) return;
  PinnedPool &pp = pinned_pool();
  std::lock_guard<std::mutex> lk(pp.mu);
  pp.idle.emplace_back(p, cap);
  if (pp.idle.size() > kPinnedKeep) {
    cudaFreeHost(pp.idle.front().first);
    pp.idle.erase(pp.idle.begin());
  }
}

void pinned_drop_cached() {
  PinnedPool &pp = pinned_pool();
  std::lock_guard<std::mutex> lk(pp.mu);
  for (auto &e : pp.idle) cudaFreeHost(e.first);
  pp.idle.clear();
}
}  // namespace cen
