// Shared internals of libcen: error handling, stream-ordered device buffers,
// the Philox4x32-10 generator, warp helpers and per-kernel accounting.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cen.h"

namespace cen {

// NVTX range for the profiler timeline (no cost when no tool is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

// ----------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string &msg);
void set_last_error(const std::string &msg);

#define CEN_CK(call)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      ::cen::fail(e_ == cudaErrorMemoryAllocation ? CEN_ENOMEM : CEN_ECUDA,                       \
                  std::string(#call) + ": " + cudaGetErrorString(e_) + " (" + __FILE__ + ":" +      \
                      std::to_string(__LINE__) + ")");                                            \
  } while (0)

#define CEN_REQUIRE(cond, code, text) \
  do {                                \
    if (!(cond)) ::cen::fail((code), (text)); \
  } while (0)

// Testing hook: when armed, the n-th device allocation from now fails with
// CEN_ENOMEM as if the device were full (see cen_debug_fail_alloc).
void alloc_fault_tick();

// ------------------------------------------------ device memory source
// An allocator installed by cen_set_allocator.  Installed ones are never
// freed, so a buffer can always go back to the one that made it.
struct Allocator {
  cen_alloc_fn alloc;
  cen_free_fn free;
  void *ctx;
};
void set_allocator(cen_alloc_fn alloc, cen_free_fn free_fn, void *ctx);
// Allocates `bytes` for use on stream s from the installed allocator (*al set
// to it) or, with none, stream-ordered from the device pool (*al = null).
void *dev_alloc(size_t bytes, cudaStream_t s, const Allocator **al);
// Returns p to its allocator: stream-ordered on s for the pool; for an
// installed allocator, once s has drained.  Never throws.
void dev_free(void *p, size_t bytes, cudaStream_t s, const Allocator *al) noexcept;

// ------------------------------------------------ stream-ordered buffers
// Device memory owned by the library, allocated and freed in stream order.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  const Allocator *al = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) dev_free(p, bytes, st, al);
    p = nullptr;
    bytes = 0;
    al = nullptr;
  }
  // Ensure capacity >= need bytes; keeps the first `keep` bytes of old content.
  void ensure(size_t need, cudaStream_t s, size_t keep = 0) {
    st = s;
    if (need <= bytes && p) return;
    size_t cap = bytes ? bytes : 256;
    while (cap < need) cap = cap + cap / 2 + 256;
    const Allocator *nal = nullptr;
    void *np = dev_alloc(cap, s, &nal);
    if (p && keep) {
      cudaError_t e = cudaMemcpyAsync(np, p, keep < bytes ? keep : bytes, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) dev_free(np, cap, s, nal);
      CEN_CK(e);
    }
    if (p) dev_free(p, bytes, s, al);
    p = np;
    bytes = cap;
    al = nal;
  }
  // Capacity of exactly `need` bytes when it has to grow (large workspaces).
  void ensure_exact(size_t need, cudaStream_t s) {
    st = s;
    if (need <= bytes && p) return;
    release();
    p = dev_alloc(need, s, &al);
    bytes = need;
  }
  template <class T>
  T *as() const { return static_cast<T *>(p); }
  void swap(DevBuf &o) {
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
    std::swap(st, o.st);
    std::swap(al, o.al);
  }
};

// ------------------------------------------------------------- Philox
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies counter words 0 and 2 by the two round multipliers, the high
// halves are mixed with words 1 and 3 and the round key; the key advances by
// the two Weyl increments.  Counter for sample j: (j_lo, j_hi, purpose, word3).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kPurposeS = 0u, kPurposeT = 1u, kPurposeWalk0 = 2u, kPurposeSign = 0xFFFFFFFFu;

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += kPhiloxW0;
    k.y += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint64_t j, uint32_t purpose, uint32_t w3) {
  return philox(make_uint4((uint32_t)j, (uint32_t)(j >> 32), purpose, w3),
                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// A job's Philox key and its map from store positions to sample ids:
// position p holds sample id p * stride + offset (stride 1 and offset 0 unless
// the job holds one shard of a sample split over several GPUs).  Every draw of
// a sample is keyed by its id, so a sample does not depend on where it is stored.
struct SampleKey {
  uint64_t seed, stride, offset;
  __host__ __device__ __forceinline__ uint64_t id(uint64_t p) const { return p * stride + offset; }
};

typedef unsigned __int128 u128;

// Uniform integer in [0, B), 1 <= B <= 2^64 - 1: bitmask rejection with
// mask = 2^ceil(log2 B) - 1 over the low 64 bits of block (j, purpose, a).
__device__ __forceinline__ uint64_t uniform_below64(uint64_t seed, uint64_t j, uint32_t purpose, uint64_t B) {
  const int bits = (B <= 1) ? 0 : 64 - __clzll((long long)(B - 1));
  const uint64_t mask = bits == 64 ? ~0ull : ((1ull << bits) - 1ull);
  for (uint32_t a = 0;; ++a) {
    const uint4 x = philox_block(seed, j, purpose, a);
    const uint64_t v = ((uint64_t)x.x | ((uint64_t)x.y << 32)) & mask;
    if (v < B) return v;
  }
}

// Same rule for 1 <= B < 2^128: 64 bits while B <= 2^64, else all 128 bits.
__device__ __forceinline__ u128 uniform_below128(uint64_t seed, uint64_t j, uint32_t purpose, u128 B) {
  const u128 bm1 = B - 1;
  const uint64_t hi = (uint64_t)(bm1 >> 64), lo = (uint64_t)bm1;
  const int bits = B <= 1 ? 0 : (hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo));
  const u128 mask = bits == 128 ? ~(u128)0 : (((u128)1 << bits) - 1);
  const bool wide = B > ((u128)1 << 64);
  for (uint32_t a = 0;; ++a) {
    const uint4 x = philox_block(seed, j, purpose, a);
    u128 v = (u128)x.x | ((u128)x.y << 32);
    if (wide) v |= ((u128)x.z << 64) | ((u128)x.w << 96);
    v &= mask;
    if (v < B) return v;
  }
}

// ----------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------- accounting
enum KClass : int {
  K_PAIRS = 0,   // pair draw + wave init
  K_TCHECK,      // target check before each level
  K_PUSH,        // top-down level expansion
  K_PULL,        // bottom-up level expansion
  K_LEVEL_FIN,   // level finalize (mask, visited, frontier list)
  K_CONE,        // backward cone pass
  K_SIGMA,       // path counts on the cone
  K_WALK,        // backward walk + hyper-edge write
  K_APPEND,      // lengths / offsets of new samples
  K_SIGN,        // sign words
  K_TRANSPOSE,   // node -> sample incidence
  K_GREEDY,      // greedy argmax + update
  K_RADE,        // R_q^u accumulation
  K_SELECT,      // top-k positive sums
  K_GRAPH,       // graph validation / in-CSR
  K_MISC,        // scans, fills
  K_BIDIR,       // bidirectional sampler (search, cone, counts, walk)
  K_SPACE,       // samplers of the kappa-path and triangle spaces
  K_COUNT
};
static_assert(K_COUNT <= CEN_NKCLASS, "too many kernel classes");
extern const char *const kClassNames[K_COUNT];

struct Stats {
  cen_kstat k[CEN_NKCLASS];
  bool timing = false;
  std::mutex mu;  // wave pipelines of one job launch from several threads
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  uint64_t *d_units = nullptr;  // device counters [K_COUNT]
  const Allocator *d_units_al = nullptr;
  Stats();
  ~Stats();
  void init(cudaStream_t st);
  cudaEvent_t ev();
  void begin(int cls, cudaStream_t st, cudaEvent_t *a, cudaEvent_t *b);
  void end(int cls, cudaStream_t st, cudaEvent_t a, cudaEvent_t b);
  void resolve();  // stream must be synchronized
  void reset(cudaStream_t st);
};

// Launch bookkeeping: counts every launch of a class and, with timing on,
// brackets it by events on the launch stream.
template <class F>
inline void launch(Stats *S, int cls, cudaStream_t st, F &&f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (S) S->begin(cls, st, &a, &b);
  f();
  CEN_CK(cudaGetLastError());
  if (S) S->end(cls, st, a, b);
}

// Blocks of `block` threads that are resident at once on the current device
// (SM count x blocks per SM for this kernel), cached per kernel.
int resident_grid(const void *kernel, int block);
// Page-locked host buffers, reused across jobs (capacity in *cap, >= bytes).
// A buffer is given back only once no copy into or out of it is in flight.
void *pinned_take(size_t bytes, size_t *cap);
void pinned_give(void *p, size_t cap);
void pinned_drop_cached();
// Blocks for a cooperative launch of `kernel` (all resident at once: one per
// SM up to what fits), or 0 when the device cannot launch cooperatively.
int cooperative_grid(const void *kernel, int block);

// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// Blocks for `items` work items at `per_block` each, at most `cap` (default:
// 32 blocks per SM of the current device).
inline int grid_for(size_t items, int per_block, int cap = 0) {
  if (cap <= 0) cap = sm_count() * 32;
  size_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------- prims
// Device-wide exclusive scan of `n` int64 values (in may equal out); writes
// the total to *d_total (device) when non-null.
void exclusive_scan_i64(const int64_t *in, int64_t *out, size_t n, int64_t *d_total, DevBuf &tmp, cudaStream_t st,
                        Stats *S);
// Exclusive scan of int32 counts into int64 offsets (out has n+1 entries, out[n] = total).
void counts_to_offsets(const int32_t *cnt, int64_t *out, size_t n, DevBuf &tmp, cudaStream_t st, Stats *S);
// Stable LSD radix sort of (key, value) uint32 pairs by key, keys < 2^key_bits.
// Result lands in keys/vals (ping-pong through the scratch buffers).
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, size_t n, int key_bits, DevBuf &k2, DevBuf &v2, DevBuf &hist,
                      DevBuf &tmp, cudaStream_t st, Stats *S);

}  // namespace cen

// -------------------------------------------------------- opaque handles
// Rows longer than kHeavyRow arcs are also split into kChunk-arc pieces so
// that one long row is spread over many warps (see the *_heavy kernels).
namespace cen {
constexpr int kHeavyRow = 256;
constexpr int kChunk = 256;
struct ChunkTable {
  DevBuf w, beg;    // chunk -> row id, first arc
  int64_t count = 0;
  const int32_t *rows() const { return w.as<int32_t>(); }
  const int64_t *begins() const { return beg.as<int64_t>(); }
};
}  // namespace cen

struct cen_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int directed = 0;
  cudaStream_t st = nullptr;
  cen::DevBuf off, col, roff, rcol;  // roff/rcol empty when undirected (alias off/col)
  // Chunk tables of the bit-parallel sampler (in_chunks_own only when
  // directed), built on first use (graph_out_chunks / graph_in_chunks).
  mutable std::mutex chunks_mu;
  mutable bool chunks_built = false;
  mutable cen::ChunkTable out_chunks, in_chunks_own;
  double param[10] = {};   // tuning defaults for jobs on this graph, by CEN_PARAM_* id
  bool param_set[10] = {};  // which of them were set
  // Set once most bidirectional searches on this graph outgrew their node
  // table: later jobs (without an explicit table size) use the large table only.
  mutable std::atomic<bool> bidir_table_off{false};
  // Set once a call handed more than 30% of its warp searches on to CTAs:
  // later jobs (without an explicit setting) search with whole CTAs only.
  mutable std::atomic<bool> bidir_warps_off{false};
  // E[d^2] / E[d] over the out- and in-degrees (the larger): how many arcs a
  // frontier node's neighbour has on average; computed when the graph loads.
  mutable std::mutex branching_mu;
  mutable double branching = -1.0;
  // Triangle ranks (triangle space): exclusive prefix of per-arc counts, built once.
  std::mutex tri_mu;
  cen::DevBuf tri_off;
  int64_t tri_total = -1;
  const int64_t *in_off() const { return directed ? roff.as<int64_t>() : off.as<int64_t>(); }
  const int32_t *in_col() const { return directed ? rcol.as<int32_t>() : col.as<int32_t>(); }
};
