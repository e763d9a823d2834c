// Internal layout of a CentRA job (the growing sample H and its workspaces).
#pragma once
#include <memory>
#include <vector>

#include "common.cuh"

namespace cen {

// Workspace of the bit-parallel sampler.  A wave handles W = 64 G samples;
// every per-vertex set is G 64-bit words (bit b of word g = slot 64 g + b),
// stored vertex-major: word (v, g) at index v * G + g.
struct WaveWS {
  int G = 0;                                  // words per vertex in the current wave
  DevBuf vis;                                 // [n][G] reached so far
  std::vector<std::unique_ptr<DevBuf>> lev;   // lev[L]: [n][G] nodes at distance exactly L
  DevBuf lev_ptrs;                            // device array of lev[L] pointers
  int lev_ptrs_n = 0;
  DevBuf tmp;                                 // [n][G] cone scratch, kept zero between uses
  DevBuf any;                                 // [n][G] cone slots of each node (all levels)
  DevBuf base;                                // [n*G+1] exclusive prefix of their popcounts
  DevBuf cnt;                                 // [n*G] popcounts (scan input)
  DevBuf sigc;                                // compact path counts, one per (node, cone slot)
  DevBuf ovf;                                 // [n][G] path-count overflow flags
  DevBuf slots;                               // per slot: j (u64), s, t, d (int32)
  DevBuf ctl;                                 // control block (see sampler.cu)
  DevBuf jlist;                               // explicit sample ids for a re-run
  DevBuf woff;                                // wave-local member offsets per slot
  DevBuf lens, exoff, scan_tmp;               // offsets of appended samples (workspace 0)
  void *host = nullptr;                       // pinned staging for this pipeline
  size_t host_bytes = 0;
  cudaStream_t own_stream = nullptr;          // stream of an extra pipeline (null for the job's)
  // Buffers of an extra pipeline are freed in order on the legacy stream
  // after that pipeline's own stream has drained, then the stream goes.
  ~WaveWS() {
    if (own_stream) {
      cudaStreamSynchronize(own_stream);
      for (DevBuf *b : {&vis, &lev_ptrs, &tmp, &any, &base, &cnt, &sigc, &ovf, &slots, &ctl, &jlist, &woff, &lens,
                        &exoff, &scan_tmp, &arcs, &arc_range})
        b->st = nullptr;
      for (auto &l : lev) l->st = nullptr;
    }
    if (host) pinned_give(host, host_bytes);  // its stream has drained (the job's stream is synced at free)
    if (own_stream) cudaStreamDestroy(own_stream);
  }
  DevBuf arcs;                                // cone arc log of the current wave
  size_t arc_cap = 0;                         // its capacity in arcs
  DevBuf arc_range;                           // per level: [first, end) of its logged arcs
};

// Workspace of the bidirectional sampler (bidir.cu): for each of `nslots`
// resident CTAs, a small table of H1 entries (0: none) and a large one of H2
// = 4 QC entries, zeroed once (entries are epoch-stamped, so nothing is
// cleared between samples), seven lists of QC entries (two ball queues, two
// cone lists, heavy rows, crossing-arc tails and heads) and H2 path counts.
// Nothing in it grows with the graph.
struct BiCtl {
  unsigned long long next;     // next sample, relative to the launch's first
  unsigned long long cursor;   // arena entries reserved
  unsigned long long nsearch;  // samples left whole to the bit-parallel sampler
  unsigned long long nwalk;    // samples whose walk is left to it (distance known)
  unsigned long long nmigrate; // searches that outgrew the small table
  unsigned long long nbig;     // warp searches handed on to the CTA launch
  unsigned long long bignext;  // next of them for the CTA launch
  int err;
  int pad;
};
struct BiWS {
  DevBuf tab1, tab2, lists, sig, epochs, ctl, aoff, dsearch, dwalk, arena;
  DevBuf tabw, epw;        // warp searches: node tables and epochs (none when WQ = 0)
  DevBuf big;              // ids the warp searches hand on to the CTA searches
  int nslots = 0;
  int64_t QC = 0;
  int64_t H1 = 0;
  int64_t H2 = 0;
  int64_t WQ = 0;          // entries of each list of a warp search; 0: CTA searches only
  int dev = -1;
};
// A finished job's workspace is kept for the next job of the same shape on the
// same device (its state words stay valid under the persisting epochs, so it
// is not cleared again); at most a few are kept.
std::unique_ptr<BiWS> bidir_take(int dev, int64_t QC, int64_t H1, int slots, int64_t WQ);
void bidir_give(std::unique_ptr<BiWS> w);
void bidir_drop_cached();
// Lets the current device's stream-ordered pool keep freed memory for reuse.
void keep_pool_memory();

}  // namespace cen

namespace cen {
// A second stream of a job, with the events that fork work onto it and join
// it back (cen_cover_and_mcera); created on first use.
struct AuxStream {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  AuxStream() = default;
  AuxStream(const AuxStream &) = delete;
  AuxStream &operator=(const AuxStream &) = delete;
  ~AuxStream() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (st) cudaStreamDestroy(st);
  }
  void ensure() {
    if (st) return;
    CEN_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CEN_CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    CEN_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  }
};
}  // namespace cen

struct cen_job {
  const cen_graph *g = nullptr;
  uint64_t seed = 0;
  // store position p holds sample id p * id_stride + id_offset (cen_job_set_ids)
  uint64_t id_stride = 1, id_offset = 0;
  int64_t shard_greedy_m = -1;  // m when cen_shard_greedy_begin last ran
  cen::SampleKey key() const { return cen::SampleKey{seed, id_stride, id_offset}; }
  int32_t t = 0;
  int32_t nw = 0;  // sign words per sample = ceil(t / 32)
  cudaStream_t st = nullptr;
  uint64_t m = 0;         // samples
  int64_t members = 0;    // sum of |h|
  // sample store (device): hoff[m+1], hmem[members], per-sample s, t, d, sign words
  cen::DevBuf hoff, hmem, ps, pt, pd, sign, bmax;
  // node -> sample incidence (rebuilt lazily when m changed)
  cen::DevBuf c, noff, nsamp, cursor;
  uint64_t inc_m = ~0ull;
  // greedy workspace
  cen::DevBuf gain, covered, gctl;
  // AMCERA workspace
  cen::DevBuf R, selh, selst;
  int32_t rade_valid_k = -1;
  // greedyCover and AMCERA side by side (cen_cover_and_mcera)
  cen::AuxStream aux;
  // sampler pipelines (workspace 0 runs on the job's stream)
  std::vector<std::unique_ptr<cen::WaveWS>> wws;
  int wave_streams = 4;  // waves of one cen_sample call run at once
  double push_ratio = 4.0;  // expand top-down while frontier out-arcs * push_ratio < arcs
  // scratch for scans
  cen::DevBuf scan_tmp;
  // pinned host staging
  void *host = nullptr;
  size_t host_bytes = 0;
  cen::Stats stats;
  size_t level_budget = (size_t)1 << 30;   // bytes allowed for one [n][G] level array
  int max_wave_words = 32;                 // upper bound on G (wave width / 64)
  // bidirectional sampler
  std::unique_ptr<cen::BiWS> bws;
  int sampler = 0;                          // 0 bidirectional (bit-parallel for what it defers), 1 bit-parallel
  size_t bidir_budget = (size_t)16 << 30;   // bytes of per-slot workspace
  int64_t bidir_queue = (int64_t)1 << 16;   // entries per ball / cone list
  int64_t bidir_table = -1;                 // small-table entries per CTA (-1: sized for L2, 0: none)
  int bidir_warps = -1;  // 1: warp searches, what they hand on by CTAs; 0: CTAs only; -1: by the graph's record
  uint64_t bidir_deferred_search = 0;       // samples it left whole to the bit-parallel sampler
  uint64_t bidir_deferred_walk = 0;         // samples whose walk it left (distance known)
  uint64_t bidir_migrated = 0;              // searches that outgrew the small table
  uint64_t bidir_escalated = 0;             // warp searches handed to their CTA
  // hyper-edge space (CEN_SPACE_*) and the kappa of the kappa-path space
  int32_t space = 0;
  int32_t kappa = 0;
  cen::DevBuf space_buf;                    // kappa-path walks before they are packed
};

namespace cen {
void sample_append(cen_job *job, uint64_t m_new);
void bidir_launch(cen_job *job, uint64_t j0, uint64_t count, int64_t arena_cap);
// Entries of each list of a warp search for a CTA queue of QC entries (0: warp searches off).
int64_t bidir_warp_queue(int64_t QC);
size_t bidir_warp_bytes_per_slot();
// E[d^2] / E[d] of the graph's degrees (out and in, the larger), computed once.
double graph_branching(const cen_graph *g, cudaStream_t st);
// The bit-parallel sampler's chunk tables of the graph's long out- and in-rows
// (built on first use, on st).
const ChunkTable &graph_out_chunks(const cen_graph *g, cudaStream_t st);
const ChunkTable &graph_in_chunks(const cen_graph *g, cudaStream_t st);
size_t bidir_warp_table_bytes_per_slot();
size_t bidir_warp_epoch_bytes_per_slot();
void kpath_sample(cen_job *job, uint64_t j0, uint64_t count, int32_t *out, const int64_t *hoff);
int64_t triangle_index(cen_job *job);
void triangle_sample(cen_job *job, uint64_t j0, uint64_t count);
int max_kappa();
int bidir_resident_slots();
void build_incidence(cen_job *job);
void greedy_cover(cen_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered);
void mcera(cen_job *job, int32_t k, int64_t *Rnum, int64_t *Wnum, int32_t *b);
void shard_greedy_begin(cen_job *job);
void shard_gains(const cen_job *job, int32_t *dst);
void shard_pick(cen_job *job, const int32_t *gains, int32_t *u, int32_t *gain);
void shard_apply(cen_job *job, int32_t u, uint64_t *newly);
void shard_rade(cen_job *job, int32_t *R_out, int32_t *b);
void shard_topk(cen_job *job, const int32_t *vals, int32_t nrows, int32_t k, int64_t *out);
size_t greedy_result_bytes(int32_t k);
void greedy_prepare(cen_job *job, int32_t k);
void greedy_enqueue(cen_job *job, int32_t k, cudaStream_t run, void *hdst);
void greedy_result(const void *h, int32_t *S, int32_t *S_size, uint64_t *covered);
size_t mcera_result_bytes(const cen_job *job);
void mcera_prepare(cen_job *job, int32_t k);
void mcera_enqueue(cen_job *job, int32_t k, cudaStream_t run, void *hdst);
void mcera_result(cen_job *job, int32_t k, const void *h, int64_t *Rnum, int64_t *Wnum, int32_t *b);
void cover_and_mcera(cen_job *job, int32_t k, int32_t *S, int32_t *S_size, uint64_t *covered, int64_t *Rnum,
                     int64_t *Wnum, int32_t *b);
void graph_build(cen_graph *g, const int64_t *off, const int32_t *col, bool on_device, Stats *S);
void graph_canonicalize(cen_graph *g, const int64_t *off, const int32_t *col, int64_t nnz, bool on_device,
                        bool symmetrize, Stats *S);
void *host_staging(cen_job *job, size_t bytes);
}  // namespace cen
