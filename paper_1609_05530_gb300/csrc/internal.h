// internal.h -- interfaces between the C-ABI layer (api.cpp) and the kernels.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "copula.h"

namespace cop {

// One subset to fit ("job"), as stored in the device schedule.
struct Job {
  int64_t off;      // first row of the subset in u / v
  int32_t m;        // rows in the subset
  int32_t family;   // COPULA_GAUSSIAN / FRANK / GUMBEL
  int32_t subset;   // output slot (global subset index)
  int32_t dataset;  // dataset index (batched calls)
  int32_t gs_mode;  // the variance's per-point store (ResidentArgs::gs_mode
                    // values), chosen from m alone so that a subset gets the
                    // same arithmetic in any batch
  int32_t pad;
};
static_assert(sizeof(Job) == 32, "Job layout");

// Spearman's rho of the Frank and Gumbel copulas on fixed parameter grids,
// used to turn the subset's rank correlation into a Newton start value.
constexpr int kStartN = 101;
constexpr double kFrankStart0 = 0.0, kFrankStartStep = 0.5;   // theta_j = 0.5 j
constexpr double kGumbelStart0 = 1.0, kGumbelStartStep = 0.49;  // theta_j = 1 + 0.49 j
struct StartTables {
  float frank_rho[kStartN];
  float gumbel_rho[kStartN];
};

// Threads per CTA for a subset of m rows (forced: 128/256/512 from the
// options, else 0).
inline int block_size_for(int m, int forced) {
  if (forced == 128 || forced == 256 || forced == 512) return forced;
  if (m <= 1536) return 128;
  if (m <= 6144) return 256;
  return 512;
}

// Fills the start tables (host; allocates nothing).
void build_start_tables(StartTables& T);

// Gauss-Legendre nodes x[i] and weights w[i] on [0, 1], n <= 128 (host).
void gauss_legendre01(int n, double* x, double* w);

// Parameter caps (a maximiser on a cap gets status BOUNDARY).
constexpr double kGaussCap = 1.0 - 1e-9;
constexpr double kFrankCap = 50.0;
constexpr double kGumbelCap = 50.0;

enum Mode : int32_t { MODE_FIT = 0, MODE_LOGLIK = 1 };

struct ResidentArgs {
  const void* u;
  const void* v;
  const Job* jobs;
  int32_t njobs;
  int32_t mode;
  int32_t* counter;       // job dispenser, zeroed before the launch
  double* theta;          // [S] fit results, indexed by Job::subset
  double* var;            // [S]
  int32_t* status;        // [S]
  double* info;           // [S] observed information -sum l_tt at theta_hat
  int32_t* iters;         // [S] Newton passes taken
  unsigned long long* phase_ns;  // [4 S] or null: global-timer stamps per subset
  const double* theta_in; // [S] (loglik mode)
  double* l_out;          // [S] (loglik mode, may be null)
  double* g_out;          // [S]
  double* h_out;          // [S]
  char* gws;              // global scratch, gws_stride bytes per CTA (blockIdx.x), or null:
  int64_t gws_stride;     //   the per-rank table and v-order scan array (2 Real per row)
  int64_t gws_gs_off;     //   when !tab_in_smem, and at gws_gs_off the variance's
                          //   per-point store of jobs with gs_mode 2
  int32_t tab_in_smem;    // (the variance's per-point store, per job: Job::gs_mode
                          // 0 none (terms evaluated again), 1 shared memory, 2 gws)
  int32_t max_iter;
  int32_t weight;         // Eq. 15 weight mode (COPULA_W_*)
  double rtol;
  double* comb;           // [B] Eq. 15 per dataset, or null: no combine
  const int64_t* dss;     // [B+1] first subset of each dataset
  int32_t* ds_done;       // [B] finished subsets per dataset, zeroed before the call
  StartTables start;
};

constexpr size_t kJobCounters = 64;  // job dispensers (one per launch bucket) ahead of the dataset counters

// Radix digit width of the block sort and its counters: 2^bits uint16 per
// thread.  4 bits: 5- and 6-bit digits save passes but their larger counter
// scans cost more (measured 4% and 23% slower on 10,000-row subsets).
constexpr int kRadixBits = 4;
constexpr int kRadixDigits = 1 << kRadixBits;
using SortCnt = uint16_t;
constexpr size_t kSortCntBytesPerThread = kRadixDigits * sizeof(SortCnt);

// Entries of the sandwich variance's per-point store of a resident subset
// of m rows at `block` threads: l_t and l_tu (and on the FP64 path the margin
// factor of the rank) for each thread's run of ((m + block - 1) / block) | 1
// consecutive points.
__host__ __device__ inline size_t var_store_entries(int m, int block, int real_bytes) {
  return (real_bytes == 8 ? 3 : 2) * (size_t)(((m + block - 1) / block) | 1) * (size_t)block;
}

// Dynamic shared memory of one resident CTA: the sort's keys and index
// arrays, later reused for the per-rank table and the v-order scan array
// (tab_smem) and the variance's per-point store (gs_smem); then pi and the
// radix counters.
struct ResLayout {
  size_t pi_off, cnt_off, total;
};
__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline ResLayout res_layout(int m, int key_bytes, int real_bytes, bool tab_smem, bool gs_smem,
                                                int block) {
  size_t sortR = (size_t)m * key_bytes + 4 * (size_t)m;
  size_t tabR = (tab_smem ? 2 * (size_t)m * real_bytes : 0) + (gs_smem ? var_store_entries(m, block, real_bytes) * real_bytes : 0);
  ResLayout L;
  L.pi_off = a16(sortR > tabR ? sortR : tabR);
  L.cnt_off = a16(L.pi_off + 2 * (size_t)m);
  L.total = L.cnt_off + (size_t)block * kSortCntBytesPerThread;  // radix counters
  return L;
}

// Raises a kernel's dynamic shared-memory limit on the current device when a
// launch needs more than any earlier one there (so steady-state launches,
// including those captured into CUDA graphs, make no attribute calls).
// granted: one entry per device, owned by the caller (one array per kernel).
// Safe to call from several host threads: the attribute is only ever raised,
// under one lock shared by all kernels.
inline std::mutex& smem_attr_mutex() {
  static std::mutex m;
  return m;
}
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t smem, std::atomic<int>* granted) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) {
    std::lock_guard<std::mutex> lock(smem_attr_mutex());
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (granted[dev].load(std::memory_order_acquire) >= (int)smem) return cudaSuccess;
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  if (granted[dev].load(std::memory_order_relaxed) >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) granted[dev].store((int)smem, std::memory_order_release);
  return e;
}

// Dynamic shared memory a resident CTA may request: the 227 KB per-CTA opt-in
// limit of sm_100-class GPUs less room for the kernels' static shared memory.
constexpr size_t kMaxSmem = 227 * 1024 - 2048;

cudaError_t launch_resident(int prec, int key_bytes, int block, int grid, size_t smem,
                            const ResidentArgs& a, cudaStream_t s);
cudaError_t launch_ranks(int key_bytes, int block, int grid, size_t smem, const void* x,
                         const Job* jobs, int njobs, int32_t* counter, int32_t* ranks,
                         cudaStream_t s);

struct CombineArgs {
  const double* theta;
  const double* var;
  const double* info;
  const int32_t* status;
  const int64_t* dataset_subset_start;  // [B+1]
  double* out;                          // [B]
  int32_t B;
  int32_t weight;
};
cudaError_t launch_combine(const CombineArgs& a, cudaStream_t s);

}  // namespace cop

namespace cop {

// ---------------------------------------------------------------------------
// Streaming path: subsets too large for one CTA's shared memory are ranked by
// a sample sort across many CTAs and fitted by one cooperative persistent
// kernel.  Work arrays are indexed by a compact position: subset s owns
// [c, c + m).
// ---------------------------------------------------------------------------
constexpr int kChunk = 16384;           // elements per chunk (bucketing, passes, scans)
constexpr int kSamplesPerBucket = 16;   // oversampling of the splitters
constexpr int kBucketMean32 = 3072;     // mean bucket size, FP32 keys
constexpr int kBucketMean64 = 2048;     // mean bucket size, FP64 keys
// Largest bucket one CTA orders in shared memory: ~3.8x the mean (with 16
// stratified samples per bucket an overflow has probability ~1e-11 per
// bucket), and small enough for two sorting CTAs per SM (keys + two uint16
// index buffers + counters <= 113 KB).  A larger bucket is ranked by direct
// pairwise counting over many CTAs instead (exact, O(size^2) work).
constexpr int kBucketCap32 = 12000;
constexpr int kBucketCap64 = 7800;
constexpr int kMaxBuckets32 = 1024;     // samples per subset <= 16384
constexpr int kMaxBuckets64 = 1024;
constexpr int64_t kStreamMax32 = (int64_t)kMaxBuckets32 * kBucketMean32;  // largest subset, FP32 keys
constexpr int64_t kStreamMax64 = (int64_t)kMaxBuckets64 * kBucketMean64;  // FP64 keys
static_assert(kStreamMax32 == COPULA_MAX_SUBSET_STREAM && kStreamMax64 == COPULA_MAX_SUBSET_STREAM_F64,
              "streaming limits in copula.h");

struct Seg {
  int64_t off;          // first row in u / v
  int64_t c;            // first compact position
  int64_t m;
  int64_t mat;          // first entry of its chunk x bucket count matrix
  int32_t family;
  int32_t subset;       // output slot
  int32_t nb;           // buckets (power of two)
  int32_t bucket_base;  // first global bucket
  int32_t chunk_first;
  int32_t chunk_count;
  int32_t dataset;
  int32_t pad;
};

struct Chunk {
  int32_t seg;
  int32_t len;
  int64_t start;  // first local position in the subset
};

struct SegState {
  double th, lo, hi, dlo, dhi, rtol;  // Newton (see Newton in fit_common.cuh)
  unsigned long long s_lo, s_hi;      // sum r_u r_v, exact 128-bit (start value)
  double mean;                        // variance: mean of xi
  double cE, ck0, ck1, ck2, cith;     // per-theta constants: Frank e^-|t|, k0, k1, k2; 1/theta
  int32_t it, max_iter, status, done;
  int32_t flags;                      // bit 0: NaN in the data; bit 2: a rank out of range reached pi
  int32_t probed;                     // bit 0 lower edge, bit 1 upper edge
  int32_t lo_natural;
  int32_t pre_it;                     // passes of the FP32 start search (FP64 path)
  unsigned long long inv;             // rank correlations: inversions of pi (discordant pairs)
};

struct StreamArgs {
  const void* u;
  const void* v;
  const Seg* segs;
  int32_t nseg;
  int32_t nchunk;
  const Chunk* chunks;
  const int32_t* bucket_seg;  // subset of each global bucket
  int32_t nbucket;
  int32_t mode;
  void* spl_key;              // splitter keys per global bucket slot
  uint32_t* spl_idx;          // splitter local indices
  uint32_t* bucket_cnt;
  uint32_t* bucket_start;
  uint32_t* mat;              // per subset [chunk][bucket] counts, then bases
  uint16_t* bucket_of;        // bucket of each compact position
  void* bkey;                 // keys in bucket order (row order inside a bucket)
  uint32_t* bidx;             // their local indices
  uint32_t* rank_u;           // ranks of u in row order (ranks call), else the rows in u-rank order
  uint32_t* rank_v;
  uint32_t* pi;               // v-rank of the point of u-rank p+1
  void* tab;                  // margin transform of u-rank p+1, in u-rank order (Real)
  void* tabv;                 // margin transform of v-rank pi[p], in u-rank order (Real)
  void* wu;                   // u-order scan array (Real)
  void* wv;                   // v-order scan array (Real)
  double* part;               // kPartStride doubles per chunk
  SegState* state;
  unsigned* barrier;          // 2 words: arrival count, generation
  int* error;                 // 1: a grid barrier gave up
  int64_t barrier_spins;      // polls (256 ns apart) before a grid barrier gives up
  int32_t barrier_phantom;    // arrivals a barrier waits for beyond the grid (0; > 0 tests the give-up path)
  int32_t nstamps;            // entries of stamps
  unsigned long long* stamps; // optional: fit kernel start and each grid barrier's release (globaltimer ns)
  int32_t* counter;           // bucket-job dispenser
  int32_t* big_count;         // buckets above the shared-memory cap in the column being ranked
  int32_t* phase_ctr;         // per chunk sweep of the fit kernel: chunk dispenser (zeroed by the init kernel)
  int32_t nphase;             // their number
  double* theta;
  double* var;
  int32_t* status;
  double* info;
  int32_t* iters;
  const double* theta_in;     // loglik mode
  double* l_out;
  double* g_out;
  double* h_out;
  int32_t max_iter;
  int32_t weight;             // Eq. 15 weight mode
  double rtol;
  double* comb;               // as in ResidentArgs
  const int64_t* dss;
  int32_t* ds_done;
  StartTables start;
};
constexpr int kPartStride = 8;
// Chunk sweeps of the fit kernel besides the Newton passes (tables, the
// Gaussian sums, five variance sweeps), with room to spare.
constexpr int kFixedPhases = 16;
// Entries of the fit kernel's barrier timestamps (profiling; later barriers
// are not recorded).
constexpr int kStreamStamps = 256;

// One-time kernel attributes and occupancy of the streaming kernels (not a
// stream operation: call it outside graph capture).
cudaError_t stream_setup(int sms);
// Enqueues the streaming fit (or log-likelihood) of all large subsets on s.
// Number of kernels it launches: kStreamLaunches.
// ev: NULL or kStreamEvents events, recorded before the ranks of u, after
// them, after the ranks of v, after pi, and after the fit kernel.
constexpr int kStreamEvents = 5;
cudaError_t launch_stream(int prec, int key_bytes, const StreamArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr);
// init, 2 x (splitter, count, scan, scatter, rank of small and of large buckets, big-bucket list, big-bucket
// rank), pi, fit
constexpr int kStreamLaunches = 19;
// Sample Kendall's tau and Spearman's rho of every large subset (the
// streaming counterpart of copula_rank_corr's shared-memory kernel):
// ranks of both columns, pi and sum r_u r_v as for a fit, then the
// inversions of pi chunk by chunk; tau[subset], rho[subset] (NaN for a subset
// holding NaN or whose ranks are incomplete).  Workspace as for a fit;
// kStreamRankCorrLaunches kernels.
cudaError_t launch_stream_rank_corr(int key_bytes, const StreamArgs& a, double* tau, double* rho, cudaStream_t s);
constexpr int kStreamRankCorrLaunches = 21;
// Ranks of one column for the large subsets, written to ranks_out at their
// rows (copula_ranks).
cudaError_t launch_stream_ranks(int key_bytes, const StreamArgs& a, const void* x, int32_t* ranks_out,
                                cudaStream_t s);

// Grows ctx's pinned schedule staging to at least bytes now (api.cpp).
int ctx_reserve_staging(copula_ctx* ctx, size_t bytes);

}  // namespace cop
