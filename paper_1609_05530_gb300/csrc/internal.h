// internal.h -- interfaces between the C-ABI layer (api.cpp) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace cop {

// One subset to fit ("job"), as stored in the device schedule.
struct Job {
  int64_t off;      // first row of the subset in u / v
  int32_t m;        // rows in the subset
  int32_t family;   // COPULA_GAUSSIAN / FRANK / GUMBEL
  int32_t subset;   // output slot (global subset index)
  int32_t dataset;  // dataset index (batched calls)
  int64_t pad;
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
  void* gws_tab;          // global fallback for the per-rank tables: 2 Real per row
  void* gws_wu;           // global fallback for the u-order scan array: 1 Real per row
  int32_t tab_in_smem;
  int32_t wu_in_smem;
  int32_t max_iter;
  int32_t pad;
  double rtol;
  StartTables start;
};

// Dynamic shared memory of one resident CTA.
struct ResLayout {
  size_t pi_off, cnt_off, total;
};
__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline ResLayout res_layout(int m, int key_bytes, int real_bytes, bool tab_smem, bool wu_smem,
                                                int block) {
  size_t sortR = (size_t)m * key_bytes + 4 * (size_t)m;
  size_t tabR = (tab_smem ? 2 * (size_t)m * real_bytes : 0) + (wu_smem ? (size_t)m * real_bytes : 0);
  ResLayout L;
  L.pi_off = a16(sortR > tabR ? sortR : tabR);
  L.cnt_off = a16(L.pi_off + 2 * (size_t)m);
  L.total = L.cnt_off + (size_t)block * 32;  // 16 uint16 radix counters per thread
  return L;
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
