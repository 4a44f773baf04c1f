// noalloc.cu -- copula_fit_noalloc: the same fit as copula_fit for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator): code running under
// a fixed memory budget that owns every byte up front, plugins handed only
// their input and output buffers by a host application, or callers that must
// not enter the driver's allocator at all (to keep allocation latency and
// fragmentation out of a serving loop).  For them this entry point keeps its
// scratch -- the job schedule, the job counters, the dataset bounds and the
// per-subset variance / information / pass-count scratch -- in one
// file-scope __device__ array of fixed size instead of a caller-supplied
// workspace, and it allocates nothing, on the device or the host.
//
// The array holds at most kNoallocMaxSubsets subsets' scratch (about 115 KB)
// and every GPU that loads the library keeps it until the process exits.
// All calls share it: a call leaves its contents behind, everything a call
// reads is written earlier in the same call on the same stream, and two
// calls that overlap in time on the GPU (different streams, or different
// host threads) race on it.
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "copula.h"
#include "internal.h"

namespace cop {
namespace {

constexpr int kNoallocMaxSubsets = 2048;

// Resident CTAs per SM of a launch (the rule copula_fit uses): by shared
// memory (the 227 KB opt-in limit) and by 2048 threads per SM.
int per_sm_of(int blk, size_t smem) {
  return std::max(1, std::min((int)((kMaxSmem + 2048) / (smem + 1024)), 2048 / blk));
}

// Byte layout of the scratch array.
constexpr size_t kOffCounters = 0;  // 64 int32 job counters
constexpr size_t kOffDss = 256;     // 2 int64 dataset bounds {0, K}
constexpr size_t kOffJobs = 512;    // kNoallocMaxSubsets Job
constexpr size_t kOffVar = kOffJobs + (size_t)kNoallocMaxSubsets * sizeof(Job);
constexpr size_t kOffInfo = kOffVar + (size_t)kNoallocMaxSubsets * sizeof(double);
constexpr size_t kOffIters = kOffInfo + (size_t)kNoallocMaxSubsets * sizeof(double);
constexpr size_t kOffStatus = kOffIters + (size_t)kNoallocMaxSubsets * sizeof(int32_t);
constexpr size_t kScratchBytes = kOffStatus + (size_t)kNoallocMaxSubsets * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Subset offsets and job slots travel in the kernel parameter block, so the
// schedule needs no host-to-device copy.
struct ScheduleArgs {
  int64_t off[kNoallocMaxSubsets + 1];
  int32_t slot[kNoallocMaxSubsets];  // position of subset k in the job array
  int8_t gs_mode[kNoallocMaxSubsets];  // Job::gs_mode of subset k
  int32_t K;
  int32_t family;
};

__global__ void noalloc_schedule_kernel(const __grid_constant__ ScheduleArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  Job* jobs = reinterpret_cast<Job*>(g_noalloc_scratch + kOffJobs);
  if (k < a.K) {
    Job j;
    j.off = a.off[k];
    j.m = (int32_t)(a.off[k + 1] - a.off[k]);
    j.family = a.family;
    j.subset = k;
    j.dataset = 0;
    j.gs_mode = a.gs_mode[k];
    j.pad = 0;
    jobs[a.slot[k]] = j;
  }
  if (k < 64) reinterpret_cast<int32_t*>(g_noalloc_scratch + kOffCounters)[k] = 0;
  if (k == 0) {
    int64_t* dss = reinterpret_cast<int64_t*>(g_noalloc_scratch + kOffDss);
    dss[0] = 0;
    dss[1] = a.K;
  }
}

// Per-device set-up: the device address of the scratch array (host code sees
// only a host-side stand-in for the symbol) and the SM count.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
bool g_tables_ready = false;
StartTables g_start;

int setup_device(int* dev_out, char** scratch, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return COPULA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_tables_ready) {
    build_start_tables(g_start);
    g_tables_ready = true;
  }
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return COPULA_ERR_CUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return COPULA_ERR_CUDA;
    g_sms[dev] = n;
    g_scratch_ptr[dev] = p;
  }
  *dev_out = dev;
  *scratch = static_cast<char*>(g_scratch_ptr[dev]);
  *sms = g_sms[dev];
  return COPULA_SUCCESS;
}

}  // namespace
}  // namespace cop

using namespace cop;

extern "C" int copula_fit_noalloc(int32_t family, int32_t dtype, const void* u, const void* v, int64_t n,
                                  const int64_t* soff, int64_t K, double* theta_out, double* var_out,
                                  int32_t* status_out, double* theta_combined_out, const copula_opts* opts,
                                  void* stream) {
  if (family < 0 || family > 2 || (dtype != COPULA_DTYPE_F32 && dtype != COPULA_DTYPE_F64)) return COPULA_ERR_ARG;
  if (!u || !v || !theta_out || !soff || K < 1 || n < 2) return COPULA_ERR_ARG;
  if (K > kNoallocMaxSubsets) return COPULA_ERR_UNSUPPORTED;
  copula_opts o;
  copula_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_iter <= 0) o.max_iter = 64;
  if (!(o.rtol > 0.0)) o.rtol = o.precision == COPULA_PREC_F64 ? 1e-13 : 1e-6;
  if (o.precision != COPULA_PREC_F64 && o.precision != COPULA_PREC_F32C) return COPULA_ERR_ARG;
  if (o.weight < 0 || o.weight > 2) return COPULA_ERR_ARG;
  if (soff[0] != 0 || soff[K] != n) return COPULA_ERR_ARG;
  const int ks = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  const int rs = o.precision == COPULA_PREC_F32C ? 4 : 8;

  // Buckets by block size (the same rule as copula_fit); every subset's
  // tables and scan arrays must fit in shared memory, since there is no
  // workspace to fall back on.
  static const int kBlocks[3] = {512, 256, 128};
  ScheduleArgs sa;
  int count[3] = {0, 0, 0};
  for (int64_t k = 0; k < K; ++k) {
    const int64_t m = soff[k + 1] - soff[k];
    if (m < 2) return COPULA_ERR_ARG;
    const int blk = block_size_for((int)std::min<int64_t>(m, 1 << 30), o.block);
    const int b = blk == 512 ? 0 : blk == 256 ? 1 : 2;
    if (m > (ks == 4 ? COPULA_MAX_SUBSET : COPULA_MAX_SUBSET_F64) ||
        res_layout((int)m, ks, rs, true, false, blk).total > kMaxSmem)
      return COPULA_ERR_UNSUPPORTED;
    ++count[b];
  }
  int first[3] = {0, count[0], count[0] + count[1]};
  int fill[3] = {first[0], first[1], first[2]};
  size_t smem_b[3] = {0, 0, 0};
  for (int64_t k = 0; k <= K; ++k) sa.off[k] = soff[k];
  for (int64_t k = 0; k < K; ++k) {
    const int m = (int)(soff[k + 1] - soff[k]);
    const int blk = block_size_for(m, o.block);
    const int b = blk == 512 ? 0 : blk == 256 ? 1 : 2;
    sa.slot[k] = fill[b]++;
    // the variance's per-point store in shared memory when the subset's own
    // layout keeps its CTAs per SM (the rule copula_fit applies), else its
    // terms are evaluated again
    const size_t s0 = res_layout(m, ks, rs, true, false, blk).total;
    const size_t s1 = res_layout(m, ks, rs, true, true, blk).total;
    const bool gs_smem = s1 <= kMaxSmem && per_sm_of(blk, s1) >= per_sm_of(blk, s0);
    sa.gs_mode[k] = gs_smem ? 1 : 0;
    smem_b[b] = std::max(smem_b[b], gs_smem ? s1 : s0);
  }
  sa.K = (int32_t)K;
  sa.family = family;

  int dev = 0, sms = 0;
  char* w = nullptr;
  int rc = setup_device(&dev, &w, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  noalloc_schedule_kernel<<<(int)((K + 63 + 255) / 256), 256, 0, st>>>(sa);
  if (cudaGetLastError() != cudaSuccess) return COPULA_ERR_CUDA;

  ResidentArgs a;
  std::memset(&a, 0, sizeof(a));
  a.u = u;
  a.v = v;
  a.mode = MODE_FIT;
  a.theta = theta_out;
  a.var = var_out ? var_out : (double*)(w + kOffVar);
  a.status = status_out ? status_out : (int32_t*)(w + kOffStatus);
  a.info = (double*)(w + kOffInfo);
  a.iters = (int32_t*)(w + kOffIters);
  a.phase_ns = nullptr;
  a.tab_in_smem = 1;
  a.gws = nullptr;
  a.max_iter = o.max_iter;
  a.rtol = o.rtol;
  a.start = g_start;
  for (int b = 0; b < 3; ++b) {
    if (count[b] == 0) continue;
    const int blk = kBlocks[b];
    const size_t smem = smem_b[b];
    a.jobs = (const Job*)(w + kOffJobs) + first[b];
    a.njobs = count[b];
    a.counter = (int32_t*)(w + kOffCounters) + b;
    const int per_sm = per_sm_of(blk, smem);
    const int grid = std::max(1, std::min(count[b], per_sm * sms));
    if (launch_resident(o.precision, ks, blk, grid, smem, a, st) != cudaSuccess) return COPULA_ERR_CUDA;
  }
  if (theta_combined_out) {
    CombineArgs c;
    c.theta = theta_out;
    c.var = a.var;
    c.info = a.info;
    c.status = a.status;
    c.dataset_subset_start = (const int64_t*)(w + kOffDss);
    c.out = theta_combined_out;
    c.B = 1;
    c.weight = o.weight;
    if (launch_combine(c, st) != cudaSuccess) return COPULA_ERR_CUDA;
  }
  return COPULA_SUCCESS;
}
