// rankcorr.cu -- sample rank correlations of every subset: Kendall's tau and
// Spearman's rho of the subset's ranks (Eq. 12, taken within the subset as
// Section 2.4 has it).  Section 2.3 lists the inversion of Kendall's tau and
// of Spearman's rho among the estimators of a copula parameter; these are
// their sample statistics, one CTA per subset on the shared-memory path.
//
// Per subset (rows [off, off+m), m <= the shared-memory sort's limit):
//   1. the ranks of u and of v by the same stable radix sort as the fit
//      kernel, giving the pairing permutation pi (pi[p] = v-rank of the point
//      of u-rank p+1) and S = sum (p+1) pi[p] exactly;
//   2. Spearman's rho = 1 - 6 D / (m (m^2 - 1)), D = sum (p+1 - pi[p])^2 =
//      m(m+1)(2m+1)/3 - 2 S, an exact integer;
//   3. Kendall's tau = (P - 2 I) / P, P = m(m-1)/2, where I, the discordant
//      pairs, are the inversions of pi: a bottom-up merge sort of pi in
//      shared memory, every element of a pass placing itself by a binary
//      search in its partner run, and each element of a left run adding the
//      partner elements below it to I.
// Both statistics are integer work up to one final FP64 division, done in
// the same order as the plain definitions, so they are exact.
#include "block_sort.cuh"
#include "common.cuh"
#include "internal.h"
#include "rankcorr.h"

namespace cop {

template <typename KeyT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) rankcorr_kernel(const void* __restrict__ u, const void* __restrict__ v,
                                                            const Job* __restrict__ jobs, int njobs,
                                                            int32_t* counter, double* __restrict__ tau_out,
                                                            double* __restrict__ rho_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t scan[40];
  __shared__ double red[4 * 32 + 8];
  __shared__ int s_job;
  using Val = typename KeyOf<KeyT>::Val;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(counter, 1);
    __syncthreads();
    const int j = s_job;
    __syncthreads();
    if (j >= njobs) return;
    const Job job = jobs[j];
    const int m = job.m;
    const ResLayout L = res_layout(m, (int)sizeof(KeyT), 4, false, false, BLOCK);
    KeyT* keys = reinterpret_cast<KeyT*>(smem);
    uint16_t* ib0 = reinterpret_cast<uint16_t*>(smem + (size_t)m * sizeof(KeyT));
    uint16_t* ib1 = ib0 + m;
    uint16_t* pi = reinterpret_cast<uint16_t*>(smem + L.pi_off);
    SortCnt* cnt = reinterpret_cast<SortCnt*>(smem + L.cnt_off);

    // Eq. 12 for u, then v
    const Val* xu = reinterpret_cast<const Val*>(u) + job.off;
    const Val* xv = reinterpret_cast<const Val*>(v) + job.off;
    KeyRange range;
    bool nan = load_keys<BLOCK, KeyT>(xu, m, keys, scan, &range);
    if (!nan) {
      const uint16_t* perm = block_rank_perm<BLOCK, KeyT>(keys, m, ib0, ib1, cnt, scan, range);
      for (int p = threadIdx.x; p < m; p += BLOCK) pi[p] = perm[p];  // perm_u
      __syncthreads();
      nan = load_keys<BLOCK, KeyT>(xv, m, keys, scan, &range);
    }
    if (nan) {
      if (threadIdx.x == 0) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        tau_out[job.subset] = qnan;
        rho_out[job.subset] = qnan;
      }
      __syncthreads();
      continue;
    }
    const uint16_t* permv = block_rank_perm<BLOCK, KeyT>(keys, m, ib0, ib1, cnt, scan, range);
    uint16_t* rv = (permv == ib0) ? ib1 : ib0;
    for (int pos = threadIdx.x; pos < m; pos += BLOCK) rv[permv[pos]] = (uint16_t)(pos + 1);
    __syncthreads();
    long long Ssum = 0;
    for (int p = threadIdx.x; p < m; p += BLOCK) {
      const uint16_t r = rv[pi[p]];
      pi[p] = r;
      Ssum += (long long)(p + 1) * (long long)r;
    }
    __syncthreads();
    Ssum = block_sum_i64<BLOCK>(Ssum, red);

    // inversions of pi by a bottom-up merge sort in the (now free) sort
    // buffers: runs of 2^lg, each element placed by a binary search in its
    // partner run
    uint16_t* A = reinterpret_cast<uint16_t*>(smem);
    uint16_t* B = A + m;
    for (int p = threadIdx.x; p < m; p += BLOCK) A[p] = pi[p];
    __syncthreads();
    long long inv = 0;
    for (int lg = 0; (1 << lg) < m; ++lg) {
      const int len = 1 << lg;
      for (int i = threadIdx.x; i < m; i += BLOCK) {
        const int r = i >> lg;
        const int rs = r << lg;
        const bool left = (r & 1) == 0;
        const int ps = left ? rs + len : rs - len;  // partner run start
        const int pl = left ? max(0, min(len, m - ps)) : len;
        const int x = A[i];
        int lo = 0, hi = pl;  // partner elements below x (values are distinct)
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((int)A[ps + mid] < x)
            lo = mid + 1;
          else
            hi = mid;
        }
        B[(left ? rs : ps) + (i - rs) + lo] = (uint16_t)x;
        if (left) inv += lo;
      }
      __syncthreads();
      uint16_t* t = A;
      A = B;
      B = t;
    }
    inv = block_sum_i64<BLOCK>(inv, red);
    if (threadIdx.x == 0) {
      const long long mm = m;
      const long long P = mm * (mm - 1) / 2;
      const double md = (double)m;
      tau_out[job.subset] = (double)(P - 2 * inv) / (0.5 * md * (double)(m - 1));
      const long long D = mm * (mm + 1) * (2 * mm + 1) / 3 - 2 * Ssum;
      rho_out[job.subset] = 1.0 - 6.0 * (double)D / (md * (md * md - 1.0));
    }
    __syncthreads();
  }
}

template <typename KeyT, int BLOCK>
static cudaError_t launch_rankcorr_t(int grid, size_t smem, const void* u, const void* v, const Job* jobs,
                                     int njobs, int32_t* counter, double* tau, double* rho, cudaStream_t s) {
  static std::atomic<int> granted[64] = {};
  auto k = rankcorr_kernel<KeyT, BLOCK>;
  cudaError_t e = ensure_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<grid, BLOCK, smem, s>>>(u, v, jobs, njobs, counter, tau, rho);
  return cudaGetLastError();
}

template <typename KeyT>
static cudaError_t launch_rankcorr_k(int block, int grid, size_t smem, const void* u, const void* v,
                                     const Job* jobs, int njobs, int32_t* counter, double* tau, double* rho,
                                     cudaStream_t s) {
  switch (block) {
    case 128: return launch_rankcorr_t<KeyT, 128>(grid, smem, u, v, jobs, njobs, counter, tau, rho, s);
    case 256: return launch_rankcorr_t<KeyT, 256>(grid, smem, u, v, jobs, njobs, counter, tau, rho, s);
    case 512: return launch_rankcorr_t<KeyT, 512>(grid, smem, u, v, jobs, njobs, counter, tau, rho, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rankcorr(int key_bytes, int block, int grid, size_t smem, const void* u, const void* v,
                            const Job* jobs, int njobs, int32_t* counter, double* tau, double* rho,
                            cudaStream_t s) {
  return key_bytes == 4 ? launch_rankcorr_k<uint32_t>(block, grid, smem, u, v, jobs, njobs, counter, tau, rho, s)
                        : launch_rankcorr_k<uint64_t>(block, grid, smem, u, v, jobs, njobs, counter, tau, rho, s);
}

}  // namespace cop
