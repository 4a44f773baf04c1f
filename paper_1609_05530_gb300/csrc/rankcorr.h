// rankcorr.h -- launcher of the per-subset sample rank correlations
// (rankcorr.cu), called by copula_rank_corr.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace cop {

// One CTA per job of `jobs` (an atomic job counter, zeroed before the
// launch); smem: res_layout(m_max, key_bytes, 4, false, false, block).total.
// Writes Kendall's tau and Spearman's rho of each job's subset to
// tau[subset], rho[subset] (NaN for a subset holding NaN).
cudaError_t launch_rankcorr(int key_bytes, int block, int grid, size_t smem, const void* u, const void* v,
                            const Job* jobs, int njobs, int32_t* counter, double* tau, double* rho,
                            cudaStream_t s);

}  // namespace cop
