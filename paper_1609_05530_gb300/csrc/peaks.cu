// peaks.cu -- issue-rate probes of the GPU units the fit kernels lean on:
// the MUFU transcendental unit (ex2, lg2, rcp approximations), the FP32 FMA
// pipe and the FP64 FMA pipe.  Their measured rates are the denominators of
// the kernels' compute rooflines (a likelihood pass costs a fixed number of
// transcendentals per pair; the FP64 path is bound by FP64 arithmetic).
//
// Every probe thread runs kChains independent dependency chains of one
// instruction, so the unit, not the latency of one chain, sets the time.
// The chains stay in a bounded range (no overflow, no denormals), and every
// thread stores its result so that nothing is optimised away.
#include <cstdint>
#include <cuda_runtime.h>

#include "copula.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

enum Unit : int { U_EX2 = 0, U_LG2 = 1, U_RCP = 2, U_FFMA = 3, U_DFMA = 4, U_COUNT = 5 };

// Iterations per thread of each probe: about a millisecond on a 152-SM GPU
// at the expected unit rate.
__host__ __device__ constexpr int probe_iters(int unit) { return unit == U_DFMA ? 256 : unit == U_FFMA ? 16384 : 4096; }

template <int UNIT>
__global__ void __launch_bounds__(kThreads) unit_probe(float* sink_f, double* sink_d, float seed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int iters = probe_iters(UNIT);
  if constexpr (UNIT == U_DFMA) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * c + 1e-9 * tid + (double)seed;
    const double a = 0.999, b = 0.001;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink_d[tid] = s;
  } else {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (UNIT == U_EX2 ? 0.0f : 1.0f) + 0.01f * c + 1e-7f * (tid & 1023) + seed;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        float y;
        if constexpr (UNIT == U_EX2) {  // [0, 1) -> [1, 2) -> [0, 1)
          asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
          x[c] = y - 1.0f;
        } else if constexpr (UNIT == U_LG2) {  // [1, 2) -> [0, 1) -> [1, 2)
          asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
          x[c] = y + 1.0f;
        } else if constexpr (UNIT == U_RCP) {  // [1, 2) -> (0.5, 1] -> (1, 1.5]
          asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
          x[c] = y + 0.5f;
        } else {  // FP32 FMA, converging to 1
          x[c] = fmaf(x[c], 0.999f, 0.001f);
        }
      }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink_f[tid] = s;
  }
}

template <int UNIT>
cudaError_t launch_probe(int blocks, float* sf, double* sd, cudaStream_t st) {
  unit_probe<UNIT><<<blocks, kThreads, 0, st>>>(sf, sd, 0.0f);
  return cudaGetLastError();
}

cudaError_t launch_unit(int unit, int blocks, float* sf, double* sd, cudaStream_t st) {
  switch (unit) {
    case U_EX2: return launch_probe<U_EX2>(blocks, sf, sd, st);
    case U_LG2: return launch_probe<U_LG2>(blocks, sf, sd, st);
    case U_RCP: return launch_probe<U_RCP>(blocks, sf, sd, st);
    case U_FFMA: return launch_probe<U_FFMA>(blocks, sf, sd, st);
    default: return launch_probe<U_DFMA>(blocks, sf, sd, st);
  }
}

}  // namespace

extern "C" int copula_measure_unit_rates(double* rates_out, int32_t count, void* stream) {
  if (!rates_out || count < 1) return COPULA_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return COPULA_ERR_CUDA;
  const int blocks = sms * kBlocksPerSm;
  const size_t nthr = (size_t)blocks * kThreads;
  cudaStream_t st = (cudaStream_t)stream;
  float* sf = nullptr;
  double* sd = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = COPULA_SUCCESS;
  if (cudaMalloc(&sf, nthr * sizeof(float)) != cudaSuccess || cudaMalloc(&sd, nthr * sizeof(double)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = COPULA_ERR_CUDA;
  }
  const int n = count < U_COUNT ? count : U_COUNT;
  for (int u = 0; u < n && rc == COPULA_SUCCESS; ++u) {
    // one warm-up launch, then the fastest of three timed ones
    float best = 0.0f;
    for (int rep = 0; rep < 4 && rc == COPULA_SUCCESS; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess || launch_unit(u, blocks, sf, sd, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = COPULA_ERR_CUDA;
        break;
      }
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = COPULA_ERR_CUDA;
      if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (rc == COPULA_SUCCESS)
      rates_out[u] = (double)nthr * (double)kChains * (double)probe_iters(u) / (1e-3 * (double)best);
  }
  for (int u = n; u < count; ++u) rates_out[u] = 0.0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sf) cudaFree(sf);
  if (sd) cudaFree(sd);
  return rc;
}
