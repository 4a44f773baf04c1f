// common.cuh -- device helpers shared by the libcopula kernels: fast MUFU
// transcendentals, compensated accumulators, block reductions and scans.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cop {

constexpr double kLog2e = 1.4426950408889634;
constexpr double kLn2 = 0.6931471805599453;
constexpr double kSqrt2Pi = 2.5066282746310002;

// ---------------------------------------------------------------------------
// MUFU instructions (PTX ex2/lg2/rcp .approx): one issue each on the SFU.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-precision elementary functions.  The float versions are single MUFU
// issues (plus one multiply); the double versions call the FP64 library.
template <typename Real>
struct Fn;

template <>
struct Fn<float> {
  static __device__ __forceinline__ float exp(float x) { return ex2_approx(x * 1.44269504088896341f); }
  static __device__ __forceinline__ float log(float x) { return lg2_approx(x) * 0.693147180559945309f; }
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
  // log(1 + x) for x >= 0; absolute error ~1e-7, which is all its users need
  static __device__ __forceinline__ float log1p_pos(float x) { return log(1.0f + x); }
};

template <>
struct Fn<double> {
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double log1p_pos(double x) { return ::log1p(x); }
};

// ---------------------------------------------------------------------------
// Accumulators.  Acc<float> is a compensated FP32 sum (Knuth TwoSum per add);
// Acc<double> a plain FP64 sum.  value() returns FP64 either way.
// ---------------------------------------------------------------------------
template <typename Real>
struct Acc;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float t, e;
    two_sum(s, x, t, e);
    s = t;
    c += e;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  __device__ __forceinline__ float value_real() const { return s + c; }
  // butterfly reduction across the warp; every lane ends with the same value
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      float c2 = __shfl_xor_sync(0xffffffffu, c, o);
      float t, e;
      two_sum(s, s2, t, e);
      s = t;
      c = (c + c2) + e;
    }
  }
};

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ double value_real() const { return s; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
};

__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ long long warp_sum_i64(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// (s, c) + (s2, c2) for compensated FP32 pairs.
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
  float t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = (c + c2) + e;
}

// Block reduction of NV accumulators.  Warp stage in the accumulator's own
// arithmetic; cross-warp stage by warp 0 in a fixed tree -- compensated FP32
// pairs for Acc<float> (no FP64 instruction until the final value), FP64 for
// Acc<double>.  The order depends only on BLOCK, so results are reproducible.
// red: shared scratch of at least NV * 64 + NV doubles.  Every thread
// receives the totals in out[].
template <int BLOCK, typename Real, int NV>
__device__ __forceinline__ void block_reduce(Acc<Real> (&a)[NV], double* red, double (&out)[NV]) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) a[v].warp_reduce();
  if constexpr (sizeof(Real) == 4) {
    float* r2 = reinterpret_cast<float*>(red);
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        r2[(v * 32 + warp) * 2] = a[v].s;
        r2[(v * 32 + warp) * 2 + 1] = a[v].c;
      }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Acc<float> x;
        if (lane < NW) {
          x.s = r2[(v * 32 + lane) * 2];
          x.c = r2[(v * 32 + lane) * 2 + 1];
        }
        x.warp_reduce();
        if (lane == 0) red[NV * 32 + v] = x.value();
      }
    }
  } else {
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) red[v * 32 + warp] = a[v].value();
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double x = lane < NW ? red[v * 32 + lane] : 0.0;
        x = warp_sum_f64(x);
        if (lane == 0) red[NV * 32 + v] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = red[NV * 32 + v];
  __syncthreads();
}

template <int BLOCK>
__device__ __forceinline__ long long block_sum_i64(long long x, double* red_as_scratch) {
  constexpr int NW = BLOCK / 32;
  long long* red = reinterpret_cast<long long*>(red_as_scratch);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum_i64(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long y = lane < NW ? red[lane] : 0;
    y = warp_sum_i64(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  long long r = red[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// A per-element factor of 1 (no factor).
struct NoScale {
  __device__ float operator()(int) const { return 1.0f; }
};

// Exclusive suffix over the threads of the block, for two per-thread totals
// at once: on return a and b hold the sums of the totals of the threads after
// this one (thread order).  FP32: compensated pairs throughout; FP64: plain
// sums.  red: >= 128 doubles.  Contains __syncthreads.
template <int BLOCK>
__device__ void block_excl_suffix2(Acc<float>& a, Acc<float>& b, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  // inclusive suffix over lanes >= lane
  float xs = a.s, xc = a.c, ys = b.s, yc = b.c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float p = __shfl_down_sync(0xffffffffu, xs, o), q = __shfl_down_sync(0xffffffffu, xc, o);
    const float r = __shfl_down_sync(0xffffffffu, ys, o), t = __shfl_down_sync(0xffffffffu, yc, o);
    if (lane + o < 32) {
      pair_add(xs, xc, p, q);
      pair_add(ys, yc, r, t);
    }
  }
  float* r2 = reinterpret_cast<float*>(red);  // a: [0, 64) totals, [64, 128) exclusive; b: +128
  if (lane == 0) {
    r2[2 * warp] = xs;
    r2[2 * warp + 1] = xc;
    r2[128 + 2 * warp] = ys;
    r2[128 + 2 * warp + 1] = yc;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float* q = r2 + 128 * k;
      const float ws = lane < NW ? q[2 * lane] : 0.0f, wc = lane < NW ? q[2 * lane + 1] : 0.0f;
      float ss = ws, sc = wc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float p = __shfl_down_sync(0xffffffffu, ss, o), t = __shfl_down_sync(0xffffffffu, sc, o);
        if (lane + o < 32) pair_add(ss, sc, p, t);
      }
      // exclusive: the warps after this one
      const float es = __shfl_down_sync(0xffffffffu, ss, 1), ec = __shfl_down_sync(0xffffffffu, sc, 1);
      if (lane < NW) {
        q[64 + 2 * lane] = lane + 1 < NW ? es : 0.0f;
        q[64 + 2 * lane + 1] = lane + 1 < NW ? ec : 0.0f;
      }
    }
  }
  __syncthreads();
  // (lanes after this one in the warp) + (warps after this one)
  const float nxs = __shfl_down_sync(0xffffffffu, xs, 1), nxc = __shfl_down_sync(0xffffffffu, xc, 1);
  const float nys = __shfl_down_sync(0xffffffffu, ys, 1), nyc = __shfl_down_sync(0xffffffffu, yc, 1);
  a.s = lane < 31 ? nxs : 0.0f;
  a.c = lane < 31 ? nxc : 0.0f;
  b.s = lane < 31 ? nys : 0.0f;
  b.c = lane < 31 ? nyc : 0.0f;
  pair_add(a.s, a.c, r2[64 + 2 * warp], r2[64 + 2 * warp + 1]);
  pair_add(b.s, b.c, r2[192 + 2 * warp], r2[192 + 2 * warp + 1]);
  __syncthreads();
}

template <int BLOCK>
__device__ void block_excl_suffix2(Acc<double>& a, Acc<double>& b, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  const double tx = a.s, ty = b.s;
  double ix = tx, iy = ty;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double p = __shfl_down_sync(0xffffffffu, ix, o), q = __shfl_down_sync(0xffffffffu, iy, o);
    if (lane + o < 32) {
      ix += p;
      iy += q;
    }
  }
  if (lane == 0) {
    red[warp] = ix;
    red[64 + warp] = iy;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      double* q = red + 64 * k;
      const double w = lane < NW ? q[lane] : 0.0;
      double s = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double p = __shfl_down_sync(0xffffffffu, s, o);
        if (lane + o < 32) s += p;
      }
      if (lane < NW) q[32 + lane] = s - w;
    }
  }
  __syncthreads();
  a.s = (ix - tx) + red[32 + warp];
  b.s = (iy - ty) + red[96 + warp];
  __syncthreads();
}

// Elements per thread of a block-wide pass over m elements in which each
// thread takes a run of consecutive elements: odd, so that the strided
// accesses of a warp fall in distinct shared-memory banks.
template <int BLOCK>
__device__ __forceinline__ int run_length(int m) {
  return ((m + BLOCK - 1) / BLOCK) | 1;
}

// Both arrays' in-place suffix sums at once (x[i] <- sum_{j >= i} x[j], the
// same for y), one set of barriers for the two: the sandwich variance needs
// both scans of Section 2.3 back to back.  Each thread takes a run of
// consecutive elements.  FP32 compensated.  red: >= 128 doubles.
template <int BLOCK, typename Real>
__device__ void block_suffix_sum2(Real* x, Real* y, int m, double* red) {
  const int C = run_length<BLOCK>(m);
  const int beg = min(m, (int)threadIdx.x * C), end = min(m, beg + C);
  Acc<Real> rx, ry;
  for (int i = beg; i < end; ++i) {
    rx.add(x[i]);
    ry.add(y[i]);
  }
  block_excl_suffix2<BLOCK>(rx, ry, red);
  for (int i = end - 1; i >= beg; --i) {
    rx.add(x[i]);
    x[i] = rx.value_real();
    ry.add(y[i]);
    y[i] = ry.value_real();
  }
}

}  // namespace cop
