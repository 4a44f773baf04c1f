// simstudy.cu -- the summaries of the paper's simulation study (Sections
// 2.5-2.6) on the GPU: the means over S simulations of the combined and the
// full-data estimates (Eq. 17, 18), the estimated bias and MSE, and the
// relative L1 and L2 distances between the copula densities at the two
// estimates (Eq. 19, 20), whose double integrals over the unit square are
// taken by a product quadrature rule.
//
// Quadrature rule (per axis, on [delta, 1 - delta]): 10-point Gauss-Legendre
// on panels graded geometrically towards both ends, where the densities'
// corner singularities sit -- 20 panels from delta (or from 1e-12 when
// delta = 0) up to 0.02; when delta = 0, for the Gaussian and Frank families,
// 40 more panels from 1e-100 up to 1e-12 (the squared Gaussian density of
// strong dependence still has mass at normal scores beyond -7); then 24
// equal panels up to 1/2.  The upper half mirrors the lower one, its nodes
// held as exact complements 1 - t (every margin transform is taken from the
// smaller of t and 1 - t).  The Gumbel density grows like
// 1/|(1 - u, 1 - v)| near (1, 1), so its squared integrals diverge like
// log(1/delta): Eq. 20 needs delta > 0 for that family, and is reported at a
// stated delta.
//
// Kernels: a node kernel fills the per-node margins and weights into the
// workspace; a tile kernel sums the four integrands over a band of rows of
// the node grid for each parameter pair (FP64, a fixed block tree); a finish
// kernel adds the bands of each pair in order.  The results do not depend on
// the launch configuration beyond that fixed order.
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "copula.h"
#include "families.cuh"
#include "fit_common.cuh"
#include "internal.h"

namespace cop {
namespace {

constexpr int kQ = 10;         // Gauss-Legendre points per panel
constexpr int kGraded = 20;    // geometric panels up to 0.02
constexpr int kTail = 40;      // geometric panels from 1e-100 to 1e-12 (delta = 0, Gaussian / Frank)
constexpr int kEqual = 24;     // equal panels from 0.02 to 1/2
constexpr int kRowsPerTile = 8;
constexpr int kDistThreads = 256;

struct DistNode {
  double u, ubar;  // the coordinate and its exact complement
  double q;        // Gaussian: Phi^{-1}(u); Gumbel: -log u; Frank: unused
  double lq;       // Gumbel: log(-log u)
  double w;        // quadrature weight
};

struct QuadRule {
  double gx[kQ], gw[kQ];  // Gauss-Legendre on [0, 1]
  int family, panels, n;  // panels on [delta, 1/2]; n = 2 panels kQ nodes
  double delta;
};

__host__ __device__ inline int dist_panels(int family, double delta) {
  const int tail = (delta > 0.0 || family == COPULA_GUMBEL) ? 0 : kTail;
  return tail + kGraded + kEqual;
}

// Left edge of panel p on [delta, 1/2] (p = panels gives 1/2).
__device__ double panel_edge(const QuadRule& R, int p) {
  const int tail = R.panels - kGraded - kEqual;
  if (p == 0) return R.delta;
  if (p <= tail) return 1e-100 * pow(1e-12 / 1e-100, (double)p / tail);
  p -= tail;
  const double lo = R.delta > 0.0 ? R.delta : 1e-12;
  if (p <= kGraded) return lo * pow(0.02 / lo, (double)p / kGraded);
  p -= kGraded;
  return 0.02 + 0.48 * (double)p / kEqual;
}

__global__ void dist_nodes_kernel(const QuadRule R, DistNode* __restrict__ nodes) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int half = R.panels * kQ;
  if (k >= half) return;
  const int p = k / kQ, i = k % kQ;
  const double a = panel_edge(R, p), b = panel_edge(R, p + 1);
  const double t = a + (b - a) * R.gx[i];
  const double w = (b - a) * R.gw[i];
  DistNode lo, hi;  // the node t and its mirror 1 - t
  lo.u = t;
  lo.ubar = 1.0 - t;
  hi.u = 1.0 - t;
  hi.ubar = t;
  lo.w = hi.w = w;
  lo.q = hi.q = lo.lq = hi.lq = 0.0;
  if (R.family == COPULA_GAUSSIAN) {
    lo.q = normcdfinv(t);
    hi.q = -lo.q;
  } else if (R.family == COPULA_GUMBEL) {
    lo.q = -log(t);
    hi.q = -log1p(-t);
    lo.lq = log(lo.q);
    hi.lq = log(hi.q);
  }
  nodes[k] = lo;
  nodes[R.n - 1 - k] = hi;
}

// log c(u, v; theta) of the family at two nodes (FP64).
__device__ __forceinline__ double log_density(int family, double th, const DistNode& A, const DistNode& B) {
  if (family == COPULA_GAUSSIAN) {
    const double x = A.q, y = B.q, om = 1.0 - th * th;
    return -0.5 * log(om) - (th * th * (x * x + y * y) - 2.0 * th * x * y) / (2.0 * om);
  }
  if (family == COPULA_FRANK) {
    if (fabs(th) < FrankSeries<double>::cut) {
      double l = 0.0;
      (void)frank_series_terms<double>(th, A.u, B.u, &l);
      return l;
    }
    // c = theta (1 - e^-theta) e^{-theta (u + v)} / D^2 with
    // D = -e^{-theta u} expm1(-theta v) - e^{-theta v} expm1(-theta (1 - v))
    const double a = exp(-th * A.u), b = exp(-th * B.u);
    const double D = -a * expm1(-th * B.u) - b * expm1(-th * B.ubar);
    return log(-th * expm1(-th)) - th * (A.u + B.u) - 2.0 * log(fabs(D));
  }
  // Gumbel, x = -log u, y = -log v, w = x^theta + y^theta, z = w^(1/theta):
  // log c = -z + x + y + (theta - 1)(log x + log y) - 2 log w + log(w)/theta + log(z + theta - 1)
  const double xt = exp(th * A.lq), yt = exp(th * B.lq);
  const double L = log(xt + yt), z = exp(L / th);
  return -z + A.q + B.q + (th - 1.0) * (A.lq + B.lq) - 2.0 * L + L / th + log(z + th - 1.0);
}

// partial[(k * tiles + tile) * 4 + c]: the four integrands over rows
// [tile R, tile R + R) of the node grid for pair k = blockIdx.y.
__global__ void __launch_bounds__(kDistThreads) dist_tile_kernel(int family, int n, const DistNode* __restrict__ nodes,
                                                                 const double* __restrict__ theta_a,
                                                                 const double* __restrict__ theta_b,
                                                                 double* __restrict__ partial) {
  const int tiles = gridDim.x, tile = blockIdx.x, k = blockIdx.y;
  const double ta = theta_a[k], tb = theta_b[k];
  const int r0 = tile * kRowsPerTile, r1 = min(n, r0 + kRowsPerTile);
  const int cells = (r1 - r0) * n;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = threadIdx.x; c < cells; c += kDistThreads) {
    const int i = r0 + c / n, j = c % n;
    const DistNode A = nodes[i], B = nodes[j];
    const double ca = exp(log_density(family, ta, A, B));
    const double cb = exp(log_density(family, tb, A, B));
    const double ww = A.w * B.w, d = ca - cb;
    s[0] += ww * fabs(d);
    s[1] += ww * fabs(ca);
    s[2] += ww * d * d;
    s[3] += ww * ca * ca;
  }
  __shared__ double red[4][kDistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double x = s[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[c][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0.0;
    for (int w = 0; w < kDistThreads / 32; ++w) x += red[threadIdx.x][w];
    partial[((size_t)k * tiles + tile) * 4 + threadIdx.x] = x;
  }
}

// out[4 k + c] = sum over tiles (in order) of the partials of pair k; with
// rel != null also rel[2 k] = out[4k] / out[4k+1] (Eq. 19) and
// rel[2 k + 1] = sqrt(out[4k+2] / out[4k+3]) (Eq. 20).
__global__ void dist_finish_kernel(int K, int tiles, const double* __restrict__ partial, double* __restrict__ out,
                                   double* __restrict__ rel) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = 0; t < tiles; ++t)
    for (int c = 0; c < 4; ++c) s[c] += partial[((size_t)k * tiles + t) * 4 + c];
  if (out)
    for (int c = 0; c < 4; ++c) out[4 * k + c] = s[c];
  if (rel) {
    rel[2 * k] = s[0] / s[1];
    rel[2 * k + 1] = sqrt(s[2] / s[3]);
  }
}

// Eq. 17, 18 and the bias and MSE of Section 2.6 from S per-simulation
// combined and full-data estimates, in simulation order (one thread; S is
// small): summary[0] = mean combined, [1] = mean full, [2] = bias,
// [3] = MSE; the pair (mean full, mean combined) goes to pair[0], pair[1]
// for the distance of Eq. 19-20.
__global__ void sim_means_kernel(int S, const double* __restrict__ comb, const double* __restrict__ full,
                                 double* __restrict__ summary, double* __restrict__ pair) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double sc = 0.0, sf = 0.0, se = 0.0;
  for (int s = 0; s < S; ++s) {
    sc += comb[s];
    sf += full[s];
    const double d = comb[s] - full[s];
    se += d * d;
  }
  const double mc = sc / S, mf = sf / S;
  summary[0] = mc;
  summary[1] = mf;
  summary[2] = mc - mf;
  summary[3] = se / S;
  pair[0] = mf;
  pair[1] = mc;
}

struct DistPlan {
  QuadRule R;
  int tiles;
  size_t off_nodes, off_partial, off_pair, bytes;
};

bool dist_plan(int family, double delta, int64_t K, DistPlan& P) {
  if (family < 0 || family > 2 || !(delta >= 0.0 && delta < 0.02) || K < 1 || K > 65535) return false;
  P.R.family = family;
  P.R.delta = delta;
  P.R.panels = dist_panels(family, delta);
  P.R.n = 2 * P.R.panels * kQ;
  gauss_legendre01(kQ, P.R.gx, P.R.gw);
  P.tiles = (P.R.n + kRowsPerTile - 1) / kRowsPerTile;
  size_t o = 0;
  P.off_nodes = o;
  o += ((size_t)P.R.n * sizeof(DistNode) + 255) & ~size_t(255);
  P.off_partial = o;
  o += ((size_t)K * P.tiles * 4 * sizeof(double) + 255) & ~size_t(255);
  P.off_pair = o;
  o += 256;
  P.bytes = o;
  return true;
}

cudaError_t dist_launch(const DistPlan& P, int64_t K, const double* ta, const double* tb, char* w, double* out,
                        double* rel, cudaStream_t st) {
  DistNode* nodes = (DistNode*)(w + P.off_nodes);
  double* partial = (double*)(w + P.off_partial);
  const int half = P.R.panels * kQ;
  dist_nodes_kernel<<<(half + 127) / 128, 128, 0, st>>>(P.R, nodes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)P.tiles, (unsigned)K);
  dist_tile_kernel<<<grid, kDistThreads, 0, st>>>(P.R.family, P.R.n, nodes, ta, tb, partial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dist_finish_kernel<<<(unsigned)((K + 127) / 128), 128, 0, st>>>((int)K, P.tiles, partial, out, rel);
  return cudaGetLastError();
}

}  // namespace
}  // namespace cop

using namespace cop;

extern "C" {

int copula_density_distance_workspace_size(int32_t family, double delta, int64_t K, size_t* bytes) {
  DistPlan P;
  if (!bytes || !dist_plan(family, delta, K, P)) return COPULA_ERR_ARG;
  *bytes = P.bytes;
  return COPULA_SUCCESS;
}

int copula_density_distance(int32_t family, double delta, int64_t K, const double* theta_a, const double* theta_b,
                            double* integrals_out, double* relative_out, void* workspace, size_t workspace_bytes,
                            void* stream) {
  DistPlan P;
  if (!theta_a || !theta_b || (!integrals_out && !relative_out) || !dist_plan(family, delta, K, P))
    return COPULA_ERR_ARG;
  if (!workspace || workspace_bytes < P.bytes || ((uintptr_t)workspace & 255u) != 0) return COPULA_ERR_WORKSPACE;
  const cudaError_t e =
      dist_launch(P, K, theta_a, theta_b, (char*)workspace, integrals_out, relative_out, (cudaStream_t)stream);
  return e == cudaSuccess ? COPULA_SUCCESS : COPULA_ERR_CUDA;
}

int copula_simulation_summary_workspace_size(int32_t family, double delta, size_t* bytes) {
  return copula_density_distance_workspace_size(family, delta, 1, bytes);
}

int copula_simulation_summary(int32_t family, double delta, int32_t S, const double* theta_combined,
                              const double* theta_full, double* summary_out, void* workspace, size_t workspace_bytes,
                              void* stream) {
  DistPlan P;
  if (S < 1 || !theta_combined || !theta_full || !summary_out || !dist_plan(family, delta, 1, P))
    return COPULA_ERR_ARG;
  if (!workspace || workspace_bytes < P.bytes || ((uintptr_t)workspace & 255u) != 0) return COPULA_ERR_WORKSPACE;
  char* w = (char*)workspace;
  double* pair = (double*)(w + P.off_pair);
  cudaStream_t st = (cudaStream_t)stream;
  sim_means_kernel<<<1, 32, 0, st>>>(S, theta_combined, theta_full, summary_out, pair);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = dist_launch(P, 1, pair, pair + 1, w, summary_out + 6, summary_out + 4, st);
  return e == cudaSuccess ? COPULA_SUCCESS : COPULA_ERR_CUDA;
}

}  // extern "C"
