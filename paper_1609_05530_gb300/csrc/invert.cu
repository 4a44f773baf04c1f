// invert.cu -- the rank-correlation inversion estimators that Section 2.3
// lists beside the maximum pseudo-likelihood: the parameter theta of a
// family whose population Kendall's tau, or Spearman's rho, equals a given
// (sample) value, one warp per value.
//
// Population maps (the values Section 2.5 prints beside each generating
// parameter):
//   Gaussian   tau = (2/pi) asin(rho),  rho_S = (6/pi) asin(rho/2)   (closed-form inverses)
//   Gumbel     tau = 1 - 1/theta                                    (closed-form inverse)
//              rho_S = 12 int_0^1 (1 + A(t))^-2 dt - 3 with the Pickands function
//              A(t) = (t^theta + (1-t)^theta)^(1/theta) of the extreme-value copula
//   Frank      tau = 1 - (4/theta)(1 - D_1(theta)),
//              rho_S = 1 - (12/theta)(D_1(theta) - D_2(theta)),
//              D_k(x) = (k / x^k) int_0^x t^k / (e^t - 1) dt (Debye functions), odd in theta
// The non-closed maps are inverted by a bracketed Newton iteration in FP64:
// each evaluation of the map and its theta-derivative is a Gauss-Legendre
// sum spread over the 32 lanes (Frank: 32 nodes on [0, theta]; Gumbel: a
// 160-node rule on [0, 1/2] graded towards t = 0, where t^theta is not
// smooth near theta = 1, and towards t = 1/2, where A sharpens into a kink
// for large theta; A is symmetric about 1/2).  Below |theta| = 0.5 Frank's
// maps come from their Bernoulli power series, where the closed forms
// cancel.
//
// Statuses: OK; BOUNDARY for Gumbel when the value is at or below the
// family's independence value 0 (theta = 1, its edge); CAPPED beyond a
// search cap (Gaussian |rho| <= 1 - 1e-9, Frank |theta| <= 50, Gumbel
// theta <= 50; theta is the cap); DEGENERATE for a value that is NaN or
// outside [-1, 1] (theta NaN); NOT_CONVERGED if the iteration cap is hit.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "copula.h"
#include "fit_common.cuh"
#include "internal.h"

namespace cop {
namespace {

constexpr int kFrankNodes = 32;
constexpr int kGumbelNodes = 160;
constexpr int kInvertMaxIter = 100;

struct InvertNodes {
  double fx[kFrankNodes], fw[kFrankNodes];  // Gauss-Legendre on [0, 1]
  double gw[kGumbelNodes];                  // weights of the rule on [0, 1/2]
  double gL[kGumbelNodes];                  // log(t / (1 - t)) at its nodes
  double gomt[kGumbelNodes];                // 1 - t at its nodes
};

struct InvertArgs {
  const double* r;
  double* theta;
  int32_t* status;
  int64_t K;
  int32_t family, which;
  InvertNodes nodes;
};

__device__ __forceinline__ double warp_sum_lane0(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return __shfl_sync(0xffffffffu, x, 0);  // lane 0's total, the same bits in every lane
}

// Frank's tau (which = 0) or rho_S (which = 1) at x > 0 and its derivative.
__device__ void frank_map(int which, double x, const InvertNodes& N, double& f, double& df) {
  if (x < 0.5) {
    // tau = 4 sum B_2j x^(2j-1) / ((2j+1)(2j)!), rho_S = 12 sum j B_2j x^(2j-1) / ((2j+1)(j+1)(2j)!)
    const double B[6] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0, -691.0 / 2730.0};
    double s = 0.0, ds = 0.0, fact = 1.0, xp = 1.0;  // xp = x^(2j-2)
    for (int j = 1; j <= 6; ++j) {
      fact *= (2.0 * j - 1.0) * (2.0 * j);
      double c = B[j - 1] / ((2.0 * j + 1.0) * fact);
      c *= which == 0 ? 4.0 : 12.0 * j / (j + 1.0);
      s += c * xp * x;
      ds += c * (2.0 * j - 1.0) * xp;
      xp *= x * x;
    }
    f = s;
    df = ds;
    return;
  }
  const int lane = threadIdx.x & 31;
  const double t = x * N.fx[lane], w = x * N.fw[lane];
  const double g = t / expm1(t);
  const double i1 = warp_sum_lane0(w * g), i2 = warp_sum_lane0(w * g * t);
  const double D1 = i1 / x, D2 = 2.0 * i2 / (x * x), E = 1.0 / expm1(x);
  if (which == 0) {
    f = 1.0 - 4.0 / x * (1.0 - D1);
    df = 4.0 / (x * x) + 4.0 * E / x - 8.0 * D1 / (x * x);
  } else {
    f = 1.0 - 12.0 / x * (D1 - D2);
    df = 12.0 * E / x + 24.0 * D1 / (x * x) - 36.0 * D2 / (x * x);
  }
}

// Gumbel's rho_S at theta >= 1 and its derivative.  With q = (t/(1-t))^theta,
// A = (1 - t)(1 + q)^(1/theta) on [0, 1/2] and
// dA/dtheta = (A / theta^2)(q log q / (1 + q) - log(1 + q)).
__device__ void gumbel_rho_map(double th, const InvertNodes& N, double& f, double& df) {
  const int lane = threadIdx.x & 31;
  double s = 0.0, ds = 0.0;
  const double ith = 1.0 / th;
  for (int i = lane; i < kGumbelNodes; i += 32) {
    const double lq = th * N.gL[i];
    const double q = exp(lq);
    const double l1q = log1p(q);
    const double A = N.gomt[i] * exp(l1q * ith);
    const double dA = A * ith * ith * (q * lq / (1.0 + q) - l1q);
    const double b = 1.0 / (1.0 + A);
    s += N.gw[i] * b * b;
    ds += N.gw[i] * b * b * b * dA;
  }
  s = warp_sum_lane0(s);
  ds = warp_sum_lane0(ds);
  f = 24.0 * s - 3.0;
  df = -48.0 * ds;
}

// The map of (family, which) at theta (Frank: theta > 0).
__device__ __forceinline__ void corr_map(int family, int which, double th, const InvertNodes& N, double& f,
                                         double& df) {
  if (family == COPULA_FRANK)
    frank_map(which, th, N, f, df);
  else
    gumbel_rho_map(th, N, f, df);
}

__global__ void invert_kernel(const __grid_constant__ InvertArgs a) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= a.K) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const double r = a.r[k];
  double th = 0.0;
  int st = ST_OK;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if (!(r >= -1.0 && r <= 1.0)) {
    th = qnan;
    st = ST_DEGENERATE;
  } else if (a.family == COPULA_GAUSSIAN) {
    th = a.which == 0 ? sin(0.5 * M_PI * r) : 2.0 * sin(M_PI * r / 6.0);
    if (fabs(th) > kGaussCap) {
      th = copysign(kGaussCap, th);
      st = ST_CAPPED;
    }
  } else if (a.family == COPULA_GUMBEL && r <= 0.0) {
    th = 1.0;
    st = ST_BOUNDARY;
  } else if (a.family == COPULA_GUMBEL && a.which == 0) {
    th = 1.0 / (1.0 - r);
    if (th > kGumbelCap) {
      th = kGumbelCap;
      st = ST_CAPPED;
    }
  } else if (a.family == COPULA_FRANK && r == 0.0) {
    th = 0.0;
  } else {
    // bracketed Newton on map(theta) = target; Frank on |r| (odd map)
    const bool frank = a.family == COPULA_FRANK;
    const double target = frank ? fabs(r) : r;
    double lo = frank ? 0.0 : 1.0, hi = frank ? kFrankCap : kGumbelCap;
    double f, df;
    corr_map(a.family, a.which, hi, a.nodes, f, df);
    if (target >= f) {
      th = hi;
      st = ST_CAPPED;
    } else {
      // start: the small-dependence slopes (tau ~ theta/9, rho_S ~ theta/6 for
      // Frank; tau ~ 2 rho_S / 3 for Gumbel), kept inside the bracket
      th = frank ? (a.which == 0 ? 9.0 : 6.0) * target / (1.0 - target) : 1.0 / (1.0 - 2.0 * target / 3.0);
      th = fmin(fmax(th, lo + 1e-3), hi - 1e-3);
      st = ST_NOT_CONVERGED;
      for (int it = 0; it < kInvertMaxIter; ++it) {
        corr_map(a.family, a.which, th, a.nodes, f, df);
        if (f == target) {
          st = ST_OK;
          break;
        }
        if (f < target)
          lo = th;
        else
          hi = th;
        double tn = th - (f - target) / df;
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const double step = fabs(tn - th);
        th = tn;
        if (step <= 1e-14 * fmax(1.0, th) || hi - lo <= 1e-15 * fmax(1.0, th)) {
          st = ST_OK;
          break;
        }
      }
      if (frank && r < 0.0) th = -th;
    }
    if (frank && st == ST_CAPPED && r < 0.0) th = -th;
  }
  if (lane == 0) {
    a.theta[k] = th;
    if (a.status) a.status[k] = st;
  }
}

InvertNodes g_nodes;
std::once_flag g_nodes_once;

void build_nodes() {
  double x[kFrankNodes], w[kFrankNodes];
  gauss_legendre01(kFrankNodes, x, w);
  for (int i = 0; i < kFrankNodes; ++i) {
    g_nodes.fx[i] = x[i];
    g_nodes.fw[i] = w[i];
  }
  // [0, 1/2]: 16-point panels on [0, 1e-6], [1e-6, 1e-5], ..., [1e-2, 1e-1],
  // then [0.1, 0.3], [0.3, 0.45], [0.45, 0.49], [0.49, 0.5]
  const double e[] = {0.0, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 0.3, 0.45, 0.49, 0.5};
  double px[16], pw[16];
  gauss_legendre01(16, px, pw);
  int n = 0;
  for (int p = 0; p < 10; ++p)
    for (int i = 0; i < 16; ++i, ++n) {
      const double t = e[p] + (e[p + 1] - e[p]) * px[i];
      g_nodes.gw[n] = (e[p + 1] - e[p]) * pw[i];
      g_nodes.gL[n] = std::log(t) - std::log1p(-t);
      g_nodes.gomt[n] = 1.0 - t;
    }
}

}  // namespace
}  // namespace cop

using namespace cop;

extern "C" int copula_theta_from_rank_corr(int32_t family, int32_t which, const double* r, int64_t K,
                                           double* theta_out, int32_t* status_out, void* stream) {
  if (family < 0 || family > 2 || (which != 0 && which != 1) || K < 0 || (K > 0 && (!r || !theta_out)))
    return COPULA_ERR_ARG;
  if (K == 0) return COPULA_SUCCESS;
  std::call_once(g_nodes_once, build_nodes);
  InvertArgs a;
  a.r = r;
  a.theta = theta_out;
  a.status = status_out;
  a.K = K;
  a.family = family;
  a.which = which;
  a.nodes = g_nodes;
  const int threads = 256;
  const int64_t blocks = (K * 32 + threads - 1) / threads;
  if (blocks > 0x7fffffff) return COPULA_ERR_UNSUPPORTED;
  invert_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? COPULA_SUCCESS : COPULA_ERR_CUDA;
}
