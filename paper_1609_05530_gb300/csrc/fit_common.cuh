// fit_common.cuh -- device pieces shared by the per-subset (resident) and
// the multi-CTA (streaming) fit kernels: status codes, the safeguarded
// Newton driver, Newton start values, the Gaussian score-cubic solver and
// the per-rank margin transforms.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace cop {

enum : int32_t { ST_OK = 0, ST_BOUNDARY = 1, ST_NOT_CONVERGED = 2, ST_DEGENERATE = 3, ST_CAPPED = 4 };

// |theta| below which the Frank terms come from the independence series.
template <typename Real>
struct FrankSeries;
template <>
struct FrankSeries<float> {
  static constexpr double cut = 1.0;
};
template <>
struct FrankSeries<double> {
  static constexpr double cut = 0.2;
};

// Tests on the bit pattern of a double (integer operations): on a single
// lane's serial path an FP64 compare-and-branch costs ~0.1 us on this GPU,
// an integer one a few ns.
__device__ __forceinline__ bool is_zero64(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_neg64(double x) { return __double_as_longlong(x) < 0 && !is_zero64(x); }
__device__ __forceinline__ bool is_nan64(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffll) > 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool same64(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }

// 1/x in FP64 from the FP32 reciprocal and two Newton corrections (four
// dependent FMAs, within an ulp) instead of an FP64 divide (~0.3 us on one
// lane): for the per-subset constants 1/m and 1/(m+1).
__device__ __forceinline__ double recip64(double x) {
  double r = (double)(1.0f / (float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// ---------------------------------------------------------------------------
// Newton driver (thread 0, FP64): bisection-safeguarded Newton on the score.
// ---------------------------------------------------------------------------
struct Newton {
  double th, lo, hi, dlo, dhi, rtol;
  int it, max_iter, status;
  bool done, probed_lo, probed_hi, lo_natural;

  // dom_lo is either the family's own edge (lo_nat: Gumbel theta = 1, reported
  // as BOUNDARY) or a search cap like dom_hi (reported as CAPPED).  A start
  // value is kept off the domain's ends by 1e-3 of its width, except a root
  // from an earlier search (clamp false), which is interior already.
  __device__ inline void init(double th0, double dom_lo, double dom_hi, double tol, int maxit, bool lo_nat,
                              bool clamp = true) {
    lo_natural = lo_nat;
    dlo = dom_lo;
    dhi = dom_hi;
    lo = dom_lo;
    hi = dom_hi;
    th = clamp ? fmin(fmax(th0, dom_lo + 1e-3 * (dom_hi - dom_lo)), dom_hi - 1e-3 * (dom_hi - dom_lo)) : th0;
    rtol = tol;
    it = 0;
    max_iter = maxit;
    status = ST_OK;
    done = false;
    probed_lo = probed_hi = false;
  }

  // g, h: score and Hessian of Eq. 13 at th.  (NaN, sign and equality tests
  // on bit patterns: this runs on one lane, where each FP64
  // compare-and-branch costs ~0.1 us.)
  __device__ inline void step(double g, double h) {
    ++it;
    if (is_nan64(g) || is_nan64(h)) {  // nothing sensible to do
      status = ST_DEGENERATE;
      done = true;
      return;
    }
    const bool g_neg = is_neg64(g), g_zero = is_zero64(g), g_pos = !g_neg && !g_zero;
    if (!g_pos && th <= dlo) {  // maximiser on the lower edge
      status = lo_natural ? ST_BOUNDARY : ST_CAPPED;
      done = true;
      return;
    }
    if (!g_neg && th >= dhi) {  // maximiser on the upper cap
      status = ST_CAPPED;
      done = true;
      return;
    }
    if (g_pos)
      lo = th;
    else if (g_neg)
      hi = th;
    else {
      done = true;
      return;
    }
    double cand = is_neg64(h) ? th - g / h : __longlong_as_double(0x7ff8000000000000ll);
    // a Newton step within the tolerance is convergence, even when it rounds
    // onto th itself or onto the bracket end th just became (at the root the
    // step is below one ulp); only then may the bracket test below fail
    if (!is_nan64(cand) && fabs(cand - th) <= rtol * fmax(1.0, fabs(th))) {
      if (cand > lo && cand < hi) th = cand;
      done = true;
      return;
    }
    if (!(cand > lo && cand < hi)) {
      if (g_neg && same64(lo, dlo) && !probed_lo) {
        cand = dlo;  // try the edge itself once
        probed_lo = true;
      } else if (g_pos && same64(hi, dhi) && !probed_hi) {
        cand = dhi;
        probed_hi = true;
      } else {
        cand = 0.5 * (lo + hi);
      }
    }
    const double tol = rtol * fmax(1.0, fabs(cand));
    const double stepsz = fabs(cand - th);
    th = cand;
    if (!same64(cand, dlo) && !same64(cand, dhi) && (stepsz <= tol || (hi - lo) <= tol)) {
      done = true;
      return;
    }
    if (it >= max_iter) {
      status = ST_NOT_CONVERGED;
      done = true;
    }
  }
};

// The FP64 path starts its Newton search at the root of an FP32-compensated
// search on the same subset: each FP64 pass costs as much as tens of FP32
// ones on this GPU, and from the FP32 root (~1e-7 relative) two FP64 passes
// reach the FP64 tolerance instead of three to five from the Spearman start.
// The FP32 root is used only when that search ended interior (status OK).
constexpr double kPresolveRtol = 1e-6;

// Start value from the subset's Spearman rho: interpolate the parameter
// whose population rho_S equals it on a tabulated grid.
// (FP32 arithmetic: it only seeds the Newton iteration.)
__device__ inline double start_from_rho(const float* tab, float th0, float dth, float rs) {
  if (!(rs > tab[0])) return th0;
  if (rs >= tab[kStartN - 1]) return th0 + (float)(kStartN - 1) * dth;
  int lo = 0, hi = kStartN - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (tab[mid] <= rs)
      lo = mid;
    else
      hi = mid;
  }
  const float f = (rs - tab[lo]) / (tab[hi] - tab[lo]);
  return (double)(th0 + ((float)lo + f) * dth);
}

// Spearman's rho of a subset from its rank products, S = sum r_u r_v, in
// FP32 (a start value only): 12 S / (m (m^2 - 1)) - 3 (m + 1) / (m - 1).
__device__ inline float spearman_rho(double S, int64_t m) {
  const float mf = (float)m;
  return 12.0f * (float)S / (mf * (mf * mf - 1.0f)) - 3.0f * (mf + 1.0f) / (mf - 1.0f);
}

// ---------------------------------------------------------------------------
// Gaussian: the score of Eq. 13 vanishes where
//   m r^3 - B r^2 + (A - m) r - B = 0,  A = sum(x^2 + y^2), B = sum(x y);
// among its real roots in (-1, 1) the MPL is the one with the largest l.
// ---------------------------------------------------------------------------
__device__ inline double gauss_l(double m, double A, double B, double r) {
  const double om = 1.0 - r * r;
  return -0.5 * m * ::log(om) - (r * r * A - 2.0 * r * B) / (2.0 * om);
}

// Root of the score cubic in the bracket [a, b] whose end a has the sign
// a_neg: bracketed Newton in FP32 from r0 (when inside, else the midpoint)
// to FP32 precision, then two FP64 Newton steps on the FP64 cubic, clamped
// to the bracket, which take the ~1e-7 FP32 root to full FP64 precision.
__device__ inline double gauss_root(double m, double A, double B, double a, double b, double r0, bool a_neg) {
  const float mf = (float)m, Bf = (float)B, Amf = (float)(A - m);
  auto f32 = [&](float r) { return ((mf * r - Bf) * r + Amf) * r - Bf; };
  auto fp32 = [&](float r) { return (3.0f * mf * r - 2.0f * Bf) * r + Amf; };
  float lo = (float)a, hi = (float)b;
  float r = (r0 > a && r0 < b) ? (float)r0 : 0.5f * (lo + hi);
  for (int it = 0; it < 64; ++it) {
    const float fr = f32(r);
    if (fr == 0.0f) break;
    if ((fr < 0.0f) == a_neg)
      lo = r;
    else
      hi = r;
    float c = r - fr / fp32(r);
    if (!(c > lo && c < hi)) c = 0.5f * (lo + hi);
    const bool stop = fabsf(c - r) <= 1e-7f * fmaxf(1.0f, fabsf(c)) || (hi - lo) <= 1e-7f;
    r = c;
    if (stop) break;
  }
  double x = fmin(fmax((double)r, a), b);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double fx = ((m * x - B) * x + (A - m)) * x - B;
    const double dx = (3.0 * m * x - 2.0 * B) * x + (A - m);
    x = fmin(fmax(x - fx / dx, a), b);
  }
  return x;
}

__device__ inline double gaussian_mpl(double m, double A, double B, int& status) {
  auto f = [&](double r) { return ((m * r - B) * r + (A - m)) * r - B; };
  // The score's sign can change only between the cap, the cubic's critical
  // points inside (-cap, cap), and the other cap: up to three brackets,
  // kept in scalars (a run-time indexed array would live in local memory).
  double e1 = kGaussCap, e2 = kGaussCap;  // interior critical points, if any
  int ne = 0;
  const double disc = B * B - 3.0 * m * (A - m);
  if (is_neg64(-disc)) {  // disc > 0
    const double sq = sqrt(disc);
    const double c1 = (B - sq) / (3.0 * m), c2 = (B + sq) / (3.0 * m);
    if (c1 > -kGaussCap && c1 < kGaussCap) e1 = c1, ne = 1;
    if (c2 > -kGaussCap && c2 < kGaussCap && c2 > c1) {
      if (ne == 1)
        e2 = c2, ne = 2;
      else
        e1 = c2, ne = 1;
    }
  }
  const double x0 = -kGaussCap, x1 = ne >= 1 ? e1 : kGaussCap, x2 = ne >= 2 ? e2 : kGaussCap, x3 = kGaussCap;
  const double f0 = f(x0), f1 = ne >= 1 ? f(x1) : 0.0, f2 = ne >= 2 ? f(x2) : 0.0, f3 = f(x3);
  // bracket i is [x_i, x_{i+1}] for i <= ne
  auto bracket = [&](int i, double& a, double& b, double& fa, double& fb) {
    a = i == 0 ? x0 : i == 1 ? x1 : x2;
    fa = i == 0 ? f0 : i == 1 ? f1 : f2;
    b = i == ne ? x3 : i == 0 ? x1 : x2;
    fb = i == ne ? f3 : i == 0 ? f1 : f2;
  };
  auto changes = [](double fa, double fb) {
    return is_zero64(fa) || is_zero64(fb) || is_neg64(fa) != is_neg64(fb);
  };
  int nsign = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i > ne) break;
    double a, b, fa, fb;
    bracket(i, a, b, fa, fb);
    if (changes(fa, fb)) ++nsign;
  }
  // Newton start: the correlation of the normal scores, 2B/A, within O(1/m)
  // of the maximiser
  const float r0 = (float)B / fmaxf((float)A, 1e-30f) * 2.0f;
  double best = 0.0, bestl = -1e300;
  bool found = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i > ne) break;
    double a, b, fa, fb;
    bracket(i, a, b, fa, fb);
    if (!changes(fa, fb)) continue;
    const double r = is_zero64(fa) ? a : is_zero64(fb) ? b : gauss_root(m, A, B, a, b, r0, is_neg64(fa));
    // with several stationary points, the one with the largest likelihood
    const double l = nsign > 1 ? gauss_l(m, A, B, r) : 0.0;
    if (!found || l > bestl) {
      best = r;
      bestl = l;
      found = true;
    }
  }
  status = ST_OK;
  if (!found) {  // no interior root: the likelihood grows towards an edge
    best = gauss_l(m, A, B, -kGaussCap) > gauss_l(m, A, B, kGaussCap) ? -kGaussCap : kGaussCap;
    status = ST_CAPPED;
  } else if (fabs(best) >= kGaussCap) {
    status = ST_CAPPED;
  }
  return best;
}

// Per-subset constants of the closed form at |theta| = at (FP64):
// k0 = log(at (1 - e^-at)), k1 = 1/at + 1/(e^at - 1),
// k2 = -1/at^2 - e^at/(e^at - 1)^2, E = e^-at.
struct FrankConsts {
  double k0, k1, k2, E;
};
__device__ inline FrankConsts frank_consts_f64(double at) {
  const double em1 = ::expm1(at);
  FrankConsts c;
  c.E = ::exp(-at);
  c.k0 = ::log(-at * ::expm1(-at));
  c.k1 = 1.0 / at + 1.0 / em1;
  c.k2 = -1.0 / (at * at) - (em1 + 1.0) / (em1 * em1);
  return c;
}

// The same constants from FP32 arithmetic, for the FP32-compensated path:
// their rounding (~1e-7 relative, k1 and k2 without cancellation for
// |theta| >= 1, where the closed form is used) moves the score by m k1 1e-7,
// i.e. theta by a few 1e-7 relative -- below that path's Newton tolerance
// (1e-6) and its 1e-5 parity bar -- while the serial FP64 exp and expm1 of
// the FP64 version cost microseconds on one lane.
__device__ inline FrankConsts frank_consts_f32(double at) {
  const float af = (float)at;
  const float em1 = expm1f(af);
  const float r = 1.0f / em1;
  FrankConsts c;
  c.E = (double)expf(-af);
  c.k0 = (double)logf(-af * expm1f(-af));
  c.k1 = (double)(1.0f / af + r);
  c.k2 = (double)(-1.0f / (af * af) - r * (1.0f + r));
  return c;
}

// Per-rank margin transforms (rank r+1 of m): the normal score
// Phi^{-1}((r+1)/(m+1)) and Gumbel's log(-log((r+1)/(m+1))), both using the
// exact complement (m-r)/(m+1) in the upper half.
__device__ __forceinline__ float normal_score(int64_t r, int64_t m, float) {
  const float inv = 1.0f / (float)(m + 1);
  return 2 * (r + 1) <= m + 1 ? normcdfinvf((float)(r + 1) * inv) : -normcdfinvf((float)(m - r) * inv);
}
__device__ __forceinline__ double normal_score(int64_t r, int64_t m, double) {
  const double inv = 1.0 / (double)(m + 1);
  return 2 * (r + 1) <= m + 1 ? normcdfinv((double)(r + 1) * inv) : -normcdfinv((double)(m - r) * inv);
}
__device__ __forceinline__ float gumbel_lx(int64_t r, int64_t m, float) {
  const float inv = 1.0f / (float)(m + 1);
  const float x = 2 * (r + 1) <= m + 1 ? -logf((float)(r + 1) * inv) : -log1pf(-(float)(m - r) * inv);
  return logf(x);
}
__device__ __forceinline__ double gumbel_lx(int64_t r, int64_t m, double) {
  const double inv = 1.0 / (double)(m + 1);
  const double x = 2 * (r + 1) <= m + 1 ? -::log((double)(r + 1) * inv) : -::log1p(-(double)(m - r) * inv);
  return ::log(x);
}

// Eq. 15 for dataset b by one full warp: the weighted mean of the subset
// estimates with status OK or BOUNDARY and a finite positive weight (weight
// 1/var, the observed information, or 1).  Lane l takes subsets l, l+32, ...
// in order and a fixed shuffle tree adds the lanes, so the bits do not depend
// on which block runs it.  Loads bypass L1: other blocks of the same launch
// wrote the estimates.
__device__ inline void combine_dataset(const double* theta, const double* var, const double* info,
                                       const int32_t* status, const int64_t* dss, int weight, int b,
                                       double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t b0 = __ldcg(dss + b), b1 = __ldcg(dss + b + 1);
  double num = 0.0, den = 0.0;
  for (int64_t k = b0 + lane; k < b1; k += 32) {
    const int32_t st = __ldcg(status + k);
    if (st != ST_OK && st != ST_BOUNDARY) continue;
    const double w = weight == 0 ? 1.0 / __ldcg(var + k) : weight == 1 ? __ldcg(info + k) : 1.0;
    const double t = __ldcg(theta + k);
    if (!isfinite(w) || !isfinite(t) || !(w > 0.0)) continue;
    num += w * t;
    den += w;
  }
  num = warp_sum_f64(num);
  den = warp_sum_f64(den);
  if (lane == 0) out[b] = den > 0.0 ? num / den : __longlong_as_double(0x7ff8000000000000ll);
}

// Counts one finished subset of dataset b (its estimates already stored by
// the calling lane); returns true, to that lane, if it was the dataset's last.
__device__ inline bool dataset_finished(int32_t* ds_done, const int64_t* dss, int b) {
  __threadfence();
  const int64_t kb = __ldcg(dss + b + 1) - __ldcg(dss + b);
  const bool last = atomicAdd(ds_done + b, 1) == (int)(kb - 1);
  if (last) __threadfence();
  return last;
}

}  // namespace cop
