// families.cuh -- per-point log-density terms of the three one-parameter
// copulas of Section 2.2 and their theta / margin derivatives, in the form the
// kernels evaluate them (Real = float for the FP32-compensated path, double
// for the FP64 path).
//
// For the pseudo-likelihood of Eq. 13 each point contributes log c(u, v; theta);
// the Newton driver needs d/dtheta and d2/dtheta2 of it, and the sandwich
// variance (Genest, Ghoudi & Rivest 1995, cited in Section 2.3) also needs the
// mixed partials d2/dtheta du and d2/dtheta dv.
#pragma once

#include "common.cuh"
#include "frank_series.h"

namespace cop {

template <typename Real>
struct Terms {
  Real g;   // d log c / d theta
  Real h;   // d2 log c / d theta2
  Real gu;  // d2 log c / d theta du
  Real gv;  // d2 log c / d theta dv
};

// ---------------------------------------------------------------------------
// Gaussian copula (Eq. 7-8) in the normal scores x = Phi^-1(u), y = Phi^-1(v):
//   log c = -1/2 log(1 - r^2) - (r^2 (x^2 + y^2) - 2 r x y) / (2 (1 - r^2)).
// Its MPL depends on the data only through A = sum(x^2 + y^2), B = sum(x y);
// the per-point terms are needed only for the variance.
// ---------------------------------------------------------------------------
// The mixed partials are d2 log c / dtheta dx times dx/du, and dx/du depends
// on the point's rank in u alone (likewise for v).  The variance therefore
// takes the partials without that margin factor and applies it per rank
// (a rank's factor serves its u-side and its v-side entry alike) instead of
// evaluating it twice per point: gaussian_terms leaves it out,
// gaussian_margin gives it.
template <typename Real>
__device__ __forceinline__ Terms<Real> gaussian_terms(Real r, Real x, Real y) {
  const Real S = x * x + y * y, P = x * y, r2 = r * r;
  const Real om = Real(1) - r2;
  const Real iom = Real(1) / om, iom2 = iom * iom;
  Terms<Real> t;
  t.g = r * iom - (r * S - P * (Real(1) + r2)) * iom2;
  t.h = (Real(1) + r2) * iom2 - (S * (Real(1) + Real(3) * r2) - Real(2) * P * r * (Real(3) + r2)) * iom2 * iom;
  t.gu = -(Real(2) * r * x - y * (Real(1) + r2)) * iom2;  // times dx/du
  t.gv = -(Real(2) * r * y - x * (Real(1) + r2)) * iom2;  // times dy/dv
  return t;
}

// dx/du = 1/phi(x) = sqrt(2 pi) exp(x^2 / 2) at the normal score x of a rank.
template <typename Real>
__device__ __forceinline__ Real gaussian_margin(Real x) {
  return Real(kSqrt2Pi) * Fn<Real>::exp(Real(0.5) * x * x);
}

// ---------------------------------------------------------------------------
// Frank copula (Eq. 10), theta > 0.  Twice differentiating C gives
//   c = theta (1 - E) e^{-theta (u + v)} / D^2,  E = e^{-theta},
//   D = a + b - a b - E,  a = e^{-theta u},  b = e^{-theta v}.
// D is formed as a (1 - b) + b (1 - e^{-theta (1 - v)}): two non-negative
// terms, no cancellation.  Negative theta is handled by the caller through
// c(u, v; -theta) = c(u, 1 - v; theta).
//
// FrankPass returns the theta-dependent, data-dependent parts only:
//   g = k1 - (u+v) - 2 D'/D, h = k2 - 2 (D''/D - (D'/D)^2),
//   l = k0 - theta (u+v) - 2 log D,
// with k0 = log(theta (1 - E)), k1 = 1/theta + 1/(e^theta - 1),
// k2 = -1/theta^2 - e^theta / (e^theta - 1)^2 added per subset.
// ---------------------------------------------------------------------------
template <typename Real>
struct FrankPoint {
  Real D, D1, D2, ab;
};

template <typename Real>
__device__ __forceinline__ FrankPoint<Real> frank_point(Real u, Real v, Real a, Real b, Real bc, Real E) {
  // bc = e^{-theta (1 - v)}
  FrankPoint<Real> f;
  f.ab = a * b;
  f.D = a * (Real(1) - b) + b * (Real(1) - bc);
  const Real s = u + v;
  f.D1 = E - u * a - v * b + s * f.ab;
  f.D2 = u * u * a + v * v * b - s * s * f.ab - E;
  return f;
}

// Variance terms (theta > 0) given the pass quantities.  dl/du =
// -theta + 2 theta a (1 - b) / D; differentiating in theta:
//   l_tu = -1 + 2 (Fu + theta dFu) / D - 2 theta Fu D' / D^2,
//   Fu = a (1 - b), dFu = -u Fu + v a b, and symmetrically for v.
template <typename Real>
__device__ __forceinline__ Terms<Real> frank_terms(Real theta, Real k1, Real k2, Real u, Real v, Real a,
                                                   Real b, const FrankPoint<Real>& f) {
  const Real iD = Real(1) / f.D;
  const Real q1 = f.D1 * iD;
  Terms<Real> t;
  t.g = k1 - (u + v) - Real(2) * q1;
  t.h = k2 - Real(2) * (f.D2 * iD - q1 * q1);
  const Real Fu = a * (Real(1) - b), Fv = b * (Real(1) - a);
  const Real dFu = -u * Fu + v * f.ab, dFv = -v * Fv + u * f.ab;
  t.gu = Real(-1) + Real(2) * (Fu + theta * dFu) * iD - Real(2) * theta * Fu * q1 * iD;
  t.gv = Real(-1) + Real(2) * (Fv + theta * dFv) * iD - Real(2) * theta * Fv * q1 * iD;
  return t;
}

// Frank near independence (|theta| small): log c = sum_{k=1..10} c_k theta^k,
// c_k = R_k(P, Q) for even k and s R_k(P, Q) for odd k, with P = u(1-u),
// Q = v(1-v), s = (1-2u)(1-2v) (coefficients in frank_series.h; the series
// converges for |theta| < 2 pi and holds for either sign of theta).  Using it
// below a cut avoids the 2/theta cancellation of the closed form.
template <typename Real>
__device__ __forceinline__ Terms<Real> frank_series_terms(Real t, Real u, Real v, Real* l_out) {
  const Real su = Real(1) - Real(2) * u, sv = Real(1) - Real(2) * v;
  const Real P = u * (Real(1) - u), Q = v * (Real(1) - v), s = su * sv;
  Real Pp[6], Qp[6];
  Pp[0] = Real(1);
  Qp[0] = Real(1);
#pragma unroll
  for (int i = 1; i < 6; ++i) {
    Pp[i] = Pp[i - 1] * P;
    Qp[i] = Qp[i - 1] * Q;
  }
  Real R[kFrankSeriesTerms], RP[kFrankSeriesTerms], RQ[kFrankSeriesTerms];
  frank_series_poly<Real>(Pp, Qp, R, RP, RQ);
  const Real fu = Real(1) - Real(4) * P, fv = Real(1) - Real(4) * Q;  // (1-2u)^2, (1-2v)^2
  Real l = 0, g = 0, h = 0, gu = 0, gv = 0;
  Real tk2 = Real(0);      // theta^{k-2}, only used for k >= 2
  Real tk1 = Real(1);      // theta^{k-1}
#pragma unroll
  for (int k = 1; k <= kFrankSeriesTerms; ++k) {
    Real c, cu, cv;
    if (k & 1) {
      c = s * R[k - 1];
      cu = sv * (Real(-2) * R[k - 1] + fu * RP[k - 1]);
      cv = su * (Real(-2) * R[k - 1] + fv * RQ[k - 1]);
    } else {
      c = R[k - 1];
      cu = su * RP[k - 1];
      cv = sv * RQ[k - 1];
    }
    const Real kk = (Real)k;
    l += c * tk1 * t;
    g += kk * c * tk1;
    if (k >= 2) h += kk * (kk - Real(1)) * c * tk2;
    gu += kk * cu * tk1;
    gv += kk * cv * tk1;
    tk2 = tk1;
    tk1 *= t;
  }
  if (l_out) *l_out = l;
  Terms<Real> r;
  r.g = g;
  r.h = h;
  r.gu = gu;
  r.gv = gv;
  return r;
}

// ---------------------------------------------------------------------------
// Gumbel copula (Eq. 11) in lx = log(-log u), ly = log(-log v):
//   w = x^theta + y^theta, L = log w, z = w^{1/theta},
//   log c = -z + x + y + (theta-1)(lx+ly) - 2L + L/theta + log(z + theta - 1).
// Evaluated with lmax = max(lx, ly), d = |lx - ly|, r = e^{-theta d},
// s = r / (1 + r):  L = theta lmax + log1p(r), L' = lmax - d s,
// L'' = d^2 s (1 - s), (log z)' = -(theta d s + log1p r) / theta^2,
// (log z)'' = L''/theta - 2 (log z)'/theta, z = e^{lmax} (1 + r)^{1/theta};
// nothing overflows for any theta >= 1.
// ---------------------------------------------------------------------------
template <typename Real>
struct GumbelPoint {
  Real g, h;           // d/dtheta, d2/dtheta2 of log c
  Real z, iQ, lz1, s;  // kept for the variance terms (iQ = 1/Q)
  Real l;              // log c (only when asked)
};

template <typename Real, bool WANT_L>
__device__ __forceinline__ GumbelPoint<Real> gumbel_point(Real th, Real ith, Real lx, Real ly) {
  const Real lmax = lx > ly ? lx : ly;
  const Real d = lx > ly ? lx - ly : ly - lx;
  const Real r = Fn<Real>::exp(-th * d);
  const Real opr = Real(1) + r;
  const Real s = r * Fn<Real>::rcp(opr);
  const Real l1p = Fn<Real>::log1p_pos(r);
  const Real L1 = lmax - d * s;
  const Real L2 = d * d * s * (Real(1) - s);
  const Real lz1 = -(th * d * s + l1p) * ith * ith;
  const Real lz2 = L2 * ith - Real(2) * lz1 * ith;
  const Real z = Fn<Real>::exp(lmax + l1p * ith);
  const Real z1 = z * lz1, z2 = z * (lz1 * lz1 + lz2);
  const Real Q = z + th - Real(1);
  const Real iQ = Fn<Real>::rcp(Q);
  const Real w1 = (z1 + Real(1)) * iQ;
  GumbelPoint<Real> p;
  p.g = -z1 + (lx + ly) - Real(2) * L1 + lz1 + w1;
  p.h = -z2 - Real(2) * L2 + lz2 + z2 * iQ - w1 * w1;
  p.z = z;
  p.iQ = iQ;
  p.lz1 = lz1;
  p.s = s;
  if (WANT_L) {
    const Real L = th * lmax + l1p;
    p.l = -z + Fn<Real>::exp(lx) + Fn<Real>::exp(ly) + (th - Real(1)) * (lx + ly) - Real(2) * L +
          L * ith + Fn<Real>::log(Q);
  } else {
    p.l = Real(0);
  }
  return p;
}

// Mixed partials for the variance.  With qx = x^theta / w, qy = 1 - qx:
//   d l_t / dx = (1/x) [ -Z1 + 1 - 2 qx (1 + theta qy (lx - ly)) + qx qy (lx - ly)
//                        + Z1 / Q - (z' + 1) z qx / Q^2 ],
//   Z1 = z qx [(log z)' + qy (lx - ly)],  and l_tu = (d l_t / dx) (-1/u).
// gumbel_mixed gives the bracket [...] for x and for y; the factor
// -1/(u x) = -(m+1)/(r x) of a point of rank r comes from gumbel_margin, once
// per rank (see gaussian_margin).
template <typename Real>
__device__ __forceinline__ void gumbel_mixed(Real th, Real lx, Real ly, const GumbelPoint<Real>& p, Real& gu,
                                             Real& gv) {
  const Real qx = lx > ly ? Real(1) - p.s : p.s;
  const Real qy = Real(1) - qx;
  const Real dxy = lx - ly;
  const Real z1 = p.z * p.lz1;
  const Real iQ = p.iQ;
  const Real Z1x = p.z * qx * (p.lz1 + qy * dxy);
  const Real Z1y = p.z * qy * (p.lz1 - qx * dxy);
  const Real cQ = (z1 + Real(1)) * p.z * iQ * iQ;
  gu = -Z1x + Real(1) - Real(2) * qx * (Real(1) + th * qy * dxy) + qx * qy * dxy + Z1x * iQ - cQ * qx;
  gv = -Z1y + Real(1) - Real(2) * qy * (Real(1) - th * qx * dxy) - qx * qy * dxy + Z1y * iQ - cQ * qy;
}

// -(m+1) / (r x) for the rank r (1-based) whose lx = log x is given: the
// factor dx/du / x of the Gumbel mixed partials, u = r/(m+1), x = -log u.
template <typename Real>
__device__ __forceinline__ Real gumbel_margin(Real lx, Real mp1, Real r) {
  return -(mp1 / r) * Fn<Real>::exp(-lx);
}

}  // namespace cop
