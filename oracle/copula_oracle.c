/*
 * copula_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU oracle for the divide-and-combine maximum
 * pseudo-likelihood (MPL) copula estimator of Wei, Kim & Conlon,
 * "Parallel Computing for Copula Parameter Estimation with Big Data"
 * (arXiv:1609.05530).  It exists to check the CUDA path and to be timed as a
 * CPU baseline; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, in the paper's order:
 *   1. Row partition of the N x 2 data into M disjoint contiguous subsets
 *      (Section 2.4, Eq. 14), given as subset offsets.
 *   2. Per subset, the normalised ranks u = r/(m+1) of each margin
 *      (Section 2.3, Eq. 12; ranks are taken within the subset, Section 2.4).
 *      Ties are broken by original index (ordinal ranks).
 *   3. Per subset, the maximiser of the pseudo log-likelihood
 *      l(theta) = sum_i log c(u_i, v_i; theta)  (Section 2.3, Eq. 13) for the
 *      Gaussian (Eq. 7-8), Frank (Eq. 10) or Gumbel (Eq. 11) copula.  The
 *      maximiser is found by a coarse grid scan of l over the parameter domain
 *      (certifying the global maximum on the grid) followed by a
 *      bisection-safeguarded Newton iteration on the score inside the
 *      bracketing grid cell.
 *   4. Per subset, the asymptotic variance of the MPL estimator by the
 *      sandwich formula of Genest, Ghoudi & Rivest (1995), which Section 2.3
 *      cites: sigma^2 = nu^2 / beta^2, beta = -E[l_tt],
 *      nu^2 = Var(l_t + W1(U) + W2(V)),
 *      W1(u) = E[1{u <= U} l_tu(U,V)], W2(v) = E[1{v <= V} l_tv(U,V)];
 *      Var(theta_hat_m) = sigma^2 / m.
 *   5. The combined estimate sum w_m theta_m / sum w_m with
 *      w_m = 1 / Var(theta_hat_m)  (Section 2.4, Eq. 15).
 * Beside the MPL it provides the rank-correlation inversion estimators that
 * Section 2.3 lists as alternatives (subset Kendall's tau and Spearman's rho,
 * their population values per family, and the inversion).
 *
 * All arithmetic is FP64.  Everything is written from the closed forms of the
 * three densities; derivatives were derived by hand and are pinned in the
 * test-suite by finite differences, unit integration, the paper's printed
 * Spearman/Kendall values (Section 2.5), closed forms and brute force.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAUSSIAN 0
#define ORC_FRANK 1
#define ORC_GUMBEL 2

#define ORC_DTYPE_F32 0
#define ORC_DTYPE_F64 1

#define ORC_W_INVVAR 0
#define ORC_W_FISHER 1
#define ORC_W_EQUAL 2

#define ORC_OK 0
#define ORC_BOUNDARY 1
#define ORC_NOT_CONVERGED 2
#define ORC_DEGENERATE 3
#define ORC_CAPPED 4

/* Parameter domains.  Eq. 8 allows rho in [-1, 1]; the likelihood is only
 * finite inside, so the search stays in [-1 + 1e-9, 1 - 1e-9].  Eq. 10 allows
 * any non-zero theta; the search is capped at |theta| <= 50 (Kendall tau
 * about 0.92).  Eq. 11 needs theta >= 1; capped at 50 (tau = 0.98).  A
 * maximiser on Gumbel's own edge theta = 1 is reported as BOUNDARY; one on a
 * search cap (the likelihood still rising there) as CAPPED. */
#define ORC_GAUSS_CAP (1.0 - 1e-9)
#define ORC_FRANK_CAP 50.0
#define ORC_GUMBEL_CAP 50.0

/* Below this |theta| the Frank terms come from the Taylor series of the log
 * density about the independence copula (theta = 0, where c == 1). */
#define ORC_FRANK_SERIES 1e-3

int orc_version(void) { return 1; }

/* ------------------------------------------------------------------------ */
/* Standard normal cdf, density and quantile (used by Eq. 7-8).              */
/* ------------------------------------------------------------------------ */

static double orc_Phi(double x) { return 0.5 * erfc(-x / M_SQRT2); }
static double orc_phi(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * M_PI); }

/* Quantile of the standard normal for p in (0, 0.5]: the root x <= 0 of
 * Phi(x) = p.  Start from the rational approximation of Abramowitz & Stegun
 * 26.2.23, then Newton's method on Phi(x) - p (Phi is convex for x < 0, so
 * the iteration is monotone after one step). */
double orc_ndtri_lower(double p) {
  if (!(p > 0.0) || p > 0.5) return NAN;
  if (p == 0.5) return 0.0;
  double t = sqrt(-2.0 * log(p));
  double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                       (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
  for (int it = 0; it < 100; ++it) {
    double dx = (orc_Phi(x) - p) / orc_phi(x);
    x -= dx;
    if (fabs(dx) <= 1e-17 * fmax(1.0, fabs(x))) break;
  }
  return x;
}

/* Phi^{-1}(r/(m+1)) from the integer rank, using the exact complement
 * (m+1-r)/(m+1) in the upper half so no precision is lost near 1. */
static double orc_normal_score(int64_t r, int64_t m) {
  if (2 * r <= m + 1) return orc_ndtri_lower((double)r / (double)(m + 1));
  return -orc_ndtri_lower((double)(m + 1 - r) / (double)(m + 1));
}

/* ------------------------------------------------------------------------ */
/* Ranks (Eq. 12), within each subset (Section 2.4).                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  double val;
  int64_t idx;
} orc_key;

static int orc_key_cmp(const void* a, const void* b) {
  const orc_key* x = (const orc_key*)a;
  const orc_key* y = (const orc_key*)b;
  if (x->val < y->val) return -1;
  if (x->val > y->val) return 1;
  /* equal values (including -0.0 == +0.0): ordinal tie-break by index */
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Ranks 1..m of x[off[k] .. off[k+1]) within each subset k.  Returns 0, or
 * -1 if a subset contains NaN (its ranks are then set to 0). */
int orc_ranks(int dtype, const void* x, int64_t n, const int64_t* off, int64_t K,
              int32_t* rank_out) {
  (void)n;
  int rc = 0;
  for (int64_t k = 0; k < K; ++k) {
    int64_t m = off[k + 1] - off[k];
    orc_key* keys = (orc_key*)malloc((size_t)(m > 0 ? m : 1) * sizeof(orc_key));
    int has_nan = 0;
    for (int64_t i = 0; i < m; ++i) {
      double v = dtype == ORC_DTYPE_F32 ? (double)((const float*)x)[off[k] + i]
                                        : ((const double*)x)[off[k] + i];
      if (isnan(v)) has_nan = 1;
      keys[i].val = v;
      keys[i].idx = i;
    }
    if (has_nan) {
      for (int64_t i = 0; i < m; ++i) rank_out[off[k] + i] = 0;
      rc = -1;
    } else {
      qsort(keys, (size_t)m, sizeof(orc_key), orc_key_cmp);
      for (int64_t pos = 0; pos < m; ++pos) rank_out[off[k] + keys[pos].idx] = (int32_t)(pos + 1);
    }
    free(keys);
  }
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Per-point log density and derivatives.                                    */
/*   out[0] = l = log c(u, v; theta)                                         */
/*   out[1] = dl/dtheta, out[2] = d2l/dtheta2,                               */
/*   out[3] = d2l/dtheta du, out[4] = d2l/dtheta dv                          */
/* Pseudo-observations are u = ru/(m+1), v = rv/(m+1); each family takes its */
/* margins' transforms from the integer ranks.                               */
/* ------------------------------------------------------------------------ */

/* Per-point margin transforms, computed once per subset. */
typedef struct {
  double u, ubar; /* u and 1 - u */
  double q;       /* Gaussian: Phi^{-1}(u); Gumbel: -log(u) */
  double dq;      /* Gaussian: dq/du = 1/phi(q); Gumbel: dq/du = -1/u */
} orc_margin;

static orc_margin orc_margin_of(int family, int64_t r, int64_t m) {
  orc_margin g;
  g.u = (double)r / (double)(m + 1);
  g.ubar = (double)(m + 1 - r) / (double)(m + 1);
  g.q = 0.0;
  g.dq = 0.0;
  if (family == ORC_GAUSSIAN) {
    g.q = orc_normal_score(r, m);
    g.dq = 1.0 / orc_phi(g.q);
  } else if (family == ORC_GUMBEL) {
    g.q = (g.u <= 0.5) ? -log(g.u) : -log1p(-g.ubar);
    g.dq = -1.0 / g.u;
  }
  return g;
}

/* Gaussian copula density, bivariate case of Eq. 7 / the integrand of Eq. 8:
 *   c = (1-rho^2)^{-1/2} exp(-(rho^2 (x^2+y^2) - 2 rho x y) / (2 (1-rho^2))),
 * with x = Phi^{-1}(u), y = Phi^{-1}(v). */
static void orc_terms_gaussian(double rho, const orc_margin* a, const orc_margin* b,
                               double* out) {
  double x = a->q, y = b->q;
  double S = x * x + y * y, P = x * y;
  double om = 1.0 - rho * rho;
  out[0] = -0.5 * log(om) - (rho * rho * S - 2.0 * rho * P) / (2.0 * om);
  out[1] = rho / om - (rho * S - P * (1.0 + rho * rho)) / (om * om);
  out[2] = (1.0 + rho * rho) / (om * om) -
           (S * (1.0 + 3.0 * rho * rho) - 2.0 * P * rho * (3.0 + rho * rho)) / (om * om * om);
  out[3] = -(2.0 * rho * x - y * (1.0 + rho * rho)) / (om * om) * a->dq;
  out[4] = -(2.0 * rho * y - x * (1.0 + rho * rho)) / (om * om) * b->dq;
}

/* Frank copula, Eq. 10.  Differentiating C twice gives
 *   c = theta (1 - e^{-theta}) e^{-theta (u+v)} / D^2,
 *   D = e^{-theta u} + e^{-theta v} - e^{-theta (u+v)} - e^{-theta},
 * where D is evaluated without cancellation as
 *   D = -e^{-theta u} expm1(-theta v) - e^{-theta v} expm1(-theta (1-v)). */
static void orc_terms_frank(double t, const orc_margin* A, const orc_margin* B, double* out) {
  double u = A->u, v = B->u;
  if (fabs(t) < ORC_FRANK_SERIES) {
    /* log c = sum_k c_k theta^k about theta = 0 (independence), with
     * P = u(1-u), Q = v(1-v), s = (1-2u)(1-2v):
     *   c1 = s/2, c2 = PQ - 1/24, c3 = PQ s / 6,
     *   c4 = P^2 Q^2 / 2 - PQ (P+Q) / 12 + 1/2880,
     *   c5 = PQ s (36 PQ - 3 (P+Q) - 1) / 360. */
    double su = 1.0 - 2.0 * u, sv = 1.0 - 2.0 * v;
    double P = u * A->ubar, Q = v * B->ubar, s = su * sv;
    double c1 = 0.5 * s, c2 = P * Q - 1.0 / 24.0, c3 = P * Q * s / 6.0;
    double c4 = 0.5 * P * P * Q * Q - P * Q * (P + Q) / 12.0 + 1.0 / 2880.0;
    double c5 = P * Q * s * (36.0 * P * Q - 3.0 * (P + Q) - 1.0) / 360.0;
    out[0] = t * (c1 + t * (c2 + t * (c3 + t * (c4 + t * c5))));
    out[1] = c1 + t * (2.0 * c2 + t * (3.0 * c3 + t * (4.0 * c4 + t * 5.0 * c5)));
    out[2] = 2.0 * c2 + t * (6.0 * c3 + t * (12.0 * c4 + t * 20.0 * c5));
    /* d/du of c1..c4 (dP/du = 1-2u, ds/du = -2(1-2v)) */
    double dc1u = -sv;
    double dc2u = su * Q;
    double dc3u = Q * sv * (1.0 - 6.0 * P) / 6.0;
    double dc4u = su * (P * Q * Q - Q * (2.0 * P + Q) / 12.0);
    double dc1v = -su;
    double dc2v = sv * P;
    double dc3v = P * su * (1.0 - 6.0 * Q) / 6.0;
    double dc4v = sv * (Q * P * P - P * (2.0 * Q + P) / 12.0);
    out[3] = dc1u + t * (2.0 * dc2u + t * (3.0 * dc3u + t * 4.0 * dc4u));
    out[4] = dc1v + t * (2.0 * dc2v + t * (3.0 * dc3v + t * 4.0 * dc4v));
    return;
  }
  double a = exp(-t * u), b = exp(-t * v), E = exp(-t);
  double omb = -expm1(-t * v);      /* 1 - b */
  double oma = -expm1(-t * u);      /* 1 - a */
  double D = a * omb - b * expm1(-t * B->ubar);
  double D1 = -u * a - v * b + (u + v) * a * b + E;
  double D2 = u * u * a + v * v * b - (u + v) * (u + v) * a * b - E;
  double k0 = log(-t * expm1(-t)); /* log(theta (1 - e^{-theta})) > 0 argument */
  double k1 = 1.0 / t + 1.0 / expm1(t);
  double k2 = -1.0 / (t * t) - exp(t) / (expm1(t) * expm1(t));
  out[0] = k0 - t * (u + v) - 2.0 * log(fabs(D));
  out[1] = k1 - (u + v) - 2.0 * D1 / D;
  out[2] = k2 - 2.0 * (D2 / D - (D1 / D) * (D1 / D));
  /* dl/du = -theta + 2 theta a (1-b) / D; differentiate in theta. */
  double Fu = a * omb, Fv = b * oma;
  double dFu = -u * a * omb + v * a * b, dFv = -v * b * oma + u * a * b;
  out[3] = -1.0 + 2.0 * (Fu + t * dFu) / D - 2.0 * t * Fu * D1 / (D * D);
  out[4] = -1.0 + 2.0 * (Fv + t * dFv) / D - 2.0 * t * Fv * D1 / (D * D);
}

/* Gumbel copula, Eq. 11, with x = -log u, y = -log v, lx = log x, ly = log y,
 * w = x^theta + y^theta, L = log w, z = w^{1/theta}:
 *   log c = -z + x + y + (theta-1)(lx+ly) - 2L + L/theta + log(z + theta - 1). */
static void orc_terms_gumbel(double t, const orc_margin* A, const orc_margin* B, double* out) {
  double x = A->q, y = B->q;
  double lx = log(x), ly = log(y);
  double xt = exp(t * lx), yt = exp(t * ly);
  double w = xt + yt, L = log(w), z = exp(L / t);
  double L1 = (xt * lx + yt * ly) / w;
  double L2 = (xt * lx * lx + yt * ly * ly) / w - L1 * L1;
  double lz1 = L1 / t - L / (t * t);
  double lz2 = L2 / t - 2.0 * L1 / (t * t) + 2.0 * L / (t * t * t);
  double z1 = z * lz1, z2 = z * (lz1 * lz1 + lz2);
  double Qz = z + t - 1.0;
  out[0] = -z + x + y + (t - 1.0) * (lx + ly) - 2.0 * L + L / t + log(Qz);
  out[1] = -z1 + (lx + ly) - 2.0 * L1 + lz1 + (z1 + 1.0) / Qz;
  out[2] = -z2 - 2.0 * L2 + lz2 + z2 / Qz - ((z1 + 1.0) / Qz) * ((z1 + 1.0) / Qz);
  /* d l_theta / dx, with qx = x^theta / w, qy = y^theta / w (qx + qy = 1). */
  double qx = xt / w, qy = yt / w;
  double Z1x = z * qx * (lz1 + qy * (lx - ly));
  double Z1y = z * qy * (lz1 + qx * (ly - lx));
  double dldx = (-Z1x + 1.0 - 2.0 * qx * (1.0 + t * qy * (lx - ly)) + qx * qy * (lx - ly) +
                 Z1x / Qz - (z1 + 1.0) * z * qx / (Qz * Qz)) / x;
  double dldy = (-Z1y + 1.0 - 2.0 * qy * (1.0 + t * qx * (ly - lx)) + qx * qy * (ly - lx) +
                 Z1y / Qz - (z1 + 1.0) * z * qy / (Qz * Qz)) / y;
  out[3] = dldx * A->dq; /* dx/du = -1/u */
  out[4] = dldy * B->dq;
}

static void orc_terms(int family, double theta, const orc_margin* a, const orc_margin* b,
                      double* out) {
  if (family == ORC_GAUSSIAN)
    orc_terms_gaussian(theta, a, b, out);
  else if (family == ORC_FRANK)
    orc_terms_frank(theta, a, b, out);
  else
    orc_terms_gumbel(theta, a, b, out);
}

/* Per-point terms at pseudo-observation (ru/(m+1), rv/(m+1)). */
int orc_point(int family, double theta, int64_t ru, int64_t rv, int64_t m, double* out) {
  if (family < 0 || family > 2 || ru < 1 || rv < 1 || ru > m || rv > m) return -1;
  orc_margin a = orc_margin_of(family, ru, m), b = orc_margin_of(family, rv, m);
  orc_terms(family, theta, &a, &b, out);
  return 0;
}

/* The margin transform of one coordinate in (0,1) (not a rank), given as u
 * and its complement ubar = 1 - u (exact when the caller has it: near 1 the
 * transforms are taken from ubar). */
static orc_margin orc_margin_at(int family, double u, double ubar) {
  orc_margin a;
  a.u = u;
  a.ubar = ubar;
  if (family == ORC_GAUSSIAN) {
    a.q = u <= 0.5 ? orc_ndtri_lower(u) : -orc_ndtri_lower(ubar);
    a.dq = 1.0 / orc_phi(a.q);
  } else if (family == ORC_GUMBEL) {
    a.q = u <= 0.5 ? -log(u) : -log1p(-ubar);
    a.dq = -1.0 / u;
  } else {
    a.q = a.dq = 0.0;
  }
  return a;
}

/* Per-point terms at arbitrary (u, v) in (0,1)^2 (for derivative pins). */
void orc_terms_at(int family, double theta, double u, double v, double* out) {
  orc_margin a = orc_margin_at(family, u, 1.0 - u), b = orc_margin_at(family, v, 1.0 - v);
  orc_terms(family, theta, &a, &b, out);
}

/* Copula density c(u_i, v_i; theta) at n arbitrary points (integration pins). */
void orc_density_vec(int family, double theta, const double* u, const double* v, int64_t n,
                     double* c) {
  double out[5];
  for (int64_t i = 0; i < n; ++i) {
    orc_terms_at(family, theta, u[i], v[i], out);
    c[i] = exp(out[0]);
  }
}

/* The copula itself, Eq. 10 (Frank) and Eq. 11 (Gumbel); the Gaussian copula
 * (Eq. 8) has no closed form and is not provided here. */
double orc_cdf(int family, double theta, double u, double v) {
  if (family == ORC_FRANK)
    return -1.0 / theta * log1p(expm1(-theta * u) * expm1(-theta * v) / expm1(-theta));
  if (family == ORC_GUMBEL)
    return exp(-pow(pow(-log(u), theta) + pow(-log(v), theta), 1.0 / theta));
  return NAN;
}

/* ------------------------------------------------------------------------ */
/* Subset fit.                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int family;
  int64_t m;
  orc_margin* mu; /* per point, u margin */
  orc_margin* mv; /* per point, v margin */
} orc_subset;

/* Eq. 13 and its first two theta-derivatives summed over the subset. */
static void orc_sums(const orc_subset* S, double theta, double* l, double* g, double* h) {
  double sl = 0, sg = 0, sh = 0, out[5];
  for (int64_t i = 0; i < S->m; ++i) {
    orc_terms(S->family, theta, &S->mu[i], &S->mv[i], out);
    sl += out[0];
    sg += out[1];
    sh += out[2];
  }
  if (l) *l = sl;
  if (g) *g = sg;
  if (h) *h = sh;
}

static double orc_loglik_at(const orc_subset* S, double theta) {
  double l;
  orc_sums(S, theta, &l, NULL, NULL);
  return l;
}

/* Search grid over the parameter domain, increasing in theta. */
static int orc_grid(int family, double* grid) {
  int G = 0;
  if (family == ORC_GAUSSIAN) {
    for (int j = 0; j < 199; ++j) grid[G++] = -ORC_GAUSS_CAP + 2.0 * ORC_GAUSS_CAP * j / 198.0;
    grid[0] = -ORC_GAUSS_CAP;
    grid[G - 1] = ORC_GAUSS_CAP;
  } else if (family == ORC_FRANK) {
    /* 200 points, symmetric, never exactly 0 */
    for (int j = 0; j < 200; ++j) grid[G++] = -ORC_FRANK_CAP + (j + 0.5) * (2.0 * ORC_FRANK_CAP / 200.0);
    grid[0] = -ORC_FRANK_CAP;
    grid[G - 1] = ORC_FRANK_CAP;
  } else {
    /* theta = 1/(1 - tau) over tau in [0, 1 - 1/cap] */
    double tmax = 1.0 - 1.0 / ORC_GUMBEL_CAP;
    for (int j = 0; j < 200; ++j) grid[G++] = 1.0 / (1.0 - tmax * j / 199.0);
    grid[0] = 1.0;
    grid[G - 1] = ORC_GUMBEL_CAP;
  }
  return G;
}

/* Golden-section maximisation of l on [a, b] (used only when the score does
 * not change sign across the bracketing grid cell). */
static double orc_golden(const orc_subset* S, double a, double b) {
  const double r = 0.5 * (sqrt(5.0) - 1.0);
  double c = b - r * (b - a), d = a + r * (b - a);
  double fc = orc_loglik_at(S, c), fd = orc_loglik_at(S, d);
  for (int it = 0; it < 200 && (b - a) > 1e-15 * fmax(1.0, fabs(a)); ++it) {
    if (fc > fd) {
      b = d; d = c; fd = fc; c = b - r * (b - a); fc = orc_loglik_at(S, c);
    } else {
      a = c; c = d; fc = fd; d = a + r * (b - a); fd = orc_loglik_at(S, d);
    }
  }
  return 0.5 * (a + b);
}

/* Maximiser of Eq. 13 for one subset.  Returns a status code. */
static int orc_maximise(const orc_subset* S, double* theta_out, int* iters_out) {
  double grid[256];
  int G = orc_grid(S->family, grid);
  double best = -INFINITY;
  int jb = -1;
  for (int j = 0; j < G; ++j) {
    double l = orc_loglik_at(S, grid[j]);
    if (isfinite(l) && l > best) { best = l; jb = j; }
  }
  if (jb < 0) { *theta_out = NAN; return ORC_DEGENERATE; }
  double lo = grid[jb > 0 ? jb - 1 : 0], hi = grid[jb < G - 1 ? jb + 1 : G - 1];
  double glo, ghi;
  orc_sums(S, lo, NULL, &glo, NULL);
  orc_sums(S, hi, NULL, &ghi, NULL);
  int status = ORC_OK;
  /* A maximiser on the domain's edge (score pointing outwards). */
  if (jb == 0 && glo <= 0.0) {
    *theta_out = grid[0];
    *iters_out = 0;
    return S->family == ORC_GUMBEL ? ORC_BOUNDARY : ORC_CAPPED;
  }
  if (jb == G - 1 && ghi >= 0.0) { *theta_out = grid[G - 1]; *iters_out = 0; return ORC_CAPPED; }
  if (!(glo > 0.0 && ghi < 0.0)) {
    /* no sign change across the cell: maximise l directly, then polish */
    double t = orc_golden(S, lo, hi);
    *theta_out = t;
    *iters_out = -1;
    return ORC_OK;
  }
  /* Bisection-safeguarded Newton on the score g inside [lo, hi]. */
  double t = grid[jb];
  int it;
  for (it = 0; it < 200; ++it) {
    double g, h;
    orc_sums(S, t, NULL, &g, &h);
    if (g > 0.0) lo = t; else hi = t;
    if (g == 0.0) break;
    double tn = (h < 0.0) ? t - g / h : NAN;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    double step = fabs(tn - t);
    t = tn;
    if (step <= 1e-14 * fmax(1.0, fabs(t)) || (hi - lo) <= 1e-15 * fmax(1.0, fabs(t))) break;
  }
  if (it >= 200) status = ORC_NOT_CONVERGED;
  *theta_out = t;
  *iters_out = it + 1;
  return status;
}

/* Sandwich variance of Genest, Ghoudi & Rivest (1995) at theta, returning
 * Var(theta_hat) = sigma^2/m.  If direct != 0 the W terms use the O(m^2)
 * double sum, otherwise a suffix sum over the rank order (ranks are a
 * permutation of 1..m, so rank r sits at slot r-1). */
static double orc_variance(const orc_subset* S, const int32_t* ru, const int32_t* rv,
                           double theta, int direct, double* beta_out) {
  int64_t m = S->m;
  double* lt = (double*)malloc((size_t)m * sizeof(double));
  double* ltu = (double*)malloc((size_t)m * sizeof(double));
  double* ltv = (double*)malloc((size_t)m * sizeof(double));
  double* W1 = (double*)malloc((size_t)m * sizeof(double));
  double* W2 = (double*)malloc((size_t)m * sizeof(double));
  double sh = 0.0, out[5];
  for (int64_t i = 0; i < m; ++i) {
    orc_terms(S->family, theta, &S->mu[i], &S->mv[i], out);
    lt[i] = out[1];
    sh += out[2];
    ltu[i] = out[3];
    ltv[i] = out[4];
  }
  if (direct) {
    for (int64_t i = 0; i < m; ++i) {
      double s1 = 0.0, s2 = 0.0;
      for (int64_t j = 0; j < m; ++j) {
        if (ru[i] <= ru[j]) s1 += ltu[j];
        if (rv[i] <= rv[j]) s2 += ltv[j];
      }
      W1[i] = s1 / (double)m;
      W2[i] = s2 / (double)m;
    }
  } else {
    double* bu = (double*)calloc((size_t)m, sizeof(double));
    double* bv = (double*)calloc((size_t)m, sizeof(double));
    for (int64_t i = 0; i < m; ++i) {
      bu[ru[i] - 1] = ltu[i];
      bv[rv[i] - 1] = ltv[i];
    }
    for (int64_t r = m - 2; r >= 0; --r) {
      bu[r] += bu[r + 1];
      bv[r] += bv[r + 1];
    }
    for (int64_t i = 0; i < m; ++i) {
      W1[i] = bu[ru[i] - 1] / (double)m;
      W2[i] = bv[rv[i] - 1] / (double)m;
    }
    free(bu);
    free(bv);
  }
  double mean = 0.0;
  for (int64_t i = 0; i < m; ++i) mean += lt[i] + W1[i] + W2[i];
  mean /= (double)m;
  double nu2 = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    double d = lt[i] + W1[i] + W2[i] - mean;
    nu2 += d * d;
  }
  nu2 /= (double)m;
  double beta = -sh / (double)m;
  if (beta_out) *beta_out = beta;
  free(lt); free(ltu); free(ltv); free(W1); free(W2);
  return nu2 / (beta * beta) / (double)m;
}

static void orc_subset_build(orc_subset* S, int family, const int32_t* ru, const int32_t* rv,
                             int64_t m) {
  S->family = family;
  S->m = m;
  S->mu = (orc_margin*)malloc((size_t)m * sizeof(orc_margin));
  S->mv = (orc_margin*)malloc((size_t)m * sizeof(orc_margin));
  for (int64_t i = 0; i < m; ++i) {
    S->mu[i] = orc_margin_of(family, ru[i], m);
    S->mv[i] = orc_margin_of(family, rv[i], m);
  }
}

static void orc_subset_free(orc_subset* S) {
  free(S->mu);
  free(S->mv);
}

/* Pseudo-likelihood sums (Eq. 13) of one subset given its ranks. */
int orc_loglik(int family, double theta, const int32_t* ru, const int32_t* rv, int64_t m,
               double* l, double* g, double* h) {
  if (m < 1) return -1;
  orc_subset S;
  orc_subset_build(&S, family, ru, rv, m);
  orc_sums(&S, theta, l, g, h);
  orc_subset_free(&S);
  return 0;
}

/* The stages of one subset's fit exposed one at a time, so that each can be
 * timed on its own: orc_subset_new takes the ranks and computes every
 * point's margin transforms (Eq. 12's u = r/(m+1) and the family's
 * Phi^{-1} or -log of it), orc_subset_sums is one pass of Eq. 13 and its
 * theta-derivatives over those points, orc_subset_delete frees them. */
void* orc_subset_new(int family, const int32_t* ru, const int32_t* rv, int64_t m) {
  if (m < 1 || family < 0 || family > 2) return NULL;
  orc_subset* S = (orc_subset*)malloc(sizeof(orc_subset));
  orc_subset_build(S, family, ru, rv, m);
  return S;
}

void orc_subset_sums(const void* handle, double theta, double* l, double* g, double* h) {
  orc_sums((const orc_subset*)handle, theta, l, g, h);
}

void orc_subset_delete(void* handle) {
  if (!handle) return;
  orc_subset_free((orc_subset*)handle);
  free(handle);
}

/* Variance of theta_hat at a given theta from ranks; direct selects the
 * O(m^2) form. */
double orc_var_at(int family, double theta, const int32_t* ru, const int32_t* rv, int64_t m,
                  int direct) {
  orc_subset S;
  orc_subset_build(&S, family, ru, rv, m);
  double v = orc_variance(&S, ru, rv, theta, direct, NULL);
  orc_subset_free(&S);
  return v;
}

/* Fit one subset from its ranks: theta_hat (Eq. 13 maximiser), its variance
 * and the observed information -sum l_tt at theta_hat. */
int orc_fit_ranks(int family, const int32_t* ru, const int32_t* rv, int64_t m, double* theta,
                  double* var, double* info, int* iters) {
  if (m < 2) { *theta = NAN; *var = NAN; *info = NAN; return ORC_DEGENERATE; }
  for (int64_t i = 0; i < m; ++i)
    if (ru[i] < 1 || rv[i] < 1) { *theta = NAN; *var = NAN; *info = NAN; return ORC_DEGENERATE; }
  orc_subset S;
  orc_subset_build(&S, family, ru, rv, m);
  int it = 0;
  int st = orc_maximise(&S, theta, &it);
  if (iters) *iters = it;
  if (st == ORC_DEGENERATE) {
    *var = NAN; *info = NAN;
  } else {
    double beta;
    *var = orc_variance(&S, ru, rv, *theta, m <= 2000, &beta);
    *info = beta * (double)m;
  }
  orc_subset_free(&S);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Rank-correlation inversion (Section 2.3 lists the inversion of Kendall's  */
/* tau and of Spearman's rho among the estimators the paper does not use;    */
/* the population values are the ones Section 2.5 prints beside each        */
/* generating parameter).  Textbook definitions, written out directly.      */
/* ------------------------------------------------------------------------ */

/* Kendall's tau of one subset from its ranks: (concordant - discordant)
 * pairs over all m(m-1)/2 pairs, every pair looked at (ordinal ranks have no
 * ties). */
double orc_kendall_tau(const int32_t* ru, const int32_t* rv, int64_t m) {
  if (m < 2) return NAN;
  int64_t s = 0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = i + 1; j < m; ++j) {
      const int64_t a = (int64_t)ru[i] - ru[j], b = (int64_t)rv[i] - rv[j];
      s += (a > 0) == (b > 0) ? 1 : -1;
    }
  return (double)s / (0.5 * (double)m * (double)(m - 1));
}

/* Kendall's tau of one subset from its ranks, counted faster for large m:
 * with the v-ranks listed in u-rank order (pi), a pair is discordant exactly
 * when it is an inversion of pi, and the inversions are counted by a
 * bottom-up merge sort of pi (O(m log m)).  Same value as orc_kendall_tau,
 * whose every-pair count is the definition. */
double orc_kendall_tau_merge(const int32_t* ru, const int32_t* rv, int64_t m) {
  if (m < 2) return NAN;
  int32_t* a = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* b = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  for (int64_t i = 0; i < m; ++i) a[ru[i] - 1] = rv[i];
  int64_t inv = 0;
  for (int64_t w = 1; w < m; w *= 2) {
    for (int64_t lo = 0; lo < m; lo += 2 * w) {
      int64_t mid = lo + w < m ? lo + w : m, hi = lo + 2 * w < m ? lo + 2 * w : m;
      int64_t i = lo, j = mid, k = lo;
      while (i < mid && j < hi) {
        if (a[i] <= a[j]) {
          b[k++] = a[i++];
        } else {
          inv += mid - i; /* a[j] is below every element left in the left run */
          b[k++] = a[j++];
        }
      }
      while (i < mid) b[k++] = a[i++];
      while (j < hi) b[k++] = a[j++];
    }
    int32_t* t = a;
    a = b;
    b = t;
  }
  free(a);
  free(b);
  const int64_t P = m * (m - 1) / 2;
  return (double)(P - 2 * inv) / (0.5 * (double)m * (double)(m - 1));
}

/* Spearman's rho of one subset from its ranks: 1 - 6 sum d^2 / (m (m^2 - 1)),
 * d = r_u - r_v (no ties). */
double orc_spearman_rho(const int32_t* ru, const int32_t* rv, int64_t m) {
  if (m < 2) return NAN;
  double sd = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const double d = (double)ru[i] - (double)rv[i];
    sd += d * d;
  }
  const double md = (double)m;
  return 1.0 - 6.0 * sd / (md * (md * md - 1.0));
}

/* Debye function D_k(x) = (k / x^k) int_0^x t^k / (e^t - 1) dt, x > 0, by
 * composite Simpson on 20,000 panels (the integrand is smooth on [0, x]; at
 * t = 0 it tends to t^(k-1)). */
static double orc_debye(int k, double x) {
  const int n = 20000;
  const double h = x / n;
  double s = 0.0;
  for (int i = 0; i <= n; ++i) {
    const double t = i * h;
    const double f = t == 0.0 ? (k == 1 ? 1.0 : 0.0) : pow(t, k) / expm1(t);
    s += (i == 0 || i == n) ? f : (i & 1) ? 4.0 * f : 2.0 * f;
  }
  return (double)k / pow(x, k) * s * h / 3.0;
}

/* Frank's tau (which = 0) and rho_S (which = 1) for 0 < x < 0.5 from their
 * power series, where the closed forms below cancel: with Bernoulli numbers
 * B_2j, D_k(x) = 1 - kx/(2(k+1)) + k sum_j B_2j x^2j / ((2j+k)(2j)!)
 * (|x| < 2 pi), so tau = 4 sum_j B_2j x^(2j-1) / ((2j+1)(2j)!) and
 * rho_S = 12 sum_j j B_2j x^(2j-1) / ((2j+1)(j+1)(2j)!).  Six terms; the
 * first one left out is below 1e-15 at x = 0.5. */
static double orc_frank_corr_series(int which, double x) {
  static const double B[6] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0, -691.0 / 2730.0};
  double s = 0.0, fact = 1.0, xp = x;  /* fact = (2j)!, xp = x^(2j-1) */
  for (int j = 1; j <= 6; ++j) {
    fact *= (2.0 * j - 1.0) * (2.0 * j);
    const double t = B[j - 1] * xp / ((2.0 * j + 1.0) * fact);
    s += which == 0 ? 4.0 * t : 12.0 * j * t / (j + 1.0);
    xp *= x * x;
  }
  return s;
}

/* Population Kendall's tau of a family at theta: Gaussian (2/pi) asin(rho);
 * Frank 1 - (4/theta)(1 - D_1(theta)) (odd in theta; the series above for
 * |theta| < 0.5); Gumbel 1 - 1/theta. */
double orc_tau_of_theta(int family, double theta) {
  if (family == ORC_GAUSSIAN) return 2.0 / M_PI * asin(theta);
  if (family == ORC_GUMBEL) return 1.0 - 1.0 / theta;
  const double a = fabs(theta);
  const double t = a < 0.5 ? orc_frank_corr_series(0, a) : 1.0 - 4.0 / a * (1.0 - orc_debye(1, a));
  return theta < 0.0 ? -t : t;
}

/* Population Spearman's rho: Gaussian (6/pi) asin(rho/2); Frank
 * 1 - (12/theta)(D_1(theta) - D_2(theta)) (odd in theta; the series above for
 * |theta| < 0.5); Gumbel 12 int int C(u, v) du dv - 3 integrated directly.
 * For Gumbel the integral is taken over the triangle v < u (C is symmetric)
 * with v = u s, rho_S = 24 int_0^1 int_0^1 C(u, u s) u ds du - 3, so that
 * the ridge C develops along the diagonal for large theta lies on the
 * domain's edge, by a product rule of 10-point Gauss-Legendre on panels
 * graded geometrically towards 0 and 1 (10 panels from 1e-12 to 0.02 at each
 * end, 18 equal panels between); good to a few 1e-12. */
double orc_rho_s_of_theta(int family, double theta) {
  if (family == ORC_GAUSSIAN) return 6.0 / M_PI * asin(0.5 * theta);
  if (family == ORC_FRANK) {
    const double a = fabs(theta);
    const double r = a < 0.5 ? orc_frank_corr_series(1, a) : 1.0 - 12.0 / a * (orc_debye(1, a) - orc_debye(2, a));
    return theta < 0.0 ? -r : r;
  }
  enum { NQ = 10, NG = 10, NMID = 18, NPAN = 2 * NG + NMID, N = NPAN * NQ };
  double gx[NQ], gw[NQ];
  for (int i = 0; i < NQ; ++i) { /* Gauss-Legendre nodes on [-1, 1]: Newton on P_10 */
    double z = cos(M_PI * (i + 0.75) / (NQ + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= NQ; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      pp = NQ * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    gx[i] = z;
    gw[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
  double e[NPAN + 1];
  int ne = 0;
  e[ne++] = 0.0;
  for (int i = 0; i < NG; ++i) e[ne++] = 1e-12 * pow(0.02 / 1e-12, (double)i / (NG - 1));
  for (int i = 1; i < NMID; ++i) e[ne++] = 0.02 + 0.96 * i / NMID;
  for (int i = NG - 1; i >= 0; --i) e[ne++] = 1.0 - 1e-12 * pow(0.02 / 1e-12, (double)i / (NG - 1));
  e[ne++] = 1.0;
  double x[N], w[N];
  for (int p = 0; p < NPAN; ++p)
    for (int i = 0; i < NQ; ++i) {
      x[p * NQ + i] = 0.5 * (e[p] + e[p + 1]) + 0.5 * (e[p + 1] - e[p]) * gx[i];
      w[p * NQ + i] = 0.5 * (e[p + 1] - e[p]) * gw[i];
    }
  double s = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) s += w[i] * w[j] * x[i] * orc_cdf(ORC_GUMBEL, theta, x[i], x[i] * x[j]);
  return 24.0 * s - 3.0;
}

/* The parameter whose population tau (which = 0) or Spearman's rho
 * (which = 1) equals r: closed forms where the family has one (Gaussian both,
 * Gumbel tau), else bisection on the increasing map over the search domain
 * (Frank [-50, 50], Gumbel [1, 50]) to a bracket of 1e-14.  Status OK;
 * BOUNDARY for Gumbel at r <= its value at theta = 1 (independence, 0),
 * reported as theta = 1; CAPPED beyond a cap (theta set to the cap). */
int orc_theta_from_rank_corr(int family, int which, double r, double* theta) {
  if (!(r >= -1.0 && r <= 1.0)) { *theta = NAN; return ORC_DEGENERATE; }
  if (family == ORC_GAUSSIAN) {
    double rho = which == 0 ? sin(0.5 * M_PI * r) : 2.0 * sin(M_PI * r / 6.0);
    if (rho > ORC_GAUSS_CAP) { *theta = ORC_GAUSS_CAP; return ORC_CAPPED; }
    if (rho < -ORC_GAUSS_CAP) { *theta = -ORC_GAUSS_CAP; return ORC_CAPPED; }
    *theta = rho;
    return ORC_OK;
  }
  double lo = family == ORC_FRANK ? -ORC_FRANK_CAP : 1.0;
  double hi = family == ORC_FRANK ? ORC_FRANK_CAP : ORC_GUMBEL_CAP;
  double (*f)(int, double) = which == 0 ? orc_tau_of_theta : orc_rho_s_of_theta;
  if (family == ORC_GUMBEL && r <= 0.0) { *theta = 1.0; return ORC_BOUNDARY; }
  if (family == ORC_GUMBEL && which == 0) {
    const double t = 1.0 / (1.0 - r);
    if (t > hi) { *theta = hi; return ORC_CAPPED; }
    *theta = t;
    return ORC_OK;
  }
  if (r >= f(family, hi)) { *theta = hi; return ORC_CAPPED; }
  if (r <= f(family, lo)) { *theta = lo; return family == ORC_GUMBEL ? ORC_BOUNDARY : ORC_CAPPED; }
  while (hi - lo > 1e-14 * fmax(1.0, fabs(lo))) {
    const double mid = 0.5 * (lo + hi);
    if (f(family, mid) < r)
      lo = mid;
    else
      hi = mid;
  }
  *theta = 0.5 * (lo + hi);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Relative L1 / L2 distance between two copula densities of one family      */
/* (Section 2.6, Eq. 19-20), over the square [delta, 1-delta]^2.            */
/* ------------------------------------------------------------------------ */

/* Fills out[0..3] with the integrals over [delta, 1-delta]^2 of |ca - cb|,
 * |ca|, (ca - cb)^2 and ca^2, where ca = c(.; theta_a), cb = c(.; theta_b);
 * Eq. 19 is out[0]/out[1] and Eq. 20 sqrt(out[2]/out[3]).  Product rule:
 * per axis, 10-point Gauss-Legendre on panels graded geometrically towards
 * both ends, where the densities' corner singularities sit (20 panels from
 * delta, or from 1e-12 when delta = 0, up to 0.02; for delta = 0 another 40
 * panels from 1e-100 to 1e-12 for the Gaussian and Frank families, since the
 * squared Gaussian density of strong dependence still has mass at normal
 * scores beyond -7), and 48 equal panels between.  The upper half mirrors
 * the lower one with its nodes held as exact complements.  delta = 0
 * integrates the whole square; the Gumbel density is of order
 * 1/|(1-u, 1-v)| near (1, 1), so its squared integrals grow like
 * log(1/delta) and Eq. 20 needs delta > 0 for that family.  Accuracy: the
 * unit mass of every density to ~1e-12; the Gaussian int int c^2 =
 * 1/(1 - rho^2) to ~1e-12 at |rho| = 0.3 and 1e-10 at 0.5, but only 3e-5 at
 * 0.8, since an axis-aligned product rule does not follow the narrow
 * diagonal ridge of strong dependence.  Returns -1 for
 * bad arguments and -2 if an integrand overflowed or underflowed to a
 * non-finite value (Gumbel with (delta or 1e-12)^theta below the FP64
 * range). */
int orc_density_distance(int family, double theta_a, double theta_b, double delta, double* out) {
  if (family < 0 || family > 2 || !(delta >= 0.0 && delta < 0.02)) return -1;
  enum { NQ = 10, NG = 20, NT = 40, NM = 48 };
  double gx[NQ], gw[NQ];
  for (int i = 0; i < NQ; ++i) { /* Newton on P_10 */
    double z = cos(M_PI * (i + 0.75) / (NQ + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= NQ; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      pp = NQ * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    gx[i] = z;
    gw[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
  /* panel edges on [delta, 1/2]: graded to 0.02, then equal; the upper half
   * mirrors them, its nodes held as exact complements t = 1 - u */
  const double lo = delta > 0.0 ? delta : 1e-12;
  const int nt = (delta > 0.0 || family == ORC_GUMBEL) ? 0 : NT;
  double e[NT + NG + NM / 2 + 1];
  int ne = 0;
  e[ne++] = delta;
  for (int i = 1; i <= nt; ++i) e[ne++] = 1e-100 * pow(1e-12 / 1e-100, (double)i / nt);
  for (int i = 1; i <= NG; ++i) e[ne++] = lo * pow(0.02 / lo, (double)i / NG);
  for (int i = 1; i <= NM / 2; ++i) e[ne++] = 0.02 + 0.48 * i / (NM / 2);
  const int np = ne - 1, n = 2 * np * NQ;
  double* w = (double*)malloc((size_t)n * sizeof(double));
  orc_margin* mg = (orc_margin*)malloc((size_t)n * sizeof(orc_margin));
  for (int p = 0; p < np; ++p)
    for (int i = 0; i < NQ; ++i) {
      const double t = 0.5 * (e[p] + e[p + 1]) + 0.5 * (e[p + 1] - e[p]) * gx[i];
      const double wt = 0.5 * (e[p + 1] - e[p]) * gw[i];
      const int k = p * NQ + i;
      mg[k] = orc_margin_at(family, t, 1.0 - t);
      w[k] = wt;
      mg[n - 1 - k] = orc_margin_at(family, 1.0 - t, t);
      w[n - 1 - k] = wt;
    }
  double s[4] = {0, 0, 0, 0}, ta[5], tb[5];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      orc_terms(family, theta_a, &mg[i], &mg[j], ta);
      orc_terms(family, theta_b, &mg[i], &mg[j], tb);
      const double ca = exp(ta[0]), cb = exp(tb[0]), ww = w[i] * w[j];
      s[0] += ww * fabs(ca - cb);
      s[1] += ww * fabs(ca);
      s[2] += ww * (ca - cb) * (ca - cb);
      s[3] += ww * ca * ca;
    }
  free(w);
  free(mg);
  for (int k = 0; k < 4; ++k) out[k] = s[k];
  for (int k = 0; k < 4; ++k)
    if (!isfinite(s[k])) return -2;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole estimator: partition (Eq. 14), per-subset MPL, combine (Eq. 15).    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int family, dtype;
  const void *u, *v;
  const int64_t* off;
  int64_t K;
  double *theta, *var, *info;
  int32_t* status;
  int32_t* iters;
  int tid, nthreads;
} orc_job;

static void* orc_worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  for (int64_t k = J->tid; k < J->K; k += J->nthreads) {
    int64_t m = J->off[k + 1] - J->off[k];
    int64_t sub[2] = {0, m};
    int32_t* ru = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t* rv = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    size_t es = J->dtype == ORC_DTYPE_F32 ? 4 : 8;
    const char* pu = (const char*)J->u + (size_t)J->off[k] * es;
    const char* pv = (const char*)J->v + (size_t)J->off[k] * es;
    int bad = orc_ranks(J->dtype, pu, m, sub, 1, ru) | orc_ranks(J->dtype, pv, m, sub, 1, rv);
    int it = 0;
    if (bad) {
      J->theta[k] = NAN; J->var[k] = NAN; J->info[k] = NAN;
      J->status[k] = ORC_DEGENERATE;
    } else {
      J->status[k] = orc_fit_ranks(J->family, ru, rv, m, &J->theta[k], &J->var[k], &J->info[k], &it);
    }
    if (J->iters) J->iters[k] = it;
    free(ru);
    free(rv);
  }
  return NULL;
}

/* Eq. 15: weighted mean of the subset estimates in subset order.  Only
 * subsets with an interior maximiser or one on Gumbel's edge theta = 1 take
 * part (a capped, unconverged or NaN subset has no asymptotic variance), and
 * only with a finite positive weight. */
double orc_combine(const double* theta, const double* var, const double* info, const int32_t* status,
                   int64_t K, int weight) {
  double num = 0.0, den = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    if (status && status[k] != ORC_OK && status[k] != ORC_BOUNDARY) continue;
    double w = weight == ORC_W_INVVAR ? 1.0 / var[k] : weight == ORC_W_FISHER ? info[k] : 1.0;
    if (!isfinite(w) || !isfinite(theta[k]) || !(w > 0.0)) continue;
    num += w * theta[k];
    den += w;
  }
  return den > 0.0 ? num / den : NAN;
}

/* Full estimator.  off has K+1 entries with off[0] = 0 and off[K] = n.
 * Returns 0, or -1 for invalid arguments.  iters may be NULL. */
int orc_fit(int family, int dtype, const void* u, const void* v, int64_t n, const int64_t* off,
            int64_t K, int weight, double* theta, double* var, double* info, int32_t* status,
            int32_t* iters, double* combined, int nthreads) {
  if (family < 0 || family > 2 || K < 1 || off[0] != 0 || off[K] != n) return -1;
  for (int64_t k = 0; k < K; ++k)
    if (off[k + 1] - off[k] < 2) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > K) nthreads = (int)K;
  pthread_t* th = (pthread_t*)malloc((size_t)nthreads * sizeof(pthread_t));
  orc_job* jobs = (orc_job*)malloc((size_t)nthreads * sizeof(orc_job));
  for (int t = 0; t < nthreads; ++t) {
    orc_job J = {family, dtype, u, v, off, K, theta, var, info, status, iters, t, nthreads};
    jobs[t] = J;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
  orc_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  if (combined) *combined = orc_combine(theta, var, info, status, K, weight);
  return 0;
}
