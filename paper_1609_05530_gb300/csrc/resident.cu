// resident.cu -- the fused per-subset fit: one CTA owns one subset at a time
// and keeps it in shared memory from the rank transform to the variance.
//
// Per subset (rows [off, off+m), Eq. 14):
//   1. ranks of u and of v within the subset (Eq. 12), by a stable radix sort
//      of (value, row) in shared memory;
//   2. the pairing permutation pi: for the point of u-rank p+1, pi[p] is its
//      v-rank.  The subset's pseudo-observations are then exactly
//      ((p+1)/(m+1), pi[p]/(m+1)), p = 0..m-1, and every per-margin transform
//      depends on a rank only, so it is tabulated once per rank and shared by
//      both margins;
//   3. the maximiser of the pseudo log-likelihood (Eq. 13): Gaussian through
//      the sufficient statistics A, B and the roots of its score cubic;
//      Frank and Gumbel by a bisection-safeguarded Newton iteration, every
//      pass a block-wide reduction of the score and Hessian (the FP64 path
//      starts it at the root of the same search in FP32);
//   4. the sandwich variance of Genest, Ghoudi & Rivest (1995) (Section 2.3):
//      l_tu summed over u-ranks >= p (a running suffix over each thread's run
//      of u-ranks) and l_tv over v-ranks >= pi[p] (scatter to pi[p]-1 and a
//      block scan) give W1, W2; sigma^2 = var(l_t + W1 + W2) / beta^2,
//      beta = -mean l_tt, and Var(theta_hat) = sigma^2 / m, the sigma_m^2 of
//      Eq. 15;
//   5. the subset is counted for its dataset, and the block that finishes a
//      dataset's last subset computes the dataset's Eq. 15.
#include "block_sort.cuh"
#include "families.cuh"
#include "fit_common.cuh"
#include "internal.h"

namespace cop {

// ---------------------------------------------------------------------------
// Per-rank tables.
// ---------------------------------------------------------------------------

// tab[r] = exp(-at (r+1)/(m+1)), r = 0..m-1 (Frank: a = e^{-theta u} for every
// possible u).  The float table takes the exponent slope c = -at log2(e)/(m+1)
// split into an FP32 head chi and tail clo, and forms r c as an FP32 product
// plus its exact FMA remainder, so each entry is good to a few ulp for any
// theta up to the cap.  The double table takes c = -at/(m+1).
template <int BLOCK>
__device__ __forceinline__ void exp_table(float* tab, int m, float chi, float clo) {
  for (int r = threadIdx.x; r < m; r += BLOCK) {
    const float rr = (float)(r + 1);
    const float p = rr * chi;
    const float e = fmaf(rr, chi, -p);
    const float t = fmaf(rr, clo, e);
    tab[r] = ex2_approx(p) * fmaf(t, 0.693147180559945309f, 1.0f);
  }
}
template <int BLOCK>
__device__ __forceinline__ void exp_table(double* tab, int m, double c) {
  for (int r = threadIdx.x; r < m; r += BLOCK) tab[r] = ::exp(c * (double)(r + 1));
}

// tab[r] = Phi^{-1}((r+1)/(m+1)).  The lower half is evaluated and the
// upper half mirrored, tab[m-1-r] = -tab[r] (Phi^{-1}(1-q) = -Phi^{-1}(q), and
// (m-r)/(m+1) is the exact complement of (r+1)/(m+1)).
template <int BLOCK>
__device__ __forceinline__ void normal_score_table(float* tab, int m) {
  const float inv = 1.0f / (float)(m + 1);
  const int h = (m + 1) >> 1;
  for (int r = threadIdx.x; r < h; r += BLOCK) {
    const float x = normcdfinvf((float)(r + 1) * inv);
    tab[r] = x;
    if (m - 1 - r != r) tab[m - 1 - r] = -x;
  }
}
template <int BLOCK>
__device__ __forceinline__ void normal_score_table(double* tab, int m) {
  const double inv = 1.0 / (double)(m + 1);
  const int h = (m + 1) >> 1;
  for (int r = threadIdx.x; r < h; r += BLOCK) {
    const double x = normcdfinv((double)(r + 1) * inv);
    tab[r] = x;
    if (m - 1 - r != r) tab[m - 1 - r] = -x;
  }
}

// tab[r] = log(-log((r+1)/(m+1))); -log u near u = 1 comes from log1p of the
// exact complement (m-r)/(m+1).
template <int BLOCK>
__device__ __forceinline__ void gumbel_table(float* tab, int m) {
  const float inv = 1.0f / (float)(m + 1);
  for (int r = threadIdx.x; r < m; r += BLOCK) {
    float x;
    if (2 * (r + 1) <= m + 1)
      x = -logf((float)(r + 1) * inv);
    else
      x = -log1pf(-(float)(m - r) * inv);
    tab[r] = logf(x);
  }
}
template <int BLOCK>
__device__ __forceinline__ void gumbel_table(double* tab, int m) {
  const double inv = 1.0 / (double)(m + 1);
  for (int r = threadIdx.x; r < m; r += BLOCK) {
    double x;
    if (2 * (r + 1) <= m + 1)
      x = -::log((double)(r + 1) * inv);
    else
      x = -::log1p(-(double)(m - r) * inv);
    tab[r] = ::log(x);
  }
}

// ---------------------------------------------------------------------------
// Shared per-CTA scratch.
// ---------------------------------------------------------------------------
struct CtaShared {
  double red[4 * 32 + 8];
  double bc[8];  // FP64 scalars broadcast by thread 0 / single lanes
  float bf[8];   // FP32 scalars broadcast by thread 0
  uint32_t scan[40];
  int job;
  int flag;
};
// bc slots: 0 theta, 1 per-pass FP64 constant (Frank -at/(m+1), Gumbel 1/theta),
// 2..5 Frank E, k0, k1, k2 (FP64 path), 6 1/m, 7 1/(m+1).  bf slots: 0, 1
// Frank exp-table slope head / tail, 2 mean of xi (variance).

struct SubsetView {
  int m;
  const uint16_t* pi;  // v-rank of the point of u-rank p+1
  long long S;         // sum (p+1) pi[p]
  int subset;
};

template <typename Real>
struct Bufs {
  Real* tab;  // per-rank table, m
  Real* wv;   // v-order scan array of the variance (then xi), m
  Real* gs;   // the variance's per-point store, var_store_entries(m, BLOCK, sizeof(Real)), or null
};

// Profiling stamps (GPU global timer, ns) per subset: 0 start, 1 ranks done,
// 2 parameter search done, 3 end.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void stamp(const ResidentArgs& A, int subset, int which) {
  if (A.phase_ns != nullptr && threadIdx.x == 0) A.phase_ns[4 * (size_t)subset + which] = global_ns();
}

// Sandwich variance (Section 2.3; Genest, Ghoudi & Rivest 1995) from the
// per-point terms (l_t, l_tt, l_tu, l_tv): for the point p of u-rank p+1,
//   xi_p = l_t(p) + (1/m) [ sum_{u-rank(q) >= p+1} l_tu(q) + sum_{v-rank(q) >= v-rank(p)} l_tv(q) ],
//   var = mean((xi - mean xi)^2) / beta^2 / m,  beta = -mean(l_tt).
// terms(p) returns Terms<Real> for point p; with MARGIN its l_tu and l_tv
// lack the margin factor of their rank and margin(q) gives that of rank q+1.
// Thread t takes the u-ranks of one run [t C, t C + C): the u-side sum is a
// running suffix over its own run plus the run totals of the threads after
// it, so no u-order array is kept.  The v-side sums are a block scan of the
// v-order array wv; point p reads entry v-rank(p)-1, its own, once, and then
// leaves xi_p there for the second moment.  B.gs, when not null, keeps each
// point's l_t and margin-scaled l_tu between the two sweeps (2 C BLOCK
// entries, run position j of thread t at j BLOCK + t); when null they are
// evaluated again; in FP64 the store also keeps the margin factor of the
// rank, which the v-side scan of the same run uses again.  var and info are
// valid in thread 0 only.
template <int BLOCK, typename Real, bool MARGIN, typename TermsFn, typename MarginFn>
__device__ void sandwich_variance(const SubsetView& S, const Bufs<Real>& B, CtaShared& sh, TermsFn terms,
                                  MarginFn margin, double& var, double& info) {
  const int m = S.m;
  const int C = run_length<BLOCK>(m);
  const int t = threadIdx.x;
  const int beg = min(m, t * C), end = min(m, beg + C);
  Real* gs = B.gs;
  Acc<Real> hacc[1], su, sv;
  constexpr bool kKeepMargin = MARGIN && sizeof(Real) == 8;
  for (int p = beg; p < end; ++p) {
    const Terms<Real> x = terms(p);
    Real gu = x.gu;
    if constexpr (MARGIN) {
      const Real f = margin(p);
      gu *= f;
      if (kKeepMargin && gs) gs[(2 * C + p - beg) * BLOCK + t] = f;
    }
    B.wv[S.pi[p] - 1] = x.gv;
    hacc[0].add(x.h);
    su.add(gu);
    if (gs) {
      gs[(p - beg) * BLOCK + t] = x.g;
      gs[(C + p - beg) * BLOCK + t] = gu;
    }
  }
  double hsum[1];
  block_reduce<BLOCK, Real, 1>(hacc, sh.red, hsum);  // contains __syncthreads: wv complete
  // v-side: margin factors (ranks of this thread's run, as above), run totals
  for (int q = beg; q < end; ++q) {
    Real w = B.wv[q];
    if constexpr (MARGIN) {
      w *= (kKeepMargin && gs) ? gs[(2 * C + q - beg) * BLOCK + t] : margin(q);
      B.wv[q] = w;
    }
    sv.add(w);
  }
  block_excl_suffix2<BLOCK>(su, sv, sh.red);  // now the totals of the runs after this one
  for (int q = end - 1; q >= beg; --q) {
    sv.add(B.wv[q]);
    B.wv[q] = sv.value_real();
  }
  __syncthreads();
  const Real im = (Real)sh.bc[6];
  Acc<Real> a1[1];
  for (int p = end - 1; p >= beg; --p) {
    Real g, gu;
    if (gs) {
      g = gs[(p - beg) * BLOCK + t];
      gu = gs[(C + p - beg) * BLOCK + t];
    } else {
      const Terms<Real> x = terms(p);
      g = x.g;
      gu = x.gu;
      if constexpr (MARGIN) gu *= margin(p);
    }
    su.add(gu);
    const int vi = S.pi[p] - 1;
    const Real xi = g + (su.value_real() + B.wv[vi]) * im;
    B.wv[vi] = xi;
    a1[0].add(xi);
  }
  double xsum[1];
  block_reduce<BLOCK, Real, 1>(a1, sh.red, xsum);
  if (threadIdx.x == 0) sh.bc[0] = xsum[0] * sh.bc[6];  // mean of xi (theta is no longer needed)
  __syncthreads();
  const Real mean = (Real)sh.bc[0];
  Acc<Real> a2[1];
  for (int q = threadIdx.x; q < m; q += BLOCK) {
    const Real d = B.wv[q] - mean;
    a2[0].add(d * d);
  }
  double dsum[1];
  block_reduce<BLOCK, Real, 1>(a2, sh.red, dsum);
  if (threadIdx.x == 0) {
    const double nu2 = dsum[0] * sh.bc[6];
    const double beta = -hsum[0] * sh.bc[6];
    var = nu2 / (beta * beta) * sh.bc[6];
    info = -hsum[0];
  }
}

// Newton search on thread 0's driver nt (initialised by the caller):
// pass(th, out) computes, on all threads, the score and Hessian of Eq. 13 at
// th into thread 0's out[1], out[2]; prep(th), on thread 0, publishes what
// the next pass needs besides th (sh.bc[0]).
template <typename PassFn, typename PrepFn>
__device__ void newton_loop(Newton& nt, CtaShared& sh, PassFn pass, PrepFn prep) {
  if (threadIdx.x == 0) {
    sh.bc[0] = nt.th;
    prep(nt.th);
    sh.flag = 0;
  }
  __syncthreads();
  for (;;) {
    const double th = sh.bc[0];
    double out[3];
    pass(th, out);
    if (threadIdx.x == 0) {
      nt.step(out[1], out[2]);
      sh.bc[0] = nt.th;
      prep(nt.th);
      sh.flag = nt.done ? 1 : 0;
    }
    __syncthreads();
    if (sh.flag) break;
  }
  __syncthreads();  // every thread has read sh.flag before thread 0 may set it again
}

template <int BLOCK, typename Real>
__device__ void fit_gaussian(const ResidentArgs& A, const SubsetView& S, const Bufs<Real>& B, CtaShared& sh) {
  const int m = S.m;
  normal_score_table<BLOCK>(B.tab, m);
  __syncthreads();
  Acc<Real> acc[2];
  for (int p = threadIdx.x; p < m; p += BLOCK) {
    const Real x = B.tab[p];
    acc[0].add(x * x);
    acc[1].add(x * B.tab[S.pi[p] - 1]);
  }
  double s[2];
  block_reduce<BLOCK, Real, 2>(acc, sh.red, s);
  if (A.mode == MODE_LOGLIK) {
    if (threadIdx.x == 0) {
      const double Asum = 2.0 * s[0], Bsum = s[1], md = (double)m;
      const double r = A.theta_in[S.subset], om = 1.0 - r * r;
      if (A.l_out) A.l_out[S.subset] = gauss_l(md, Asum, Bsum, r);
      if (A.g_out) A.g_out[S.subset] = md * r / om - (r * Asum - Bsum * (1.0 + r * r)) / (om * om);
      if (A.h_out)
        A.h_out[S.subset] = md * (1.0 + r * r) / (om * om) -
                            (Asum * (1.0 + 3.0 * r * r) - 2.0 * Bsum * r * (3.0 + r * r)) / (om * om * om);
    }
    return;
  }
  if (threadIdx.x == 0) {
    int st;
    sh.bc[1] = gaussian_mpl((double)m, 2.0 * s[0], s[1], st);
    sh.flag = st;
  }
  __syncthreads();
  stamp(A, S.subset, 2);
  const double rho = sh.bc[1];
  const int st = sh.flag;
  const Real r = (Real)rho;
  double var = 0.0, info = 0.0;
  sandwich_variance<BLOCK, Real, true>(
      S, B, sh, [&](int p) { return gaussian_terms<Real>(r, B.tab[p], B.tab[S.pi[p] - 1]); },
      [&](int q) { return gaussian_margin<Real>(B.tab[q]); }, var, info);
  if (threadIdx.x == 0) {
    A.theta[S.subset] = rho;
    A.var[S.subset] = var;
    A.status[S.subset] = st;
    A.info[S.subset] = info;
    A.iters[S.subset] = 0;
  }
}

// ---------------------------------------------------------------------------
// Frank.
// ---------------------------------------------------------------------------
// Thread 0: constants the next Frank pass needs before its table is built.
__device__ __forceinline__ void frank_prepare(CtaShared& sh, double th) {
  const double at = fabs(th);
  const double c = -at * kLog2e * sh.bc[7];
  const float chi = (float)c;
  sh.bf[0] = chi;
  sh.bf[1] = (float)(c - (double)chi);
  sh.bc[1] = -at * sh.bc[7];
}

// One likelihood pass at theta (sh.bc[0]): the data-dependent sums
// (sum l, sum l_t, sum l_tt) without the per-subset constants in raw[], and
// for thread 0 the totals in out[].
template <int BLOCK, typename Real, bool WANT_L>
__device__ void frank_pass(const SubsetView& S, const Bufs<Real>& B, CtaShared& sh, double th, double (&out)[3]) {
  const int m = S.m;
  const Real inv = Real(1) / (Real)(m + 1);
  Acc<Real> acc[3];
  const double at = fabs(th);
  if (at < FrankSeries<Real>::cut) {
    const Real t = (Real)th;
    for (int p = threadIdx.x; p < m; p += BLOCK) {
      Real l = 0;
      const Terms<Real> x = frank_series_terms<Real>(t, (Real)(p + 1) * inv, (Real)S.pi[p] * inv, WANT_L ? &l : nullptr);
      acc[0].add(l);
      acc[1].add(x.g);
      acc[2].add(x.h);
    }
    block_reduce<BLOCK, Real, 3>(acc, sh.red, out);
    return;
  }
  const bool flip = th < 0.0;
  {
    // The per-subset constants come from single lanes, in parallel with the
    // table build; the barrier below publishes them.  FP64 path: from FP64
    // lanes of three warps; FP32C path: from one lane in FP32 (see
    // frank_consts_f32).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(Real) == 4) {
      if (lane == 0 && warp == 1) {
        const FrankConsts c = frank_consts_f32(at);
        sh.bc[2] = c.E;
        sh.bc[4] = c.k1;
        sh.bc[5] = c.k2;
        if (WANT_L) sh.bc[3] = c.k0;
      }
    } else {
      if (lane == 0 && warp == 1) sh.bc[2] = ::exp(-at);
      if (lane == 0 && warp == 2) {
        const double em1 = ::expm1(at);
        sh.bc[4] = 1.0 / at + 1.0 / em1;
        sh.bc[5] = -1.0 / (at * at) - (em1 + 1.0) / (em1 * em1);
      }
      if (WANT_L && lane == 0 && warp == 3) sh.bc[3] = ::log(-at * ::expm1(-at));
    }
  }
  if constexpr (sizeof(Real) == 4)
    exp_table<BLOCK>(B.tab, m, sh.bf[0], sh.bf[1]);
  else
    exp_table<BLOCK>(B.tab, m, sh.bc[1]);
  __syncthreads();
  const Real E = (Real)sh.bc[2];
  const Real atr = (Real)at;
  for (int p = threadIdx.x; p < m; p += BLOCK) {
    const int vr = flip ? m + 1 - (int)S.pi[p] : (int)S.pi[p];
    const Real u = (Real)(p + 1) * inv, v = (Real)vr * inv;
    const Real a = B.tab[p], b = B.tab[vr - 1], bc = B.tab[m - vr];
    const FrankPoint<Real> f = frank_point<Real>(u, v, a, b, bc, E);
    const Real iD = Fn<Real>::rcp(f.D);
    const Real q1 = f.D1 * iD;
    if (WANT_L) acc[0].add(-atr * (u + v) - Real(2) * Fn<Real>::log(f.D));
    acc[1].add(-(u + v) - Real(2) * q1);
    acc[2].add(Real(-2) * (f.D2 * iD - q1 * q1));
  }
  double s[3];
  block_reduce<BLOCK, Real, 3>(acc, sh.red, s);
  if (threadIdx.x == 0) {
    const double md = (double)m;
    out[0] = md * (WANT_L ? sh.bc[3] : 0.0) + s[0];
    out[1] = (md * sh.bc[4] + s[1]) * (flip ? -1.0 : 1.0);
    out[2] = md * sh.bc[5] + s[2];
  }
}

template <int BLOCK, typename Real>
__device__ void fit_frank(const ResidentArgs& A, const SubsetView& S, const Bufs<Real>& B, CtaShared& sh) {
  const int m = S.m;
  if (A.mode == MODE_LOGLIK) {
    if (threadIdx.x == 0) frank_prepare(sh, A.theta_in[S.subset]);
    __syncthreads();
    double out[3];
    frank_pass<BLOCK, Real, true>(S, B, sh, A.theta_in[S.subset], out);
    if (threadIdx.x == 0) {
      if (A.l_out) A.l_out[S.subset] = out[0];
      if (A.g_out) A.g_out[S.subset] = out[1];
      if (A.h_out) A.h_out[S.subset] = out[2];
    }
    return;
  }
  Newton nt;
  double th0 = 0.0;
  int pre_it = 0;
  bool from_root = false;
  if (threadIdx.x == 0) {
    const float rs = spearman_rho((double)S.S, m);
    th0 = start_from_rho(A.start.frank_rho, kFrankStart0, kFrankStartStep, fabsf(rs));
    if (rs < 0.0f) th0 = -th0;
  }
  if constexpr (sizeof(Real) == 8) {
    // FP32 start search; its exp table takes the first m floats of tab
    const Bufs<float> Bf{reinterpret_cast<float*>(B.tab), nullptr, nullptr};
    if (threadIdx.x == 0) nt.init(th0, -kFrankCap, kFrankCap, kPresolveRtol, A.max_iter, false);
    newton_loop(
        nt, sh, [&](double th, double(&out)[3]) { frank_pass<BLOCK, float, false>(S, Bf, sh, th, out); },
        [&](double th) { frank_prepare(sh, th); });
    if (threadIdx.x == 0) {
      pre_it = nt.it;
      from_root = nt.status == ST_OK;
      if (from_root) th0 = nt.th;
    }
  }
  if (threadIdx.x == 0) nt.init(th0, -kFrankCap, kFrankCap, A.rtol, A.max_iter, false, !from_root);
  newton_loop(
      nt, sh, [&](double th, double(&out)[3]) { frank_pass<BLOCK, Real, false>(S, B, sh, th, out); },
      [&](double th) { frank_prepare(sh, th); });
  stamp(A, S.subset, 2);
  const double th = sh.bc[0];
  const double at = fabs(th);
  const bool flip = th < 0.0;
  const Real inv = Real(1) / (Real)(m + 1);
  double var = 0.0, info = 0.0;
  if (at < FrankSeries<Real>::cut) {
    const Real t = (Real)th;
    sandwich_variance<BLOCK, Real, false>(
        S, B, sh,
        [&](int p) { return frank_series_terms<Real>(t, (Real)(p + 1) * inv, (Real)S.pi[p] * inv, nullptr); },
        NoScale(), var, info);
  } else {
    if (threadIdx.x == 0) {
      const FrankConsts c = sizeof(Real) == 4 ? frank_consts_f32(at) : frank_consts_f64(at);
      sh.bc[2] = c.E;
      sh.bc[4] = c.k1;
      sh.bc[5] = c.k2;
    }
    if constexpr (sizeof(Real) == 4)
      exp_table<BLOCK>(B.tab, m, sh.bf[0], sh.bf[1]);
    else
      exp_table<BLOCK>(B.tab, m, sh.bc[1]);
    __syncthreads();
    const Real E = (Real)sh.bc[2], k1 = (Real)sh.bc[4], k2 = (Real)sh.bc[5], atr = (Real)at;
    sandwich_variance<BLOCK, Real, false>(
        S, B, sh,
        [&](int p) {
          const int vr = flip ? m + 1 - (int)S.pi[p] : (int)S.pi[p];
          const Real u = (Real)(p + 1) * inv, v = (Real)vr * inv;
          const Real a = B.tab[p], b = B.tab[vr - 1], bc = B.tab[m - vr];
          const FrankPoint<Real> f = frank_point<Real>(u, v, a, b, bc, E);
          Terms<Real> t = frank_terms<Real>(atr, k1, k2, u, v, a, b, f);
          if (flip) {  // c(u, v; -theta) = c(u, 1 - v; theta)
            t.g = -t.g;
            t.gu = -t.gu;
          }
          return t;
        },
        NoScale(), var, info);
  }
  if (threadIdx.x == 0) {
    A.theta[S.subset] = th;
    A.var[S.subset] = var;
    A.status[S.subset] = nt.status;
    A.info[S.subset] = info;
    A.iters[S.subset] = pre_it + nt.it;
  }
}

// ---------------------------------------------------------------------------
// Gumbel.
// ---------------------------------------------------------------------------
template <int BLOCK, typename Real, bool WANT_L>
__device__ void gumbel_pass(const SubsetView& S, const Bufs<Real>& B, CtaShared& sh, double th, double (&out)[3]) {
  const int m = S.m;
  const Real t = (Real)th;
  Real it;
  if constexpr (sizeof(Real) == 4)
    it = 1.0f / (float)th;
  else
    it = sh.bc[1];  // 1/theta from thread 0
  Acc<Real> acc[3];
  for (int p = threadIdx.x; p < m; p += BLOCK) {
    const GumbelPoint<Real> q = gumbel_point<Real, WANT_L>(t, it, B.tab[p], B.tab[S.pi[p] - 1]);
    acc[0].add(q.l);
    acc[1].add(q.g);
    acc[2].add(q.h);
  }
  block_reduce<BLOCK, Real, 3>(acc, sh.red, out);
}

template <int BLOCK, typename Real>
__device__ void fit_gumbel(const ResidentArgs& A, const SubsetView& S, const Bufs<Real>& B, CtaShared& sh) {
  const int m = S.m;
  if (A.mode == MODE_LOGLIK) {
    gumbel_table<BLOCK>(B.tab, m);
    if (threadIdx.x == 0) sh.bc[1] = 1.0 / A.theta_in[S.subset];
    __syncthreads();
    double out[3];
    gumbel_pass<BLOCK, Real, true>(S, B, sh, A.theta_in[S.subset], out);
    if (threadIdx.x == 0) {
      if (A.l_out) A.l_out[S.subset] = out[0];
      if (A.g_out) A.g_out[S.subset] = out[1];
      if (A.h_out) A.h_out[S.subset] = out[2];
    }
    return;
  }
  Newton nt;
  double th0 = 0.0;
  int pre_it = 0;
  bool from_root = false;
  if (threadIdx.x == 0) {
    const float rs = spearman_rho((double)S.S, m);
    th0 = start_from_rho(A.start.gumbel_rho, kGumbelStart0, kGumbelStartStep, rs);
  }
  if constexpr (sizeof(Real) == 8) {
    // FP32 start search on an FP32 table in the (not yet used) wv array
    const Bufs<float> Bf{reinterpret_cast<float*>(B.wv), nullptr, nullptr};
    gumbel_table<BLOCK>(Bf.tab, m);
    if (threadIdx.x == 0) nt.init(th0, 1.0, kGumbelCap, kPresolveRtol, A.max_iter, true);
    newton_loop(
        nt, sh, [&](double th, double(&out)[3]) { gumbel_pass<BLOCK, float, false>(S, Bf, sh, th, out); },
        [](double) {});
    if (threadIdx.x == 0) {
      pre_it = nt.it;
      from_root = nt.status == ST_OK;
      if (from_root) th0 = nt.th;
    }
  }
  gumbel_table<BLOCK>(B.tab, m);
  if (threadIdx.x == 0) nt.init(th0, 1.0, kGumbelCap, A.rtol, A.max_iter, true, !from_root);
  newton_loop(
      nt, sh, [&](double th, double(&out)[3]) { gumbel_pass<BLOCK, Real, false>(S, B, sh, th, out); },
      [&](double th) {
        if constexpr (sizeof(Real) == 8) sh.bc[1] = 1.0 / th;  // the FP32 passes form 1/theta themselves
      });
  stamp(A, S.subset, 2);
  const double th = sh.bc[0];
  const Real t = (Real)th, mp1 = (Real)(m + 1);
  Real it;
  if constexpr (sizeof(Real) == 4)
    it = 1.0f / t;
  else
    it = sh.bc[1];
  double var = 0.0, info = 0.0;
  sandwich_variance<BLOCK, Real, true>(
      S, B, sh,
      [&](int p) {
        const Real lx = B.tab[p], ly = B.tab[S.pi[p] - 1];
        const GumbelPoint<Real> q = gumbel_point<Real, false>(t, it, lx, ly);
        Terms<Real> r;
        r.g = q.g;
        r.h = q.h;
        gumbel_mixed<Real>(t, lx, ly, q, r.gu, r.gv);
        return r;
      },
      [&](int q) { return gumbel_margin<Real>(B.tab[q], mp1, (Real)(q + 1)); }, var, info);
  if (threadIdx.x == 0) {
    A.theta[S.subset] = th;
    A.var[S.subset] = var;
    A.status[S.subset] = nt.status;
    A.info[S.subset] = info;
    A.iters[S.subset] = pre_it + nt.it;
  }
}

// A job's estimates are stored (by thread 0, before a __syncthreads): count
// it for its dataset, and the block that finishes a dataset's last subset
// computes the dataset's Eq. 15 with its first warp.
template <int BLOCK>
__device__ void finish_job(const ResidentArgs& A, const Job& job, CtaShared& sh) {
  if (!A.comb) return;
  if (threadIdx.x == 0) sh.flag = dataset_finished(A.ds_done, A.dss, job.dataset) ? 1 : 0;
  __syncthreads();
  if (sh.flag && threadIdx.x < 32)
    combine_dataset(A.theta, A.var, A.info, A.status, A.dss, A.weight, job.dataset, A.comb);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <typename Real, typename KeyT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) resident_kernel(const __grid_constant__ ResidentArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaShared sh;
  using Val = typename KeyOf<KeyT>::Val;
  for (;;) {
    if (threadIdx.x == 0) sh.job = atomicAdd(A.counter, 1);
    __syncthreads();
    const int j = sh.job;
    __syncthreads();
    if (j >= A.njobs) return;
    const Job job = A.jobs[j];
    const int m = job.m;
    // The jobs leave the counter in order, so while the grid fits jobs
    // j - gridDim.x ... j the next ones taken are about j + gridDim.x: this
    // CTA asks the L2 for that job's two columns meanwhile (whichever CTA
    // takes it), so that key loads do not wait on HBM (or, for inputs in
    // mapped host memory, on the host link).
    const int ahead = j + (int)gridDim.x;
    if (ahead < A.njobs) {
      const Job nj = A.jobs[ahead];
      const char* pu = reinterpret_cast<const char*>(A.u) + (size_t)nj.off * sizeof(Val);
      const char* pv = reinterpret_cast<const char*>(A.v) + (size_t)nj.off * sizeof(Val);
      const size_t bytes = (size_t)nj.m * sizeof(Val);
      for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)BLOCK * 128) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pu + o));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pv + o));
      }
    }
    stamp(A, job.subset, 0);
    const ResLayout L = res_layout(m, (int)sizeof(KeyT), (int)sizeof(Real), A.tab_in_smem != 0,
                                   job.gs_mode == 1, BLOCK);
    KeyT* keys = reinterpret_cast<KeyT*>(smem);
    uint16_t* ib0 = reinterpret_cast<uint16_t*>(smem + (size_t)m * sizeof(KeyT));
    uint16_t* ib1 = ib0 + m;
    uint16_t* pi = reinterpret_cast<uint16_t*>(smem + L.pi_off);
    SortCnt* cnt = reinterpret_cast<SortCnt*>(smem + L.cnt_off);

    // Eq. 12: ranks of u within the subset
    const Val* xu = reinterpret_cast<const Val*>(A.u) + job.off;
    const Val* xv = reinterpret_cast<const Val*>(A.v) + job.off;
    KeyRange range;
    bool nan = load_keys<BLOCK, KeyT>(xu, m, keys, sh.scan, &range);
    if (!nan) {
      const uint16_t* perm = block_rank_perm<BLOCK, KeyT>(keys, m, ib0, ib1, cnt, sh.scan, range);
      for (int p = threadIdx.x; p < m; p += BLOCK) pi[p] = perm[p];  // perm_u
      __syncthreads();
      nan = load_keys<BLOCK, KeyT>(xv, m, keys, sh.scan, &range);
    }
    if (nan) {
      if (threadIdx.x == 0) {
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        if (A.mode == MODE_FIT) {
          A.theta[job.subset] = qnan;
          A.var[job.subset] = qnan;
          A.status[job.subset] = ST_DEGENERATE;
          A.info[job.subset] = qnan;
          A.iters[job.subset] = 0;
        } else {
          if (A.l_out) A.l_out[job.subset] = qnan;
          if (A.g_out) A.g_out[job.subset] = qnan;
          if (A.h_out) A.h_out[job.subset] = qnan;
        }
      }
      __syncthreads();
      finish_job<BLOCK>(A, job, sh);
      continue;
    }
    // ranks of v, then pi[p] = v-rank of the point with u-rank p+1
    const uint16_t* permv = block_rank_perm<BLOCK, KeyT>(keys, m, ib0, ib1, cnt, sh.scan, range);
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
    Ssum = block_sum_i64<BLOCK>(Ssum, sh.red);
    stamp(A, job.subset, 1);

    if (threadIdx.x == 0) {
      sh.bc[6] = recip64((double)m);
      sh.bc[7] = recip64((double)(m + 1));
    }
    __syncthreads();
    SubsetView S{m, pi, Ssum, job.subset};
    Bufs<Real> B;
    char* region = A.gws ? A.gws + (size_t)blockIdx.x * (size_t)A.gws_stride : nullptr;
    B.tab = A.tab_in_smem ? reinterpret_cast<Real*>(smem) : reinterpret_cast<Real*>(region);
    B.wv = B.tab + m;
    if (job.gs_mode == 1)
      B.gs = reinterpret_cast<Real*>(smem + (A.tab_in_smem ? 2 * (size_t)m * sizeof(Real) : 0));
    else if (job.gs_mode == 2)
      B.gs = reinterpret_cast<Real*>(region + A.gws_gs_off);
    else
      B.gs = nullptr;
    if (job.family == 0)
      fit_gaussian<BLOCK, Real>(A, S, B, sh);
    else if (job.family == 1)
      fit_frank<BLOCK, Real>(A, S, B, sh);
    else
      fit_gumbel<BLOCK, Real>(A, S, B, sh);
    __syncthreads();
    finish_job<BLOCK>(A, job, sh);
    stamp(A, job.subset, 3);
  }
}

// Ranks alone (Eq. 12 per subset), one column.
template <typename KeyT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) ranks_kernel(const void* __restrict__ x, const Job* __restrict__ jobs,
                                                         int njobs, int32_t* counter, int32_t* __restrict__ ranks) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t scan[40];
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
    KeyT* keys = reinterpret_cast<KeyT*>(smem);
    uint16_t* ib0 = reinterpret_cast<uint16_t*>(smem + (size_t)m * sizeof(KeyT));
    uint16_t* ib1 = ib0 + m;
    const ResLayout L = res_layout(m, (int)sizeof(KeyT), 4, false, false, BLOCK);
    SortCnt* cnt = reinterpret_cast<SortCnt*>(smem + L.cnt_off);
    KeyRange range;
    const bool nan = load_keys<BLOCK, KeyT>(reinterpret_cast<const Val*>(x) + job.off, m, keys, scan, &range);
    int32_t* out = ranks + job.off;
    if (nan) {
      for (int i = threadIdx.x; i < m; i += BLOCK) out[i] = 0;
    } else {
      const uint16_t* perm = block_rank_perm<BLOCK, KeyT>(keys, m, ib0, ib1, cnt, scan, range);
      for (int pos = threadIdx.x; pos < m; pos += BLOCK) out[perm[pos]] = pos + 1;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename Real, typename KeyT, int BLOCK>
static cudaError_t launch_res_t(int grid, size_t smem, const ResidentArgs& a, cudaStream_t s) {
  static std::atomic<int> granted[64] = {};
  auto k = resident_kernel<Real, KeyT, BLOCK>;
  cudaError_t e = ensure_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<grid, BLOCK, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, typename KeyT>
static cudaError_t launch_res_b(int block, int grid, size_t smem, const ResidentArgs& a, cudaStream_t s) {
  switch (block) {
    case 128: return launch_res_t<Real, KeyT, 128>(grid, smem, a, s);
    case 256: return launch_res_t<Real, KeyT, 256>(grid, smem, a, s);
    case 512: return launch_res_t<Real, KeyT, 512>(grid, smem, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_resident(int prec, int key_bytes, int block, int grid, size_t smem, const ResidentArgs& a,
                            cudaStream_t s) {
  if (prec == 1) {
    return key_bytes == 4 ? launch_res_b<float, uint32_t>(block, grid, smem, a, s)
                          : launch_res_b<float, uint64_t>(block, grid, smem, a, s);
  }
  return key_bytes == 4 ? launch_res_b<double, uint32_t>(block, grid, smem, a, s)
                        : launch_res_b<double, uint64_t>(block, grid, smem, a, s);
}

template <typename KeyT, int BLOCK>
static cudaError_t launch_ranks_t(int grid, size_t smem, const void* x, const Job* jobs, int njobs,
                                  int32_t* counter, int32_t* ranks, cudaStream_t s) {
  static std::atomic<int> granted[64] = {};
  auto k = ranks_kernel<KeyT, BLOCK>;
  cudaError_t e = ensure_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<grid, BLOCK, smem, s>>>(x, jobs, njobs, counter, ranks);
  return cudaGetLastError();
}

cudaError_t launch_ranks(int key_bytes, int block, int grid, size_t smem, const void* x, const Job* jobs,
                         int njobs, int32_t* counter, int32_t* ranks, cudaStream_t s) {
  if (key_bytes == 4) {
    switch (block) {
      case 128: return launch_ranks_t<uint32_t, 128>(grid, smem, x, jobs, njobs, counter, ranks, s);
      case 256: return launch_ranks_t<uint32_t, 256>(grid, smem, x, jobs, njobs, counter, ranks, s);
      case 512: return launch_ranks_t<uint32_t, 512>(grid, smem, x, jobs, njobs, counter, ranks, s);
    }
  } else {
    switch (block) {
      case 128: return launch_ranks_t<uint64_t, 128>(grid, smem, x, jobs, njobs, counter, ranks, s);
      case 256: return launch_ranks_t<uint64_t, 256>(grid, smem, x, jobs, njobs, counter, ranks, s);
      case 512: return launch_ranks_t<uint64_t, 512>(grid, smem, x, jobs, njobs, counter, ranks, s);
    }
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Eq. 15 as a kernel of its own (copula_fit_noalloc; the fit paths compute it
// in their last block instead): per dataset, sum w theta / sum w over its
// subsets, FP64.  One warp per dataset; lanes stride over the subsets in
// order and the lane partials are combined in a fixed tree.  Only subsets with an interior maximiser or
// one on the family's own edge (status OK or BOUNDARY) take part: a
// maximiser on a search cap, an unconverged one or a NaN subset has no
// asymptotic variance to weight it by.
// ---------------------------------------------------------------------------
__global__ void combine_kernel(const CombineArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= a.B) return;
  combine_dataset(a.theta, a.var, a.info, a.status, a.dataset_subset_start, a.weight, warp, a.out);
}

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t s) {
  if (a.B <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (a.B * 32 + threads - 1) / threads;
  combine_kernel<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cop
