"""Writes frank_series.h: the Taylor coefficients of the Frank copula's
log-density about theta = 0 (the independence copula), used by the kernels
for small |theta| where the closed form of Eq. 10's density cancels.

log c(u, v; theta) = sum_{k=1..10} c_k theta^k with
  c_k = R_k(P, Q)            for even k,
  c_k = s * R_k(P, Q)        for odd k,
P = u(1-u), Q = v(1-v), s = (1-2u)(1-2v), R_k a polynomial with rational
coefficients.  Derived with sympy from
  log c = log((1 - e^-t)/t) - t(u+v) - 2 log(D/t),
  D = e^-tu + e^-tv - e^-t(u+v) - e^-t.
Run: python gen_frank_series.py  (needs sympy; takes ~20 s).
"""
import os

import sympy as sp

NTERMS = 10


def coefficients():
    t, u, v = sp.symbols("t u v")
    E, a, b = sp.exp(-t), sp.exp(-t * u), sp.exp(-t * v)
    N = NTERMS + 1
    Dhat = sp.series((a + b - a * b - E) / t, t, 0, N + 1).removeO()
    phi1 = sp.series((1 - E) / t, t, 0, N + 1).removeO()
    L = sp.expand(sp.series(sp.log(phi1), t, 0, N + 1).removeO() - t * (u + v)
                  - 2 * sp.series(sp.log(sp.expand(Dhat)), t, 0, N + 1).removeO())
    P, Q = sp.symbols("P Q")
    out = {}
    for k in range(1, NTERMS + 1):
        ck = sp.factor(L.coeff(t, k))
        deg = k // 2
        idx = [(i, j) for i in range(deg + 1) for j in range(deg + 1)]
        xs = sp.symbols(f"x0:{len(idx)}")
        base = 1 if k % 2 == 0 else (1 - 2 * u) * (1 - 2 * v)
        cand = base * sum(x * P ** i * Q ** j for x, (i, j) in zip(xs, idx))
        cand = cand.subs({P: u * (1 - u), Q: v * (1 - v)})
        sol = sp.solve(sp.Poly(sp.expand(cand - ck), u, v).coeffs(), xs, dict=True)[0]
        out[k] = {ij: sol.get(x, 0) for x, ij in zip(xs, idx)}
    return out


def _num(c):
    return f"Real({float(sp.Rational(c)):.17g})"


def main():
    co = coefficients()
    lines = ["// frank_series.h -- generated by gen_frank_series.py; do not edit.",
             "// Taylor coefficients of the Frank log-density about theta = 0:",
             "// R[k-1] = R_k(P, Q), RP = dR_k/dP, RQ = dR_k/dQ, with Pp[i] = P^i,",
             "// Qp[j] = Q^j; c_k = R_k (k even) or s R_k (k odd).",
             "#pragma once", "", "namespace cop {", "",
             f"constexpr int kFrankSeriesTerms = {NTERMS};", "",
             "template <typename Real>",
             "__device__ __forceinline__ void frank_series_poly(const Real* Pp, const Real* Qp, Real* R, Real* RP,",
             "                                                  Real* RQ) {"]
    for k in range(1, NTERMS + 1):
        terms, tp, tq = [], [], []
        for (i, j), c in sorted(co[k].items()):
            if c == 0:
                continue
            terms.append(f"{_num(c)} * Pp[{i}] * Qp[{j}]")
            if i:
                tp.append(f"{_num(i * c)} * Pp[{i - 1}] * Qp[{j}]")
            if j:
                tq.append(f"{_num(j * c)} * Pp[{i}] * Qp[{j - 1}]")
        lines.append(f"  R[{k - 1}] = " + (" + ".join(terms) if terms else "Real(0)") + ";")
        lines.append(f"  RP[{k - 1}] = " + (" + ".join(tp) if tp else "Real(0)") + ";")
        lines.append(f"  RQ[{k - 1}] = " + (" + ".join(tq) if tq else "Real(0)") + ";")
    lines += ["}", "", "}  // namespace cop", ""]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "frank_series.h")
    with open(path, "w") as f:
        f.write("\n".join(lines))
    print(path)


if __name__ == "__main__":
    main()
