// 1D rules and tables for the sum-factorised tensor-product basis B (Sec. 2.1 of
// arXiv 2402.15940: the basis action is applied dimension by dimension with 1D
// matrices).  Host code, long double, run once per operator.
//
//   gll_nodes(p)       Gauss-Lobatto-Legendre nodes of order p on [0,1]
//   gauss_rule(q)      Gauss-Legendre points/weights on [0,1] (weights sum to 1)
//   lagrange_tables    B[i][a] = phi_a(t_i), G[i][a] = phi_a'(t_i), barycentric form
#pragma once
#include <cmath>
#include <vector>

namespace fepa {
namespace basis {

// Legendre P_n(t) and P_n'(t) by the Bonnet recurrence.
inline void legendre(int n, long double t, long double* pn, long double* dpn) {
  long double p0 = 1.0L, p1 = t, dp0 = 0.0L, dp1 = 1.0L;
  if (n == 0) { *pn = 1.0L; *dpn = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    long double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
    long double dp2 = dp0 + (2 * k - 1) * p1;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2;
  }
  *pn = p1; *dpn = dp1;
}

// Gauss-Legendre rule with q points mapped to [0,1].
inline void gauss_rule(int q, std::vector<long double>& x, std::vector<long double>& w) {
  x.assign(q, 0.0L); w.assign(q, 0.0L);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < q; ++i) {
    long double t = -std::cos(pi * (i + 0.75L) / (q + 0.5L));  // ascending initial guesses
    for (int it = 0; it < 100; ++it) {
      long double pn, dpn;
      legendre(q, t, &pn, &dpn);
      long double dt = pn / dpn;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    long double pn, dpn;
    legendre(q, t, &pn, &dpn);
    x[i] = 0.5L * (t + 1.0L);
    w[i] = 1.0L / ((1.0L - t * t) * dpn * dpn);  // 2/((1-t^2)P'^2), halved for [0,1]
  }
}

// GLL nodes: endpoints and the zeros of P_p'.  Newton on P_p' with P_p'' taken from
// the Legendre equation (1-t^2)P'' = 2tP' - p(p+1)P.
inline std::vector<long double> gll_nodes(int p) {
  std::vector<long double> r(p + 1);
  r[0] = 0.0L; r[p] = 1.0L;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 1; i < p; ++i) {
    long double t = -std::cos(pi * i / p);
    for (int it = 0; it < 100; ++it) {
      long double pn, dpn;
      legendre(p, t, &pn, &dpn);
      long double d2 = (2.0L * t * dpn - p * (p + 1.0L) * pn) / (1.0L - t * t);
      long double dt = dpn / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    r[i] = 0.5L * (t + 1.0L);
  }
  return r;
}

// B[i*n + a] = phi_a(t_i), G[i*n + a] = phi_a'(t_i) for the Lagrange basis on `nodes`,
// through the barycentric weights lambda_a = 1/prod_{m!=a}(x_a - x_m).
inline void lagrange_tables(const std::vector<long double>& nodes, const std::vector<long double>& pts,
                            std::vector<double>& B, std::vector<double>& G) {
  const int n = (int)nodes.size(), q = (int)pts.size();
  std::vector<long double> lam(n, 1.0L);
  for (int a = 0; a < n; ++a)
    for (int m = 0; m < n; ++m)
      if (m != a) lam[a] /= (nodes[a] - nodes[m]);
  B.assign((size_t)q * n, 0.0); G.assign((size_t)q * n, 0.0);
  for (int i = 0; i < q; ++i) {
    const long double t = pts[i];
    int hit = -1;
    for (int a = 0; a < n; ++a)
      if (t == nodes[a]) hit = a;
    if (hit >= 0) {
      // t is a node: phi_a(t) = delta; derivative from the differentiation matrix
      long double diag = 0.0L;
      for (int a = 0; a < n; ++a) {
        B[i * n + a] = (a == hit) ? 1.0 : 0.0;
        if (a != hit) {
          long double d = (lam[a] / lam[hit]) / (nodes[hit] - nodes[a]);
          G[i * n + a] = (double)d;
          diag -= d;
        }
      }
      G[i * n + hit] = (double)diag;
      continue;
    }
    // l(t) = prod (t - x_m); phi_a = l * lam_a / (t - x_a);
    // phi_a' = lam_a * (l' / (t - x_a) - l / (t - x_a)^2), l' = l * sum 1/(t - x_m)
    long double l = 1.0L, s = 0.0L;
    for (int m = 0; m < n; ++m) { l *= (t - nodes[m]); s += 1.0L / (t - nodes[m]); }
    for (int a = 0; a < n; ++a) {
      long double inv = 1.0L / (t - nodes[a]);
      B[i * n + a] = (double)(l * lam[a] * inv);
      G[i * n + a] = (double)(lam[a] * (l * s * inv - l * inv * inv));
    }
  }
}

}  // namespace basis
}  // namespace fepa
