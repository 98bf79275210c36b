// Specific heat from an energy curve (arXiv:2409.05285, Sec. III.A: C_v from the derivative of
// a spline fitted to E against beta): C/N = dE/dT = -beta^2 dE/dbeta.
//
// The fit is a natural cubic smoothing spline (Reinsch's construction): with knots x_1 < ... <
// x_n, values g and second derivatives gamma (gamma_1 = gamma_n = 0), it minimises
// lambda * integral f''^2 subject to sum_i (y_i - g_i)^2 <= s; s = 0 interpolates.  For a given
// lambda, (R + lambda Q^T Q) gamma = Q^T y (a symmetric pentadiagonal system, Q the n x (n-2)
// second-difference matrix and R the (n-2)-square tridiagonal of the knot spacings) and
// g = y - lambda Q gamma; lambda is found by bisection on log lambda so that the residual sum
// of squares meets s.  Host code, double precision, no GPU involved.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/peps_vmc.h"

namespace {

// Solves the symmetric positive definite pentadiagonal system (diagonals d0 main, d1 first and
// d2 second off-diagonal) by an LDL^T factorisation; b is overwritten with the solution.
void penta_solve(std::vector<double> d0, std::vector<double> d1, std::vector<double> d2,
                 std::vector<double>& b) {
  const int m = (int)d0.size();
  // LDL^T with L unit lower triangular of bandwidth 2: l1[i] = L(i+1, i), l2[i] = L(i+2, i)
  std::vector<double> D(m), l1(m, 0.0), l2(m, 0.0);
  for (int i = 0; i < m; ++i) {
    double di = d0[i];
    if (i >= 1) di -= l1[i - 1] * l1[i - 1] * D[i - 1];
    if (i >= 2) di -= l2[i - 2] * l2[i - 2] * D[i - 2];
    D[i] = di;
    if (i + 1 < m) {
      double v = d1[i];
      if (i >= 1) v -= l2[i - 1] * l1[i - 1] * D[i - 1];
      l1[i] = v / di;
    }
    if (i + 2 < m) l2[i] = d2[i] / di;
  }
  for (int i = 0; i < m; ++i) {   // L z = b
    if (i >= 1) b[i] -= l1[i - 1] * b[i - 1];
    if (i >= 2) b[i] -= l2[i - 2] * b[i - 2];
  }
  for (int i = 0; i < m; ++i) b[i] /= D[i];
  for (int i = m - 1; i >= 0; --i) {   // L^T x = z
    if (i + 1 < m) b[i] -= l1[i] * b[i + 1];
    if (i + 2 < m) b[i] -= l2[i] * b[i + 2];
  }
}

struct Spline {
  std::vector<double> x, g, gam;   // knots, values, second derivatives (natural: ends zero)

  // Fit for a given lambda; returns the residual sum of squares.
  double fit(const std::vector<double>& y, double lambda) {
    const int n = (int)x.size(), m = n - 2;
    std::vector<double> h(n - 1);
    for (int i = 0; i + 1 < n; ++i) h[i] = x[i + 1] - x[i];
    // Q column j (j = 0..m-1, interior knot j+1): Q[j][j] = 1/h_j, Q[j+1][j] = -1/h_j - 1/h_{j+1},
    // Q[j+2][j] = 1/h_{j+1}.  R tridiagonal: R[j][j] = (h_j + h_{j+1}) / 3, R[j][j+1] = h_{j+1} / 6.
    std::vector<double> qa(m), qb(m), qc(m);
    for (int j = 0; j < m; ++j) {
      qa[j] = 1.0 / h[j];
      qb[j] = -1.0 / h[j] - 1.0 / h[j + 1];
      qc[j] = 1.0 / h[j + 1];
    }
    std::vector<double> d0(m), d1(m, 0.0), d2(m, 0.0), rhs(m);
    for (int j = 0; j < m; ++j) {
      // (Q^T Q)[j][j] = qa^2 + qb^2 + qc^2; [j][j+1] = qb_j qa_{j+1} + qc_j qb_{j+1}; [j][j+2] = qc_j qa_{j+2}
      d0[j] = (h[j] + h[j + 1]) / 3.0 + lambda * (qa[j] * qa[j] + qb[j] * qb[j] + qc[j] * qc[j]);
      if (j + 1 < m) d1[j] = h[j + 1] / 6.0 + lambda * (qb[j] * qa[j + 1] + qc[j] * qb[j + 1]);
      if (j + 2 < m) d2[j] = lambda * (qc[j] * qa[j + 2]);
      rhs[j] = qa[j] * y[j] + qb[j] * y[j + 1] + qc[j] * y[j + 2];
    }
    penta_solve(d0, d1, d2, rhs);
    gam.assign(n, 0.0);
    for (int j = 0; j < m; ++j) gam[j + 1] = rhs[j];
    g = y;
    double rss = 0.0;
    for (int i = 0; i < n; ++i) {
      // (Q gamma)_i: row i of Q touches columns i-2 (qc), i-1 (qb), i (qa)
      double qg = 0.0;
      if (i - 2 >= 0 && i - 2 < m) qg += qc[i - 2] * rhs[i - 2];
      if (i - 1 >= 0 && i - 1 < m) qg += qb[i - 1] * rhs[i - 1];
      if (i < m) qg += qa[i] * rhs[i];
      g[i] = y[i] - lambda * qg;
      rss += (y[i] - g[i]) * (y[i] - g[i]);
    }
    return rss;
  }

  double deriv(double t) const {
    const int n = (int)x.size();
    int i = (int)(std::upper_bound(x.begin(), x.end(), t) - x.begin()) - 1;
    i = std::max(0, std::min(n - 2, i));
    const double h = x[i + 1] - x[i];
    const double a = (x[i + 1] - t) / h, b = (t - x[i]) / h;
    return (g[i + 1] - g[i]) / h + (-(3 * a * a - 1) * gam[i] + (3 * b * b - 1) * gam[i + 1]) * h / 6.0;
  }
};

}  // namespace

extern "C" int peps_cv_spline(const double* beta, const double* E_site, int n, double smoothing,
                              const double* beta_eval, double* cv, int m) {
  if (!beta || !E_site || n < 3 || !(smoothing >= 0) || m < 0 || (m > 0 && (!beta_eval || !cv)))
    return PEPS_EINVAL;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return beta[a] < beta[b]; });
  Spline sp;
  std::vector<double> y(n);
  sp.x.resize(n);
  for (int i = 0; i < n; ++i) {
    sp.x[i] = beta[order[i]];
    y[i] = E_site[order[i]];
    if (!std::isfinite(sp.x[i]) || !std::isfinite(y[i])) return PEPS_EINVAL;
    if (i > 0 && !(sp.x[i] > sp.x[i - 1])) return PEPS_EINVAL;   // distinct abscissae
  }
  if (smoothing == 0.0) {
    sp.fit(y, 0.0);
  } else {
    // the residual sum of squares grows with lambda: bisect on log lambda
    double lo = -30.0, hi = 30.0;
    if (sp.fit(y, std::exp(hi)) <= smoothing) {
      lo = hi;
    } else {
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sp.fit(y, std::exp(mid)) > smoothing) hi = mid;
        else lo = mid;
      }
    }
    sp.fit(y, std::exp(lo));
  }
  for (int k = 0; k < m; ++k) {
    const double b = beta_eval[k];
    if (!std::isfinite(b)) return PEPS_EINVAL;
    cv[k] = -b * b * sp.deriv(b);
  }
  return PEPS_OK;
}
