// Host-only scalar formulas of the method (no GPU involved).
#include <math.h>

#include "bem.h"

namespace {

// Table 1 (Sec. 3.1): corrected c1(k) for k = -0.9, -0.8, ..., 0.9.
const double kTableK[19] = {-0.9, -0.8, -0.7, -0.6, -0.5, -0.4, -0.3, -0.2, -0.1, 0.0,
                            0.1,  0.2,  0.3,  0.4,  0.5,  0.6,  0.7,  0.8,  0.9};
const double kTableC1[19] = {0.14, 0.31, 0.495, 0.71, 0.96, 1.24, 1.58, 1.97, 2.43, 2.97,
                             3.66, 4.52, 5.62,  7.10, 9.15, 12.25, 17.50, 27.65, 58.00};

// Second derivatives of the natural cubic spline through (kTableK, ln c1),
// by the Thomas algorithm on the tridiagonal system of the interior knots.
struct Spline {
  double y[19], m[19];
  Spline() {
    const int n = 19;
    for (int i = 0; i < n; ++i) y[i] = log(kTableC1[i]);
    double sub[19], diag[19], sup[19], rhs[19];
    for (int i = 1; i < n - 1; ++i) {
      const double h0 = kTableK[i] - kTableK[i - 1], h1 = kTableK[i + 1] - kTableK[i];
      sub[i] = h0;
      diag[i] = 2.0 * (h0 + h1);
      sup[i] = h1;
      rhs[i] = 6.0 * ((y[i + 1] - y[i]) / h1 - (y[i] - y[i - 1]) / h0);
    }
    m[0] = m[n - 1] = 0.0;
    // forward elimination over i = 1..n-2 (m[0] = 0 drops sub[1])
    for (int i = 2; i < n - 1; ++i) {
      const double w = sub[i] / diag[i - 1];
      diag[i] -= w * sup[i - 1];
      rhs[i] -= w * rhs[i - 1];
    }
    m[n - 2] = rhs[n - 2] / diag[n - 2];
    for (int i = n - 3; i >= 1; --i) m[i] = (rhs[i] - sup[i] * m[i + 1]) / diag[i];
  }
  double eval(double k) const {
    int i = 0;
    while (i < 17 && k > kTableK[i + 1]) ++i;
    const double h = kTableK[i + 1] - kTableK[i];
    const double a = (kTableK[i + 1] - k) / h, b = (k - kTableK[i]) / h;
    return a * y[i] + b * y[i + 1] + ((a * a * a - a) * m[i] + (b * b * b - b) * m[i + 1]) * h * h / 6.0;
  }
};

}  // namespace

extern "C" double bem_alpha(double k, double nu) {
  if (!(k > -1.0 && k < 1.0) || !(nu > -1.0 && nu <= 0.5)) return NAN;
  const double b2 = (1.0 + k) * (1.0 - k * nu / (1.0 - nu));  // Eq. 4
  if (!(b2 > 0.0)) return NAN;
  const double b = sqrt(b2);
  const double pi = 3.14159265358979323846;
  // Eq. 3
  const double num = pow(2.0, k) * b * sin(0.5 * pi * b) * tgamma(0.5 * (3.0 + k + b)) *
                     tgamma(0.5 * (3.0 + k - b));
  const double den = sqrt(pi) * (1.0 + k) * cos(0.5 * pi * k) * tgamma(2.0 + k) *
                     tgamma(1.0 + 0.5 * k) * tgamma(0.5 * (1.0 - k));
  return num / den;
}

extern "C" double bem_c1_corrected(double k) {
  if (!(k >= -0.9 - 1e-12 && k <= 0.9 + 1e-12)) return NAN;
  for (int i = 0; i < 19; ++i)
    if (k == kTableK[i]) return kTableC1[i];
  static const Spline sp;
  return exp(sp.eval(k));
}

extern "C" double bem_p_crit(double k, double nu, double E0, double c0, double dgamma, double delta) {
  const double a = bem_alpha(k, nu), c1 = bem_c1_corrected(k);
  if (!(a > 0.0) || !(c1 > 0.0) || !(E0 > 0.0) || !(c0 > 0.0) || !(dgamma >= 0.0) || !(delta > 0.0))
    return NAN;
  // Eq. 24
  return sqrt(2.0 * E0 * dgamma / (a * (1.0 - nu * nu) * c1 * pow(c0, k) * pow(delta, 1.0 - k)));
}
