// Weights of the accelerated weak-coupling series (Sec. 3.1, convergence acceleration).
//
// The weak-coupling preconditioner of order d is a weighted sum of its terms,
// P_d r = sum_{n=0}^{d} c_n t_n with t_n = (-A M0^{-1} M1)^n M0^{-1} r (Sec. 3, Eq. WCE), so every
// acceleration of the series only changes the weights c_n, computed here on the host in FP64:
//   UFG_ACCEL_NONE     the partial sum S_{0,d}: c_n = 1;
//   UFG_ACCEL_EULER    S_{d,0} of the recursion S_{j+1,k} = p S_{j,k} + (1 - p) S_{j,k+1}
//                      (Eq. Euler), run until one term is left;
//   UFG_ACCEL_EULER23  S_{j,d-j} with j the integer nearest 2d/3 (the paper's S_{2kmax/3,kmax/3},
//                      whose rounding it leaves open), the last entry of level j, so it still
//                      uses every term;
//   UFG_ACCEL_VANW     the special van Wijngaarden transformation: the terms are multiplied by
//                      lambda_k = s^k / k!, Euler transformed into
//                      b_n = sum_{j<=n} C(n, j) p^(n-j) (1-p)^(j+1) lambda_j t_j, and summed as
//                      sum_{n<=d} mu_n b_n with mu_n = int_0^inf s e^(-s t) t^n / (1-p+pt)^(n+1) dt.
// The Euler weights are the recursion applied to the coefficient vectors of the partial sums;
// mu_n is integrated by 32-point Gauss-Legendre rules on panels that double in length.
#include <cmath>
#include <vector>

#include "ufg_internal.h"

namespace ufg {

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the Legendre recurrence).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// mu_k = int_0^inf e^(-u) (u/s)^k / (1 - p + p u/s)^(k+1) du (u = s t).  The integrand is analytic
// on [0, inf) with its nearest singularity at u = -s (1-p)/p, so the first panel is kept within
// a quarter of that distance and the panels double up to u = 160 (e^-160 is far below rounding).
double vanw_mu(int k, double s, double p) {
  static std::vector<double> gx, gw;
  if (gx.empty()) gauss_legendre(32, gx, gw);
  auto f = [&](double u) {
    const double t = u / s;
    return std::exp(-u) * std::pow(t, k) / std::pow(1.0 - p + p * t, k + 1);
  };
  double a = 0.0, h = std::fmin(0.25, 0.25 * s * (1.0 - p) / p), total = 0.0;
  while (a < 160.0) {
    const double b = a + h, mid = 0.5 * (a + b), half = 0.5 * h;
    double acc = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) acc += gw[i] * f(mid + half * gx[i]);
    total += half * acc;
    a = b;
    if (a >= 2.0 * h) h *= 2.0;
  }
  return total;
}

}  // namespace

bool wce_series_weights(int d, int accel, double p, double s, std::vector<double>& c) {
  c.assign(d + 1, 1.0);
  if (d < 0 || !(p > 0.0 && p < 1.0) || !(s > 0.0)) return false;
  if (accel == UFG_ACCEL_NONE) return true;
  if (accel == UFG_ACCEL_EULER || accel == UFG_ACCEL_EULER23) {
    const int j = accel == UFG_ACCEL_EULER ? d : (2 * d + 1) / 3;
    // row k of `rows` holds the coefficients of S_{level,k} in the terms t_0..t_d
    std::vector<std::vector<double>> rows(d + 1, std::vector<double>(d + 1, 0.0));
    for (int k = 0; k <= d; ++k)
      for (int n = 0; n <= k; ++n) rows[k][n] = 1.0;
    for (int level = 0; level < j; ++level) {
      for (int k = 0; k + 1 < (int)rows.size(); ++k)
        for (int n = 0; n <= d; ++n) rows[k][n] = p * rows[k][n] + (1.0 - p) * rows[k + 1][n];
      rows.pop_back();
    }
    c = rows[d - j];
    return true;
  }
  if (accel == UFG_ACCEL_VANW) {
    std::vector<double> lam(d + 1), mu(d + 1);
    double fact = 1.0;
    for (int k = 0; k <= d; ++k) {
      if (k > 0) fact *= k;
      lam[k] = std::pow(s, k) / fact;
      mu[k] = vanw_mu(k, s, p);
    }
    for (int j = 0; j <= d; ++j) {
      double acc = 0.0, binom = 1.0;  // C(n, j) for n = j, j+1, ...
      for (int n = j; n <= d; ++n) {
        if (n > j) binom = binom * n / (n - j);
        acc += binom * std::pow(p, n - j) * mu[n];
      }
      c[j] = lam[j] * std::pow(1.0 - p, j + 1) * acc;
    }
    return true;
  }
  return false;
}

ufg_status normalize_pc(int kind, const ufg_pc_params* in, ufg_pc_params* out) {
  *out = *in;
  if (out->euler_p == 0.0) out->euler_p = 0.5;
  if (out->vw_s == 0.0) out->vw_s = 1.0;
  if (kind == UFG_PC_WCE) {
    if (out->order < 0 || out->order > 16) {
      set_error("WCE: order must be in 0..16");
      return UFG_INVALID_ARG;
    }
    if (out->euler < UFG_ACCEL_NONE || out->euler > UFG_ACCEL_VANW) {
      set_error("WCE: euler must be a ufg_accel value (0..3), got %d", out->euler);
      return UFG_INVALID_ARG;
    }
    if (!(out->euler_p > 0.0 && out->euler_p < 1.0) || !(out->vw_s > 0.0) ||
        !std::isfinite(out->vw_s)) {
      set_error("WCE: need 0 < euler_p < 1 and vw_s > 0 (got %g, %g)", out->euler_p, out->vw_s);
      return UFG_INVALID_ARG;
    }
  }
  return UFG_OK;
}

}  // namespace ufg

extern "C" ufg_status ufg_wce_series_weights(int order, int accel, double euler_p, double vw_s,
                                             double* weights) {
  ufg::clear_error();
  if (weights == nullptr) {
    ufg::set_error("wce_series_weights: weights is null");
    return UFG_INVALID_ARG;
  }
  ufg_pc_params in = {}, pc = {};
  in.order = order;
  in.euler = accel;
  in.euler_p = euler_p;
  in.vw_s = vw_s;
  const ufg_status st = ufg::normalize_pc(UFG_PC_WCE, &in, &pc);
  if (st != UFG_OK) return st;
  std::vector<double> c;
  if (!ufg::wce_series_weights(pc.order, pc.euler, pc.euler_p, pc.vw_s, c)) {
    ufg::set_error("wce_series_weights: invalid acceleration parameters");
    return UFG_INVALID_ARG;
  }
  for (int n = 0; n <= pc.order; ++n) weights[n] = c[(size_t)n];
  return UFG_OK;
}
