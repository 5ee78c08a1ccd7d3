// Weights of the imaginary-time <-> imaginary-frequency transforms (host code,
// FP64): the cosine transform chi(i tau) -> chi(i omega) and W(i omega) ->
// W(i tau) of the screening chain (the passage before Eq. 7 and after Eq. 9),
// and the half-line sine transform of the self-energy (the quasiparticle step
// after Eq. 11).
//
// Every term of chi(i tau) and of Sigma^c(i tau) decays like exp(-x|tau|) for a
// transition energy x in [E_min, E_max].  The weights make each transform exact
// for those functions in the least-squares sense over x:
//   cosine:  sum_j gamma_kj exp(-x tau_j)           ~ 2x / (x^2 + omega_k^2)
//   inverse: sum_k delta_jk 2x / (x^2 + omega_k^2)  ~ exp(-x tau_j)
//   sine:    sum_j s_kj exp(-x tau_j)               ~ omega_k / (x^2 + omega_k^2)
// on 400 points log-spaced over [E_min, E_max].  The minimum-norm solution
// keeps the singular values above 1e-14 of the largest (the columns are nearly
// dependent when the grid is dense for the energy range).  One-sided Jacobi
// SVD: a handful of small matrices per calculation, host code.

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/gwchi.h"

namespace {

constexpr int kFitPoints = 400;    // x samples of the least-squares fit
constexpr int kCheckPoints = 997;  // x samples of the reported fit error
constexpr double kRcond = 1e-14;

// Thin SVD A = U diag(s) V^T of A (m x n, m >= n, row-major) by one-sided
// Jacobi rotations: U m x n (row-major), s n, V n x n (row-major).
void jacobi_svd(const std::vector<double>& A, int m, int n, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& V) {
  U = A;
  V.assign(static_cast<size_t>(n) * n, 0.0);
  for (int j = 0; j < n; ++j) V[j * n + j] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = 0; i < m; ++i) {
          const double up = U[i * n + p], uq = U[i * n + q];
          a += up * up;
          b += uq * uq;
          g += up * uq;
        }
        if (g == 0.0 || std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          const double up = U[i * n + p], uq = U[i * n + q];
          U[i * n + p] = c * up - sn * uq;
          U[i * n + q] = sn * up + c * uq;
        }
        for (int i = 0; i < n; ++i) {
          const double vp = V[i * n + p], vq = V[i * n + q];
          V[i * n + p] = c * vp - sn * vq;
          V[i * n + q] = sn * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  s.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += U[i * n + j] * U[i * n + j];
    s[j] = std::sqrt(nrm);
    if (s[j] > 0.0)
      for (int i = 0; i < m; ++i) U[i * n + j] /= s[j];
  }
}

// Minimum-norm least-squares solutions X (n x r, row-major) of A X ~ F for
// A m x n and F m x r, singular values below kRcond * max dropped.
std::vector<double> lstsq(const std::vector<double>& A, int m, int n, const std::vector<double>& F,
                          int r) {
  std::vector<double> U, s, V;
  jacobi_svd(A, m, n, U, s, V);
  const double smax = *std::max_element(s.begin(), s.end());
  std::vector<double> X(static_cast<size_t>(n) * r, 0.0), y(n);
  for (int c = 0; c < r; ++c) {
    for (int j = 0; j < n; ++j) {
      y[j] = 0.0;
      if (!(s[j] > kRcond * smax)) continue;
      double d = 0.0;
      for (int i = 0; i < m; ++i) d += U[i * n + j] * F[i * r + c];
      y[j] = d / s[j];
    }
    for (int i = 0; i < n; ++i) {
      double v = 0.0;
      for (int j = 0; j < n; ++j) v += V[i * n + j] * y[j];
      X[i * r + c] = v;
    }
  }
  return X;
}

std::vector<double> samples(double lo, double hi, int m) {
  std::vector<double> x(m);
  for (int i = 0; i < m; ++i) x[i] = lo * std::pow(hi / lo, static_cast<double>(i) / (m - 1));
  return x;
}

// exp(-x tau_j): [m][n_tau]
std::vector<double> exp_cols(const std::vector<double>& x, const double* tau, int n_tau) {
  std::vector<double> e(x.size() * n_tau);
  for (size_t i = 0; i < x.size(); ++i)
    for (int j = 0; j < n_tau; ++j) e[i * n_tau + j] = std::exp(-x[i] * tau[j]);
  return e;
}

// 2x/(x^2 + omega_k^2) (cosine) or omega_k/(x^2 + omega_k^2) (sine): [m][n_omega]
std::vector<double> freq_cols(const std::vector<double>& x, const double* omega, int n_omega,
                              bool sine) {
  std::vector<double> f(x.size() * n_omega);
  for (size_t i = 0; i < x.size(); ++i)
    for (int k = 0; k < n_omega; ++k) {
      const double d = x[i] * x[i] + omega[k] * omega[k];
      f[i * n_omega + k] = (sine ? omega[k] : 2.0 * x[i]) / d;
    }
  return f;
}

// max_i,c |sum_j B[i][j] W[c][j] - T[i][c]| / max |T| with W given as [r][n]
double fit_error(const std::vector<double>& B, int m, int n, const double* W,
                 const std::vector<double>& T, int r) {
  double num = 0.0, den = 0.0;
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < r; ++c) {
      double v = 0.0;
      for (int j = 0; j < n; ++j) v += B[i * n + j] * W[c * n + j];
      num = std::max(num, std::fabs(v - T[i * r + c]));
      den = std::max(den, std::fabs(T[i * r + c]));
    }
  return den > 0.0 ? num / den : num;
}

// Transposes X (n x r) into out (r x n).
void store_transposed(const std::vector<double>& X, int n, int r, double* out) {
  for (int c = 0; c < r; ++c)
    for (int j = 0; j < n; ++j) out[c * n + j] = X[j * r + c];
}

}  // namespace

extern "C" int gw_transform_weights(const double* tau, int n_tau, const double* omega,
                                    int n_omega, double e_min, double e_max, double* gamma,
                                    double* delta, double* s_weights, double* fit_err) {
  if (!tau || !omega || n_tau < 1 || n_omega < 1 || n_tau > kFitPoints || n_omega > kFitPoints)
    return GW_ERR_INVALID_ARG;
  if (!std::isfinite(e_min) || !std::isfinite(e_max)) return GW_ERR_NONFINITE;
  if (!(e_min > 0.0) || !(e_max > e_min)) return GW_ERR_INVALID_ARG;
  for (int j = 0; j < n_tau; ++j) {
    if (!std::isfinite(tau[j])) return GW_ERR_NONFINITE;
    if (!(tau[j] > 0.0)) return GW_ERR_INVALID_ARG;
  }
  for (int k = 0; k < n_omega; ++k) {
    if (!std::isfinite(omega[k])) return GW_ERR_NONFINITE;
    if (!(omega[k] > 0.0)) return GW_ERR_INVALID_ARG;
  }
  const std::vector<double> x = samples(e_min, e_max, kFitPoints);
  const std::vector<double> xc = samples(e_min, e_max, kCheckPoints);
  const std::vector<double> E = exp_cols(x, tau, n_tau), Ec = exp_cols(xc, tau, n_tau);
  const std::vector<double> C = freq_cols(x, omega, n_omega, false),
                            Cc = freq_cols(xc, omega, n_omega, false);
  double err[3] = {0.0, 0.0, 0.0};
  if (gamma) {
    store_transposed(lstsq(E, kFitPoints, n_tau, C, n_omega), n_tau, n_omega, gamma);
    err[0] = fit_error(Ec, kCheckPoints, n_tau, gamma, Cc, n_omega);
  }
  if (delta) {
    store_transposed(lstsq(C, kFitPoints, n_omega, E, n_tau), n_omega, n_tau, delta);
    err[1] = fit_error(Cc, kCheckPoints, n_omega, delta, Ec, n_tau);
  }
  if (s_weights) {
    const std::vector<double> S = freq_cols(x, omega, n_omega, true),
                              Sc = freq_cols(xc, omega, n_omega, true);
    store_transposed(lstsq(E, kFitPoints, n_tau, S, n_omega), n_tau, n_omega, s_weights);
    err[2] = fit_error(Ec, kCheckPoints, n_tau, s_weights, Sc, n_omega);
  }
  if (fit_err)
    for (int i = 0; i < 3; ++i) fit_err[i] = err[i];
  return GW_OK;
}
