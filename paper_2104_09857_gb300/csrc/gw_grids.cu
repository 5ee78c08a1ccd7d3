// Minimax imaginary-time and imaginary-frequency grids (host code, FP64).
//
// chi(i tau) is computed on a minimax time grid and cosine-transformed onto a
// minimax frequency grid (the passage before Eq. 7; 12-point grids in the
// Computational Details).  The grids are those of the space-time GW method:
// with x = E / E_min in [1, R], R = E_max / E_min, the n-term best
// approximation of 1/x in the maximum norm
//   time:       1/x ~ sum_j a_j exp(-p_j x)                (1/x = int e^{-x t} dt)
//   frequency:  1/x ~ sum_k b_k x^2 / (x^2 + p_k^2)^2      (1/x = 4/pi int x^2/(x^2+w^2)^2 dw)
// whose error equioscillates at 2n + 1 points (signs +, -, ..., +).
//
// Remez exchange: levelling on a reference set by Levenberg-Marquardt in
// (ln a, ln p, lambda) with Householder-QR steps; exchange from the local
// extrema of the error on a dense ln x grid, refined by parabolas.  Starting
// values by continuation in n on [1, 1e10] and then downward in R.  The work is
// a few hundred small dense solves: host code, not a GPU kernel.

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/gwchi.h"

namespace {

constexpr double kRHalfLine = 1e10;
// Arithmetic allowed per grid, in floating-point operations of the QR solves
// and error sweeps (a few seconds); past it the call reports
// GW_ERR_NOT_CONVERGED instead of searching on.
constexpr double kWorkBudget = 3e10;

struct Approx {
  int kind = GW_GRID_TIME;
  std::vector<double> a, p;  // weights, nodes
};

inline double basis(int kind, double x, double p) {
  if (kind == GW_GRID_TIME) return std::exp(-p * x);
  const double x2 = x * x, d = x2 + p * p;
  return x2 / (d * d);
}

// d basis / d ln p
inline double basis_dlogp(int kind, double x, double p) {
  if (kind == GW_GRID_TIME) {
    const double t = p * x;
    return -t * std::exp(-t);
  }
  const double x2 = x * x, p2 = p * p, d = x2 + p2;
  return -4.0 * p2 * x2 / (d * d * d);
}

double eta(const Approx& f, double x) {
  double s = 0.0;
  for (size_t j = 0; j < f.a.size(); ++j) s += f.a[j] * basis(f.kind, x, f.p[j]);
  return 1.0 / x - s;
}

// Least-squares solution of A z = b (A: m x k row-major, m >= k) by
// Householder QR.  False when a diagonal entry of R vanishes.
bool qr_lstsq(std::vector<double> A, int m, int k, std::vector<double> b, std::vector<double>& z) {
  for (int c = 0; c < k; ++c) {
    double nrm = 0.0;
    for (int r = c; r < m; ++r) nrm += A[r * k + c] * A[r * k + c];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    const double alpha = A[c * k + c] > 0 ? -nrm : nrm;
    // v = column c below the diagonal minus alpha e_c
    std::vector<double> v(m - c);
    for (int r = c; r < m; ++r) v[r - c] = A[r * k + c];
    v[0] -= alpha;
    double vv = 0.0;
    for (double t : v) vv += t * t;
    if (vv == 0.0) continue;
    for (int cc = c; cc < k; ++cc) {
      double s = 0.0;
      for (int r = c; r < m; ++r) s += v[r - c] * A[r * k + cc];
      s = 2.0 * s / vv;
      for (int r = c; r < m; ++r) A[r * k + cc] -= s * v[r - c];
    }
    double s = 0.0;
    for (int r = c; r < m; ++r) s += v[r - c] * b[r];
    s = 2.0 * s / vv;
    for (int r = c; r < m; ++r) b[r] -= s * v[r - c];
  }
  z.assign(k, 0.0);
  for (int c = k - 1; c >= 0; --c) {
    double s = b[c];
    for (int cc = c + 1; cc < k; ++cc) s -= A[c * k + cc] * z[cc];
    const double d = A[c * k + c];
    if (d == 0.0 || !std::isfinite(d)) return false;
    z[c] = s / d;
  }
  return true;
}

// Residuals of the levelled system eta(X_i) - (-1)^i lambda for the
// unknowns z = (ln a, ln p, lambda).  False on a non-finite value.
bool level_residual(int kind, const std::vector<double>& X, const std::vector<double>& z,
                    std::vector<double>& F) {
  const int n = static_cast<int>((z.size() - 1) / 2);
  Approx f;
  f.kind = kind;
  f.a.resize(n);
  f.p.resize(n);
  for (int j = 0; j < n; ++j) {
    f.a[j] = std::exp(z[j]);
    f.p[j] = std::exp(z[n + j]);
  }
  F.resize(X.size());
  for (size_t i = 0; i < X.size(); ++i) {
    const double sgn = (i % 2 == 0) ? 1.0 : -1.0;
    F[i] = eta(f, X[i]) - sgn * z[2 * n];
    if (!std::isfinite(F[i])) return false;
  }
  return true;
}

double sumsq(const std::vector<double>& v) {
  double s = 0.0;
  for (double t : v) s += t * t;
  return s;
}

// Levenberg-Marquardt with Marquardt's column scaling: each step solves
// [J; sqrt(mu) D] dz = [-F; 0] in the least-squares sense.  The damping starts
// near Gauss-Newton (the levelled system is square and usually well started)
// and follows Nielsen's rule: scaled by max(1/3, 1 - (2 rho - 1)^3) after an
// accepted step with gain ratio rho, by 2, 4, 8, ... after rejected ones.
void level(int kind, const std::vector<double>& X, Approx& f, double& lam, double& budget) {
  const int n = static_cast<int>(f.a.size());
  const int N = 2 * n + 1;
  std::vector<double> z(N), F, Fn, zn, dz, D(N, 0.0);
  for (int j = 0; j < n; ++j) {
    z[j] = std::log(f.a[j]);
    z[n + j] = std::log(f.p[j]);
  }
  z[2 * n] = lam;
  if (!level_residual(kind, X, z, F)) return;
  double mu = 1e-12, fs = sumsq(F), nu = 2.0;
  std::vector<double> A(static_cast<size_t>(2 * N) * N), b(2 * N);
  for (int it = 0; it < 2000 && fs > 0.0 && budget > 0; ++it) {
    // Jacobian rows at z
    for (int i = 0; i < N; ++i) {
      const double x = X[i];
      for (int j = 0; j < n; ++j) {
        const double a = std::exp(z[j]), p = std::exp(z[n + j]);
        A[i * N + j] = -a * basis(kind, x, p);
        A[i * N + n + j] = -a * basis_dlogp(kind, x, p);
      }
      A[i * N + 2 * n] = (i % 2 == 0) ? -1.0 : 1.0;
      b[i] = -F[i];
    }
    for (int c = 0; c < N; ++c) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) s += A[i * N + c] * A[i * N + c];
      D[c] = std::max(D[c], std::sqrt(s));
    }
    bool accepted = false;
    double step = 0.0;
    while (mu < 1e30 && budget > 0) {
      budget -= 4.0 * N * N * N;
      std::vector<double> Aa(A.begin(), A.begin() + static_cast<size_t>(N) * N);
      Aa.resize(static_cast<size_t>(2 * N) * N, 0.0);
      std::vector<double> ba(b.begin(), b.begin() + N);
      ba.resize(2 * N, 0.0);
      for (int c = 0; c < N; ++c) Aa[(N + c) * N + c] = std::sqrt(mu) * (D[c] > 0 ? D[c] : 1.0);
      if (!qr_lstsq(Aa, 2 * N, N, ba, dz)) {
        mu *= 10.0;
        continue;
      }
      zn = z;
      step = 0.0;
      for (int c = 0; c < N; ++c) {
        zn[c] += dz[c];
        step = std::max(step, std::fabs(dz[c]) / (1.0 + std::fabs(z[c])));
      }
      if (level_residual(kind, X, zn, Fn) && sumsq(Fn) < fs) {
        const double fs_old = fs;
        // gain ratio against the linear model ||F + J dz||^2
        double model = 0.0;
        for (int i = 0; i < N; ++i) {
          double r = F[i];
          for (int c = 0; c < N; ++c) r += A[i * N + c] * dz[c];
          model += r * r;
        }
        const double rho = (fs_old - sumsq(Fn)) / std::max(fs_old - model, 1e-300);
        z.swap(zn);
        F.swap(Fn);
        fs = sumsq(F);
        const double t = 2.0 * rho - 1.0;
        mu = std::max(mu * std::max(1.0 / 3.0, 1.0 - t * t * t), 1e-20);
        nu = 2.0;
        accepted = true;
        // converged: the residual no longer falls, or sits at rounding level
        if (fs_old - fs <= 1e-12 * fs_old || fs <= 1e-30 * N) step = 0.0;
        break;
      }
      mu *= nu;
      nu *= 2.0;
      if (step < 1e-16) break;
    }
    if (!accepted || step < 1e-15) break;
  }
  for (int j = 0; j < n; ++j) {
    f.a[j] = std::exp(z[j]);
    f.p[j] = std::exp(z[n + j]);
  }
  lam = z[2 * n];
}

struct Extremum {
  double x, e;
};

// Local extrema of eta on [1, R] with both ends: dense ln x grid of m points,
// interior extrema refined by five parabola fits with shrinking spacing; runs
// of equal sign merged to their largest |eta|.  emax = max |eta| seen.
std::vector<Extremum> extrema(const Approx& f, double R, int m, double& emax) {
  const double tR = std::log(R), h = tR / (m - 1);
  std::vector<double> e(m);
  emax = 0.0;
  for (int i = 0; i < m; ++i) {
    e[i] = eta(f, std::exp(i * h));
    emax = std::max(emax, std::fabs(e[i]));
  }
  std::vector<double> ts{0.0};
  for (int i = 1; i + 1 < m; ++i) {
    if ((e[i] - e[i - 1]) * (e[i + 1] - e[i]) >= 0) continue;
    double t = i * h, step = h;
    for (int r = 0; r < 5; ++r) {
      const double em = eta(f, std::exp(t - step)), e0 = eta(f, std::exp(t)),
                   ep = eta(f, std::exp(t + step));
      const double den = ep - 2.0 * e0 + em;
      if (den != 0.0) t -= 0.5 * step * (ep - em) / den;
      step /= 8.0;
    }
    ts.push_back(std::min(std::max(t, 0.0), tR));
  }
  ts.push_back(tR);
  std::vector<Extremum> out;
  for (double t : ts) {
    const double x = std::exp(t), v = eta(f, x);
    emax = std::max(emax, std::fabs(v));
    if (!out.empty() && ((v > 0) == (out.back().e > 0))) {
      if (std::fabs(v) > std::fabs(out.back().e)) out.back() = {x, v};
    } else {
      out.push_back({x, v});
    }
  }
  return out;
}

// 2n + 1 consecutive alternating extrema, positive at both ends, containing
// the largest |eta|; among those, the window with the largest smallest |eta|.
bool choose_reference(const std::vector<Extremum>& ex, int n, std::vector<double>& X,
                      double& emin) {
  const int k = 2 * n + 1, cnt = static_cast<int>(ex.size());
  int g = 0;
  for (int i = 1; i < cnt; ++i)
    if (std::fabs(ex[i].e) > std::fabs(ex[g].e)) g = i;
  int best = -1;
  double key = -1.0;
  for (int s = 0; s + k <= cnt; ++s) {
    if (ex[s].e <= 0 || ex[s + k - 1].e <= 0 || g < s || g >= s + k) continue;
    double v = INFINITY;
    for (int i = s; i < s + k; ++i) v = std::min(v, std::fabs(ex[i].e));
    if (v > key) {
      key = v;
      best = s;
    }
  }
  if (best < 0) return false;
  X.resize(k);
  for (int i = 0; i < k; ++i) X[i] = ex[best + i].x;
  emin = key;
  return true;
}

// Remez exchange from f and reference X.  On success f holds the best
// approximation on [1, R], X its reference and E the maximum error.
bool remez(Approx& f, double R, std::vector<double>& X, double& E, double& budget) {
  const int n = static_cast<int>(f.a.size());
  const int m = 200 * n + 400;
  double lam = 0.0;
  for (double x : X) lam += std::fabs(eta(f, x));
  lam /= X.size();
  double prev = -1.0;
  for (int it = 0; it < 100; ++it) {
    level(f.kind, X, f, lam, budget);
    if (budget <= 0) return false;
    double emax = 0.0, emin = 0.0;
    const std::vector<Extremum> ex = extrema(f, R, m, emax);
    budget -= 20.0 * m * n;
    if (!std::isfinite(emax) || !choose_reference(ex, n, X, emin)) return false;
    E = emax;
    if (emax - emin <= 1e-9 * emax + 1e-15) return true;
    if (prev >= 0 && std::fabs(emax - prev) <= 1e-12 * emax) return true;  // level to rounding
    prev = emax;
  }
  return false;
}

// Weights of the n nodes p that fit 1/x on the points X in least squares,
// non-positive ones replaced by 1e-6 (the levelling fixes them).
std::vector<double> fit_weights(int kind, const std::vector<double>& X, const std::vector<double>& p) {
  const int m = static_cast<int>(X.size()), k = static_cast<int>(p.size());
  std::vector<double> A(static_cast<size_t>(m) * k), b(m), w;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < k; ++j) A[i * k + j] = basis(kind, X[i], p[j]);
    b[i] = 1.0 / X[i];
  }
  if (!qr_lstsq(A, m, k, b, w)) w.assign(k, 1.0 / k);
  for (double& t : w)
    if (!(t > 0)) t = 1e-6;
  return w;
}

// Values y at cell centres (k + 1/2)/len moved to (k + 1/2)/m, linear,
// extrapolated past the end cells.
std::vector<double> stretch(const std::vector<double>& y, int m) {
  const int k = static_cast<int>(y.size());
  std::vector<double> out(m);
  for (int i = 0; i < m; ++i) {
    const double t = (i + 0.5) / m, u = t * k - 0.5;  // position in cell units
    int lo = static_cast<int>(std::floor(u));
    lo = std::min(std::max(lo, 0), k - 2);
    out[i] = y[lo] + (u - lo) * (y[lo + 1] - y[lo]);
  }
  return out;
}

// Values at i/(len-1) moved to i/(m-1), linear.
std::vector<double> resample(const std::vector<double>& y, int m) {
  const int k = static_cast<int>(y.size());
  std::vector<double> out(m);
  for (int i = 0; i < m; ++i) {
    const double u = (m > 1 ? static_cast<double>(i) / (m - 1) : 0.0) * (k - 1);
    int lo = std::min(static_cast<int>(std::floor(u)), k - 2);
    out[i] = y[lo] + (u - lo) * (y[lo + 1] - y[lo]);
  }
  return out;
}

// Best n-term approximation on [1, R].
int minimax_unit(int kind, int n, double R, Approx& f, double& E) {
  const double Rhi = std::max(R, kRHalfLine);
  double budget = kWorkBudget;
  f.kind = kind;
  f.p = {kind == GW_GRID_TIME ? 0.5 : 1.0};
  std::vector<double> X{1.0, std::sqrt(12.0), 12.0};
  f.a = fit_weights(kind, X, f.p);
  if (!remez(f, Rhi, X, E, budget)) return GW_ERR_NOT_CONVERGED;
  std::vector<double> errs{E};
  // continuation in n on the half line
  for (int m = 2; m <= n; ++m) {
    std::vector<double> lp(f.p.size());
    for (size_t j = 0; j < lp.size(); ++j) lp[j] = std::log(f.p[j]);
    if (m == 2)
      lp = {lp[0] - 1.0, lp[0] + 1.0};
    else
      lp = stretch(lp, m);
    std::vector<double> lx(X.size());
    for (size_t i = 0; i < X.size(); ++i) lx[i] = std::log(X[i]);
    lx = resample(lx, 2 * m + 1);
    const double ratio = errs.size() > 1 ? errs[errs.size() - 2] / errs.back() : 4.0;
    if (X.back() < Rhi) {
      const double top = std::min(std::log(Rhi), lx.back() + std::log(ratio));
      const double s = top / lx.back();
      for (double& t : lx) t *= s;
    }
    Approx g;
    g.kind = kind;
    g.p.resize(m);
    for (int j = 0; j < m; ++j) g.p[j] = std::exp(lp[j]);
    std::vector<double> Xn(lx.size());
    for (size_t i = 0; i < lx.size(); ++i) Xn[i] = std::exp(lx[i]);
    g.a = fit_weights(kind, Xn, g.p);
    if (!remez(g, Rhi, Xn, E, budget)) return GW_ERR_NOT_CONVERGED;
    f = g;
    X = Xn;
    errs.push_back(E);
  }
  // continuation downward in R, halving a step that fails
  double Rc = std::min(Rhi, X.back() * (1.0 + 1e-7)), fac = 2.0;
  while (Rc > R) {
    const double Rn = std::max(R, Rc / fac);
    const double s = std::log(Rn) / std::log(X.back());
    std::vector<double> Xn(X.size());
    for (size_t i = 0; i < X.size(); ++i) Xn[i] = std::exp(std::log(X[i]) * s);
    Approx g = f;
    double En = 0.0;
    if (!remez(g, Rn, Xn, En, budget)) {
      fac = std::sqrt(fac);
      if (fac < 1.001 || budget <= 0) return GW_ERR_NOT_CONVERGED;
      continue;
    }
    f = g;
    X = Xn;
    E = En;
    Rc = Rn;
    fac = std::min(2.0, fac * fac);
  }
  // nodes ascending
  std::vector<int> ord(f.p.size());
  for (size_t j = 0; j < ord.size(); ++j) ord[j] = static_cast<int>(j);
  std::sort(ord.begin(), ord.end(), [&](int u, int v) { return f.p[u] < f.p[v]; });
  Approx s = f;
  for (size_t j = 0; j < ord.size(); ++j) {
    s.p[j] = f.p[ord[j]];
    s.a[j] = f.a[ord[j]];
  }
  f = s;
  return GW_OK;
}

}  // namespace

extern "C" int gw_minimax_grid(int kind, int n, double e_min, double e_max, double* nodes,
                               double* weights, double* max_err) {
  if ((kind != GW_GRID_TIME && kind != GW_GRID_FREQ) || n < 1 || n > GW_GRID_MAX_N || !nodes ||
      !weights || !max_err)
    return GW_ERR_INVALID_ARG;
  if (!(std::isfinite(e_min) && std::isfinite(e_max))) return GW_ERR_NONFINITE;
  if (!(e_min > 0.0) || !(e_max > e_min * (1.0 + 1e-9))) return GW_ERR_INVALID_ARG;
  Approx f;
  double E = 0.0;
  const int rc = minimax_unit(kind, n, e_max / e_min, f, E);
  if (rc != GW_OK) return rc;
  for (int j = 0; j < n; ++j) {
    if (kind == GW_GRID_TIME) {
      nodes[j] = f.p[j] / e_min;
      weights[j] = f.a[j] / e_min;
    } else {
      nodes[j] = f.p[j] * e_min;
      weights[j] = f.a[j] * e_min;
    }
  }
  *max_err = E / e_min;
  return GW_OK;
}
