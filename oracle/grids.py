"""Oracle for the minimax imaginary-time and imaginary-frequency grids on
which chi(i tau) is computed and cosine-transformed (the passage before Eq. 7;
12-point grids in the Computational Details).  FP64 numpy, with scipy's
Levenberg-Marquardt least-squares solver as a library step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper takes its grids from the space-time GW literature it cites and does
not restate how they are made.  Reading (restated from that published method,
in this module's own notation):

* Energies are scaled by the smallest transition energy, x = E / E_min, so
  x lies in [1, R] with R = E_max / E_min.
* Time grid ("T"): nodes tau_j and weights a_j of the n-term exponential sum
  that best approximates 1/x = int_0^inf e^{-x tau} dtau in the maximum norm,
      E_n(R) = min max_{1<=x<=R} | 1/x - sum_j a_j exp(-tau_j x) |.
* Frequency grid ("F"): nodes w_k and weights b_k of the n-term sum that best
  approximates 1/x = (4/pi) int_0^inf dw x^2 / (x^2 + w^2)^2 in the same
  norm, basis x^2 / (x^2 + w_k^2)^2 (the frequency integrand of the
  second-order ring term).
* Both families have 2n parameters; the best approximation is the one whose
  error equioscillates at 2n + 1 points 1 <= x_0 < ... < x_2n <= R with signs
  +, -, ..., + (the error is positive where 1/x outlasts every term).  When R
  exceeds the last point of the half-line solution, the grid is that of
  [1, inf).
* Physical grids: tau_j / E_min, a_j / E_min; w_k E_min, b_k E_min.

Algorithm (Remez exchange):
  1. level: for a reference set X, solve eta(x_i) = (-1)^i lam (2n + 1
     equations in log a, log p and lam) by Levenberg-Marquardt;
  2. exchange: the local extrema of eta on a dense ln x grid (refined by
     parabolas), merged by sign, give a new reference of 2n + 1 alternating
     points that contains the largest |eta|;
  repeat until max |eta| and min over the reference agree to 1e-9.
Starting values come from continuation: in n on [1, 1e10] (a node grid
stretched from the (n-1)-term solution), then downward in R (geometric steps,
the reference scaled in ln x), halving a step that fails.
"""

from __future__ import annotations

import numpy as np
import scipy.optimize as so

R_HI = 1e10   # stands for the half line in the continuation in n


def basis(kind: str, x: np.ndarray, p: np.ndarray) -> np.ndarray:
    """[len(x), len(p)]: exp(-p x) (time) or x^2 / (x^2 + p^2)^2 (frequency)."""
    x = np.asarray(x, float)
    if kind == "T":
        return np.exp(-np.outer(x, p))
    x2 = x[:, None] ** 2
    return x2 / (x2 + p[None, :] ** 2) ** 2


def basis_dlogp(kind: str, x: np.ndarray, p: np.ndarray) -> np.ndarray:
    """d basis / d ln p."""
    x = np.asarray(x, float)
    if kind == "T":
        t = np.outer(x, p)
        return -t * np.exp(-t)
    x2 = x[:, None] ** 2
    p2 = p[None, :] ** 2
    return -4.0 * p2 * x2 / (x2 + p2) ** 3


def error(kind: str, x, a, p) -> np.ndarray:
    """eta(x) = 1/x - sum_j a_j basis_j(x)."""
    x = np.asarray(x, float)
    return 1.0 / x - basis(kind, x, p) @ a


def extrema(kind: str, R: float, a, p, m: int):
    """Local extrema of eta on [1, R] (both ends included): dense ln x grid of
    m points, each interior extremum refined by four parabola fits; points of
    equal sign in a row are merged, keeping the largest |eta|.  Returns
    (x, eta(x), max |eta| on the dense grid)."""
    t = np.linspace(0.0, np.log(R), m)
    h = t[1] - t[0]
    e = error(kind, np.exp(t), a, p)
    i = np.nonzero((e[1:-1] - e[:-2]) * (e[2:] - e[1:-1]) < 0)[0] + 1
    ti = t[i].copy()
    step = h
    for _ in range(5):
        em, e0, ep = (error(kind, np.exp(ti + o), a, p) for o in (-step, 0.0, step))
        den = ep - 2.0 * e0 + em
        ti = ti - np.where(den != 0, 0.5 * step * (ep - em) / np.where(den != 0, den, 1.0), 0.0)
        step /= 8.0
    ti = np.clip(ti, 0.0, np.log(R))
    pts = np.concatenate([[0.0], ti, [np.log(R)]])
    ev = error(kind, np.exp(pts), a, p)
    xs, es = [pts[0]], [ev[0]]
    for tt, ee in zip(pts[1:], ev[1:]):
        if np.sign(ee) == np.sign(es[-1]):
            if abs(ee) > abs(es[-1]):
                xs[-1], es[-1] = tt, ee
        else:
            xs.append(tt)
            es.append(ee)
    return np.exp(np.array(xs)), np.array(es), float(np.abs(np.concatenate([e, ev])).max())


def choose_reference(x, e, n: int):
    """2n + 1 consecutive alternating extrema with sign + at both ends that
    contain the largest |eta|; among those windows the one whose smallest
    |eta| is largest.  None if no such window exists."""
    k = 2 * n + 1
    best, key = None, -1.0
    g = int(np.argmax(np.abs(e)))
    for s in range(0, len(x) - k + 1):
        if e[s] <= 0 or e[s + k - 1] <= 0 or not (s <= g < s + k):
            continue
        v = np.abs(e[s:s + k]).min()
        if v > key:
            best, key = s, v
    if best is None:
        return None
    return x[best:best + k], e[best:best + k]


def level(kind: str, X, a, p, lam):
    """Levelled approximation on the reference X: solve
    eta(x_i) - (-1)^i lam = 0 for (ln a, ln p, lam)."""
    n = len(a)
    sgn = (-1.0) ** np.arange(2 * n + 1)

    def F(z):
        with np.errstate(all="ignore"):
            f = error(kind, X, np.exp(z[:n]), np.exp(z[n:2 * n])) - sgn * z[-1]
        return np.where(np.isfinite(f), f, 1e30)

    def J(z):
        a_, p_ = np.exp(z[:n]), np.exp(z[n:2 * n])
        return np.hstack([-basis(kind, X, p_) * a_, -basis_dlogp(kind, X, p_) * a_, -sgn[:, None]])

    z0 = np.concatenate([np.log(a), np.log(p), [lam]])
    r = so.least_squares(F, z0, jac=J, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                         max_nfev=2000)
    return np.exp(r.x[:n]), np.exp(r.x[n:2 * n]), r.x[-1]


def remez(kind: str, n: int, R: float, a, p, X, max_iter: int = 100):
    """Remez exchange from weights a, nodes p and reference X.  Returns
    (a, p, E, reference) with E = max |eta| over [1, R], or None."""
    lam = float(np.abs(error(kind, X, a, p)).mean())
    m = 200 * n + 400
    prev = None
    for _ in range(max_iter):
        a, p, lam = level(kind, X, a, p, lam)
        x, e, emax = extrema(kind, R, a, p, m)
        ref = choose_reference(x, e, n)
        if ref is None:
            return None
        X, ev = ref
        emin = float(np.abs(ev).min())
        if emax - emin <= 1e-9 * emax + 1e-15:
            break
        if prev is not None and abs(emax - prev) <= 1e-12 * emax:
            break   # levelled to rounding
        prev = emax
    else:
        return None
    order = np.argsort(p)
    return a[order], p[order], emax, X


def _stretch(y: np.ndarray, m: int) -> np.ndarray:
    """Values y at cell centres (k + 1/2)/len -> (k + 1/2)/m, linear,
    extrapolated past the end cells."""
    k = len(y)
    s = (np.arange(k) + 0.5) / k
    t = (np.arange(m) + 0.5) / m
    slope_lo = (y[1] - y[0]) / (s[1] - s[0])
    slope_hi = (y[-1] - y[-2]) / (s[-1] - s[-2])
    out = np.interp(t, s, y)
    out = np.where(t < s[0], y[0] + (t - s[0]) * slope_lo, out)
    return np.where(t > s[-1], y[-1] + (t - s[-1]) * slope_hi, out)


def _resample(y: np.ndarray, m: int) -> np.ndarray:
    """Values at i/(len-1) -> i/(m-1), linear."""
    return np.interp(np.linspace(0.0, 1.0, m), np.linspace(0.0, 1.0, len(y)), y)


def minimax_unit(kind: str, n: int, R: float):
    """Minimax grid on [1, R]: (nodes ascending, weights, E_n(R)).
    Raises RuntimeError where the exchange does not converge (errors near the
    FP64 rounding level)."""
    if kind not in ("T", "F") or n < 1 or not R > 1.0:
        raise ValueError("kind T or F, n >= 1, R > 1")
    Rhi = max(R, R_HI)
    # continuation in n on the half line
    p = np.array([0.5 if kind == "T" else 1.0])
    X = np.exp(np.linspace(0.0, np.log(12.0), 3))
    a = np.linalg.lstsq(basis(kind, X, p), 1.0 / X, rcond=None)[0]
    r = remez(kind, 1, Rhi, np.abs(a), p, X)
    errs = [r[2]]
    for m in range(2, n + 1):
        a, p, e, X = r
        lp = np.log(p[0]) + np.array([-1.0, 1.0]) if m == 2 else _stretch(np.log(p), m)
        lx = _resample(np.log(X), 2 * m + 1)
        ratio = errs[-2] / errs[-1] if len(errs) > 1 else 4.0
        if X[-1] < Rhi:
            lx = lx * (min(np.log(Rhi), lx[-1] + np.log(ratio)) / lx[-1])
        Xn = np.exp(lx)
        an = np.linalg.lstsq(basis(kind, Xn, np.exp(lp)), 1.0 / Xn, rcond=None)[0]
        an = np.where(an > 0, an, 1e-6)
        r = remez(kind, m, Rhi, an, np.exp(lp), Xn)
        if r is None:
            raise RuntimeError(f"minimax {kind}: no convergence at n = {m} on the half line")
        errs.append(r[2])
    a, p, e, X = r
    # continuation downward in R
    Rc = min(Rhi, X[-1] * (1.0 + 1e-7))
    f = 2.0
    while Rc > R:
        Rn = max(R, Rc / f)
        Xn = np.exp(np.log(X) * (np.log(Rn) / np.log(X[-1])))
        rn = remez(kind, n, Rn, a, p, Xn)
        if rn is None:
            f = np.sqrt(f)
            if f < 1.001:
                raise RuntimeError(f"minimax {kind}: no convergence at n = {n}, R = {Rn:.6g}")
            continue
        a, p, e, X = rn
        Rc = Rn
        f = min(2.0, f * f)
    return p, a, e


def minimax_grid(kind: str, n: int, e_min: float, e_max: float):
    """Physical grid for transition energies in [e_min, e_max]:
    time:      (tau_j = p_j / e_min, a_j / e_min, E / e_min)
    frequency: (omega_k = p_k e_min, b_k e_min,   E / e_min),
    so that 1/E ~ sum_j a_j exp(-tau_j E) or sum_k b_k E^2 / (E^2 + omega_k^2)^2
    within the returned maximum error for every E in [e_min, e_max]."""
    p, a, e = minimax_unit(kind, n, e_max / e_min)
    if kind == "T":
        return p / e_min, a / e_min, e / e_min
    return p * e_min, a * e_min, e / e_min


def _fit_x(e_min: float, e_max: float, m: int) -> np.ndarray:
    return e_min * (e_max / e_min) ** (np.arange(m) / (m - 1))


def transform_weights(tau, omega, e_min: float, e_max: float):
    """Least-squares transform weights for decaying exponentials exp(-x|tau|),
    x on 400 log-spaced energies of [e_min, e_max] (minimum-norm, singular
    values below 1e-14 of the largest dropped):
      gamma [n_omega, n_tau]: sum_j gamma_kj exp(-x tau_j) ~ 2x/(x^2 + omega_k^2)
      delta [n_tau, n_omega]: sum_k delta_jk 2x/(x^2 + omega_k^2) ~ exp(-x tau_j)
      s     [n_omega, n_tau]: sum_j s_kj exp(-x tau_j) ~ omega_k/(x^2 + omega_k^2)
    and the three fit errors (max deviation over 997 energies / max target)."""
    tau = np.asarray(tau, float)
    omega = np.asarray(omega, float)

    def parts(x):
        e = np.exp(-np.outer(x, tau))
        c = 2.0 * x[:, None] / (x[:, None] ** 2 + omega[None, :] ** 2)
        s = omega[None, :] / (x[:, None] ** 2 + omega[None, :] ** 2)
        return e, c, s

    e, c, s = parts(_fit_x(e_min, e_max, 400))
    gamma = np.linalg.lstsq(e, c, rcond=1e-14)[0].T
    delta = np.linalg.lstsq(c, e, rcond=1e-14)[0].T
    sw = np.linalg.lstsq(e, s, rcond=1e-14)[0].T
    e, c, s = parts(_fit_x(e_min, e_max, 997))
    err = np.array([np.abs(e @ gamma.T - c).max() / np.abs(c).max(),
                    np.abs(c @ delta.T - e).max() / np.abs(e).max(),
                    np.abs(e @ sw.T - s).max() / np.abs(s).max()])
    return gamma, delta, sw, err
