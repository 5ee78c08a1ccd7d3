"""Inputs of the screening chain: frequency grid, cosine-transform weights and
the synthetic Coulomb matrix of the auxiliary basis.

* omega_k: log-spaced in [0.5 gap, 2 (eps_max - eps_min)], as many points as
  tau points.
* gamma[k][j] (tau -> i omega): least-squares weights with
      sum_j gamma_kj exp(-x tau_j) ~= 2x / (x^2 + omega_k^2)
  for x on a log grid over [gap, eps_max - eps_min] -- the transform of one
  decaying exponential, exp(-x|tau|), which is what every term of chi(i tau)
  is (the approach of minimax-type time/frequency grids).
* delta[j][k] (i omega -> tau): least-squares weights with
      sum_k delta_jk 2x / (x^2 + omega_k^2) ~= exp(-x tau_j)
  over the same x.
* s[k][j] (half-line sine transform, for the self-energy): least-squares
  weights with sum_j s_kj exp(-x tau_j) ~= omega_k / (x^2 + omega_k^2).
* V_PQ = 1 / sqrt(r_PQ^2 + 1 A^2) + 1.0 delta_PQ over the RI-function centres:
  a regularised Coulomb kernel (positive Fourier transform, hence positive
  semidefinite) plus a diagonal shift, so V is symmetric positive definite.

The weights are data for both sides of every comparison; their quadrature
error against the closed forms is reported by `fit_error`.
"""

from __future__ import annotations

import numpy as np


def omega_grid(n: int, gap: float, width: float) -> np.ndarray:
    lo, hi = 0.5 * gap, 2.0 * width
    if n == 1:
        return np.array([lo])
    return lo * (hi / lo) ** (np.arange(n) / (n - 1))


def _x_samples(gap: float, width: float, m: int = 400) -> np.ndarray:
    return gap * (width / gap) ** (np.arange(m) / (m - 1))


def transform_weights(tau: np.ndarray, omega: np.ndarray, gap: float, width: float):
    """(gamma [n_omega, n_tau], delta [n_tau, n_omega])."""
    x = _x_samples(gap, width)
    e = np.exp(-np.outer(x, tau))                                    # [m, n_tau]
    f = 2.0 * x[:, None] / (x[:, None] ** 2 + omega[None, :] ** 2)   # [m, n_omega]
    gamma = np.linalg.lstsq(e, f, rcond=1e-14)[0].T                  # [n_omega, n_tau]
    delta = np.linalg.lstsq(f, e, rcond=1e-14)[0].T                  # [n_tau, n_omega]
    return np.ascontiguousarray(gamma), np.ascontiguousarray(delta)


def fit_error(tau, omega, gamma, delta, gap, width) -> tuple[float, float]:
    """Max relative error of the two fitted transforms over the x range."""
    x = _x_samples(gap, width, 997)
    e = np.exp(-np.outer(x, tau))
    f = 2.0 * x[:, None] / (x[:, None] ** 2 + omega[None, :] ** 2)
    eg = np.abs(e @ gamma.T - f).max() / np.abs(f).max()
    ed = np.abs(f @ delta.T - e).max() / np.abs(e).max()
    return float(eg), float(ed)


def sine_weights(tau: np.ndarray, omega: np.ndarray, gap: float, width: float) -> np.ndarray:
    """s [n_omega, n_tau]: least-squares weights of the half-line sine
    transform, sum_j s_kj exp(-x tau_j) ~= omega_k / (x^2 + omega_k^2), for x
    on the same log grid over [gap, width] (the half-line cosine weights are
    gamma / 2)."""
    x = _x_samples(gap, width)
    e = np.exp(-np.outer(x, tau))
    f = omega[None, :] / (x[:, None] ** 2 + omega[None, :] ** 2)
    return np.ascontiguousarray(np.linalg.lstsq(e, f, rcond=1e-14)[0].T)


def sine_fit_error(tau, omega, s, gap, width) -> float:
    """Max relative error of the fitted sine transform over the x range."""
    x = _x_samples(gap, width, 997)
    e = np.exp(-np.outer(x, tau))
    f = omega[None, :] / (x[:, None] ** 2 + omega[None, :] ** 2)
    return float(np.abs(e @ s.T - f).max() / np.abs(f).max())


def coulomb_matrix(system) -> np.ndarray:
    centres = np.repeat(system.xyz, system.n_ri, axis=0)
    r2 = np.sum((centres[:, None, :] - centres[None, :, :]) ** 2, axis=2)
    v = 1.0 / np.sqrt(r2 + 1.0)
    v[np.diag_indices_from(v)] += 1.0
    return v


def synthetic_w(nri: int, tau: np.ndarray, seed: int) -> np.ndarray:
    """Seeded negative semidefinite W(tau_j) = -(R^T R / n_RI) exp(-0.1 tau_j),
    R [n_RI, n_RI] with N(0,1) entries: a stand-in screened interaction for
    self-energy tests that do not run the chain."""
    from .rng import normal_stream

    r = normal_stream(seed, 13, 0, nri * nri).reshape(nri, nri)
    w0 = -(r.T @ r) / nri
    return np.stack([w0 * np.exp(-0.1 * t) for t in tau])


def chain_inputs(case):
    """omega, gamma, delta and V for a synth Case."""
    eps = case.eps
    gap = float(eps[case.n_occ] - eps[case.n_occ - 1])
    width = float(eps[-1] - eps[0])
    omega = omega_grid(len(case.tau), gap, width)
    gamma, delta = transform_weights(case.tau, omega, gap, width)
    return omega, gamma, delta, coulomb_matrix(case.system), gap, width
