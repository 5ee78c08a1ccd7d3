"""Oracle for the screening chain between chi(i tau) and W^c(i tau):
the cosine transform to imaginary frequency, the symmetric dielectric matrix
(Eq. 7) with the Cholesky factor of the Coulomb matrix (Eq. 8), its inverse by
Cholesky factorisation, the correlation part of the screened interaction
(Eq. 9), and the cosine transform back to imaginary time.  FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* The RI overlap metric S is the identity for the synthetic inputs (the
  tilde quantities of Eqs. 5-6 equal the plain ones); apply_metric forms
  S^-1 M S^-1 for a general symmetric positive definite S (chi~ of Eq. 5,
  W~ of Eq. 10, V~ of Eq. 11).
* chi here is real and negative semidefinite (chi^0 / i); eps = 1 - L^T chi L
  is then >= 1 and positive definite, as the paper requires of it.
* The transform weights gamma (tau -> omega) and delta (omega -> tau) are
  inputs, shared with the GPU path.
* The Cholesky factorisation and the triangular solves are written out as
  the textbook column algorithms; no LAPACK routine is used.
"""

from __future__ import annotations

import numpy as np


def cholesky_lower(a: np.ndarray) -> np.ndarray:
    """A = L L^T, L lower triangular (Cholesky-Banachiewicz, one column at a
    time).  Raises ValueError on a non-positive pivot."""
    n = a.shape[0]
    low = np.zeros_like(a)
    for j in range(n):
        d = a[j, j] - low[j, :j] @ low[j, :j]
        if not d > 0.0:
            raise ValueError(f"matrix not positive definite at pivot {j}")
        low[j, j] = np.sqrt(d)
        low[j + 1:, j] = (a[j + 1:, j] - low[j + 1:, :j] @ low[j, :j]) / low[j, j]
    return low


def solve_lower(low: np.ndarray, b: np.ndarray) -> np.ndarray:
    """X with L X = B, L lower triangular (forward substitution by rows)."""
    n = low.shape[0]
    x = np.zeros_like(b)
    for i in range(n):
        x[i] = (b[i] - low[i, :i] @ x[:i]) / low[i, i]
    return x


def chi_to_omega(chi_tau: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """chi(i omega_k) = sum_j gamma_kj chi(i tau_j)."""
    return np.einsum("kj,jpq->kpq", gamma, chi_tau)


def dielectric(chi_w: np.ndarray, low_v: np.ndarray) -> np.ndarray:
    """Eq. 7: eps = 1 - L^T chi L."""
    n = low_v.shape[0]
    return np.eye(n) - low_v.T @ chi_w @ low_v


def wc_omega(chi_w: np.ndarray, low_v: np.ndarray) -> np.ndarray:
    """Eq. 9: W^c = L (eps^-1 - 1) L^T, eps inverted through eps = R R^T:
    with Z = R^-1 L^T, L eps^-1 L^T = Z^T Z and L L^T = V."""
    eps = dielectric(chi_w, low_v)
    r = cholesky_lower(eps)
    z = solve_lower(r, low_v.T)
    return z.T @ z - low_v @ low_v.T


def omega_to_tau(w_omega: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """W(i tau_j) = sum_k delta_jk W(i omega_k)."""
    return np.einsum("jk,kpq->jpq", delta, w_omega)


def chi_to_w(chi_tau: np.ndarray, v: np.ndarray, gamma: np.ndarray, delta: np.ndarray):
    """The whole chain: (W^c(i tau) [n_tau], W^c(i omega) [n_omega])."""
    low = cholesky_lower(v)
    chi_w = chi_to_omega(chi_tau, gamma)
    w_w = np.stack([wc_omega(c, low) for c in chi_w])
    return omega_to_tau(w_w, delta), w_w


def chi_omega_closed_form(t: np.ndarray, C: np.ndarray, eps: np.ndarray, n_occ: int,
                          omega: float) -> np.ndarray:
    """Exact chi(i omega) = -sum_ia 2 D_ia / (D_ia^2 + omega^2) B^ia B^ia^T,
    D_ia = eps_a - eps_i, from the MO route of Eq. 3 (unfiltered)."""
    co = C[:, :n_occ]
    cv = C[:, n_occ:]
    b = np.einsum("li,lsp,sa->iap", co, t, cv, optimize=True)
    d = eps[None, n_occ:] - eps[:n_occ, None]
    w = 2.0 * d / (d * d + omega * omega)
    nb = b.shape[0] * b.shape[1]
    return -((b * w[:, :, None]).reshape(nb, -1).T @ b.reshape(nb, -1))


def apply_metric(s: np.ndarray, m: np.ndarray) -> np.ndarray:
    """S^-1 M S^-1 (Eq. 5 and the tilde quantities of Eqs. 10-11) through the
    Cholesky factor S = R R^T: S^-1 = R^-T R^-1."""
    r = cholesky_lower(s)
    rinv = solve_lower(r, np.eye(s.shape[0]))
    sinv = rinv.T @ rinv
    return sinv @ m @ sinv
