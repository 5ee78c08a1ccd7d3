"""Oracle for the steps after the self-energy: the exchange self-energy of
Eq. 11, the transform of Sigma^c_n(+-i tau) to imaginary frequency by a cosine
and a sine transform, the analytic continuation to the real axis by a Pade
interpolant, and the Newton-Raphson solve of the quasiparticle equation,
Eq. 12.  FP64 / complex128 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* Fourier convention: Sigma(i omega) = int dtau e^{-i omega tau} Sigma(i tau)
  with the real representation of the self-energy oracle, S+(tau) =
  Sigma^c_n(i tau) (occupied side) and S-(tau) = Sigma^c_n(-i tau) (virtual
  side), tau > 0.  Hence
      Sigma(i omega) = int_0^inf cos(omega tau) [S+ + S-] dtau
                     - i int_0^inf sin(omega tau) [S+ - S-] dtau,
  and one pole a / (z - p) is S+(tau) = a e^{p tau} for p < 0 and
  S-(tau) = -a e^{-p tau} for p > 0.
* Quadrature: half-line cosine weights gamma / 2 (gamma fits the full-line
  transform of e^{-x|tau|}) and fitted half-line sine weights
  (synth.chain_inputs.sine_weights): data for both sides.
* Pade interpolant: Thiele's continued fraction through all N points
  (z_k = i omega_k), its coefficients by the Vidberg-Serene recursion
      g_1(z_i) = u_i,
      g_p(z) = (g_{p-1}(z_{p-1}) - g_{p-1}(z)) / ((z - z_{p-1}) g_{p-1}(z)),
      a_p = g_p(z_p),
      C(z) = a_1 / (1 + a_2 (z - z_1) / (1 + a_3 (z - z_2) / (1 + ...))).
  Real-axis values at z = eps (eta = 0).
* Exchange (Eq. 11) with the RI metric S = 1: Sigma^x_n = -sum D_{mu nu}
  B^n_{mu P} V_PQ B^n_{nu Q}, D = C_occ C_occ^T, filtered like Eq. 10.
* Quasiparticle equation: eps = eps_n - vxc_n + Sigma^x_n + Re Sigma^c_n(eps),
  Newton steps with the derivative of Re Sigma^c by central differences,
  starting at eps_n.  vxc_n is an input (no DFT here).
"""

from __future__ import annotations

import numpy as np

from . import chi as oc
from . import sigma as osg


def tau_to_omega(s_plus: np.ndarray, s_minus: np.ndarray, gamma: np.ndarray,
                 s_weights: np.ndarray) -> np.ndarray:
    """Sigma(i omega_k) [.., n_omega] from S+(tau_j), S-(tau_j) [.., n_tau]."""
    even = s_plus + s_minus
    odd = s_plus - s_minus
    return even @ (0.5 * gamma).T - 1j * (odd @ s_weights.T)


def pade_coefficients(z: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Thiele continued-fraction coefficients a_1..a_N through (z_i, u_i)."""
    n = len(z)
    g = np.zeros((n, n), dtype=complex)
    g[0] = u
    for p in range(1, n):
        g[p, p:] = (g[p - 1, p - 1] - g[p - 1, p:]) / ((z[p:] - z[p - 1]) * g[p - 1, p:])
    return np.diag(g).copy()


def pade_eval(z: np.ndarray, a: np.ndarray, w):
    """The continued fraction at w (scalar or array), nodes z."""
    w = np.asarray(w, dtype=complex)
    acc = np.ones_like(w)
    for p in range(len(a) - 1, 0, -1):
        acc = 1.0 + a[p] * (w - z[p - 1]) / acc
    return a[0] / acc


def sigma_x_dense(case, v: np.ndarray, orbitals, thr: float | None = None) -> np.ndarray:
    """Sigma^x_n of Eq. 11 for the listed orbitals (dense route)."""
    sysm = case.system
    thr = case.thr if thr is None else thr
    ao = oc.offsets(sysm.n_ao)
    ri = oc.offsets(sysm.n_ri)
    t = oc.dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                              case.t3c.data, thr)
    c_occ = case.C[:, :case.n_occ]
    d = oc.filter_sym_2d(c_occ @ c_occ.T, ao, thr)
    out = np.zeros(len(orbitals))
    for a, n in enumerate(orbitals):
        b = osg.b_half(t, case.C, n)
        if thr > 0.0:
            nrm = np.sqrt(oc.block_sq_sums(b, [ao, ri]))
            keep = np.repeat(np.repeat(nrm >= thr, np.diff(ao), 0), np.diff(ri), 1)
            b = np.where(keep, b, 0.0)
        out[a] = -osg.s_term(d, b, v)
    return out


def sigma_x_mo(t: np.ndarray, C: np.ndarray, n_occ: int, n: int, v: np.ndarray) -> float:
    """MO route of Eq. 11 (unfiltered): -sum_{i occ} b_i^T V b_i with
    b_i[P] = sum_{mu nu} C_mu,i C_nu,n (mu nu | P)."""
    bm = np.einsum("um,vn,uvp->mp", C[:, :n_occ], C[:, [n]], t)
    return float(-np.einsum("mp,pq,mq->", bm, v, bm))


def qp_newton(eps_n: float, vxc_n: float, sx_n: float, re_sigma_c, max_iter: int = 100,
              tol: float = 1e-12, h: float = 1e-6) -> tuple[float, int]:
    """Root of e - (eps_n - vxc_n + sx_n + re_sigma_c(e)) by Newton-Raphson from
    eps_n; returns (e, iterations)."""
    e = float(eps_n)
    for it in range(1, max_iter + 1):
        f = e - (eps_n - vxc_n + sx_n + re_sigma_c(e))
        d = 1.0 - (re_sigma_c(e + h) - re_sigma_c(e - h)) / (2.0 * h)
        step = f / d
        e -= step
        if abs(step) < tol * max(1.0, abs(e)):
            return e, it
    return e, max_iter


def quasiparticle_energies(sig_c_tau: np.ndarray, omega: np.ndarray, gamma: np.ndarray,
                           s_weights: np.ndarray, eps: np.ndarray, vxc: np.ndarray,
                           sx: np.ndarray) -> np.ndarray:
    """G0W0 energies of Eq. 12 for the orbitals whose Sigma^c_n(+-i tau) are
    given ([n_orb][n_tau][2], the layout of the self-energy oracle)."""
    sig_w = tau_to_omega(sig_c_tau[:, :, 0], sig_c_tau[:, :, 1], gamma, s_weights)
    z = 1j * omega
    out = np.zeros(len(eps))
    for a in range(len(eps)):
        coef = pade_coefficients(z, sig_w[a])
        out[a] = qp_newton(eps[a], vxc[a], sx[a], lambda e: float(pade_eval(z, coef, e).real))[0]
    return out
