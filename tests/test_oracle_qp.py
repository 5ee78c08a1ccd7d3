"""Pins of the post-self-energy oracle (oracle/qp.py) against closed forms:
Pade interpolation and exact reproduction of rational functions, the
transform of a pole model, the quadratic root of the quasiparticle equation
for one pole, and Eq. 11 against its MO route."""

import numpy as np
import pytest

from oracle import chi as oc
from oracle import qp
from synth import make_case
from synth.chain_inputs import omega_grid, sine_fit_error, sine_weights, transform_weights


def _poles(z, amps, poles):
    return sum(a / (z - p) for a, p in zip(amps, poles))


def test_pade_interpolates_its_nodes():
    rng = np.random.default_rng(1)
    z = 1j * np.linspace(0.1, 3.0, 9)
    u = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    a = qp.pade_coefficients(z, u)
    assert np.allclose(qp.pade_eval(z, a, z), u, rtol=1e-10, atol=0)


@pytest.mark.parametrize("n_nodes", [7, 12])
def test_pade_reproduces_a_rational_function(n_nodes):
    """Three simple poles on the real axis: a [2/3] rational function, fixed
    by 6 values; Thiele's fraction through 7 or more points on the imaginary
    axis reproduces it on the real axis."""
    amps, poles = [0.7, -0.3, 1.1], [-0.9, 0.4, 1.7]
    z = 1j * np.geomspace(0.05, 4.0, n_nodes)
    a = qp.pade_coefficients(z, _poles(z, amps, poles))
    x = np.array([-1.5, -0.3, 0.1, 0.9, 1.3, 2.5])
    got = qp.pade_eval(z, a, x)
    ref = _poles(x, amps, poles)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-8


def test_transform_of_a_pole_model():
    """S+(tau) = a e^{p tau} (p < 0) and S-(tau) = -a e^{-p tau} (p > 0) give
    Sigma(i omega) = sum a / (i omega - p) up to the quadrature fit error."""
    gap, width = 0.3, 2.0
    tau = 0.01 * 5000.0 ** (np.arange(20) / 19)
    omega = omega_grid(20, gap, width)
    gamma, _ = transform_weights(tau, omega, gap, width)
    s = sine_weights(tau, omega, gap, width)
    amps, poles = [0.4, -0.25, 0.6], [-0.5, -1.2, 0.8]
    sp = sum(a * np.exp(p * tau) for a, p in zip(amps, poles) if p < 0)
    sm = sum(-a * np.exp(-p * tau) for a, p in zip(amps, poles) if p > 0)
    got = qp.tau_to_omega(sp, sm, gamma, s)
    ref = _poles(1j * omega, amps, poles)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 1e-6  # measured 1.5e-8
    assert sine_fit_error(tau, omega, s, gap, width) < 1e-6  # measured 3e-8


def test_qp_newton_single_pole_closed_form():
    """Re Sigma^c(e) = a / (e - p): e - e0 - a / (e - p) = 0 is a quadratic;
    Newton from eps_n reaches its root on eps_n's side of the pole."""
    eps_n, vxc, sx, a, p = -0.4, -0.35, -0.6, 0.05, 0.9
    e0 = eps_n - vxc + sx
    e, it = qp.qp_newton(eps_n, vxc, sx, lambda x: a / (x - p))
    roots = np.roots([1.0, -(e0 + p), e0 * p - a]).real
    ref = roots[np.argmin(np.abs(roots - e0))]
    assert abs(e - ref) < 1e-10
    assert it < 30


def test_qp_pipeline_on_a_pole_model():
    """tau -> i omega -> Pade -> Newton on a two-pole self-energy reproduces
    the quasiparticle energy of the exact pole model."""
    gap, width = 0.3, 2.0
    tau = 0.01 * 5000.0 ** (np.arange(20) / 19)
    omega = omega_grid(20, gap, width)
    gamma, _ = transform_weights(tau, omega, gap, width)
    s = sine_weights(tau, omega, gap, width)
    amps, poles = [0.03, 0.05], [-1.0, 1.1]
    sp = sum(a * np.exp(p * tau) for a, p in zip(amps, poles) if p < 0)
    sm = sum(-a * np.exp(-p * tau) for a, p in zip(amps, poles) if p > 0)
    sig = np.stack([sp, sm], axis=-1)[None]
    eps, vxc, sx = np.array([-0.2]), np.array([-0.3]), np.array([-0.25])
    got = qp.quasiparticle_energies(sig, omega, gamma, s, eps, vxc, sx)[0]
    ref = qp.qp_newton(eps[0], vxc[0], sx[0], lambda x: float(_poles(x, amps, poles)))[0]
    assert abs(got - ref) < 1e-7  # measured 2e-9


@pytest.mark.parametrize("name", ["chain_CHCH", "benzene"])
def test_sigma_x_ao_route_matches_mo_route(name):
    case = make_case(name, n_tau=1, thr=0.0) if name == "benzene" else make_case(name, n_tau=1)
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data, 0.0)
    rng = np.random.default_rng(4)
    r = rng.standard_normal((s.nri_total, s.nri_total))
    v = r @ r.T / s.nri_total + np.eye(s.nri_total)
    orbs = [case.n_occ - 1, case.n_occ]
    got = qp.sigma_x_dense(case, v, orbs, thr=0.0)
    ref = [qp.sigma_x_mo(t, case.C, case.n_occ, n, v) for n in orbs]
    assert np.allclose(got, ref, rtol=1e-11, atol=0)
    assert np.all(got < 0)  # V positive definite: exchange lowers every level
