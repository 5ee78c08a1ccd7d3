"""Pins of the screening-chain oracle (cosine transforms, Eq. 7-9): library
factorisations, the closed-form transform of chi, and the sign and limit
properties of eps and W^c.  No GPU."""

import numpy as np
import pytest

from oracle import chain as och
from oracle import chi as oc
from synth import make_case
from synth.chain_inputs import chain_inputs, fit_error


@pytest.fixture(scope="module")
def benzene():
    case = make_case("benzene")
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data)
    chi = np.stack([oc.chi_mo_route(t, case.C, case.eps, case.n_occ, tau) for tau in case.tau])
    omega, gamma, delta, v, gap, width = chain_inputs(case)
    return dict(case=case, t=t, chi=chi, omega=omega, gamma=gamma, delta=delta, v=v, gap=gap,
                width=width)


def test_cholesky_and_solve_match_library(benzene):
    v = benzene["v"]
    low = och.cholesky_lower(v)
    assert np.allclose(low, np.linalg.cholesky(v), rtol=1e-12, atol=1e-13)
    assert np.allclose(low @ low.T, v, rtol=1e-12, atol=1e-12)
    b = np.random.default_rng(1).standard_normal(v.shape)
    assert np.allclose(och.solve_lower(low, b), np.linalg.solve(low, b), rtol=1e-10, atol=1e-12)
    with pytest.raises(ValueError):
        och.cholesky_lower(-v)


def test_cosine_transform_matches_closed_form(benzene):
    """chi(i omega) from the fitted weights against the exact transform of the
    MO route, within the fitted kernel's own error."""
    b = benzene
    eg, ed = fit_error(b["case"].tau, b["omega"], b["gamma"], b["delta"], b["gap"], b["width"])
    assert eg < 1e-3 and ed < 1e-3
    cw = och.chi_to_omega(b["chi"], b["gamma"])
    for k, w in enumerate(b["omega"]):
        exact = och.chi_omega_closed_form(b["t"], b["case"].C, b["case"].eps, b["case"].n_occ, w)
        assert np.linalg.norm(cw[k] - exact) <= 5 * eg * np.linalg.norm(exact) + 1e-12


def test_epsilon_at_least_one_and_w_negative(benzene):
    b = benzene
    low = np.linalg.cholesky(b["v"])
    cw = och.chi_to_omega(b["chi"], b["gamma"])
    for c in cw:
        ev = np.linalg.eigvalsh(och.dielectric(c, low))
        assert ev.min() >= 1.0 - 1e-10
        w = och.wc_omega(c, low)
        assert np.abs(w - w.T).max() <= 1e-10 * np.abs(w).max()
        assert np.linalg.eigvalsh(0.5 * (w + w.T)).max() <= 1e-10 * np.abs(w).max()


def test_zero_chi_gives_zero_w_and_small_chi_limit(benzene):
    """chi = 0 -> W^c = 0; for small chi, W^c = V chi V + O(chi^2)."""
    b = benzene
    v = b["v"]
    low = och.cholesky_lower(v)
    n = v.shape[0]
    w0 = och.wc_omega(np.zeros((n, n)), low)
    assert np.abs(w0).max() <= 1e-12 * np.abs(v).max()
    c = b["chi"][0] / np.abs(b["chi"][0]).max()
    errs = []
    for s in (1e-3, 1e-4):
        lin = v @ (s * c) @ v
        errs.append(np.linalg.norm(och.wc_omega(s * c, low) - lin) / np.linalg.norm(lin))
    assert errs[1] < errs[0] / 5.0  # the remainder is second order
    assert errs[1] < 1e-2


def test_inverse_transform_roundtrip(benzene):
    """The two fitted transforms invert each other on exponentials."""
    b = benzene
    tau = b["case"].tau
    x = 0.9
    f_tau = np.exp(-x * tau)[:, None, None] * np.ones((1, 2, 2))
    back = och.omega_to_tau(och.chi_to_omega(f_tau, b["gamma"]), b["delta"])
    assert np.allclose(back[:, 0, 0], f_tau[:, 0, 0], rtol=5e-3, atol=5e-4)


def test_chain_end_to_end_shapes_and_sign(benzene):
    b = benzene
    w_tau, w_w = och.chi_to_w(b["chi"], b["v"], b["gamma"], b["delta"])
    assert w_tau.shape == b["chi"].shape and w_w.shape[0] == len(b["omega"])
    assert np.all(np.isfinite(w_tau))
    # every W^c(i omega) is negative semidefinite
    for w in w_w:
        assert np.linalg.eigvalsh(0.5 * (w + w.T)).max() <= 1e-10 * np.abs(w).max()


def test_apply_metric_pins():
    """S^-1 M S^-1: identity metric, diagonal metric in closed form, and the
    defining equation S X S = M for a random SPD metric."""
    from oracle import chain as och

    rng = np.random.default_rng(11)
    n = 24
    a = rng.standard_normal((n, n))
    m = a + a.T
    assert np.allclose(och.apply_metric(np.eye(n), m), m, rtol=0, atol=1e-13)
    d = rng.uniform(0.5, 2.0, n)
    assert np.allclose(och.apply_metric(np.diag(d), m), m / np.outer(d, d), rtol=1e-12, atol=0)
    b = rng.standard_normal((n, n))
    s = b @ b.T / n + np.eye(n)
    x = och.apply_metric(s, m)
    assert np.allclose(s @ x @ s, m, rtol=0, atol=1e-10 * np.abs(m).max())
    assert np.allclose(x, x.T, rtol=0, atol=1e-12 * np.abs(x).max())
