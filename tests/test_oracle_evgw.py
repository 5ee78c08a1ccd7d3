"""Pins of the evGW oracle (oracle/evgw.py): the level update by hand, the
first cycle against G0W0 composed from the pinned oracle steps, the
zero-coupling limit, and the fixed point the loop stops at.

Inputs: benzene, 10 tau points, V scaled by c (the synthetic 3c tensor has
unit-normal entries, so c = 3e-4 gives quasiparticle shifts of a few mHa) and
vxc = Sigma^x (a mean field that already holds exchange)."""

import numpy as np
import pytest

from oracle import chain as och
from oracle import chi as oc
from oracle import evgw as oe
from oracle import qp
from oracle import sigma as osg
from synth import make_case
from synth.chain_inputs import chain_inputs, sine_weights


@pytest.fixture(scope="module")
def setup():
    case = make_case("benzene", n_tau=10)
    omega, gamma, delta, v, gap, width = chain_inputs(case)
    s = sine_weights(case.tau, omega, gap, width)
    orbs = [case.n_occ - 1, case.n_occ]
    return case, omega, gamma, delta, v, s, orbs


def test_level_update_by_hand():
    eps = np.array([-3.0, -2.0, -1.0, 1.0, 2.0, 3.0])
    # HOMO-1 and LUMO computed: the occupied side moves with HOMO-1, the
    # virtual side with the LUMO
    got = oe.shifted_levels(eps, 3, [1, 3], [-2.5, 1.2])
    np.testing.assert_array_equal(got, [-3.5, -2.5, -1.5, 1.2, 2.2, 3.2])
    # occupied 0 and 2 computed: 1 is equally far from both and follows 2
    got = oe.shifted_levels(eps, 3, [0, 2, 4], [-3.1, -0.8, 2.5])
    np.testing.assert_allclose(got, [-3.1, -1.8, -0.8, 1.5, 2.5, 3.5], rtol=0, atol=1e-15)
    # virtual 3 and 5 computed: 4 follows 3
    got = oe.shifted_levels(eps, 3, [3, 5], [1.1, 3.3])
    np.testing.assert_allclose(got, [-3.0, -2.0, -1.0, 1.1, 2.1, 3.3], rtol=0, atol=1e-15)


def test_first_cycle_is_g0w0(setup):
    case, omega, gamma, delta, v, s, orbs = setup
    vc = 3e-4 * v
    sx = qp.sigma_x_dense(case, vc, orbs, thr=case.thr)
    chi = oc.chi_dense(case)
    w_tau, _ = och.chi_to_w(chi, vc, gamma, delta)
    sig = osg.sigma_dense(case, w_tau, orbs, thr=case.thr)
    g0w0 = qp.quasiparticle_energies(sig, omega, gamma, s, case.eps[orbs], sx, sx)
    e, cycles, converged, _ = oe.evgw(case, vc, omega, gamma, delta, s, orbs, sx, max_cycles=1)
    assert cycles == 1 and not converged
    np.testing.assert_array_equal(e, g0w0)


def test_weak_coupling_limit(setup):
    """V -> cV, c -> 0: Sigma^x = vxc cancels, and W^c = L(eps^-1 - 1)L^T
    with eps = 1 - c L^T chi L is c^2 V chi V + O(c^3), so the shifts from
    eps_n vanish like c^2 (ratio 100 between c = 1e-6 and 1e-7) and the
    second cycle already confirms them."""
    case, omega, gamma, delta, v, s, orbs = setup
    shifts = []
    for c in (1e-6, 1e-7):
        vc = c * v
        sx = qp.sigma_x_dense(case, vc, orbs, thr=case.thr)
        e, cycles, converged, _ = oe.evgw(case, vc, omega, gamma, delta, s, orbs, sx, tol=1e-12)
        assert converged and cycles <= 3
        shifts.append(e - case.eps[orbs])
    assert np.max(np.abs(shifts[1])) < 1e-8
    np.testing.assert_allclose(shifts[0] / shifts[1], 100.0, rtol=0.02)


def test_converged_energies_are_a_fixed_point(setup):
    """At convergence one more cycle, built from the levels the result
    implies, returns the same energies; the gap moved away from G0W0's."""
    case, omega, gamma, delta, v, s, orbs = setup
    vc = 3e-4 * v
    sx = qp.sigma_x_dense(case, vc, orbs, thr=case.thr)
    tol = 1e-8
    e, cycles, converged, _ = oe.evgw(case, vc, omega, gamma, delta, s, orbs, sx, tol=tol)
    assert converged and 2 < cycles < 20
    again = oe.gw_cycle(case, oe.shifted_levels(case.eps, case.n_occ, orbs, e), vc, omega, gamma,
                        delta, s, orbs, sx, sx)
    assert np.max(np.abs(again - e)) < 10 * tol
    g0w0 = oe.gw_cycle(case, case.eps, vc, omega, gamma, delta, s, orbs, sx, sx)
    assert np.max(np.abs(e - g0w0)) > 1e-5
    assert e[0] < 0.0 < e[1]                   # HOMO below, LUMO above mu_F = 0
