"""Quasiparticle step on the GPU (gw_qp_g0w0, FP64) against the oracle
(oracle/qp.py): transform of Sigma^c to imaginary frequency, Pade
continuation and the Newton solve of Eq. 12.  The Pade interpolant amplifies
input rounding ~1e5-fold (1e-15 relative perturbations of Sigma^c move the
energies by ~3e-10 Ha), so the two sides, which sum in different orders, are
compared at 1e-8 Ha."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import qp  # noqa: E402
from oracle import sigma as osg  # noqa: E402
from synth import make_case  # noqa: E402
from synth.chain_inputs import chain_inputs, omega_grid, sine_weights, synthetic_w, transform_weights  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def _pole_model(tau, amps, poles):
    sp = np.zeros_like(tau)
    sm = np.zeros_like(tau)
    for a, p in zip(amps, poles):
        if p < 0:
            sp += a * np.exp(p * tau)
        else:
            sm -= a * np.exp(-p * tau)
    return np.stack([sp, sm], axis=-1)


def test_qp_pole_models_match_oracle_and_closed_form(pkg):
    from paper_2104_09857_gb300 import _lib

    gap, width = 0.3, 2.0
    tau = 0.01 * 5000.0 ** (np.arange(20) / 19)
    omega = omega_grid(20, gap, width)
    gamma, _ = transform_weights(tau, omega, gap, width)
    s = sine_weights(tau, omega, gap, width)
    models = [([0.03, 0.05], [-1.0, 1.1]), ([0.02], [-0.8]), ([0.04, 0.01, 0.03], [-1.5, 0.9, 1.6])]
    sig = np.stack([_pole_model(tau, a, p) for a, p in models])
    eps = np.array([-0.2, -0.1, 0.25])
    vxc = np.array([-0.3, -0.2, -0.1])
    sx = np.array([-0.25, -0.3, -0.05])
    with pkg.Context(0) as ctx:
        got, it = _lib.gw_qp_g0w0(ctx.ctx, sig, omega, gamma, s, eps, vxc, sx)
    ref = qp.quasiparticle_energies(sig, omega, gamma, s, eps, vxc, sx)
    assert np.max(np.abs(got - ref)) < 1e-8
    assert np.all((it > 0) & (it < 100))
    for b, (a, p) in enumerate(models):
        exact = qp.qp_newton(eps[b], vxc[b], sx[b],
                             lambda x: float(sum(ai / (x - pi) for ai, pi in zip(a, p))))[0]
        assert abs(got[b] - exact) < 1e-6


def test_qp_from_benzene_self_energy(pkg):
    """HOMO and LUMO of benzene: Sigma^c(+-i tau) and Sigma^x (Eq. 11) from the
    oracle with a synthetic W (scaled to ~0.1 Ha), then the GPU step."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("benzene", n_tau=10)
    omega, gamma, _, v, gap, width = chain_inputs(case)
    s = sine_weights(case.tau, omega, gap, width)
    w = 1e-3 * synthetic_w(case.system.nri_total, case.tau, 9)
    orbs = [case.n_occ - 1, case.n_occ]
    sig = osg.sigma_dense(case, w, orbs, thr=case.thr)
    sx = qp.sigma_x_dense(case, 1e-3 * v, orbs, thr=case.thr)
    eps = case.eps[orbs]
    vxc = 0.5 * eps
    with pkg.Context(0) as ctx:
        got, _ = _lib.gw_qp_g0w0(ctx.ctx, sig, omega, gamma, s, eps, vxc, sx)
    ref = qp.quasiparticle_energies(sig, omega, gamma, s, eps, vxc, sx)
    assert np.max(np.abs(got - ref)) < 1e-8


def test_qp_rejects_bad_input(pkg):
    from paper_2104_09857_gb300 import _lib

    sig = np.zeros((1, 4, 2))
    w = np.ones((3, 4))
    with pkg.Context(0) as ctx:
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_qp_g0w0(ctx.ctx, sig, [0.1, 0.1, 0.5], w, w, [0.0], [0.0], [0.0])
        assert e.value.code == -1
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_qp_g0w0(ctx.ctx, sig, [0.1, 0.2, 0.5], w, w, [np.nan], [0.0], [0.0])
        assert e.value.code == -4
        # the first frequency is checked like the others
        for om in ([0.0, 0.2, 0.5], [-0.1, 0.2, 0.5]):
            with pytest.raises(_lib.GwError) as e:
                _lib.gw_qp_g0w0(ctx.ctx, sig, om, w, w, [0.0], [0.0], [0.0])
            assert e.value.code == -1


def test_qp_reports_a_newton_solve_that_does_not_converge(pkg):
    """A self-energy that is the same at every frequency point leaves the
    continued fraction's third coefficient 0/0: the Newton solve meets a
    non-finite value and the call says so (GW_ERR_NOT_CONVERGED) instead of
    returning the iterate as an energy."""
    from paper_2104_09857_gb300 import _lib

    sig = np.ones((1, 1, 2))              # S+ = S- = 1 on one tau point
    gamma = np.full((4, 1), 0.2)          # Sigma(i omega_k) = 0.2 for every k
    sw = np.zeros((4, 1))
    with pkg.Context(0) as ctx:
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_qp_g0w0(ctx.ctx, sig, [0.1, 0.3, 0.7, 1.5], gamma, sw, [0.0], [0.0], [0.0])
        assert e.value.code == -10
        assert "did not converge" in str(e.value)


@pytest.mark.parametrize("name,precision,tol", [("benzene", "fp64", 1e-10), ("ribbon28", "fp64", 1e-10),
                                                ("ribbon28", "fp16x3", 1e-6)])
def test_sigma_x_matches_oracle(pkg, name, precision, tol):
    """Eq. 11 through gw_sigma_x against the oracle's dense route."""
    from paper_2104_09857_gb300 import _lib

    case = make_case(name, n_tau=2)
    _, _, _, v, _, _ = chain_inputs(case)
    orbs = [case.n_occ - 2, case.n_occ - 1, case.n_occ]
    ref = qp.sigma_x_dense(case, v, orbs, thr=case.thr)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got = _lib.gw_sigma_x(ctx.ctx, v, orbs, case.thr, _lib.PRECISIONS[precision])
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
