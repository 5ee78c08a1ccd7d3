"""Eigenvalue-self-consistent GW on the GPU (gw_evgw, FP64) against the
oracle (oracle/evgw.py).  It chains every GPU entry point (chi, the screening
chain, Sigma^x, Sigma^c, the quasiparticle step) cycle after cycle, so it is
the last file of the suite.

Inputs as in tests/test_oracle_evgw.py: benzene, 10 tau points, V scaled by
3e-4, vxc = Sigma^x.  The Pade step amplifies rounding about 1e5-fold and
each cycle feeds the last one's energies back, so the energies are compared
at 1e-6 Ha (0.03 meV)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from oracle import evgw as oe  # noqa: E402
from oracle import qp  # noqa: E402
from synth import make_case  # noqa: E402
from synth.chain_inputs import chain_inputs, sine_weights  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def _inputs():
    case = make_case("benzene", n_tau=10)
    omega, gamma, delta, v, gap, width = chain_inputs(case)
    s = sine_weights(case.tau, omega, gap, width)
    orbs = [case.n_occ - 1, case.n_occ]
    vc = 3e-4 * v
    sx = qp.sigma_x_dense(case, vc, orbs, thr=case.thr)
    return case, omega, gamma, delta, s, orbs, vc, sx


def test_evgw_matches_oracle_and_restores_levels(pkg):
    from paper_2104_09857_gb300 import _lib

    case, omega, gamma, delta, s, orbs, vc, sx = _inputs()
    ref, ref_cycles, ok, _ = oe.evgw(case, vc, omega, gamma, delta, s, orbs, sx, tol=1e-8)
    assert ok
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got, cycles = _lib.gw_evgw(ctx.ctx, vc, omega, gamma, delta, s, orbs, sx, case.thr,
                                   _lib.GW_FP64, 20, 1e-8)
        chi = ctx.chi_tau(case.thr, "fp64", 0, 1).cpu().numpy()
    print(f"evGW HOMO/LUMO {got} after {cycles} cycles; oracle {ref} after {ref_cycles}")
    assert abs(cycles - ref_cycles) <= 1
    assert np.max(np.abs(got - ref)) < 1e-6
    # the context is back on the levels given to gw_set_greens
    chi_ref = oc.chi_dense(case, tau_index=0)[0]
    assert np.linalg.norm(chi[0] - chi_ref) <= 1e-10 * np.linalg.norm(chi_ref)


def test_evgw_rejects_bad_input(pkg):
    from paper_2104_09857_gb300 import _lib

    case, omega, gamma, delta, s, orbs, vc, sx = _inputs()
    with pkg.Context(0) as ctx:
        with pytest.raises(_lib.GwError) as ei:
            _lib.gw_evgw(ctx.ctx, vc, omega, gamma, delta, s, orbs, sx, case.thr)
        assert ei.value.code == -2                       # no inputs set yet
        ctx.load_case(case)
        with pytest.raises(_lib.GwError) as ei:
            _lib.gw_evgw(ctx.ctx, vc, omega, gamma, delta, s, [0, 10_000], sx, case.thr)
        assert ei.value.code == -1                       # orbital out of range
        with pytest.raises(_lib.GwError) as ei:
            _lib.gw_evgw(ctx.ctx, vc, omega, gamma, delta, s, orbs, sx, case.thr, tol=0.0)
        assert ei.value.code == -1
