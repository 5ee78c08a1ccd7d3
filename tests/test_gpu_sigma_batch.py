"""Batched self-energy (Eq. 10) over molecules of uneven size in one call:
each grouped product is one persistent tensor-core launch over every
(molecule, orbital) pair.  Per-molecule error against the block oracle, and
agreement with the one-molecule entry point."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import sigma as osg  # noqa: E402
from synth.chain_inputs import synthetic_w  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def _molecules(k):
    """k molecules of the 64-molecule set spread over its size range."""
    from synth import case_from_system, molecule_set

    mols = molecule_set(64, 10, 150, 20210425)
    order = np.argsort([m.n_atoms for m in mols])
    pick = sorted({int(order[int(round(x))]) for x in np.linspace(0, 40, k)})
    cases = [case_from_system(mols[i], 20, 1e-9, 20210425 + i) for i in pick]
    ws = [synthetic_w(c.system.nri_total, c.tau, 100 + i) for c, i in zip(cases, pick)]
    return cases, ws


@pytest.mark.parametrize("precision,tol", [("fp16x3", 1e-6), ("bf16x6", 1e-6), ("fp64", 1e-10)])
def test_batch_matches_oracle_per_molecule(pkg, precision, tol):
    from paper_2104_09857_gb300 import _lib

    cases, ws = _molecules(6)
    taus = [0, 9, 19]
    orbs = [[c.n_occ - 1, c.n_occ] for c in cases]
    ctxs = [pkg.Context(0) for _ in cases]
    try:
        for ctx, c in zip(ctxs, cases):
            ctx.load_case(c)
        got = _lib.gw_sigma_tau_batch([c.ctx for c in ctxs], ws, orbs, 1e-9, _lib.PRECISIONS[precision])
        one = ctxs[-1].sigma_tau(ws[-1], orbs[-1], 1e-9, precision=precision)
    finally:
        for ctx in ctxs:
            ctx.close()
    for c, w, o, g in zip(cases, ws, orbs, got):
        ref = osg.sigma_blocks(c, w, o, taus)
        err = np.abs(g[:, taus] - ref).max() / np.abs(ref).max()
        print(f"{precision} {c.system.name} ({c.system.n_atoms} atoms): error {err:.2e}")
        assert err <= tol, (c.system.name, err)
    # the batch and the one-molecule entry point agree
    assert np.abs(got[-1] - one).max() <= tol * np.abs(one).max()


def test_batch_rejects_mismatched_contexts(pkg):
    from paper_2104_09857_gb300 import _lib

    cases, ws = _molecules(2)
    a, b = pkg.Context(0), pkg.Context(0)
    try:
        a.load_case(cases[0])
        with pytest.raises(_lib.GwError) as e:  # b has no inputs
            _lib.gw_sigma_tau_batch([a.ctx, b.ctx], ws, [[0], [0]], 1e-9, _lib.GW_FP16X3)
        assert e.value.code == -2
        b.load_case(cases[1])
        with pytest.raises(_lib.GwError) as e:  # orbital out of range
            _lib.gw_sigma_tau_batch([a.ctx, b.ctx], ws, [[0], [10 ** 6]], 1e-9, _lib.GW_FP16X3)
        assert e.value.code == -1
    finally:
        a.close()
        b.close()
