"""Parity of the diagonal self-energy (Eq. 10, gw_sigma_tau, FP64) with the
CPU oracle, and the whole chain chi -> W -> Sigma on one small system."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chain as och  # noqa: E402
from oracle import chi as oc  # noqa: E402
from oracle import sigma as osg  # noqa: E402
from synth import make_case  # noqa: E402
from synth.chain_inputs import chain_inputs, synthetic_w  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


@pytest.mark.parametrize("name,thr", [("chain_CHCH", 0.0), ("benzene", 0.0), ("ribbon28", 1e-9),
                                      ("ribbon28", 1e-3)])
def test_sigma_matches_oracle_synthetic_w(pkg, name, thr):
    case = make_case(name, n_tau=4)
    w = synthetic_w(case.system.nri_total, case.tau, 5)
    orbs = [case.n_occ - 1, case.n_occ, 0]
    ref = osg.sigma_dense(case, w, orbs, thr=thr)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got = ctx.sigma_tau(w, orbs, thr)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL * scale
    assert np.all(got[:, :, 0] >= -TOL * scale) and np.all(got[:, :, 1] <= TOL * scale)


def test_chi_w_sigma_chain_on_device(pkg):
    """chi (GPU) -> W^c (GPU chain) -> Sigma (GPU), all on the device, against
    the same composition of oracles."""
    case = make_case("benzene")
    omega, gamma, delta, v, _, _ = chain_inputs(case)
    orbs = [case.n_occ - 1, case.n_occ]
    chi_ref = oc.chi_dense(case)
    w_ref, _ = och.chi_to_w(chi_ref, v, gamma, delta)
    s_ref = osg.sigma_dense(case, w_ref, orbs)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, "fp64")
        w = ctx.chi_to_w(chi, v, gamma, delta)
        got = ctx.sigma_tau(w, orbs, case.thr)
    assert np.abs(got - s_ref).max() <= 1e-9 * np.abs(s_ref).max()


@pytest.mark.parametrize("name,precision", [("benzene", "bf16x6"), ("ribbon28", "bf16x6"),
                                            ("benzene", "fp16x3"), ("ribbon28", "fp16x3")])
def test_sigma_mixed_matches_oracle(pkg, name, precision):
    """The two products of Eq. 10 on the tensor cores (split bf16, 6 products,
    or scaled binary16, 3 products): within the 1e-6 mixed-precision bar of
    the oracle."""
    case = make_case(name, n_tau=3)
    w = synthetic_w(case.system.nri_total, case.tau, 9)
    orbs = [case.n_occ - 1, case.n_occ]
    ref = osg.sigma_dense(case, w, orbs, thr=case.thr)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got = ctx.sigma_tau(w, orbs, case.thr, precision=precision)
        fp64 = ctx.sigma_tau(w, orbs, case.thr, precision="fp64")
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-6 * scale
    assert np.abs(fp64 - ref).max() <= 1e-10 * scale


def test_uneven_molecule_set_mixed_and_fp64(pkg):
    """Self-energy (HOMO, LUMO) of molecules of uneven size drawn like the
    batched self-energy workload (rings and ribbon segments, 10-150 atoms,
    thr 1e-9): per-molecule error of BF16x6, FP16x3 and FP64 against the block oracle
    on three of the twenty tau points."""
    from synth import case_from_system, molecule_set

    mols = molecule_set(64, 10, 150, 20210425)
    sizes = np.array([m.n_atoms for m in mols])
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argsort(sizes)[32]),
            int(np.argsort(sizes)[16])]
    taus = [0, 9, 19]
    for i in pick:
        case = case_from_system(mols[i], 20, 1e-9, 20210425 + i)
        w = synthetic_w(case.system.nri_total, case.tau, 100 + i)
        orbs = [case.n_occ - 1, case.n_occ]
        ref = osg.sigma_blocks(case, w, orbs, taus)
        with pkg.Context(0) as ctx:
            ctx.load_case(case)
            mixed = ctx.sigma_tau(w, orbs, case.thr, precision="bf16x6")[:, taus]
            half = ctx.sigma_tau(w, orbs, case.thr, precision="fp16x3")[:, taus]
            fp64 = ctx.sigma_tau(w, orbs, case.thr, precision="fp64")[:, taus]
        scale = np.abs(ref).max()
        e_mixed = np.abs(mixed - ref).max() / scale
        e_half = np.abs(half - ref).max() / scale
        e_fp64 = np.abs(fp64 - ref).max() / scale
        print(f"{case.system.name}: {case.system.n_atoms} atoms, bf16x6 err {e_mixed:.2e}, "
              f"fp16x3 err {e_half:.2e}, fp64 err {e_fp64:.2e}")
        assert e_mixed <= 1e-6
        assert e_half <= 1e-6
        assert e_fp64 <= 1e-10
