"""Parity at the benchmark's full size (298-atom ribbon, 3090 AO / 7176 RI,
thr 1e-9), in the configuration bench.py times: chi(i tau) on sampled atom
blocks that the block oracle computes one by one (the dense oracle is out of
reach at this size).

Every tau point of the grid is checked.  At tau index j the sample is the
5 x 5 atom blocks (p, q) of an atom set S_j (25 blocks, 5 of them diagonal);
the sets are consecutive runs of one seeded permutation of the atoms, so the
20 tau points cover 100 different atoms and 500 blocks.  The FP64 form is
checked on three of the tau points with the same samples."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402

SET = 5
FP64_TAUS = (0, 10, 19)


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as pkg

    case = make_case("ribbon300")
    bo = oc.BlockOracle(case)
    perm = np.random.default_rng(20210420).permutation(case.system.n_atoms)
    sets = [sorted(int(a) for a in perm[SET * j:SET * (j + 1)]) for j in range(len(case.tau))]
    refs = {}
    return pkg, case, bo, sets, refs


def _pairs(atoms):
    return [(p, q) for p in atoms for q in atoms]


def _reference(bo, refs, j, atoms):
    """Oracle blocks at tau index j, computed once per module."""
    if j not in refs:
        cache = {}
        refs[j] = [bo.block(j, p, q, cache) for p, q in _pairs(atoms)]
    return refs[j]


def _blocks(chi, ri, pairs):
    return [chi[ri[p]:ri[p + 1], ri[q]:ri[q + 1]].cpu().numpy() for p, q in pairs]


def _errors(got_blocks, ref_blocks):
    num = sum(np.sum((g - r) ** 2) for g, r in zip(got_blocks, ref_blocks))
    den = sum(np.sum(r ** 2) for r in ref_blocks)
    mx = max(np.abs(r).max() for r in ref_blocks)
    err = max(np.abs(g - r).max() for g, r in zip(got_blocks, ref_blocks))
    assert den > 0.0
    return float(np.sqrt(num / den)), float(err / mx)


@pytest.mark.parametrize("precision", ["fp16x3"])
def test_mixed_full_size_every_tau(setup, precision):
    """All 20 tau points of the timed form in one call, 25 sampled blocks each:
    relative Frobenius and element-wise errors <= 1e-6 at every tau."""
    pkg, case, bo, sets, refs = setup
    ri = oc.offsets(case.system.n_ri)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, precision)
        got = [_blocks(chi[j], ri, _pairs(sets[j])) for j in range(len(case.tau))]
        # exact mirror across atom blocks
        p, q = sets[0][0], sets[0][-1]
        assert torch.equal(chi[0, ri[p]:ri[p + 1], ri[q]:ri[q + 1]],
                           chi[0, ri[q]:ri[q + 1], ri[p]:ri[p + 1]].T)
        del chi
    worst = 0.0
    for j in range(len(case.tau)):
        rel, el = _errors(got[j], _reference(bo, refs, j, sets[j]))
        print(f"{precision} tau[{j}] atoms {sets[j]}: rel Frobenius {rel:.2e}, element {el:.2e}")
        assert rel <= 1e-6, f"tau index {j}: relative Frobenius error {rel:.3e}"
        assert el <= 1e-6, f"tau index {j}: element error {el:.3e} of max |chi|"
        worst = max(worst, rel, el)
    print(f"{precision}: worst sampled error over 20 tau points {worst:.2e}")


@pytest.mark.parametrize("j", FP64_TAUS)
def test_fp64_full_size_sampled_blocks(setup, j):
    """The plain FP64 GPU form on three tau points of the full workload."""
    pkg, case, bo, sets, refs = setup
    ri = oc.offsets(case.system.n_ri)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, "fp64", j, 1)[0]
        got = _blocks(chi, ri, _pairs(sets[j]))
        st = ctx.stats()
    rel, el = _errors(got, _reference(bo, refs, j, sets[j]))
    print(f"fp64 tau[{j}]: rel Frobenius {rel:.2e}, element {el:.2e}")
    assert rel <= 1e-10 and el <= 1e-10
    # the useful-flop count equals the oracle's own count where one was taken
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "flops_ribbon298.json")
    golden = json.load(open(path))["per_tau"].get(str(j))
    if golden is not None:
        for k in ("flops_a", "flops_b", "flops_c"):
            assert st[k] == pytest.approx(golden[k], rel=1e-12), (k, st[k], golden[k])
