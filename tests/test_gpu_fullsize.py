"""Parity at the benchmark's full size (298-atom ribbon, 3090 AO / 7176 RI,
thr 1e-9), in the configuration bench.py times: chi(i tau) for one tau point
per call, compared on sampled atom blocks that the block oracle computes one
by one (the dense oracle is out of reach at this size)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402

# (p-atom, q-atom) samples: both ribbon ends, the middle, diagonal and
# off-diagonal blocks, near and far
PAIRS = [(0, 0), (0, 5), (3, 60), (149, 149), (149, 170), (149, 40), (120, 260), (297, 297),
         (297, 280), (200, 150)]


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as pkg

    case = make_case("ribbon300")
    bo = oc.BlockOracle(case)
    return pkg, case, bo


def _blocks(chi, ri, pairs):
    return [chi[ri[p]:ri[p + 1], ri[q]:ri[q + 1]] for p, q in pairs]


def _compare(got_blocks, ref_blocks, tol):
    num = sum(np.sum((g - r) ** 2) for g, r in zip(got_blocks, ref_blocks))
    den = sum(np.sum(r ** 2) for r in ref_blocks)
    rel = np.sqrt(num / den)
    mx = max(np.abs(r).max() for r in ref_blocks)
    err = max(np.abs(g - r).max() for g, r in zip(got_blocks, ref_blocks))
    assert rel <= tol, f"sampled relative Frobenius error {rel:.3e} > {tol}"
    assert err <= tol * mx, f"sampled element error {err:.3e} > {tol} * {mx:.3e}"
    return rel


@pytest.mark.parametrize("precision,tau_index", [("bf16x6", 3), ("bf16x6", 19), ("fp16x3", 3),
                                                 ("fp16x3", 19)])
def test_mixed_full_size_sampled_blocks(setup, precision, tau_index):
    pkg, case, bo = setup
    ri = oc.offsets(case.system.n_ri)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, precision, tau_index, 1)[0]
        got = [b.cpu().numpy() for b in _blocks(chi, ri, PAIRS)]
        # exact mirror across atom blocks
        p, q = PAIRS[5]
        assert torch.equal(chi[ri[p]:ri[p + 1], ri[q]:ri[q + 1]],
                           chi[ri[q]:ri[q + 1], ri[p]:ri[p + 1]].T)
    cache = {}
    ref = [bo.block(tau_index, p, q, cache) for p, q in PAIRS]
    _compare(got, ref, 1e-6)


def test_fp64_full_size_sampled_blocks(setup):
    """The plain FP64 GPU form on one tau point of the full workload."""
    pkg, case, bo = setup
    j = 19
    ri = oc.offsets(case.system.n_ri)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, "fp64", j, 1)[0]
        got = [b.cpu().numpy() for b in _blocks(chi, ri, PAIRS[:6])]
    cache = {}
    ref = [bo.block(j, p, q, cache) for p, q in PAIRS[:6]]
    _compare(got, ref, 1e-10)
