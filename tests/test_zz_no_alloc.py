"""The allocation-free chi entry point (gw_chi_tau_noalloc) against the
regular one (gw_chi_tau, FP64) and against the CPU oracle, called twice in a
row through the C ABI, with the device's free memory unchanged across calls.

It exists for callers that cannot call cudaMalloc when they need chi (a host
framework whose caching allocator owns the device memory budget, a process
that reserved all device memory up front, latency-bound code that cannot
afford cudaMalloc's implicit synchronisation): its work buffers live in one
fixed array inside the library.  Kept in a file of its own that pytest
collects last.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402

TOL = 1e-10  # the FP64 tolerance of the parity tests


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,thr", [("benzene", 0.0), ("ribbon28", 1e-9), ("ribbon28", 1e-3)])
def test_noalloc_matches_chi_tau_twice(pkg, name, thr):
    from paper_2104_09857_gb300 import _lib

    case = make_case(name, n_tau=4)
    oracle = oc.chi_dense(case, thr=thr)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        ref = ctx.chi_tau(thr, "fp64").cpu().numpy()
        out = torch.full((ctx.nri, ctx.nri), float("nan"), dtype=torch.float64, device="cuda:0")
        _lib.gw_chi_tau_noalloc(ctx.ctx, 0, thr, out.data_ptr())  # first call: address look-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        for j in (1, 2):
            for _ in range(2):
                _lib.gw_chi_tau_noalloc(ctx.ctx, j, thr, out.data_ptr())
                got = out.cpu().numpy()
                assert np.all(np.isfinite(got))
                for want in (ref[j], oracle[j]):
                    assert _rel(got, want) <= TOL
                    assert np.abs(got - want).max() <= TOL * np.abs(want).max()
                out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(0)[0] == free0, "device memory was allocated"


def test_noalloc_requires_panels_and_rejects_bad_arguments(pkg):
    from paper_2104_09857_gb300 import _lib

    case = make_case("chain_CH")
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        out = torch.zeros((ctx.nri, ctx.nri), dtype=torch.float64, device="cuda:0")
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_chi_tau_noalloc(ctx.ctx, 0, 0.0, out.data_ptr())
        assert e.value.code == -2
        # the tensor-core route builds no FP64 panels
        ctx.chi_tau(0.0, "fp16x3", 0, 1)
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_chi_tau_noalloc(ctx.ctx, 0, 0.0, out.data_ptr())
        assert e.value.code == -2
        ctx.chi_tau(0.0, "fp64", 0, 1)
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_chi_tau_noalloc(ctx.ctx, 99, 0.0, out.data_ptr())
        assert e.value.code == -1
        _lib.gw_chi_tau_noalloc(ctx.ctx, 0, 0.0, out.data_ptr())


def test_noalloc_rejects_system_too_large(pkg):
    """A system whose work does not fit the fixed array is refused cleanly."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("ribbon120", n_tau=1)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        out = ctx.chi_tau(case.thr, "fp64")
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_chi_tau_noalloc(ctx.ctx, 0, case.thr, out.data_ptr())
        assert e.value.code == -1
        assert "MiB" in str(e.value)
