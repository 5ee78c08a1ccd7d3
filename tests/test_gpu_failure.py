"""Failure detection without a GPU fault: an injected never-met dependency in
the tensor-core kernels comes back as GW_ERR_TIMEOUT (bounded waits, about 2 s)
and an injected work-buffer allocation failure as GW_ERR_OOM; in both cases
the same context then computes chi correctly."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def _rel(got, ref):
    return max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(got, ref))


def test_injected_stall_times_out_and_context_recovers(pkg):
    from paper_2104_09857_gb300 import _lib

    case = make_case("benzene", n_tau=2)
    ref = oc.chi_dense(case)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        ctx.set_option("test_stall_tc", 1)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(case.thr, "fp16x3", 0, 1)
        assert e.value.code == -7  # GW_ERR_TIMEOUT
        ctx.set_option("test_stall_tc", 0)
        got = ctx.chi_tau(case.thr, "fp16x3").cpu().numpy()
    assert _rel(got, ref) <= 1e-6


def test_injected_allocation_failure_and_context_recovers(pkg):
    from paper_2104_09857_gb300 import _lib

    case = make_case("benzene", n_tau=2)
    ref = oc.chi_dense(case)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        ctx.set_option("test_fail_alloc", 1)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(case.thr, "fp64")
        assert e.value.code == -5  # GW_ERR_OOM
        assert "injected" in str(e.value)
        got = ctx.chi_tau(case.thr, "fp64").cpu().numpy()
    assert _rel(got, ref) <= 1e-10


def test_allocation_failure_during_panel_rebuild_leaves_no_stale_cache(pkg):
    """An injected allocation failure while the 3c panels are rebuilt for a new
    threshold must not leave them cached under the old one: the next calls
    with the old threshold (the regular and the allocation-free entry point)
    rebuild and match the oracle."""
    from paper_2104_09857_gb300 import _lib

    thr1 = 1e-3
    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case, thr=thr1)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        assert _rel(ctx.chi_tau(thr1, "fp64").cpu().numpy(), ref) <= 1e-10
        # thr 0 keeps more 3c blocks than thr1: the rebuild needs a larger
        # host-table buffer, whose allocation is the injected failure
        ctx.set_option("test_fail_alloc", 1)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(0.0, "fp64")
        assert e.value.code == -5  # GW_ERR_OOM
        got = ctx.chi_tau(thr1, "fp64").cpu().numpy()
        assert _rel(got, ref) <= 1e-10
        # (tau index 0: at tau = 50 a.u. every block is below thr1 and chi is zero)
        out = torch.full((ctx.nri, ctx.nri), float("nan"), dtype=torch.float64, device="cuda:0")
        _lib.gw_chi_tau_noalloc(ctx.ctx, 0, thr1, out.data_ptr())
        assert _rel([out.cpu().numpy()], [ref[0]]) <= 1e-10
        _lib.gw_chi_tau_noalloc(ctx.ctx, 1, thr1, out.data_ptr())
        assert not np.any(out.cpu().numpy()) and not np.any(ref[1])
