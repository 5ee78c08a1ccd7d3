"""Parity of the FP64 screening chain on the GPU (gw_chi_to_w) with the CPU
oracle: chi -> chi(i omega) -> eps -> W^c(i omega) -> W^c(i tau)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chain as och  # noqa: E402
from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402
from synth.chain_inputs import chain_inputs  # noqa: E402

TOL = 1e-10


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


@pytest.mark.parametrize("name", ["benzene", "ribbon28"])
def test_chain_matches_oracle_on_oracle_chi(pkg, name):
    """Same chi in, W^c(i tau) out: GPU chain vs oracle chain."""
    case = make_case(name, n_tau=8)
    chi = oc.chi_dense(case)
    omega, gamma, delta, v, _, _ = chain_inputs(case)
    ref, _ = och.chi_to_w(chi, v, gamma, delta)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got = ctx.chi_to_w(chi, v, gamma, delta).cpu().numpy()
    for j in range(len(case.tau)):
        assert _rel(got[j], ref[j]) <= TOL, f"tau {j}: {_rel(got[j], ref[j]):.3e}"


def test_chain_from_gpu_chi_host_output(pkg):
    """chi computed on the device feeds the chain directly; host output."""
    case = make_case("benzene")
    omega, gamma, delta, v, _, _ = chain_inputs(case)
    ref, _ = och.chi_to_w(oc.chi_dense(case), v, gamma, delta)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, "fp64")
        out = np.zeros(ref.shape)
        ctx.chi_to_w(chi, v, gamma, delta, out=out)
    for j in range(len(case.tau)):
        assert _rel(out[j], ref[j]) <= TOL
        assert np.abs(out[j] - out[j].T).max() <= 1e-10 * np.abs(out[j]).max()


def test_chain_rejects_non_spd(pkg):
    from paper_2104_09857_gb300 import _lib

    case = make_case("chain_CH")
    chi = oc.chi_dense(case)
    omega, gamma, delta, v, _, _ = chain_inputs(case)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_to_w(chi, -v, gamma, delta)
        assert e.value.code == -8
        # a positive chi makes eps indefinite for a large enough scale
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_to_w(-1e6 * chi, v, gamma, delta)
        assert e.value.code == -8


def test_ri_metric_matches_oracle(pkg):
    """S^-1 M S^-1 on the GPU against the oracle for a random SPD metric of
    the benzene RI size; the identity metric returns M; an indefinite metric
    is refused with GW_ERR_NOT_SPD."""
    from oracle import chain as och
    from paper_2104_09857_gb300 import _lib

    case = make_case("benzene", n_tau=2)
    n = case.system.nri_total
    rng = np.random.default_rng(21)
    b = rng.standard_normal((n, n))
    s = b @ b.T / n + np.eye(n)
    ms = []
    for _ in range(3):
        a = rng.standard_normal((n, n))
        ms.append(a + a.T)
    ms = np.stack(ms)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        got = _lib.gw_ri_metric(ctx.ctx, s, ms)
        same = _lib.gw_ri_metric(ctx.ctx, np.eye(n), ms[0])
        bad = np.eye(n)
        bad[3, 3] = -1.0
        with pytest.raises(_lib.GwError) as e:
            _lib.gw_ri_metric(ctx.ctx, bad, ms[0])
        assert e.value.code == -8
    for k in range(3):
        ref = och.apply_metric(s, ms[k])
        assert np.abs(got[k] - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(same - ms[0]).max() <= 1e-14 * np.abs(ms[0]).max()


def test_chain_at_the_benchmark_ri_size(pkg):
    """The chain at the benchmark's RI size (298-atom ribbon, 7176 RI
    functions): chi(i tau) of the timed FP16x3 form on 3 tau points feeds both
    the GPU chain and the oracle chain; W^c(i tau) agree within 1e-10."""
    import time

    case = make_case("ribbon300", n_tau=3)
    omega, gamma, delta, v, _, _ = chain_inputs(case)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        chi = ctx.chi_tau(case.thr, "fp16x3")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = ctx.chi_to_w(chi, v, gamma, delta)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - t0
        got = got.cpu().numpy()
        chi_h = chi.cpu().numpy()
        del chi
    t0 = time.perf_counter()
    ref, _ = och.chi_to_w(chi_h, v, gamma, delta)
    t_cpu = time.perf_counter() - t0
    errs = [_rel(got[j], ref[j]) for j in range(len(case.tau))]
    print(f"chain, n_RI {chi_h.shape[1]}, {len(case.tau)} points: GPU {t_gpu:.2f} s, oracle {t_cpu:.1f} s, "
          f"max rel error {max(errs):.2e}")
    for j, e in enumerate(errs):
        assert e <= TOL, f"tau {j}: {e:.3e}"
