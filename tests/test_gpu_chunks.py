"""The tensor-core route with its operands cut into 2-D batches (sigma-atom
batches x mu-atom chunks, each chunk's Y restricted to the RI window of its
atoms' 3c blocks), and the useful-flop count of every route against the
oracle's own count (oracle.chi.useful_flops_dense)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as pkg

    return pkg


def _run(pkg, case, precision, thr, options=None):
    with pkg.Context(0) as ctx:
        for k, v in (options or {}).items():
            ctx.set_option(k, v)
        ctx.load_case(case)
        got = ctx.chi_tau(thr, precision).cpu().numpy()
        return got, ctx.stats()


def _check(got, ref, tol):
    for j in range(ref.shape[0]):
        r, g = ref[j], got[j]
        if not np.any(r):
            assert not np.any(g)
            continue
        rel = np.linalg.norm(g - r) / np.linalg.norm(r)
        el = np.abs(g - r).max() / np.abs(r).max()
        assert rel <= tol and el <= tol, (j, rel, el)


@pytest.mark.parametrize("precision,tol", [("fp16x3", 1e-6), ("bf16x6", 1e-6)])
@pytest.mark.parametrize("thr", [1e-9, 1e-3])
@pytest.mark.parametrize("chunk,batch_atoms", [(5, 0), (9, 3), (1, 2)])
def test_chunked_batches_match_oracle(lib, precision, tol, thr, chunk, batch_atoms):
    """mu chunks of 1, 5 and 9 atoms (ragged last chunk, windows cut inside
    the ribbon), with and without small owner batches: chi within the form's
    tolerance of the oracle, and the same useful-flop count as one chunk."""
    case = make_case("ribbon28", n_tau=3)
    ref = oc.chi_dense(case, thr=thr)
    opts = {"mu_chunk_atoms": chunk}
    if batch_atoms:
        opts["batch_atoms"] = batch_atoms
    got, st = _run(lib, case, precision, thr, opts)
    _check(got, ref, tol)
    one, st1 = _run(lib, case, precision, thr)
    assert st["n_batches"] > st1["n_batches"]
    for k in ("flops_a", "flops_b", "flops_c"):
        assert st[k] == pytest.approx(st1[k], rel=1e-12), k


@pytest.mark.parametrize("precision", ["fp64", "fp16x3"])
@pytest.mark.parametrize("name,thr", [("ribbon28", 1e-9), ("ribbon28", 1e-3), ("benzene", 0.0)])
def test_useful_flops_match_oracle_count(lib, precision, name, thr):
    """The library's useful flops per step equal the oracle's count of the
    atom-block products whose operands survive the filter, at every tau."""
    case = make_case(name, n_tau=3)
    with lib.Context(0) as ctx:
        ctx.load_case(case)
        for j in range(len(case.tau)):
            ctx.chi_tau(thr, precision, j, 1)
            st = ctx.stats()
            # a skipped batch's flops are not credited; here a batch is skipped
            # only where every G block is filtered (tau = 50 a.u. at thr 1e-3),
            # so that both counts are zero
            fa, fb, fc = oc.useful_flops_dense(case, j, thr=thr)
            assert st["flops_a"] == fa and st["flops_b"] == fb, (j, st["flops_a"], fa)
            assert st["flops_c"] == pytest.approx(fc, rel=1e-12), (j, st["flops_c"], fc)


def test_filtered_chunks_are_skipped(lib):
    """At a threshold that filters the Green's-function blocks between the
    ribbon's two ends, batches whose X or Y is entirely filtered are skipped,
    and chi still matches the oracle."""
    case = make_case("ribbon60", n_tau=2)
    thr = 3e-2
    ref = oc.chi_dense(case, thr=thr)
    got, st = _run(lib, case, "fp16x3", thr, {"mu_chunk_atoms": 6, "batch_atoms": 6})
    _check(got, ref, 1e-6)
    assert st["batches_skipped"] > 0


@pytest.mark.parametrize("name", ["benzene", "ribbon28"])
@pytest.mark.parametrize("chunk", [0, 7])
def test_staged_epilogue_writes_the_same_operands(lib, name, chunk):
    """The staged step-A/B epilogue (whole runs of X and Y from a tile staged
    in shared memory) computes every operand element in the same order as
    the per-element one: with whole-tile step-C units (a fixed summation
    order) and nothing filtered, chi is bitwise the same."""
    case = make_case(name, n_tau=2)
    opts = {"c_split_k": 0, "mu_chunk_atoms": chunk}
    a, _ = _run(lib, case, "fp16x3", 0.0, dict(opts, panel_staged=1))
    b, _ = _run(lib, case, "fp16x3", 0.0, dict(opts, panel_staged=0))
    assert np.array_equal(a, b)
    _check(a, oc.chi_dense(case, thr=0.0), 1e-6)


def test_autotune_keeps_the_fastest_schedule_and_the_result(lib):
    """The schedule search logs every timing, leaves the context on a
    setting at least as fast as where it started, and chi computed with the
    chosen schedule still matches the oracle."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case)
    with lib.Context(0) as ctx:
        ctx.load_case(case)
        trials = _lib.gw_autotune(ctx.ctx, 1, case.thr, _lib.GW_FP16X3)
        got = ctx.chi_tau(case.thr, "fp16x3").cpu().numpy()
    assert trials[0]["knob"] == "start" and len(trials) >= 6
    best = min(t["ms"] for t in trials)
    assert best <= trials[0]["ms"]
    assert all(t["ms"] > 0 for t in trials)
    _check(got, ref, 1e-6)


def test_tensor_kept_in_fp32(lib):
    """With the tensor kept in FP32 on the device the split forms still match
    the oracle within 1e-6 and count the same useful flops (the filter
    decisions come from the FP64 input); the FP64 form is refused."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("ribbon28", n_tau=3)
    ref = oc.chi_dense(case)
    a, sa = _run(lib, case, "fp16x3", case.thr, {"tensor_fp32": 1, "mu_chunk_atoms": 7})
    b, sb = _run(lib, case, "fp16x3", case.thr, {"mu_chunk_atoms": 7})
    _check(a, ref, 1e-6)
    for k in ("flops_a", "flops_b", "flops_c"):
        assert sa[k] == sb[k]
    with lib.Context(0) as ctx:
        ctx.set_option("tensor_fp32", 1)
        ctx.load_case(case)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(case.thr, "fp64", 0, 1)
        assert e.value.code == -9


def test_learned_screening_with_chunks(lib):
    """The learned screen on 2-D batches (7-atom mu chunks): the logged task
    features and targets feed the same network, and the screened chi stays
    within 1e-6 of the oracle at thr 1e-9."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("ribbon28", n_tau=3)
    ref = oc.chi_dense(case)
    with lib.Context(0) as ctx:
        ctx.set_option("mu_chunk_atoms", 7)
        ctx.load_case(case)
        feat, tgt = _lib.gw_mlp_log(ctx.ctx, 0, 3, case.thr, _lib.GW_FP16X3)
        keep = tgt > -39.0
        assert feat.shape[0] > 100 and np.all(tgt[keep] <= feat[keep, 7] + 1e-3)
        _lib.gw_mlp_init(ctx.ctx, 17)
        _lib.gw_mlp_train(ctx.ctx, feat[keep], tgt[keep], epochs=200, batch=0, lr=3e-3, seed=5)
        ctx.set_option("mlp_margin", float(np.max(tgt[keep] - _lib.gw_mlp_predict(ctx.ctx, feat[keep]))) + 0.25)
        got = ctx.chi_tau(case.thr, "fp16x3", screening=lib.GW_SCREEN_MLP).cpu().numpy()
        st = ctx.stats()
    assert st["n_batches"] > 1 and st["tasks_seen"] > 0
    _check(got, ref, 1e-6)


@pytest.mark.parametrize("chunk", [0, 7])
@pytest.mark.parametrize("fp32", [0, 1])
def test_streamed_panels_give_the_same_chi(lib, chunk, fp32):
    """Split panels streamed per batch (the owners' for step A, the chunk's for
    step B, built from the stored blocks) hold the same values as the resident
    set: with whole-tile step-C units chi is bitwise the same."""
    case = make_case("ribbon28", n_tau=2)
    opts = {"c_split_k": 0, "mu_chunk_atoms": chunk, "batch_atoms": 5, "tensor_fp32": fp32}
    a, sa = _run(lib, case, "fp16x3", case.thr, dict(opts, panel_stream=1))
    b, sb = _run(lib, case, "fp16x3", case.thr, opts)
    assert np.array_equal(a, b)
    assert sa["flops_useful"] == sb["flops_useful"]
    _check(a, oc.chi_dense(case), 1e-6)


@pytest.mark.parametrize("dynamic", [0, 1])
def test_step_c_unit_distribution(lib, dynamic):
    """Step-C units taken in order from a shared counter (default) or as a
    fixed share per CTA give the same chi within the bar, with the same
    useful flops (only the order of the FP64 atomic adds differs)."""
    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case)
    got, st = _run(lib, case, "fp16x3", case.thr, {"c_dynamic": dynamic, "c_split_k": 1024})
    _check(got, ref, 1e-6)
    got0, st0 = _run(lib, case, "fp16x3", case.thr, {"c_dynamic": 1 - dynamic, "c_split_k": 1024})
    assert st["flops_c"] == st0["flops_c"]
    assert np.allclose(got, got0, rtol=0, atol=1e-12 * np.abs(got0).max())
