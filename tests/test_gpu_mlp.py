"""Learned block-norm screening on the GPU: gradients of the library's
backward kernels against the CPU oracle, training, and what the trained
network gains over the exact-filter method at the same threshold."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from synth import make_case  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as p

    return p


def test_mlp_gradients_match_oracle(pkg):
    from paper_2104_09857_gb300 import _lib

    rng = np.random.default_rng(11)
    x = rng.standard_normal((500, 8)).astype(np.float32)
    t = rng.standard_normal(500).astype(np.float32)
    theta = omlp.init_params(8, 5)
    theta[512:576] = 0.05 * rng.standard_normal(64)  # nonzero b1
    with pkg.Context(0) as ctx:
        _lib.gw_mlp_set_params(ctx.ctx, theta)
        loss, g = _lib.gw_mlp_grad(ctx.ctx, x, t)
        assert np.array_equal(_lib.gw_mlp_get_params(ctx.ctx), theta)
        pred = _lib.gw_mlp_predict(ctx.ctx, x)
    ref_loss, ref_g = omlp.loss_and_grad(theta, x.astype(np.float64), t.astype(np.float64))
    ref_y, _ = omlp.forward(theta, x.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert np.abs(pred - ref_y).max() <= 1e-4 * np.abs(ref_y).max()
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)


def test_logged_targets_match_block_contractions(pkg):
    """Each logged target is log10 of a task's contribution norm; their sum of
    squares over all tasks of a tile bounds nothing exactly, but the largest
    targets must reach the scale of chi and none may exceed its log-bound
    feature (norm product)."""
    from paper_2104_09857_gb300 import _lib

    case = make_case("ribbon28", n_tau=2)
    with pkg.Context(0) as ctx:
        ctx.load_case(case)
        feat, tgt = _lib.gw_mlp_log(ctx.ctx, 0, 2, case.thr, _lib.GW_BF16X6)
    assert feat.shape[0] == tgt.shape[0] > 100
    assert np.all(tgt <= feat[:, 7] + 1e-3)  # ||X^T Y|| <= ||X|| ||Y||
    chi = oc.chi_dense(case, tau_index=0)[0]
    assert tgt.max() > np.log10(np.abs(chi).max()) - 2


def _train_screen(pkg, ctx, thr, precision):
    """Train the network on task logs of two systems at thr and return the
    margin calibrated on held-out tasks (the largest under-prediction plus a
    quarter decade)."""
    from paper_2104_09857_gb300 import _lib

    feats, tgts = [], []
    for name, nt in (("ribbon28", 4), ("benzene", 4)):
        case = make_case(name, n_tau=nt, thr=1e-9)
        with pkg.Context(0) as lc:
            lc.load_case(case)
            f, t = _lib.gw_mlp_log(lc.ctx, 0, nt, thr, _lib.PRECISIONS[precision])
        feats.append(f)
        tgts.append(t)
    x = np.concatenate(feats)
    y = np.concatenate(tgts)
    keep = y > -39.0  # a task whose contribution is exactly zero carries no norm to learn
    x, y = x[keep], y[keep]
    rng = np.random.default_rng(3)
    idx = rng.permutation(len(y))
    n_tr = int(0.8 * len(y))
    tr, va = idx[:n_tr], idx[n_tr:]
    _lib.gw_mlp_init(ctx.ctx, 17)
    losses = _lib.gw_mlp_train(ctx.ctx, x[tr], y[tr], epochs=400, batch=0, lr=3e-3, seed=5)
    assert losses[-1] < 0.3 * losses[0]
    pv = _lib.gw_mlp_predict(ctx.ctx, x[va])
    return float(np.max(y[va] - pv)) + 0.25


def test_trained_screening_gain_and_error(pkg):
    """Train on task logs of two systems at the benchmark threshold 1e-9,
    calibrate the margin on held-out tasks, then screen a third system in the
    timed form: tasks are skipped (fewer issued flops), and at every tau point
    both the learned and the plain filtered chi match the oracle within 1e-6
    relative (Frobenius and element-wise), with no absolute allowance."""
    import time

    thr, precision = 1e-9, "fp16x3"
    case = make_case("ribbon60", n_tau=6, thr=thr)
    ref = oc.chi_dense(case, thr=thr)
    with pkg.Context(0) as ctx:
        margin = _train_screen(pkg, ctx, thr, precision)
        ctx.set_option("mlp_margin", margin)
        ctx.load_case(case)
        ctx.chi_tau(thr, precision)  # warm-up: panels and work buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = ctx.chi_tau(thr, precision).cpu().numpy()
        t_plain = time.perf_counter() - t0
        st_plain = ctx.stats()
        t0 = time.perf_counter()
        learned = ctx.chi_tau(thr, precision, screening=pkg.GW_SCREEN_MLP).cpu().numpy()
        t_learned = time.perf_counter() - t0
        st = ctx.stats()
    assert st["tasks_seen"] > 0
    assert st["tasks_skipped"] > 0, "the trained network skipped nothing"
    assert st["flops_issued"] < st_plain["flops_issued"]
    for j in range(len(case.tau)):
        nrm = np.linalg.norm(ref[j])
        assert nrm > 0.0
        for name, got in (("plain", plain[j]), ("learned", learned[j])):
            rel = np.linalg.norm(got - ref[j]) / nrm
            el = np.abs(got - ref[j]).max() / np.abs(ref[j]).max()
            print(f"tau[{j}] {name}: rel Frobenius {rel:.2e}, element {el:.2e}")
            assert rel <= 1e-6 and el <= 1e-6, (j, name, rel, el)
    print(f"learned screening at thr {thr:g}: skipped {st['tasks_skipped']}/{st['tasks_seen']} "
          f"tasks, issued flops {st['flops_issued']:.3e} vs {st_plain['flops_issued']:.3e}, "
          f"{t_learned * 1e3:.1f} ms vs {t_plain * 1e3:.1f} ms for {len(case.tau)} tau, "
          f"margin {margin:.2f}")
