"""Parity of the CUDA chi(i tau) path (through the C ABI) with the CPU oracle.

FP64 bar: per tau, ||chi - chi_ref||_F <= 1e-10 ||chi_ref||_F and element-wise
|chi - chi_ref| <= 1e-10 max|chi_ref|.  FP32/split forms: the same with 1e-6
(FP32 accumulation over one 64-function slab, FP64 across slabs).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402

TOL = {"fp64": 1e-10, "fp32": 1e-6, "bf16x6": 1e-6, "fp16x3": 1e-6}


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_09857_gb300 as pkg

    return pkg


def _check(got, ref, tol):
    for j in range(ref.shape[0]):
        r = ref[j]
        g = got[j]
        if not np.any(r):
            # every block filtered: the result must be exactly zero
            assert not np.any(g), f"tau {j}: reference is zero, result is not"
            continue
        rel = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert rel <= tol, f"tau {j}: relative Frobenius error {rel:.3e} > {tol}"
        assert np.abs(g - r).max() <= tol * np.abs(r).max(), f"tau {j}: element error"


def _run(pkg, case, precision="fp64", thr=None, tau_first=0, tau_count=None, options=None,
         host_out=False):
    thr = case.thr if thr is None else thr
    with pkg.Context(0) as ctx:
        for k, v in (options or {}).items():
            ctx.set_option(k, v)
        ctx.load_case(case)
        if host_out:
            n = tau_count if tau_count is not None else len(case.tau) - tau_first
            out = np.zeros((n, ctx.nri, ctx.nri))
            ctx.chi_tau(thr, precision, tau_first, tau_count, out=out)
            return out, ctx.stats()
        got = ctx.chi_tau(thr, precision, tau_first, tau_count)
        torch.cuda.synchronize()
        return got.cpu().numpy(), ctx.stats()


@pytest.mark.parametrize("name", ["chain_HH", "chain_CH", "chain_CHCH", "benzene"])
def test_fp64_matches_dense_oracle(lib, name):
    case = make_case(name)
    got, st = _run(lib, case)
    ref = oc.chi_dense(case)
    _check(got, ref, TOL["fp64"])
    assert st["flops_c"] > 0 and st["tiles_active"] > 0


def test_fp64_symmetric_and_nsd(lib):
    """Off-diagonal atom blocks are mirrored (exactly symmetric); inside a
    diagonal atom block both halves are computed, symmetric to rounding."""
    case = make_case("benzene")
    got, _ = _run(lib, case)
    atom = np.repeat(np.arange(case.system.n_atoms), case.system.n_ri)
    off = atom[:, None] != atom[None, :]
    for x in got:
        assert np.array_equal(x[off], x.T[off])
        assert np.abs(x - x.T).max() <= 1e-13 * np.abs(x).max()
        ev = np.linalg.eigvalsh(0.5 * (x + x.T))
        assert ev.max() <= 1e-12 * np.abs(ev).max()


@pytest.mark.parametrize("thr", [1e-9, 1e-3, 3e-2])
def test_fp64_filtered_ribbon_matches_oracle(lib, thr):
    """Ribbon with stored-block sparsity; thr > 0 exercises the filters of T,
    G and both intermediates."""
    case = make_case("ribbon28", n_tau=4)
    got, st = _run(lib, case, thr=thr)
    ref = oc.chi_dense(case, thr=thr)
    _check(got, ref, TOL["fp64"])
    if thr >= 1e-3:
        assert st["slabs_active"] < st["slabs_total"]


def test_fp64_many_batches_and_ragged_tiles(lib):
    """Force one sigma-atom per batch: ragged P windows and K segments."""
    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case)
    for atoms in (1, 3, 7):
        got, st = _run(lib, case, options={"batch_atoms": atoms})
        assert st["n_batches"] >= case.system.n_atoms // atoms
        _check(got, ref, TOL["fp64"])


def test_tau_subset_and_host_output(lib):
    case = make_case("benzene")
    ref = oc.chi_dense(case)
    got, _ = _run(lib, case, tau_first=3, tau_count=4, host_out=True)
    _check(got, ref[3:7], TOL["fp64"])
    got0, _ = _run(lib, case, tau_first=9, tau_count=0, host_out=True)
    assert got0.shape[0] == 0


def test_fp64_deterministic(lib):
    case = make_case("ribbon28", n_tau=2)
    a, _ = _run(lib, case)
    b, _ = _run(lib, case)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["benzene", "ribbon28"])
def test_fp32_matches_oracle(lib, name):
    case = make_case(name, n_tau=4)
    got, _ = _run(lib, case, precision="fp32")
    ref = oc.chi_dense(case)
    _check(got, ref, TOL["fp32"])


def test_useful_flop_count_matches_dense_formula(lib):
    """At thr = 0 with every block stored, step C's useful flops are
    sum over (s, m, p <= q) of 2 n_s n_m n_p n_q for nonzero blocks; on a
    fully dense small case this is 2 nao^2 * (sum_{p<=q} n_p n_q)."""
    case = make_case("chain_CHCH", n_tau=1)
    _, st = _run(lib, case)
    nri = case.system.n_ri.astype(float)
    pairs = sum(nri[p] * nri[q] for p in range(len(nri)) for q in range(p, len(nri)))
    nao = case.system.nao_total
    assert st["flops_c"] == pytest.approx(2.0 * nao * nao * pairs, rel=1e-12)
    nblk_elems = 0.0
    t3 = case.t3c
    for (a, b, p) in t3.blocks:
        w = case.system.n_ao[a] * case.system.n_ao[b] * case.system.n_ri[p]
        nblk_elems += w * (1 if a == b else 2)
    assert st["flops_a"] == pytest.approx(2.0 * nao * nblk_elems, rel=1e-12)
    assert st["flops_b"] == pytest.approx(st["flops_a"], rel=1e-12)


# ---------------------------------------------------------------------------
# error handling through the C ABI (host-side checks; no device fault)
# ---------------------------------------------------------------------------

def test_errors_order_and_arguments(lib):
    from paper_2104_09857_gb300 import _lib

    case = make_case("chain_CH")
    s = case.system
    with lib.Context(0) as ctx:
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(0.0, "fp64", 0, 1)
        assert e.value.code == -2
        ctx.set_basis(s.xyz, s.n_ao, s.n_ri)
        blocks = case.t3c.blocks.copy()
        with pytest.raises(_lib.GwError) as e:
            ctx.set_3c_tensor(blocks[::-1].copy(), case.t3c.data)
        assert e.value.code == -1
        bad = case.t3c.data.copy()
        bad[5] = np.nan
        with pytest.raises(_lib.GwError) as e:
            ctx.set_3c_tensor(blocks, bad)
        assert e.value.code == -4
        asym = case.t3c.data.copy()
        # element (mu=0, sigma=1, P=0) of the first (0, 0, 0) block; its mirror
        # (1, 0, 0) is left unchanged
        asym[case.system.n_ri[0]] += 0.5
        with pytest.raises(_lib.GwError) as e:
            ctx.set_3c_tensor(blocks, asym)
        assert e.value.code == -3
        ctx.set_3c_tensor(blocks, case.t3c.data)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(0.0, "fp64", 0, 1)
        assert e.value.code == -2
        ctx.set_greens(case.C, case.eps, case.n_occ, 0.0, case.tau)
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(-1.0, "fp64", 0, 1)
        assert e.value.code == -1
        with pytest.raises(_lib.GwError) as e:
            ctx.chi_tau(0.0, "fp64", 2, 5)
        assert e.value.code == -1
        out = ctx.chi_tau(0.0, "fp64", 0, 1)
        assert torch.isfinite(out).all()


# ---------------------------------------------------------------------------
# tensor-core split-BF16 forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,thr", [("benzene", 0.0), ("ribbon28", 1e-9), ("ribbon28", 1e-3)])
def test_bf16x6_matches_oracle(lib, name, thr):
    """Three-slice split, 6 products: within the 1e-6 mixed-precision bar."""
    case = make_case(name, n_tau=4)
    got, st = _run(lib, case, precision="bf16x6", thr=thr)
    ref = oc.chi_dense(case, thr=thr)
    _check(got, ref, TOL["bf16x6"])
    assert st["c_launches"] > 0


def _rel_err(got, ref):
    return max(np.linalg.norm(g - r) / np.linalg.norm(r) for g, r in zip(got, ref))


def test_bf16x6_many_batches_ragged_tiles_and_flush(lib):
    """Ragged 128-row tiles over one- and five-atom batches; the accuracy bar
    holds for drains of the main accumulator every 16..64 reduction elements.
    Each 16-element MMA step rounds toward zero, so draining rarely (4096)
    lets the error grow, which is why the default is 64."""
    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case)
    for atoms, flush in ((1, 16), (5, 32), (0, 64)):
        got, _ = _run(lib, case, precision="bf16x6", options={"batch_atoms": atoms, "flush_k": flush})
        _check(got, ref, TOL["bf16x6"])
    whole = {"c_split_k": 0}  # whole tiles, so that a 4096 drain interval is reached
    e_short = _rel_err(_run(lib, case, precision="bf16x6", options={"flush_k": 64, **whole})[0], ref)
    e_long = _rel_err(_run(lib, case, precision="bf16x6", options={"flush_k": 4096, **whole})[0], ref)
    assert e_long > e_short


def test_bf16x6_split_k_units(lib):
    """Step C over work units that split tiles along the reduction (FP64
    atomic adds into chi): every split, from one slab per unit to whole
    tiles, meets the bar; whole tiles are bitwise reproducible."""
    case = make_case("ribbon28", n_tau=2)
    ref = oc.chi_dense(case)
    for split in (0, 1, 700, 2048, 1 << 20):
        got, _ = _run(lib, case, precision="bf16x6", options={"c_split_k": split, "batch_atoms": 4})
        _check(got, ref, TOL["bf16x6"])
    a = _run(lib, case, precision="bf16x6", options={"c_split_k": 0})[0]
    b = _run(lib, case, precision="bf16x6", options={"c_split_k": 0})[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name,thr", [("benzene", 0.0), ("ribbon28", 1e-9), ("ribbon28", 1e-3)])
def test_fp16x3_matches_oracle(lib, name, thr):
    """Two binary16 slices of power-of-two scaled operands, 3 products."""
    case = make_case(name, n_tau=4)
    got, st = _run(lib, case, precision="fp16x3", thr=thr)
    ref = oc.chi_dense(case, thr=thr)
    _check(got, ref, TOL["fp16x3"])
    assert st["c_launches"] > 0


@pytest.mark.parametrize("factor", [1e-7, 1e7])
def test_fp16x3_scaling_covers_tensor_magnitude(lib, factor):
    """A tensor scaled by 1e-7 or 1e7 lies far outside the binary16 range
    unscaled (chi scales by factor^2); the power-of-two operand scales keep
    the result within the bar, whole tiles or split units alike."""
    import dataclasses

    base = make_case("ribbon28", n_tau=2)
    t3 = dataclasses.replace(base.t3c, data=base.t3c.data * factor)
    case = dataclasses.replace(base, t3c=t3, thr=base.thr * factor)
    ref = oc.chi_dense(case)
    for split in (0, 2048):
        got, _ = _run(lib, case, precision="fp16x3", options={"c_split_k": split})
        _check(got, ref, TOL["fp16x3"])


def test_bf16x3_error_is_split_limited(lib):
    """Two-slice split, 3 products: the dropped low-low product and the 16-bit
    representation bound the error near 2^-17; it does not meet 1e-6."""
    case = make_case("benzene", n_tau=4)
    got, _ = _run(lib, case, precision="bf16x3")
    ref = oc.chi_dense(case)
    _check(got, ref, 2e-5)
