"""Pins of the CPU oracle for Eq. 2 and Eq. 3 against what the mathematics
fixes: an independent algebraic route, brute force, a closed form, and the
invariants of the Green's functions and of chi.  No GPU."""

import numpy as np
import pytest

from oracle import chi as oc
from synth import make_case


def _dense_t(case, thr=0.0):
    s = case.system
    return oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets,
                                 case.t3c.data, thr)


def _offs(case):
    return oc.offsets(case.system.n_ao), oc.offsets(case.system.n_ri)


@pytest.mark.parametrize("name", ["chain_CH", "chain_HCH", "chain_CHCH", "benzene"])
def test_dense_equals_mo_route(name):
    """Eq. 3 in the AO bracketing == Eq. 3 with Eq. 2 inserted (MO sums)."""
    case = make_case(name)
    t = _dense_t(case)
    chi = oc.chi_dense(case, thr=0.0)
    for j, tau in enumerate(case.tau):
        mo = oc.chi_mo_route(t, case.C, case.eps, case.n_occ, tau)
        assert np.linalg.norm(chi[j] - mo) <= 1e-12 * np.linalg.norm(mo)


def test_bruteforce_loops_equal_dense():
    """Eq. 3 summed one scalar term at a time agrees with the oracle."""
    case = make_case("chain_HH")
    t = _dense_t(case)
    ao, ri = _offs(case)
    for tau in case.tau[:2]:
        go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, tau)
        ref = oc.chi_bruteforce(t, go, gv)
        got = oc.chi_dense_from_g(t, go, gv, ao, ri, 0.0, mirror=False)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_single_pair_closed_form():
    """One occupied i and one virtual a: chi = -exp(-(e_a - e_i) tau) b b^T,
    b_P = sum_{lambda sigma} c_i[lambda] c_a[sigma] T[lambda, sigma, P]; rank 1."""
    case = make_case("chain_CH")
    t = _dense_t(case)
    ao, ri = _offs(case)
    i, a = case.n_occ - 1, case.n_occ
    ci, ca = case.C[:, i], case.C[:, a]
    tau = 0.7
    go = np.exp(case.eps[i] * tau) * np.outer(ci, ci)
    gv = np.exp(-case.eps[a] * tau) * np.outer(ca, ca)
    got = oc.chi_dense_from_g(t, go, gv, ao, ri, 0.0, mirror=False)
    nao, _, nri = t.shape
    b = np.zeros(nri)
    for lam in range(nao):
        for sg in range(nao):
            b += ci[lam] * ca[sg] * t[lam, sg, :]
    ref = -np.exp(-(case.eps[a] - case.eps[i]) * tau) * np.outer(b, b)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    sv = np.linalg.svd(got, compute_uv=False)
    assert sv[1] <= 1e-12 * sv[0]


def test_chi_symmetric_and_negative_semidefinite():
    case = make_case("benzene")
    chi = oc.chi_dense(case, thr=0.0, mirror=False)
    for x in chi:
        scale = np.abs(x).max()
        assert np.abs(x - x.T).max() <= 1e-13 * scale
        ev = np.linalg.eigvalsh(0.5 * (x + x.T))
        assert ev.max() <= 1e-12 * np.abs(ev).max()
        assert ev.min() < 0.0


def test_trace_strictly_decreasing_in_tau():
    """-Tr chi(tau) = sum_ia exp(-(e_a - e_i) tau) |B^ia|^2 decreases with tau."""
    case = make_case("benzene")
    tr = [-np.trace(x) for x in oc.chi_dense(case, thr=0.0)]
    assert all(tr[k] > tr[k + 1] for k in range(len(tr) - 1))
    assert tr[-1] > 0.0


def test_fermi_level_invariance():
    case = make_case("chain_CHCH")
    t = _dense_t(case)
    ao, ri = _offs(case)
    tau = 1.3
    g0 = oc.greens(case.C, case.eps, case.n_occ, 0.0, tau)
    g1 = oc.greens(case.C, case.eps, case.n_occ, 0.11, tau)
    assert not np.allclose(g0[0], g1[0])
    c0 = oc.chi_dense_from_g(t, *g0, ao, ri)
    c1 = oc.chi_dense_from_g(t, *g1, ao, ri)
    assert np.linalg.norm(c0 - c1) <= 1e-12 * np.linalg.norm(c0)


def test_greens_invariants_at_tau_zero():
    """Orthonormal basis: G^occ(0) + G^virt(0) = 1, Tr G^occ(0) = n_occ,
    G^occ(0) is idempotent; both are PSD at tau > 0."""
    case = make_case("benzene")
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, 0.0)
    n = go.shape[0]
    assert np.abs(go + gv - np.eye(n)).max() < 1e-12
    assert abs(np.trace(go) - case.n_occ) < 1e-10
    assert np.abs(go @ go - go).max() < 1e-12
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, 2.0)
    assert np.linalg.eigvalsh(go).min() > -1e-12
    assert np.linalg.eigvalsh(gv).min() > -1e-12
    # eps measured from mu_F: occupied factors < 1, virtual factors < 1
    assert np.all(case.eps[:case.n_occ] < 0) and np.all(case.eps[case.n_occ:] > 0)


def test_threshold_zero_filters_nothing_and_tiny_threshold_matches():
    case = make_case("chain_CHCH")
    full = oc.chi_dense(case, thr=0.0)
    tiny = oc.chi_dense(case, thr=1e-300)
    assert np.array_equal(full, tiny)


def test_three_center_filter_drops_small_block():
    """A stored 3c block with norm < thr is excluded, its mirror too."""
    case = make_case("chain_CH")
    t3 = case.t3c
    data = t3.data.copy()
    # the (0, 1, 1) block (C, H, RI of H) scaled to norm 1e-6
    i = int(np.nonzero((t3.blocks[:, 0] == 0) & (t3.blocks[:, 1] == 1) & (t3.blocks[:, 2] == 1))[0][0])
    blk = data[t3.offsets[i]:t3.offsets[i + 1]]
    blk *= 1e-6 / np.linalg.norm(blk)
    s = case.system
    t_f = oc.dense_three_center(s.n_ao, s.n_ri, t3.blocks, t3.offsets, data, thr=2e-6)
    t_k = oc.dense_three_center(s.n_ao, s.n_ri, t3.blocks, t3.offsets, data, thr=5e-7)
    ao, ri = _offs(case)
    sl = (slice(ao[0], ao[1]), slice(ao[1], ao[2]), slice(ri[1], ri[2]))
    slt = (slice(ao[1], ao[2]), slice(ao[0], ao[1]), slice(ri[1], ri[2]))
    assert np.all(t_f[sl] == 0) and np.all(t_f[slt] == 0)
    assert np.linalg.norm(t_k[sl]) == pytest.approx(1e-6)
    assert np.array_equal(t_k[slt], t_k[sl].transpose(1, 0, 2))


def test_intermediate_block_filter_by_loops():
    """filter_3idx zeroes exactly the atom blocks whose norm is < thr."""
    rng = np.random.default_rng(3)
    cuts = [oc.offsets([2, 3]), oc.offsets([3, 1]), oc.offsets([2, 2])]
    x = rng.standard_normal((5, 4, 4))
    x[0:2, 3:4, 2:4] *= 1e-5
    thr = 1e-3
    got = oc.filter_3idx(x, cuts, thr)
    ref = x.copy()
    for a in range(2):
        for b in range(2):
            for c in range(2):
                sl = tuple(slice(o[i], o[i + 1]) for o, i in zip(cuts, (a, b, c)))
                if np.sqrt(np.sum(x[sl] ** 2)) < thr:
                    ref[sl] = 0.0
    assert np.array_equal(got, ref)
    assert np.all(got[0:2, 3:4, 2:4] == 0.0)


def test_green_filter_symmetric_decision():
    rng = np.random.default_rng(4)
    ao = oc.offsets([2, 3, 1])
    g = rng.standard_normal((6, 6))
    g = g + g.T
    g[0:2, 5:6] *= 1e-9
    g[5:6, 0:2] *= 1e-9
    f = oc.filter_sym_2d(g, ao, 1e-6)
    assert np.all(f[0:2, 5:6] == 0) and np.all(f[5:6, 0:2] == 0)
    assert np.array_equal(f[2:5], g[2:5])


@pytest.mark.parametrize("thr", [0.0, 1e-9, 1e-3])
def test_block_oracle_matches_dense(thr):
    """The per-block route used at large sizes reproduces the dense oracle on
    every atom block of a 28-atom ribbon (its M and N slices sum only over
    the stored 3c blocks, so a dropped partner atom would show here)."""
    case = make_case("ribbon28", n_tau=2, thr=1e-9)
    dense = oc.chi_dense(case, tau_index=1, thr=thr)[0]
    bo = oc.BlockOracle(case, thr=thr)
    ri = oc.offsets(case.system.n_ri)
    n_at = case.system.n_atoms
    cache = {}
    for p in range(n_at):
        for q in range(n_at):
            blk = bo.block(1, p, q, cache)
            ref = dense[ri[p]:ri[p + 1], ri[q]:ri[q + 1]]
            assert np.allclose(blk, ref, rtol=1e-11, atol=1e-12 * np.abs(dense).max()), (p, q)


@pytest.mark.parametrize("thr", [0.0, 1e-3])
def test_useful_flops_two_routes_and_closed_form(thr):
    """The useful-flop count of one tau point from the dense route equals the
    count from the block oracle's slices, and at thr 0 (nothing filtered,
    every stored block kept) steps A and B each equal 2 n_AO times the
    stored elements of both block orientations."""
    case = make_case("ribbon28", n_tau=2, thr=1e-9)
    dense = oc.useful_flops_dense(case, 1, thr=thr)
    blocks = oc.useful_flops_blocks(oc.BlockOracle(case, thr=thr), 1)
    assert dense == pytest.approx(blocks, rel=1e-14)
    if thr == 0.0:
        s = case.system
        b = case.t3c.blocks
        elems = s.n_ao[b[:, 0]] * s.n_ao[b[:, 1]] * s.n_ri[b[:, 2]] * np.where(b[:, 0] == b[:, 1], 1, 2)
        assert dense[0] == dense[1] == 2.0 * s.nao_total * float(np.sum(elems))


def test_useful_flops_step_c_by_loops():
    """F_C by explicit loops over (mu-atom, sigma-atom, p <= q) on a 3-atom
    chain at a threshold that drops some M/N blocks."""
    case = make_case("chain_CHCH", n_tau=2, thr=0.0)
    thr = 1e-2
    s = case.system
    ao, ri = oc.offsets(s.n_ao), oc.offsets(s.n_ri)
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data, thr)
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[1])
    go, gv = oc.filter_sym_2d(go, ao, thr), oc.filter_sym_2d(gv, ao, thr)
    m = oc.filter_3idx(np.einsum("ml,lsp->msp", go, t), [ao, ao, ri], thr)
    n = oc.filter_3idx(np.einsum("mnq,ns->msq", t, gv), [ao, ao, ri], thr)
    n_at = s.n_atoms
    fc = 0.0
    for a in range(n_at):
        for b in range(n_at):
            for p in range(n_at):
                for q in range(p, n_at):
                    mb = m[ao[a]:ao[a + 1], ao[b]:ao[b + 1], ri[p]:ri[p + 1]]
                    nb = n[ao[a]:ao[a + 1], ao[b]:ao[b + 1], ri[q]:ri[q + 1]]
                    if np.any(mb) and np.any(nb):
                        fc += 2.0 * s.n_ao[a] * s.n_ao[b] * s.n_ri[p] * s.n_ri[q]
    assert oc.useful_flops_dense(case, 1, thr=thr)[2] == fc
    assert fc < oc.useful_flops_dense(case, 1, thr=0.0)[2]  # the filter dropped some blocks
