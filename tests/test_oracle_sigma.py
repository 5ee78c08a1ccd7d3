"""Pins of the self-energy oracle (Eq. 10): the AO route against the MO
route, the W = 1 special case, the sign for negative semidefinite W, and
linearity in W.  No GPU."""

import numpy as np
import pytest

from oracle import chi as oc
from oracle import sigma as osg
from synth import make_case
from synth.chain_inputs import synthetic_w


@pytest.fixture(scope="module")
def setup():
    case = make_case("chain_CHCH", n_tau=3)
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data)
    w = synthetic_w(s.nri_total, case.tau, 5)
    orbs = [case.n_occ - 1, case.n_occ]
    return case, t, w, orbs


def test_ao_route_equals_mo_route(setup):
    case, t, w, orbs = setup
    got = osg.sigma_dense(case, w, orbs, thr=0.0)
    for a, n in enumerate(orbs):
        for j, tau in enumerate(case.tau):
            ref = osg.sigma_mo(t, case.C, case.eps, case.n_occ, case.mu_fermi, n, w[j], tau)
            assert got[a, j, 0] == pytest.approx(ref[0], rel=1e-11)
            assert got[a, j, 1] == pytest.approx(ref[1], rel=1e-11)


def test_identity_w_is_trace_of_g_b_bt(setup):
    case, t, _, orbs = setup
    n = orbs[0]
    b = osg.b_half(t, case.C, n)
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, 0.4)
    eye = np.eye(b.shape[1])
    # sum_{mu nu} G_{mu nu} sum_P B_{mu P} B_{nu P}, by loops over P
    ref = sum(float(b[:, p] @ go @ b[:, p]) for p in range(b.shape[1]))
    assert osg.s_term(go, b, eye) == pytest.approx(ref, rel=1e-12)


def test_sign_and_linearity(setup):
    """W <= 0 and G >= 0 give S <= 0, so Sigma(i tau) >= 0 and Sigma(-i tau) <= 0;
    Sigma is linear in W."""
    case, _, w, orbs = setup
    sg = osg.sigma_dense(case, w, orbs, thr=0.0)
    assert np.all(sg[:, :, 0] >= 0.0) and np.all(sg[:, :, 1] <= 0.0)
    sg2 = osg.sigma_dense(case, 2.5 * w, orbs, thr=0.0)
    assert np.allclose(sg2, 2.5 * sg, rtol=1e-12)


def test_filter_threshold_zero_and_tiny_agree(setup):
    case, _, w, orbs = setup
    a = osg.sigma_dense(case, w, orbs, thr=0.0)
    b = osg.sigma_dense(case, w, orbs, thr=1e-300)
    assert np.array_equal(a, b)


def test_block_route_equals_dense_route(setup):
    """B^n from the stored blocks equals the dense half transform (both filters)."""
    case, t, w, orbs = setup
    for thr in (0.0, 1e-2):
        a = osg.sigma_dense(case, w, orbs, thr=thr)
        b = osg.sigma_blocks(case, w, orbs, list(range(len(case.tau))), thr=thr)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(a).max())


def test_molecule_set_shapes():
    from synth import molecule_set

    mols = molecule_set(8, 10, 150, 20210425)
    assert len(mols) == 8
    for m in mols:
        assert 8 <= m.n_atoms <= 160
        nc = m.species.count("C")
        assert abs(nc - 2 * (m.n_atoms - nc)) <= 4  # about 2:1


def _sigma_ao_case():
    from synth.chain_inputs import synthetic_w

    case = make_case("chain_CHCH")
    w = synthetic_w(case.system.nri_total, case.tau, 4)
    return case, w


def test_sigma_ao_projects_onto_the_diagonal_self_energy():
    """C_n^T Sigma_AO C_n is Sigma^c_n of the half-transformed route."""
    case, w = _sigma_ao_case()
    full = osg.sigma_ao_dense(case, w, thr=0.0)
    orbs = list(range(case.system.nao_total))
    diag = osg.sigma_dense(case, w, orbs, thr=0.0)
    proj = np.einsum("mn,jkmv,vn->njk", case.C, full, case.C)
    np.testing.assert_allclose(proj, diag, rtol=1e-11, atol=1e-13 * np.abs(diag).max())


def test_sigma_ao_symmetry_and_signs():
    """Symmetric; with W negative semidefinite, Sigma(i tau) is positive
    semidefinite (G^occ >= 0 between T^P-weighted factors) and Sigma(-i tau)
    negative semidefinite."""
    case, w = _sigma_ao_case()
    full = osg.sigma_ao_dense(case, w, thr=0.0)
    for j in range(len(case.tau)):
        for k, sign in ((0, 1.0), (1, -1.0)):
            m = full[j, k]
            np.testing.assert_allclose(m, m.T, rtol=0, atol=1e-13 * np.abs(m).max())
            ev = np.linalg.eigvalsh(0.5 * (m + m.T))
            assert np.all(sign * ev >= -1e-12 * np.abs(ev).max())


def test_sigma_ao_brute_force_on_two_atoms():
    """Explicit loops over mu, nu, lambda, sigma, P, Q on the two-atom chain."""
    from synth.chain_inputs import synthetic_w

    case = make_case("chain_HH")
    sysm = case.system
    w = synthetic_w(sysm.nri_total, case.tau, 5)
    full = osg.sigma_ao_dense(case, w, thr=0.0)
    t = oc.dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                              case.t3c.data, 0.0)
    nao, nri = t.shape[0], t.shape[2]
    j = 1
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[j])
    for g, k, sign in ((go, 0, -1.0), (gv, 1, 1.0)):
        ref = np.zeros((nao, nao))
        for mu in range(nao):
            for nu in range(nao):
                acc = 0.0
                for lam in range(nao):
                    for sig in range(nao):
                        for p in range(nri):
                            for q in range(nri):
                                acc += t[mu, lam, p] * g[lam, sig] * w[j, p, q] * t[sig, nu, q]
                ref[mu, nu] = sign * acc
        np.testing.assert_allclose(full[j, k], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_sigma_ao_filter_drops_blocks_like_explicit_loops():
    """thr > 0 on the four-atom chain: explicit per-block masks of the 3c
    tensor and of G (blocks with Frobenius norm < thr zeroed, mirrors
    together) reproduce the filtered AO self-energy."""
    case = make_case("chain_CHCH")
    s = case.system
    w = synthetic_w(s.nri_total, case.tau, 6)
    t_full = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets,
                                   case.t3c.data, 0.0)
    ao, ri = oc.offsets(s.n_ao), oc.offsets(s.n_ri)
    n_at = len(s.n_ao)
    j = 2
    go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[j])
    norms = [np.linalg.norm(t_full[ao[a]:ao[a + 1], ao[b]:ao[b + 1], ri[p]:ri[p + 1]])
             for a in range(n_at) for b in range(a, n_at) for p in range(n_at)]
    gnorms = [np.linalg.norm(g[ao[a]:ao[a + 1], ao[b]:ao[b + 1]])
              for g in (go, gv) for a in range(n_at) for b in range(a, n_at)]
    thr = float(np.median([x for x in norms + gnorms if x > 0]))   # drops about half
    t = t_full.copy()
    for a in range(n_at):
        for b in range(a, n_at):
            for p in range(n_at):
                blk = (slice(ao[a], ao[a + 1]), slice(ao[b], ao[b + 1]), slice(ri[p], ri[p + 1]))
                if np.linalg.norm(t[blk]) < thr:
                    t[blk] = 0.0
                    t[blk[1], blk[0], blk[2]] = 0.0
    ref = []
    for g, sign in ((go, -1.0), (gv, 1.0)):
        g = g.copy()
        for a in range(n_at):
            for b in range(a, n_at):
                if np.linalg.norm(g[ao[a]:ao[a + 1], ao[b]:ao[b + 1]]) < thr:
                    g[ao[a]:ao[a + 1], ao[b]:ao[b + 1]] = 0.0
                    g[ao[b]:ao[b + 1], ao[a]:ao[a + 1]] = 0.0
        ref.append(sign * np.einsum("mlp,ls,pq,snq->mn", t, g, w[j], t, optimize=True))
    got = osg.sigma_ao_dense(case, w, thr=thr)[j]
    for k in range(2):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-12, atol=1e-14 * np.abs(ref[k]).max())
    full = osg.sigma_ao_dense(case, w, thr=0.0)[j]
    assert np.abs(full - got).max() > 1e-6 * np.abs(full).max()      # the filter did act
