"""Oracle for the diagonal correlation self-energy of Eq. 10 (and, with the
density matrix and the Coulomb matrix in place of G(i tau) and W^c(i tau),
the exchange term of Eq. 11).  FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* (n mu | P) = sum_nu C_nu,n (nu mu | P) is the half-transformed 3c tensor
  B^n[mu][P] (its sparsity in mu-P is what the paper exploits).
* With the real G^occ/G^virt of the chi oracle (phases removed) and the real
  W^c(i tau) of the chain, Eq. 10 reads
      S^occ_n(tau)  = sum_{mu nu} G^occ_{mu nu}(tau) sum_{PQ} B^n_{mu P} W_PQ(tau) B^n_{nu Q}
      Sigma^c_n(i tau)  = i * i * S^occ_n  = -S^occ_n(tau)
      Sigma^c_n(-i tau) = i * (-i) * S^virt_n = +S^virt_n(tau)
  (W^c is even in tau).
* The RI metric S is the identity (W~ = W).
* Filter: 3c blocks, G blocks and the atom blocks (mu-atom, P-atom) of B^n
  with Frobenius norm < thr are dropped.
"""

from __future__ import annotations

import numpy as np

from . import chi as oc


def b_half(t: np.ndarray, C: np.ndarray, n: int) -> np.ndarray:
    """B^n[mu][P] = sum_nu C[nu][n] T[nu][mu][P]."""
    return np.einsum("v,vmp->mp", C[:, n], t)


def s_term(g: np.ndarray, b: np.ndarray, w: np.ndarray) -> float:
    """sum_{mu nu} G[mu][nu] sum_{PQ} B[mu][P] W[P][Q] B[nu][Q]."""
    return float(np.sum(g * (b @ w @ b.T)))


def sigma_dense(case, w_tau: np.ndarray, orbitals, thr: float | None = None) -> np.ndarray:
    """[n_orb][n_tau][2]: (Sigma^c_n(i tau), Sigma^c_n(-i tau)) for each orbital."""
    sysm = case.system
    thr = case.thr if thr is None else thr
    ao = oc.offsets(sysm.n_ao)
    ri = oc.offsets(sysm.n_ri)
    t = oc.dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                              case.t3c.data, thr)
    out = np.zeros((len(orbitals), len(case.tau), 2))
    for a, n in enumerate(orbitals):
        b = b_half(t, case.C, n)
        if thr > 0.0:
            nrm = np.sqrt(oc.block_sq_sums(b, [ao, ri]))
            keep = np.repeat(np.repeat(nrm >= thr, np.diff(ao), 0), np.diff(ri), 1)
            b = np.where(keep, b, 0.0)
        for j, tau in enumerate(case.tau):
            go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, tau)
            go = oc.filter_sym_2d(go, ao, thr)
            gv = oc.filter_sym_2d(gv, ao, thr)
            out[a, j, 0] = -s_term(go, b, w_tau[j])
            out[a, j, 1] = s_term(gv, b, w_tau[j])
    return out


def sigma_mo(t: np.ndarray, C: np.ndarray, eps: np.ndarray, n_occ: int, mu_fermi: float, n: int,
             w: np.ndarray, tau: float) -> tuple[float, float]:
    """MO route of Eq. 10 (unfiltered): with b_m[P] = sum_{mu nu} C_mu,m C_nu,n
    T[mu][nu][P],
        S^occ_n  = sum_{i occ}  exp( (eps_i - mu_F) tau) b_i^T W b_i
        S^virt_n = sum_{a virt} exp(-(eps_a - mu_F) tau) b_a^T W b_a."""
    bm = np.einsum("um,vn,uvp->mp", C, C[:, [n]], t)  # [all m][P]
    q = np.einsum("mp,pq,mq->m", bm, w, bm)
    e = eps - mu_fermi
    s_occ = float(np.sum(np.exp(e[:n_occ] * tau) * q[:n_occ]))
    s_virt = float(np.sum(np.exp(-e[n_occ:] * tau) * q[n_occ:]))
    return -s_occ, s_virt


def b_half_blocks(case, n: int, thr: float) -> np.ndarray:
    """B^n[mu][P] = sum_nu C[nu][n] (nu mu|P) from the stored atom blocks
    (no dense 3c tensor), with the 3c and B^n block filters of sigma_dense."""
    s = case.system
    ao = oc.offsets(s.n_ao)
    ri = oc.offsets(s.n_ri)
    t3 = case.t3c
    c = case.C[:, n]
    b = np.zeros((ao[-1], ri[-1]))
    for i, (a, bb, p) in enumerate(t3.blocks):
        blk = t3.data[t3.offsets[i]:t3.offsets[i + 1]].reshape(s.n_ao[a], s.n_ao[bb], s.n_ri[p])
        if thr > 0.0 and np.sqrt(np.sum(blk * blk)) < thr:
            continue
        # (nu in A, mu in B): B[mu][P] += C[nu] blk[nu][mu][P]
        b[ao[bb]:ao[bb + 1], ri[p]:ri[p + 1]] += np.einsum("v,vmp->mp", c[ao[a]:ao[a + 1]], blk)
        if a != bb:
            # (nu in B, mu in A): T[nu][mu][P] = blk[mu][nu][P]
            b[ao[a]:ao[a + 1], ri[p]:ri[p + 1]] += np.einsum("v,mvp->mp", c[ao[bb]:ao[bb + 1]], blk)
    if thr > 0.0:
        nrm = np.sqrt(oc.block_sq_sums(b, [ao, ri]))
        keep = np.repeat(np.repeat(nrm >= thr, np.diff(ao), 0), np.diff(ri), 1)
        b = np.where(keep, b, 0.0)
    return b


def sigma_blocks(case, w_tau: np.ndarray, orbitals, tau_indices, thr: float | None = None) -> np.ndarray:
    """Like sigma_dense for the given tau indices, without the dense 3c tensor
    (for systems of a few hundred basis functions and more)."""
    thr = case.thr if thr is None else thr
    ao = oc.offsets(case.system.n_ao)
    out = np.zeros((len(orbitals), len(tau_indices), 2))
    for a, n in enumerate(orbitals):
        b = b_half_blocks(case, n, thr)
        for jj, j in enumerate(tau_indices):
            go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[j])
            go = oc.filter_sym_2d(go, ao, thr)
            gv = oc.filter_sym_2d(gv, ao, thr)
            out[a, jj, 0] = -s_term(go, b, w_tau[j])
            out[a, jj, 1] = s_term(gv, b, w_tau[j])
    return out


def sigma_ao_dense(case, w_tau: np.ndarray, thr: float | None = None) -> np.ndarray:
    """The full atomic-orbital matrix of Eq. 10 (the form before it is
    projected on orbital n): [n_tau][2][n_AO][n_AO] with
        [j][0] = Sigma^c_{mu nu}(i tau_j)  = -sum_{lam sig P Q} (mu lam|P) G^occ_{lam sig} W_PQ (sig nu|Q)
        [j][1] = Sigma^c_{mu nu}(-i tau_j) = +sum ... G^virt ...
    (the real representation of the diagonal oracle: C_n^T Sigma C_n is
    Sigma^c_n).  The filter acts on the inputs: 3c blocks and G blocks with
    Frobenius norm < thr are dropped."""
    sysm = case.system
    thr = case.thr if thr is None else thr
    ao = oc.offsets(sysm.n_ao)
    t = oc.dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                              case.t3c.data, thr)
    nao = t.shape[0]
    out = np.zeros((len(case.tau), 2, nao, nao))
    for j, tau in enumerate(case.tau):
        go, gv = oc.greens(case.C, case.eps, case.n_occ, case.mu_fermi, tau)
        go = oc.filter_sym_2d(go, ao, thr)
        gv = oc.filter_sym_2d(gv, ao, thr)
        tw = np.einsum("snq,pq->snp", t, w_tau[j])          # (sig nu|Q) W_PQ summed over Q
        for k, (g, sign) in enumerate(((go, -1.0), (gv, 1.0))):
            out[j, k] = sign * np.einsum("mlp,ls,snp->mn", t, g, tw, optimize=True)
    return out
