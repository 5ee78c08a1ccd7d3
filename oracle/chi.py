"""Oracle for the imaginary-time Green's functions (Eq. 2) and the
irreducible polarizability chi_PQ(i tau) (Eq. 3), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (readings of the paper, stated once here):

* Phase (Eq. 2, Eq. 3): G(i tau) carries a factor +i for tau > 0 (occupied sum)
  and -i for tau < 0 (virtual sum); Eq. 3 multiplies by -i.  The routines
  return the real, positive-semidefinite matrices
      G^occ(tau)  = sum_{i occ}  C_mu,i C_nu,i exp( (eps_i - mu_F) tau)
      G^virt(tau) = sum_{a virt} C_mu,a C_nu,a exp(-(eps_a - mu_F) tau)
  and the real polarizability chi = -sum M N (which is chi^0 of Eq. 3 divided
  by i): negative semidefinite, so that eps = 1 - L^T chi L (Eq. 7) is
  positive definite as the paper requires of it.
* Energy zero: energies enter relative to the Fermi level mu_F; chi does not
  depend on mu_F (each term carries one occupied and one virtual factor).
* Bracketing of Eq. 3:
      M[mu, sigma, P] = sum_lambda G^occ[mu, lambda] T[lambda, sigma, P]
      N[mu, sigma, Q] = sum_nu     T[mu, nu, Q] G^virt[nu, sigma]
      chi[P, Q]       = - sum_{mu, sigma} M[mu, sigma, P] N[mu, sigma, Q]
* Filtering (Computational Methods: atom blocks whose Frobenius norm is below
  the threshold are filtered in the sparse tensor operations of Eq. 3): every
  stored atom block of every tensor of the contraction -- T (A, B, P),
  G^occ/G^virt (A, B), M and N (mu-atom, sigma-atom, RI-atom) -- whose
  Frobenius norm is < thr is set to zero (kept on equality).  A symmetric
  tensor's mirror blocks share one decision, taken on the block with the
  smaller first atom index.  With thr = 0 nothing is filtered.
* The filtered contraction is not exactly symmetric in P <-> Q; chi is defined
  by its atom-block upper triangle (atom(P) <= atom(Q)) and mirrored.
"""

from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# helpers on atom-blocked layouts
# ----------------------------------------------------------------------------

def offsets(sizes) -> np.ndarray:
    s = np.asarray(sizes, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(s)])


def block_sq_sums(x: np.ndarray, cuts: list[np.ndarray]) -> np.ndarray:
    """Sum of squares of x over the atom blocks given by per-axis offsets."""
    s = x * x
    for ax, off in enumerate(cuts):
        s = np.add.reduceat(s, off[:-1], axis=ax)
    return s


def dense_three_center(n_ao, n_ri, blocks, offs, data, thr: float = 0.0) -> np.ndarray:
    """Dense T[lambda, sigma, P] from the stored A <= B atom blocks.

    The (B, A, P) block is the (A, B, P) block transposed in its two primary
    indices (Eq. 4 is symmetric under that exchange).  A stored block whose
    Frobenius norm is < thr is dropped, together with its mirror.
    """
    ao = offsets(n_ao)
    ri = offsets(n_ri)
    t = np.zeros((ao[-1], ao[-1], ri[-1]))
    for i, (a, b, p) in enumerate(blocks):
        blk = data[offs[i]:offs[i + 1]].reshape(n_ao[a], n_ao[b], n_ri[p])
        if thr > 0.0 and np.sqrt(np.sum(blk * blk)) < thr:
            continue
        t[ao[a]:ao[a + 1], ao[b]:ao[b + 1], ri[p]:ri[p + 1]] = blk
        if a != b:
            t[ao[b]:ao[b + 1], ao[a]:ao[a + 1], ri[p]:ri[p + 1]] = blk.transpose(1, 0, 2)
    return t


# ----------------------------------------------------------------------------
# Eq. 2
# ----------------------------------------------------------------------------

def greens(C: np.ndarray, eps: np.ndarray, n_occ: int, mu_fermi: float, tau: float):
    """(G^occ(tau), G^virt(tau)), Eq. 2 without its phase factors.

    C[mu, n] holds orbital n (the paper's C_{n mu}); eps ascending; the first
    n_occ orbitals are occupied.
    """
    co = C[:, :n_occ]
    cv = C[:, n_occ:]
    wo = np.exp((eps[:n_occ] - mu_fermi) * tau)
    wv = np.exp(-(eps[n_occ:] - mu_fermi) * tau)
    g_occ = (co * wo) @ co.T
    g_virt = (cv * wv) @ cv.T
    return g_occ, g_virt


def filter_sym_2d(g: np.ndarray, ao: np.ndarray, thr: float) -> np.ndarray:
    """Zero the atom blocks (A, B) of a symmetric matrix with norm < thr.

    The decision for (A, B) and (B, A) is the one of the block with A <= B.
    """
    if thr <= 0.0:
        return g
    nrm = np.sqrt(block_sq_sums(g, [ao, ao]))
    up = np.triu(nrm)
    nrm = up + np.triu(up, 1).T
    keep = nrm >= thr
    sizes = np.diff(ao)
    mask = np.repeat(np.repeat(keep, sizes, axis=0), sizes, axis=1)
    return np.where(mask, g, 0.0)


def filter_3idx(x: np.ndarray, cuts: list[np.ndarray], thr: float) -> np.ndarray:
    """Zero the atom blocks of a 3-index tensor with Frobenius norm < thr."""
    if thr <= 0.0:
        return x
    nrm = np.sqrt(block_sq_sums(x, cuts))
    keep = nrm >= thr
    for ax, off in enumerate(cuts):
        keep = np.repeat(keep, np.diff(off), axis=ax)
    return np.where(keep, x, 0.0)


def mirror_upper(chi: np.ndarray, ri: np.ndarray) -> np.ndarray:
    """chi[P, Q] := chi[Q, P] wherever atom(P) > atom(Q)."""
    atom = np.repeat(np.arange(len(ri) - 1), np.diff(ri))
    lower = atom[:, None] > atom[None, :]
    return np.where(lower, chi.T, chi)


# ----------------------------------------------------------------------------
# Eq. 3, dense in all indices (small systems)
# ----------------------------------------------------------------------------

def chi_dense_from_g(t: np.ndarray, g_occ: np.ndarray, g_virt: np.ndarray,
                     ao: np.ndarray, ri: np.ndarray, thr: float = 0.0,
                     mirror: bool = True) -> np.ndarray:
    """chi[P, Q] of Eq. 3 with the block filter, from dense T and G."""
    g_occ = filter_sym_2d(g_occ, ao, thr)
    g_virt = filter_sym_2d(g_virt, ao, thr)
    m = np.einsum("ml,lsp->msp", g_occ, t, optimize=True)
    m = filter_3idx(m, [ao, ao, ri], thr)
    n = np.einsum("mnq,ns->msq", t, g_virt, optimize=True)
    n = filter_3idx(n, [ao, ao, ri], thr)
    nao = t.shape[0]
    chi = -(m.reshape(nao * nao, -1).T @ n.reshape(nao * nao, -1))
    return mirror_upper(chi, ri) if mirror else chi


def chi_dense(case, tau_index: int | None = None, thr: float | None = None,
              mirror: bool = True) -> np.ndarray:
    """chi for every tau of a synth Case (or one tau): [n_tau, n_RI, n_RI]."""
    sysm = case.system
    thr = case.thr if thr is None else thr
    ao = offsets(sysm.n_ao)
    ri = offsets(sysm.n_ri)
    t = dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                           case.t3c.data, thr)
    taus = case.tau if tau_index is None else case.tau[[tau_index]]
    out = []
    for tau in taus:
        go, gv = greens(case.C, case.eps, case.n_occ, case.mu_fermi, tau)
        out.append(chi_dense_from_g(t, go, gv, ao, ri, thr, mirror))
    return np.stack(out)


# ----------------------------------------------------------------------------
# independent routes (pins)
# ----------------------------------------------------------------------------

def chi_mo_route(t: np.ndarray, C: np.ndarray, eps: np.ndarray, n_occ: int,
                 tau: float) -> np.ndarray:
    """Eq. 3 with Eq. 2 inserted and the AO sums done first:
    chi_PQ = - sum_{i occ, a virt} exp(-(eps_a - eps_i) tau) B^{ia}_P B^{ia}_Q,
    B^{ia}_P = sum_{lambda sigma} C_lambda,i C_sigma,a T[lambda, sigma, P].
    Unfiltered; independent of any atom blocking and of mu_F."""
    co = C[:, :n_occ]
    cv = C[:, n_occ:]
    b = np.einsum("li,lsp,sa->iap", co, t, cv, optimize=True)
    w = np.exp(-(eps[None, n_occ:] - eps[:n_occ, None]) * tau)
    bw = b * w[:, :, None]
    nb = b.shape[0] * b.shape[1]
    return -(bw.reshape(nb, -1).T @ b.reshape(nb, -1))


def chi_bruteforce(t: np.ndarray, g_occ: np.ndarray, g_virt: np.ndarray) -> np.ndarray:
    """Eq. 3 as written, one scalar term at a time (pure-Python loops).

    chi_PQ = - sum_{mu sigma} sum_lambda T[lambda, sigma, P] G^occ[mu, lambda]
                              * sum_nu T[mu, nu, Q] G^virt[nu, sigma]
    Only for a handful of basis functions.
    """
    nao, _, nri = t.shape
    chi = [[0.0] * nri for _ in range(nri)]
    tl = t.tolist()
    go = g_occ.tolist()
    gv = g_virt.tolist()
    for p in range(nri):
        for q in range(nri):
            acc = 0.0
            for mu in range(nao):
                for sg in range(nao):
                    left = 0.0
                    for lam in range(nao):
                        left += tl[lam][sg][p] * go[mu][lam]
                    right = 0.0
                    for nu in range(nao):
                        right += tl[mu][nu][q] * gv[nu][sg]
                    acc += left * right
            chi[p][q] = -acc
    return np.array(chi)


# ----------------------------------------------------------------------------
# Eq. 3 one atom block at a time (large systems)
# ----------------------------------------------------------------------------

class BlockOracle:
    """chi atom blocks (p-atom, q-atom) of Eq. 3 for systems too large for the
    dense route, with the same filter semantics as chi_dense.

    M[:, :, P in p] needs only T[:, :, P in p] and is computed for all
    (mu, sigma); N[:, :, Q in q] likewise; the block is - sum M N.  Each block
    is independent of every other, so any subset can be checked.
    """

    def __init__(self, case, thr: float | None = None):
        sysm = case.system
        self.case = case
        self.thr = case.thr if thr is None else thr
        self.n_ao = sysm.n_ao
        self.n_ri = sysm.n_ri
        self.ao = offsets(sysm.n_ao)
        self.ri = offsets(sysm.n_ri)
        t3 = case.t3c
        self.blocks = t3.blocks
        self.offs = t3.offsets
        self.data = t3.data
        # per RI atom: indices of stored blocks that survive the T filter
        keep = np.ones(len(self.blocks), dtype=bool)
        if self.thr > 0.0:
            for i in range(len(self.blocks)):
                blk = self.data[self.offs[i]:self.offs[i + 1]]
                keep[i] = np.sqrt(np.sum(blk * blk)) >= self.thr
        self.by_p: dict[int, np.ndarray] = {}
        ps = self.blocks[:, 2]
        for p in range(len(self.n_ri)):
            self.by_p[p] = np.nonzero((ps == p) & keep)[0]
        self._g = {}

    def greens(self, tau_index: int):
        if tau_index not in self._g:
            c = self.case
            go, gv = greens(c.C, c.eps, c.n_occ, c.mu_fermi, c.tau[tau_index])
            self._g = {tau_index: (filter_sym_2d(go, self.ao, self.thr),
                                   filter_sym_2d(gv, self.ao, self.thr))}
        return self._g[tau_index]

    def t_slice(self, p: int):
        """(idx, Tp): AO indices touched by RI atom p and T[idx, idx, P in p]."""
        ids = self.by_p[p]
        atoms = np.unique(np.concatenate([self.blocks[ids, 0], self.blocks[ids, 1]]))
        pos = {}
        idx = []
        for a in atoms:
            pos[a] = len(idx)
            idx.extend(range(self.ao[a], self.ao[a + 1]))
        idx = np.array(idx, dtype=np.int64)
        npp = self.n_ri[p]
        tp = np.zeros((len(idx), len(idx), npp))
        for i in ids:
            a, b, _ = self.blocks[i]
            blk = self.data[self.offs[i]:self.offs[i + 1]].reshape(self.n_ao[a], self.n_ao[b], npp)
            ia, ib = pos[a], pos[b]
            tp[ia:ia + self.n_ao[a], ib:ib + self.n_ao[b]] = blk
            if a != b:
                tp[ib:ib + self.n_ao[b], ia:ia + self.n_ao[a]] = blk.transpose(1, 0, 2)
        return idx, atoms, tp

    def _atom_cuts(self, atoms):
        sizes = self.n_ao[atoms]
        return offsets(sizes)

    def _partners(self, atoms, tp):
        """Per atom b of the slice: positions (in idx) of the functions of the
        atoms a with a stored block (a, b, P) or (b, a, P) -- the only rows of
        T[:, b, P] (and, T being symmetric in its primary indices, of
        T[b, :, P]) that can be nonzero."""
        sizes = self.n_ao[atoms]
        cuts = offsets(sizes)
        nz = np.abs(tp).sum(axis=2) > 0.0                        # [k, k]
        nza = np.add.reduceat(np.add.reduceat(nz, cuts[:-1], axis=0), cuts[:-1], axis=1) > 0
        out = []
        for j in range(len(atoms)):
            rows = [np.arange(cuts[i], cuts[i + 1]) for i in np.nonzero(nza[:, j])[0]]
            out.append(np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64))
        return cuts, out

    def m_slice(self, tau_index: int, p: int):
        """M[mu, sigma in idx_p, P in p] = sum_lambda G^occ[mu, lambda] T[lambda, sigma, P], filtered.

        Computed one sigma-atom b at a time: the lambda sum runs over the
        functions of the atoms that share a stored block with b at this RI
        atom (every other term is an exact zero of T), and each atom block
        (mu-atom, b, p) of the result is dropped when its Frobenius norm is
        < thr, the filter of chi_dense."""
        go, _ = self.greens(tau_index)
        idx, atoms, tp = self.t_slice(p)
        k = len(idx)
        npp = self.n_ri[p]
        nao = go.shape[0]
        cuts, part = self._partners(atoms, tp)
        m = np.empty((nao, k, npp))
        for j in range(len(atoms)):
            lam = part[j]
            c0, c1 = cuts[j], cuts[j + 1]
            if lam.size == 0:
                m[:, c0:c1, :] = 0.0
                continue
            tb = tp[lam, c0:c1, :].reshape(lam.size, (c1 - c0) * npp)
            # G^occ is symmetric (Eq. 2): its columns idx[lam] are read as rows
            r = go[idx[lam], :].T @ tb                            # [nao, nb * nP]
            if self.thr > 0.0:
                nrm = np.sqrt(np.add.reduceat(np.einsum("ij,ij->i", r, r), self.ao[:-1]))
                r[np.repeat(nrm < self.thr, self.n_ao)] = 0.0
            m[:, c0:c1, :] = r.reshape(nao, c1 - c0, npp)
        return idx, m

    def n_slice(self, tau_index: int, q: int):
        """N[mu in idx_q, sigma, Q in q] = sum_nu T[mu, nu, Q] G^virt[nu, sigma], filtered.

        Computed one mu-atom a at a time: the nu sum runs over the functions of
        the atoms that share a stored block with a at this RI atom, and each
        atom block (a, sigma-atom, q) with Frobenius norm < thr is dropped."""
        _, gv = self.greens(tau_index)
        idx, atoms, tq = self.t_slice(q)
        k = len(idx)
        nq = self.n_ri[q]
        nao = gv.shape[0]
        cuts, part = self._partners(atoms, tq)
        n = np.empty((k, nao, nq))
        for i in range(len(atoms)):
            nu = part[i]
            c0, c1 = cuts[i], cuts[i + 1]
            if nu.size == 0:
                n[c0:c1] = 0.0
                continue
            ta = tq[c0:c1, nu, :].transpose(0, 2, 1).reshape((c1 - c0) * nq, nu.size)
            r = ta @ gv[idx[nu], :]                               # [na * nQ, nao]
            if self.thr > 0.0:
                nrm = np.sqrt(np.add.reduceat(np.einsum("ij,ij->j", r, r), self.ao[:-1]))
                r[:, np.repeat(nrm < self.thr, self.n_ao)] = 0.0
            n[c0:c1] = r.reshape(c1 - c0, nq, nao).transpose(0, 2, 1)
        return idx, n

    def block(self, tau_index: int, p: int, q: int, cache: dict | None = None) -> np.ndarray:
        """chi[P in p, Q in q] with the atom upper-triangle convention."""
        if p > q:
            return self.block(tau_index, q, p, cache).T
        cache = {} if cache is None else cache
        key_m = ("m", tau_index, p)
        key_n = ("n", tau_index, q)
        if key_m not in cache:
            cache[key_m] = self.m_slice(tau_index, p)
        if key_n not in cache:
            cache[key_n] = self.n_slice(tau_index, q)
        idx_p, m = cache[key_m]
        idx_q, n = cache[key_n]
        # sum over mu in idx_q (where N lives) and sigma in idx_p (where M lives)
        mm = m[idx_q]                     # [|idx_q|, |idx_p|, nP]
        nn = n[:, idx_p]                  # [|idx_q|, |idx_p|, nQ]
        kk = mm.shape[0] * mm.shape[1]
        return -(mm.reshape(kk, -1).T @ nn.reshape(kk, -1))


# ----------------------------------------------------------------------------
# useful work of one tau point (the flops the method must do after filtering)
# ----------------------------------------------------------------------------

def _count_c(n_ao, n_ri, keep_m, keep_n) -> float:
    """F_C = sum over (mu-atom m, sigma-atom s) and RI atoms p <= q of
    2 n(m) n(s) n(p) n(q), for kept nonzero M(m, s, p) and N(m, s, q)."""
    nao = np.asarray(n_ao, dtype=float)
    nri = np.asarray(n_ri, dtype=float)
    xm = keep_m * nri[None, None, :]                         # [m, s, p]
    xn = keep_n * nri[None, None, :]                         # [m, s, q]
    suffix = np.cumsum(xn[:, :, ::-1], axis=2)[:, :, ::-1]   # sum over q >= p
    per_pair = np.sum(xm * suffix, axis=2)                   # [m, s]
    return float(2.0 * nao @ per_pair @ nao)


def _count_ab(case, thr, keep_go, keep_gv):
    """(F_A, F_B): every stored T block orientation (lambda-atom, sigma-atom,
    P) that survives the T filter, times every kept G block (mu-atom,
    lambda-atom): 2 n(mu) n(lambda) n(sigma) n(P) flops (G^occ for step A,
    G^virt for step B)."""
    s = case.system
    blk = case.t3c.blocks
    fa = fb = 0.0
    for i, (a, b, p) in enumerate(blk):
        d = case.t3c.data[case.t3c.offsets[i]:case.t3c.offsets[i + 1]]
        if thr > 0.0 and np.sqrt(np.sum(d * d)) < thr:
            continue
        w = 2.0 * s.n_ao[a] * s.n_ao[b] * s.n_ri[p]
        for lam in ((a,) if a == b else (a, b)):
            fa += w * float(s.n_ao @ keep_go[:, lam])
            fb += w * float(s.n_ao @ keep_gv[:, lam])
    return fa, fb


def _g_keep(g, ao, thr):
    """Kept nonzero atom blocks of a filtered symmetric G (thr 0 keeps all)."""
    if thr <= 0.0:
        return np.ones((len(ao) - 1, len(ao) - 1), dtype=bool)
    return np.sqrt(block_sq_sums(filter_sym_2d(g, ao, thr), [ao, ao])) > 0.0


def useful_flops_dense(case, tau_index: int, thr: float | None = None):
    """(F_A, F_B, F_C) of one tau point from the dense route (small systems):
    the flops of the atom-block products of Eq. 3 whose operands survive the
    filter (kept and nonzero), each product counted once; chi's atom-block
    upper triangle p <= q for step C."""
    sysm = case.system
    thr = case.thr if thr is None else thr
    ao, ri = offsets(sysm.n_ao), offsets(sysm.n_ri)
    t = dense_three_center(sysm.n_ao, sysm.n_ri, case.t3c.blocks, case.t3c.offsets,
                           case.t3c.data, thr)
    go, gv = greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau[tau_index])
    go, gv = filter_sym_2d(go, ao, thr), filter_sym_2d(gv, ao, thr)
    m = filter_3idx(np.einsum("ml,lsp->msp", go, t, optimize=True), [ao, ao, ri], thr)
    n = filter_3idx(np.einsum("mnq,ns->msq", t, gv, optimize=True), [ao, ao, ri], thr)
    keep_m = np.sqrt(block_sq_sums(m, [ao, ao, ri])) > 0.0
    keep_n = np.sqrt(block_sq_sums(n, [ao, ao, ri])) > 0.0
    fa, fb = _count_ab(case, thr, _g_keep(go, ao, thr), _g_keep(gv, ao, thr))
    return fa, fb, _count_c(sysm.n_ao, sysm.n_ri, keep_m, keep_n)


def useful_flops_blocks(bo: BlockOracle, tau_index: int):
    """(F_A, F_B, F_C) of one tau point from the block oracle's M and N slices
    (large systems): the same count as useful_flops_dense."""
    n_at = len(bo.n_ao)
    keep_m = np.zeros((n_at, n_at, n_at), dtype=bool)
    keep_n = np.zeros((n_at, n_at, n_at), dtype=bool)
    for p in range(n_at):
        idx, m = bo.m_slice(tau_index, p)
        _, atoms, _ = bo.t_slice(p)
        cuts = bo._atom_cuts(atoms)
        nm = np.add.reduceat(np.add.reduceat(np.sum(m * m, axis=2), bo.ao[:-1], axis=0),
                             cuts[:-1], axis=1)
        keep_m[:, atoms, p] = nm > 0.0
        idx, n = bo.n_slice(tau_index, p)
        nn = np.add.reduceat(np.add.reduceat(np.sum(n * n, axis=2), cuts[:-1], axis=0),
                             bo.ao[:-1], axis=1)
        keep_n[atoms, :, p] = nn > 0.0
    go, gv = bo.greens(tau_index)
    fa, fb = _count_ab(bo.case, bo.thr, _g_keep(go, bo.ao, bo.thr), _g_keep(gv, bo.ao, bo.thr))
    return fa, fb, _count_c(bo.n_ao, bo.n_ri, keep_m, keep_n)
