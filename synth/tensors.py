"""Synthetic three-centre tensor, model Hamiltonian, orbitals and tau grid.

Recipe (units: Angstrom for distances, Hartree for energies, a.u. for tau):

* three-centre tensor (mu sigma | P), stored in atom blocks (A, B, P) with
  A <= B, data [n_ao(A)][n_ao(B)][n_ri(P)] row-major.  Entry =
  z * exp(-0.5 r_AB^2) * exp(-0.8 r_mid,P), z ~ N(0,1), r_AB the distance of
  the two primary-basis atoms and r_mid,P the distance from their midpoint to
  the auxiliary atom.  A == B blocks are symmetrised in their two primary
  indices, (X + X^T)/2, so the tensor is symmetric under mu <-> sigma as the
  overlap integral of Eq. 4 is.  A block is stored iff thr == 0 or its expected
  Frobenius norm scale * sqrt(nA nB nP) >= thr.
* model Hamiltonian in an orthonormal primary basis: H = (X + X^T)/2 with
  X_mu,nu = z * exp(-r_AB) for r_AB <= 5 A, else 0, z ~ N(0,1).
* orbitals: eigenpairs of H; energies scaled to a 2 Ha spectral width, then
  the n_occ lowest shifted so that HOMO = -0.15 Ha and the rest so that
  LUMO = +0.15 Ha (gap 0.3 Ha, Fermi level 0).
* tau grid: tau_j = 0.01 * 5000^((j-1)/(n_tau-1)), j = 1..n_tau (0.01 .. 50 a.u.).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import normal_stream
from .systems import System, armchair_ribbon, benzene_ring, random_cluster, tiny_chain

STREAM_3C = 11
STREAM_H = 12
STREAM_W = 13

DECAY_AO = 0.5      # exp(-0.5 r_AB^2)
DECAY_RI = 0.8      # exp(-0.8 r_mid,P)
H_CUTOFF = 5.0
SPECTRAL_WIDTH = 2.0
HALF_GAP = 0.15


@dataclass
class ThreeCenter:
    """Atom-blocked three-centre tensor with A <= B blocks only.

    blocks  : [n_blocks, 3] int32 (A, B, P), sorted lexicographically
    offsets : [n_blocks + 1] int64 start of each block in `data`
    data    : [n_elems] float64
    """

    blocks: np.ndarray
    offsets: np.ndarray
    data: np.ndarray

    @property
    def n_blocks(self) -> int:
        return int(self.blocks.shape[0])

    def block(self, i: int, sysm: System) -> np.ndarray:
        a, b, p = self.blocks[i]
        return self.data[self.offsets[i]:self.offsets[i + 1]].reshape(
            sysm.n_ao[a], sysm.n_ao[b], sysm.n_ri[p])


def block_scales(sysm: System) -> np.ndarray:
    """[n_at, n_at, n_at] expected element scale of block (A, B, P)."""
    x = sysm.xyz
    r_ab = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    mid = 0.5 * (x[:, None, :] + x[None, :, :])
    r_mp = np.linalg.norm(mid[:, :, None, :] - x[None, None, :, :], axis=3)
    return np.exp(-DECAY_AO * r_ab * r_ab)[:, :, None] * np.exp(-DECAY_RI * r_mp)


def make_three_center(sysm: System, thr: float, seed: int) -> ThreeCenter:
    n = sysm.n_atoms
    nao = sysm.n_ao.astype(np.int64)
    nri = sysm.n_ri.astype(np.int64)
    # per A: scales against all (B, P) -- avoids an n^3 x 3 temporary
    blk_list = []
    size_list = []
    scale_list = []
    x = sysm.xyz
    for a in range(n):
        bs = np.arange(a, n)
        r_ab = np.linalg.norm(x[bs] - x[a], axis=1)
        mid = 0.5 * (x[bs] + x[a])
        r_mp = np.linalg.norm(mid[:, None, :] - x[None, :, :], axis=2)
        sc = np.exp(-DECAY_AO * r_ab * r_ab)[:, None] * np.exp(-DECAY_RI * r_mp)
        sizes = (nao[a] * nao[bs])[:, None] * nri[None, :]
        if thr > 0.0:
            keep = sc * np.sqrt(sizes.astype(np.float64)) >= thr
        else:
            keep = np.ones_like(sc, dtype=bool)
        bi, pi = np.nonzero(keep)
        blk_list.append(np.stack([np.full(bi.shape, a), bs[bi], pi], axis=1))
        size_list.append(sizes[bi, pi])
        scale_list.append(sc[bi, pi])
    blocks = np.concatenate(blk_list).astype(np.int32)
    sizes = np.concatenate(size_list).astype(np.int64)
    scales = np.concatenate(scale_list)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(offsets[-1])
    data = normal_stream(seed, STREAM_3C, 0, total)
    # scale each block (runs of blocks of at most 2^26 elements at a time, so
    # that no second array of the tensor's size is needed)
    b0 = 0
    step = 1 << 26
    while b0 < len(sizes):
        b1 = int(np.searchsorted(offsets, offsets[b0] + step, side="right")) - 1
        b1 = min(max(b1, b0 + 1), len(sizes))
        data[offsets[b0]:offsets[b1]] *= np.repeat(scales[b0:b1], sizes[b0:b1])
        b0 = b1
    # symmetrise A == B blocks, (X + X^T) / 2 in the primary indices, grouped by
    # block shape
    diag = np.nonzero(blocks[:, 0] == blocks[:, 1])[0]
    shapes = np.stack([nao[blocks[diag, 0]], nri[blocks[diag, 2]]], axis=1)
    for na, npp in np.unique(shapes, axis=0):
        ids = diag[(shapes[:, 0] == na) & (shapes[:, 1] == npp)]
        sz = int(na * na * npp)
        for c0 in range(0, len(ids), 4096):
            sel = ids[c0:c0 + 4096]
            pos = offsets[sel][:, None] + np.arange(sz)[None, :]
            blk = data[pos].reshape(-1, na, na, npp)
            data[pos] = (0.5 * (blk + blk.transpose(0, 2, 1, 3))).reshape(len(sel), sz)
    return ThreeCenter(blocks, offsets, data)


def make_hamiltonian(sysm: System, seed: int) -> np.ndarray:
    nao = sysm.nao_total
    atom_of = np.repeat(np.arange(sysm.n_atoms), sysm.n_ao)
    x = sysm.xyz
    r = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    env = np.where(r <= H_CUTOFF, np.exp(-r), 0.0)
    h = normal_stream(seed, STREAM_H, 0, nao * nao).reshape(nao, nao)
    h *= env[atom_of][:, atom_of]
    return 0.5 * (h + h.T)


def orbitals_from_hamiltonian(h: np.ndarray, n_occ: int) -> tuple[np.ndarray, np.ndarray]:
    """(C, eps): C[mu, n] columns are orbitals, eps ascending, gap 0.3 Ha at 0."""
    w, c = np.linalg.eigh(h)
    w = w * (SPECTRAL_WIDTH / (w[-1] - w[0]))
    eps = w.copy()
    eps[:n_occ] = w[:n_occ] - w[n_occ - 1] - HALF_GAP
    eps[n_occ:] = w[n_occ:] - w[n_occ] + HALF_GAP
    return np.ascontiguousarray(c), eps


def log_tau_grid(n_tau: int, tau_min: float = 0.01, tau_max: float = 50.0) -> np.ndarray:
    if n_tau == 1:
        return np.array([tau_min])
    j = np.arange(n_tau)
    return tau_min * (tau_max / tau_min) ** (j / (n_tau - 1))


@dataclass
class Case:
    name: str
    system: System
    t3c: ThreeCenter
    C: np.ndarray        # [n_ao, n_ao], columns = orbitals
    eps: np.ndarray      # [n_ao]
    n_occ: int
    mu_fermi: float
    tau: np.ndarray
    thr: float
    seed: int


CASES = {
    # name: (system builder, n_tau, thr, seed)
    "benzene": (benzene_ring, 10, 0.0, 20210421),
    "ribbon300": (lambda: armchair_ribbon(25), 20, 1e-9, 20210422),
    "ribbon28": (lambda: armchair_ribbon(2.5), 4, 1e-9, 20210425),
    "ribbon60": (lambda: armchair_ribbon(5), 6, 1e-9, 20210426),
    "ribbon120": (lambda: armchair_ribbon(10), 6, 1e-9, 20210427),
    # 144.5 cells: 1156 C + 576 H = 1732 atoms, 17 908 AO / 41 592 RI
    "ribbon1734": (lambda: armchair_ribbon(144.5), 30, 1e-9, 20210423),
    # 500 atoms uniform in a 17.1 A cube (0.1 atoms/A^3, >= 1.0 A apart), C with
    # probability 2/3: 5220 AO / 12 120 RI
    "cluster500": (lambda: random_cluster(500, 0.1, 1.0, 20210424), 6, 1e-9, 20210424),
    "chain_HH": (lambda: tiny_chain("HH", 1.0), 3, 0.0, 6),
    "chain_CH": (lambda: tiny_chain("CH"), 3, 0.0, 7),
    "chain_HCH": (lambda: tiny_chain("HCH"), 3, 0.0, 8),
    "chain_CHCH": (lambda: tiny_chain("CHCH", 1.2), 4, 0.0, 9),
}


def case_from_system(sysm: System, n_tau: int, thr: float, seed: int) -> Case:
    """A Case for an arbitrary system with the standard recipe."""
    n_occ = max(1, min(sysm.n_electrons // 2, sysm.nao_total - 1))
    t3c = make_three_center(sysm, thr, seed)
    h = make_hamiltonian(sysm, seed)
    c, eps = orbitals_from_hamiltonian(h, n_occ)
    return Case(sysm.name, sysm, t3c, c, eps, n_occ, 0.0, log_tau_grid(n_tau), thr, seed)


def make_case(name: str, n_tau: int | None = None, thr: float | None = None,
              seed: int | None = None, n_occ: int | None = None) -> Case:
    builder, nt, th, sd = CASES[name]
    sysm = builder()
    nt = nt if n_tau is None else n_tau
    th = th if thr is None else thr
    sd = sd if seed is None else seed
    if n_occ is None:
        n_occ = sysm.n_electrons // 2
        n_occ = max(1, min(n_occ, sysm.nao_total - 1))
    t3c = make_three_center(sysm, th, sd)
    h = make_hamiltonian(sysm, sd)
    c, eps = orbitals_from_hamiltonian(h, n_occ)
    return Case(name, sysm, t3c, c, eps, n_occ, 0.0, log_tau_grid(nt), th, sd)
