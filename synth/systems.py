"""Atom geometries and per-atom basis sizes of the synthetic workloads.

Species carry only basis sizes: a 'C' atom holds 13 primary Gaussian functions
and 30 auxiliary (RI) functions, an 'H' atom 5 and 12.  Distances are in
Angstrom.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import uniform_stream

CC_BOND = 1.4
CH_BOND = 1.09

_BASIS = {"C": (13, 30), "H": (5, 12)}


def species_basis(species: str) -> tuple[int, int]:
    """(n_ao, n_ri) of one atom of the given species."""
    return _BASIS[species]


@dataclass
class System:
    name: str
    xyz: np.ndarray            # [n_atoms, 3] float64, Angstrom
    species: list[str]
    n_ao: np.ndarray = field(init=False)   # [n_atoms] int32
    n_ri: np.ndarray = field(init=False)   # [n_atoms] int32

    def __post_init__(self) -> None:
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64)
        self.n_ao = np.array([_BASIS[s][0] for s in self.species], dtype=np.int32)
        self.n_ri = np.array([_BASIS[s][1] for s in self.species], dtype=np.int32)

    @property
    def n_atoms(self) -> int:
        return len(self.species)

    @property
    def nao_total(self) -> int:
        return int(self.n_ao.sum())

    @property
    def nri_total(self) -> int:
        return int(self.n_ri.sum())

    @property
    def ao_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_ao)]).astype(np.int64)

    @property
    def ri_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_ri)]).astype(np.int64)

    @property
    def n_electrons(self) -> int:
        """All-electron count (C = 6, H = 1)."""
        return sum(6 if s == "C" else 1 for s in self.species)


def benzene_ring() -> System:
    """Planar hexagon: six C on a 1.4 A ring, one H 1.09 A radially outside each."""
    ang = np.arange(6) * (np.pi / 3.0)
    c = np.stack([CC_BOND * np.cos(ang), CC_BOND * np.sin(ang), np.zeros(6)], axis=1)
    h = np.stack([(CC_BOND + CH_BOND) * np.cos(ang), (CC_BOND + CH_BOND) * np.sin(ang),
                  np.zeros(6)], axis=1)
    return System("benzene-ring-12", np.concatenate([c, h]), ["C"] * 6 + ["H"] * 6)


def armchair_ribbon(n_cells: float, width: int = 4) -> System:
    """Armchair graphene-nanoribbon-shaped chain along x.

    `width` dimer lines across the ribbon; rows k = 0..width-1 sit at
    y = k * (sqrt(3)/2) * a with two carbons per 3a period along x (offset by
    1.5 a on odd rows).  Each carbon of the two edge rows is two-coordinated
    and gets one hydrogen at 1.09 A along the outward bisector of its bonds.
    A 4-wide ribbon has 8 C + 4 H per 4.2 A cell (C:H = 2:1).  A fractional
    `n_cells` adds the atoms of the next cell whose x lies inside the length.
    """
    a = CC_BOND
    period = 3.0 * a
    length = n_cells * period
    ncell_int = int(np.ceil(n_cells)) + 1
    carb = []
    for k in range(width):
        y = k * (np.sqrt(3.0) / 2.0) * a
        base = [0.0, a] if k % 2 == 0 else [1.5 * a, 2.5 * a]
        for c in range(ncell_int):
            for x0 in base:
                x = c * period + x0
                if x < length - 1e-9:
                    carb.append((x, y, 0.0))
    carb = np.array(carb)
    # bonds: neighbours at distance a
    d = np.linalg.norm(carb[:, None, :] - carb[None, :, :], axis=2)
    nb = (d > 0.1) & (d < a * 1.05)
    hyd = []
    ymax = (width - 1) * (np.sqrt(3.0) / 2.0) * a
    for i, p in enumerate(carb):
        on_edge = abs(p[1]) < 1e-9 or abs(p[1] - ymax) < 1e-9
        if not on_edge or nb[i].sum() != 2:
            continue
        v = (carb[nb[i]] - p).sum(axis=0)
        v = -v / np.linalg.norm(v)
        hyd.append(p + CH_BOND * v)
    hyd = np.array(hyd).reshape(-1, 3)
    # order atoms along the ribbon axis (C and H interleaved by x), stable
    xyz = np.concatenate([carb, hyd])
    spec = ["C"] * len(carb) + ["H"] * len(hyd)
    order = np.lexsort((xyz[:, 1], np.round(xyz[:, 0], 6)))
    return System(f"armchair-ribbon-{len(spec)}", xyz[order], [spec[i] for i in order])


def tiny_chain(species: str, spacing: float = 1.4) -> System:
    """Linear chain of the given species string (e.g. 'CHC'), for brute-force tests."""
    n = len(species)
    xyz = np.stack([np.arange(n) * spacing, np.zeros(n), np.zeros(n)], axis=1)
    return System(f"chain-{species}", xyz, list(species))


def random_cluster(n_atoms: int, density: float, min_dist: float, seed: int,
                   p_carbon: float = 2.0 / 3.0) -> System:
    """Uniform random positions in a cube of n/density volume, rejection-sampled
    to a minimum separation; each atom is 'C' with probability p_carbon."""
    box = (n_atoms / density) ** (1.0 / 3.0)
    pts = np.zeros((0, 3))
    ctr = 0
    while len(pts) < n_atoms:
        u = uniform_stream(seed, 1, ctr, 3 * 256).reshape(256, 3) * box
        ctr += 3 * 256
        for p in u:
            if len(pts) == n_atoms:
                break
            if len(pts) == 0 or np.min(np.linalg.norm(pts - p, axis=1)) >= min_dist:
                pts = np.vstack([pts, p])
    sp = uniform_stream(seed, 2, 0, n_atoms)
    species = ["C" if s < p_carbon else "H" for s in sp]
    return System(f"cluster-{n_atoms}", pts, species)


def carbon_ring_with_h(n_atoms: int) -> System:
    """Planar ring: n_c carbons 1.4 A apart on a circle, an H 1.09 A radially
    outside every other carbon (C:H = 2:1); n_atoms = n_c + n_c // 2."""
    n_c = max(3, int(round(n_atoms * 2 / 3)))
    radius = CC_BOND / (2.0 * np.sin(np.pi / n_c))
    ang = 2.0 * np.pi * np.arange(n_c) / n_c
    c = np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n_c)], axis=1)
    hi = np.arange(0, n_c, 2)
    h = np.stack([(radius + CH_BOND) * np.cos(ang[hi]), (radius + CH_BOND) * np.sin(ang[hi]),
                  np.zeros(len(hi))], axis=1)
    return System(f"ring-{n_c + len(hi)}", np.concatenate([c, h]), ["C"] * n_c + ["H"] * len(hi))


def molecule_set(n_mol: int, lo: int, hi: int, seed: int) -> list[System]:
    """n_mol molecules with atom counts uniform on [lo, hi]: odd index a
    ribbon segment (cells chosen to reach the count), even index a ring."""
    counts = lo + np.floor(uniform_stream(seed, 3, 0, n_mol) * (hi - lo + 1)).astype(int)
    out = []
    for i, n in enumerate(counts):
        if i % 2 == 1:
            out.append(armchair_ribbon(max(1.0, n / 12.0)))
        else:
            out.append(carbon_ring_with_h(int(n)))
    return out
