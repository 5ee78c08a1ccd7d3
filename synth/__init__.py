"""Seeded synthetic inputs for the imaginary-time polarizability chi_PQ(i tau).

This package builds the *inputs* of the method and nothing else: atom
geometries, per-atom basis sizes, the three-centre tensor (mu sigma | P),
a model Hamiltonian whose eigenpairs stand in for the mean-field orbitals
(C, eps) of the expansion in Gaussian orbitals (Eq. 1), and the imaginary-time
grid.  It holds none of the method's arithmetic (no Green's function, no
contraction, no screening): both the CPU oracle and the CUDA path consume what
it returns.

Every random number comes from one counter-based generator (SplitMix64 over a
global element counter, then Box-Muller), so any block of any tensor can be
regenerated on its own, on any machine, from (seed, stream, index).
"""

from .rng import normal_stream, uniform_stream
from .systems import (
    System,
    benzene_ring,
    armchair_ribbon,
    random_cluster,
    species_basis,
    tiny_chain,
    carbon_ring_with_h,
    molecule_set,
)
from .tensors import (
    ThreeCenter,
    make_three_center,
    make_hamiltonian,
    orbitals_from_hamiltonian,
    log_tau_grid,
    make_case,
    case_from_system,
    Case,
)

__all__ = [
    "normal_stream",
    "uniform_stream",
    "System",
    "benzene_ring",
    "armchair_ribbon",
    "random_cluster",
    "species_basis",
    "tiny_chain",
    "carbon_ring_with_h",
    "molecule_set",
    "case_from_system",
    "ThreeCenter",
    "make_three_center",
    "make_hamiltonian",
    "orbitals_from_hamiltonian",
    "log_tau_grid",
    "make_case",
    "Case",
]
