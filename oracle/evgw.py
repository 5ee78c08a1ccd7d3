"""Oracle for eigenvalue-self-consistent GW (evGW): the quasiparticle
energies of Eq. 12 replace the mean-field levels in the Green's functions of
Eq. 2, and the cycle chi (Eq. 3) -> W (Eqs. 7-9) -> Sigma^c (Eq. 10) ->
quasiparticle equation (Eq. 12) repeats until the energies stop changing
(the paragraph after Eq. 12).  FP64 numpy, built from the other oracle
modules.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* Only the levels of the listed orbitals are computed.  Every other level
  moves by the shift e_n - eps_n of the nearest computed level on its side of
  the gap (nearest by index; on a tie, the one nearer the gap).  With HOMO and
  LUMO computed this is the usual scissor shift of the occupied and virtual
  levels.  A side with no computed level keeps its mean-field levels.
* The quasiparticle equation keeps its mean-field part,
  e = eps_n - vxc_n + Sigma^x_n + Re Sigma^c_n(e), with eps_n the input level:
  only G (hence chi, W and Sigma^c) sees the updated levels.  Sigma^x depends
  on the occupied orbitals alone and is computed once.
* The orbitals C, the Fermi level, the tau and omega grids and the transform
  weights stay fixed.  No mixing between cycles.
* Converged when no computed energy changes by tol or more between two
  cycles; the first cycle is G0W0.
"""

from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import chain as och
from . import chi as oc
from . import qp
from . import sigma as osg


def shifted_levels(eps: np.ndarray, n_occ: int, orbitals, e_qp) -> np.ndarray:
    """Levels of the next cycle: computed orbitals at their quasiparticle
    energies, every other level shifted with the nearest computed level on
    its side of the gap."""
    orbitals = [int(n) for n in orbitals]
    shift = np.asarray(e_qp, dtype=float) - eps[orbitals]
    out = np.array(eps, dtype=float)
    for i in range(len(eps)):
        occ = i < n_occ
        same = [k for k, n in enumerate(orbitals) if (n < n_occ) == occ]
        if not same:
            continue
        # distance first; on a tie the higher index for occupied levels and
        # the lower for virtual ones (the one nearer the gap)
        k = min(same, key=lambda k: (abs(orbitals[k] - i), -orbitals[k] if occ else orbitals[k]))
        out[i] = eps[i] + shift[k]
    return out


def gw_cycle(case, levels, v, omega, gamma, delta, s_weights, orbitals, vxc, sx) -> np.ndarray:
    """One GW cycle with G of Eq. 2 built from `levels`: chi (Eq. 3), W^c
    (Eqs. 7-9), Sigma^c (Eq. 10) and the quasiparticle equation (Eq. 12) with
    the mean-field levels of `case`."""
    cur = replace(case, eps=np.asarray(levels, dtype=float))
    chi = oc.chi_dense(cur)
    w_tau, _ = och.chi_to_w(chi, v, gamma, delta)
    sig = osg.sigma_dense(cur, w_tau, orbitals, thr=case.thr)
    eps_n = case.eps[np.asarray(orbitals)]
    return qp.quasiparticle_energies(sig, omega, gamma, s_weights, eps_n, vxc, sx)


def evgw(case, v, omega, gamma, delta, s_weights, orbitals, vxc, max_cycles: int = 20,
         tol: float = 1e-6):
    """(energies of the listed orbitals, cycles run, converged, the levels G
    was built from in the last cycle)."""
    sx = qp.sigma_x_dense(case, v, orbitals, thr=case.thr)
    levels = np.array(case.eps, dtype=float)
    prev = None
    for cycle in range(1, max_cycles + 1):
        e = gw_cycle(case, levels, v, omega, gamma, delta, s_weights, orbitals, vxc, sx)
        if prev is not None and np.max(np.abs(e - prev)) < tol:
            return e, cycle, True, levels
        prev = e
        levels = shifted_levels(case.eps, case.n_occ, orbitals, e)
    return prev, max_cycles, False, levels
