"""Writes flops_ribbon298.json: the useful flops (F_A, F_B, F_C) of one tau
point of the 298-atom ribbon workload (3090 AO / 7176 RI, thr 1e-9), counted
by the oracle from its own filtered blocks (oracle.chi.useful_flops_blocks).

Both CPU legs of bench.py divide by this count, and a GPU test checks the
library's own count against it.  Run from the repository root:
    python tests/golden/make_flops_ribbon298.py [tau_index ...]
(about ten minutes per tau point on eight cores)."""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import chi as oc  # noqa: E402
from synth import make_case  # noqa: E402


def main():
    taus = [int(a) for a in sys.argv[1:]] or [10]
    case = make_case("ribbon300")
    bo = oc.BlockOracle(case)
    out = {"workload": "ribbon300 (298 atoms, 3090 AO / 7176 RI, 20 tau, thr 1e-9)",
           "counted_by": "oracle.chi.useful_flops_blocks", "per_tau": {}}
    for j in taus:
        t0 = time.perf_counter()
        fa, fb, fc = oc.useful_flops_blocks(bo, j)
        out["per_tau"][str(j)] = {"tau": float(case.tau[j]), "flops_a": fa, "flops_b": fb,
                                  "flops_c": fc, "seconds": time.perf_counter() - t0}
        print(j, out["per_tau"][str(j)], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flops_ribbon298.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
