"""Writes the stored expected values of the sweep tests (calls only oracle/ and qcinputs/).

  python tests/golden/make_golden.py

u1_L10_sweeps.json: energies and largest discarded weights of 6 full sweeps
of the oracle DMRG on the L=10, N=10, 2Sz=0, D=64 U(1) workload, starting
from the seeded random MPS (centre 4), plus the FCI ground-state energy.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import qcinputs as q  # noqa: E402
from oracle.dmrgu1 import DMRGU1  # noqa: E402
from oracle.fci import FCI  # noqa: E402
from oracle.mpsu1 import MPSU1  # noqa: E402


def main():
    w = q.workload("u1_L10_N10_D64")
    L, N, D = w["L"], w["N"], w["D"]
    h, V = q.make_integrals(L, w["int_seed"])
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, w["mps_seed"], 4))
    E, err, _ = DMRGU1(h, V, N, 0).sweeps(m, D, nsweeps=6, tol=1e-12)
    e0, _ = FCI(h, V, N, 0).ground_state()
    out = {"workload": "u1_L10_N10_D64", "center": 4, "sweep_energies": E,
           "sweep_max_discarded_weight": err, "fci_energy": e0,
           "source": "oracle.dmrgu1.DMRGU1.sweeps (tol 1e-12) and oracle.fci.FCI"}
    with open(os.path.join(HERE, "u1_L10_sweeps.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
