"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the DMRG method itself: it only draws the
random numbers (integrals, raw MPS block entries) and fixes the shapes of the
workloads, so that both sides of every parity test start from identical data.

Integral recipe (chemist notation V_pqrs = (pq|rs), 8-fold symmetric, PSD):
  1. off-diagonal h_pq, p<q, row-major upper triangle: N(0, 0.1), mirrored;
  2. diagonal h_pp = linspace(-2, 0.5, L) (or the open-shell profile);
  3. for k = 0 .. 2L-1: B^k upper triangle incl. diagonal, row-major, N(0,1),
     mirrored, scaled by 0.5**(k/4);
  4. V_pqrs = sum_k B^k_pq B^k_rs.
"""

from .integrals import make_integrals, open_shell_diagonal, write_integrals, read_integrals
from .mps import (batched_instances, site_qns, fuse, mps_structure, random_mps_blocks, SYM_U1, SYM_SU2,
                  workload)

__all__ = [
    "make_integrals", "open_shell_diagonal", "write_integrals", "read_integrals",
    "site_qns", "fuse", "mps_structure", "random_mps_blocks", "SYM_U1", "SYM_SU2",
    "workload",
]
