"""SU(2) sweeps through the C ABI against the operator-based SU(2) oracle.

qcdmrg_sweep moves the centre to the left end by exact steps and then optimises every
two-site centre left to right and back (2L-4 Davidson solves, SU(2) truncation of
multiplet weights, renormalization of the reduced operators and the 6j recoupling
of the two-site guess at each move), as the oracle's sweeps do. Six sweeps at a
truncated bond dimension match the oracle's energies after each sweep (1e-8); at the
exact bond dimension the energy is the spin-filtered FCI energy (1e-9); the mixed
precision Davidson policy (BF16, BF16x3, FP64 residual correction) reaches the FP64
solve's energy (1e-6, in practice far below).
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ctx(L, N, two_s, D, c, seed, int_seed):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))
    h, V = q.make_integrals(L, int_seed)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, c, *export_abi_su2(mps))
    ctx.build_env()
    return ctx, mps, h, V


@pytest.mark.parametrize("L,N,two_s,D,c", [(6, 6, 0, 8, 2), (6, 5, 1, 8, 2)])
def test_su2_six_sweeps_match_oracle(L, N, two_s, D, c):
    from oracle.dmrgsu2 import DMRGSU2
    ctx, mps, h, V = _ctx(L, N, two_s, D, c, 2, 13)
    E = [ctx.sweep(D, tol=1e-10)["energy"] for _ in range(6)]
    Eo, _, _ = DMRGSU2(h, V, N, two_s).sweeps(mps, D, nsweeps=6, tol=1e-12)
    assert np.abs(np.array(E) - np.array(Eo)).max() <= 1e-8
    ctx.close()


def test_su2_exact_sweeps_reach_spin_filtered_fci():
    from oracle.fci import FCI
    L, N, two_s, D = 6, 6, 2, 400
    ctx, mps, h, V = _ctx(L, N, two_s, D, 2, 3, 17)
    for _ in range(2):
        e = ctx.sweep(D, tol=1e-10)["energy"]
    e_fci, _ = FCI(h, V, N, two_s).ground_state(two_s=two_s)
    assert abs(e - e_fci) <= 1e-9
    ctx.close()


def test_su2_mixed_policy_energy_matches_fp64():
    ctx, mps, h, V = _ctx(8, 8, 0, 24, 3, 5, 12)
    psi0 = ctx.psi()
    e64, r64, _ = ctx.davidson(tol=1e-8)
    n64 = ctx.stats()["dav_hpsi"][0]
    ctx.set_psi(psi0)
    emx, rmx, _ = ctx.davidson(tol=1e-8, policy=1)
    nmix = ctx.stats()["dav_hpsi"]
    assert r64 <= 1e-8 and rmx <= 1e-8
    assert abs(emx - e64) <= 1e-6
    assert nmix[0] < n64                   # fewer FP64 products than the FP64 solve
    ctx.close()
