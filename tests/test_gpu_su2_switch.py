"""SU(2) with the normal/complementary switch (the N/2 rule) through the C ABI.

Left blocks past the switch cut keep P^k, Q^k of the orbitals to their right and right
blocks beyond it A^k, B^k of their own orbitals. The FP64 sigma equals the SU(2) oracle's
(which keeps normal operators on both sides, so it does not depend on the switch) at
switch cuts before, at and after the centre; sweeps across the switch cut match the
oracle's energies; at the CAS(54,36) shape the switched environment gives the unswitched
sigma with a smaller device footprint.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ctx(L, N, two_s, D, c, seed, int_seed, switch):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))
    h, V = q.make_integrals(L, int_seed)
    ctx = qd.Context(symmetry=qd.SU2, pair_switch=switch)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, c, *export_abi_su2(mps))
    ctx.build_env()
    return ctx, mps, h, V


@pytest.mark.parametrize("L,N,two_s,D,c,switch", [(8, 8, 0, 20, 3, 1), (8, 8, 0, 20, 3, 4), (8, 8, 0, 20, 3, 5),
                                                  (7, 6, 2, 8, 2, 1), (6, 5, 1, 6, 4, 2)])
def test_su2_switched_sigma_matches_oracle(L, N, two_s, D, c, switch):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import DMRGSU2
    ctx, mps, h, V = _ctx(L, N, two_s, D, c, 5, 11, switch)
    psi = mps.psi_to_flat()
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    s64 = ctx.apply_heff(psi, qd.FP64)
    assert np.linalg.norm(s64 - ref) <= 1e-10 * np.linalg.norm(ref)
    s3 = ctx.apply_heff(psi, qd.BF16X3)
    assert np.linalg.norm(s3 - s64) <= 2.0 ** -14 * np.linalg.norm(s64)
    ctx.close()


def test_su2_switched_sweeps_match_oracle():
    from oracle.dmrgsu2 import DMRGSU2
    L, N, two_s, D, c = 6, 6, 0, 8, 2
    ctx, mps, h, V = _ctx(L, N, two_s, D, c, 2, 13, 3)
    E = [ctx.sweep(D, tol=1e-10)["energy"] for _ in range(3)]
    Eo, _, _ = DMRGSU2(h, V, N, two_s).sweeps(mps, D, nsweeps=3, tol=1e-12)
    assert np.abs(np.array(E) - np.array(Eo)).max() <= 1e-8
    ctx.close()


def test_su2_switch_at_the_cas54_36_shape():
    """L=36, N=54, S=0, D=256, centre (17, 18): the switch one cut past the centre (the
    bench's setting) reproduces the unswitched FP64 sigma and holds fewer device bytes."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    h, V = q.make_integrals(36, q.integrals.BASE_SEED + 2)
    out = {}
    for switch in (0, 19):
        ctx = qd.Context(symmetry=qd.SU2, pair_switch=switch)
        ctx.load_integrals(h, V)
        ctx.set_target(54, 0)
        ctx.init_mps(256, q.integrals.BASE_SEED + 1002, 17)
        ctx.build_env()
        psi = ctx.psi()
        out[switch] = (ctx.apply_heff(psi, qd.FP64), ctx.stats()["live_bytes"])
        ctx.close()
    s0, b0 = out[0]
    s1, b1 = out[19]
    assert np.linalg.norm(s1 - s0) <= 1e-12 * np.linalg.norm(s0)
    assert b1 < b0
