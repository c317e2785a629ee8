"""Dynamic block-state selection through the C ABI.

With trunc_eps > 0 each truncation of qcdmrg_sweep keeps the smallest bond dimension in
[D_min, D] whose discarded weight is at most trunc_eps. Two SU(2) sweeps match the SU(2)
oracle's sweeps with the same rule (energies 1e-8, the largest number of multiplets
kept), and qcdmrg_truncate_dbss reports the states it kept.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ctx(L, N, two_s, D, c):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 2, c))
    h, V = q.make_integrals(L, 13)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, c, *export_abi_su2(mps))
    ctx.build_env()
    return ctx, mps, h, V


@pytest.mark.parametrize("L,N,two_s,D,c,eps,dmin", [(6, 5, 1, 12, 2, 1e-3, 3), (6, 6, 0, 12, 2, 1e-2, 2)])
def test_dynamic_selection_sweeps_match_oracle(L, N, two_s, D, c, eps, dmin):
    from oracle.dmrgsu2 import DMRGSU2
    ctx, mps, h, V = _ctx(L, N, two_s, D, c)
    reps = [ctx.sweep(D, tol=1e-10, trunc_eps=eps, D_min=dmin) for _ in range(2)]
    orc = DMRGSU2(h, V, N, two_s)
    Eo, _, _ = orc.sweeps(mps, D, nsweeps=2, tol=1e-12, trunc_eps=eps, D_min=dmin)
    assert np.abs(np.array([r["energy"] for r in reps]) - np.array(Eo)).max() <= 1e-8
    assert max(r["max_D"] for r in reps) == orc.max_kept
    ctx.close()


def test_truncate_dbss_keeps_fewer_states_for_a_larger_error():
    L, N, two_s, D, c = 6, 6, 0, 12, 2
    kept = []
    for eps in (1e-8, 1e-1):
        ctx, _, _, _ = _ctx(L, N, two_s, D, c)
        ctx.davidson(tol=1e-8)
        err, k = ctx.truncate_dbss(1, D, eps, +1)
        assert 1 <= k <= D
        assert err <= eps or k == D
        kept.append(k)
        ctx.close()
    assert kept[1] < kept[0]
