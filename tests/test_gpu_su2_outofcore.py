"""Out-of-core operator store with SU(2) reduced operators.

The store moves renormalized blocks between the device and pinned host memory without
looking at what they hold, so SU(2) blocks (reduced elements between multiplets) take the
same path as U(1) ones. Sweeps under a budget of one byte (every block the centre and the
next move do not use leaves the device) and of a tenth of the resident footprint give the
energies of the all-resident context (1e-10), and at L=6 the SU(2) oracle's sweep
energies (1e-8).
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ctx(L, N, two_s, D, c, seed, int_seed, hbm_budget_gb):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))
    h, V = q.make_integrals(L, int_seed)
    ctx = qd.Context(symmetry=qd.SU2, hbm_budget_gb=hbm_budget_gb)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, c, *export_abi_su2(mps))
    ctx.build_env()
    return ctx, mps, h, V


@pytest.mark.parametrize("fraction", [0.0, 0.1])
def test_su2_budgeted_sweeps_match_resident(fraction):
    """fraction: budget as a fraction of the resident context's device bytes (which also
    count the enlarged centre blocks and the operand mirrors, not only renormalized
    blocks); 0 is a budget of one byte."""
    L, N, two_s, D, c = 8, 7, 1, 12, 3
    ref, _, _, _ = _ctx(L, N, two_s, D, c, 4, 14, 0.0)
    budget_gb = max(1e-9, fraction * ref.stats()["live_bytes"] / 1e9)
    ctx, _, _, _ = _ctx(L, N, two_s, D, c, 4, 14, budget_gb)
    for _ in range(3):
        e_ref = ref.sweep(D, tol=1e-10)["energy"]
        e = ctx.sweep(D, tol=1e-10)["energy"]
        assert abs(e - e_ref) <= 1e-10
    st = ctx.stats()
    assert st["evictions"] > 0 and st["d2h_bytes"] > 0
    assert st["restores"] > 0 and st["h2d_bytes"] > 0
    assert st["d2h_bytes"] >= st["h2d_bytes"]
    assert ref.stats()["evictions"] == 0
    if fraction == 0.0:
        assert st["live_bytes"] < ref.stats()["live_bytes"]
    ref.close()
    ctx.close()


def test_su2_budgeted_sweeps_match_oracle():
    from oracle.dmrgsu2 import DMRGSU2
    L, N, two_s, D, c = 6, 6, 0, 8, 2
    ctx, mps, h, V = _ctx(L, N, two_s, D, c, 2, 13, 1e-9)
    E = [ctx.sweep(D, tol=1e-10)["energy"] for _ in range(3)]
    Eo, _, _ = DMRGSU2(h, V, N, two_s).sweeps(mps, D, nsweeps=3, tol=1e-12)
    assert np.abs(np.array(E) - np.array(Eo)).max() <= 1e-8
    assert ctx.stats()["h2d_bytes"] > 0
    ctx.close()
