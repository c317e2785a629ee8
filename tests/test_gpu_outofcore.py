"""Out-of-core operator store: sweeps with renormalized blocks moved to pinned
host memory give the energies of the all-resident run."""
import json
import os

import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "u1_L10_sweeps.json")


def _ctx(hbm_budget_gb):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    g = json.load(open(GOLDEN))
    w = q.workload("u1_L10_N10_D64")
    m = MPSU1.from_raw(q.random_mps_blocks(w["L"], w["N"], w["N"] % 2, w["D"], q.SYM_U1,
                                           w["mps_seed"], g["center"]))
    h, V = q.make_integrals(w["L"], w["int_seed"])
    ctx = qd.Context(hbm_budget_gb=hbm_budget_gb)
    ctx.load_integrals(h, V)
    ctx.set_target(w["N"], w["N"] % 2)
    ctx.import_mps(w["L"], g["center"], *export_abi(m))
    ctx.build_env()
    return ctx, w, g


@pytest.mark.parametrize("fraction", [0.0, 0.5])
def test_budgeted_sweeps_match_resident(fraction):
    """Budget of one byte (everything evictable leaves the device) and of half
    the all-resident footprint."""
    ref, w, g = _ctx(0.0)
    budget_gb = max(1e-9, fraction * ref.stats()["live_bytes"] / 1e9)
    ctx, _, _ = _ctx(budget_gb)
    s0 = ctx.stats()
    assert s0["evictions"] > 0 and s0["d2h_bytes"] > 0
    for s in range(3):
        e_ref = ref.sweep(w["D"], tol=1e-10)["energy"]
        e = ctx.sweep(w["D"], tol=1e-10)["energy"]
        assert abs(e - e_ref) <= 1e-10
        assert abs(e - g["sweep_energies"][s]) <= 1e-8
    st = ctx.stats()
    assert st["restores"] > 0 and st["h2d_bytes"] > 0
    assert st["d2h_bytes"] >= st["h2d_bytes"]
    assert st["copy_wait_seconds"] >= 0.0
    assert ref.stats()["evictions"] == 0 and ref.stats()["h2d_bytes"] == 0


def test_budget_bounds_resident_blocks():
    """With a budget of one byte, only the blocks the centre and the next move
    use stay on the device: the device footprint of the budgeted context stays
    below the resident one after a sweep."""
    ref, w, g = _ctx(0.0)
    ctx, _, _ = _ctx(1e-9)
    ref.sweep(w["D"], tol=1e-8)
    ctx.sweep(w["D"], tol=1e-8)
    assert ctx.stats()["live_bytes"] < ref.stats()["live_bytes"]
