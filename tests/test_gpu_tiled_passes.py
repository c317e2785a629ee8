"""The BF16 forms with the stage-1 intermediates split into passes.

QCDMRG_TILED_T_BYTES bounds the bytes of one plane of the T arena; the T_t are then
written and read pass by pass (a stage-1 and a stage-2 launch per pass, sigma blocks whose
segments fall in several passes adding with atomics). Sigma stays within the form's
rounding bound of the FP64 sigma, which equals the SU(2) oracle's, and the statistics show
the passes.
"""
import os

import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _products(budget, L, N, two_s, D, c):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    ensure_built()
    old = os.environ.get("QCDMRG_TILED_T_BYTES")
    os.environ["QCDMRG_TILED_T_BYTES"] = str(budget)
    try:
        mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
        h, V = q.make_integrals(L, 11)
        ctx = qd.Context(symmetry=qd.SU2)
        ctx.load_integrals(h, V)
        ctx.set_target(N, two_s)
        ctx.import_mps(L, c, *export_abi_su2(mps))
        ctx.build_env()
        psi = mps.psi_to_flat()
        out = {p: ctx.apply_heff(psi, p) for p in (qd.FP64, qd.BF16X3, qd.BF16)}
        st = ctx.stats()
        ctx.close()
    finally:
        if old is None:
            os.environ.pop("QCDMRG_TILED_T_BYTES", None)
        else:
            os.environ["QCDMRG_TILED_T_BYTES"] = old
    return out, st, mps, h, V


@pytest.mark.parametrize("budget", [4096, 1])
def test_tiled_passes_within_rounding_bounds(budget):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import DMRGSU2
    L, N, two_s, D, c = 8, 8, 0, 20, 3
    out, st, mps, h, V = _products(budget, L, N, two_s, D, c)
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    nrm = np.linalg.norm(ref)
    assert np.linalg.norm(out[qd.FP64] - ref) <= 1e-10 * nrm
    assert np.linalg.norm(out[qd.BF16X3] - out[qd.FP64]) <= 2.0 ** -14 * nrm
    assert np.linalg.norm(out[qd.BF16] - out[qd.FP64]) <= 8 * 2.0 ** -8 * nrm
    assert st["tile_passes"] > 1
    assert 0 < st["tile_t_bytes"]


def test_one_pass_without_a_budget():
    import paper_2603_28648_b300 as qd
    out, st, mps, h, V = _products(0, 8, 8, 0, 20, 3)
    assert st["tile_passes"] == 1
    assert np.linalg.norm(out[qd.BF16X3] - out[qd.FP64]) <= 2.0 ** -14 * np.linalg.norm(out[qd.FP64])


def test_passes_at_the_cas54_36_shape():
    """L=36, N=54, S=0, D=256 (SU(2), random MPS, centre bond): the BF16x3 product with the
    T arena split into about eight passes stays within the form's bound of the FP64 product
    and of the one-pass product."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    h, V = q.make_integrals(36, q.integrals.BASE_SEED + 2)
    out = {}
    for budget in (0, None):
        old = os.environ.get("QCDMRG_TILED_T_BYTES")
        if budget is None:
            # an eighth of the one-pass arena
            os.environ["QCDMRG_TILED_T_BYTES"] = str(max(1, out[0][2] // 8))
        try:
            ctx = qd.Context(symmetry=qd.SU2, pair_switch=19)
            ctx.load_integrals(h, V)
            ctx.set_target(54, 0)
            ctx.init_mps(256, q.integrals.BASE_SEED + 1002, 17)
            ctx.build_env()
            psi = ctx.psi()
            s64 = ctx.apply_heff(psi, qd.FP64)
            s3 = ctx.apply_heff(psi, qd.BF16X3)
            st = ctx.stats()
            out[budget] = (s64, s3, st["tile_t_bytes"], st["tile_passes"])
            ctx.close()
        finally:
            if old is None:
                os.environ.pop("QCDMRG_TILED_T_BYTES", None)
            else:
                os.environ["QCDMRG_TILED_T_BYTES"] = old
    s64, s3a, _, p1 = out[0]
    _, s3b, _, p8 = out[None]
    nrm = np.linalg.norm(s64)
    assert p1 == 1 and p8 >= 6
    assert np.linalg.norm(s3b - s64) <= 2.0 ** -14 * nrm
    assert np.linalg.norm(s3b - s3a) <= 2.0 ** -14 * nrm
