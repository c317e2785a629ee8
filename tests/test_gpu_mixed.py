"""tcgen05 forms of H_eff psi (TF32, BF16, BF16x3) against the FP64 form.

Bounds: the relative Frobenius error of a product of two rounded operands is a
few units of roundoff u of the input format, independent of K for random
signs; sigma goes through two such contractions. u(BF16) = 2^-9,
u(TF32) = 2^-11, and the three-term BF16 split reproduces FP32 inputs to
about 2^-24 relative. Bounds below are 8u (BF16, TF32) and 2^-14 (BF16x3)."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

BOUND = {"tf32": 8 * 2.0 ** -11, "bf16": 8 * 2.0 ** -9, "bf16x3": 2.0 ** -14}


def _ctx(L, N, D, c, seed):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, N % 2, D, q.SYM_U1, seed, c))
    h, V = q.make_integrals(L, seed + 1)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, N % 2)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    return ctx, m


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("L,N,D,c", [(4, 4, 16, 1), (6, 6, 16, 2), (8, 8, 32, 3), (10, 10, 64, 4)])
def test_tensor_core_forms_vs_fp64(prec, L, N, D, c):
    import paper_2603_28648_b300 as qd
    ctx, m = _ctx(L, N, D, c, 30 + L)
    psi = m.psi_to_flat()
    ref = ctx.apply_heff(psi, qd.FP64)
    out = ctx.apply_heff(psi, qd.PRECISIONS[prec])
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err <= BOUND[prec], err


def test_bf16_forms_two_row_panels_L14():
    """psi blocks of more than 128 rows (two A panels) in the bulk-copy-fed
    BF16 path; stage-2 items split over segment ranges."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 14, 14, 1024
    h, V = q.make_integrals(L, 77)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 7, 6)
    ctx.build_env()
    psi = ctx.psi()
    ref = ctx.apply_heff(psi, qd.FP64)
    for prec in ["bf16", "bf16x3"]:
        out = ctx.apply_heff(psi, qd.PRECISIONS[prec])
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= BOUND[prec], (prec, err)
        again = ctx.apply_heff(psi, qd.PRECISIONS[prec])
        assert np.linalg.norm(again - out) <= 1e-6 * np.linalg.norm(ref)   # only atomics order differs


def test_tensor_core_large_blocks_L36():
    """Blocks larger than one 128x128 tile and K spanning several chunks."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 36, 54, 512
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 5, 17)
    ctx.build_env()
    psi = ctx.psi()
    ref = ctx.apply_heff(psi, qd.FP64)
    for prec in ["tf32", "bf16", "bf16x3"]:
        out = ctx.apply_heff(psi, qd.PRECISIONS[prec])
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= BOUND[prec], (prec, err)


def test_autotuner_picks_a_shape_and_keeps_results():
    """The autotuner times the candidate work-item shapes on the first BF16
    product; its choice changes the schedule, not the result."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 12, 12, 256
    h, V = q.make_integrals(L, 5)
    out = {}
    for tune in (False, True):
        ctx = qd.Context(autotune=tune)
        ctx.load_integrals(h, V)
        ctx.set_target(N, 0)
        ctx.init_mps(D, 9, 5)
        ctx.build_env()
        psi = ctx.psi()
        out[tune] = ctx.apply_heff(psi, qd.BF16)
        st = ctx.stats()
        assert st["tile_kmax"] > 0 and st["tile_width"] in (128, 256)
        if tune:
            assert st["tune_seconds"] >= 0.0
    # shapes differ in how the FP32 partial sums are grouped (split items add
    # in FP64): a difference far below the BF16 form's own error (~2e-3)
    assert np.linalg.norm(out[True] - out[False]) <= 1e-4 * np.linalg.norm(out[False])
