"""GPU parity with the normal/complementary switch (config pair_switch), through the C ABI.

Left blocks at cuts <= pair_switch and right blocks beyond it hold the normal pair
operators; the cases put the switch left of, at and right of the centre cut, so the
switching enlargement runs in either chain or at the centre and the centre uses either
decomposition. Bounds as in the unswitched tests: FP64 1e-10 relative against the oracle,
the tensor-core forms 8u (BF16, TF32) and 2^-14 (BF16x3) against the FP64 form, sweep
energies 1e-8 against the oracle's."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
BOUND = {"tf32": 8 * 2.0 ** -11, "bf16": 8 * 2.0 ** -9, "bf16x3": 2.0 ** -14}


def _ctx(m, h, V, N, two, switch):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import export_abi
    ensure_built()
    ctx = qd.Context(pair_switch=switch)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two)
    ctx.import_mps(m.L, m.center, *export_abi(m))
    ctx.build_env()
    return ctx


@pytest.mark.parametrize("L,N,D,c,switch", [(6, 6, 16, 2, 1), (6, 6, 16, 2, 2), (6, 6, 16, 2, 3),
                                            (7, 5, 24, 0, 3), (7, 5, 24, 5, 3), (8, 8, 32, 3, 2),
                                            (8, 8, 32, 3, 4), (8, 8, 32, 3, 6)])
def test_switched_sigma_matches_oracle(L, N, D, c, switch):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, 40 + L, c))
    h, V = q.make_integrals(L, 41 + L)
    ctx = _ctx(m, h, V, N, two, switch)
    psi = m.psi_to_flat()
    ref = m.psi_to_flat(DMRGU1(h, V, N, two).sigma(m))
    sig = ctx.apply_heff(psi)
    assert np.linalg.norm(sig - ref) <= TOL_FP64 * np.linalg.norm(ref)
    for prec in ("tf32", "bf16", "bf16x3"):
        out = ctx.apply_heff(psi, qd.PRECISIONS[prec])
        assert np.linalg.norm(out - sig) <= BOUND[prec] * np.linalg.norm(sig), prec


def test_switched_sweeps_match_oracle():
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    L, N, D, c = 7, 5, 12, 3
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, D, q.SYM_U1, 5, c))
    h, V = q.make_integrals(L, 6)
    ctx = _ctx(m, h, V, N, 1, 3)
    E = [ctx.sweep(D, tol=1e-10)["energy"] for _ in range(2)]
    Eo, _, _ = DMRGU1(h, V, N, 1).sweeps(m, D, 2, tol=1e-12)
    assert np.abs(np.array(E) - np.array(Eo)).max() <= 1e-8


def test_switched_rdm1_equals_unswitched():
    """The one-particle density matrix needs normal pairs on the left at the last centre:
    with the switch on, the library rebuilds that environment unswitched and restores it."""
    from oracle.mpsu1 import MPSU1
    L, N, D = 6, 6, 16
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 9, L - 2))
    h, V = q.make_integrals(L, 10)
    g0 = _ctx(m, h, V, N, 0, 0).rdm1(L)
    ctx = _ctx(m, h, V, N, 0, 3)
    g1 = ctx.rdm1(L)
    assert np.abs(g1 - g0).max() <= 1e-12
    psi = m.psi_to_flat()
    from oracle.dmrgu1 import DMRGU1
    ref = m.psi_to_flat(DMRGU1(h, V, N, 0).sigma(m))
    assert np.linalg.norm(ctx.apply_heff(psi) - ref) <= TOL_FP64 * np.linalg.norm(ref)


@pytest.mark.parametrize("switch,sum_gemm", [(0, 1), (3, -1)])
def test_operator_sum_forms_match_oracle(switch, sum_gemm):
    """Operator sums as GEMMs without the switch, block by block with it."""
    import paper_2603_28648_b300 as qd
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    L, N, D, c = 8, 8, 32, 3
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 7, c))
    h, V = q.make_integrals(L, 8)
    ctx = qd.Context(pair_switch=switch, sum_gemm=sum_gemm)
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    ref = m.psi_to_flat(DMRGU1(h, V, N, 0).sigma(m))
    assert np.linalg.norm(ctx.apply_heff(m.psi_to_flat()) - ref) <= TOL_FP64 * np.linalg.norm(ref)


def test_switch_leaves_sigma_unchanged_L36():
    """CAS(54,36)-shaped problem at D=512: the switch at the centre cut and two cuts left of it
    gives the unswitched FP64 sigma (to summation order), and its BF16 forms stay within their
    bounds of it."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 36, 54, 512
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    out = {}
    for switch in (0, 18, 16):
        ctx = qd.Context(pair_switch=switch)
        ctx.load_integrals(h, V)
        ctx.set_target(N, 0)
        ctx.init_mps(D, 5, 17)
        ctx.build_env()
        psi = ctx.psi()
        out[switch] = ctx.apply_heff(psi, qd.FP64)
        if switch:
            ref = out[0]
            assert np.linalg.norm(out[switch] - ref) <= 1e-12 * np.linalg.norm(ref)
            for prec in ("bf16", "bf16x3"):
                x = ctx.apply_heff(psi, qd.PRECISIONS[prec])
                assert np.linalg.norm(x - ref) <= BOUND[prec] * np.linalg.norm(ref), prec
        ctx.close()

