"""Two-orbital density matrices by a walk of the centre (qcdmrg_orbital_rdm) through the C
ABI on the GPU: every rho_ij element against the partial trace of the expanded state (U(1),
and for an SU(2) state the average over its multiplet's components), the state restored
afterwards, and at L = 12 the identities of density matrices of one state (unit trace,
symmetry, positivity, the one-orbital matrices of different pairs agreeing) with the
mutual-information order a permutation."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ref(dets, v, L):
    from oracle import orbital_qi as qi
    R = np.zeros((L, L, 16, 16))
    for i in range(L):
        for j in range(i + 1, L):
            R[i, j] = qi.two_orbital_rdm(dets, v, i, j)
    return R


def test_orbital_rdm_u1_matches_the_partial_trace():
    import paper_2603_28648_b300 as qd
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1, Projector, export_abi
    ensure_built()
    L, N, D, c = 6, 5, 16, 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, D, q.SYM_U1, 6, c))
    h, V = q.make_integrals(L, 7)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 1)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    psi0 = m.psi_to_flat()
    s0 = ctx.apply_heff(psi0)
    R = ctx.orbital_rdm(L)
    f = FCI(h, V, N, 1)
    v = Projector(m, f.space).apply(m.psi)
    assert np.abs(R - _ref(f.space.dets, v, L)).max() <= 1e-10
    assert np.array_equal(ctx.psi(), psi0)
    assert np.linalg.norm(ctx.apply_heff(psi0) - s0) <= 1e-12 * np.linalg.norm(s0)
    ctx.close()


@pytest.mark.parametrize("L,N,two_s,D,c", [(5, 5, 1, 8, 1), (6, 6, 0, 8, 2)])
def test_orbital_rdm_su2_matches_the_partial_trace(L, N, two_s, D, c):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2, export_abi_su2
    from tests.test_oracle_dmrgsu2 import projector
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, c, *export_abi_su2(mps))
    ctx.build_env()
    psi = mps.psi_to_flat()
    s0 = ctx.apply_heff(psi, qd.FP64)
    R = ctx.orbital_rdm(L)
    from oracle import orbital_qi as qi
    P, pairs, space = projector(mps)
    v = P @ np.array([mps.psi[a, b] for a, b in pairs])
    for i in range(L):
        for j in range(i + 1, L):
            assert np.abs(R[i, j] - qi.multiplet_rdm(L, N, two_s, v, i, j)).max() <= 1e-10
    s1 = ctx.apply_heff(psi, qd.FP64)
    assert np.linalg.norm(s1 - s0) <= 1e-12 * np.linalg.norm(s0)
    ctx.close()


def test_orbital_rdm_identities_at_L12():
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 12, 12, 32
    h, V = q.make_integrals(L, 21)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 3, 5)
    ctx.build_env()
    R = ctx.orbital_rdm(L)
    ctx.close()
    one = {}
    for i in range(L):
        for j in range(i + 1, L):
            r = R[i, j]
            assert abs(np.trace(r) - 1) <= 1e-10
            assert np.abs(r - r.T).max() <= 1e-12
            assert np.linalg.eigvalsh(r).min() >= -1e-10
            t = r.reshape(4, 4, 4, 4)
            one.setdefault(i, []).append(np.einsum("xyzy->xz", t))
            one.setdefault(j, []).append(np.einsum("xyxz->yz", t))
    for i, mats in one.items():
        assert max(np.abs(m - mats[0]).max() for m in mats) <= 1e-10
    s1, I = qd.orbital_entanglement(R)
    assert (I >= -1e-10).all() and I.max() > 0
    order, _ = qd.fiedler_order(I)
    assert sorted(order) == list(range(L))
