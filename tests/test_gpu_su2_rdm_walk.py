"""SU(2) two-particle density matrix by the walk of the centre, through the C ABI.

qcdmrg_rdm2_sweep on an SU(2) context walks the state's M = S expansion with the U(1)
centre walk. At L = 5, 6 the result equals the FCI 2-RDM of the determinant-expanded
state element by element; at L = 12 (beyond the environment probes) the traces, the
symmetries of a real state and E = sum h gamma + 1/2 sum V Gamma hold; the SU(2) context
still gives the same sigma afterwards.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _ctx(mps, h, V):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import export_abi_su2
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(mps.N, mps.two_s)
    ctx.import_mps(mps.L, mps.center, *export_abi_su2(mps))
    ctx.build_env()
    return ctx


@pytest.mark.parametrize("L,N,two_s,D,c", [(5, 5, 1, 8, 1), (6, 6, 0, 8, 2)])
def test_su2_walk_equals_fci_rdm(L, N, two_s, D, c):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2
    from oracle.fci import FCI
    from tests.test_oracle_dmrgsu2 import projector
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    ctx = _ctx(mps, h, V)
    psi = mps.psi_to_flat()
    s0 = ctx.apply_heff(psi, qd.FP64)
    G = ctx.rdm2_sweep(L)
    P, pairs, space = projector(mps)
    v = P @ np.array([mps.psi[a, b] for a, b in pairs])
    _, Gf = FCI(h, V, N, two_s).rdm12(v / np.linalg.norm(v))
    assert np.abs(G - Gf).max() <= 1e-10
    s1 = ctx.apply_heff(psi, qd.FP64)
    assert np.linalg.norm(s1 - s0) <= 1e-12 * np.linalg.norm(s0)
    ctx.close()


def test_su2_walk_identities_at_L12():
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import MPSSU2
    ensure_built()
    L, N, two_s, D = 12, 12, 0, 16
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 3, L - 2))
    h, V = q.make_integrals(L, 17)
    ctx = _ctx(mps, h, V)
    E, _, g1, _ = ctx.energy_grad(L, dpsi=False, gamma1=True, gamma2=False)
    G = ctx.rdm2_sweep(L)
    assert abs(np.einsum("pprr->", G) - N * (N - 1)) <= 1e-9
    assert np.abs(G - G.transpose(2, 3, 0, 1)).max() <= 1e-10
    assert np.abs(G - G.transpose(1, 0, 3, 2)).max() <= 1e-10
    assert abs(np.sum(h * g1) + 0.5 * np.sum(V * G) - E) <= 1e-9 * abs(E)
    ctx.close()
