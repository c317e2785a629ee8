"""SU(2) density matrices and the energy gradient through the C ABI.

gamma (reduced B^0 and c at the right end) and Gamma (environment builds with unit
integrals on each permutation orbit of (pq|rs)) of an SU(2) two-site state against the
plain definition: the state expanded to determinants by the Clebsch-Gordan map of its
reduced elements, its density matrices by the FCI oracle's E_pq action (Gamma averaged
over the 8 permutations). qcdmrg_energy_grad returns the same matrices, the energy of the
state and dE/dpsi = 2 (H psi - E psi) / psi.psi; E = sum h gamma + 1/2 sum V Gamma.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]

AXES = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
        (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]


@pytest.mark.parametrize("L,N,two_s,D", [(5, 5, 1, 8), (6, 6, 0, 8)])
def test_su2_density_matrices_and_gradient(L, N, two_s, D):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2, export_abi_su2
    from oracle.fci import FCI
    from tests.test_oracle_dmrgsu2 import projector
    ensure_built()
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 7, L - 2))
    h, V = q.make_integrals(L, 21)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, L - 2, *export_abi_su2(mps))
    ctx.build_env()
    P, pairs, space = projector(mps)
    x = np.array([mps.psi[a, b] for a, b in pairs])
    v = P @ x
    g1, Gf = FCI(h, V, N, two_s).rdm12(v / np.linalg.norm(v))
    Gs = sum(Gf.transpose(a) for a in AXES) / 8.0
    E, dpsi, g, G = ctx.energy_grad(L, dpsi=True, gamma1=True, gamma2=True)
    assert np.abs(g - g1).max() <= 1e-10
    assert np.abs(G - Gs).max() <= 1e-10
    assert np.abs(ctx.rdm2(L) - Gs).max() <= 1e-10
    psi = mps.psi_to_flat()
    sig = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    nn = psi @ psi
    Eo = psi @ sig / nn
    assert abs(E - Eo) <= 1e-11 * abs(Eo)
    assert np.linalg.norm(dpsi - 2.0 * (sig - Eo * psi) / nn) <= 1e-10 * np.linalg.norm(sig)
    assert abs(np.sum(h * g) + 0.5 * np.sum(V * G) - E) <= 1e-10 * abs(E)
    ctx.close()
