"""qcdmrg_psi_layout against the oracle's block order of the two-site wavefunction, and
qcdmrg_energy_grad against the separate calls it bundles (apply_heff, rdm1, rdm2)."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def test_psi_layout_and_energy_grad():
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    L, N, D, c = 5, 5, 8, 1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 1)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    lay = ctx.psi_layout()
    bX, bY = m.lbonds[c], m.rbonds[c + 2]
    ref = [(qX[0], qX[1], i, j, qY[0], qY[1], bX.sectors[qX][1], bY.sectors[qY][1])
           for qX, i, j, qY in m.psi_keys()]
    assert [tuple(int(x) for x in r) for r in lay] == ref
    assert int(np.sum(lay[:, 6] * lay[:, 7])) == ctx.psi_size()
    ctx.move_center(L - 2)
    psi = ctx.psi()
    sig = ctx.apply_heff(psi)
    E, dpsi, g1, g2 = ctx.energy_grad(L, dpsi=True, gamma1=True, gamma2=True)
    nn = psi @ psi
    assert abs(E - psi @ sig / nn) <= 1e-13 * abs(E)
    assert np.abs(dpsi - 2.0 * (sig - E * psi) / nn).max() <= 1e-12 * np.abs(sig).max()
    assert np.abs(g1 - ctx.rdm1(L)).max() <= 1e-13
    assert np.abs(g2 - ctx.rdm2(L)).max() <= 1e-13
    assert abs(np.sum(h * g1) + 0.5 * np.sum(V * g2) - E) <= 1e-10 * abs(E)
    ctx.close()
