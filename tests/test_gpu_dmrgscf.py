"""One DMRG-SCF macro-iteration through the C ABI.

Frozen-core active-space integrals (qcdmrg_active_space) go into an SU(2) context; sweeps
at the exact bond dimension give the active-space ground state; its gamma (qcdmrg_rdm1)
and Gamma (qcdmrg_rdm2) give the orbital gradient (qcdmrg_orbital_gradient), which equals
the one from the FCI density matrices of the same active space; a steepest-descent
rotation (qcdmrg_rotate_orbitals) and new active-space integrals, re-optimised by sweeps,
lower the energy.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


def _solve(qd, h, V, ncore, nact, nel, two_s, D):
    """Active-space ground state by SU(2) sweeps; returns (energy, gamma, Gamma)."""
    e_core, ha, Va = qd.active_space(h, V, ncore, nact)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(ha, Va, e_core)
    ctx.set_target(nel, two_s)
    ctx.init_mps(D, 7, 1)
    ctx.build_env()
    for _ in range(3):
        e = ctx.sweep(D, tol=1e-10)["energy"]
    ctx.move_center(nact - 2)
    g1 = ctx.rdm1(nact)
    g2 = ctx.rdm2(nact)
    ctx.close()
    return e, g1, g2


def test_dmrgscf_macro_iteration():
    import paper_2603_28648_b300 as qd
    from oracle import casscf
    from oracle.fci import FCI
    ensure_built()
    n, ncore, nact, nel, two_s, D = 7, 1, 5, 4, 0, 64
    h, V = q.make_integrals(n, 41)
    e0, g1, g2 = _solve(qd, h, V, ncore, nact, nel, two_s, D)
    # the active space at exact bond dimension: FCI energy and density matrices
    ec, ha, Va = casscf.active_space(h, V, ncore, nact)
    f = FCI(ha, Va, nel, two_s)
    e_fci, c = f.ground_state(two_s=two_s)
    assert abs(e0 - (e_fci + ec)) <= 1e-8
    f1, f2 = f.rdm12(c)
    G = qd.orbital_gradient(h, V, ncore, nact, g1, g2)
    Gf = qd.orbital_gradient(h, V, ncore, nact, f1, f2)
    assert np.abs(G - Gf).max() <= 1e-7 * max(1.0, np.abs(Gf).max())
    assert abs(casscf.energy(h, V, ncore, nact, g1, g2) - e0) <= 1e-8
    # one steepest-descent step, then the active space re-optimised
    _, h1, V1 = qd.rotate_orbitals(-2e-3 * G, h, V)
    e1, _, _ = _solve(qd, h1, V1, ncore, nact, nel, two_s, D)
    assert e1 < e0 - 0.5 * 2e-3 * 0.5 * np.sum(G * G)
