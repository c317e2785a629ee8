"""DMRG-SCF orbital step through the C ABI (host code, no device) against the plain
definitions of oracle/casscf.py.

Density matrices come from the FCI oracle for the active space of a random synthetic
orbital set (core, active and virtual orbitals), so gamma and Gamma are those of a real
spin-adapted state. Checked: the frozen-core active-space integrals; the rotated integrals
and exp(kappa) against scipy's expm and an einsum of the definition; the orbital gradient
against central differences of the energy of rotated orbitals at fixed density matrices
for every pair type (core-active, core-virtual, active-active, active-virtual); and a
steepest-descent step lowering that energy.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built


def _setup(n=7, ncore=2, nact=4, nel=4, two_s=0, seed=31):
    from oracle.fci import FCI
    from oracle import casscf
    h, V = q.make_integrals(n, seed)
    e_core, h_act, V_act = casscf.active_space(h, V, ncore, nact)
    f = FCI(h_act, V_act, nel, two_s)
    _, c = f.ground_state(two_s=two_s)
    g1, g2 = f.rdm12(c)
    return h, V, ncore, nact, g1, g2


def test_active_space_matches_the_definition():
    import paper_2603_28648_b300 as qd
    from oracle import casscf
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(7, 31)
    e, ha, Va = qd.active_space(h, V, 2, 4, lib=lib)
    e0, ha0, Va0 = casscf.active_space(h, V, 2, 4)
    assert abs(e - e0) < 1e-12 * max(1.0, abs(e0))
    assert np.abs(ha - ha0).max() < 1e-12 and np.abs(Va - Va0).max() < 1e-14


def test_rotation_matches_expm_and_the_definition():
    import paper_2603_28648_b300 as qd
    from scipy.linalg import expm
    from oracle import casscf
    lib = qd.load(ensure_built())
    n = 6
    h, V = q.make_integrals(n, 32)
    rng = np.random.default_rng(5)
    k = rng.normal(0, 0.7, (n, n))
    k = k - k.T
    U, h2, V2 = qd.rotate_orbitals(k, h, V, lib=lib)
    assert np.abs(U - expm(k)).max() < 1e-13
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-13
    h0, V0 = casscf.rotate(h, V, expm(k))
    assert np.abs(h2 - h0).max() < 1e-12 and np.abs(V2 - V0).max() < 1e-12
    with pytest.raises(qd.QcdmrgError):
        qd.rotate_orbitals(k + np.eye(n) * 1e-3, h, V, lib=lib)   # not antisymmetric


@pytest.mark.parametrize("ncore,nact,nel,two_s", [(2, 4, 4, 0), (1, 4, 3, 1), (0, 5, 4, 2)])
def test_orbital_gradient_equals_finite_differences(ncore, nact, nel, two_s):
    import paper_2603_28648_b300 as qd
    from oracle import casscf
    lib = qd.load(ensure_built())
    h, V, ncore, nact, g1, g2 = _setup(7, ncore, nact, nel, two_s)
    G = qd.orbital_gradient(h, V, ncore, nact, g1, g2, lib=lib)
    Gfd = casscf.gradient_fd(h, V, ncore, nact, g1, g2)
    assert np.abs(G + G.T).max() < 1e-12
    assert np.abs(G - Gfd).max() < 1e-7 * max(1.0, np.abs(Gfd).max())
    # every kind of pair carries a gradient here (a plausible index slip zeroes or
    # misplaces one of these blocks)
    a = slice(ncore, ncore + nact)
    v = slice(ncore + nact, 7)
    assert np.abs(G[v, a]).max() > 1e-3
    if ncore:
        assert np.abs(G[a, :ncore]).max() > 1e-3 and np.abs(G[v, :ncore]).max() > 1e-3


def test_steepest_descent_step_lowers_the_energy():
    import paper_2603_28648_b300 as qd
    from oracle import casscf
    lib = qd.load(ensure_built())
    h, V, ncore, nact, g1, g2 = _setup()
    e0 = casscf.energy(h, V, ncore, nact, g1, g2)
    G = qd.orbital_gradient(h, V, ncore, nact, g1, g2, lib=lib)
    step = 1e-3
    _, h2, V2 = qd.rotate_orbitals(-step * G, h, V, lib=lib)
    e1 = casscf.energy(h2, V2, ncore, nact, g1, g2)
    # first order: dE = -step * sum_{p>q} G_pq^2
    pred = -step * 0.5 * np.sum(G * G)
    assert e1 < e0
    assert abs((e1 - e0) - pred) <= 0.05 * abs(pred)


def test_invalid_orbital_spaces_are_rejected():
    """EINVAL for orbital spaces that do not fit (core + active > n, no active orbital,
    negative core) and for NULL arrays, before any work."""
    import ctypes
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(5, 3)
    for ncore, nact in ((3, 3), (0, 0), (-1, 2)):
        with pytest.raises(qd.QcdmrgError):
            qd.active_space(h, V, ncore, nact, lib=lib)
        with pytest.raises(qd.QcdmrgError):
            qd.orbital_gradient(h, V, ncore, nact, np.zeros((2, 2)), np.zeros((2,) * 4), lib=lib)
    dp = ctypes.POINTER(ctypes.c_double)
    null = ctypes.cast(None, dp)
    assert lib.qcdmrg_rotate_orbitals(5, null, null, null, null, null, null) == -1
    assert lib.qcdmrg_active_space(5, 1, 2, null, null, null, null, null) == -1
