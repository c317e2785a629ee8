"""Pins of the operator-based U(1) DMRG oracle against the projection definition."""
import numpy as np
import pytest

import qcinputs as q
from oracle.fci import FCI
from oracle.mpsu1 import MPSU1, Projector
from oracle.dmrgu1 import DMRGU1


@pytest.mark.parametrize("L,N,D,c", [(4, 4, 16, 1), (5, 5, 16, 1), (6, 6, 16, 2), (6, 4, 12, 3)])
def test_sigma_equals_projection(L, N, D, c):
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, 5 + L, c))
    h, V = q.make_integrals(L, 7 + L)
    f = FCI(h, V, N, two)
    P = Projector(m, f.space)
    s_op = DMRGU1(h, V, N, two).sigma(m)
    s_pr = P.heff(f, m.psi)
    assert np.linalg.norm(s_op - s_pr) <= 1e-12 * np.linalg.norm(s_pr)


def test_projector_isometry_and_heff_hermitian():
    L, N = 6, 6
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, 16, q.SYM_U1, 1, 2))
    h, V = q.make_integrals(L, 2)
    f = FCI(h, V, N, 0)
    P = Projector(m, f.space)
    rng = np.random.default_rng(0)
    mask = m.psi_from_flat(np.ones(m.psi_to_flat().size)) != 0
    x = rng.normal(size=m.psi.shape) * mask
    y = rng.normal(size=m.psi.shape) * mask
    assert abs(np.linalg.norm(P.apply(x)) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    d = DMRGU1(h, V, N, 0)
    a = np.vdot(y, d.sigma(m, x))
    b = np.vdot(d.sigma(m, y), x)
    assert abs(a - b) < 1e-10 * abs(a)


def test_sigma_conserves_quantum_numbers():
    L, N = 6, 5
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, 16, q.SYM_U1, 4, 2))
    h, V = q.make_integrals(L, 4)
    s = DMRGU1(h, V, N, 1).sigma(m)
    mask = m.psi_from_flat(np.ones(m.psi_to_flat().size)) != 0
    assert np.abs(s[~mask]).max(initial=0.0) == 0.0


@pytest.mark.parametrize("N", [6, 5])
def test_exact_bond_dimension_reproduces_ed(N):
    L, D = 6, 64   # 4**(L/2) = 64: no truncation at any bond
    two = N % 2
    h, V = q.make_integrals(L, 11)
    E0, _ = FCI(h, V, N, two).ground_state()
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, 3, 2))
    E, err, _ = DMRGU1(h, V, N, two).sweeps(m, D, nsweeps=2)
    assert abs(E[-1] - E0) < 1e-9
    assert max(err) < 1e-20


def test_truncated_dmrg_is_variational():
    L, N, D = 6, 6, 8
    h, V = q.make_integrals(L, 12)
    E0, _ = FCI(h, V, N, 0).ground_state()
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 8, 2))
    E, err, _ = DMRGU1(h, V, N, 0).sweeps(m, D, nsweeps=2)
    assert E[-1] >= E0 - 1e-10
    assert E[-1] <= E[0] + 1e-9
