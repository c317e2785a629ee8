"""Pins of the SU(2) spin-adapted two-site tangent space (oracle/mpssu2.py).

Closed forms of Clebsch-Gordan coefficients; P has orthonormal columns of
total spin S (S^2 applied to every column by the determinant-space operator of
the FCI oracle); at exact bond dimension the tangent space is the whole spin-S,
M = S space (its dimension is #(2Sz = 2S) - #(2Sz = 2S + 2) determinants) and
the lowest eigenvalue of P^T H P is the spin-filtered FCI ground-state energy;
at truncated bond dimension the energy is variational and H_eff Hermitian."""
import math

import numpy as np
import pytest

import qcinputs as q
from oracle.fci import FCI, DetSpace
from oracle.mpssu2 import TangentSU2, cg


def test_clebsch_gordan_closed_forms():
    r2 = 1 / math.sqrt(2)
    assert abs(cg(1, 1, 1, -1, 0, 0) - r2) < 1e-15          # <1/2 1/2; 1/2 -1/2 | 0 0>
    assert abs(cg(1, -1, 1, 1, 0, 0) + r2) < 1e-15          # <1/2 -1/2; 1/2 1/2 | 0 0>
    assert abs(cg(1, 1, 1, 1, 2, 2) - 1.0) < 1e-15          # stretched state
    assert abs(cg(1, 1, 1, -1, 2, 0) - r2) < 1e-15          # triplet M = 0
    assert abs(cg(2, 2, 1, -1, 1, 1) - math.sqrt(2 / 3)) < 1e-15   # <1 1; 1/2 -1/2 | 1/2 1/2>
    assert abs(cg(2, 0, 1, 1, 1, 1) + math.sqrt(1 / 3)) < 1e-15    # <1 0; 1/2 1/2 | 1/2 1/2>
    assert cg(1, 1, 1, 1, 0, 0) == 0.0                       # M mismatch


CASES = [(4, 4, 0, 1), (5, 5, 1, 1), (5, 3, 1, 2), (6, 6, 2, 2), (6, 6, 0, 2)]


@pytest.mark.parametrize("L,N,two_s,l", CASES)
def test_exact_tangent_space_is_the_spin_sector(L, N, two_s, l):
    t = TangentSU2(L, N, two_s, l)
    P = t.P
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < 1e-12
    # dimension of the spin-S, M = S space
    above = DetSpace(L, N, two_s + 2).dim if (N + two_s + 2) // 2 <= L else 0
    assert P.shape[1] == DetSpace(L, N, two_s).dim - above
    h, V = q.make_integrals(L, 7)
    f = FCI(h, V, N, two_s)
    ss = (two_s / 2) * (two_s / 2 + 1)
    S2P = np.column_stack([f.s2_apply(P[:, k]) for k in range(P.shape[1])])
    assert np.abs(S2P - ss * P).max() < 1e-11
    Heff = t.heff_matrix(f)
    assert np.abs(Heff - Heff.T).max() < 1e-11
    e_fci, _ = f.ground_state(two_s=two_s)
    e = np.linalg.eigvalsh(0.5 * (Heff + Heff.T))[0]
    assert abs(e - e_fci) < 1e-9


@pytest.mark.parametrize("L,N,two_s,l,cap", [(6, 6, 0, 2, 2), (7, 7, 1, 2, 2), (8, 8, 0, 3, 3)])
def test_truncated_tangent_space(L, N, two_s, l, cap):
    t = TangentSU2(L, N, two_s, l, cap=cap, seed=5)
    P = t.P
    assert P.shape[1] > 0
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < 1e-12
    h, V = q.make_integrals(L, 11)
    f = FCI(h, V, N, two_s)
    ss = (two_s / 2) * (two_s / 2 + 1)
    for k in range(0, P.shape[1], max(1, P.shape[1] // 7)):
        assert np.abs(f.s2_apply(P[:, k]) - ss * P[:, k]).max() < 1e-11
    Heff = t.heff_matrix(f)
    assert np.abs(Heff - Heff.T).max() < 1e-10
    e_fci, _ = f.ground_state(two_s=two_s)
    assert np.linalg.eigvalsh(0.5 * (Heff + Heff.T))[0] >= e_fci - 1e-10
    # H_eff psi by the definition equals the matrix on a random vector
    psi = np.random.default_rng(2).normal(size=P.shape[1])
    assert np.abs(t.heff(f, psi) - Heff @ psi).max() < 1e-10


@pytest.mark.parametrize("L,N,two_s,l,cap", [(6, 6, 0, 2, 2), (7, 7, 1, 2, 2), (7, 5, 1, 3, 2)])
def test_su2_space_as_u1_mps_matches_operator_oracle(L, N, two_s, l, cap):
    """The SU(2) space written as a U(1) MPS (bond states = all M components): the
    Clebsch-Gordan map C is an isometry, the U(1) expansion of every SU(2) basis state is
    its determinant vector, and sigma of the plain SU(2) definition equals C^T applied to
    the operator-based U(1) oracle's sigma (a separately written code path)."""
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpssu2 import to_u1
    from oracle.mpsu1 import Projector
    t = TangentSU2(L, N, two_s, l, cap=cap, seed=5)
    mps, C = to_u1(t)
    assert np.abs(C.T @ C - np.eye(C.shape[1])).max() < 1e-13
    pr = Projector(mps, t.space)
    for k in range(C.shape[1]):
        assert np.abs(pr.apply(mps.psi_from_flat(C[:, k])) - t.P[:, k]).max() < 1e-13
    h, V = q.make_integrals(L, 11)
    f = FCI(h, V, N, two_s)
    psi = np.random.default_rng(3).normal(size=C.shape[1])
    s_su2 = t.heff(f, psi)
    s_u1 = DMRGU1(h, V, N, two_s).sigma(mps, mps.psi_from_flat(C @ psi))
    s_via = C.T @ mps.psi_to_flat(s_u1)
    assert np.linalg.norm(s_su2 - s_via) <= 1e-12 * np.linalg.norm(s_su2)
