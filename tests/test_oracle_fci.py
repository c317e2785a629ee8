"""Pins of the determinant-space oracle against closed forms and invariants."""
import numpy as np
import pytest

import qcinputs as q
from oracle.fci import FCI, DetSpace


def test_hubbard_dimer_closed_form():
    # two sites, two electrons, hopping -t, on-site U: E0 = (U - sqrt(U^2 + 16 t^2)) / 2
    for t, U in [(1.0, 3.0), (0.7, 0.0), (0.3, 8.0)]:
        h = np.array([[0.0, -t], [-t, 0.0]])
        V = np.zeros((2, 2, 2, 2))
        V[0, 0, 0, 0] = V[1, 1, 1, 1] = U
        E, _ = FCI(h, V, 2, 0).ground_state()
        assert abs(E - (U - np.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_noninteracting_diagonal():
    # V = 0, diagonal h: E0 = 2 * (sum of the N/2 lowest h_pp)
    L, N = 6, 4
    d = np.array([0.3, -1.2, 0.5, -0.7, 2.0, -0.1])
    E, _ = FCI(np.diag(d), np.zeros((L,) * 4), N, 0).ground_state()
    assert abs(E - 2 * np.sort(d)[: N // 2].sum()) < 1e-12


def test_dimension_cas10_10():
    assert DetSpace(10, 10, 0).dim == 63504


def test_hermitian_and_rdm_identities():
    L, N = 5, 4
    h, V = q.make_integrals(L, 3)
    f = FCI(h, V, N, 0)
    H = f.matrix().toarray()
    assert np.abs(H - H.T).max() < 1e-12
    E, c = f.ground_state()
    assert abs(E - np.linalg.eigvalsh(H)[0]) < 1e-10
    g1, g2 = f.rdm12(c)
    assert abs(np.trace(g1) - N) < 1e-10
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-9
    assert np.abs(np.einsum("pqrr->pq", g2) - (N - 1) * g1).max() < 1e-9
    assert abs(np.einsum("pq,pq->", h, g1) + 0.5 * np.einsum("pqrs,pqrs->", V, g2) - E) < 1e-9


def test_integral_symmetry_and_psd():
    h, V = q.make_integrals(6, 9)
    assert np.allclose(h, h.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2)]:
        assert np.allclose(V, V.transpose(perm))
    M = V.reshape(36, 36)
    assert np.linalg.eigvalsh(M).min() > -1e-10
    assert np.allclose(np.diag(h), np.linspace(-2, 0.5, 6))


def test_spin_filter_selects_singlet():
    L, N = 4, 4
    h, V = q.make_integrals(L, 5)
    f = FCI(h, V, N, 0)
    E0, c0 = f.ground_state(two_s=0)
    assert abs(c0 @ f.s2_apply(c0)) < 1e-8
    E2, c2 = f.ground_state(two_s=2)
    assert abs(c2 @ f.s2_apply(c2) - 2.0) < 1e-8
