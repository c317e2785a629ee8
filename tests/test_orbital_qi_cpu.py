"""Orbital entanglement and ordering through the C ABI (host code, no device) against
oracle/orbital_qi.py: one-orbital entropies and mutual information from two-orbital density
matrices of FCI ground states, the Fiedler order and vector of mutual-information matrices
(random ones, and a path graph with hidden labels), and the argument checks."""
import ctypes
import itertools

import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built


def _rho_blocks(L, N, two_s, seed):
    from oracle import orbital_qi as qi
    from oracle.fci import FCI
    h, V = q.make_integrals(L, seed)
    f = FCI(h, V, N, two_s)
    _, c = f.ground_state(two_s=two_s)
    R = np.zeros((L, L, 16, 16))
    nested = [[None] * L for _ in range(L)]
    for i, j in itertools.combinations(range(L), 2):
        R[i, j] = nested[i][j] = qi.two_orbital_rdm(f.space.dets, c, i, j)
    return R, nested


@pytest.mark.parametrize("L,N,two_s,seed", [(4, 4, 0, 3), (5, 5, 1, 4), (6, 6, 0, 5), (6, 4, 2, 8)])
def test_entropies_and_mutual_information_match_the_oracle(L, N, two_s, seed):
    import paper_2603_28648_b300 as qd
    from oracle import orbital_qi as qi
    lib = qd.load(ensure_built())
    R, nested = _rho_blocks(L, N, two_s, seed)
    s1, I = qd.orbital_entanglement(R, lib=lib)
    s1o, Io = qi.mutual_information(nested, L)
    assert np.abs(s1 - s1o).max() <= 1e-12
    assert np.abs(I - Io).max() <= 1e-12
    assert np.array_equal(I, I.T) and not np.diag(I).any()


@pytest.mark.parametrize("L,seed", [(2, 1), (5, 2), (12, 3), (30, 4)])
def test_fiedler_order_matches_the_oracle(L, seed):
    import paper_2603_28648_b300 as qd
    from oracle import orbital_qi as qi
    lib = qd.load(ensure_built())
    rng = np.random.default_rng(seed)
    A = rng.exponential(size=(L, L))
    A = A + A.T
    np.fill_diagonal(A, 0.0)
    order, f = qd.fiedler_order(A, lib=lib)
    oo, fo = qi.fiedler_order(A)
    assert np.abs(f - fo).max() <= 1e-10
    assert list(order) == list(oo)
    assert sorted(order) == list(range(L))


def test_fiedler_order_recovers_a_hidden_path():
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    n = 20
    perm = np.random.default_rng(9).permutation(n)
    I = np.zeros((n, n))
    for k in range(n - 1):
        I[perm[k], perm[k + 1]] = I[perm[k + 1], perm[k]] = 0.5 + 0.01 * k
    order, _ = qd.fiedler_order(I, lib=lib)
    assert list(order) in (list(perm), list(perm[::-1]))
    h, V = q.make_integrals(n, 1)
    h2, V2 = qd.reorder_integrals(h, V, order)
    assert h2[3, 5] == h[order[3], order[5]] and V2[1, 2, 3, 4] == V[order[1], order[2], order[3], order[4]]


def test_invalid_entanglement_arguments_are_rejected():
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    null_d, null_i = ctypes.cast(None, dp), ctypes.cast(None, ip)
    R = np.zeros((3, 3, 16, 16))
    m = np.zeros((3, 3))
    rp = R.ctypes.data_as(dp)
    mp = m.ctypes.data_as(dp)
    order = np.zeros(3, dtype=np.int32)
    op = order.ctypes.data_as(ip)
    assert lib.qcdmrg_orbital_entanglement(1, rp, null_d, mp) == -1
    assert lib.qcdmrg_orbital_entanglement(3, null_d, null_d, mp) == -1
    R[0, 1, 2, 2] = np.nan
    assert lib.qcdmrg_orbital_entanglement(3, rp, null_d, mp) == -1
    assert lib.qcdmrg_fiedler_order(1, mp, op, null_d) == -1
    assert lib.qcdmrg_fiedler_order(3, mp, null_i, null_d) == -1
    m[0, 1] = 1.0                                   # not symmetric
    assert lib.qcdmrg_fiedler_order(3, mp, op, null_d) == -1
    m[1, 0] = 1.0
    assert lib.qcdmrg_fiedler_order(3, mp, op, null_d) == 0
    with pytest.raises(qd.QcdmrgError):
        qd.fiedler_order(np.array([[0.0, 1.0], [2.0, 0.0]]), lib=lib)
