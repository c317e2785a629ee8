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


@pytest.mark.parametrize("L,eta,seed", [(5, 2.0, 1), (8, 2.0, 2), (8, 1.0, 3), (12, 1.5, 4)])
def test_ordering_cost_and_refinement(L, eta, seed):
    """The cost equals its plain definition; the refined order is never worse than its start
    and no single exchange of two orbitals lowers it further (checked over all exchanges)."""
    import itertools
    import paper_2603_28648_b300 as qd
    from oracle import orbital_qi as qi
    lib = qd.load(ensure_built())
    rng = np.random.default_rng(seed)
    A = rng.exponential(size=(L, L))
    A = A + A.T
    np.fill_diagonal(A, 0.0)
    start = rng.permutation(L)
    c0 = qd.ordering_cost(A, start, eta, lib=lib)
    assert abs(c0 - qi.ordering_cost(A, start, eta)) <= 1e-12 * c0
    o, n = qd.refine_order(A, start, eta, lib=lib)
    assert sorted(o) == list(range(L))
    c1 = qi.ordering_cost(A, o, eta)
    assert c1 <= c0 + 1e-12 and (n == 0 or c1 < c0)
    for a, b in itertools.combinations(range(L), 2):
        t = o.copy()
        t[a], t[b] = t[b], t[a]
        assert qi.ordering_cost(A, t, eta) >= c1 - 1e-9 * c1


def test_path_graph_order_is_the_global_minimum():
    """On a path graph with hidden labels the Fiedler order has the smallest possible cost
    (brute force over all 720 orders of six orbitals) and the refinement leaves it alone."""
    import paper_2603_28648_b300 as qd
    from oracle import orbital_qi as qi
    lib = qd.load(ensure_built())
    n = 6
    perm = np.random.default_rng(5).permutation(n)
    I = np.zeros((n, n))
    for k in range(n - 1):
        I[perm[k], perm[k + 1]] = I[perm[k + 1], perm[k]] = 1.0
    order, _ = qd.fiedler_order(I, lib=lib)
    best = qi.best_order(I)
    assert qd.ordering_cost(I, order, lib=lib) == qi.ordering_cost(I, best) == n - 1
    o, swaps = qd.refine_order(I, order, lib=lib)
    assert swaps == 0 and list(o) == list(order)


def test_invalid_ordering_arguments_are_rejected():
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    I = np.ones((4, 4)) - np.eye(4)
    for order, eta in (([0, 1, 1, 3], 2.0), ([0, 1, 2, 4], 2.0), ([0, 1, 2, 3], 0.0), ([0, 1, 2, 3], np.nan)):
        with pytest.raises(qd.QcdmrgError):
            qd.ordering_cost(I, order, eta, lib=lib)
        with pytest.raises(qd.QcdmrgError):
            qd.refine_order(I, order, eta, lib=lib)
    J = I.copy()
    J[0, 1] = 2.0
    with pytest.raises(qd.QcdmrgError):
        qd.ordering_cost(J, [0, 1, 2, 3], lib=lib)
