"""Pins of oracle/configs.py against closed forms and the mathematics.

* spin states: the two-open-shell singlet equals (|a_up b_dn> - |a_dn b_up>)/sqrt(2) in the
  determinant basis; the couplings of one spatial occupation are orthonormal, have
  S^2 = S(S+1) by the FCI oracle's spin operator and M = S, and their number is the
  branching-diagram count C(k, k/2 - S) - C(k, k/2 - S - 1);
* the aufbau reference's energy equals the closed-shell formula
  2 sum_i h_ii + sum_ij (2 (ii|jj) - (ij|ji)) computed from the integrals directly;
* the candidate counts equal the combinatorial counts of determinants within two
  electrons of the reference;
* the energy of a spatial occupation with two open shells is the 1:3 weighted mean of its
  singlet and triplet energies (<CSF|H|CSF> from the FCI matrix).
"""
import math

import numpy as np
import pytest

import qcinputs as q
from oracle import configs as oc
from oracle.fci import FCI, DetSpace


def test_two_shell_singlet_closed_form():
    space, v = oc.config_vector([(1, 2, 0)], [1.0], 3, 2, 0, True)
    ref = np.zeros(space.dim)
    ref[int(space.index(np.uint64(0b1001))[0])] = 1 / math.sqrt(2)    # a+_{0 up} a+_{1 dn}
    ref[int(space.index(np.uint64(0b0110))[0])] = -1 / math.sqrt(2)   # a+_{0 dn} a+_{1 up}
    assert np.abs(v - ref).max() <= 1e-15


@pytest.mark.parametrize("n,two_s", [((1, 1, 1, 1, 0), 0), ((1, 1, 1, 1, 0), 2), ((1, 2, 1, 1, 0), 1),
                                     ((1, 1, 1, 1, 1, 1), 0), ((1, 1, 1, 1, 1, 1), 2), ((2, 1, 0, 1, 1), 3)])
def test_couplings_are_orthonormal_spin_eigenstates(n, two_s):
    L, N = len(n), sum(n)
    h, V = q.make_integrals(L, 2)
    f = FCI(h, V, N, two_s)
    sts = oc.couplings(n, two_s)
    k = sum(1 for x in n if x == 1)
    count = math.comb(k, k // 2 - two_s // 2) - (math.comb(k, k // 2 - two_s // 2 - 1) if k // 2 - two_s // 2 >= 1 else 0)
    assert len(sts) == count
    vs = np.stack([oc.config_vector([st], [1.0], L, N, two_s, True)[1] for st in sts])
    assert np.abs(vs @ vs.T - np.eye(len(sts))).max() <= 1e-13
    S = two_s / 2
    for v in vs:
        assert np.abs(f.s2_apply(v) - S * (S + 1) * v).max() <= 1e-12


@pytest.mark.parametrize("L,N", [(5, 6), (6, 4)])
def test_reference_energy_closed_shell_formula(L, N):
    h, V = q.make_integrals(L, 7)
    cands = oc.candidates_u1(h, V, N, 0)
    ref = [c for c in cands if c[1] == 0]
    assert len(ref) == 1
    occ = [p for p in range(L) if ref[0][2][p] == 3]
    e = 2 * sum(h[i, i] for i in occ) + sum(2 * V[i, i, j, j] - V[i, j, j, i] for i in occ for j in occ)
    assert abs(ref[0][0] - e) <= 1e-12
    su = oc.candidates_su2(h, V, N, 0)
    assert abs([c for c in su if c[1] == 0][0][0] - e) <= 1e-12


@pytest.mark.parametrize("L,N,two_s", [(5, 4, 0), (6, 5, 1), (5, 6, 2)])
def test_candidate_counts(L, N, two_s):
    h, V = q.make_integrals(L, 3)
    na, nb = (N + two_s) // 2, (N - two_s) // 2
    va, vb = L - na, L - nb
    c2 = math.comb
    expect = 1 + na * va + nb * vb + c2(na, 2) * c2(va, 2) + c2(nb, 2) * c2(vb, 2) + na * va * nb * vb
    assert len(oc.candidates_u1(h, V, N, two_s)) == expect


def test_two_open_shell_average_is_the_spin_weighted_mean():
    L, N = 4, 4
    h, V = q.make_integrals(L, 9)
    n = (2, 1, 1, 0)
    occ = {0: 0, 1: 1, 2: 1, 3: 2}
    e_avg = [c[0] for c in oc.candidates_su2(h, V, N, 0) if tuple(occ[s] for s in c[2]) == n]
    # singlet and triplet couplings at M = S, their energies from the FCI matrices
    es = []
    for two_s in (0, 2):
        f = FCI(h, V, N, two_s)
        _, v = oc.config_vector(oc.couplings(n, two_s), [1.0], L, N, two_s, True)
        es.append(v @ (f.matrix() @ v))
    assert len(e_avg) == 1
    assert abs(e_avg[0] - (es[0] + 3 * es[1]) / 4) <= 1e-12
