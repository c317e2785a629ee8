"""Pins of oracle/orbital_qi.py against what the definitions and the mathematics fix.

* rho_ij against a brute-force construction: every determinant built by applying its
  creation operators, one by one, to the vacuum of a Jordan-Wigner chain whose first
  modes are those of orbitals i and j (no sign formula), then the partial trace by a
  reshape;
* rho_ij against the FCI oracle's density matrices (its own excitation code): every
  <E_pq> and <E_pq E_rs - delta_qr E_ps> with p, q, r, s in {i, j} equals
  Tr rho_ij O for O built from 4-mode Jordan-Wigner matrices, and the spin-resolved
  hopping <a+_{i up} a_{j up}> likewise;
* closed forms: a pair a|20> + b|02> (entropies -a^2 ln a^2 - b^2 ln b^2, mutual
  information twice that), a single determinant (all zero), an orbital that is always
  empty (no mutual information with anything);
* the Fiedler vector of a path graph with hidden labels (closed form
  cos(pi (k + 1/2) / n) along the path; the order recovers the path up to reversal), and
  the mutual-information ordering recovering a hidden chain of a strongly repulsive
  hopping model.
"""
import itertools

import numpy as np
import pytest

import qcinputs as q
from oracle import orbital_qi as qi
from oracle.fci import FCI, DetSpace, excitation_matrix


def _brute_rho(dets, c, i, j, L):
    """rho_ij by applying creation operators in a Jordan-Wigner chain ordered
    (i up, i dn, j up, j dn, the other orbitals' modes in index order)."""
    order = [2 * i, 2 * i + 1, 2 * j, 2 * j + 1] + [k for k in range(2 * L) if k // 2 not in (i, j)]
    pos = {k: n for n, k in enumerate(order)}
    c = np.asarray(c, float) / np.linalg.norm(c)
    vec = {}
    for b, cd in zip(dets, c):
        b = int(b)
        modes = [k for k in range(2 * L) if (b >> k) & 1]
        state, sign = 0, 1.0
        for k in reversed(modes):            # a+_{k1} a+_{k2} ... |vac>: rightmost first
            p = pos[k]
            assert not (state >> p) & 1
            if bin(state & ((1 << p) - 1)).count("1") % 2:
                sign = -sign
            state |= 1 << p
        vec[state] = vec.get(state, 0.0) + sign * cd
    rest = 4 ** (L - 2)
    M = np.zeros((16, rest))
    for state, a in vec.items():
        x = (state & 1) + 2 * ((state >> 1) & 1)
        y = ((state >> 2) & 1) + 2 * ((state >> 3) & 1)
        M[4 * x + y, state >> 4] += a
    return M @ M.T


def _local_ops():
    """Jordan-Wigner a+ for the 4 modes (i up, i dn, j up, j dn) on 16 states; basis index
    4 x + y with x = n_{i up} + 2 n_{i dn}, y = n_{j up} + 2 n_{j dn}."""
    def idx(bits):
        return 4 * (bits[0] + 2 * bits[1]) + bits[2] + 2 * bits[3]
    cre = []
    for m in range(4):
        A = np.zeros((16, 16))
        for bits in itertools.product((0, 1), repeat=4):
            if bits[m]:
                continue
            nb = list(bits)
            nb[m] = 1
            A[idx(nb), idx(bits)] = (-1) ** sum(bits[:m])
        cre.append(A)
    return cre


def _ground(L, N, two_s, seed):
    h, V = q.make_integrals(L, seed)
    f = FCI(h, V, N, two_s)
    _, c = f.ground_state(two_s=two_s)
    return f, c


@pytest.mark.parametrize("L,N,two_s,seed", [(4, 4, 0, 3), (5, 5, 1, 4), (5, 4, 2, 6)])
def test_rho_equals_the_brute_force_partial_trace(L, N, two_s, seed):
    f, c = _ground(L, N, two_s, seed)
    for i, j in itertools.combinations(range(L), 2):
        r = qi.two_orbital_rdm(f.space.dets, c, i, j)
        assert np.abs(r - _brute_rho(f.space.dets, c, i, j, L)).max() <= 1e-14
        assert abs(np.trace(r) - 1) <= 1e-13
        assert np.abs(r - r.T).max() <= 1e-15
        assert np.linalg.eigvalsh(r).min() >= -1e-14


@pytest.mark.parametrize("L,N,two_s,seed", [(5, 4, 0, 7), (5, 5, 1, 8)])
def test_rho_reproduces_the_fci_density_matrices(L, N, two_s, seed):
    f, c = _ground(L, N, two_s, seed)
    g1, G = f.rdm12(c)
    cre = _local_ops()
    ann = [a.T for a in cre]
    orb = lambda which: (0, 1) if which == 0 else (2, 3)     # local modes of orbital 0 (i) or 1 (j)
    E = {(a, b): sum(cre[orb(a)[s]] @ ann[orb(b)[s]] for s in range(2)) for a in (0, 1) for b in (0, 1)}
    for i, j in itertools.combinations(range(L), 2):
        r = qi.two_orbital_rdm(f.space.dets, c, i, j)
        lab = (i, j)
        for a, b in itertools.product((0, 1), repeat=2):
            assert abs(np.trace(r @ E[a, b].T) - g1[lab[a], lab[b]]) <= 1e-12
        for a, b, x, y in itertools.product((0, 1), repeat=4):
            O = E[a, b] @ E[x, y] - (E[a, y] if b == x else 0)
            assert abs(np.trace(r @ O.T) - G[lab[a], lab[b], lab[x], lab[y]]) <= 1e-12
        # spin-resolved hopping a+_{i up} a_{j up}, straight from the determinant space
        hop = excitation_matrix(f.space, f.space, 2 * i, 2 * j)
        assert abs(np.trace(r @ (cre[0] @ ann[2]).T) - c @ (hop @ c)) <= 1e-12


@pytest.mark.parametrize("a", [1.0, 0.8, np.sqrt(0.5)])
def test_pair_state_closed_forms(a):
    b = np.sqrt(1 - a * a)
    # L = 3, orbital 2 always empty: |20 0> and |02 0>
    sp = DetSpace(3, 2, 0)
    c = np.zeros(sp.dim)
    c[sp.index(np.uint64(0b11))[0]] = a
    c[sp.index(np.uint64(0b1100))[0]] = b
    rho = [[qi.two_orbital_rdm(sp.dets, c, i, j) if i < j else None for j in range(3)] for i in range(3)]
    S1, I = qi.mutual_information(rho, 3)
    w = np.array([a * a, b * b])
    w = w[w > 0]
    s = float(-np.sum(w * np.log(w)))
    assert np.allclose(S1, [s, s, 0.0], atol=1e-14)
    assert abs(I[0, 1] - 2 * s) <= 1e-14
    assert abs(I[0, 2]) <= 1e-14 and abs(I[1, 2]) <= 1e-14
    assert abs(qi.entropy(rho[0][1])) <= 1e-14            # the pair is pure


def test_mutual_information_is_nonnegative_and_bounded():
    f, c = _ground(5, 5, 1, 9)
    rho = [[qi.two_orbital_rdm(f.space.dets, c, i, j) if i < j else None for j in range(5)] for i in range(5)]
    S1, I = qi.mutual_information(rho, 5)
    assert (S1 >= -1e-14).all() and (S1 <= np.log(4) + 1e-12).all()
    assert (I >= -1e-12).all() and (I <= 2 * np.log(4) + 1e-12).all()
    assert np.abs(I - I.T).max() == 0 and np.abs(np.diag(I)).max() == 0
    assert I.max() > 1e-3


@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2), (14, 3)])
def test_fiedler_vector_of_a_hidden_path(n, seed):
    perm = np.random.default_rng(seed).permutation(n)       # perm[k]: label of the k-th vertex
    I = np.zeros((n, n))
    for k in range(n - 1):
        I[perm[k], perm[k + 1]] = I[perm[k + 1], perm[k]] = 1.0
    order, f = qi.fiedler_order(I)
    assert list(order) in (list(perm), list(perm[::-1]))
    ref = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    ref /= np.linalg.norm(ref)
    along = f[perm]
    assert min(np.abs(along - ref).max(), np.abs(along + ref).max()) <= 1e-12


@pytest.mark.parametrize("seed", [1, 4, 7])
def test_mutual_information_order_recovers_a_hidden_chain(seed):
    """A half-filled hopping chain in a hidden order (t = -1 between neighbours along it,
    on-site repulsion 4, weak random couplings elsewhere): in this strongly repulsive regime
    the entanglement is local and the ordering from the ground state's mutual information
    is that chain, up to reversal. (At weak repulsion the half-filled chain's mutual
    information reaches across the chain and the Fiedler order need not be the chain.)"""
    L, N = 6, 6
    rng = np.random.default_rng(seed)
    perm = rng.permutation(L)
    h = 0.01 * rng.normal(size=(L, L))
    h = h + h.T
    for k in range(L - 1):
        h[perm[k], perm[k + 1]] = h[perm[k + 1], perm[k]] = -1.0
    V = np.zeros((L,) * 4)
    for p in range(L):
        V[p, p, p, p] = 4.0
    f = FCI(h, V, N, 0)
    _, c = f.ground_state(two_s=0)
    rho = [[qi.two_orbital_rdm(f.space.dets, c, i, j) if i < j else None for j in range(L)] for i in range(L)]
    _, I = qi.mutual_information(rho, L)
    order, _ = qi.fiedler_order(I)
    assert list(order) in (list(perm), list(perm[::-1]))


def _pair_spin_ops():
    """S_z and S_+ of orbitals i and j together on the 16 states of the pair."""
    cre = _local_ops()
    ann = [a.T for a in cre]
    sz = 0.5 * sum(cre[2 * o] @ ann[2 * o] - cre[2 * o + 1] @ ann[2 * o + 1] for o in (0, 1))
    sp = sum(cre[2 * o] @ ann[2 * o + 1] for o in (0, 1))
    return sz, sp


@pytest.mark.parametrize("L,N,two_s,seed", [(4, 4, 0, 3), (5, 5, 1, 4), (5, 4, 2, 6), (5, 5, 3, 2)])
def test_multiplet_average_is_spin_invariant(L, N, two_s, seed):
    """The multiplet average of rho_ij commutes with the total spin of the pair (it is the
    partial trace of a rotation-invariant operator); for a singlet it is the plain rho_ij, and
    for S > 0 the M = S component alone does not commute with S_+ (so the average matters)."""
    f, c = _ground(L, N, two_s, seed)
    sz, sp = _pair_spin_ops()
    broken = 0.0
    for i, j in itertools.combinations(range(L), 2):
        r = qi.multiplet_rdm(L, N, two_s, c, i, j)
        assert abs(np.trace(r) - 1) <= 1e-12
        assert np.abs(r @ sz - sz @ r).max() <= 1e-12
        assert np.abs(r @ sp - sp @ r).max() <= 1e-12
        r0 = qi.two_orbital_rdm(f.space.dets, c, i, j)
        if two_s == 0:
            assert np.abs(r - r0).max() <= 1e-13
        broken = max(broken, np.abs(r0 @ sp - sp @ r0).max())
    if two_s > 0:
        assert broken > 1e-3
