"""SU(2) spin-adapted two-site tangent space and the plain definition of H_eff.

TEST INFRASTRUCTURE (oracle): imported only by tests/.

Conventions (the paper states none; these readings are fixed here):
  * site multiplets: |0> (N=0, S=0); the doublet |1; 1/2, m> with m=+1/2 ->
    a+_up|0>, m=-1/2 -> a+_dn|0> (S_- a+_up|0> = +a+_dn|0>, Condon-Shortley);
    |2> = a+_up a+_dn|0> (N=2, S=0); local configuration index = n_up + 2 n_dn,
    as in the U(1) oracle;
  * Clebsch-Gordan coefficients <j1 m1; j2 m2 | J M> in the Condon-Shortley
    phase convention (sympy.physics.wigner.clebsch_gordan);
  * the left block is coupled left to right, (block) x (site) -> block'; the
    right block right to left, (site) x (block) -> block'; the two-site
    wavefunction couples a = (left block x site l) to j_a, b = (site l+1 x
    right block) to j_b, and (j_a x j_b) -> (S, M = S). Spin-orbitals are in
    chain order, so a product of a state of the sites before a cut with a
    state of the sites after it is the determinant product with sign +1.
A multiplet is stored with all its 2S+1 components as vectors in the Fock
space of its sites (4 states per site, configuration index = sum over sites of
local index * 4^position). The reduced two-site wavefunction psi[(a, b)] is
mapped to the determinant vector of the (N, 2Sz = 2S) space by P, and
  H_eff psi = P^T H_FCI P psi,
the projection of the Hamiltonian onto the SU(2)-adapted two-site tangent
space; P has orthonormal columns of total spin S.
"""

from functools import lru_cache

import numpy as np
from sympy import Rational
from sympy.physics.wigner import clebsch_gordan

from .fci import DetSpace

# site multiplets: (particle number, 2S, local configuration of each component m = S, S-1, ...)
SITE = [(0, 0, [0]), (1, 1, [1, 2]), (2, 0, [3])]


@lru_cache(maxsize=None)
def cg(two_j1, two_m1, two_j2, two_m2, two_J, two_M):
    """<j1 m1; j2 m2 | J M> from doubled angular momenta."""
    if two_m1 + two_m2 != two_M:
        return 0.0
    h = Rational(1, 2)
    return float(clebsch_gordan(two_j1 * h, two_j2 * h, two_J * h, two_m1 * h, two_m2 * h, two_M * h))


class Mult:
    """One multiplet: particle number n, doubled spin s, components vec[i] for 2m = s - 2i."""

    def __init__(self, n, s, vec):
        self.n, self.s, self.vec = n, s, np.asarray(vec, float)


def site_mults():
    out = []
    for n, s, cfg in SITE:
        v = np.zeros((s + 1, 4))
        for i, c in enumerate(cfg):
            v[i, c] = 1.0
        out.append(Mult(n, s, v))
    return out


def couple(m1, m2, two_J, first_dim_left=True):
    """Components of |(m1 m2) J M> = sum CG <j1 m1; j2 m2|J M> |m1> (x) |m2>, with m1's sites
    before m2's sites in chain order (Fock index = idx1 + dim1 * idx2)."""
    d1, d2 = m1.vec.shape[1], m2.vec.shape[1]
    out = np.zeros((two_J + 1, d1 * d2))
    for i in range(two_J + 1):
        two_M = two_J - 2 * i
        for i1 in range(m1.s + 1):
            two_m1 = m1.s - 2 * i1
            two_m2 = two_M - two_m1
            if abs(two_m2) > m2.s or (m2.s - two_m2) % 2:
                continue
            c = cg(m1.s, two_m1, m2.s, two_m2, two_J, two_M)
            if c == 0.0:
                continue
            i2 = (m2.s - two_m2) // 2
            # Fock index of the product: site configurations of m1 first
            out[i] += c * np.kron(m2.vec[i2], m1.vec[i1])
    return out


def coupled_candidates(A, B):
    """All coupled multiplets (A_k x B_l) -> J, as Mult objects with their labels."""
    out = []
    for ka, a in enumerate(A):
        for kb, b in enumerate(B):
            for two_J in range(abs(a.s - b.s), a.s + b.s + 1, 2):
                out.append(((ka, kb, two_J), Mult(a.n + b.n, two_J, couple(a, b, two_J))))
    return out


def grow(block, left, rng, dims=None):
    """Enlarge a block by one site and keep, per (N, 2S) sector, dims[(N, 2S)] random
    orthonormal combinations of the coupled candidates (all of them when dims is None).
    Left blocks: (block) x (site); right blocks: (site) x (block)."""
    cands = coupled_candidates(block, site_mults()) if left else coupled_candidates(site_mults(), block)
    by = {}
    for lab, m in cands:
        by.setdefault((m.n, m.s), []).append(m)
    new = []
    for key in sorted(by):
        ms = by[key]
        k = len(ms) if dims is None else min(len(ms), dims.get(key, 0))
        if k == 0:
            continue
        if dims is None:
            U = np.eye(len(ms))
        else:
            Q, _ = np.linalg.qr(rng.normal(size=(len(ms), len(ms))))
            U = Q[:, :k]
        stack = np.stack([m.vec for m in ms])            # (ncand, 2S+1, fock)
        comb = np.einsum("cmf,ck->kmf", stack, U)
        for j in range(k):
            new.append(Mult(key[0], key[1], comb[j]))
    return new


def vacuum():
    return [Mult(0, 0, np.ones((1, 1)))]


class TangentSU2:
    """Two-site tangent space at the centre (l, l+1) of an SU(2)-adapted MPS of L sites with
    N electrons and total spin S = two_s / 2; bond multiplet counts capped per sector by
    `cap` (None: exact, nothing discarded)."""

    def __init__(self, L, N, two_s, l, cap=None, seed=0):
        self.L, self.N, self.two_s, self.l = L, N, two_s, l
        rng = np.random.default_rng(seed)
        left = vacuum()
        self.lefts = [left]            # left blocks of 0, 1, ..., l sites
        for _ in range(l):
            left = grow(left, True, rng, None if cap is None else _caps(left, cap, True))
            self.lefts.append(left)
        right = vacuum()
        self.rights = [right]          # right blocks of the last 0, 1, ..., L-l-2 sites
        for _ in range(L - l - 2):
            right = grow(right, False, rng, None if cap is None else _caps(right, cap, False))
            self.rights.append(right)
        self.left, self.right = left, right
        a = coupled_candidates(left, site_mults())     # (left block x site l)
        b = coupled_candidates(site_mults(), right)    # (site l+1 x right block)
        self.space = DetSpace(L, N, two_s)
        cols, labels = [], []
        nl = 4 ** (l + 1)
        for la, ma in a:
            for lb, mb in b:
                if ma.n + mb.n != N:
                    continue
                if not (abs(ma.s - mb.s) <= two_s <= ma.s + mb.s) or (ma.s + mb.s - two_s) % 2:
                    continue
                v = np.zeros(nl * mb.vec.shape[1])
                for ia in range(ma.s + 1):
                    two_ma = ma.s - 2 * ia
                    two_mb = two_s - two_ma
                    if abs(two_mb) > mb.s or (mb.s - two_mb) % 2:
                        continue
                    c = cg(ma.s, two_ma, mb.s, two_mb, two_s, two_s)
                    if c:
                        v += c * np.kron(mb.vec[(mb.s - two_mb) // 2], ma.vec[ia])
                cols.append(self._to_dets(v))
                labels.append((la, lb))
        self.labels = labels
        self.cand_a, self.cand_b = a, b
        self.P = np.stack(cols, axis=1) if cols else np.zeros((self.space.dim, 0))

    def _to_dets(self, v):
        """Fock vector (local configs, site 0 fastest) -> coefficients on the (N, 2Sz) determinants."""
        out = np.zeros(self.space.dim)
        nz = np.nonzero(v)[0]
        L = self.L
        for f in nz:
            bits, x = 0, int(f)
            for p in range(L):
                c = x % 4
                x //= 4
                if c & 1:
                    bits |= 1 << (2 * p)
                if c & 2:
                    bits |= 1 << (2 * p + 1)
            idx, ok = self.space.index(np.array([bits], dtype=np.uint64))
            if not ok[0]:
                raise AssertionError("state outside the (N, 2Sz) space")
            out[idx[0]] += v[f]
        return out

    def heff(self, fci, psi):
        """H_eff psi = P^T H P psi (plain definition)."""
        return self.P.T @ fci.apply(self.P @ psi)

    def heff_matrix(self, fci):
        HP = np.column_stack([fci.apply(self.P[:, k]) for k in range(self.P.shape[1])])
        return self.P.T @ HP


def _caps(block, cap, left):
    """Per-sector multiplet caps of the next block: at most `cap` per (N, 2S)."""
    cands = coupled_candidates(block, site_mults()) if left else coupled_candidates(site_mults(), block)
    keys = {(m.n, m.s) for _, m in cands}
    return {k: cap for k in keys}


def _states(block):
    """All components of a block's multiplets as U(1) states: labels (N, 2M) and Fock vectors,
    sorted by label (stable within a label)."""
    st = []
    for m in block:
        for i in range(m.s + 1):
            st.append(((m.n, m.s - 2 * i), m.vec[i]))
    st.sort(key=lambda t: t[0])
    return st


def to_u1(t):
    """The same state space as a U(1)xU(1) MPS: bond states are all M components of the
    multiplets. Returns (mps, C) with mps an oracle.mpsu1.MPSU1 (left- and right-canonical
    tensors, psi = 0) and C[flat U(1) psi index, SU(2) column] the Clebsch-Gordan map of the
    reduced two-site wavefunction onto the U(1) one (orthonormal columns)."""
    from .mpsu1 import MPSU1, Bond
    L, l = t.L, t.l
    lst = [_states(b) for b in t.lefts]            # bond b = 0..l
    rst = [_states(b) for b in t.rights]           # right block of k sites -> bond L - k

    def bond(states):
        d = {}
        for lab, _ in states:
            d[lab] = d.get(lab, 0) + 1
        return Bond(d)

    lbonds = {b: bond(lst[b]) for b in range(l + 1)}
    rbonds = {L - k: bond(rst[k]) for k in range(L - l - 1)}
    A, R = {}, {}
    for p in range(l):
        old, new = lst[p], lst[p + 1]
        n_old = 4 ** p
        T = np.zeros((len(old), 4, len(new)))
        Vo = np.stack([v for _, v in old])                    # (D_p, 4^p)
        for c, (_, v) in enumerate(new):
            T[:, :, c] = Vo @ v.reshape(4, n_old).T            # site p is the slowest digit
        A[p] = T
    for k in range(1, L - l - 1):
        p = L - k                                              # site of this step
        new, old = rst[k], rst[k - 1]
        Vo = np.stack([v for _, v in old])                    # (D_{p+1}, 4^(k-1))
        T = np.zeros((len(new), 4, len(old)))
        for r, (_, v) in enumerate(new):
            T[r] = (Vo @ v.reshape(-1, 4)).T                   # site p is the fastest digit
        R[p] = T
    mps = MPSU1(L, t.N, t.two_s, l, lbonds, rbonds, A, R,
                np.zeros((lbonds[l].dim, 4, 4, rbonds[l + 2].dim)))
    VX = np.stack([v for _, v in lst[l]])                     # (D_X, 4^l)
    VY = np.stack([v for _, v in rst[L - l - 2]])             # (D_Y, 4^(L-l-2))
    nX = 4 ** l
    cols = []
    for (la, lb) in t.labels:
        ma = dict(t.cand_a)[la]
        mb = dict(t.cand_b)[lb]
        psi = np.zeros((VX.shape[0], 4, 4, VY.shape[0]))
        for ia in range(ma.s + 1):
            two_ma = ma.s - 2 * ia
            two_mb = t.two_s - two_ma
            if abs(two_mb) > mb.s or (mb.s - two_mb) % 2:
                continue
            c = cg(ma.s, two_ma, mb.s, two_mb, t.two_s, t.two_s)
            if not c:
                continue
            alpha = VX @ ma.vec[ia].reshape(4, nX).T          # (D_X, 4): <x i | a, m_a>
            beta = (VY @ mb.vec[(mb.s - two_mb) // 2].reshape(-1, 4)).T   # (4, D_Y): <j y | b, m_b>
            psi += c * np.einsum("xi,jy->xijy", alpha, beta)
        cols.append(mps.psi_to_flat(psi))
    C = np.stack(cols, axis=1) if cols else np.zeros((len(mps.psi_to_flat()), 0))
    return mps, C
