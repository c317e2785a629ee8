"""Operator-based two-site DMRG with SU(2) spin adaptation, dense FP64 (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The renormalized-operator formulation of spin-adapted quantum-chemical DMRG
(the paper's Method section; its bond dimensions count SU(2) multiplets,
Numerical procedure section). Every quantity is a reduced matrix element
between multiplets (Wigner-Eckart convention of oracle/su2alg.py), so the cost
is that of the multiplet basis, not of its M components.

Tensor operators (spatial orbital p; ranks in brackets):
    c_p = a+_p          (1/2)  components c_{p,+1/2} = a+_{p up}, c_{p,-1/2} = a+_{p dn}
    d_p = a~_p          (1/2)  d_{p,+1/2} = a_{p dn}, d_{p,-1/2} = -a_{p up}
    A^k_pq = [c_p x c_q]^k, B^k_pq = [c_p x d_q]^k, DD^k_pq = [d_p x d_q]^k  (k = 0, 1)
    T_m = 1/2 sum_{q in B} h_mq d_q + sum_{q,r,s in B} (ms|qr) E_qr d_s      (1/2)
with E_pq = sum_sigma a+_{p sigma} a_{q sigma} = -sqrt(2) B^0_pq. T_m is the
complementary operator of a block B for an orbital m outside it: its
components are (-1)^(1/2-mu) S_{m,-mu} of the spin-orbital complementary
operator S_{m sigma} = 1/2 sum h_mq a_{q sigma} + sum (ms|qr) E_qr a_{s sigma}.
A block keeps c, d, A, B, DD of its own orbitals, T of every orbital outside
and its Hamiltonian H; P and Q are formed at a cut from the other side's
normal operators.

Decomposition of H = sum h_pq E_pq + 1/2 sum (pq|rs) sum a+_{p s} a+_{r t} a_{s t} a_{q s}
at a cut L|R into scalar couplings [O_L^k x O_R^k]^0 ("+ h.c." adds the
Hermitian conjugate of the whole term):
    H = H_L + H_R
      - sqrt(2) sum_{p in L} [c_p x T_p(R)]^0 + h.c.
      - sqrt(2) sum_{m in R} [T_m(L) x c_m]^0 + h.c.
      + 1/2 sum_{p,r in L} sum_k (-1)^(1+k) sqrt(2k+1) [A^k_pr x P^k_pr(R)]^0 + h.c.,
            P^k_pr(R) = sum_{s,q in R} (pq|rs) DD^k_sq
      + sum_{i,j in L} sum_k [B^k_ij x Q^k_ij(R)]^0,
            Q^0_ij = sum_{k,l in R} (2 (ij|kl) - (il|kj)) B^0_kl,
            Q^1_ij = sqrt(3) sum_{k,l in R} (il|kj) B^1_kl.
The two pair lines follow from recoupling the four spin-orbital operators
(sum over spins of a+ a+ a a with two indices on each side) into ranks 0 and
1. A product O_1 O_2 of operators on the two parts of a coupled basis (part 1
first in the fermion order) has reduced elements given by the 9j formula
(su2alg.coupled_factor) times (-1)^(parity of O_2 x particle number of the
part-1 ket). Three-operator products of T are recoupled with su2alg.recouple.
Single-site reduced elements are obtained from the explicit 4 x 4 matrices by
the Wigner-Eckart theorem.
"""

import math

import numpy as np
import scipy.sparse.linalg as spla

from .su2alg import cg, coupled_factor, recouple

R2 = math.sqrt(2.0)

# ---------------------------------------------------------------------------
# single site: configurations |0>, |up>, |dn>, |updn>; multiplets |0>, |1/2 m>, |2>
# ---------------------------------------------------------------------------
_CUP = np.zeros((4, 4))
_CUP[1, 0] = 1.0
_CUP[3, 2] = 1.0
_CDN = np.zeros((4, 4))
_CDN[2, 0] = 1.0
_CDN[3, 1] = -1.0
# site multiplets: (n, 2S, configuration of each component 2m = 2S, 2S-2, ...)
SITE_MULT = [(0, 0, [0]), (1, 1, [1, 2]), (2, 0, [3])]
SITE_N = np.array([0, 1, 2])
SITE_S = np.array([0, 1, 0])


def site_c():
    """Components {2q: 4x4} of c = a+ (rank 1/2)."""
    return {1: _CUP, -1: _CDN}


def site_d():
    """Components of d = a~: d_{+1/2} = a_dn, d_{-1/2} = -a_up."""
    return {1: _CDN.T.copy(), -1: -_CUP.T}


def site_couple(X, kx, Y, ky, k):
    """Components of [X^kx x Y^ky]^k on one site (product X Y, doubled ranks)."""
    out = {}
    for q in range(-k, k + 1, 2):
        m = np.zeros((4, 4))
        for q1, Xm in X.items():
            q2 = q - q1
            if q2 in Y:
                c = cg(kx, q1, ky, q2, k, q)
                if c:
                    m += c * (Xm @ Y[q2])
        out[q] = m
    return out


def site_reduced(comps, k):
    """3 x 3 reduced matrix <s||O^k||s'> of a site tensor operator from its
    components, by the Wigner-Eckart theorem; every component must agree."""
    red = np.zeros((3, 3))
    seen = np.zeros((3, 3), bool)
    for a, (na, sa, ca) in enumerate(SITE_MULT):
        for b, (nb, sb, cb) in enumerate(SITE_MULT):
            for ia, conf_a in enumerate(ca):
                ma = sa - 2 * ia
                for ib, conf_b in enumerate(cb):
                    mb = sb - 2 * ib
                    q = ma - mb
                    if abs(q) > k:
                        continue
                    v = comps.get(q, np.zeros((4, 4)))[conf_a, conf_b]
                    c = cg(sb, mb, k, q, sa, ma)
                    if abs(c) < 1e-14:
                        if abs(v) > 1e-12:
                            raise AssertionError("site operator is not a tensor operator of this rank")
                        continue
                    r = v / c
                    if seen[a, b] and abs(red[a, b] - r) > 1e-12:
                        raise AssertionError("components disagree on the reduced element")
                    red[a, b], seen[a, b] = r, True
    return red


class Block:
    """Dense reduced operators of a block of consecutive orbitals (or of one site)."""

    def __init__(self, modes, outside, n, s):
        self.modes, self.outside = list(modes), list(outside)
        self.n, self.s = np.asarray(n, int), np.asarray(s, int)   # multiplet labels (n, 2S)
        self.dim = len(self.n)
        self.C, self.Dd, self.T = {}, {}, {}          # rank 1/2, odd
        self.A, self.B, self.DD = {}, {}, {}          # keys (2k, p, q), even
        self.H = np.zeros((self.dim, self.dim))
        self.I = np.eye(self.dim)

    def pair(self, kind):
        return {"A": self.A, "B": self.B, "DD": self.DD}[kind]


def vacuum_block(L):
    b = Block([], range(L), [0], [0])
    b.T = {m: np.zeros((1, 1)) for m in range(L)}
    return b


def site_block(p, h, V):
    """Exact reduced operators of orbital p as a one-site block."""
    L = h.shape[0]
    b = Block([p], [m for m in range(L) if m != p], SITE_N, SITE_S)
    c, d = site_c(), site_d()
    b.C[p] = site_reduced(c, 1)
    b.Dd[p] = site_reduced(d, 1)
    for k in (0, 2):
        b.A[(k, p, p)] = site_reduced(site_couple(c, 1, c, 1, k), k)
        b.B[(k, p, p)] = site_reduced(site_couple(c, 1, d, 1, k), k)
        b.DD[(k, p, p)] = site_reduced(site_couple(d, 1, d, 1, k), k)
    n = _CUP @ _CUP.T + _CDN @ _CDN.T
    for m in b.outside:
        # T_m = 1/2 h_mp d_p + (mp|pp) E_pp d_p
        comps = {q: 0.5 * h[m, p] * dq + V[m, p, p, p] * (n @ dq) for q, dq in d.items()}
        b.T[m] = site_reduced(comps, 1)
    Hs = h[p, p] * n + V[p, p, p, p] * (_CUP @ _CUP.T @ _CDN @ _CDN.T)
    b.H = site_reduced({0: Hs}, 0)
    return b


# ---------------------------------------------------------------------------
# coupled product bases and coupled products
# ---------------------------------------------------------------------------
class Product:
    """Coupled basis of two parts (part 1 first in the fermion order).

    Entries (i1, i2, 2J) for every multiplet pair and allowed total spin,
    ordered by label (n, 2J), then (block sector, site channel) for a left
    product or (site channel, block sector) for a right one, then the index of
    the block multiplet -- the row (column) order of the library's
    site-tensor import layout. `left`: part 1 is the block, part 2 the site;
    otherwise part 1 is the site.
    """

    def __init__(self, b1, b2, left):
        ent = []
        for i1 in range(b1.dim):
            for i2 in range(b2.dim):
                s1, s2 = b1.s[i1], b2.s[i2]
                for J in range(abs(s1 - s2), s1 + s2 + 1, 2):
                    ent.append((i1, i2, J))
        blk, site = (b1, b2) if left else (b2, b1)

        def key(e):
            i1, i2, J = e
            ib, isite = (i1, i2) if left else (i2, i1)
            n = b1.n[i1] + b2.n[i2]
            ch = channel(site.n[isite], blk.s[ib], J)
            if left:
                return ((n, J), (blk.n[ib], blk.s[ib]), ch, ib)
            return ((n, J), ch, (blk.n[ib], blk.s[ib]), ib)
        ent.sort(key=key)
        self.left = left
        self.i1 = np.array([e[0] for e in ent], int)
        self.i2 = np.array([e[1] for e in ent], int)
        self.J = np.array([e[2] for e in ent], int)
        self.s1, self.s2 = b1.s[self.i1], b2.s[self.i2]
        self.n = b1.n[self.i1] + b2.n[self.i2]
        self.n1 = b1.n[self.i1]
        self.s = self.J            # label (n, 2S) of every entry
        self.dim = len(ent)
        kinds = {}
        self.kid = np.array([kinds.setdefault((a, b, c), len(kinds))
                             for a, b, c in zip(self.s1, self.s2, self.J)], int)
        self.kinds = list(kinds)

    def cp(self, O1, k1, O2, k2, k, odd2):
        """Reduced matrix of [O1^k1 x O2^k2]^k (product O1 O2) on this basis."""
        F = np.zeros((len(self.kinds), len(self.kinds)))
        for a, (s1, s2, J) in enumerate(self.kinds):
            for b, (t1, t2, Jp) in enumerate(self.kinds):
                F[a, b] = coupled_factor(s1, s2, J, t1, t2, Jp, k1, k2, k)
        M = O1[np.ix_(self.i1, self.i1)] * O2[np.ix_(self.i2, self.i2)] * F[np.ix_(self.kid, self.kid)]
        if odd2:
            M = M * np.where(self.n1 % 2 == 0, 1.0, -1.0)[None, :]
        return M


def channel(nsite, two_s_block, two_J):
    """Site channel of a coupled pair: 0 |0>, 1 doublet up, 2 doublet down, 3 |2>."""
    if nsite == 0:
        return 0
    if nsite == 2:
        return 3
    return 1 if two_J == two_s_block + 1 else 2


# ---------------------------------------------------------------------------
# decomposition of H at a cut
# ---------------------------------------------------------------------------
def decomposition(Lb, Rb, V):
    """Scalar-coupling terms of H at the cut Lb|Rb, excluding H_L and H_R:
    list of (O_L, O_R, 2k, coefficient, odd(O_R), hermitian_conjugate_too)."""
    terms = []
    for p in Lb.modes:
        terms.append((Lb.C[p], Rb.T[p], 1, -R2, True, True))
    for m in Rb.modes:
        terms.append((Lb.T[m], Rb.C[m], 1, -R2, True, True))
    for k in (0, 2):
        kk = k // 2
        for p in Lb.modes:
            for r in Lb.modes:
                P = np.zeros((Rb.dim, Rb.dim))
                for s in Rb.modes:
                    for q in Rb.modes:
                        v = V[p, q, r, s]
                        if v:
                            P += v * Rb.DD[(k, s, q)]
                c = 0.5 * (-1) ** (1 + kk) * math.sqrt(2 * kk + 1)
                terms.append((Lb.A[(k, p, r)], P, k, c, False, True))
        for i in Lb.modes:
            for j in Lb.modes:
                Q = np.zeros((Rb.dim, Rb.dim))
                for kx in Rb.modes:
                    for l in Rb.modes:
                        if k == 0:
                            v = 2 * V[i, j, kx, l] - V[i, l, kx, j]
                        else:
                            v = math.sqrt(3.0) * V[i, l, kx, j]
                        if v:
                            Q += v * Rb.B[(k, kx, l)]
                terms.append((Lb.B[(k, i, j)], Q, k, 1.0, False, False))
    return terms


# ---------------------------------------------------------------------------
# enlargement: block (x) site (left) and site (x) block (right)
# ---------------------------------------------------------------------------
_OPS = {"c": "C", "d": "Dd"}
_PAIR = {("c", "c"): "A", ("c", "d"): "B", ("d", "d"): "DD"}


def _single(b, kind, p):
    return getattr(b, _OPS[kind])[p]


def _pair_op(b, k, kinds, p, q):
    return b.pair(_PAIR[kinds])[(k, p, q)]


def enlarge(X, S, h, V, left):
    """Operators of the enlarged block X (x) S (left) or S (x) X (right), S a one-site block."""
    b1, b2 = (X, S) if left else (S, X)
    pb = Product(b1, b2, left)
    o = S.modes[0]
    modes = sorted(X.modes + [o])
    outside = [m for m in X.outside if m != o]
    E = Block(modes, outside, pb.n, pb.J)
    E.prod = pb

    def cp(O1, k1, O2, k2, k, odd2):
        return pb.cp(O1, k1, O2, k2, k, odd2)

    def on(part, O, k, odd):
        """Operator of one part only (identity on the other)."""
        if (part == "X") == left:   # part 1
            return cp(O, k, b2.I, 0, k, False)
        return cp(b1.I, 0, O, k, k, odd)

    # single-mode normal operators
    for kind in ("c", "d"):
        dst = getattr(E, _OPS[kind])
        for p in X.modes:
            dst[p] = on("X", _single(X, kind, p), 1, True)
        dst[o] = on("S", _single(S, kind, o), 1, True)
    # pair operators [f1_p x f2_q]^k for p, q in X + o
    for kinds, name in _PAIR.items():
        dst = E.pair(name)
        for k in (0, 2):
            kk = k // 2
            for p in modes:
                for q in modes:
                    if p in X.modes and q in X.modes:
                        val = on("X", _pair_op(X, k, kinds, p, q), k, False)
                    elif p == o and q == o:
                        val = on("S", _pair_op(S, k, kinds, o, o), k, False)
                    else:
                        # one operator on each part; write the product with the
                        # part-1 operator first: [Y x Z]^k = (-1)^k [Z x Y]^k
                        # for two odd operators on different parts
                        f1 = (X if p in X.modes else S, kinds[0], p)
                        f2 = (X if q in X.modes else S, kinds[1], q)
                        first_is_1 = (f1[0] is b1)
                        a, b = (f1, f2) if first_is_1 else (f2, f1)
                        sgn = 1.0 if first_is_1 else (-1.0) ** kk
                        val = sgn * cp(_single(a[0], a[1], a[2]), 1, _single(b[0], b[1], b[2]), 1, k, True)
                    dst[(k, p, q)] = val
    # complementary T_m
    for m in outside:
        E.T[m] = on("X", X.T[m], 1, True) + on("S", S.T[m], 1, True) + _t_cross(X, S, V, m, left, pb)
    # Hamiltonian
    H = on("X", X.H, 0, False) + on("S", S.H, 0, False)
    for OL, OR, k, coef, odd, hc in decomposition(b1, b2, V):
        M = coef * cp(OL, k, OR, k, 0, odd)
        H += M + M.T if hc else M
    E.H = H
    return E


def _t_cross(X, S, V, m, left, pb):
    """Mixed part of T_m on the enlarged block: sum over (q, r, s) with some on X
    and some on the site o of (ms|qr) E_qr d_s = -sqrt(2) (ms|qr) [[c_q x d_r]^0 x d_s]^1/2.
    Each product is reordered so that the part-1 operators come first (the sign of
    the permutation of odd operators on different parts) and recoupled so that the
    two operators on one part form a rank-K composite."""
    o = S.modes[0]
    cp = pb.cp
    out = np.zeros((pb.dim, pb.dim))
    ops = ("c", "d", "d")
    js = (1, 1, 1)
    tree_in = ((0, 1, 0), 2)
    for pattern in range(1, 7):   # bit i set: operator i on the site
        on_site = [(pattern >> i) & 1 == 1 for i in range(3)]
        xi = [i for i in range(3) if not on_site[i]]
        si = [i for i in range(3) if on_site[i]]
        # product order after moving: part-1 operators first (relative order kept)
        order = (xi + si) if left else (si + xi)
        perm_sign = _perm_sign(order)
        # X indices to sum over
        nx = len(xi)
        xsets = [X.modes] * nx
        grids = np.meshgrid(*[np.array(s) for s in xsets], indexing="ij") if nx else []
        idx_lists = [g.reshape(-1) for g in grids]
        nterms = len(idx_lists[0]) if nx else 1
        # group the sum by the rank K of the two-operator composite
        part1_ops = xi if left else si
        for K in (0, 2):
            if len(part1_ops) == 2:
                tree_out = ((order[0], order[1], K), order[2])
            else:
                tree_out = (order[0], (order[1], order[2], K))
            w = recouple(js, tree_in, tree_out, 1)
            if abs(w) < 1e-15:
                continue
            acc_x = None
            for t in range(nterms):
                orb = [o, o, o]
                for j, i in enumerate(xi):
                    orb[i] = int(idx_lists[j][t])
                q, r, s = orb
                v = V[m, s, q, r]
                if v == 0.0:
                    continue
                # X-side factor: one operator or a rank-K composite of two
                if nx == 1:
                    ox = _single(X, ops[xi[0]], orb[xi[0]])
                else:
                    a, b = xi
                    ox = _pair_op(X, K, (ops[a], ops[b]), orb[a], orb[b])
                acc_x = v * ox if acc_x is None else acc_x + v * ox
            if acc_x is None:
                continue
            # site-side factor
            if len(si) == 1:
                os_ = _single(S, ops[si[0]], o)
                ks = 1
            else:
                a, b = si
                os_ = _pair_op(S, K, (ops[a], ops[b]), o, o)
                ks = K
            kx = 1 if nx == 1 else K
            coef = -R2 * perm_sign * w
            if left:
                out += coef * cp(acc_x, kx, os_, ks, 1, ks == 1)
            else:
                out += coef * cp(os_, ks, acc_x, kx, 1, kx == 1)
    return out


def _perm_sign(order):
    s = 1
    o = list(order)
    for i in range(len(o)):
        for j in range(i + 1, len(o)):
            if o[i] > o[j]:
                s = -s
    return s


def renormalize(E, U, left, bond):
    """O -> U^T O U (left, U: product x new) or V O V^T (right, V: new x product)."""
    g = (lambda O: U.T @ O @ U) if left else (lambda O: U @ O @ U.T)
    n = np.array([q[0] for q in bond.labels], int)
    s = np.array([q[1] for q in bond.labels], int)
    B = Block(E.modes, E.outside, n, s)
    for name in ("C", "Dd", "T", "A", "B", "DD"):
        getattr(B, name).update({k: g(v) for k, v in getattr(E, name).items()})
    B.H = g(E.H)
    return B


# ---------------------------------------------------------------------------
# SU(2) MPS around a two-site centre
# ---------------------------------------------------------------------------
CH_SHIFT = [(0, 0), (1, 1), (1, -1), (2, 0)]   # channel -> (dn, d2S) of the coupled label


class Labels:
    """Multiplet labels of a bond (sectors sorted, multiplets of a sector consecutive)."""

    def __init__(self, sectors):
        from .mpsu1 import Bond
        self.bond = Bond(dict(sectors))
        self.n, self.s, self.dim = self.bond.n, self.bond.s, self.bond.dim
        self.sectors = self.bond.sectors
        self.labels = self.bond.labels


SITE_LABELS = Labels({(0, 0): 1, (1, 1): 1, (2, 0): 1})


def _rows_of(pb, label):
    return np.nonzero((pb.n == label[0]) & (pb.J == label[1]))[0]


def _lift(pb, C, on_first):
    """Matrix C acting on the block part of a product basis (identity on the site)."""
    i_blk = pb.i1 if on_first else pb.i2
    i_site = pb.i2 if on_first else pb.i1
    same = (i_site[:, None] == i_site[None, :]) & (pb.J[:, None] == pb.J[None, :])
    return C[np.ix_(i_blk, i_blk)] * same


def allowed(sa, sb, two_s):
    return abs(sa - sb) <= two_s <= sa + sb


class MPSSU2:
    """Mixed-canonical SU(2) MPS around the two-site centre (l, l+1).

    lbonds[b] (b <= l) and rbonds[b] (b >= l+2) are Labels; A[p] (p < l) is the
    dense left-canonical tensor [product (bond p x site p) entries, bond p+1],
    R[p] (p > l+1) the right-canonical [bond p, product (site p x bond p+1)];
    psi is dense [product (bond l x site l), product (site l+1 x bond l+2)],
    zero outside the pairs that couple to (N, S).
    """

    def __init__(self, L, N, two_s, center, lbonds, rbonds, A, R, psi):
        self.L, self.N, self.two_s, self.center = L, N, two_s, center
        self.lbonds, self.rbonds, self.A, self.R, self.psi = lbonds, rbonds, A, R, psi

    def lprod(self):
        return Product(self.lbonds[self.center], SITE_LABELS, True)

    def rprod(self):
        return Product(SITE_LABELS, self.rbonds[self.center + 2], False)

    @classmethod
    def from_raw(cls, raw):
        """Canonical MPS from the raw random blocks of qcinputs (SU(2) keys):
        per-sector QR from the left, LQ from the right, carries into psi."""
        L, N, two_s, c = raw["L"], raw["N"], raw["two_s"], raw["center"]
        lb = {b: Labels(d) for b, d in raw["left_bonds"].items()}
        rb = {b: Labels(d) for b, d in raw["right_bonds"].items()}
        A, R = {}, {}
        carry = np.ones((1, 1))
        for p in range(c):
            pb = Product(lb[p], SITE_LABELS, True)
            M = np.zeros((pb.dim, lb[p + 1].dim))
            for (qL, si, qR), blk in raw["left"][p].items():
                rows = np.nonzero((lb[p].n[pb.i1] == qL[0]) & (lb[p].s[pb.i1] == qL[1]) &
                                  (pb.i2 == si) & (pb.J == qR[1]))[0]
                c0, dc = lb[p + 1].sectors[qR]
                M[np.ix_(rows, np.arange(c0, c0 + dc))] = blk
            M = _lift(pb, carry, True) @ M
            U = np.zeros_like(M)
            carry = np.zeros((lb[p + 1].dim, lb[p + 1].dim))
            for q, (c0, dc) in lb[p + 1].sectors.items():
                rows = _rows_of(pb, q)
                cols = np.arange(c0, c0 + dc)
                qm, rm = np.linalg.qr(M[np.ix_(rows, cols)])
                U[np.ix_(rows, cols)] = qm
                carry[np.ix_(cols, cols)] = rm
            A[p] = U
        cl = carry
        carry = np.ones((1, 1))
        for p in range(L - 1, c + 1, -1):
            pb = Product(SITE_LABELS, rb[p + 1], False)
            M = np.zeros((rb[p].dim, pb.dim))
            for (qn, si, qR), blk in raw["right"][p].items():
                cols = np.nonzero((rb[p + 1].n[pb.i2] == qR[0]) & (rb[p + 1].s[pb.i2] == qR[1]) &
                                  (pb.i1 == si) & (pb.J == qn[1]))[0]
                r0, dr = rb[p].sectors[qn]
                M[np.ix_(np.arange(r0, r0 + dr), cols)] = blk
            M = M @ _lift(pb, carry, False).T
            V = np.zeros_like(M)
            carry = np.zeros((rb[p].dim, rb[p].dim))
            for q, (r0, dr) in rb[p].sectors.items():
                cols = _rows_of(pb, q)
                rows = np.arange(r0, r0 + dr)
                qm, rm = np.linalg.qr(M[np.ix_(rows, cols)].T)
                V[np.ix_(rows, cols)] = qm.T
                carry[np.ix_(rows, rows)] = rm.T
            R[p] = V
        cr = carry
        m = cls(L, N, two_s, c, lb, rb, A, R, None)
        Lp, Rp = m.lprod(), m.rprod()
        psi = np.zeros((Lp.dim, Rp.dim))
        bX, bY = lb[c], rb[c + 2]
        for (qX, i, sL, j, qY, sR), blk in raw["psi"].items():
            rows = np.nonzero((bX.n[Lp.i1] == qX[0]) & (bX.s[Lp.i1] == qX[1]) & (Lp.i2 == i) & (Lp.J == sL))[0]
            cols = np.nonzero((bY.n[Rp.i2] == qY[0]) & (bY.s[Rp.i2] == qY[1]) & (Rp.i1 == j) & (Rp.J == sR))[0]
            psi[np.ix_(rows, cols)] = blk
        psi = _lift(Lp, cl, True) @ psi @ _lift(Rp, cr, False).T
        psi /= np.linalg.norm(psi)
        m.psi = psi
        return m

    # ---- flat layout of the two-site wavefunction (the library's order) ----
    def psi_blocks(self):
        """[(rows, cols)] of the sub-blocks (x, i, j, y) in the flat order: x a
        sector of bond l, i its site channel, j the channel of site l+1, y a
        sector of bond l+2, with the coupled labels fusing to (N, S)."""
        c = self.center
        bX, bY = self.lbonds[c], self.rbonds[c + 2]
        Lp, Rp = self.lprod(), self.rprod()
        lch = np.array([channel(SITE_LABELS.n[i], bX.s[x], J) for x, i, J in zip(Lp.i1, Lp.i2, Lp.J)])
        rch = np.array([channel(SITE_LABELS.n[j], bY.s[y], J) for j, y, J in zip(Rp.i1, Rp.i2, Rp.J)])
        out = []
        for qX in sorted(bX.sectors):
            for i in range(4):
                rows = np.nonzero((bX.n[Lp.i1] == qX[0]) & (bX.s[Lp.i1] == qX[1]) & (lch == i))[0]
                if len(rows) == 0:
                    continue
                na, sa = Lp.n[rows[0]], Lp.J[rows[0]]
                for j in range(4):
                    for qY in sorted(bY.sectors):
                        cols = np.nonzero((bY.n[Rp.i2] == qY[0]) & (bY.s[Rp.i2] == qY[1]) & (rch == j))[0]
                        if len(cols) == 0:
                            continue
                        nb, sb = Rp.n[cols[0]], Rp.J[cols[0]]
                        if na + nb == self.N and allowed(sa, sb, self.two_s):
                            out.append((rows, cols))
        return out

    def psi_to_flat(self, psi=None):
        psi = self.psi if psi is None else psi
        parts = [psi[np.ix_(r, c)].reshape(-1) for r, c in self.psi_blocks()]
        return np.concatenate(parts) if parts else np.zeros(0)

    def psi_from_flat(self, flat):
        psi = np.zeros((self.lprod().dim, self.rprod().dim))
        pos = 0
        for r, c in self.psi_blocks():
            psi[np.ix_(r, c)] = flat[pos:pos + len(r) * len(c)].reshape(len(r), len(c))
            pos += len(r) * len(c)
        if pos != len(flat):
            raise ValueError("flat vector has the wrong length")
        return psi

    def mask(self):
        Lp, Rp = self.lprod(), self.rprod()
        m = np.zeros((Lp.dim, Rp.dim), bool)
        for r, c in self.psi_blocks():
            m[np.ix_(r, c)] = True
        return m


def export_abi_su2(mps):
    """Flatten an SU(2) MPS into the C-ABI import layout: bonds as (n, 2S, dim)
    triples; left sites as U_q [product rows in (x, channel) order, dim_q],
    right sites as V_q [dim_q, product columns in (channel, y) order]; then psi."""
    L, c = mps.L, mps.center
    bonds = {b: mps.lbonds[b] for b in range(c + 1)}
    bonds.update({b: mps.rbonds[b] for b in range(c + 2, L + 1)})
    nsec, sec = [], []
    for b in range(L + 1):
        if b in bonds:
            items = sorted(bonds[b].sectors.items())
            nsec.append(len(items))
            for q, (st, d) in items:
                sec += [q[0], q[1], d]
        else:
            nsec.append(0)
    data = []
    for p in range(c):
        pb = Product(mps.lbonds[p], SITE_LABELS, True)
        for q, (c0, dc) in sorted(mps.lbonds[p + 1].sectors.items()):
            rows = _rows_of(pb, q)
            data.append(mps.A[p][np.ix_(rows, np.arange(c0, c0 + dc))].reshape(-1))
    for p in range(c + 2, L):
        pb = Product(SITE_LABELS, mps.rbonds[p + 1], False)
        for q, (r0, dr) in sorted(mps.rbonds[p].sectors.items()):
            cols = _rows_of(pb, q)
            data.append(mps.R[p][np.ix_(np.arange(r0, r0 + dr), cols)].reshape(-1))
    data.append(mps.psi_to_flat())
    return (np.array(nsec, dtype=np.int32), np.array(sec, dtype=np.int32),
            np.concatenate(data).astype(np.float64))


# ---------------------------------------------------------------------------
# H_eff at the centre
# ---------------------------------------------------------------------------
class Heff:
    """H_eff on psi[(L' entries), (R' entries)] from the enlarged blocks.

    A term c [O_L^k x O_R^k]^0 maps psi to
        sigma[a, b] = c F(a, b, a', b') O_L[a, a'] O_R[b, b'] (-1)^(p(O_R) n(a')) psi[a', b']
    with F the scalar-coupling factor of su2alg.coupled_factor at total spin S;
    its Hermitian conjugate is applied as the transpose of the same map.
    """

    def __init__(self, Lp, Rp, V, N, two_s, e_core=0.0):
        self.Lp, self.Rp = Lp, Rp
        self.terms = decomposition(Lp, Rp, V)
        self.e_core = e_core
        self.two_s = two_s
        pa, pb = Lp.prod, Rp.prod
        na, sa = Lp.n, Lp.s
        nb, sb = Rp.n, Rp.s
        self.mask_n = N
        self.mask = (na[:, None] + nb[None, :] == N) & \
            (np.abs(sa[:, None] - sb[None, :]) <= two_s) & (sa[:, None] + sb[None, :] >= two_s)
        self.sign = np.where(na % 2 == 0, 1.0, -1.0)
        self.lspins = {v: np.nonzero(sa == v)[0] for v in np.unique(sa)}
        self.rspins = {v: np.nonzero(sb == v)[0] for v in np.unique(sb)}
        self.shape = (Lp.dim, Rp.dim)

    def _apply_term(self, OL, OR, k, coef, odd, x, sig, transpose):
        S = self.two_s
        xs = x * self.sign[:, None] if (odd and not transpose) else x
        for sa, Ia in self.lspins.items():
            for sap, Iap in self.lspins.items():
                OLb = OL[np.ix_(Ia, Iap)]
                if not OLb.any():
                    continue
                for sb, Ib in self.rspins.items():
                    if not allowed(sa, sb, S):
                        continue
                    for sbp, Ibp in self.rspins.items():
                        if not allowed(sap, sbp, S):
                            continue
                        f = coupled_factor(sa, sb, S, sap, sbp, S, k, k, 0)
                        if f == 0.0:
                            continue
                        ORb = OR[np.ix_(Ib, Ibp)]
                        if not ORb.any():
                            continue
                        if not transpose:
                            sig[np.ix_(Ia, Ib)] += coef * f * (OLb @ xs[np.ix_(Iap, Ibp)] @ ORb.T)
                        else:
                            t = coef * f * (OLb.T @ x[np.ix_(Ia, Ib)] @ ORb)
                            if odd:
                                t = t * self.sign[Iap][:, None]
                            sig[np.ix_(Iap, Ibp)] += t

    def algorithmic_flops(self):
        """Flops of one H_eff psi counted per quantum-number sector: for every term
        and every pair of nonzero (n, 2S) sector blocks of O_L and O_R that meet a
        psi block, 2 d_a' d_b' d_b (psi O_R^T) + 2 d_a d_a' d_b (O_L times that);
        the Hermitian conjugates and the block Hamiltonians counted the same way."""
        def sectors(n, s):
            labs = sorted(set(zip(n.tolist(), s.tolist())))
            ind = np.zeros((len(labs), len(n)))
            for k, lab in enumerate(labs):
                ind[k, (n == lab[0]) & (s == lab[1])] = 1.0
            return labs, ind, ind.sum(axis=1)
        la, Ia, da = sectors(self.Lp.n, self.Lp.s)
        lb, Ib, db = sectors(self.Rp.n, self.Rp.s)
        allow = np.array([[1.0 if (a[0] + b[0] == self.mask_n and allowed(a[1], b[1], self.two_s)) else 0.0
                           for b in lb] for a in la])

        def nz(O, ind):
            return (ind @ (np.abs(O) > 0) @ ind.T) > 0

        def count(nzl, nzr):
            # stage 1: X[a', b] = sum_b' allow[a', b'] nzr[b, b'] d_b' d_b
            X = (allow * db[None, :]) @ (nzr.T * db[None, :])
            s1 = float(np.sum((nzl * da[None, :]) @ X * allow))
            # stage 2: sum over (a, a', b) of 2 d_a d_a' d_b where the stage-1 output exists
            Y = allow @ nzr.T                       # [a', b]: some b' reaches b
            s2 = float(np.sum(((nzl * (da[:, None] * da[None, :])) @ ((Y > 0) * db[None, :])) * allow))
            return 2.0 * (s1 + s2)
        tot = 0.0
        idL, idR = np.eye(len(la)) > 0, np.eye(len(lb)) > 0
        tot += count(nz(self.Lp.H, Ia), idR) + count(idL, nz(self.Rp.H, Ib))
        for OL, OR, k, coef, odd, hc in self.terms:
            f = count(nz(OL, Ia), nz(OR, Ib))
            tot += 2 * f if hc else f
        return tot

    def apply_mat(self, x):
        x = x * self.mask
        sig = self.Lp.H @ x + x @ self.Rp.H.T + self.e_core * x
        for OL, OR, k, coef, odd, hc in self.terms:
            self._apply_term(OL, OR, k, coef, odd, x, sig, False)
            if hc:
                self._apply_term(OL, OR, k, coef, odd, x, sig, True)
        return sig * self.mask


def lowest_eig(heff, guess, tol=1e-12):
    """Lanczos (ARPACK) on the masked H_eff: ground state of the two-site problem."""
    sel = heff.mask.reshape(-1)
    nsel = int(sel.sum())

    def mv(v):
        full = np.zeros(sel.shape[0])
        full[sel] = v
        return heff.apply_mat(full.reshape(heff.shape)).reshape(-1)[sel]
    v0 = guess.reshape(-1)[sel]
    if np.linalg.norm(v0) == 0:
        v0 = np.ones(nsel)
    if nsel <= 64:
        M = np.column_stack([mv(np.eye(nsel)[:, k]) for k in range(nsel)])
        wv, vv = np.linalg.eigh(0.5 * (M + M.T))
    else:
        op = spla.LinearOperator((nsel, nsel), matvec=mv, dtype=float)
        wv, vv = spla.eigsh(op, k=1, which="SA", v0=v0, tol=tol)
    full = np.zeros(sel.shape[0])
    full[sel] = vv[:, 0]
    return float(wv[0]), full.reshape(heff.shape)


# ---------------------------------------------------------------------------
# truncation and centre moves
# ---------------------------------------------------------------------------
def svd_left(x, Lp, Rp, mask):
    """Per L' sector q: SVD of psi[rows of q, every R' column coupled with q]."""
    blocks = {}
    for q in sorted(set(zip(Lp.n.tolist(), Lp.s.tolist()))):
        rows = np.nonzero((Lp.n == q[0]) & (Lp.s == q[1]))[0]
        cols = np.nonzero(mask[rows[0]])[0]
        if len(cols) == 0:
            continue
        u, sv, vt = np.linalg.svd(x[np.ix_(rows, cols)], full_matrices=False)
        blocks[q] = (rows, cols, u, sv, vt)
    return blocks


def svd_right(x, Lp, Rp, mask):
    """Per R' sector r: SVD of psi[every L' row coupled with r, columns of r]."""
    blocks = {}
    for r in sorted(set(zip(Rp.n.tolist(), Rp.s.tolist()))):
        cols = np.nonzero((Rp.n == r[0]) & (Rp.s == r[1]))[0]
        rows = np.nonzero(mask[:, cols[0]])[0]
        if len(rows) == 0:
            continue
        u, sv, vt = np.linalg.svd(x[np.ix_(rows, cols)], full_matrices=False)
        blocks[r] = (rows, cols, u, sv, vt)
    return blocks


def recouple_right_move(Lnew, pb_old_R, Rt, SV, two_s, rbond_y):
    """psi'' [(a s1) Ja, (s2 y') Jb] from SV[a, (s1 y) Jold] and R_{l+2}[y, (s2 y') Jb]:
    |a, (s1 y) Jold; S> = sum_Ja <(a s1) Ja, y; S | a, (s1 y) Jold; S> |(a s1) Ja, y; S>."""
    Tm = np.zeros((Lnew.dim, rbond_y.dim))
    for e1 in range(Lnew.dim):
        a, s1, Ja = Lnew.i1[e1], Lnew.i2[e1], Lnew.J[e1]
        sa_ = Lnew.s1[e1]
        for eo in np.nonzero(pb_old_R.i1 == s1)[0]:
            y, Jold = pb_old_R.i2[eo], pb_old_R.J[eo]
            v = SV[a, eo]
            if v == 0.0:
                continue
            js = (int(sa_), int(SITE_LABELS.s[s1]), int(rbond_y.s[y]))
            w = recouple(js, (0, (1, 2, int(Jold))), ((0, 1, int(Ja)), 2), two_s)
            Tm[e1, y] += w * v
    return Tm @ Rt


def recouple_left_move(At, US, pb_old_L, Rnew, two_s, lbond_x):
    """psi'' [(x' s0) Jx, (s1 b') Jb] from A_{l-1}[(x' s0) Jx, x] and US[(x s1) Ja, b']:
    |(x s1) Ja, b'; S> = sum_Jb <x, (s1 b') Jb; S | (x s1) Ja, b'; S> |x, (s1 b') Jb; S>."""
    Tm = np.zeros((lbond_x.dim, Rnew.dim))
    for e2 in range(Rnew.dim):
        s1, b, Jb = Rnew.i1[e2], Rnew.i2[e2], Rnew.J[e2]
        sb_ = Rnew.s2[e2]
        for eo in np.nonzero(pb_old_L.i2 == s1)[0]:
            x, Ja = pb_old_L.i1[eo], pb_old_L.J[eo]
            v = US[eo, b]
            if v == 0.0:
                continue
            js = (int(lbond_x.s[x]), int(SITE_LABELS.s[s1]), int(sb_))
            w = recouple(js, ((0, 1, int(Ja)), 2), (0, (1, 2, int(Jb))), two_s)
            Tm[x, e2] += w * v
    return At @ Tm


class DMRGSU2:
    """Plain spin-adapted two-site DMRG driver (oracle)."""

    def __init__(self, h, V, N, two_s, e_core=0.0):
        self.h, self.V = np.asarray(h, float), np.asarray(V, float)
        self.L = self.h.shape[0]
        self.N, self.two_s, self.e_core = N, two_s, e_core
        self.sites = [site_block(p, self.h, self.V) for p in range(self.L)]

    def left_block(self, mps, upto):
        blk = vacuum_block(self.L)
        for p in range(upto):
            E = enlarge(blk, self.sites[p], self.h, self.V, True)
            blk = renormalize(E, mps.A[p], True, mps.lbonds[p + 1])
        return blk

    def right_block(self, mps, frm):
        blk = vacuum_block(self.L)
        for p in range(self.L - 1, frm - 1, -1):
            E = enlarge(blk, self.sites[p], self.h, self.V, False)
            blk = renormalize(E, mps.R[p], False, mps.rbonds[p])
        return blk

    def heff_at_center(self, mps):
        l = mps.center
        Lp = enlarge(self.left_block(mps, l), self.sites[l], self.h, self.V, True)
        Rp = enlarge(self.right_block(mps, l + 2), self.sites[l + 1], self.h, self.V, False)
        return Heff(Lp, Rp, self.V, self.N, self.two_s, self.e_core)

    def sigma(self, mps, psi=None):
        heff = self.heff_at_center(mps)
        return heff.apply_mat(mps.psi if psi is None else psi)

    def _factor_left(self, blocks, kept, Lp, Rp):
        lab = {q: len(ks) for q, ks in kept.items()}
        bnew = Labels(lab)
        U = np.zeros((Lp.dim, bnew.dim))
        SV = np.zeros((bnew.dim, Rp.dim))
        for q, ks in kept.items():
            rows, cols, u, sv, vt = blocks[q]
            st, dq = bnew.sectors[q]
            r = np.arange(st, st + dq)
            U[np.ix_(rows, r)] = u[:, ks]
            SV[np.ix_(r, cols)] = sv[ks][:, None] * vt[ks]
        return bnew, U, SV

    def _factor_right(self, blocks, kept, Lp, Rp):
        lab = {q: len(ks) for q, ks in kept.items()}
        bnew = Labels(lab)
        Vt = np.zeros((bnew.dim, Rp.dim))
        US = np.zeros((Lp.dim, bnew.dim))
        for q, ks in kept.items():
            rows, cols, u, sv, vt = blocks[q]
            st, dq = bnew.sectors[q]
            rr = np.arange(st, st + dq)
            Vt[np.ix_(rr, cols)] = vt[ks]
            US[np.ix_(rows, rr)] = u[:, ks] * sv[ks][None, :]
        return bnew, Vt, US

    def move_center_left(self, mps, target):
        """Shift the two-site centre left by exact (untruncated) SVDs."""
        from .dmrgu1 import select_kept
        A, R = dict(mps.A), dict(mps.R)
        lb, rb = dict(mps.lbonds), dict(mps.rbonds)
        psi = mps.psi
        l = mps.center
        while l > target:
            cur = MPSSU2(self.L, self.N, self.two_s, l, lb, rb, A, R, psi)
            Lp, Rp = cur.lprod(), cur.rprod()
            blocks = svd_right(psi, Lp, Rp, cur.mask())
            kept, _ = select_kept(blocks, 10 ** 9)
            bnew, Vt, US = self._factor_right(blocks, kept, Lp, Rp)
            R[l + 1] = Vt
            rb[l + 1] = bnew
            Rnew = Product(SITE_LABELS, bnew, False)
            psi = recouple_left_move(A.pop(l - 1), US, Lp, Rnew, self.two_s, lb[l])
            del lb[l]
            l -= 1
        return MPSSU2(self.L, self.N, self.two_s, l, lb, rb, A, R, psi)

    def sweeps(self, mps, D, nsweeps=1, tol=1e-12, trunc_eps=0.0, D_min=1):
        """Full sweeps at bond dimension D (SU(2) multiplets); as the U(1)
        oracle: the centre starts at 0, each sweep optimises centres 0..L-3
        moving right and L-2..1 moving left and ends at 0. Returns (energies,
        max discarded weights, final MPS). trunc_eps > 0: dynamic block-state
        selection in [D_min, D] (dmrgu1.dbss_bond_dimension on the multiplet
        weights); self.max_kept and self.total_kept are the largest and the summed
        numbers of multiplets kept."""
        from .dmrgu1 import select_kept, dbss_bond_dimension
        self.max_kept = 0
        self.total_kept = 0

        def choose(blocks):
            Dk = dbss_bond_dimension(blocks, trunc_eps, D_min, D) if trunc_eps > 0 else D
            kept, disc = select_kept(blocks, Dk)
            self.max_kept = max(self.max_kept, sum(len(v) for v in kept.values()))
            self.total_kept += sum(len(v) for v in kept.values())
            return kept, disc
        L = self.L
        mps = self.move_center_left(mps, 0)
        A, R = dict(mps.A), dict(mps.R)
        lb, rb = dict(mps.lbonds), dict(mps.rbonds)
        lblocks = {0: vacuum_block(L)}
        rblocks = {L: vacuum_block(L)}
        for p in range(L - 1, 1, -1):
            E = enlarge(rblocks[p + 1], self.sites[p], self.h, self.V, False)
            rblocks[p] = renormalize(E, R[p], False, rb[p])
        psi = mps.psi
        energies, terrs = [], []
        for _ in range(nsweeps):
            maxerr, En = 0.0, None
            order = [(l, +1) for l in range(0, L - 2)] + [(l, -1) for l in range(L - 2, 0, -1)]
            for l, d in order:
                Lp = enlarge(lblocks[l], self.sites[l], self.h, self.V, True)
                Rp = enlarge(rblocks[l + 2], self.sites[l + 1], self.h, self.V, False)
                heff = Heff(Lp, Rp, self.V, self.N, self.two_s, self.e_core)
                En, x = lowest_eig(heff, psi, tol=tol)
                if d > 0:
                    blocks = svd_left(x, Lp.prod, Rp.prod, heff.mask)
                    kept, disc = choose(blocks)
                    bnew, U, SV = self._factor_left(blocks, kept, Lp, Rp)
                    A[l] = U
                    lb[l + 1] = bnew
                    lblocks[l + 1] = renormalize(Lp, U, True, bnew)
                    Lnew = Product(bnew, SITE_LABELS, True)
                    psi = recouple_right_move(Lnew, Rp.prod, R.pop(l + 2), SV, self.two_s, rb[l + 2])
                else:
                    blocks = svd_right(x, Lp.prod, Rp.prod, heff.mask)
                    kept, disc = choose(blocks)
                    bnew, Vt, US = self._factor_right(blocks, kept, Lp, Rp)
                    R[l + 1] = Vt
                    rb[l + 1] = bnew
                    rblocks[l + 1] = renormalize(Rp, Vt, False, bnew)
                    Rnew = Product(SITE_LABELS, bnew, False)
                    psi = recouple_left_move(A.pop(l - 1), US, Lp.prod, Rnew, self.two_s, lb[l])
                maxerr = max(maxerr, disc)
            energies.append(En)
            terrs.append(maxerr)
        out = MPSSU2(L, self.N, self.two_s, 0, {0: lb[0]}, {b: rb[b] for b in range(2, L + 1)},
                     {}, {p: R[p] for p in range(2, L)}, psi)
        return energies, terrs, out
