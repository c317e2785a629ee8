"""SU(2) angular-momentum algebra for the spin-adapted oracle (FP64, plain).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

All angular momenta are passed doubled (two_j = 2j) so that half-integers are
integers. Conventions (the paper states none; these readings are fixed here):
  * Clebsch-Gordan coefficients <j1 m1; j2 m2 | J M> in the Condon-Shortley
    phase convention, from the Racah formula;
  * Wigner-Eckart theorem with the reduced matrix element defined by
        <j m | T^k_q | j' m'> = <j' m'; k q | j m> <j || T^k || j'>;
  * 6j symbols from the Racah formula, 9j symbols as the sum over one 6j
    product (the standard expansion in the 6j symbols).

coupled_factor gives the reduced matrix element of a tensor product of two
operators acting on two subsystems (subsystem 1 first in the fermion order),
    X^k_q = [T^{k1}(1) x U^{k2}(2)]^k_q = sum <k1 q1; k2 q2|k q> T_q1 U_q2,
between coupled states |(j1 j2) J> and |(j1' j2') J'>, as a multiple of
<j1||T||j1'> <j2||U||j2'> (fermion signs are applied by the caller). Two
forms are provided: the plain definition (a sum of Clebsch-Gordan products,
coupled_factor_def) and the closed form with the 9j symbol (coupled_factor);
the tests pin one against the other.

recouple gives the overlap of two coupling orders of three angular momenta
(the plain Clebsch-Gordan sum); operator products of three tensor operators
recouple with the same coefficients.
"""

import math
from fractions import Fraction
from functools import lru_cache


def _f(n):
    return math.factorial(n)


def _tri(a, b, c):
    """Doubled triangle condition (a, b, c doubled): |a-b| <= c <= a+b, a+b+c even."""
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0


def _delta_sq(a, b, c):
    """Squared triangle coefficient Delta(abc)^2 as a Fraction (doubled args)."""
    return Fraction(_f((a + b - c) // 2) * _f((a - b + c) // 2) * _f((-a + b + c) // 2),
                    _f((a + b + c) // 2 + 1))


@lru_cache(maxsize=None)
def cg(two_j1, two_m1, two_j2, two_m2, two_J, two_M):
    """<j1 m1; j2 m2 | J M> (Racah formula, Condon-Shortley phases)."""
    j1, m1, j2, m2, J, M = two_j1, two_m1, two_j2, two_m2, two_J, two_M
    if m1 + m2 != M or not _tri(j1, j2, J):
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    if (j1 + m1) % 2 or (j2 + m2) % 2 or (J + M) % 2:
        return 0.0
    pre = Fraction((J + 1) * _f((J + j1 - j2) // 2) * _f((J - j1 + j2) // 2) * _f((j1 + j2 - J) // 2),
                   _f((j1 + j2 + J) // 2 + 1))
    pre *= Fraction(_f((J + M) // 2) * _f((J - M) // 2) * _f((j1 - m1) // 2) * _f((j1 + m1) // 2) *
                    _f((j2 - m2) // 2) * _f((j2 + m2) // 2))
    s = Fraction(0)
    for k in range(0, j1 + j2 + 1):
        a = [k, (j1 + j2 - J) // 2 - k, (j1 - m1) // 2 - k, (j2 + m2) // 2 - k,
             (J - j2 + m1) // 2 + k, (J - j1 - m2) // 2 + k]
        if min(a) < 0:
            continue
        den = 1
        for x in a:
            den *= _f(x)
        s += Fraction((-1) ** k, den)
    return float(s) * math.sqrt(float(pre)) if s >= 0 else -float(-s) * math.sqrt(float(pre))


@lru_cache(maxsize=None)
def sixj(a, b, c, d, e, f):
    """Wigner 6j symbol {a b c; d e f} (doubled arguments), Racah formula."""
    for t in ((a, b, c), (a, e, f), (d, b, f), (d, e, c)):
        if not _tri(*t):
            return 0.0
    tri = _delta_sq(a, b, c) * _delta_sq(a, e, f) * _delta_sq(d, b, f) * _delta_sq(d, e, c)
    s = Fraction(0)
    t_lo = max((a + b + c) // 2, (a + e + f) // 2, (d + b + f) // 2, (d + e + c) // 2)
    t_hi = min((a + b + d + e) // 2, (a + c + d + f) // 2, (b + c + e + f) // 2)
    for t in range(t_lo, t_hi + 1):
        den = (_f(t - (a + b + c) // 2) * _f(t - (a + e + f) // 2) * _f(t - (d + b + f) // 2) *
               _f(t - (d + e + c) // 2) * _f((a + b + d + e) // 2 - t) * _f((a + c + d + f) // 2 - t) *
               _f((b + c + e + f) // 2 - t))
        s += Fraction((-1) ** t * _f(t + 1), den)
    v = float(s) * math.sqrt(float(tri))
    return v


@lru_cache(maxsize=None)
def ninej(a, b, c, d, e, f, g, h, i):
    """Wigner 9j symbol {a b c; d e f; g h i} (doubled arguments):
    sum_x (-1)^(2x) (2x+1) {a b c; f i x} {d e f; b x h} {g h i; x a d}."""
    lo = max(abs(a - i), abs(d - h), abs(b - f))
    hi = min(a + i, d + h, b + f)
    s = 0.0
    for x in range(lo, hi + 1, 2):
        s += (x + 1) * sixj(a, b, c, f, i, x) * sixj(d, e, f, b, x, h) * sixj(g, h, i, x, a, d)
    # (-1)^(2x): x is doubled, 2x -> x
    return s if lo % 2 == 0 else -s


def reduced_from_components(two_j, two_m, two_jp, two_mp, two_k, two_q, value):
    """<j||T^k||j'> from one matrix element <j m|T^k_q|j' m'> (Wigner-Eckart)."""
    c = cg(two_jp, two_mp, two_k, two_q, two_j, two_m)
    return value / c


@lru_cache(maxsize=None)
def coupled_factor_def(j1, j2, J, j1p, j2p, Jp, k1, k2, k):
    """Plain definition (sum of CG products) of
    <(j1 j2)J || [T^k1 x U^k2]^k || (j1' j2')J'> / (<j1||T||j1'> <j2||U||j2'>), doubled args."""
    if not (_tri(j1, j2, J) and _tri(j1p, j2p, Jp) and _tri(k1, k2, k) and _tri(Jp, k, J)):
        return 0.0
    if not (_tri(j1p, k1, j1) and _tri(j2p, k2, j2)):
        return 0.0
    # pick M, M', q with a nonzero <J' M'; k q | J M>
    for M in range(-J, J + 1, 2):
        for Mp in range(-Jp, Jp + 1, 2):
            q = M - Mp
            if abs(q) > k:
                continue
            den = cg(Jp, Mp, k, q, J, M)
            if abs(den) < 1e-12:
                continue
            s = 0.0
            for m1 in range(-j1, j1 + 1, 2):
                m2 = M - m1
                if abs(m2) > j2:
                    continue
                c1 = cg(j1, m1, j2, m2, J, M)
                if c1 == 0.0:
                    continue
                for m1p in range(-j1p, j1p + 1, 2):
                    m2p = Mp - m1p
                    if abs(m2p) > j2p:
                        continue
                    c2 = cg(j1p, m1p, j2p, m2p, Jp, Mp)
                    if c2 == 0.0:
                        continue
                    q1, q2 = m1 - m1p, m2 - m2p
                    if abs(q1) > k1 or abs(q2) > k2:
                        continue
                    c3 = cg(k1, q1, k2, q2, k, q)
                    if c3 == 0.0:
                        continue
                    # <j1 m1|T_q1|j1' m1'> = <j1' m1'; k1 q1|j1 m1> <j1||T||j1'>, same for U
                    s += c1 * c2 * c3 * cg(j1p, m1p, k1, q1, j1, m1) * cg(j2p, m2p, k2, q2, j2, m2)
            return s / den
    return 0.0


@lru_cache(maxsize=None)
def coupled_factor(j1, j2, J, j1p, j2p, Jp, k1, k2, k):
    """Closed form of coupled_factor_def with the 9j symbol (doubled args):
    sqrt((2J'+1)(2k+1)(2j1+1)(2j2+1)) {j1 j1' k1; j2 j2' k2; J J' k}."""
    if not (_tri(j1p, k1, j1) and _tri(j2p, k2, j2) and _tri(Jp, k, J)):
        return 0.0
    return math.sqrt((Jp + 1) * (k + 1) * (j1 + 1) * (j2 + 1)) * ninej(j1, j1p, k1, j2, j2p, k2, J, Jp, k)


@lru_cache(maxsize=None)
def recouple(js, tree_in, tree_out, J):
    """Overlap <tree_out; J M | tree_in; J M> of two coupling orders of three
    angular momenta js = (j1, j2, j3) (doubled), each tree given as
    ((a, b, Jab), c) for ((a b)Jab, c) or (a, (b, c, Jbc)) for (a, (b c)Jbc)
    with a, b, c indices 0..2 into js. Plain sum of Clebsch-Gordan products
    at M = J (the overlap does not depend on M)."""
    M = J

    def amp(tree, ms):
        if isinstance(tree[0], tuple):
            (a, b, Jab), c = tree
            s = 0.0
            Mab = ms[a] + ms[b]
            if abs(Mab) > Jab:
                return 0.0
            return cg(js[a], ms[a], js[b], ms[b], Jab, Mab) * cg(Jab, Mab, js[c], ms[c], J, M)
        a, (b, c, Jbc) = tree
        Mbc = ms[b] + ms[c]
        if abs(Mbc) > Jbc:
            return 0.0
        return cg(js[b], ms[b], js[c], ms[c], Jbc, Mbc) * cg(js[a], ms[a], Jbc, Mbc, J, M)

    s = 0.0
    for m0 in range(-js[0], js[0] + 1, 2):
        for m1 in range(-js[1], js[1] + 1, 2):
            m2 = M - m0 - m1
            if abs(m2) > js[2] or (js[2] - m2) % 2:
                continue
            ms = (m0, m1, m2)
            s += amp(tree_in, ms) * amp(tree_out, ms)
    return s


def adjoint_factor(two_jr, two_jc, two_k):
    """<j'||T~||j> / <j||T||j'> for the adjoint tensor T~_q = (-1)^(k-q) (T_-q)^+,
    with j the bra (row) and j' the ket (column) of T: (-1)^(j+k-j') sqrt((2j+1)/(2j'+1))."""
    e = (two_jr + two_k - two_jc) // 2
    return (-1) ** e * math.sqrt((two_jr + 1) / (two_jc + 1))
