"""Configuration spaces of the warm-up sweep (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The paper converges its runs with an SU(2)-aware dynamically extended active space
procedure (DEAS; Numerical benchmark section), whose warm-up sweep draws its environment
from a small configuration space. The plain definitions used to check the library's
configuration selection and configuration MPS:

* a configuration is a step vector over the orbitals in chain order: for determinants
  0 = |0>, 1 = a+_up|0>, 2 = a+_dn|0>, 3 = a+_up a+_dn|0> and the determinant is
  prod_k (a+_k)^{n_k}|vac> (k = 2p + sigma increasing, the FCI oracle's basis); for spin
  states 0 = empty, 3 = doubly occupied, and on a singly occupied orbital 1 / 2 couple the
  spin of the orbitals before it to S_prev + 1/2 / S_prev - 1/2 (a configuration state
  function in the genealogical coupling), expanded to determinants with Clebsch-Gordan
  coefficients at M = S;
* the aufbau reference fills the orbitals of lowest h_pp (ties by index): (N + 2Sz)/2 up
  and (N - 2Sz)/2 down electrons, or, for spin states, (N - 2S)/2 doubly occupied orbitals
  and the next 2S singly occupied with every step up;
* the candidates are the configurations at most two electrons away from it (electrons
  moved: the number of spin-orbitals (orbitals, counted with multiplicity) the reference
  occupies and the configuration does not);
* their energy is the diagonal element <D|H|D> of the FCI matrix for a determinant, and
  for a spatial occupation the mean of those diagonal elements over every determinant of
  that occupation (all spin assignments, every Sz), shared by all of its couplings;
* the selection is the nmax lowest by (energy, electrons moved, step vector).

Written by enumerating the whole determinant space (small L only); numpy, scipy.
"""
import itertools

import numpy as np

from oracle.fci import FCI, DetSpace
from oracle.su2alg import cg


def det_bits(steps):
    """Bit string of a determinant step vector (bit 2p up, bit 2p + 1 down)."""
    b = 0
    for p, s in enumerate(steps):
        if s in (1, 3):
            b |= 1 << (2 * p)
        if s in (2, 3):
            b |= 1 << (2 * p + 1)
    return b


def csf_components(steps):
    """{determinant bits: coefficient} of a genealogical spin state at M = S."""
    # states[M2] = {bits: coefficient} of the coupled state so far with 2M = M2
    states = {0: {0: 1.0}}
    two_s = 0
    for p, s in enumerate(steps):
        if s == 0:
            continue
        if s == 3:
            states = {m: {b | (3 << (2 * p)): c for b, c in d.items()} for m, d in states.items()}
            continue
        new_s = two_s + (1 if s == 1 else -1)
        if new_s < 0:
            raise ValueError("spin below zero")
        new = {}
        for M2 in range(-new_s, new_s + 1, 2):
            out = {}
            for m in (1, -1):                  # electron spin up / down
                Mp = M2 - m
                if abs(Mp) > two_s or Mp not in states:
                    continue
                w = cg(two_s, Mp, 1, m, new_s, M2)
                if w == 0.0:
                    continue
                bit = 1 << (2 * p + (0 if m == 1 else 1))
                for b, c in states[Mp].items():
                    out[b | bit] = out.get(b | bit, 0.0) + w * c
            new[M2] = out
        states, two_s = new, new_s
    return states[two_s]


def config_vector(configs, coef, L, N, two_s, su2):
    """sum_k coef[k] |config_k> in DetSpace(L, N, two_s) (M = S for spin states)."""
    space = DetSpace(L, N, two_s)
    v = np.zeros(space.dim)
    for st, c in zip(configs, coef):
        comps = csf_components(st) if su2 else {det_bits(st): 1.0}
        for b, w in comps.items():
            idx, ok = space.index(np.uint64(b))
            assert ok, "configuration outside the target space"
            v[int(idx)] += c * w
    return space, v


def _aufbau(h, N, two_s, su2):
    L = h.shape[0]
    order = sorted(range(L), key=lambda p: (h[p, p], p))
    if su2:
        n = np.zeros(L, int)
        nd = (N - two_s) // 2
        for p in order[:nd]:
            n[p] = 2
        for p in order[nd:nd + two_s]:
            n[p] = 1
        return n
    na, nb = (N + two_s) // 2, (N - two_s) // 2
    bits = 0
    for p in order[:na]:
        bits |= 1 << (2 * p)
    for p in order[:nb]:
        bits |= 1 << (2 * p + 1)
    return bits


def _steps_of(bits, L):
    return tuple(((bits >> (2 * p)) & 1) + 2 * ((bits >> (2 * p + 1)) & 1) for p in range(L))


def candidates_u1(h, V, N, two_s):
    """[(energy, electrons moved, steps)] of every determinant within two of the reference."""
    L = h.shape[0]
    f = FCI(h, V, N, two_s)
    diag = f.matrix().diagonal()
    ref = _aufbau(h, N, two_s, False)
    out = []
    for b, e in zip(f.space.dets, diag):
        moved = bin(ref & ~int(b)).count("1")
        if moved <= 2:
            out.append((float(e), moved, _steps_of(int(b), L)))
    return out


def couplings(n, two_s):
    """Every genealogical step vector of the spatial occupation n with final spin two_s."""
    L = len(n)
    open_ = [p for p in range(L) if n[p] == 1]
    base = [3 if n[p] == 2 else 0 for p in range(L)]
    out = []
    for seq in itertools.product((1, 2), repeat=len(open_)):
        s, ok = 0, True
        for x in seq:
            s += 1 if x == 1 else -1
            if s < 0:
                ok = False
                break
        if ok and s == two_s:
            st = list(base)
            for p, x in zip(open_, seq):
                st[p] = x
            out.append(tuple(st))
    return out


def candidates_su2(h, V, N, two_s):
    """[(energy, electrons moved, steps)] of every coupling of every spatial occupation within
    two electrons of the reference; energy = mean FCI diagonal over the occupation's
    determinants."""
    L = h.shape[0]
    diag = {}
    for tz in range(-N, N + 1, 2):
        try:
            f = FCI(h, V, N, tz)
        except ValueError:
            continue
        for b, e in zip(f.space.dets, f.matrix().diagonal()):
            diag[int(b)] = float(e)
    ref = _aufbau(h, N, two_s, True)
    sums = {}
    for b, e in diag.items():
        n = tuple(((b >> (2 * p)) & 1) + ((b >> (2 * p + 1)) & 1) for p in range(L))
        s = sums.setdefault(n, [0.0, 0])
        s[0] += e
        s[1] += 1
    out = []
    for n, (tot, cnt) in sums.items():
        moved = int(sum(max(0, ref[p] - n[p]) for p in range(L)))
        if moved > 2:
            continue
        for st in couplings(n, two_s):
            out.append((tot / cnt, moved, st))
    return out


def select_configs(h, V, N, two_s, nmax, su2):
    """The nmax lowest candidates by (energy, electrons moved, step vector)."""
    cands = candidates_su2(h, V, N, two_s) if su2 else candidates_u1(h, V, N, two_s)
    cands.sort()
    return cands[:nmax], cands
