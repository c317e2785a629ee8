"""Pins of the operator-based SU(2) oracle (oracle/su2alg.py, oracle/dmrgsu2.py).

* 6j and 9j symbols (Racah formula) against tabulated special values, the
  orthogonality sums of the 6j symbols and the 9j symbols of the
  independent-coupling expansion; Clebsch-Gordan closed forms.
* The 9j closed form of a coupled product against its plain definition.
* Single-site reduced operators: every M component of c, d and the pair
  operators agrees with one reduced element (Wigner-Eckart).
* Every reduced block operator (c, d, A^k, B^k, DD^k, T and H) of left and
  right blocks built site by site, expanded to the determinant (Fock) space of
  the block's orbitals through its multiplets' M components, equals the
  operator written with spin-orbital creation and annihilation matrices
  (Jordan-Wigner signs in chain order), for every component: 1e-12. This
  fixes every recoupling factor and sign of the enlargement rules.
* H_eff psi equals P^T H_FCI P psi, with P the map of the reduced two-site
  wavefunction to determinants (Clebsch-Gordan coupling of the two enlarged
  blocks to S, M = S), for S = 0, 1/2, 1 and edge centres: 1e-12.
* Sweeps at exact bond dimension reach the spin-filtered FCI energy; truncated
  sweeps are variational and H_eff is symmetric.
"""
import itertools
import math

import numpy as np
import pytest

import qcinputs as q
from oracle import dmrgsu2 as ds
from oracle.fci import FCI, DetSpace
from oracle.mpssu2 import Mult, couple, site_mults
from oracle.su2alg import cg, coupled_factor, coupled_factor_def, ninej, recouple, sixj


# ---------------------------------------------------------------------------
# algebra
# ---------------------------------------------------------------------------
def test_sixj_special_values_and_orthogonality():
    # {a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))
    for a, b, c in itertools.product(range(0, 5), repeat=3):
        if abs(b - c) <= a <= b + c and (a + b + c) % 2 == 0:
            ref = (-1) ** ((a + b + c) // 2) / math.sqrt((b + 1) * (c + 1))
            assert abs(sixj(a, b, c, 0, c, b) - ref) < 1e-14
    # {1/2 1/2 1; 1/2 1/2 0} = 1/2 (doubled: {1 1 2; 1 1 0}); {1 1 1; 1 1 1} = 1/6
    assert abs(sixj(1, 1, 2, 1, 1, 0) - 0.5) < 1e-15
    assert abs(sixj(2, 2, 2, 2, 2, 2) - 1.0 / 6.0) < 1e-15
    # sum_x (2x+1)(2c+1) {a b x; d e c}{a b x; d e c'} = delta_cc'
    for a, b, d, e in itertools.product(range(0, 4), repeat=4):
        for c in range(0, 7):
            for cp in range(0, 7):
                s = sum((x + 1) * (c + 1) * sixj(a, b, x, d, e, c) * sixj(a, b, x, d, e, cp)
                        for x in range(0, 8))
                ok = abs(a - e) <= c <= a + e and abs(d - b) <= c <= d + b and (a + e + c) % 2 == 0 \
                    and (d + b + c) % 2 == 0
                assert abs(s - (1.0 if (c == cp and ok) else 0.0)) < 1e-12


def test_ninej_orthogonality_and_reduction_to_sixj():
    # {a b c; d e f; g h 0} = delta_cf delta_gh (-1)^(b+c+d+g) / sqrt((2c+1)(2g+1)) {a b c; e d g}
    for a, b, c, d, e, g in itertools.product(range(0, 4), repeat=6):
        v = ninej(a, b, c, d, e, c, g, g, 0)
        ref = (-1) ** ((b + c + d + g) // 2) / math.sqrt((c + 1) * (g + 1)) * sixj(a, b, c, e, d, g) \
            if (b + c + d + g) % 2 == 0 else 0.0
        assert abs(v - ref) < 1e-13
    # sum_{c,f} (2c+1)(2f+1)(2g+1)(2h+1) {a b c; d e f; g h i}{a b c; d e f; g' h' i} = delta
    a, b, d, e, i = 1, 1, 1, 1, 2
    for g, h, gp, hp in itertools.product(range(0, 3), repeat=4):
        s = 0.0
        for c in range(0, 3):
            for f in range(0, 3):
                s += (c + 1) * (f + 1) * math.sqrt((g + 1) * (h + 1) * (gp + 1) * (hp + 1)) * \
                    ninej(a, b, c, d, e, f, g, h, i) * ninej(a, b, c, d, e, f, gp, hp, i)
        okg = abs(a - d) <= g <= a + d and (a + d + g) % 2 == 0
        okh = abs(b - e) <= h <= b + e and (b + e + h) % 2 == 0
        oki = abs(g - h) <= i <= g + h
        ref = 1.0 if (g, h) == (gp, hp) and okg and okh and oki else 0.0
        assert abs(s - ref) < 1e-12


def test_clebsch_gordan_and_coupled_factor_definition():
    r2 = 1 / math.sqrt(2)
    assert abs(cg(1, 1, 1, -1, 0, 0) - r2) < 1e-15
    assert abs(cg(1, -1, 1, 1, 0, 0) + r2) < 1e-15
    assert abs(cg(2, 0, 1, 1, 1, 1) + math.sqrt(1 / 3)) < 1e-15
    for args in itertools.product(range(0, 3), repeat=9):
        assert abs(coupled_factor(*args) - coupled_factor_def(*args)) < 1e-13


def test_recoupling_is_orthogonal():
    js = (1, 1, 1)
    for J in (1, 3):
        for tin in (((0, 1, 0), 2), ((0, 1, 2), 2)):
            s = sum(recouple(js, tin, ((0, 2, K), 1), J) ** 2 for K in (0, 2))
            ok = abs(tin[0][2] - 1) <= J <= tin[0][2] + 1
            assert abs(s - (1.0 if ok else 0.0)) < 1e-14


def test_site_operators_are_tensor_operators():
    c, d = ds.site_c(), ds.site_d()
    assert np.allclose(ds.site_reduced(c, 1), [[0, 0, 0], [1, 0, 0], [0, -math.sqrt(2), 0]])
    for k in (0, 2):
        ds.site_reduced(ds.site_couple(c, 1, d, 1, k), k)   # raises if components disagree
    # d is the adjoint tensor of c: <0||d||1/2> = -sqrt(2) <1/2||c||0>
    assert abs(ds.site_reduced(d, 1)[0, 1] + math.sqrt(2)) < 1e-15


# ---------------------------------------------------------------------------
# Fock-space expansion of blocks
# ---------------------------------------------------------------------------
def fock_cre(nsites):
    """a+_{p sigma} on the Fock space of nsites sites (configuration index: site
    0 the least significant base-4 digit, local index n_up + 2 n_dn), with the
    Jordan-Wigner sign of chain order 0up, 0dn, 1up, ..."""
    dim = 4 ** nsites
    ops = {}
    for p in range(nsites):
        for sg in range(2):
            M = np.zeros((dim, dim))
            mode = 2 * p + sg
            for f in range(dim):
                occ = []
                x = f
                for _ in range(nsites):
                    loc = x % 4
                    x //= 4
                    occ += [loc & 1, (loc >> 1) & 1]
                if occ[mode]:
                    continue
                sign = (-1) ** sum(occ[:mode])
                occ2 = list(occ)
                occ2[mode] = 1
                g = sum((occ2[2 * s] + 2 * occ2[2 * s + 1]) * 4 ** s for s in range(nsites))
                M[g, f] = sign
            ops[(p, sg)] = M
    return ops


def fock_tensors(nsites, orbs, h, V):
    """Components {2q: matrix} of c_p, d_p, pair operators, T_m and H for orbitals
    `orbs` of a block whose Fock space covers local sites 0..nsites-1 (orbital
    orbs[i] on local site i), from spin-orbital matrices."""
    cr = fock_cre(nsites)
    loc = {p: i for i, p in enumerate(orbs)}
    c = {p: {1: cr[(loc[p], 0)], -1: cr[(loc[p], 1)]} for p in orbs}
    d = {p: {1: cr[(loc[p], 1)].T, -1: -cr[(loc[p], 0)].T} for p in orbs}

    def coup(X, kx, Y, ky, k):
        out = {}
        for qq in range(-k, k + 1, 2):
            M = 0
            for q1, Xm in X.items():
                if qq - q1 in Y:
                    w = cg(kx, q1, ky, qq - q1, k, qq)
                    if w:
                        M = M + w * (Xm @ Y[qq - q1])
            out[qq] = M if not isinstance(M, int) else np.zeros_like(cr[(0, 0)])
        return out
    E = {(p, r): sum(cr[(loc[p], s)] @ cr[(loc[r], s)].T for s in range(2)) for p in orbs for r in orbs}
    return c, d, coup, E, cr, loc


def build_states(mps, upto, left):
    """Multiplets (Fock vectors of all components) of the oracle's left block of
    sites 0..upto-1 or right block of sites upto..L-1, from its tensors."""
    L = mps.L
    mults = [Mult(0, 0, np.ones((1, 1)))]
    site = site_mults()
    sites = range(upto) if left else range(L - 1, upto - 1, -1)
    for p in sites:
        labels = _labels(mults)
        pb = ds.Product(labels, ds.SITE_LABELS, True) if left else ds.Product(ds.SITE_LABELS, labels, False)
        ent = []
        for e in range(pb.dim):
            i1, i2, J = pb.i1[e], pb.i2[e], pb.J[e]
            if left:
                ent.append(couple(mults[i1], site[i2], J))
            else:
                ent.append(couple(site[i1], mults[i2], J))
        T = mps.A[p] if left else mps.R[p].T
        bond = mps.lbonds[p + 1] if left else mps.rbonds[p]
        new = []
        for k in range(bond.dim):
            vec = sum(T[e, k] * ent[e] for e in range(pb.dim) if T[e, k] != 0.0)
            new.append(Mult(int(bond.n[k]), int(bond.s[k]), vec))
        mults = new
    return mults


def _labels(mults):
    class _L:
        pass
    o = _L()
    o.n = np.array([m.n for m in mults])
    o.s = np.array([m.s for m in mults])
    o.dim = len(mults)
    return o


def check_operator(red, comps, k, mults, tol=1e-11):
    """<a m|O_q|b m'> = <S_b m'; k q|S_a m> red[a, b] for every component."""
    err = 0.0
    for a, ma in enumerate(mults):
        for b, mb in enumerate(mults):
            for ia in range(ma.s + 1):
                for ib in range(mb.s + 1):
                    m1, m2 = ma.s - 2 * ia, mb.s - 2 * ib
                    qq = m1 - m2
                    if abs(qq) > k:
                        continue
                    v = ma.vec[ia] @ comps[qq] @ mb.vec[ib] if qq in comps else 0.0
                    ref = cg(mb.s, m2, k, qq, ma.s, m1) * red[a, b]
                    err = max(err, abs(v - ref))
    assert err < tol, err


def _mps(L, N, two_s, D, c, seed=3):
    return ds.MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))


@pytest.mark.parametrize("L,N,two_s,D,c,left", [(5, 5, 1, 6, 3, True), (5, 4, 0, 6, 1, False),
                                                (4, 4, 2, 16, 2, True), (4, 3, 1, 16, 1, False)])
def test_block_operators_expand_to_determinant_matrices(L, N, two_s, D, c, left):
    h, V = q.make_integrals(L, 7)
    mps = _mps(L, N, two_s, D, c)
    dm = ds.DMRGSU2(h, V, N, two_s)
    if left:
        nb = c
        blk = dm.left_block(mps, nb)
        orbs = list(range(nb))
    else:
        nb = L - (c + 2)
        blk = dm.right_block(mps, c + 2)
        orbs = list(range(c + 2, L))
    mults = build_states(mps, nb if left else c + 2, left)
    # local site i of the Fock space holds orbital orbs[i] for a left block; a right
    # block's Fock index has its first site (orbital c+2) as the least significant digit
    cfock, dfock, coup, E, cr, loc = fock_tensors(len(orbs), orbs, h, V)
    for p in orbs:
        check_operator(blk.C[p], cfock[p], 1, mults)
        check_operator(blk.Dd[p], dfock[p], 1, mults)
    for k in (0, 2):
        for p in orbs:
            for r in orbs:
                check_operator(blk.A[(k, p, r)], coup(cfock[p], 1, cfock[r], 1, k), k, mults)
                check_operator(blk.B[(k, p, r)], coup(cfock[p], 1, dfock[r], 1, k), k, mults)
                check_operator(blk.DD[(k, p, r)], coup(dfock[p], 1, dfock[r], 1, k), k, mults)
    for m in blk.outside:
        comps = {}
        for qq in (1, -1):
            M = sum(0.5 * h[m, qo] * dfock[qo][qq] for qo in orbs)
            for qo, ro, so in itertools.product(orbs, repeat=3):
                M = M + V[m, so, qo, ro] * (E[(qo, ro)] @ dfock[so][qq])
            comps[qq] = M
        check_operator(blk.T[m], comps, 1, mults)
    Hf = sum(h[p, r] * E[(p, r)] for p in orbs for r in orbs)
    for p, r, s, t in itertools.product(orbs, repeat=4):
        if V[p, r, s, t]:
            for a, b in itertools.product(range(2), repeat=2):
                Hf = Hf + 0.5 * V[p, r, s, t] * (cr[(loc[p], a)] @ cr[(loc[s], b)] @ cr[(loc[t], b)].T @
                                                 cr[(loc[r], a)].T)
    check_operator(blk.H, {0: Hf}, 0, mults, tol=1e-10)


# ---------------------------------------------------------------------------
# H_eff against the plain definition P^T H P
# ---------------------------------------------------------------------------
def projector(mps):
    """P[det, (a, b) pair of the psi layout]: |(a b) S, M = S> expanded to determinants."""
    c, L = mps.center, mps.L
    lm = build_states(mps, c, True)
    rm = build_states(mps, c + 2, False)
    site = site_mults()
    Lp, Rp = mps.lprod(), mps.rprod()
    La = [couple(lm[Lp.i1[e]], site[Lp.i2[e]], Lp.J[e]) for e in range(Lp.dim)]
    Rb = [couple(site[Rp.i1[e]], rm[Rp.i2[e]], Rp.J[e]) for e in range(Rp.dim)]
    space = DetSpace(L, mps.N, mps.two_s)
    nl = 4 ** (c + 1)
    cols = []
    mask = mps.mask()
    pairs = [(a, b) for a in range(Lp.dim) for b in range(Rp.dim) if mask[a, b]]
    for a, b in pairs:
        sa, sb, S = Lp.J[a], Rp.J[b], mps.two_s
        v = np.zeros(nl * Rb[b].shape[1])
        for ia in range(sa + 1):
            ma = sa - 2 * ia
            mb = S - ma
            if abs(mb) > sb:
                continue
            w = cg(sa, ma, sb, mb, S, S)
            if w:
                v += w * np.kron(Rb[b][(sb - mb) // 2], La[a][ia])
        cols.append(_to_dets(v, L, space))
    return np.stack(cols, axis=1), pairs, space


def _to_dets(v, L, space):
    out = np.zeros(space.dim)
    for f in np.nonzero(v)[0]:
        bits, x = 0, int(f)
        for p in range(L):
            cc = x % 4
            x //= 4
            if cc & 1:
                bits |= 1 << (2 * p)
            if cc & 2:
                bits |= 1 << (2 * p + 1)
        idx, ok = space.index(np.array([bits], dtype=np.uint64))
        assert ok[0]
        out[idx[0]] += v[f]
    return out


@pytest.mark.parametrize("L,N,two_s,D,c", [(4, 4, 0, 16, 1), (5, 5, 1, 8, 1), (5, 4, 2, 8, 2),
                                           (6, 6, 0, 6, 0), (6, 5, 1, 6, 4), (6, 6, 2, 5, 2)])
def test_sigma_equals_projected_fci(L, N, two_s, D, c):
    h, V = q.make_integrals(L, 11)
    mps = _mps(L, N, two_s, D, c, seed=5)
    P, pairs, space = projector(mps)
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < 1e-12
    f = FCI(h, V, N, two_s)
    x = np.array([mps.psi[a, b] for a, b in pairs])
    ref = P.T @ f.apply(P @ x)
    sig = ds.DMRGSU2(h, V, N, two_s).sigma(mps)
    got = np.array([sig[a, b] for a, b in pairs])
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("L,N,two_s", [(6, 6, 0), (5, 5, 1), (6, 4, 2)])
def test_exact_sweeps_reach_spin_filtered_fci(L, N, two_s):
    h, V = q.make_integrals(L, 13)
    mps = _mps(L, N, two_s, 400, L // 2 - 1, seed=2)
    e, terr, _ = ds.DMRGSU2(h, V, N, two_s).sweeps(mps, 400, nsweeps=2, tol=1e-12)
    e_fci, _ = FCI(h, V, N, two_s).ground_state(two_s=two_s)
    assert abs(e[-1] - e_fci) < 1e-9
    assert max(terr) < 1e-12


def test_truncated_sweeps_are_variational_and_heff_symmetric():
    L, N, two_s, D = 8, 8, 0, 12
    h, V = q.make_integrals(L, 17)
    mps = _mps(L, N, two_s, D, 3, seed=4)
    dm = ds.DMRGSU2(h, V, N, two_s)
    heff = dm.heff_at_center(mps)
    rng = np.random.default_rng(0)
    x = rng.normal(size=heff.shape) * heff.mask
    y = rng.normal(size=heff.shape) * heff.mask
    assert abs(np.sum(x * heff.apply_mat(y)) - np.sum(heff.apply_mat(x) * y)) < 1e-11 * np.abs(x).sum()
    e, terr, out = dm.sweeps(mps, D, nsweeps=2, tol=1e-10)
    e_fci, _ = FCI(h, V, N, two_s).ground_state(two_s=two_s)
    assert e[-1] >= e_fci - 1e-10
    assert e[-1] <= e[0] + 1e-9
    assert max(terr) > 0.0
