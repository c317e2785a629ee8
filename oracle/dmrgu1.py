"""Operator-based two-site DMRG in U(1)xU(1) symmetry, dense FP64 (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

Follows the renormalized-operator formulation of quantum-chemical DMRG that
the paper's Method section relies on (memory O(N^2 D^2), compute O(N^4 D^3)):
every block keeps normal operators (a+_k, a+_k a+_l, a+_k a_l for its own
spin-orbitals) and complementary operators (S_m for every spin-orbital m
outside the block, and the block Hamiltonian). Two-index complementary
operators P, Q are formed on the fly from the other side's normal operators.

Spin-orbital form of H (k = 2p + sigma):
    H = sum t_kl a+_k a_l + 1/2 sum w_ijkl a+_i a+_j a_k a_l,
    t_kl = h_{p_k p_l} d(s_k,s_l),  w_ijkl = (p_i p_l | p_j p_k) d(s_i,s_l) d(s_j,s_k).
Complementary one-index operator of a block B for m outside B:
    S^B_m = 1/2 sum_{j in B} t_mj a_j + sum_{jkl in B} w_mjkl a+_j a_k a_l
(the one-body cross terms appear once through S^R and once through S^L, so
each carries half of t).
Decomposition at a cut L|R (operator products written left part first):
    H = H_L + H_R
      + sum_{i in L} ( a+_i S^R_i - a_i (S^R_i)^+ )
      + sum_{m in R} ( -S^L_m a+_m + (S^L_m)^+ a_m )
      + 1/2 sum_{ij in L, kl in R} w_ijkl (a+_i a+_j)(a_k a_l)
      + 1/2 sum_{kl in L, ij in R} w_ijkl (a_k a_l)(a+_i a+_j)
      + sum_{il in L, jk in R} (w_ijkl - w_ijlk) (a+_i a_l)(a+_j a_k).
A product O_L O_R acts on |x>|y> as (O_L P_L^{p(O_R)}) (x) O_R, with P_L the
fermion parity of the left part (Jordan-Wigner order follows the chain).
"""

import numpy as np
import scipy.sparse.linalg as spla

from .mpsu1 import SITE_N, SITE_S, Bond, MPSU1

# single-site matrices, basis |0>, |up>, |dn>, |updn>
_CUP = np.zeros((4, 4))
_CUP[1, 0] = 1.0   # a+_up |0> = |up>
_CUP[3, 2] = 1.0   # a+_up |dn> = a+_up a+_dn |0> = |updn>
_CDN = np.zeros((4, 4))
_CDN[2, 0] = 1.0   # a+_dn |0> = |dn>
_CDN[3, 1] = -1.0  # a+_dn a+_up |0> = -|updn>
_PS = np.diag([1.0, -1.0, -1.0, 1.0])
SITE_CRE = (_CUP, _CDN)


def spin_orbital_integrals(h, V):
    L = h.shape[0]
    n = 2 * L
    p = np.arange(n) // 2
    s = np.arange(n) % 2
    t = h[np.ix_(p, p)] * (s[:, None] == s[None, :])
    # w_ijkl = V[p_i, p_l, p_j, p_k] d(s_i, s_l) d(s_j, s_k)
    w = V[p[:, None, None, None], p[None, None, None, :], p[None, :, None, None], p[None, None, :, None]]
    w = w * (s[:, None, None, None] == s[None, None, None, :]) * (s[None, :, None, None] == s[None, None, :, None])
    return t, w


class Block:
    """Dense renormalized operators of a block of consecutive sites."""

    def __init__(self, modes, outside, n, s, C, AA, BB, S, H):
        self.modes = list(modes)          # spin-orbitals of the block (ascending)
        self.outside = list(outside)      # spin-orbitals not in the block (ascending)
        self.n, self.s = np.asarray(n), np.asarray(s)   # labels per basis state
        self.P = np.where(self.n % 2 == 0, 1.0, -1.0)
        self.C, self.AA, self.BB, self.S, self.H = C, AA, BB, S, H
        self.dim = len(self.n)


def vacuum_block(nmodes):
    z = np.zeros((0, 1, 1))
    return Block([], list(range(nmodes)), [0], [0], z,
                 np.zeros((0, 0, 1, 1)), np.zeros((0, 0, 1, 1)),
                 np.zeros((nmodes, 1, 1)), np.zeros((1, 1)))


def site_block(site, t, w):
    """Exact operators of one site (no truncation: products are exact)."""
    nm = t.shape[0]
    modes = [2 * site, 2 * site + 1]
    outside = [m for m in range(nm) if m not in modes]
    c = SITE_CRE
    C = np.stack(c)
    AA = np.stack([[c[a] @ c[b] for b in range(2)] for a in range(2)])
    BB = np.stack([[c[a] @ c[b].T for b in range(2)] for a in range(2)])
    S = np.zeros((len(outside), 4, 4))
    for mi, m in enumerate(outside):
        op = np.zeros((4, 4))
        for j in range(2):
            op += 0.5 * t[m, modes[j]] * c[j].T
            for k in range(2):
                for l in range(2):
                    op += w[m, modes[j], modes[k], modes[l]] * (c[j] @ c[k].T @ c[l].T)
        S[mi] = op
    H = np.zeros((4, 4))
    for a in range(2):
        for b in range(2):
            H += t[modes[a], modes[b]] * (c[a] @ c[b].T)
            for k in range(2):
                for l in range(2):
                    H += 0.5 * w[modes[a], modes[b], modes[k], modes[l]] * (c[a] @ c[b] @ c[k].T @ c[l].T)
    return Block(modes, outside, SITE_N.copy(), SITE_S.copy(), C, AA, BB, S, H)


def decomposition(Lb, Rb, t, w):
    """Terms (O_L, O_R, odd) of H at the cut Lb|Rb, excluding H_L and H_R.

    Each term stands for the operator product O_L O_R; 'odd' is the fermion
    parity of O_R. Two-index complementary operators are formed here from the
    other side's normal operators.
    """
    ML, MR = Lb.modes, Rb.modes
    terms = []
    iR = {m: k for k, m in enumerate(Rb.outside)}
    iL = {m: k for k, m in enumerate(Lb.outside)}
    for a, i in enumerate(ML):
        SR = Rb.S[iR[i]]
        terms.append((Lb.C[a], SR, True))
        terms.append((-Lb.C[a].T, SR.T, True))
    for b, m in enumerate(MR):
        SL = Lb.S[iL[m]]
        terms.append((-SL, Rb.C[b], True))
        terms.append((SL.T, Rb.C[b].T, True))
    if ML and MR:
        AAtR = Rb.AA.transpose(1, 0, 3, 2)            # AAtR[k,l] = a_k a_l
        PR = 0.5 * np.einsum("ijkl,klab->ijab", w[np.ix_(ML, ML, MR, MR)], AAtR)
        AAtL = Lb.AA.transpose(1, 0, 3, 2)            # a_k a_l on the left
        PL = 0.5 * np.einsum("ijkl,ijab->klab", w[np.ix_(MR, MR, ML, ML)], Rb.AA)
        wLRRL = w[np.ix_(ML, MR, MR, ML)]             # [i, j, k, l]
        wLRLR = w[np.ix_(ML, MR, ML, MR)]             # [i, j, l, k]
        coef = wLRRL - wLRLR.transpose(0, 1, 3, 2)    # w_ijkl - w_ijlk
        QR = np.einsum("ijkl,jkab->ilab", coef, Rb.BB)
        for a in range(len(ML)):
            for b in range(len(ML)):
                terms.append((Lb.AA[a, b], PR[a, b], False))
                terms.append((AAtL[a, b], PL[a, b], False))
                terms.append((Lb.BB[a, b], QR[a, b], False))
    return terms


def _site_three(w, m, sm):
    op = np.zeros((4, 4))
    c = SITE_CRE
    for ja in range(2):
        for ka in range(2):
            for la in range(2):
                op += w[m, sm[ja], sm[ka], sm[la]] * (c[ja] @ c[ka].T @ c[la].T)
    return op


def enlarge_left(X, site, t, w):
    """Operators of L' = X (x) site from those of X and of the site."""
    DX = X.dim
    I4 = np.eye(4)
    IX = np.eye(DX)
    PX = np.diag(X.P)
    sm = site.modes
    c = SITE_CRE
    modes = X.modes + sm
    outside = [m for m in X.outside if m not in sm]
    n = (X.n[:, None] + SITE_N[None, :]).reshape(-1)
    s = (X.s[:, None] + SITE_S[None, :]).reshape(-1)
    D = DX * 4
    nx = len(X.modes)
    nb = nx + 2
    C = np.zeros((nb, D, D))
    for a in range(nx):
        C[a] = np.kron(X.C[a], I4)
    for b in range(2):
        C[nx + b] = np.kron(PX, c[b])
    AA = np.zeros((nb, nb, D, D))
    BB = np.zeros((nb, nb, D, D))
    for a in range(nx):
        for b in range(nx):
            AA[a, b] = np.kron(X.AA[a, b], I4)
            BB[a, b] = np.kron(X.BB[a, b], I4)
    for a in range(nx):
        CP = X.C[a] @ PX
        CtP = X.C[a].T @ PX
        for b in range(2):
            AA[a, nx + b] = np.kron(CP, c[b])          # a+_k(X) a+_l(s)
            AA[nx + b, a] = -np.kron(CP, c[b])         # a+_l(s) a+_k(X) = -a+_k a+_l
            BB[a, nx + b] = np.kron(CP, c[b].T)        # a+_k(X) a_l(s)
            BB[nx + b, a] = -np.kron(CtP, c[b])        # a+_k(s) a_l(X) = -a_l a+_k
    for a in range(2):
        for b in range(2):
            AA[nx + a, nx + b] = np.kron(IX, c[a] @ c[b])
            BB[nx + a, nx + b] = np.kron(IX, c[a] @ c[b].T)
    iX = {m: k for k, m in enumerate(X.outside)}
    BBXP = np.einsum("jkab,bc->jkac", X.BB, PX)
    AAtXP = np.einsum("klab,bc->klac", X.AA.transpose(1, 0, 3, 2), PX)
    XC = X.C
    XCt = X.C.transpose(0, 2, 1)
    XM = X.modes
    S = np.zeros((len(outside), D, D))
    for mi, m in enumerate(outside):
        op = np.kron(X.S[iX[m]], I4)
        for j in range(2):
            op += 0.5 * t[m, sm[j]] * np.kron(PX, c[j].T)
        if nx:
            wm = w[m]
            for sj in range(2):
                js = sm[sj]
                # (X, X, s): (a+_j a_k)_X (a_l)_s
                op += np.kron(np.einsum("jk,jkab->ab", wm[np.ix_(XM, XM)][:, :, js], BBXP), c[sj].T)
                # (X, s, X): -(a+_j a_l)_X (a_k)_s
                op -= np.kron(np.einsum("jl,jlab->ab", wm[XM][:, js][:, XM], BBXP), c[sj].T)
                # (s, X, X): (a_k a_l)_X (a+_j)_s
                op += np.kron(np.einsum("kl,klab->ab", wm[js][np.ix_(XM, XM)], AAtXP), c[sj])
            for sa in range(2):
                for sb in range(2):
                    ka, kb = sm[sa], sm[sb]
                    # (X, s, s): a+_j(X) (a_ka a_kb)_s
                    op += np.kron(np.einsum("j,jab->ab", wm[XM, ka, kb], XC), c[sa].T @ c[sb].T)
                    # (s, X, s): a+_ka a_k a_kb = -(a_k)_X (a+_ka a_kb)_s
                    op -= np.kron(np.einsum("k,kab->ab", wm[ka, XM, kb], XCt), c[sa] @ c[sb].T)
                    # (s, s, X): a+_ka a_kb a_l = (a_l)_X (a+_ka a_kb)_s
                    op += np.kron(np.einsum("l,lab->ab", wm[ka, kb, XM], XCt), c[sa] @ c[sb].T)
        op += np.kron(PX, _site_three(w, m, sm))
        S[mi] = op
    H = np.kron(X.H, I4) + np.kron(IX, site.H)
    for OL, OR, odd in decomposition(X, site, t, w):
        H += np.kron(OL @ PX if odd else OL, OR)
    return Block(modes, outside, n, s, C, AA, BB, S, H)


def enlarge_right(site, Y, t, w):
    """Operators of R' = site (x) Y (site modes first in the fermion order)."""
    DY = Y.dim
    I4 = np.eye(4)
    IY = np.eye(DY)
    P4 = _PS
    sm = site.modes
    c = SITE_CRE
    modes = sm + Y.modes
    outside = [m for m in Y.outside if m not in sm]
    n = (SITE_N[:, None] + Y.n[None, :]).reshape(-1)
    s = (SITE_S[:, None] + Y.s[None, :]).reshape(-1)
    D = 4 * DY
    ny = len(Y.modes)
    nb = ny + 2
    C = np.zeros((nb, D, D))
    for b in range(2):
        C[b] = np.kron(c[b], IY)
    for a in range(ny):
        C[2 + a] = np.kron(P4, Y.C[a])
    AA = np.zeros((nb, nb, D, D))
    BB = np.zeros((nb, nb, D, D))
    for a in range(2):
        for b in range(2):
            AA[a, b] = np.kron(c[a] @ c[b], IY)
            BB[a, b] = np.kron(c[a] @ c[b].T, IY)
    for sa in range(2):
        for y in range(ny):
            AA[sa, 2 + y] = np.kron(c[sa] @ P4, Y.C[y])          # a+_s a+_y
            AA[2 + y, sa] = -np.kron(c[sa] @ P4, Y.C[y])         # a+_y a+_s = -a+_s a+_y
            BB[sa, 2 + y] = np.kron(c[sa] @ P4, Y.C[y].T)        # a+_s a_y
            BB[2 + y, sa] = -np.kron(c[sa].T @ P4, Y.C[y])       # a+_y a_s = -a_s a+_y
    for a in range(ny):
        for b in range(ny):
            AA[2 + a, 2 + b] = np.kron(I4, Y.AA[a, b])
            BB[2 + a, 2 + b] = np.kron(I4, Y.BB[a, b])
    iY = {m: k for k, m in enumerate(Y.outside)}
    YM = Y.modes
    AAtY = Y.AA.transpose(1, 0, 3, 2)
    YC = Y.C
    YCt = Y.C.transpose(0, 2, 1)
    S = np.zeros((len(outside), D, D))
    for mi, m in enumerate(outside):
        op = np.kron(P4, Y.S[iY[m]])
        for j in range(2):
            op += 0.5 * t[m, sm[j]] * np.kron(c[j].T, IY)
        if ny:
            wm = w[m]
            for sj in range(2):
                js = sm[sj]
                # (s, Y, Y): (a+_j)_s (a_k a_l)_Y
                op += np.kron(c[sj], np.einsum("kl,klab->ab", wm[js][np.ix_(YM, YM)], AAtY))
                # (Y, s, Y): a+_j a_k a_l = -(a_k)_s (a+_j a_l)_Y
                op -= np.kron(c[sj].T, np.einsum("jl,jlab->ab", wm[YM][:, js][:, YM], Y.BB))
                # (Y, Y, s): a+_j a_k a_l = (a_l)_s (a+_j a_k)_Y
                op += np.kron(c[sj].T, np.einsum("jk,jkab->ab", wm[np.ix_(YM, YM)][:, :, js], Y.BB))
            for sa in range(2):
                for sb in range(2):
                    ka, kb = sm[sa], sm[sb]
                    # (s, s, Y): (a+_ka a_kb)_s (a_l)_Y
                    op += np.kron(c[sa] @ c[sb].T @ P4, np.einsum("l,lab->ab", wm[ka, kb, YM], YCt))
                    # (s, Y, s): a+_ka a_k a_kb = -(a+_ka a_kb)_s (a_k)_Y
                    op -= np.kron(c[sa] @ c[sb].T @ P4, np.einsum("k,kab->ab", wm[ka, YM, kb], YCt))
                    # (Y, s, s): a+_j a_ka a_kb = (a_ka a_kb)_s (a+_j)_Y
                    op += np.kron(c[sa].T @ c[sb].T @ P4, np.einsum("j,jab->ab", wm[YM, ka, kb], YC))
        op += np.kron(_site_three(w, m, sm), IY)
        S[mi] = op
    H = np.kron(site.H, IY) + np.kron(I4, Y.H)
    for OL, OR, odd in decomposition(site, Y, t, w):
        H += np.kron(OL @ P4 if odd else OL, OR)
    return Block(modes, outside, n, s, C, AA, BB, S, H)


def project_block(blk, U, n, s, left=True):
    """Renormalize: O -> U^T O U (left, U: (D', Dnew)) or V O V^T (right, V: (Dnew, D'))."""
    if left:
        g = lambda O: np.einsum("ia,...ij,jb->...ab", U, O, U, optimize=True)
    else:
        g = lambda O: np.einsum("ai,...ij,bj->...ab", U, O, U, optimize=True)
    return Block(blk.modes, blk.outside, n, s, g(blk.C), g(blk.AA), g(blk.BB), g(blk.S), g(blk.H))


class Heff:
    """H_eff at the two-site centre from the enlarged blocks L', R'.

    psi is the matrix psi[(x i), (j y)]; a term O_L O_R maps it to
    O_L P_L'^{p(O_R)} psi O_R^T.
    """

    def __init__(self, Lp, Rp, t, w, N, two_sz, e_core=0.0):
        self.Lp, self.Rp = Lp, Rp
        self.terms = decomposition(Lp, Rp, t, w)
        self.e_core = e_core
        tn = Lp.n[:, None] + Rp.n[None, :]
        ts = Lp.s[:, None] + Rp.s[None, :]
        self.mask = (tn == N) & (ts == two_sz)
        self.shape = (Lp.dim, Rp.dim)

    def apply_mat(self, x):
        sig = self.Lp.H @ x + x @ self.Rp.H.T + self.e_core * x
        Px = self.Lp.P[:, None] * x
        for OL, OR, odd in self.terms:
            sig += OL @ (Px if odd else x) @ OR.T
        return sig * self.mask


def to_mat(psi4):
    DX, _, _, DY = psi4.shape
    return psi4.reshape(DX * 4, 4 * DY)


def from_mat(m, DX, DY):
    return m.reshape(DX, 4, 4, DY)


def lowest_eig(heff, guess_mat, tol=1e-12):
    """Lanczos (ARPACK) on the masked H_eff: ground state of the two-site problem."""
    sel = heff.mask.reshape(-1)
    nsel = int(sel.sum())

    def mv(x):
        full = np.zeros(sel.shape[0])
        full[sel] = x
        return heff.apply_mat(full.reshape(heff.shape)).reshape(-1)[sel]
    v0 = guess_mat.reshape(-1)[sel]
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


def svd_sectors(x, Ln, Ls, Rn, Rs, N, two_sz):
    """Per-sector SVD of psi[(x i), (j y)]; returns {qL: (rows, cols, u, sv, vt)}."""
    blocks = {}
    for qn in sorted(set(zip(Ln.tolist(), Ls.tolist()))):
        rows = np.nonzero((Ln == qn[0]) & (Ls == qn[1]))[0]
        cols = np.nonzero((Rn == N - qn[0]) & (Rs == two_sz - qn[1]))[0]
        if len(rows) == 0 or len(cols) == 0:
            continue
        u, sv, vt = np.linalg.svd(x[np.ix_(rows, cols)], full_matrices=False)
        blocks[qn] = (rows, cols, u, sv, vt)
    return blocks


TIE_REL = 1e-8
# Weights at or below this are rounding noise of the density-matrix eigenvalues
# (absolute error ~1e-16 of the unit trace) and are always discarded, so that
# zero-weight states never enter a basis.
WEIGHT_FLOOR = 1e-14


def select_kept(blocks, D, drop_below=WEIGHT_FLOOR):
    """Keep the D largest weights sv^2 above drop_below; ties by label
    ascending, then index.

    Weights that are equal up to rounding (within TIE_REL relative of the D-th
    weight) are kept or discarded together: when such a group straddles the
    cut it is discarded as a whole, so fewer than D states are kept. Exact
    ties arise from the spin-flip symmetry of Sz = 0 states (sectors Sz and
    -Sz carry equal weights), and a cut through them would otherwise be
    decided by rounding.

    Returns ({qL: [k...]}, discarded weight).
    """
    cand = []
    for qn, (_, _, _, sv, _) in blocks.items():
        for k, x in enumerate(sv):
            cand.append((-x * x, qn, k))
    cand.sort()
    keep = cand[:D]
    if len(cand) > D:
        lam_cut = -cand[D - 1][0]
        if -cand[D][0] >= lam_cut - TIE_REL * lam_cut:
            keep = [c for c in keep if -c[0] > lam_cut + TIE_REL * lam_cut]
    keep = [c for c in keep if -c[0] > drop_below]
    kept_set = set(keep)
    disc = sum(-c[0] for c in cand if c not in kept_set)
    kept = {}
    for _, qn, k in keep:
        kept.setdefault(qn, []).append(k)
    return {q: sorted(v) for q, v in kept.items()}, float(disc)


def dbss_bond_dimension(blocks, eps, D_min, D_max):
    """Dynamic block-state selection (the fixed-truncation-error alternative to
    a fixed D in the paper's Numerical procedure section): the smallest D in
    [D_min, D_max] whose discarded weight, the sum of all weights sv^2 beyond
    the D largest, is at most eps; D_max (or the number of weights) when none
    is. The selection itself then runs select_kept with that D."""
    w = sorted((float(x) * float(x) for (_, _, _, sv, _) in blocks.values() for x in sv), reverse=True)
    top = min(D_max, len(w))
    for D in range(max(1, D_min), top + 1):
        if sum(w[D:]) <= eps:
            return D
    return max(1, top)


def left_factor(blocks, kept, dL, dR):
    bnew = Bond({qn: len(ks) for qn, ks in kept.items()})
    U = np.zeros((dL, bnew.dim))
    SV = np.zeros((bnew.dim, dR))
    for qn, ks in kept.items():
        rows, cols, u, sv, vt = blocks[qn]
        st, dq = bnew.sectors[qn]
        r = np.arange(st, st + dq)
        U[np.ix_(rows, r)] = u[:, ks]
        SV[np.ix_(r, cols)] = sv[ks][:, None] * vt[ks]
    return bnew, U, SV


def right_factor(blocks, kept, dL, dR, N, two_sz):
    lab = {(N - qn[0], two_sz - qn[1]): qn for qn in kept}
    bnew = Bond({r: len(kept[qn]) for r, qn in lab.items()})
    Vt = np.zeros((bnew.dim, dR))
    US = np.zeros((dL, bnew.dim))
    for r, qn in lab.items():
        rows, cols, u, sv, vt = blocks[qn]
        ks = kept[qn]
        st, dq = bnew.sectors[r]
        rr = np.arange(st, st + dq)
        Vt[np.ix_(rr, cols)] = vt[ks]
        US[np.ix_(rows, rr)] = u[:, ks] * sv[ks][None, :]
    return bnew, Vt, US


class DMRGU1:
    """Plain two-site DMRG driver (oracle)."""

    def __init__(self, h, V, N, two_sz, e_core=0.0):
        self.h, self.V = np.asarray(h, float), np.asarray(V, float)
        self.L = self.h.shape[0]
        self.N, self.two_sz, self.e_core = N, two_sz, e_core
        self.t, self.w = spin_orbital_integrals(self.h, self.V)
        self.sites = [site_block(p, self.t, self.w) for p in range(self.L)]

    def left_block(self, mps, upto):
        """Renormalized block of sites 0..upto-1 from the left-canonical tensors."""
        blk = vacuum_block(2 * self.L)
        for p in range(upto):
            Lp = enlarge_left(blk, self.sites[p], self.t, self.w)
            bnew = mps.lbonds[p + 1]
            blk = project_block(Lp, mps.A[p].reshape(-1, bnew.dim), bnew.n, bnew.s, left=True)
        return blk

    def right_block(self, mps, frm):
        """Renormalized block of sites frm..L-1 from the right-canonical tensors."""
        blk = vacuum_block(2 * self.L)
        for p in range(self.L - 1, frm - 1, -1):
            Rp = enlarge_right(self.sites[p], blk, self.t, self.w)
            bnew = mps.rbonds[p]
            blk = project_block(Rp, mps.R[p].reshape(bnew.dim, -1), bnew.n, bnew.s, left=False)
        return blk

    def heff_at_center(self, mps):
        l = mps.center
        Lp = enlarge_left(self.left_block(mps, l), self.sites[l], self.t, self.w)
        Rp = enlarge_right(self.sites[l + 1], self.right_block(mps, l + 2), self.t, self.w)
        return Heff(Lp, Rp, self.t, self.w, self.N, self.two_sz, self.e_core)

    def sigma(self, mps, psi4=None):
        """sigma = H_eff psi at the centre of mps (psi defaults to mps.psi)."""
        heff = self.heff_at_center(mps)
        psi4 = mps.psi if psi4 is None else psi4
        return from_mat(heff.apply_mat(to_mat(psi4)), psi4.shape[0], psi4.shape[3])

    def move_center_left(self, mps, target):
        """Shift the two-site centre left by exact (untruncated) SVDs."""
        A, R = dict(mps.A), dict(mps.R)
        lb, rb = dict(mps.lbonds), dict(mps.rbonds)
        psi = mps.psi
        l = mps.center
        while l > target:
            DX, DY = psi.shape[0], psi.shape[3]
            Ln = (lb[l].n[:, None] + SITE_N[None, :]).reshape(-1)
            Ls = (lb[l].s[:, None] + SITE_S[None, :]).reshape(-1)
            Rn = (SITE_N[:, None] + rb[l + 2].n[None, :]).reshape(-1)
            Rs = (SITE_S[:, None] + rb[l + 2].s[None, :]).reshape(-1)
            blocks = svd_sectors(to_mat(psi), Ln, Ls, Rn, Rs, self.N, self.two_sz)
            kept, _ = select_kept(blocks, 10 ** 9)
            bnew, Vt, US = right_factor(blocks, kept, len(Ln), len(Rn), self.N, self.two_sz)
            R[l + 1] = Vt.reshape(bnew.dim, 4, DY)
            rb[l + 1] = bnew
            psi = np.einsum("cha,aib->chib", A.pop(l - 1), US.reshape(DX, 4, bnew.dim))
            del lb[l]
            l -= 1
        return MPSU1(self.L, self.N, self.two_sz, l, lb, rb, A, R, psi)

    def sweeps(self, mps, D, nsweeps=1, tol=1e-12, trunc_eps=0.0, D_min=1):
        """Full sweeps; returns (energies, max discarded weights, final MPS).

        The MPS is first moved to centre 0. Each sweep optimises centres
        0..L-3 moving right and L-2..1 moving left (2L-4 optimisations) and
        ends with the centre back at 0. The energy of a sweep is that of its
        last optimisation. trunc_eps > 0: each truncation keeps the bond
        dimension dbss_bond_dimension gives in [D_min, D]; self.max_kept and
        self.total_kept are the largest and the summed numbers of states kept.
        """
        self.max_kept = 0
        self.total_kept = 0
        L = self.L
        mps = self.move_center_left(mps, 0)
        A, R = dict(mps.A), dict(mps.R)
        lb, rb = dict(mps.lbonds), dict(mps.rbonds)
        lblocks = {0: vacuum_block(2 * L)}
        rblocks = {L: vacuum_block(2 * L)}
        for p in range(L - 1, 1, -1):
            Rp = enlarge_right(self.sites[p], rblocks[p + 1], self.t, self.w)
            rblocks[p] = project_block(Rp, R[p].reshape(rb[p].dim, -1), rb[p].n, rb[p].s, left=False)
        psi = mps.psi
        energies, terrs = [], []
        for _ in range(nsweeps):
            maxerr, E = 0.0, None
            order = [(l, +1) for l in range(0, L - 2)] + [(l, -1) for l in range(L - 2, 0, -1)]
            for l, d in order:
                Lp = enlarge_left(lblocks[l], self.sites[l], self.t, self.w)
                Rp = enlarge_right(self.sites[l + 1], rblocks[l + 2], self.t, self.w)
                heff = Heff(Lp, Rp, self.t, self.w, self.N, self.two_sz, self.e_core)
                DX, DY = psi.shape[0], psi.shape[3]
                E, x = lowest_eig(heff, to_mat(psi), tol=tol)
                blocks = svd_sectors(x, Lp.n, Lp.s, Rp.n, Rp.s, self.N, self.two_sz)
                Dk = dbss_bond_dimension(blocks, trunc_eps, D_min, D) if trunc_eps > 0 else D
                kept, disc = select_kept(blocks, Dk)
                self.max_kept = max(self.max_kept, sum(len(v) for v in kept.values()))
                self.total_kept += sum(len(v) for v in kept.values())
                maxerr = max(maxerr, disc)
                if d > 0:
                    bnew, U, SV = left_factor(blocks, kept, Lp.dim, Rp.dim)
                    A[l] = U.reshape(DX, 4, bnew.dim)
                    lb[l + 1] = bnew
                    lblocks[l + 1] = project_block(Lp, U, bnew.n, bnew.s, left=True)
                    psi = np.einsum("ajb,bkc->ajkc", SV.reshape(bnew.dim, 4, DY), R.pop(l + 2))
                else:
                    bnew, Vt, US = right_factor(blocks, kept, Lp.dim, Rp.dim, self.N, self.two_sz)
                    R[l + 1] = Vt.reshape(bnew.dim, 4, DY)
                    rb[l + 1] = bnew
                    rblocks[l + 1] = project_block(Rp, Vt, bnew.n, bnew.s, left=False)
                    psi = np.einsum("cha,aib->chib", A.pop(l - 1), US.reshape(DX, 4, bnew.dim))
            energies.append(E)
            terrs.append(maxerr)
        lb0 = {0: lb[0]}
        rbo = {b: rb[b] for b in range(2, L + 1)}
        out = MPSU1(L, self.N, self.two_sz, 0, lb0, rbo, {}, {p: R[p] for p in range(2, L)}, psi)
        return energies, terrs, out
