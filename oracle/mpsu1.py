"""Dense U(1)xU(1) MPS with quantum-number labels (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The MPS of Eq. (mps) of the Method section, written around a two-site centre
(l, l+1):
    |Psi> = sum psi[a, i, j, b] |a>_L |i>_l |j>_{l+1} |b>_R
with |a'>_L = sum A_p[a, i, a'] |a>_L |i>_p            (left-canonical, p < l)
     |b'>_R = sum R_p[b', j, b] |j>_p |b>_R            (right-canonical, p > l+1)
Bond labels are block-local: left bonds carry (n, 2Sz) of the block on their
left, right bonds those of the block on their right. Tensors are dense arrays;
entries that break the labels are exactly zero.

Site basis index: 0 = |0>, 1 = a+_up|0>, 2 = a+_dn|0>, 3 = a+_up a+_dn|0>.
"""

import numpy as np

SITE_QN = [(0, 0), (1, 1), (1, -1), (2, 0)]
SITE_N = np.array([q[0] for q in SITE_QN])
SITE_S = np.array([q[1] for q in SITE_QN])


class Bond:
    """Sorted list of states with labels; sectors map label -> (start, dim)."""

    def __init__(self, sectors):
        self.labels = []
        self.sectors = {}
        pos = 0
        for q, d in sorted(sectors.items()):
            self.sectors[q] = (pos, d)
            self.labels += [q] * d
            pos += d
        self.dim = pos
        self.n = np.array([q[0] for q in self.labels], dtype=int)
        self.s = np.array([q[1] for q in self.labels], dtype=int)

    def sector_dims(self):
        return {q: d for q, (st, d) in self.sectors.items()}


def dense_left(raw, bl, br):
    A = np.zeros((bl.dim, 4, br.dim))
    for (qL, i, qR), blk in raw.items():
        a0, da = bl.sectors[qL]
        b0, db = br.sectors[qR]
        A[a0:a0 + da, i, b0:b0 + db] = blk
    return A


def dense_right(raw, bnew, bR):
    R = np.zeros((bnew.dim, 4, bR.dim))
    for (qn, j, qR), blk in raw.items():
        a0, da = bnew.sectors[qn]
        b0, db = bR.sectors[qR]
        R[a0:a0 + da, j, b0:b0 + db] = blk
    return R


def left_qr(M, bl, br):
    """Per-sector QR of M[(a i), a'] (a' in sector q takes rows with n(a)+n(i)=q).

    Returns the left-canonical tensor Q and the carry matrix C with M = Q C.
    """
    Dl, _, Dr = M.shape
    rows_n = (bl.n[:, None] + SITE_N[None, :]).reshape(-1)
    rows_s = (bl.s[:, None] + SITE_S[None, :]).reshape(-1)
    Mf = M.reshape(Dl * 4, Dr)
    Q = np.zeros_like(Mf)
    C = np.zeros((Dr, Dr))
    for q, (c0, dc) in br.sectors.items():
        rows = np.nonzero((rows_n == q[0]) & (rows_s == q[1]))[0]
        cols = np.arange(c0, c0 + dc)
        if len(rows) < dc:
            raise ValueError("sector larger than its product space")
        qm, rm = np.linalg.qr(Mf[np.ix_(rows, cols)])
        Q[np.ix_(rows, cols)] = qm
        C[np.ix_(cols, cols)] = rm
    return Q.reshape(Dl, 4, Dr), C


def right_lq(M, bnew, bR):
    """Per-sector LQ of M[a', (j b)]; a' labels are fused from site j and block b."""
    Dn, _, DR = M.shape
    cols_n = (SITE_N[:, None] + bR.n[None, :]).reshape(-1)
    cols_s = (SITE_S[:, None] + bR.s[None, :]).reshape(-1)
    Mf = M.reshape(Dn, 4 * DR)
    Q = np.zeros_like(Mf)
    C = np.zeros((Dn, Dn))
    for q, (r0, dr) in bnew.sectors.items():
        cols = np.nonzero((cols_n == q[0]) & (cols_s == q[1]))[0]
        rows = np.arange(r0, r0 + dr)
        if len(cols) < dr:
            raise ValueError("sector larger than its product space")
        qm, rm = np.linalg.qr(Mf[np.ix_(rows, cols)].T)
        Q[np.ix_(rows, cols)] = qm.T
        C[np.ix_(rows, rows)] = rm.T
    return Q.reshape(Dn, 4, DR), C


class MPSU1:
    """Mixed-canonical MPS around the two-site centre (l, l+1)."""

    def __init__(self, L, N, two_sz, center, lbonds, rbonds, A, R, psi):
        self.L, self.N, self.two_sz, self.center = L, N, two_sz, center
        self.lbonds = lbonds      # dict b -> Bond, b = 0..center
        self.rbonds = rbonds      # dict b -> Bond, b = center+2..L
        self.A = A                # dict p -> (D_p, 4, D_p+1), p < center
        self.R = R                # dict p -> (D'_p, 4, D'_p+1), p > center+1
        self.psi = psi            # (D_X, 4, 4, D_Y)

    @classmethod
    def from_raw(cls, raw):
        L, N, two_sz, c = raw["L"], raw["N"], raw["two_s"], raw["center"]
        lb = {b: Bond(d) for b, d in raw["left_bonds"].items()}
        rb = {b: Bond(d) for b, d in raw["right_bonds"].items()}
        A, R = {}, {}
        carry = np.ones((1, 1))
        for p in range(c):
            M = np.einsum("xa,aib->xib", carry, dense_left(raw["left"][p], lb[p], lb[p + 1]))
            A[p], carry = left_qr(M, lb[p], lb[p + 1])
        cl = carry
        carry = np.ones((1, 1))
        for p in range(L - 1, c + 1, -1):
            M = np.einsum("aib,by->aiy", dense_right(raw["right"][p], rb[p], rb[p + 1]), carry)
            R[p], carry = right_lq(M, rb[p], rb[p + 1])
        cr = carry
        bX, bY = lb[c], rb[c + 2]
        psi = np.zeros((bX.dim, 4, 4, bY.dim))
        for (qX, i, j, qY), blk in raw["psi"].items():
            a0, da = bX.sectors[qX]
            b0, db = bY.sectors[qY]
            psi[a0:a0 + da, i, j, b0:b0 + db] = blk
        psi = np.einsum("xa,aijb,by->xijy", cl, psi, cr)
        psi /= np.linalg.norm(psi)
        return cls(L, N, two_sz, c, lb, rb, A, R, psi)

    # ---- flat block layout of the two-site wavefunction --------------------
    def psi_keys(self):
        """Sorted sub-block keys (qX, i, j, qY) coupled to the target."""
        bX, bY = self.lbonds[self.center], self.rbonds[self.center + 2]
        keys = []
        for qX in bX.sectors:
            for i, si in enumerate(SITE_QN):
                for j, sj in enumerate(SITE_QN):
                    for qY in bY.sectors:
                        if (qX[0] + si[0] + sj[0] + qY[0] == self.N and
                                qX[1] + si[1] + sj[1] + qY[1] == self.two_sz):
                            keys.append((qX, i, j, qY))
        return sorted(keys)

    def psi_to_flat(self, psi=None):
        psi = self.psi if psi is None else psi
        bX, bY = self.lbonds[self.center], self.rbonds[self.center + 2]
        out = []
        for qX, i, j, qY in self.psi_keys():
            a0, da = bX.sectors[qX]
            b0, db = bY.sectors[qY]
            out.append(psi[a0:a0 + da, i, j, b0:b0 + db].reshape(-1))
        return np.concatenate(out) if out else np.zeros(0)

    def psi_from_flat(self, flat):
        bX, bY = self.lbonds[self.center], self.rbonds[self.center + 2]
        psi = np.zeros((bX.dim, 4, 4, bY.dim))
        pos = 0
        for qX, i, j, qY in self.psi_keys():
            a0, da = bX.sectors[qX]
            b0, db = bY.sectors[qY]
            psi[a0:a0 + da, i, j, b0:b0 + db] = flat[pos:pos + da * db].reshape(da, db)
            pos += da * db
        if pos != len(flat):
            raise ValueError("flat vector has the wrong length")
        return psi

    # ---- expansion to the determinant space ---------------------------------
    def left_states(self):
        """Lvec[config of sites 0..l-1, a] (site 0 is the most significant digit)."""
        v = np.ones((1, 1))
        for p in range(self.center):
            v = np.einsum("ca,aib->cib", v, self.A[p]).reshape(-1, self.A[p].shape[2])
        return v

    def right_states(self):
        """Rvec[b, config of sites l+2..L-1]."""
        v = np.ones((1, 1))
        for p in range(self.L - 1, self.center + 1, -1):
            v = np.einsum("bjc,cx->bjx", self.R[p], v).reshape(self.R[p].shape[0], -1)
        return v

    def config_to_det(self):
        """Determinant bit string of every site configuration (base-4 digits)."""
        L = self.L
        nconf = 4 ** L
        bits = np.zeros(nconf, dtype=np.uint64)
        conf = np.arange(nconf, dtype=np.int64)
        for p in range(L - 1, -1, -1):
            d = conf % 4
            conf //= 4
            bits |= np.where((d == 1) | (d == 3), np.uint64(1) << np.uint64(2 * p), np.uint64(0))
            bits |= np.where((d == 2) | (d == 3), np.uint64(1) << np.uint64(2 * p + 1), np.uint64(0))
        return bits


class Projector:
    """Two-site tangent map P: psi -> determinant vector (projection definition).

    H_eff psi = P^T H_FCI P psi, exact for any bond dimension. P is an
    isometry when the environment tensors are canonical. The product of site
    configurations is the determinant with modes in chain order, so P carries
    no extra fermion signs.
    """

    def __init__(self, mps, space):
        self.mps = mps
        self.space = space
        self.Lv = mps.left_states()
        self.Rv = mps.right_states()
        idx, ok = space.index(mps.config_to_det())
        self.map = np.where(ok, idx, -1)

    def apply(self, psi):
        full = np.einsum("ca,aijb,bd->cijd", self.Lv, psi, self.Rv).reshape(-1)
        sel = self.map >= 0
        if np.abs(full[~sel]).max(initial=0.0) > 1e-12:
            raise ValueError("state leaves the determinant space")
        out = np.zeros(self.space.dim)
        out[self.map[sel]] = full[sel]
        return out

    def apply_t(self, vec):
        full = np.zeros(self.map.shape[0])
        sel = self.map >= 0
        full[sel] = vec[self.map[sel]]
        full = full.reshape(self.Lv.shape[0], 4, 4, self.Rv.shape[1])
        return np.einsum("ca,cijd,bd->aijb", self.Lv, full, self.Rv)

    def heff(self, fci, psi):
        return self.apply_t(fci.apply(self.apply(psi)))


def export_abi(mps):
    """Flatten a mixed-canonical MPS into the C-ABI import layout.

    Returns (bond_nsec, bond_sec, data) as numpy arrays: left sites as
    product-sector matrices U_q [(x, i) rows, kept states], right sites as
    V_q [kept states, (j, y) columns], then the two-site wavefunction.
    """
    L, c = mps.L, mps.center
    bonds = {}
    for b in range(0, c + 1):
        bonds[b] = mps.lbonds[b]
    for b in range(c + 2, L + 1):
        bonds[b] = mps.rbonds[b]
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
        bl, br = mps.lbonds[p], mps.lbonds[p + 1]
        prods = {}
        for q, (x0, dx) in sorted(bl.sectors.items()):
            for i, si in enumerate(SITE_QN):
                lab = (q[0] + si[0], q[1] + si[1])
                prods.setdefault(lab, []).append((q, i))
        for lab in sorted(prods):
            if lab not in br.sectors:
                continue
            c0, dc = br.sectors[lab]
            rows = [mps.A[p][bl.sectors[q][0]:bl.sectors[q][0] + bl.sectors[q][1], i, c0:c0 + dc]
                    for q, i in sorted(prods[lab], key=lambda t: (t[0], t[1]))]
            data.append(np.concatenate(rows, axis=0).reshape(-1))
    for p in range(c + 2, L):
        bn, bR = mps.rbonds[p], mps.rbonds[p + 1]
        prods = {}
        for j, sj in enumerate(SITE_QN):
            for q, (y0, dy) in sorted(bR.sectors.items()):
                lab = (sj[0] + q[0], sj[1] + q[1])
                prods.setdefault(lab, []).append((j, q))
        for lab in sorted(prods):
            if lab not in bn.sectors:
                continue
            r0, dr = bn.sectors[lab]
            cols = [mps.R[p][r0:r0 + dr, j, bR.sectors[q][0]:bR.sectors[q][0] + bR.sectors[q][1]]
                    for j, q in sorted(prods[lab], key=lambda t: (t[0], t[1]))]
            data.append(np.concatenate(cols, axis=1).reshape(-1))
    data.append(mps.psi_to_flat())
    return (np.array(nsec, dtype=np.int32), np.array(sec, dtype=np.int32),
            np.concatenate(data).astype(np.float64))
