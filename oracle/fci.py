"""Full configuration interaction in the determinant basis (plain definition).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The Hamiltonian is the ab initio active-space Hamiltonian that the paper's
DMRG (Method section, Eq. (mps)) approximates:
    H = sum_pq h_pq E_pq + 1/2 sum_pqrs V_pqrs (E_pq E_rs - delta_qr E_ps)
with chemist-notation V_pqrs = (pq|rs). Determinants |n> = prod_k (a+_k)^{n_k}|vac>
in increasing spin-orbital index k = 2p + sigma (sigma = 0 up, 1 down).

Everything below is the literal second-quantised action of E_pq on bit
strings, with the Jordan-Wigner sign counted as the number of occupied modes
passed over.
"""

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def popcount(x):
    x = np.asarray(x, dtype=np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    y = x.copy()
    while np.any(y):
        c += (y & np.uint64(1)).astype(np.int64)
        y >>= np.uint64(1)
    return c


class DetSpace:
    """All determinants of L spatial orbitals with N electrons and 2Sz = two_sz."""

    def __init__(self, L, N, two_sz):
        if (N + two_sz) % 2:
            raise ValueError("N and 2Sz parity mismatch")
        nup = (N + two_sz) // 2
        ndn = (N - two_sz) // 2
        if nup < 0 or ndn < 0 or nup > L or ndn > L:
            raise ValueError("empty determinant space")
        self.L, self.N, self.two_sz = L, N, two_sz
        dets = []
        for up in itertools.combinations(range(L), nup):
            for dn in itertools.combinations(range(L), ndn):
                b = 0
                for p in up:
                    b |= 1 << (2 * p)
                for p in dn:
                    b |= 1 << (2 * p + 1)
                dets.append(b)
        self.dets = np.array(sorted(dets), dtype=np.uint64)
        self.dim = len(self.dets)

    def index(self, bits):
        idx = np.searchsorted(self.dets, bits)
        idx = np.minimum(idx, self.dim - 1)
        ok = self.dets[idx] == bits
        return idx, ok


def excitation_matrix(space_from, space_to, k_cre, k_ann):
    """Sparse matrix of a+_{k_cre} a_{k_ann} from space_from to space_to."""
    d = space_from.dets
    one = np.uint64(1)
    mk_a = one << np.uint64(k_ann)
    mk_c = one << np.uint64(k_cre)
    has = (d & mk_a) != 0
    src = np.nonzero(has)[0]
    b = d[src]
    s1 = popcount(b & (mk_a - one))     # modes passed by a_{k_ann}
    b = b & ~mk_a
    ok = (b & mk_c) == 0
    src, b, s1 = src[ok], b[ok], s1[ok]
    s2 = popcount(b & (mk_c - one))     # modes passed by a+_{k_cre}
    b = b | mk_c
    sign = np.where((s1 + s2) % 2 == 0, 1.0, -1.0)
    tgt, found = space_to.index(b)
    return sp.csr_matrix((sign[found], (tgt[found], src[found])),
                         shape=(space_to.dim, space_from.dim))


class FCI:
    """Hamiltonian action, ground state, spin and reduced density matrices."""

    def __init__(self, h, V, N, two_sz, e_core=0.0):
        self.h = np.asarray(h, float)
        self.V = np.asarray(V, float)
        self.L = self.h.shape[0]
        self.N, self.two_sz, self.e_core = N, two_sz, e_core
        self.space = DetSpace(self.L, N, two_sz)
        L = self.L
        # E_pq = a+_{p up} a_{q up} + a+_{p dn} a_{q dn}
        self.E = [[None] * L for _ in range(L)]
        for p in range(L):
            for q in range(L):
                self.E[p][q] = (excitation_matrix(self.space, self.space, 2 * p, 2 * q)
                                + excitation_matrix(self.space, self.space, 2 * p + 1, 2 * q + 1)).tocsr()
        # one-body part with the -1/2 sum_q V_pqqs E_ps term folded in
        self.k1 = self.h - 0.5 * np.einsum("pqqs->ps", self.V)

    def apply(self, c):
        """H c = sum_pq k_pq E_pq c + 1/2 sum_pq E_pq (sum_rs V_pqrs E_rs c) + e_core c."""
        L = self.L
        c = np.asarray(c, float)
        Y = np.stack([self.E[r][s] @ c for r in range(L) for s in range(L)])  # (L^2, dim)
        Z = self.V.reshape(L * L, L * L) @ Y
        out = self.e_core * c
        for p in range(L):
            for q in range(L):
                out = out + self.E[p][q] @ (self.k1[p, q] * c + 0.5 * Z[p * L + q])
        return out

    def matrix(self):
        """Explicit sparse H (small spaces only)."""
        L = self.L
        H = sp.csr_matrix((self.space.dim, self.space.dim))
        for p in range(L):
            for q in range(L):
                H = H + self.k1[p, q] * self.E[p][q]
        for p in range(L):
            for q in range(L):
                for r in range(L):
                    for s in range(L):
                        v = self.V[p, q, r, s]
                        if v != 0.0:
                            H = H + 0.5 * v * (self.E[p][q] @ self.E[r][s])
        return (H + self.e_core * sp.identity(self.space.dim)).tocsr()

    def spin_plus(self):
        """S_+ from this Sz space to the Sz+1 space."""
        up = DetSpace(self.L, self.N, self.two_sz + 2)
        Sp = None
        for p in range(self.L):
            m = excitation_matrix(self.space, up, 2 * p, 2 * p + 1)
            Sp = m if Sp is None else Sp + m
        return Sp.tocsr()

    def s2_apply(self, c):
        """S^2 = S_- S_+ + Sz (Sz + 1)."""
        sz = self.two_sz / 2.0
        if not hasattr(self, "_Sp"):
            try:
                self._Sp = self.spin_plus()
            except ValueError:
                self._Sp = None
        out = sz * (sz + 1.0) * c
        if self._Sp is not None:
            out = out + self._Sp.T @ (self._Sp @ c)
        return out

    def ground_state(self, two_s=None, penalty=10.0, tol=1e-12):
        """Lowest eigenpair; with two_s given, of H + penalty (S^2 - S(S+1))^2."""
        dim = self.space.dim
        if two_s is None:
            mv = self.apply
        else:
            ss = (two_s / 2.0) * (two_s / 2.0 + 1.0)

            def mv(c):
                t = self.s2_apply(c) - ss * c
                return self.apply(c) + penalty * (self.s2_apply(t) - ss * t)
        if dim <= 400:
            M = np.column_stack([mv(np.eye(dim)[:, i]) for i in range(dim)])
            w, v = np.linalg.eigh(0.5 * (M + M.T))
            c = v[:, 0]
        else:
            op = spla.LinearOperator((dim, dim), matvec=mv, dtype=float)
            w, v = spla.eigsh(op, k=1, which="SA", tol=tol, v0=np.ones(dim) / np.sqrt(dim))
            c = v[:, 0]
        c = c / np.linalg.norm(c)
        return float(c @ self.apply(c)), c

    def rdm12(self, c):
        """gamma_pq = <E_pq>, Gamma_pqrs = <E_pq E_rs> - delta_qr <E_ps>."""
        L = self.L
        gamma = np.array([[c @ (self.E[p][q] @ c) for q in range(L)] for p in range(L)])
        Y = np.stack([self.E[r][s] @ c for r in range(L) for s in range(L)])  # E_rs c
        G = np.zeros((L, L, L, L))
        for p in range(L):
            for q in range(L):
                G[p, q] = (Y[q * L + p] @ Y.T).reshape(L, L)   # (E_qp c).(E_rs c)
        for q in range(L):
            G[:, q, q, :] -= gamma
        return gamma, G
