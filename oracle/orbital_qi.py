"""Orbital entanglement from a determinant-space vector (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The paper pre-optimises its chain ordering with quantum-information protocols
(Numerical procedure section): one- and two-orbital entropies, the mutual information
of orbital pairs and an ordering from it. Their plain definitions, for a state given
as FCI coefficients over determinants |D> = prod_k (a+_k)^{n_k}|vac> (k = 2p + sigma):

* write each determinant with the creation operators of orbitals i and j moved to the
  front, |D> = s(D) |x_i y_j> (x) |rest>, s(D) the sign of that reordering, x, y in
  {|0>, |up>, |dn>, |up dn> = a+_up a+_dn|0>};
* rho_ij[(x y), (x' y')] = sum over determinant pairs with the same rest of
  s(D) c_D s(D') c_D' (the partial trace over the other orbitals);
  rho_i likewise with orbital i alone; for a spin multiplet, the average of rho_ij over its
  2S + 1 components (the components of one multiplet give different rho_ij when S > 0);
* S = -sum lambda ln lambda over the eigenvalues; I_ij = S_i + S_j - S_ij;
* the ordering sorts the orbitals by the eigenvector of the second smallest eigenvalue
  (the Fiedler vector) of the graph Laplacian diag(sum_j I_ij) - I (Barcza et al. 2011,
  the protocol the paper cites for its chain topology).
"""
import numpy as np


def _occ(bits, p):
    """Site state of orbital p in a determinant: 0, 1 (up), 2 (dn), 3 (up dn)."""
    up = (bits >> (2 * p)) & 1
    dn = (bits >> (2 * p + 1)) & 1
    return int(up + 2 * dn) if not (up and dn) else 3


def _count_below(bits, k):
    return bin(bits & ((1 << k) - 1)).count("1")


def two_orbital_rdm(dets, c, i, j):
    """rho_ij (16 x 16, row 4 x + y) of the normalised state sum_D c_D |D>, i < j."""
    assert i < j
    c = np.asarray(c, float) / np.linalg.norm(c)
    mask = (3 << (2 * i)) | (3 << (2 * j))
    groups = {}
    for b, cd in zip(dets, c):
        b = int(b)
        if cd == 0.0:
            continue
        ni = ((b >> (2 * i)) & 1) + ((b >> (2 * i + 1)) & 1)
        nj = ((b >> (2 * j)) & 1) + ((b >> (2 * j + 1)) & 1)
        # move orbital i's operators past the occupied modes before it, then
        # orbital j's past the occupied modes before it other than orbital i's
        t = ni * _count_below(b, 2 * i) + nj * (_count_below(b, 2 * j) - ni)
        s = -1.0 if t & 1 else 1.0
        groups.setdefault(b & ~mask, []).append((4 * _occ(b, i) + _occ(b, j), s * cd))
    rho = np.zeros((16, 16))
    for items in groups.values():
        for r, a in items:
            for q, bb in items:
                rho[r, q] += a * bb
    return rho


def one_orbital_rdm(rho_ij, first=True):
    """rho_i (4 x 4) from rho_ij by tracing out the other orbital (first: keep i)."""
    r = rho_ij.reshape(4, 4, 4, 4)
    return np.einsum("xyzy->xz", r) if first else np.einsum("xyxz->yz", r)


def entropy(rho):
    w = np.linalg.eigvalsh(0.5 * (rho + rho.T))
    w = w[w > 1e-300]
    return float(-np.sum(w * np.log(w)))


def mutual_information(rho2, L):
    """(S_i, I_ij) from the two-orbital matrices rho2[i][j] (i < j)."""
    S1 = np.zeros(L)
    for i in range(L):
        if i + 1 < L:
            S1[i] = entropy(one_orbital_rdm(rho2[i][i + 1], first=True))
        else:
            S1[i] = entropy(one_orbital_rdm(rho2[i - 1][i], first=False))
    I = np.zeros((L, L))
    for i in range(L):
        for j in range(i + 1, L):
            I[i, j] = I[j, i] = S1[i] + S1[j] - entropy(rho2[i][j])
    return S1, I


def fiedler_order(I):
    """Orbitals sorted by the Fiedler vector of diag(sum_j I_ij) - I (ties by index).

    The eigenvector's sign is free; it is fixed here by making its first component of
    magnitude above 1e-8 of the largest negative."""
    I = np.array(I, float)
    np.fill_diagonal(I, 0.0)
    lap = np.diag(I.sum(axis=1)) - I
    w, v = np.linalg.eigh(lap)
    f = v[:, 1] / np.linalg.norm(v[:, 1])
    lead = np.flatnonzero(np.abs(f) > 1e-8 * np.abs(f).max())[0]
    if f[lead] > 0:
        f = -f
    return np.argsort(f, kind="stable"), f


def ordering_cost(I, order, eta=2.0):
    """sum_{i<j} I_ij |pos_i - pos_j|^eta, pos_i the position of orbital i in order."""
    L = len(order)
    pos = np.empty(L, int)
    pos[np.asarray(order)] = np.arange(L)
    return float(sum(I[i, j] * abs(pos[i] - pos[j]) ** eta for i in range(L) for j in range(i + 1, L)))


def best_order(I, eta=2.0):
    """The lowest-cost chain order by brute force over all permutations (small L only)."""
    import itertools
    L = I.shape[0]
    return min(itertools.permutations(range(L)), key=lambda o: ordering_cost(I, o, eta))


def multiplet_components(L, N, two_s, v):
    """[(dets, vector)] of the 2S + 1 components of the spin multiplet whose M = S component
    is v (a vector of DetSpace(L, N, two_s)): S_- = sum_p a+_{p dn} a_{p up} applied again and
    again, each result normalised."""
    from oracle.fci import DetSpace, excitation_matrix
    sp = DetSpace(L, N, two_s)
    cur = np.asarray(v, float) / np.linalg.norm(v)
    out = [(sp.dets, cur)]
    for m in range(two_s - 2, -two_s - 1, -2):
        sp2 = DetSpace(L, N, m)
        lower = sum(excitation_matrix(sp, sp2, 2 * p + 1, 2 * p) for p in range(L))
        cur = lower @ cur
        cur = cur / np.linalg.norm(cur)
        out.append((sp2.dets, cur))
        sp = sp2
    return out


def multiplet_rdm(L, N, two_s, v, i, j):
    """rho_ij averaged over the 2S + 1 components of the multiplet (independent of M)."""
    comps = multiplet_components(L, N, two_s, v)
    return sum(two_orbital_rdm(d, c, i, j) for d, c in comps) / len(comps)
