"""Quantum-number sector structure and raw random entries of an initial MPS.

Only shapes and random draws live here (no method arithmetic): which
(N, S) or (N, 2Sz) sectors a bond carries, their dimensions, and i.i.d. normal
numbers for every allowed block. Orthonormalisation is the method's job and is
done independently by the oracle and by the CUDA library.

Symmetries
  SYM_U1  : U(1)xU(1), sector label (n, 2Sz), site states 0, up, down, updown.
  SYM_SU2 : SU(2),     sector label (n, 2S),  site multiplets 0, 1/2, 2.

Bond labels are block-local: a bond left of the two-site centre carries the
quantum numbers of the block to its left, a bond right of the centre those of
the block to its right. Because every site is identical, the structure of the
right block of L-b sites equals the left structure of bond L-b.

Sector rule at a bond with b sites on the labelled side (deterministic):
  cap(q)   = min(exact number of block states/multiplets with q,
                 number of complementary-block states that couple q to the target,
                 product dimension reachable from the neighbouring bond)
  w(q)     = cap(q) * exp(-(n - N b/L)^2 / (2*3^2)) * exp(-(s/2)^2 / (2*1.5^2))
  the bond dimension min(D, sum cap) is split in proportion to w by water
  filling with caps, then floors plus largest remainders (ties: smaller
  (n, s) first); a final right-to-left pass caps every sector by the number of
  states it can continue into.
"""

import math
from functools import lru_cache

import numpy as np

SYM_U1 = 0
SYM_SU2 = 1


def site_qns(sym):
    if sym == SYM_U1:
        return [(0, 0), (1, 1), (1, -1), (2, 0)]
    return [(0, 0), (1, 1), (2, 0)]


def fuse(sym, a, b):
    """Labels reachable by coupling a and b."""
    if sym == SYM_U1:
        return [(a[0] + b[0], a[1] + b[1])]
    lo, hi = abs(a[1] - b[1]), a[1] + b[1]
    return [(a[0] + b[0], s) for s in range(lo, hi + 1, 2)]


@lru_cache(maxsize=None)
def _counts(sym, nsites):
    """Exact number of states (U1) or multiplets (SU2) of nsites sites per label."""
    cur = {(0, 0): 1}
    for _ in range(nsites):
        nxt = {}
        for q, c in cur.items():
            for s in site_qns(sym):
                for r in fuse(sym, q, s):
                    nxt[r] = nxt.get(r, 0) + c
        cur = nxt
    return dict(cur)


def _complement_count(sym, L, b, q, N, two_s):
    """Number of states of the other L-b sites that couple q to the target."""
    cnt = _counts(sym, L - b)
    tot = 0
    for r, c in cnt.items():
        if (N, two_s) in fuse(sym, q, r):
            tot += c
    return tot


def _allocate(D, caps, weights):
    keys = sorted(caps)
    total_cap = sum(caps[k] for k in keys)
    Dt = min(D, total_cap)
    alloc = {k: 0.0 for k in keys}
    free = [k for k in keys if caps[k] > 0 and weights[k] > 0]
    remaining = float(Dt)
    while free and remaining > 1e-12:
        wsum = sum(weights[k] for k in free)
        over = []
        for k in free:
            share = remaining * weights[k] / wsum
            if alloc[k] + share >= caps[k]:
                over.append(k)
        if not over:
            for k in free:
                alloc[k] += remaining * weights[k] / wsum
            remaining = 0.0
            break
        for k in over:
            remaining -= caps[k] - alloc[k]
            alloc[k] = float(caps[k])
            free.remove(k)
    ints = {k: int(math.floor(alloc[k] + 1e-9)) for k in keys}
    left = Dt - sum(ints.values())
    order = sorted(keys, key=lambda k: (-(alloc[k] - ints[k]), k))
    for k in order:
        if left <= 0:
            break
        if ints[k] < caps[k]:
            ints[k] += 1
            left -= 1
    return {k: v for k, v in ints.items() if v > 0}


@lru_cache(maxsize=None)
def _structure(L, N, two_s, D, sym):
    bonds = [None] * (L + 1)
    bonds[0] = {(0, 0): 1}
    bonds[L] = {(N, two_s): 1}
    for b in range(1, L):
        prod = {}
        for q, d in bonds[b - 1].items():
            for s in site_qns(sym):
                for r in fuse(sym, q, s):
                    prod[r] = prod.get(r, 0) + d
        cnt = _counts(sym, b)
        caps, weights = {}, {}
        for q, c in cnt.items():
            cap = min(c, _complement_count(sym, L, b, q, N, two_s), prod.get(q, 0))
            if cap <= 0:
                continue
            caps[q] = cap
            n, s = q
            weights[q] = cap * math.exp(-((n - N * b / L) ** 2) / 18.0) * \
                math.exp(-((s / 2.0) ** 2) / (2 * 1.5 ** 2))
        bonds[b] = _allocate(D, caps, weights)
    for b in range(L - 1, 0, -1):
        for q in list(bonds[b]):
            cont = 0
            for s in site_qns(sym):
                for r in fuse(sym, q, s):
                    cont += bonds[b + 1].get(r, 0)
            bonds[b][q] = min(bonds[b][q], cont)
            if bonds[b][q] <= 0:
                del bonds[b][q]
    return tuple(tuple(sorted(d.items())) for d in bonds)


def mps_structure(L, N, two_s, D, sym):
    """Left-labelled sector dimensions for bonds 0..L (bond b: b sites on the left).

    Returns a list of dicts {label: dim}. Bond 0 is the vacuum, bond L the target.
    """
    return [dict(t) for t in _structure(L, N, two_s, D, sym)]


def random_mps_blocks(L, N, two_s, D, sym, seed, center):
    """Raw random MPS around the two-site centre (center, center+1).

    Returns a dict with
      left_bonds[b]  for b = 0..center      (left labels, {label: dim})
      right_bonds[b] for b = center+2..L    (labels of the block of sites b..L-1)
      left[p]  for p < center:   {(qL, s, qR): array (dL, dR)}    qR in fuse(qL, s)
      right[p] for p > center+1: {(qnew, s, qR): array (dnew, dR)} qnew in fuse(s, qR)
      psi: U1  {(qX, i, j, qY): array (dX, dY)}
           SU2 {(qX, i, sL, j, qY, sR): array (dX, dY)}, with sL (sR) the
           coupled spin of qX (x) i (of j (x) qY) and sL (x) sR containing the target.
    Draw order: left sites ascending, right sites descending, then psi; within a
    tensor blocks sorted by key, each block row-major.
    """
    struct = mps_structure(L, N, two_s, D, sym)
    left_bonds = {b: struct[b] for b in range(0, center + 1)}
    right_bonds = {}
    for b in range(center + 2, L):
        right_bonds[b] = dict(struct[L - b])
    right_bonds[L] = {(0, 0): 1}
    rng = np.random.default_rng(seed)
    sq = site_qns(sym)
    left = {}
    for p in range(center):
        keys = []
        for qL in sorted(left_bonds[p]):
            for si, s in enumerate(sq):
                for qR in fuse(sym, qL, s):
                    if qR in left_bonds[p + 1]:
                        keys.append((qL, si, qR))
        left[p] = {k: rng.normal(size=(left_bonds[p][k[0]], left_bonds[p + 1][k[2]]))
                   for k in sorted(keys)}
    right = {}
    for p in range(L - 1, center + 1, -1):
        keys = []
        for qR in sorted(right_bonds[p + 1]):
            for si, s in enumerate(sq):
                for qn in fuse(sym, s, qR):
                    if qn in right_bonds[p]:
                        keys.append((qn, si, qR))
        right[p] = {k: rng.normal(size=(right_bonds[p][k[0]], right_bonds[p + 1][k[2]]))
                    for k in sorted(keys)}
    keys = []
    target = (N, two_s)
    for qX in left_bonds[center]:
        for i, si in enumerate(sq):
            for qL in fuse(sym, qX, si):
                for qY in right_bonds[center + 2]:
                    for j, sj in enumerate(sq):
                        for qR in fuse(sym, sj, qY):
                            if target in fuse(sym, qL, qR):
                                if sym == SYM_U1:
                                    keys.append((qX, i, j, qY))
                                else:
                                    keys.append((qX, i, qL[1], j, qY, qR[1]))
    psi = {}
    for k in sorted(set(keys)):
        qX = k[0]
        qY = k[3] if sym == SYM_U1 else k[4]
        psi[k] = rng.normal(size=(left_bonds[center][qX], right_bonds[center + 2][qY]))
    return dict(L=L, N=N, two_s=two_s, D=D, sym=sym, center=center,
                left_bonds=left_bonds, right_bonds=right_bonds,
                left=left, right=right, psi=psi)


def workload(name):
    """Named synthetic workloads (sizes of the paper's active spaces)."""
    from .integrals import BASE_SEED, open_shell_diagonal
    table = {
        # U(1)xU(1), L=10, N=10, Sz=0, D=64 (FCI dimension 63504)
        "u1_L10_N10_D64": dict(L=10, N=10, two_s=0, D=64, sym=SYM_U1,
                               int_seed=BASE_SEED + 1, mps_seed=BASE_SEED + 1001),
        # CAS(54,36)-shaped singlet, SU(2)
        "su2_L36_N54_S0_D1024": dict(L=36, N=54, two_s=0, D=1024, sym=SYM_SU2,
                                     int_seed=BASE_SEED + 2, mps_seed=BASE_SEED + 1002),
        "su2_L36_N54_S0_D2048": dict(L=36, N=54, two_s=0, D=2048, sym=SYM_SU2,
                                     int_seed=BASE_SEED + 2, mps_seed=BASE_SEED + 1002),
        "su2_L36_N54_S0_D4096": dict(L=36, N=54, two_s=0, D=4096, sym=SYM_SU2,
                                     int_seed=BASE_SEED + 2, mps_seed=BASE_SEED + 1002),
        # CAS(89,102)-shaped sextet, SU(2), open-shell orbital profile
        "su2_L102_N89_S5_D2048": dict(L=102, N=89, two_s=5, D=2048, sym=SYM_SU2,
                                      int_seed=BASE_SEED + 5, mps_seed=BASE_SEED + 1005,
                                      diag=open_shell_diagonal()),
    }
    return dict(table[name])


def batched_instances(n=16, seed=99):
    """Independent problems of the batched workload: L uniform in 12..24,
    N = L, 2S = N mod 2, D uniform in {128, 256, 512}, integral seeds
    100, 101, ..., MPS seeds 1100, 1101, ..."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(rng.integers(12, 25))
        D = int(rng.choice([128, 256, 512]))
        out.append(dict(L=L, N=L, two_s=L % 2, D=D, int_seed=100 + i, mps_seed=1100 + i))
    return out
