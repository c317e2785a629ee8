"""Synthetic one- and two-electron integrals (seeded)."""

import struct

import numpy as np

BASE_SEED = 20260328


def open_shell_diagonal(n_docc=32, n_open=25, n_virt=45):
    """Orbital-energy profile of the large sextet workload: n_docc doubly occupied
    like orbitals, n_open near-degenerate open-shell orbitals (spread 0.05) and
    n_virt virtuals, in chain order."""
    return np.concatenate([
        np.linspace(-2.0, -1.0, n_docc),
        -0.5 + np.linspace(-0.025, 0.025, n_open),
        np.linspace(0.0, 0.5, n_virt),
    ])


def make_integrals(L, seed, diag=None, nvec=None):
    """Return (h, V) with h (L,L) symmetric and V (L,L,L,L) = sum_k B^k (x) B^k.

    The draw order is fixed: h upper triangle (i<j) row-major, then for each k
    the upper triangle of B^k including the diagonal, row-major.
    """
    rng = np.random.default_rng(seed)
    h = np.zeros((L, L))
    iu = np.triu_indices(L, 1)
    h[iu] = rng.normal(0.0, 0.1, size=len(iu[0]))
    h = h + h.T
    if diag is None:
        diag = np.linspace(-2.0, 0.5, L)
    h[np.arange(L), np.arange(L)] = np.asarray(diag, dtype=float)
    if nvec is None:
        nvec = 2 * L
    iu0 = np.triu_indices(L, 0)
    Bs = np.zeros((nvec, L, L))
    for k in range(nvec):
        b = np.zeros((L, L))
        b[iu0] = rng.normal(0.0, 1.0, size=len(iu0[0]))
        b = b + np.triu(b, 1).T
        Bs[k] = b * 0.5 ** (k / 4.0)
    Bf = Bs.reshape(nvec, L * L)
    V = (Bf.T @ Bf).reshape(L, L, L, L)
    return h, V


_MAGIC = b"QCINT001"


def write_integrals(path, h, V, N, two_s, seed, e_core=0.0):
    """Binary file: magic, header (L, N, 2S, seed as int64; e_core f64), h, V."""
    L = h.shape[0]
    with open(path, "wb") as f:
        f.write(_MAGIC)
        f.write(struct.pack("<qqqqd", L, N, two_s, seed, e_core))
        f.write(np.ascontiguousarray(h, dtype="<f8").tobytes())
        f.write(np.ascontiguousarray(V, dtype="<f8").tobytes())


def read_integrals(path):
    with open(path, "rb") as f:
        if f.read(8) != _MAGIC:
            raise ValueError("not an integral file")
        L, N, two_s, seed, e_core = struct.unpack("<qqqqd", f.read(40))
        h = np.frombuffer(f.read(8 * L * L), dtype="<f8").reshape(L, L).copy()
        V = np.frombuffer(f.read(8 * L ** 4), dtype="<f8").reshape(L, L, L, L).copy()
    return dict(L=L, N=N, two_s=two_s, seed=seed, e_core=e_core, h=h, V=V)
