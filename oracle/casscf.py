"""Plain orbital-optimisation pieces of DMRG-SCF (oracle).

TEST INFRASTRUCTURE (oracle): imported only by tests/, smoke() and bench.py's
CPU-baseline leg.

The paper couples its spin-adapted DMRG to a CAS-SCF orbital optimisation (New benchmark
system section): the active-space solver supplies the one- and two-particle density
matrices, and the orbitals are rotated to lower the energy. The formulas are not printed
there; this module holds their plain definitions, written out so that each can be checked
by eye, for the tests of the library's orbital gradient and integral rotation:

* orbitals are the columns of an orthogonal U acting on the given basis,
  h' = U^T h U, (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd);
* core orbitals 0..ncore-1 are doubly occupied, active orbitals ncore..ncore+nact-1 carry the
  density matrices, the rest are empty; the frozen-core energy and active integrals are
  E_core = sum_c 2 h_cc + sum_cd (2 (cc|dd) - (cd|dc)),
  h_act_tu = h_tu + sum_c (2 (tu|cc) - (tc|cu)),  V_act = (tu|vw) over active indices;
* the energy at fixed density matrices is E = E_core + sum h_act gamma + 1/2 sum V_act Gamma,
  with gamma_tu = <E_tu> and Gamma_tuvw = <E_tu E_vw - delta_uv E_tw>;
* the orbital gradient is the derivative of E(expm(kappa)) at kappa = 0 for the
  antisymmetric generator kappa, one parameter per pair p > q (kappa_pq = -kappa_qp),
  taken here by central differences of that energy.

Nothing here is shared with the library; numpy and scipy only.
"""
import numpy as np
from scipy.linalg import expm


def rotate(h, V, U):
    """Integrals in the orbitals given by the columns of U."""
    h2 = U.T @ h @ U
    V2 = np.einsum("abcd,ap,bq,cr,ds->pqrs", V, U, U, U, U, optimize=True)
    return h2, V2


def active_space(h, V, ncore, nact):
    """(E_core, h_act, V_act) of the frozen-core active space."""
    c = slice(0, ncore)
    a = slice(ncore, ncore + nact)
    e_core = 2.0 * np.trace(h[c, c])
    for i in range(ncore):
        for j in range(ncore):
            e_core += 2.0 * V[i, i, j, j] - V[i, j, j, i]
    h_act = h[a, a].copy()
    for i in range(ncore):
        h_act += 2.0 * V[a, a, i, i] - V[a, i, i, a]
    return e_core, h_act, V[a, a, a, a].copy()


def energy(h, V, ncore, nact, gamma, Gamma):
    e_core, h_act, V_act = active_space(h, V, ncore, nact)
    return e_core + np.sum(h_act * gamma) + 0.5 * np.sum(V_act * Gamma)


def energy_rotated(h, V, ncore, nact, gamma, Gamma, kappa):
    return energy(*rotate(h, V, expm(kappa)), ncore, nact, gamma, Gamma)


def gradient_fd(h, V, ncore, nact, gamma, Gamma, step=1e-5):
    """G[p, q] = dE/dkappa_pq for p > q (kappa_qp = -kappa_pq), central differences;
    G is returned antisymmetric (G[q, p] = -G[p, q])."""
    n = h.shape[0]
    G = np.zeros((n, n))
    for p in range(n):
        for q in range(p):
            k = np.zeros((n, n))
            k[p, q], k[q, p] = step, -step
            ep = energy_rotated(h, V, ncore, nact, gamma, Gamma, k)
            em = energy_rotated(h, V, ncore, nact, gamma, Gamma, -k)
            G[p, q] = (ep - em) / (2 * step)
            G[q, p] = -G[p, q]
    return G
