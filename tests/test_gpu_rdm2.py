"""2-RDM (dE/dV) through the C ABI: against the brute-force 2-RDM of the expanded MPS
vector (averaged over the 8 permutations of (pq|rs)), E = sum h gamma + 1/2 sum V Gamma,
the context restored afterwards, a central difference in one integral orbit, and the
autograd gradient dE/dV = 1/2 Gamma."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

AXES = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
        (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]


def _ctx(m, h, V):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import export_abi
    ensure_built()
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(m.N, m.two_sz)
    ctx.import_mps(m.L, m.center, *export_abi(m))
    ctx.build_env()
    return ctx


def test_rdm2_matches_expanded_vector():
    import torch
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1, Projector
    from paper_2603_28648_b300.autograd import DMRGEnergy
    L, N, D, c = 5, 5, 8, 1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    ctx = _ctx(m, h, V)
    psi0 = m.psi_to_flat()
    sig0 = ctx.apply_heff(psi0)
    G = ctx.rdm2(L)
    # the context is back to its integrals and environment
    sig1 = ctx.apply_heff(psi0)
    assert np.linalg.norm(sig1 - sig0) <= 1e-13 * np.linalg.norm(sig0)
    f = FCI(h, V, N, 1)
    v = Projector(m, f.space).apply(m.psi)
    g1, Gf = f.rdm12(v / np.linalg.norm(v))
    Gs = sum(Gf.transpose(a) for a in AXES) / 8.0
    assert np.abs(G - Gs).max() <= 1e-10
    # energy from the density matrices
    E = psi0 @ sig0 / (psi0 @ psi0)
    assert abs(np.sum(h * g1) + 0.5 * np.sum(V * G) - E) <= 1e-10 * abs(E)
    # central difference in one permutation orbit of V (E is linear in V at fixed MPS)
    p, qq, r, s = 0, 2, 1, 3
    dV = np.zeros_like(V)
    for a in AXES:
        idx = tuple(np.array((p, qq, r, s))[list(np.argsort(a))])
        dV[idx] = 1.0
    eps = 1e-6
    Es = []
    for sgn in (+1, -1):
        c2 = _ctx(m, h, V + sgn * eps * dV)
        Es.append(psi0 @ c2.apply_heff(psi0) / (psi0 @ psi0))
        c2.close()
    fd = (Es[0] - Es[1]) / (2 * eps)
    assert abs(fd - 0.5 * np.sum(dV * G)) <= 1e-7 * max(1.0, abs(fd))
    # autograd: dE/dV = 1/2 Gamma
    tV = torch.tensor(V, requires_grad=True)
    En = DMRGEnergy.apply(torch.tensor(psi0, device="cuda"), torch.tensor(h), tV, ctx)
    En.backward()
    assert np.abs(tV.grad.numpy() - 0.5 * G).max() <= 1e-12
    ctx.close()
