"""Adjoint of E(psi, h, V): dE/dpsi against finite differences, the 1-RDM
(dE/dh) against finite differences in h (E is linear in h at fixed MPS, so the
central difference is exact up to rounding), against the brute-force RDM of the
expanded MPS vector, and against FCI at exact bond dimension."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


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


def _setup(L=6, N=5, D=16, c=2):
    from oracle.mpsu1 import MPSU1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, N % 2, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    return m, h, V


def test_dpsi_matches_finite_difference():
    import torch
    from paper_2603_28648_b300.autograd import DMRGEnergy
    m, h, V = _setup()
    ctx = _ctx(m, h, V)
    th, tV = torch.tensor(h), torch.tensor(V)
    psi = torch.tensor(m.psi_to_flat() * 1.3, device="cuda", requires_grad=True)
    E = DMRGEnergy.apply(psi, th, tV, ctx)
    E.backward()
    d = torch.tensor(np.random.default_rng(1).normal(size=psi.numel()), device="cuda")
    eps = 1e-6
    with torch.no_grad():
        Ep = DMRGEnergy.apply(psi + eps * d, th, tV, ctx)
        Em = DMRGEnergy.apply(psi - eps * d, th, tV, ctx)
    fd = (Ep - Em).item() / (2 * eps)
    an = torch.dot(psi.grad, d).item()
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_rdm1_matches_expanded_vector_and_fd_in_h():
    import torch
    from oracle.fci import FCI
    from oracle.mpsu1 import Projector
    from paper_2603_28648_b300.autograd import DMRGEnergy
    m, h, V = _setup()
    L = m.L
    f = FCI(h, V, m.N, m.two_sz)
    v = Projector(m, f.space).apply(m.psi)
    g_ref, _ = f.rdm12(v / np.linalg.norm(v))
    ctx = _ctx(m, h, V)
    ctx.move_center(L - 2)
    g = ctx.rdm1(L)
    assert np.abs(g - g_ref).max() <= 1e-11
    assert abs(np.trace(g) - m.N) <= 1e-11
    # autograd dE/dh at the moved centre equals gamma
    psi = torch.tensor(ctx.psi(), device="cuda")
    th = torch.tensor(h, requires_grad=True)
    E = DMRGEnergy.apply(psi, th, torch.tensor(V), ctx)
    E.backward()
    assert np.abs(th.grad.numpy() - g).max() <= 1e-12
    # central difference in a symmetric perturbation of h (same MPS tensors)
    eps = 1e-6
    for (p, r) in [(0, 0), (1, 3), (2, 5)]:
        dh = np.zeros_like(h)
        dh[p, r] += 1.0
        dh[r, p] += 1.0 if p != r else 0.0
        Es = []
        for sgn in (+1, -1):
            c2 = _ctx(m, h + sgn * eps * dh, V)
            Es.append(c2.psi() @ c2.apply_heff(c2.psi()) / (c2.psi() @ c2.psi()))
        fd = (Es[0] - Es[1]) / (2 * eps)
        an = g[p, r] + (g[r, p] if p != r else 0.0)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_rdm1_equals_fci_at_exact_bond_dimension():
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1
    L, N, D = 6, 6, 64
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, 2))
    h, V = q.make_integrals(L, 11)
    ctx = _ctx(m, h, V)
    for _ in range(2):
        ctx.sweep(D, tol=1e-10)
    ctx.move_center(L - 2)
    ctx.davidson(tol=1e-10)
    g = ctx.rdm1(L)
    e0, c0 = FCI(h, V, N, 0).ground_state()
    g0, _ = FCI(h, V, N, 0).rdm12(c0)
    assert np.abs(g - g0).max() <= 1e-7
