"""GPU tests of the 2-RDM by a walk of the centre (qcdmrg_rdm2_sweep), through the C ABI:
element by element against the 2-RDM of the expanded MPS vector, its permutation average
against qcdmrg_rdm2, the MPS restored after the walk, and at L=16 the identities every 2-RDM
of the state satisfies."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def test_rdm2_by_centre_walk_matches_brute_force():
    """qcdmrg_rdm2_sweep (every element at its centre, exact moves) against the 2-RDM of the
    expanded MPS vector, its permutation average against qcdmrg_rdm2, and the MPS restored
    after the walk (same psi, same H_eff psi)."""
    import paper_2603_28648_b300 as qd
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1, Projector, export_abi
    ensure_built()
    L, N, D, c = 6, 5, 16, 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 1, D, q.SYM_U1, 6, c))
    h, V = q.make_integrals(L, 7)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 1)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    psi0 = m.psi_to_flat()
    e0 = psi0 @ ctx.apply_heff(psi0) / (psi0 @ psi0)
    G = ctx.rdm2_sweep(L)
    f = FCI(h, V, N, 1)
    v = Projector(m, f.space).apply(m.psi)
    g1, Gf = f.rdm12(v / np.linalg.norm(v))
    assert np.abs(G - Gf).max() <= 1e-10
    axes = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
            (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    Gs = sum(G.transpose(a) for a in axes) / 8.0
    assert np.abs(Gs - ctx.rdm2(L)).max() <= 1e-10
    assert np.array_equal(ctx.psi(), psi0)      # the MPS is restored after the walk
    e1 = psi0 @ ctx.apply_heff(psi0) / (psi0 @ psi0)
    assert abs(e1 - e0) <= 1e-13 * abs(e0)


def test_rdm2_by_centre_walk_identities_L16():
    """Beyond brute-force sizes (L=16, N=16, D=128, GPU-initialised MPS): the traces, the
    symmetries and the energy identity E = sum h gamma + 1/2 sum V Gamma with gamma from the
    contraction of Gamma."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 16, 16, 128
    h, V = q.make_integrals(L, 21)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 3, 7)
    ctx.build_env()
    psi = ctx.psi()
    E = psi @ ctx.apply_heff(psi) / (psi @ psi)
    G = ctx.rdm2_sweep(L)
    assert abs(np.einsum("pprr->", G) - N * (N - 1)) <= 1e-9
    assert np.abs(G - G.transpose(2, 3, 0, 1)).max() <= 1e-12
    g = np.einsum("pqrr->pq", G) / (N - 1)
    assert abs(np.sum(h * g) + 0.5 * np.sum(V * G) - E) <= 1e-10 * abs(E)
