"""GPU Davidson, H_eff diagonal, truncation and full sweeps against the oracle."""
import json
import os

import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "u1_L10_sweeps.json")


def _ctx(L, N, D, c, mps_seed, int_seed):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, mps_seed, c))
    h, V = q.make_integrals(L, int_seed)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, two)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    return ctx, m, h, V


def test_heff_diagonal_matches_probes():
    ctx, m, h, V = _ctx(6, 5, 16, 2, 3, 4)
    d = ctx.heff_diag()
    n = d.size
    probe = np.array([ctx.apply_heff(np.eye(n)[i])[i] for i in range(n)])
    assert np.abs(d - probe).max() <= 1e-12 * np.abs(probe).max()


@pytest.mark.parametrize("L,N,D,c", [(6, 6, 16, 2), (8, 8, 32, 3), (7, 5, 24, 0)])
def test_davidson_matches_oracle_lanczos(L, N, D, c):
    from oracle.dmrgu1 import DMRGU1, lowest_eig, to_mat
    ctx, m, h, V = _ctx(L, N, D, c, 3, 11)
    e, r, it = ctx.davidson(tol=1e-10)
    heff = DMRGU1(h, V, N, N % 2).heff_at_center(m)
    e0, _ = lowest_eig(heff, to_mat(m.psi))
    assert r <= 1e-10
    assert abs(e - e0) <= 1e-9


def test_mixed_policy_energy_within_1e6():
    """BF16 -> BF16x3 -> FP64-corrected Davidson reaches the FP64 energy."""
    import paper_2603_28648_b300 as qd
    ctx, m, h, V = _ctx(8, 8, 32, 3, 5, 12)
    e64, _, _ = ctx.davidson(tol=1e-8)
    ctx2, _, _, _ = _ctx(8, 8, 32, 3, 5, 12)
    emx, r, _ = ctx2.davidson(tol=1e-8, policy=1)
    assert r <= 1e-8
    assert abs(emx - e64) <= 1e-6


def test_sweeps_match_oracle_config_L10_D64():
    """6 sweeps at L=10, N=10, D=64 (U(1)) from the same MPS: energies as the
    oracle's, and variational with respect to FCI."""
    g = json.load(open(GOLDEN))
    w = q.workload("u1_L10_N10_D64")
    ctx, m, h, V = _ctx(w["L"], w["N"], w["D"], g["center"], w["mps_seed"], w["int_seed"])
    E = []
    for s in range(6):
        rep = ctx.sweep(w["D"], tol=1e-10)
        E.append(rep["energy"])
        assert rep["n_steps"] == 2 * w["L"] - 4
        assert rep["max_trunc_err"] >= 0.0
    assert np.abs(np.array(E) - np.array(g["sweep_energies"])).max() <= 1e-8
    assert E[-1] >= g["fci_energy"] - 1e-10


def test_exact_bond_dimension_reproduces_fci():
    from oracle.fci import FCI
    L, N, D = 6, 6, 64
    ctx, m, h, V = _ctx(L, N, D, 2, 3, 11)
    e0, _ = FCI(h, V, N, 0).ground_state()
    for _ in range(2):
        rep = ctx.sweep(D, tol=1e-10)
    assert abs(rep["energy"] - e0) <= 1e-9
    # only rounding-level density-matrix eigenvalues (each <= 1e-14) are dropped
    assert rep["max_trunc_err"] <= 1e-12


def test_truncate_moves_and_keeps_norm():
    ctx, m, h, V = _ctx(8, 8, 32, 3, 7, 8)
    ctx.davidson(tol=1e-8)
    err = ctx.truncate(16, +1)
    assert err >= 0.0
    psi = ctx.psi()
    assert abs(psi @ psi - (1.0 - err)) <= 1e-10
    err2 = ctx.truncate(16, -1)
    assert err2 >= 0.0
