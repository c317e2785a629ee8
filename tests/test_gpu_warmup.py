"""Configuration-space warm start through the C ABI on the GPU: selected configurations
imported as an MPS (qcdmrg_config_mps + qcdmrg_import_mps), the warm-up half sweep
(qcdmrg_sweep_left) and full sweeps; the first solve is at or below the CI energy of the
selected configurations and the sweeps reach the FCI energy at a bond dimension that
truncates nothing, in both symmetries."""
import numpy as np
import pytest
import scipy.linalg as sl

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]


@pytest.mark.parametrize("sym,L,N,two_s,nmax", [(0, 6, 6, 0, 30), (1, 6, 6, 0, 30), (1, 6, 5, 1, 20)])
def test_warm_start_sweeps_reach_fci(sym, L, N, two_s, nmax):
    import paper_2603_28648_b300 as qd
    from oracle import configs as oc
    from oracle.fci import FCI
    ensure_built()
    h, V = q.make_integrals(L, 5)
    steps, _ = qd.select_configs(sym, h, V, N, two_s, nmax)
    coef = np.zeros(len(steps))
    coef[0] = 1.0
    ctx = qd.Context(symmetry=sym)
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    assert ctx.import_configs(L, N, two_s, steps, coef) == L - 2
    ctx.build_env()
    first = ctx.davidson(tol=1e-10)[0]
    rep = ctx.sweep_left(64, tol=1e-10)
    assert rep["n_steps"] == L - 2
    for _ in range(2):
        rep = ctx.sweep(64, tol=1e-10)
    ctx.close()
    f = FCI(h, V, N, two_s)
    P = np.stack([oc.config_vector([tuple(int(x) for x in s)], [1.0], L, N, two_s, bool(sym))[1] for s in steps], 1)
    H = f.matrix()
    e_ci = sl.eigh(P.T @ (H @ P), P.T @ P, eigvals_only=True)[0]
    e_fci, _ = f.ground_state(two_s=two_s)
    assert first <= e_ci + 1e-9
    assert abs(rep["energy"] - e_fci) <= 1e-8
