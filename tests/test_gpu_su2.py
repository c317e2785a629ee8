"""SU(2)-adapted H_eff psi through the library's U(1) path: the SU(2) MPS of the oracle
written with all M components as bond states is imported through the C ABI, the library's
FP64 H_eff psi is applied to the Clebsch-Gordan expansion C psi of a reduced two-site
wavefunction, and C^T of the result is compared element by element with the oracle's
plain-definition SU(2) sigma (relative Frobenius error <= 1e-10, the FP64 parity bound)."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,two_s,l,cap", [(6, 6, 0, 2, 2), (7, 7, 1, 2, 2), (8, 8, 0, 3, 3)])
def test_su2_sigma_through_u1_library(L, N, two_s, l, cap):
    import paper_2603_28648_b300 as qd
    from oracle.fci import FCI
    from oracle.mpssu2 import TangentSU2, to_u1
    from oracle.mpsu1 import export_abi
    ensure_built()
    t = TangentSU2(L, N, two_s, l, cap=cap, seed=9)
    mps, C = to_u1(t)
    h, V = q.make_integrals(L, 13)
    psi = np.random.default_rng(4).normal(size=C.shape[1])
    mps.psi = mps.psi_from_flat(C @ psi)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, two_s)
    ctx.import_mps(L, l, *export_abi(mps))
    ctx.build_env()
    sig_u1 = ctx.apply_heff(mps.psi_to_flat())
    ref = t.heff(FCI(h, V, N, two_s), psi)
    got = C.T @ sig_u1
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    ctx.close()
