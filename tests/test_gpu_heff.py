"""GPU parity of H_eff psi (FP64 form) against the oracle, through the C ABI."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10   # relative Frobenius error bound of the FP64 form


def _ctx_from_oracle(m, h, V, N, two):
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import export_abi
    ensure_built()
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, two)
    ns, sec, data = export_abi(m)
    ctx.import_mps(m.L, m.center, ns, sec, data)
    ctx.build_env()
    return ctx


@pytest.mark.parametrize("L,N,D,c", [(3, 2, 8, 0), (4, 4, 16, 1), (5, 5, 16, 1), (6, 6, 16, 2),
                                     (6, 5, 16, 2), (7, 6, 24, 0), (7, 6, 24, 5), (8, 8, 32, 3)])
def test_sigma_matches_oracle(L, N, D, c):
    from oracle.mpsu1 import MPSU1
    from oracle.dmrgu1 import DMRGU1
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, 5 + L, c))
    h, V = q.make_integrals(L, 7 + L)
    ctx = _ctx_from_oracle(m, h, V, N, two)
    psi = m.psi_to_flat()
    sig = ctx.apply_heff(psi)
    ref = m.psi_to_flat(DMRGU1(h, V, N, two).sigma(m))
    assert np.linalg.norm(sig - ref) <= TOL_FP64 * np.linalg.norm(ref)


def test_sigma_config_u1_L10_D64_against_projection():
    """L=10, N=10, Sz=0, D=64 at the centre bond, against P^T H_FCI P psi."""
    from oracle.mpsu1 import MPSU1, Projector
    from oracle.fci import FCI
    w = q.workload("u1_L10_N10_D64")
    L, N = w["L"], w["N"]
    h, V = q.make_integrals(L, w["int_seed"])
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, w["D"], q.SYM_U1, w["mps_seed"], 4))
    ctx = _ctx_from_oracle(m, h, V, N, 0)
    f = FCI(h, V, N, 0)
    P = Projector(m, f.space)
    rng = np.random.default_rng(3)
    for trial in range(2):
        x = m.psi if trial == 0 else m.psi_from_flat(rng.normal(size=m.psi_to_flat().size))
        ref = m.psi_to_flat(P.heff(f, x))
        sig = ctx.apply_heff(m.psi_to_flat(x))
        assert np.linalg.norm(sig - ref) <= TOL_FP64 * np.linalg.norm(ref)


def test_e_core_shift_and_linearity():
    from oracle.mpsu1 import MPSU1, export_abi
    import paper_2603_28648_b300 as qd
    L, N = 6, 6
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, 16, q.SYM_U1, 2, 2))
    h, V = q.make_integrals(L, 3)
    a = _ctx_from_oracle(m, h, V, N, 0)
    b = qd.Context()
    b.load_integrals(h, V, e_core=1.25)
    b.set_target(N, 0)
    b.import_mps(L, 2, *export_abi(m))
    b.build_env()
    x = m.psi_to_flat()
    y = np.random.default_rng(1).normal(size=x.size)
    sa, sb = a.apply_heff(x), b.apply_heff(x)
    assert np.allclose(sb - sa, 1.25 * x, atol=1e-12)
    lin = a.apply_heff(2.0 * x - 3.0 * y)
    assert np.allclose(lin, 2.0 * sa - 3.0 * a.apply_heff(y), atol=1e-10 * np.abs(lin).max())


def test_device_entry_point_matches_host():
    import torch
    from oracle.mpsu1 import MPSU1
    L, N = 6, 6
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, 16, q.SYM_U1, 4, 2))
    h, V = q.make_integrals(L, 5)
    ctx = _ctx_from_oracle(m, h, V, N, 0)
    x = m.psi_to_flat()
    xd = torch.tensor(x, device="cuda")
    sd = torch.empty_like(xd)
    s = torch.cuda.current_stream()
    ctx.apply_heff_dev(xd.data_ptr(), sd.data_ptr(), s.cuda_stream)
    s.synchronize()
    assert np.allclose(sd.cpu().numpy(), ctx.apply_heff(x), rtol=0, atol=1e-13)


def test_init_mps_structure_and_hermiticity_L36():
    """Sector rule equals the input generator's; H_eff of the GPU-initialised
    MPS at the centre of a CAS(54,36)-shaped U(1) problem is symmetric."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 36, 54, 128
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 11, 17)
    st = q.mps_structure(L, N, 0, D, q.SYM_U1)
    for b in range(0, 18):
        assert ctx.bond(b) == st[b]
    for b in range(19, L + 1):
        assert ctx.bond(b) == st[L - b]
    ctx.build_env()
    n = ctx.psi_size()
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=n), rng.normal(size=n)
    a, b = y @ ctx.apply_heff(x), x @ ctx.apply_heff(y)
    assert abs(a - b) <= 1e-11 * abs(a)
    psi = ctx.psi()
    assert abs(psi @ psi - 1.0) < 1e-12


def test_error_codes():
    import paper_2603_28648_b300 as qd
    ensure_built()
    ctx = qd.Context()
    with pytest.raises(qd.QcdmrgError) as e:
        ctx.build_env()
    assert e.value.code == -4
    h, V = q.make_integrals(4, 1)
    hb = h.copy()
    hb[0, 1] += 1.0
    with pytest.raises(qd.QcdmrgError) as e:
        ctx.load_integrals(hb, V)
    assert e.value.code == -1
    Vn = V.copy()
    Vn[0, 0, 0, 0] = np.nan
    with pytest.raises(qd.QcdmrgError):
        ctx.load_integrals(h, Vn)
    ctx.load_integrals(h, V)
    with pytest.raises(qd.QcdmrgError):
        ctx.set_target(5, 0)
    ctx.set_target(4, 0)
    with pytest.raises(qd.QcdmrgError):
        ctx.apply_heff(np.zeros(4))
