"""SU(2) spin-adapted H_eff psi at multiplet cost, through the C ABI.

The library keeps reduced operators between multiplets (rules_su2.cpp) and runs
the same grouped kernels as the U(1) path, with the recoupling factors as
segment scalars. sigma is compared element by element with the operator-based
SU(2) oracle (oracle/dmrgsu2.py, itself pinned by the Fock-space expansion of
every block operator and by P^T H_FCI P psi) on imported MPS: S = 0, 1/2, 1,
edge centres, and a case whose sectors of 40 multiplets need the 64-wide FP64
tiles. FP64: relative Frobenius error <= 1e-10; the tensor-core forms against
the FP64 form within the bounds of the U(1) tests (8u for BF16 and TF32,
2^-14 for the three-term BF16 split). At the CAS(54,36) shape (L = 36, N = 54,
S = 0, random MPS of 256 multiplets) the library's H_eff is symmetric and its
diagonal equals the probes e_i^T H e_i.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]

TOL_FP64 = 1e-10
BOUND = {"tf32": 8 * 2.0 ** -11, "bf16": 8 * 2.0 ** -9, "bf16x3": 2.0 ** -14}


def _ctx(mps, h, V):
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import export_abi_su2
    ensure_built()
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(mps.N, mps.two_s)
    ctx.import_mps(mps.L, mps.center, *export_abi_su2(mps))
    ctx.build_env()
    return ctx


def _mps(L, N, two_s, D, c, seed):
    from oracle.dmrgsu2 import MPSSU2
    return MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))


CASES = [(4, 4, 0, 16, 1), (5, 5, 1, 8, 1), (5, 4, 2, 8, 2), (6, 6, 0, 6, 0), (6, 5, 1, 6, 4),
         (8, 8, 0, 20, 3), (8, 7, 1, 24, 6), (8, 8, 2, 24, 0), (12, 5, 1, 100, 5)]


@pytest.mark.parametrize("L,N,two_s,D,c", CASES)
def test_su2_fp64_sigma_matches_oracle(L, N, two_s, D, c):
    from oracle.dmrgsu2 import DMRGSU2
    mps = _mps(L, N, two_s, D, c, 5)
    h, V = q.make_integrals(L, 11)
    ctx = _ctx(mps, h, V)
    psi = mps.psi_to_flat()
    sig = ctx.apply_heff(psi)
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    assert np.linalg.norm(sig - ref) <= TOL_FP64 * np.linalg.norm(ref)
    if L == 12:
        t = ctx.stats()["f64_tiles"]
        assert t[0] + t[1] + t[2] > 0, t      # sectors of 40 multiplets: 64-wide tiles
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
def test_su2_tensor_core_forms_vs_fp64(prec):
    import paper_2603_28648_b300 as qd
    mps = _mps(8, 7, 1, 24, 3, 8)
    h, V = q.make_integrals(8, 12)
    ctx = _ctx(mps, h, V)
    psi = mps.psi_to_flat()
    ref = ctx.apply_heff(psi, qd.FP64)
    out = ctx.apply_heff(psi, qd.PRECISIONS[prec])
    assert np.linalg.norm(out - ref) <= BOUND[prec] * np.linalg.norm(ref)
    ctx.close()


def test_su2_cas54_shape_symmetric_with_probe_diagonal():
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 36, 54, 256
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    ctx = qd.Context(symmetry=qd.SU2)
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 3, 17)
    ctx.build_env()
    n = ctx.psi_size()
    rng = np.random.default_rng(1)
    x, y = rng.normal(size=n), rng.normal(size=n)
    hx, hy = ctx.apply_heff(x), ctx.apply_heff(y)
    assert abs(x @ hy - y @ hx) <= 1e-11 * np.linalg.norm(hx) * np.linalg.norm(y)
    d = ctx.heff_diag()
    for i in rng.choice(n, 8, replace=False):
        e = np.zeros(n)
        e[i] = 1.0
        assert abs(ctx.apply_heff(e)[i] - d[i]) <= 1e-10 * max(1.0, abs(d[i]))
    for prec in ["bf16", "bf16x3"]:
        out = ctx.apply_heff(x, qd.PRECISIONS[prec])
        assert np.linalg.norm(out - hx) <= BOUND[prec] * np.linalg.norm(hx)
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_su2_chunk_targets_give_the_fixed_depth_sigma(prec):
    """The chunk byte target only regroups the K steps the kernels issue (same MMAs in
    the same order per accumulator column), so every target reproduces the fixed-depth
    sigma up to the order of the FP64 atomics of split items; each is within the form's
    bound of FP64. CAS(54,36) shape at D = 256 multiplets: many chunks per item."""
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 36, 54, 256
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    x = None
    out = {}
    for chunk in [0, 32768, 49152, 65536]:
        ctx = qd.Context(symmetry=qd.SU2, autotune=False, tile_chunk=chunk)
        ctx.load_integrals(h, V)
        ctx.set_target(N, 0)
        ctx.init_mps(D, 3, 17)
        ctx.build_env()
        if x is None:
            x = np.random.default_rng(5).normal(size=ctx.psi_size())
            ref = ctx.apply_heff(x, qd.FP64)
        out[chunk] = ctx.apply_heff(x, qd.PRECISIONS[prec])
        assert ctx.stats()["tile_chunk"] == chunk
        ctx.close()
    for chunk, o in out.items():
        assert np.linalg.norm(o - ref) <= BOUND[prec] * np.linalg.norm(ref), chunk
        assert np.linalg.norm(o - out[0]) <= 1e-12 * np.linalg.norm(out[0]), chunk

