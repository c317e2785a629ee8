"""MPS export and checkpoint/restore through the C ABI: an imported MPS comes back
bit for bit; after a sweep (moved centre, truncated bonds) the exported MPS imported
into a new context, and a checkpoint restored into a new context, give the same
H_eff psi as the original context; missing, truncated and foreign files are file errors."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def test_export_returns_the_imported_mps():
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    L, N, D, c = 6, 6, 16, 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    nsec, sec, data = export_abi(m)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.import_mps(L, c, nsec, sec, data)
    L2, c2, nsec2, sec2, data2 = ctx.export_mps()
    assert (L2, c2) == (L, c)
    assert np.array_equal(nsec2, nsec)
    assert np.array_equal(sec2, sec)
    assert np.array_equal(data2, data)
    ctx.close()


def test_export_and_checkpoint_after_a_sweep(tmp_path):
    import paper_2603_28648_b300 as qd
    ensure_built()
    L, N, D = 8, 8, 16
    h, V = q.make_integrals(L, 6)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 11, L // 2 - 1)
    ctx.build_env()
    ctx.sweep(D, tol=1e-8)
    ctx.move_center(2)
    psi = ctx.psi()
    ref = ctx.apply_heff(psi)

    ctx2 = qd.Context()
    ctx2.load_integrals(h, V)
    ctx2.set_target(N, 0)
    Lx, cx, nsec, sec, data = ctx.export_mps()
    ctx2.import_mps(Lx, cx, nsec, sec, data)
    ctx2.build_env()
    assert np.linalg.norm(ctx2.apply_heff(psi) - ref) <= 1e-13 * np.linalg.norm(ref)

    path = str(tmp_path / "state.qcdmrg")
    ctx.checkpoint(path)
    ctx3 = qd.Context()
    ctx3.restore(path)
    ctx3.build_env()
    assert np.array_equal(ctx3.psi(), psi)
    assert np.linalg.norm(ctx3.apply_heff(psi) - ref) <= 1e-13 * np.linalg.norm(ref)
    with pytest.raises(qd.QcdmrgError) as e:
        ctx3.restore(str(tmp_path / "missing.qcdmrg"))
    assert e.value.code == -7
    # a truncated checkpoint and a file that is not one are file errors, not crashes
    raw = open(path, "rb").read()
    for name, blob in (("short.qcdmrg", raw[: len(raw) // 2]), ("other.qcdmrg", b"NOTACHECKPOINT" + raw[14:])):
        bad = str(tmp_path / name)
        with open(bad, "wb") as f:
            f.write(blob)
        with pytest.raises(qd.QcdmrgError) as e:
            ctx3.restore(bad)
        assert e.value.code == -7
    for c in (ctx, ctx2, ctx3):
        c.close()
