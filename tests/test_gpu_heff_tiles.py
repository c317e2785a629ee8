"""FP64 H_eff psi at block sizes that reach every work-item form of the FP64 kernel.

At L = 10, N = 10 with the full bond dimension 256 at the centre bond (4, 5),
the blocks of four sites carry sectors of 36 states (two up and two down
electrons among four orbitals), so the sigma blocks need the 64-row and
64-column tiles of the FP64 grouped GEMM, and a sigma block collects segments
from a few hundred operator-product terms, so its summed K exceeds one work
item and the split-K path (partial tiles added with FP64 atomics) runs. The
library's statistics report which tile shapes and how many split tiles the
prepared task lists hold; sigma is compared element by element with the
oracle's operator-based sigma (relative Frobenius error <= 1e-10, the FP64
bound).
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def test_fp64_sigma_with_64_tiles_and_split_k_matches_oracle():
    import paper_2603_28648_b300 as qd
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    L, N, D, c = 10, 10, 256, 4
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, c))
    assert max(d for _, d in m.lbonds[c].sectors.values()) > 32
    h, V = q.make_integrals(L, 4)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.import_mps(L, c, *export_abi(m))
    ctx.build_env()
    st = ctx.stats()
    tiles = st["f64_tiles"]
    assert tiles[0] + tiles[1] + tiles[2] > 0, tiles     # a 64-wide tile shape runs
    assert tiles[3] > 0, tiles
    assert st["f64_split_tiles"] > 0                      # split-K tiles with FP64 atomics
    psi = m.psi_to_flat()
    sig = ctx.apply_heff(psi)
    ref = m.psi_to_flat(DMRGU1(h, V, N, 0).sigma(m))
    err = np.linalg.norm(sig - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err
    ctx.close()
