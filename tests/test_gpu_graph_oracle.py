"""Several independent SU(2) problems captured in one CUDA graph, each result checked
against the operator-based SU(2) oracle (not only against eager replay).

Four problems of different lengths, particle numbers and spins (the shape of the batched
workload, at sizes the oracle computes in seconds) run as parallel branches of one graph
(`qcdmrg_graph_create`); after two replays every FP64 sigma equals the oracle's sigma of its
problem (relative Frobenius error <= 1e-10) and every BF16 sigma is within the BF16 bound
(8 x 2^-9) of it.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.run_last]

PROBLEMS = [(6, 6, 0, 8, 2, 31), (7, 7, 1, 10, 3, 32), (8, 6, 2, 16, 3, 33), (10, 10, 0, 24, 4, 34)]


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-10), ("bf16", 8 * 2.0 ** -9)])
def test_graph_of_su2_problems_matches_oracle(prec, bound):
    import torch
    import paper_2603_28648_b300 as qd
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2, export_abi_su2
    ensure_built()
    ctxs, psis, sigs, refs = [], [], [], []
    for L, N, two_s, D, c, seed in PROBLEMS:
        mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, seed, c))
        h, V = q.make_integrals(L, seed + 100)
        ctx = qd.Context(symmetry=qd.SU2)
        ctx.load_integrals(h, V)
        ctx.set_target(N, two_s)
        ctx.import_mps(L, c, *export_abi_su2(mps))
        ctx.build_env()
        ctxs.append(ctx)
        psis.append(torch.tensor(mps.psi_to_flat(), device="cuda"))
        sigs.append(torch.full_like(psis[-1], float("nan")))
        refs.append(mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps)))
    g = qd.HeffGraph(ctxs, [p.data_ptr() for p in psis], [s.data_ptr() for s in sigs], qd.PRECISIONS[prec])
    stream = torch.cuda.current_stream()
    for _ in range(2):
        g.launch(stream.cuda_stream)
    stream.synchronize()
    for s, ref in zip(sigs, refs):
        out = s.cpu().numpy()
        assert np.all(np.isfinite(out))
        assert np.linalg.norm(out - ref) <= bound * np.linalg.norm(ref)
    g.close()
    for c in ctxs:
        c.close()
