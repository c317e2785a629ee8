"""H_eff psi captured in CUDA graphs: one context, and 16 independent instances
(L in 12..24, N = L, D in {128, 256, 512}) replayed as parallel graph branches."""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def _instance(L, D, seed):
    import paper_2603_28648_b300 as qd
    h, V = q.make_integrals(L, seed)
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(L, L % 2)
    ctx.init_mps(D, seed + 1000, L // 2 - 1)
    ctx.build_env()
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_graph_replay_equals_eager(prec):
    import torch
    import paper_2603_28648_b300 as qd
    ensure_built()
    ctx = _instance(10, 64, 21)
    x = torch.tensor(ctx.psi(), device="cuda")
    y_eager = torch.empty_like(x)
    y_graph = torch.full_like(x, float("nan"))
    p = qd.PRECISIONS[prec]
    s = torch.cuda.current_stream()
    ctx.apply_heff_dev(x.data_ptr(), y_eager.data_ptr(), s.cuda_stream, p)
    g = qd.HeffGraph([ctx], [x.data_ptr()], [y_graph.data_ptr()], p)
    for _ in range(2):
        g.launch(s.cuda_stream)
    s.synchronize()
    a, b = y_eager.cpu().numpy(), y_graph.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
    flops, nodes = g.info()
    assert flops > 0 and nodes >= 3


def test_sixteen_instances_in_one_graph():
    import torch
    import paper_2603_28648_b300 as qd
    ensure_built()
    rng = np.random.default_rng(99)
    Ls = rng.integers(12, 25, size=16)
    Ds = rng.choice([128, 256, 512], size=16)
    ctxs, xs, ys, refs = [], [], [], []
    s = torch.cuda.current_stream()
    for i, (L, D) in enumerate(zip(Ls, Ds)):
        c = _instance(int(L), int(D), 100 + i)
        x = torch.tensor(c.psi(), device="cuda")
        r = torch.empty_like(x)
        c.apply_heff_dev(x.data_ptr(), r.data_ptr(), s.cuda_stream)
        ctxs.append(c); xs.append(x); refs.append(r); ys.append(torch.full_like(x, float("nan")))
    g = qd.HeffGraph(ctxs, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys])
    g.launch(s.cuda_stream)
    s.synchronize()
    for r, y in zip(refs, ys):
        a, b = r.cpu().numpy(), y.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
