"""The no-allocation H_eff psi entry point against the regular device entry point.

qcdmrg_apply_heff_noalloc exists for callers that cannot allocate device memory
at the moment they need a product (work being captured into a CUDA graph, a
GPU whose free memory is held by another framework's caching allocator, a
solver with a fixed memory budget). It must give the same sigma as
qcdmrg_apply_heff_dev on two calls in a row (the second call finds the
previous call's data in the shared scratch array). This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _ctx():
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1, export_abi
    ensure_built()
    w = q.workload("u1_L10_N10_D64")
    L, N = w["L"], w["N"]
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, w["D"], q.SYM_U1, w["mps_seed"], 4))
    h, V = q.make_integrals(L, w["int_seed"])
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.import_mps(L, 4, *export_abi(m))
    ctx.build_env()
    return ctx


def test_noalloc_matches_device_entry_point_twice():
    import torch
    ctx = _ctx()
    n = ctx.psi_size()
    rng = np.random.default_rng(7)
    stream = torch.cuda.current_stream()
    for trial in range(2):
        x = torch.tensor(rng.normal(size=n), device="cuda")
        ref = torch.empty_like(x)
        out = torch.full_like(x, float("nan"))
        ctx.apply_heff_dev(x.data_ptr(), ref.data_ptr(), stream.cuda_stream)
        ctx.apply_heff_noalloc(x.data_ptr(), out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= TOL_FP64 * np.linalg.norm(r), trial


def test_noalloc_allocates_nothing_and_runs_inside_graph_capture():
    """After one warm call the entry point allocates no device memory (free bytes
    unchanged around an eager call), and it can be captured into a CUDA graph
    (capture rejects any allocation or synchronisation); the replayed sigma equals
    the device entry point's."""
    import torch
    ctx = _ctx()
    n = ctx.psi_size()
    x = torch.tensor(np.random.default_rng(11).normal(size=n), device="cuda")
    ref = torch.empty_like(x)
    out = torch.full_like(x, float("nan"))
    stream = torch.cuda.current_stream()
    ctx.apply_heff_dev(x.data_ptr(), ref.data_ptr(), stream.cuda_stream)
    ctx.apply_heff_noalloc(x.data_ptr(), out.data_ptr(), stream.cuda_stream)   # warm call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx.apply_heff_noalloc(x.data_ptr(), out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    out.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ctx.apply_heff_noalloc(x.data_ptr(), out.data_ptr(), side.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert np.linalg.norm(o - r) <= TOL_FP64 * np.linalg.norm(r)
    ctx.close()


def test_noalloc_rejects_too_large_problem():
    import paper_2603_28648_b300 as qd
    import torch
    ensure_built()
    L, N, D = 36, 54, 1024
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    ctx = qd.Context(tmp_budget_gb=8.0)
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, 3, 17)
    ctx.build_env()
    n = ctx.psi_size()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(qd.QcdmrgError) as e:
        ctx.apply_heff_noalloc(x.data_ptr(), y.data_ptr(), 0)
    assert e.value.code == -1 and "scratch" in str(e.value)
