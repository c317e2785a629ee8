"""The N > 1 path of the benchmark on the CPU: two gloo ranks (replicas, no data-path
collective) agree on the maximum over ranks of their timed seconds, and the whole-job
throughput counts the work of every replica over that slowest time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], dist, "cpu")
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == [2.0, 10.0] and res[1] == [2.0, 10.0]


def test_replica_throughput_counts_every_replica():
    import bench
    assert bench.replica_throughput(2e12, 0.5, 1) == pytest.approx(4.0)
    assert bench.replica_throughput(2e12, 0.5, 4) == pytest.approx(16.0)


def test_bench_defaults_and_modes_parse(monkeypatch):
    """The default bench line keeps N = 1, the SU(2) CAS(54,36) shape at D = 2048 and the switch one
    cut past the centre; U(1) and the adjoint keep normal pairs everywhere; the opt-in modes
    parse without touching the default."""
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.symmetry, a.L, a.N, a.D, a.pair_switch) == (1, "su2", 36, 54, 2048, 19)
    assert a.warmup >= 3 and not a.qi and a.warm_start == 0 and a.scf_step == "steepest"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--symmetry", "u1"])
    assert bench.parse().pair_switch == 0
    monkeypatch.setattr(sys, "argv", ["bench.py", "--adjoint"])
    assert bench.parse().pair_switch == 0
    monkeypatch.setattr(sys, "argv", ["bench.py", "--qi", "--warm-start", "64", "--scf", "--scf-step", "newton"])
    a = bench.parse()
    assert a.qi and a.warm_start == 64 and a.scf and a.scf_step == "newton"
