"""Benchmark of the two-site DMRG H_eff psi hot path (one JSON line on rank 0).

Default workload: U(1)xU(1) H_eff psi at the centre bond of a CAS(54,36)-shaped
synthetic problem (L=36, N=54, 2Sz=0), random canonical MPS of bond dimension
D, operator blocks built on the device by the library's renormalization.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--D 1024] [--precision fp64]
Under torchrun every rank runs an independent replica (the path does not
shard across GPUs); the line reports the whole-job throughput.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("H·ψ TFLOP/s & sweep s, CAS(54,36)-shape D=4096: mixed vs FP64, "
          "same energy err")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--D", type=int, default=1024)
    ap.add_argument("--symmetry", default="su2", choices=["su2", "u1"],
                    help="su2: spin-adapted (D counts SU(2) multiplets, the paper's D_SU(2)); u1: U(1)xU(1)")
    ap.add_argument("--L", type=int, default=36)
    ap.add_argument("--N", type=int, default=54)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "tf32", "bf16", "bf16x3"],
                    help="form whose throughput is the headline value (all forms are timed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="one full sweep (L->R->L) with FP64 Davidson and with the mixed policy, same start")
    ap.add_argument("--batched", action="store_true",
                    help="16 independent problems (L 12..24, D 128..512) in one CUDA graph vs one by one")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the backward of E(psi, h, V): dE/dpsi, gamma and the centre-walk 2-RDM")
    ap.add_argument("--max-iter", type=int, default=300,
                    help="Davidson iteration cap per two-site step of --sweep (a step that hits it is kept)")
    ap.add_argument("--sweep-budget", type=float, default=300.0,
                    help="seconds of sweep steps per form in --sweep mode before it stops early")
    ap.add_argument("--hbm-budget", type=float, default=0.0,
                    help="device GB for renormalized operator blocks (0: unlimited); blocks beyond it "
                         "live in pinned host memory, so only the centre's blocks stay on the device")
    ap.add_argument("--pair-switch", type=int, default=0,
                    help="cut of the normal/complementary switch (0: normal pairs on the left at every "
                         "cut; L/2: the N/2 rule, which the D=4096 environment needs to fit)")
    ap.add_argument("--sum-gemm", type=int, default=0, choices=[-1, 0, 1],
                    help="operator sums of the renormalization side as GEMMs (1), block by block (-1), "
                         "or as GEMMs only with the switch (0)")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (read + write) of one H_eff psi on the tiled tensor-core kernel,
# from one ncu capture of both stage launches (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (form, L, N, D); the capture and its command
# are summarised in profiles/tiled_gemm_bf16_u1_L36_N54_D1024.md. A key that is
# absent reports null.
DRAM_TRAFFIC = {("bf16", 36, 54, 1024): 2.58e9 + 1.64e9 + 3.52e9 + 0.0024e9}


def measured_peaks():
    """Measured peaks of this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16": float(d["bf16_tflops"]), "hbm": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16": 1800.0, "hbm": 6400.0, "source": "fallback"}


def fp64_peak_tflops(torch):
    """Measured cuBLAS DGEMM rate (no FP64 peak is recorded for this box)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def cpu_sample():
    """Oracle H_eff psi on the L=10, N=10, D=64 U(1) workload (centre bond)."""
    import numpy as np
    import qcinputs as q
    from oracle.mpsu1 import MPSU1
    from oracle.dmrgu1 import DMRGU1
    w = q.workload("u1_L10_N10_D64")
    L, N = w["L"], w["N"]
    h, V = q.make_integrals(L, w["int_seed"])
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, w["D"], q.SYM_U1, w["mps_seed"], L // 2 - 1))
    d = DMRGU1(h, V, N, 0)
    heff = d.heff_at_center(m)
    from oracle.dmrgu1 import to_mat
    x = to_mat(m.psi)
    return m, h, V, heff, x


def time_oracle(reps):
    m, h, V, heff, x = cpu_sample()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        heff.apply_mat(x)
        ts.append(time.perf_counter() - t0)
    return m, h, V, ts


def time_oracle_for(seconds, min_reps=4):
    """Oracle H_eff psi repeated until about `seconds` of CPU time (first repetition untimed)."""
    m, h, V, heff, x = cpu_sample()
    ts, t_all = [], time.perf_counter()
    while len(ts) < min_reps or time.perf_counter() - t_all < seconds:
        t0 = time.perf_counter()
        heff.apply_mat(x)
        ts.append(time.perf_counter() - t0)
    return m, h, V, ts


def sample_flops(m, h, V):
    """Algorithmic flops of the sample as counted by the library's task list."""
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import export_abi
    ctx = qd.Context()
    ctx.load_integrals(h, V)
    ctx.set_target(m.N, m.two_sz)
    ctx.import_mps(m.L, m.center, *export_abi(m))
    ctx.build_env()
    f = ctx.stats()["heff_flops"]
    ctx.close()
    return f


def max_over_ranks(values, dist, device):
    """Element-wise maximum over the ranks of per-rank seconds (the slowest replica
    sets the job's time)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(flops_per_step, seconds_per_step, world):
    """Whole-job TFLOP/s of `world` independent replicas, each doing flops_per_step in
    at most seconds_per_step (the maximum over ranks)."""
    return world * flops_per_step / seconds_per_step / 1e12


def cores():
    return len(os.sched_getaffinity(0))


def run_reference(args, rank, world):
    if rank != 0:
        return
    reps = args.steps + args.warmup
    m, h, V, ts = time_oracle(reps)
    t = statistics.mean(ts[args.warmup:]) if len(ts) > args.warmup else statistics.mean(ts)
    try:
        flops = sample_flops(m, h, V)
    except Exception:
        flops = None
    val = flops / t / 1e12 if flops else None
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "u1_L10_N10_D64 centre-bond H_eff psi (oracle sample)",
                   "note": "oracle: dense FP64 numpy, H_eff psi with environments built",
                   "flops": "algorithmic count of the library's task list for the same product "
                            "(qcdmrg_stats.heff_flops, planned outside the timed region)"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores(), "kind": "oracle",
                         "sample": "U(1) L=10 N=10 D=64 centre-bond H_eff psi (environment excluded)"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import qcinputs as q
    import paper_2603_28648_b300 as qd
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    L, N, D = args.L, args.N, args.D
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    sym = qd.SU2 if args.symmetry == "su2" else qd.U1
    ctx = qd.Context(device=local, symmetry=sym, hbm_budget_gb=args.hbm_budget, pair_switch=args.pair_switch,
                     sum_gemm=args.sum_gemm)
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    center = L // 2 - 1
    ctx.init_mps(D, q.integrals.BASE_SEED + 1002, center)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.build_env()
    torch.cuda.synchronize()
    env_s = time.perf_counter() - t0
    st = ctx.stats()
    flops = st["heff_flops"]
    psi = torch.tensor(ctx.psi(), device="cuda")
    sig = torch.empty_like(psi)
    stream = torch.cuda.current_stream()

    head = qd.PRECISIONS[args.precision]

    def step(prec):
        ctx.apply_heff_dev(psi.data_ptr(), sig.data_ptr(), stream.cuda_stream, prec)

    def timed(prec, steps, clocks=None, profile=False):
        for _ in range(args.warmup):
            step(prec)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        if dist:
            dist.barrier()
        ctx.check_device()
        return e0.elapsed_time(e1) / 1e3

    forms = {}
    energies = {}
    step(0)  # FP64 reference product for the per-form sigma errors
    torch.cuda.synchronize()
    sig64 = sig.clone()
    errs = {}
    for name, prec in qd.PRECISIONS.items():
        if name == args.precision:
            continue
        t = timed(prec, max(2, args.steps // 2))
        energies[name] = float(torch.dot(psi, sig).item())
        errs[name] = float((torch.linalg.norm(sig - sig64) / torch.linalg.norm(sig64)).item())
        forms[name] = {"tflops": flops / (t / max(2, args.steps // 2)) / 1e12,
                       "ms_per_step": t / max(2, args.steps // 2) * 1e3}
    clocks = Clocks(local)
    elapsed = timed(head, args.steps, clocks, args.profile)
    clk = clocks.stop()
    energies[args.precision] = float(torch.dot(psi, sig).item())
    errs[args.precision] = float((torch.linalg.norm(sig - sig64) / torch.linalg.norm(sig64)).item())
    forms[args.precision] = {"tflops": flops / (elapsed / args.steps) / 1e12,
                             "ms_per_step": elapsed / args.steps * 1e3}
    for name in forms:
        forms[name]["energy_minus_fp64"] = energies[name] - energies["fp64"]
        forms[name]["sigma_rel_err_vs_fp64"] = errs[name]
        forms[name]["speedup_vs_fp64"] = forms["fp64"]["ms_per_step"] / forms[name]["ms_per_step"]
    # end to end through the public API: pinned host psi -> device, H psi, sigma -> host
    hpsi = psi.cpu().pin_memory()
    hsig = torch.empty_like(hpsi).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        psi.copy_(hpsi, non_blocking=True)
        step(head)
        hsig.copy_(sig, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_t = e0.elapsed_time(e1) / 1e3
    energy = energies[args.precision]
    if dist:
        elapsed, e2e_t = max_over_ranks([elapsed, e2e_t], dist, "cuda")
    peak = fp64_peak_tflops(torch)
    per_step = elapsed / args.steps
    value = replica_throughput(flops, per_step, world)
    e2e_val = replica_throughput(flops, e2e_t / args.steps, world)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        m, hh, VV, ts = time_oracle_for(10.0)
        t_cpu = statistics.mean(ts[1:])
        f_cpu = sample_flops(m, hh, VV)
        cpu = {"value": f_cpu / t_cpu / 1e12, "unit": "TFLOP/s", "cores": cores(), "kind": "oracle",
               "sample": "U(1) L=10 N=10 D=64 centre-bond H_eff psi, oracle dense FP64 "
                         f"(environment build excluded), {len(ts) - 1} timed repetitions, "
                         f"{sum(ts[1:]):.1f} s of CPU work"}
    st2 = ctx.stats()
    tile = {"stage2_kmax": st2["tile_kmax"], "stage1_width": st2["tile_width"], "autotuner_runs": st2["tunes"],
            "autotuner_s": st2["tune_seconds"]}
    pk = measured_peaks()
    # algorithmic minimum traffic of one product in each form's operand type:
    # every referenced operator element once (8 B FP64, 4 B TF32, 2 B BF16,
    # 6 B for the three BF16 planes), psi and sigma (FP64 in every form)
    nelem = st["heff_bytes"] / 8.0
    npsi = 2.0 * st["psi_size"]
    esize = {"fp64": 8, "tf32": 4, "bf16": 2, "bf16x3": 6}
    form_bytes = {k: (nelem - npsi) * e + 8 * npsi for k, e in esize.items()}
    tensor_ratio = {"fp64": None, "bf16": 1.0, "tf32": 1.1 / 2.25, "bf16x3": 1.0 / 6.0}
    for name, f in forms.items():
        t_s = f["ms_per_step"] / 1e3
        f["algorithmic_bytes"] = form_bytes[name]
        f["hbm_gbs_algorithmic"] = form_bytes[name] / t_s / 1e9
        f["hbm_frac"] = f["hbm_gbs_algorithmic"] / pk["hbm"]
        r = tensor_ratio[name]
        f["compute_frac"] = f["tflops"] / (pk["bf16"] * r if r else peak)
    # the dominant kernel (the grouped block GEMM, every launch of the step) is
    # bound by HBM: flops / algorithmic bytes is below the ridge point of every
    # tensor form, so its roofline is the measured copy bandwidth
    nbytes = form_bytes[args.precision]
    achieved = nbytes / per_step / 1e9
    traffic = DRAM_TRAFFIC.get((args.precision, L, N, D))
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm"], "unit": "GB/s",
            "frac": achieved / pk["hbm"], "traffic": traffic,
            "algorithmic_bytes_per_step": nbytes,
            "intensity_flop_per_byte": flops / nbytes,
            "peak_source": f"{pk['source']} copy bandwidth (of {pk['source']})",
            "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the stage-1 and stage-2 "
                             "launches of one product (profiles/)") if traffic else
                            "null: no DRAM counter capture of this kernel build at this size",
            "compute_frac": forms[args.precision]["compute_frac"]}
    if args.precision in ("bf16", "bf16x3"):
        launches_per_step = 3
        launches_note = ("per step: psi tiling, stage-1 and stage-2 launches of the bulk-copy-fed "
                         "tcgen05 kernel (plus one cudaMemsetAsync of sigma)")
    else:
        launches_per_step = int(st["nlaunch"])
        launches_note = ("per step: the grouped GEMM launches of every task-list chunk "
                         "(plus one cudaMemsetAsync of sigma)")
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision.replace("fp", "f"), "data": "synthetic",
        "config": {"workload": (f"su2_L{L}_N{N}_S0_D{D} centre-bond H_eff psi" if args.symmetry == "su2"
                                else f"u1_L{L}_N{N}_Sz0_D{D} centre-bond H_eff psi"),
                   "symmetry": "SU(2)" if args.symmetry == "su2" else "U(1)xU(1)",
                   "precision": args.precision, "L": L, "N": N, "D": D,
                   "psi_size": st["psi_size"], "terms": st["nterms"],
                   "heff_gflop": flops / 1e9, "env_build_s": env_s,
                   "env_build_tflops": st["env_flops"] / env_s / 1e12,
                   "l2": "operator blocks read per step exceed L2 (no flush needed)",
                   "device_bytes": st2["device_bytes"], "energy_psi_h_psi": energy, "tile": tile,
                   "forms": forms, "fp64_peak_tflops_measured": peak,
                   "pair_switch": args.pair_switch, "sum_gemm": args.sum_gemm, "hbm_budget_gb": args.hbm_budget,
                   "parallelism": f"replicas{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": int(psi.numel() * 8),
                "d2h_bytes_per_step": int(sig.numel() * 8)},
        "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_note": launches_note,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batched(args, rank, world, local):
    """All H_eff psi of 16 independent problems in one captured CUDA graph
    (parallel branches), against the same products launched one by one."""
    import torch
    import qcinputs as q
    import paper_2603_28648_b300 as qd
    torch.cuda.set_device(local)
    prec = qd.PRECISIONS[args.precision]
    ctxs, psis, sigs, shapes = [], [], [], []
    flops = nbytes = 0.0
    t0 = time.perf_counter()
    for w in q.batched_instances():
        h, V = q.make_integrals(w["L"], w["int_seed"])
        c = qd.Context(device=local)
        c.load_integrals(h, V)
        c.set_target(w["N"], w["two_s"])
        c.init_mps(w["D"], w["mps_seed"], w["L"] // 2 - 1)
        c.build_env()
        st = c.stats()
        flops += st["heff_flops"]
        e = {"fp64": 8, "tf32": 4, "bf16": 2, "bf16x3": 6}[args.precision]
        npsi = 2.0 * st["psi_size"]
        nbytes += (st["heff_bytes"] / 8.0 - npsi) * e + 8 * npsi
        p = torch.tensor(c.psi(), device="cuda")
        ctxs.append(c)
        psis.append(p)
        sigs.append(torch.empty_like(p))
        shapes.append(f"L{w['L']}D{w['D']}")
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def one_by_one():
        for c, p, sg in zip(ctxs, psis, sigs):
            c.apply_heff_dev(p.data_ptr(), sg.data_ptr(), stream.cuda_stream, prec)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / args.steps

    t_seq = timed(one_by_one)
    ref = [sg.clone() for sg in sigs]
    g = qd.HeffGraph(ctxs, [p.data_ptr() for p in psis], [sg.data_ptr() for sg in sigs], prec)
    clocks = Clocks(local)
    clocks.start()
    t_graph = timed(lambda: g.launch(stream.cuda_stream))
    clk = clocks.stop()
    for c in ctxs:
        c.check_device()
    diff = max(float((torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()) for a, b in zip(sigs, ref))
    gflops, nodes = g.info()
    pk = measured_peaks()
    line = {
        "metric": "batched H_eff psi TFLOP/s, 16 independent problems in one CUDA graph",
        "value": flops / t_graph / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_graph * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision.replace("fp", "f"), "data": "synthetic",
        "config": {"workload": "16 U(1) problems, L uniform 12..24, N = L, D in {128, 256, 512} (seed 99)",
                   "instances": shapes, "gflop_per_step": flops / 1e9, "graph_nodes": nodes,
                   "one_by_one_ms": t_seq * 1e3, "graph_speedup": t_seq / t_graph,
                   "graph_vs_one_by_one_max_rel_diff": diff, "env_build_s": build_s,
                   "l2": "all operators of the 16 problems stay resident; replays are L2-warm"},
        "roofline": {"bound": "hbm", "achieved": nbytes / t_graph / 1e9, "peak": pk["hbm"], "unit": "GB/s",
                     "frac": nbytes / t_graph / 1e9 / pk["hbm"], "traffic": None},
        "clocks": clk,
    }
    g.close()
    print(json.dumps(line), flush=True)


def run_sweep(args, rank, world, local):
    """Two-site sweep at bond dimension D through the public API, with every
    H_eff psi in FP64 and with the mixed policy (BF16 -> BF16x3 -> FP64
    residual correction), from the same random MPS. The sweep starts at the
    centre bond, runs right to the end, left to the other end and right back
    to the centre: 2(L-2) two-site steps, each a Davidson solve followed by
    truncation, renormalization and preparation of the next centre, timed
    separately. A form stops early when its time budget runs out; the line
    then reports the steps it completed."""
    import torch
    import qcinputs as q
    import paper_2603_28648_b300 as qd
    torch.cuda.set_device(local)
    L, N, D = args.L, args.N, args.D
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    c0 = L // 2 - 1
    order = [+1] * (L - 2 - c0) + [-1] * (L - 2) + [+1] * c0
    out = {}
    for name, kw in (("fp64", dict(policy=0, precision=qd.FP64)), ("mixed", dict(policy=1))):
        ctx = qd.Context(device=local, hbm_budget_gb=args.hbm_budget, pair_switch=args.pair_switch,
                     sum_gemm=args.sum_gemm)
        ctx.load_integrals(h, V)
        ctx.set_target(N, 0)
        ctx.init_mps(D, q.integrals.BASE_SEED + 1002, c0)
        t0 = time.perf_counter()
        ctx.build_env()
        torch.cuda.synchronize()
        env_s = time.perf_counter() - t0
        clocks = Clocks(local)
        clocks.start()
        dav_s, move_s, energies, iters = [], [], [], []
        t_start = time.perf_counter()
        for step, d in enumerate(order):
            t1 = time.perf_counter()
            e, r, it = ctx.davidson(allow_notconv=True, tol=1e-6, max_iter=args.max_iter, **kw)
            t2 = time.perf_counter()
            ctx.truncate(D, d)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            dav_s.append(t2 - t1)
            move_s.append(t3 - t2)
            energies.append(e)
            iters.append(it)
            if t3 - t_start > args.sweep_budget:
                break
        wall = time.perf_counter() - t_start
        out[name] = {"steps_done": len(dav_s), "steps_sweep": len(order), "complete": len(dav_s) == len(order),
                     "wall_s": wall, "davidson_s": sum(dav_s), "truncate_renormalize_s": sum(move_s),
                     "centre_step_s": (dav_s[0] + move_s[0]) if dav_s else None,
                     "step_s": [a + b for a, b in zip(dav_s, move_s)],
                     "energy_last": energies[-1] if energies else None, "energies": energies,
                     "davidson_iters": iters, "env_build_s": env_s, "clocks": clocks.stop()}
        ctx.close()
    f, m = out["fp64"], out["mixed"]
    n = min(f["steps_done"], m["steps_done"])
    line = {
        "metric": f"sweep seconds, one two-site sweep (2(L-2) = {2 * (L - 2)} steps) at L={L}",
        "value": m["wall_s"] if m["complete"] else None, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "dtype": "mixed", "data": "synthetic",
        "config": {"workload": f"u1_L{L}_N{N}_Sz0_D{D} sweep from a random MPS, centre start",
                   "davidson": {"tol": 1e-6, "max_iter": args.max_iter}, "budget_s": args.sweep_budget,
                   "pair_switch": args.pair_switch, "sum_gemm": args.sum_gemm, "hbm_budget_gb": args.hbm_budget,
                   "fp64": f, "mixed": m,
                   "same_steps_compared": n,
                   "speedup_vs_fp64_same_steps": (sum(f["step_s"][:n]) / sum(m["step_s"][:n])) if n else None,
                   "energy_mixed_minus_fp64_last_common_step": (m["energies"][n - 1] - f["energies"][n - 1]) if n else None},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args, rank, world, local):
    """Backward of E(psi, h, V) through the public API at the last centre (L-2, L-1):
    dE/dpsi (one FP64 H_eff psi), gamma = dE/dh from the stored operators, and the spin-summed
    2-RDM element by element by the walk of the centre (qcdmrg_rdm2_sweep, O(L^4) single-term
    products), each timed; checks E = sum h gamma + 1/2 sum V Gamma and the trace of Gamma."""
    import numpy as np
    import torch
    import qcinputs as q
    import paper_2603_28648_b300 as qd
    torch.cuda.set_device(local)
    L, N, D = args.L, args.N, args.D
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    ctx = qd.Context(device=local, hbm_budget_gb=args.hbm_budget, pair_switch=args.pair_switch,
                     sum_gemm=args.sum_gemm)
    ctx.load_integrals(h, V)
    ctx.set_target(N, 0)
    ctx.init_mps(D, q.integrals.BASE_SEED + 1002, L - 2)
    ctx.build_env()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, dpsi, g1, _ = ctx.energy_grad(L, dpsi=True, gamma1=True, gamma2=False)
    t1 = time.perf_counter()
    G = ctx.rdm2_sweep(L)
    t2 = time.perf_counter()
    st = ctx.stats()
    ident = float(np.sum(h * g1) + 0.5 * np.sum(V * G) - E)
    line = {
        "metric": f"adjoint seconds: dE/dpsi, gamma and the 2-RDM (centre walk) at L={L}",
        "value": t2 - t0, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"u1_L{L}_N{N}_Sz0_D{D} random MPS, centre (L-2, L-1)",
                   "dpsi_gamma_s": t1 - t0, "rdm2_walk_s": t2 - t1,
                   "rdm2_elements_measured": (L ** 4 + 3 * L ** 2) // 4,
                   "energy": E, "energy_identity_residual": ident,
                   "trace_gamma2_minus_N(N-1)": float(np.einsum("pprr->", G) - N * (N - 1)),
                   "device_bytes_peak": st["device_bytes"],
                   "pair_switch": args.pair_switch, "hbm_budget_gb": args.hbm_budget},
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.batched:
        if rank == 0:
            run_batched(args, rank, world, local)
    elif args.sweep:
        if rank == 0:
            run_sweep(args, rank, world, local)
    elif args.adjoint:
        if rank == 0:
            run_adjoint(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
