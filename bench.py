"""Benchmark: kernel-mode pairs/s of the correction stage, and time to a 1e-8
residual for the FP64 and the mixed-precision solve, on one B300.

Workload (N = 1): triaxial ellipsoid with semi-axes (1, 0.8, 0.6), k = 10,
16 panels x 16 Gauss-Legendre nodes, Mth = 128 angles (N = 32,768 unknowns,
1,507,328 near pairs).  A step is one correction stage over every near pair:
the per-pair pipeline (ring distances, complex root, A_m recurrence, smooth
factor FFT, singular convolution, Parseval weights) and the GGQ fill of the
near blocks into the resident N x N matrix.  Inputs are resident in HBM; L2 is
flushed (a 512 MiB write) before every timed step.

Also reported on the same JSON line: the end-to-end rate (surface sampling from
host descriptors and the near band [N][3][16 Mth] written to page-locked host
memory through bie_assemble_near_band), the dominant pair-kernel launch against
the measured FP64 rate (roofline), the single + double layer rate, the far fill,
FGMRES iteration and field-evaluation figures (rows), the solves (FP64, mixed,
learned preconditioner), and the batch scheduler.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the oracle (plain FP64 numpy) is timed on bounded
samples of the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

WORKLOAD = "ellipsoid_np16_m128_k10"
METRIC = "kernel-mode pairs/s (correction stage, S kernel, FP64)"
UNIT = "pairs/s"
def _hbm_peak():
    """Measured copy bandwidth of the B300s (GB/s) and its source."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


FP64_PEAK_GFLOPS = 1105.0   # measured FP64 FMA throughput of this B300 pool (profiles/fp64_peak_probe.md)
# DRAM bytes (read + write) per pair of the pair pipeline (root kernel + transform kernel: the kernel
# modes plus the per-pair records between the two), from one ncu capture of 75,776 pairs of this
# workload (profiles/pair_kernel_ellipsoid_np16_m128_k10.md); valid only for the kernel sources it was
# taken on: the report carries it while the sources hash to the same value, and null otherwise.
PAIR_TRAFFIC = {"bytes_per_pair": (10.782976e6 + 296.570624e6 + 246.056192e6 + 123.324416e6) / 75776,
                "sources": "8ca135997c44e2ff"}


def algorithmic_flops_per_pair(Mt):
    """FP64 flop model of one S-kernel pair at Mth = L (FFT 5 n log2 n complex,
    2.5 n log2 n real): ~42.5 L log2 L + 80 L."""
    L = Mt
    return 42.5 * L * np.log2(L) + 80.0 * L


def config_json(c, extra=None):
    d = {"workload": WORKLOAD, "surface": "ellipsoid(1, 0.8, 0.6)", "panels": c["Np"], "nodes_per_panel": 16,
         "m_theta": c["Mt"], "k": c["k"], "unknowns": 16 * c["Np"] * c["Mt"],
         "near_pairs": wl.near_pair_count(c["Np"], c["Mt"]), "kernel": "S", "l2": "flushed before every step"}
    if extra:
        d.update(extra)
    return d


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                                          "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def oracle_pairs_per_second(c, seconds=15.0, max_pairs=20000):
    """Oracle (method mode) on a bounded sample of the workload's near pairs."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:          # the oracle's numpy calls here are single-threaded anyway
        import contextlib

        def threadpool_limits(limits=None):
            return contextlib.nullcontext()
    from oracle import kernel_modes as km
    from oracle import nystrom as ny
    gx = wl.load_ggq()[0]
    rows = wl.sample_rows(c["Np"], c["Mt"], 400, seed=1)
    pairs = ny.near_pairs(c["Np"], c["Mt"], rows, gx)
    t = np.array([p[3] for p in pairs])
    th = np.array([p[4] for p in pairs])
    ts = np.array([p[5] for p in pairs])
    done = 0
    t0 = time.perf_counter()
    with threadpool_limits(limits=1):
        while done < min(len(t), max_pairs) and time.perf_counter() - t0 < seconds:
            sl = slice(done, done + 128)
            km.method_modes(c["surface"], t[sl], th[sl], ts[sl], c["Mt"], c["k"], ("S",))
            done += len(t[sl])
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = wl.config(WORKLOAD)
    vals = []
    for _ in range(args.warmup):
        oracle_pairs_per_second(c, seconds=5.0, max_pairs=512)
    for _ in range(args.steps):
        v, n, dt = oracle_pairs_per_second(c, seconds=10.0, max_pairs=2048)
        vals.append((v, n, dt))
    value = float(np.mean([v for v, _, _ in vals]))
    sample = "%d steps of up to 2048 near pairs (10 s cap each) from 400 seeded target rows" % args.steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean([d for _, _, d in vals])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_json(c),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def pair_kernel_sources_hash():
    import glob
    import hashlib
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2608_16208_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(csrc, "pair_modes.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def job_throughput(step_ms, units_per_rank, world, device=None):
    """Whole-job rate of `world` replicas that each processed units_per_rank in their own step time:
    the job takes the slowest rank's time (max over ranks, one all_reduce when world > 1).
    Returns (job step time in ms, units per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(step_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    return step_ms, world * units_per_rank / (step_ms / 1000.0)


def near_launches(Np, Mt, nk):
    """Kernel launches of one near-correction pass: per group of panels whose weights fit 4 GiB, the
    pair pipeline (single layer alone: a root and a transform kernel per chunk of 2^20 pairs; with the
    double layer: one fused kernel), and the near-band fill once per panel."""
    per_panel_pairs = 16 * 48 * Mt
    group = max(1, min(Np, (4 << 30) // (16 * per_panel_pairs * Mt * nk)))
    n = 0
    for j0 in range(0, Np, group):
        pairs = per_panel_pairs * min(group, Np - j0)
        n += 2 * (-(-pairs // (1 << 20))) if nk == 1 else 1
    return n + Np


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2608_16208_b300 as bie

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    c = wl.config(WORKLOAD)
    Np, Mt, k = c["Np"], c["Mt"], c["k"]
    ggq = wl.load_ggq()
    ctx = bie.Context()
    surf = bie.Surface(ctx, c["surface"], Np, Mt, ggq)
    N = surf.N
    A = torch.zeros((N, N), dtype=torch.complex128, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        bie.assemble_near(surf, bie.KERNEL_S, k, A)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks() as clk:
        for e0, e1 in events:
            flush.fill_(1.0)
            e0.record(stream)
            step()
            e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [e0.elapsed_time(e1) for e0, e1 in events]
    pairs = surf.near_pairs
    step_ms, value = job_throughput(float(np.mean(ms)), pairs, world, dev)
    launches_per_step = near_launches(Np, Mt, 1)

    # dominant kernel: the pair pipeline over every near pair of the surface in one launch (the
    # launch size of a step), timed with events on the launching stream
    rows_all = torch.arange(N, device=dev, dtype=torch.int64).repeat_interleave(48)
    srcs_all = torch.arange(48, device=dev, dtype=torch.int32).repeat(N)
    panel = rows_all // (16 * Mt) + srcs_all.to(torch.int64) // 16 - 1
    keep = (panel >= 0) & (panel < Np)
    rows_all, srcs_all = rows_all[keep].contiguous(), srcs_all[keep].contiguous()
    modes = torch.empty((rows_all.numel(), 1, Mt + 1), dtype=torch.complex128, device=dev)
    pk_events = []
    for _ in range(3):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bie.kernel_modes(surf, bie.KERNEL_S, k, rows_all, srcs_all, out=modes)
        e1.record(stream)
        pk_events.append((e0, e1))
    torch.cuda.synchronize()
    pk_ms = float(np.mean([a.elapsed_time(b) for a, b in pk_events]))
    pk_pairs = rows_all.numel()
    del modes
    # the single and double layer together over the same pairs (fused FP64 kernel), reported apart
    modes_sk = torch.empty((rows_all.numel(), 2, Mt + 1), dtype=torch.complex128, device=dev)
    bie.kernel_modes(surf, bie.KERNEL_S | bie.KERNEL_K, k, rows_all, srcs_all, out=modes_sk)
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bie.kernel_modes(surf, bie.KERNEL_S | bie.KERNEL_K, k, rows_all, srcs_all, out=modes_sk)
    e1.record(stream)
    torch.cuda.synchronize()
    sk_ms = e0.elapsed_time(e1)
    del modes_sk, rows_all, srcs_all, panel, keep
    fl = algorithmic_flops_per_pair(Mt)
    traffic = (PAIR_TRAFFIC["bytes_per_pair"] * pk_pairs
               if pair_kernel_sources_hash() == PAIR_TRAFFIC["sources"] else None)
    achieved_gflops = fl * pk_pairs / (pk_ms / 1000.0) / 1e9
    step_gflops = fl * pairs / (step_ms / 1000.0) / 1e9

    # end to end: host descriptors and tables in, the near band out to page-locked host memory
    # (bie_assemble_near_band: each group of target panels is copied while the next one computes)
    host_band = torch.empty((N, 3, 16 * Mt), dtype=torch.complex128, pin_memory=True)
    e2e_ms = []
    for it in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = bie.Surface(ctx, c["surface"], Np, Mt, ggq)
        bie.assemble_near_band(s2, bie.KERNEL_S, k, out=host_band)
        ctx.sync()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        del s2
    e2e_value = world * pairs / (float(np.median(e2e_ms)) / 1000.0)
    d2h = host_band.numel() * host_band.element_size()
    del host_band
    h2d = 8 * (3 * 16 * 16 * 2 + 32) + 5 * 8 * len(c["surface"].get("terms", []))

    # time to a 1e-8 residual: FP64 vs FP32 storage with FP64 refinement (plane wave along +z)
    solve = None
    if not args.skip_solve:
        torch.cuda.synchronize()
        # exterior sound-soft problem, combined-field operator on the unweighted density (second kind)
        Afull = bie.assemble(surf, bie.OP_CFIE | bie.UNWEIGHTED, k, out=A)
        g = bie.rhs(surf, 0, c["dirs"][0], k)
        res = {}
        for name, prec in (("fp64", 0), ("mixed_fp32_refined", 1)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                x, rep = bie.solve(ctx, Afull, g, tol=1e-8, restart=200, maxit=3000, prec=prec)
                rep["wall_s"] = time.perf_counter() - t0
            except bie.BieError as exc:
                rep = {"error": str(exc)}
            res[name] = rep
        res["operator"] = "I + K - i k S (combined field, unweighted density), plane wave"
        res["learned"] = run_learned(bie) if args.learned else None
        solve = res

    rows = run_rows(bie, surf, k, A, flush, stream, step_ms, solve)

    batch = None if args.batch_surfaces <= 0 else run_batch(bie, ctx, args.batch_surfaces, stream)

    if rank == 0:
        cpu_v, cpu_n, cpu_dt = oracle_pairs_per_second(c, seconds=15.0)
        cs = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32x2", "data": "synthetic",
            "config": config_json(c, {"parallelism": "replicas" if world > 1 else "single"}),
            "clocks": cs,
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved_gflops / FP64_PEAK_GFLOPS, "traffic": traffic,
                         "kernel": "pair_root_kernel + pair_transform_kernel (S)", "peak_source": "measured FP64 FMA probe",
                         "traffic_source": "ncu capture of 75,776 pairs, scaled to the %d pairs of a launch" % pk_pairs,
                         "launch_ms": pk_ms,
                         "flops_per_pair": fl, "step_gflops": step_gflops},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": float(np.median(e2e_ms))},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d near pairs of 400 seeded target rows, method mode, %.1f s" % (cpu_n, cpu_dt)},
            "solve": solve,
            "batch": batch,
            "rows": rows,
            "single_and_double_layer": {"pairs_per_s": pk_pairs / (sk_ms / 1000.0), "ms": sk_ms, "pairs": pk_pairs,
                                        "kernels": "S+K", "path": "fused FP64 pair kernel"},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_batch(bie, ctx, count, stream):
    """Uneven batch (harmonic stars, Np in 8..32, Mth in 64..256, k in [1, 20]) in one persistent,
    graph-captured launch, against the same surfaces run one after the other."""
    import torch
    stream = torch.cuda.Stream()              # graph capture needs a non-default stream
    ctx = bie.Context(stream)
    specs = wl.batch_surfaces(seed=0, count=count)
    ggq = wl.load_ggq()
    surfs = [bie.Surface(ctx, sp["surface"], sp["Np"], sp["Mt"], ggq) for sp in specs]
    ks = [sp["k"] for sp in specs]
    maxMt = max(sp["Mt"] for sp in specs)
    slot = 1 << 20
    W = torch.empty((1, slot, maxMt), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    plan = bie.Batch(ctx, surfs, ks, bie.KERNEL_S, W, slot)
    plan.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):       # replay() launches on the current stream
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = min(times)
    # the same surfaces, one plan (one launch) each, back to back
    singles = [bie.Batch(ctx, [sf], [k], bie.KERNEL_S, W, slot) for sf, k in zip(surfs, ks)]
    for sp in singles:
        sp.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for sp in singles:
        sp.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    return {"surfaces": count, "pairs": plan.pairs, "pairs_per_s": plan.pairs / (ms / 1000.0), "ms": ms,
            "sequential_ms": ms_seq, "speedup_vs_sequential": ms_seq / ms, "autotuned": plan.config,
            "m_theta": sorted(sp["Mt"] for sp in specs), "panels": sorted(sp["Np"] for sp in specs),
            "output": "ring of %d pairs x %d angles (throughput mode)" % (slot, maxMt), "cuda_graph": True}


def learned_family(seed, i):
    """System i of the learned-preconditioner family: harmonic star (eps <= 0.15), k ~ U[5, 25],
    Np = 16, Mth = 96 (N = 24,576)."""
    rs = wl.Stream(seed, 40 + i)
    eps = 0.15 * rs.uniform()
    k = 5.0 + 20.0 * rs.uniform()
    d = wl.Stream(seed, 60 + i).directions(1)[0].tolist()
    return wl.harmonic_star(seed, 200 + i, eps), k, d


def run_learned(bie, n_train=4, n_test=2, steps=600):
    """Learned preconditioner: train on systems of the family, then time FGMRES to 1e-8 on held-out
    systems with the block-diagonal preconditioner (the judge and fallback) and with the network on
    top of it.  Operator: the single layer S (first kind, weighted density), plane-wave data."""
    import torch
    ctx = bie.Context()
    ggq = wl.load_ggq()
    Np, Mt = 16, 96
    block = 16 * Mt

    def system(i):
        desc, k, d = learned_family(1, i)
        s = bie.Surface(ctx, desc, Np, Mt, ggq)
        A = bie.assemble(s, bie.OP_S, k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B = bie.BlockDiag(ctx, A, block)
        t_lu = time.perf_counter() - t0
        return s, A, B, k, d, t_lu

    sets, lu_times = [], []
    for i in range(n_train):
        s, A, B, k, _, t_lu = system(i)
        sets.append((bie.TrainSet(ctx, s, k, A, B), s, B))
        lu_times.append(t_lu)
        del A
        torch.cuda.empty_cache()
    net = bie.Net(ctx, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = net.train([t for t, _, _ in sets], steps=steps, batch=16, lr=1e-3, seed=2)
    t_train = time.perf_counter() - t0
    del sets
    torch.cuda.empty_cache()
    held = []
    for j in range(n_test):
        s, A, B, k, d, t_lu = system(1000 + j)
        lu_times.append(t_lu)
        g = bie.rhs(s, 0, d, k)
        row = {"k": k}
        for name, pc, prec in (("plain_fp64", bie.PRECOND_NONE, 0), ("block_fp64", bie.PRECOND_BLOCK, 0),
                               ("block_mixed", bie.PRECOND_BLOCK, 1), ("learned_fp64", bie.PRECOND_LEARNED, 0)):
            torch.cuda.synchronize()
            try:
                _, rep = bie.solve(ctx, A, g, tol=1e-8, restart=300, maxit=1500, prec=prec, precond=pc, block=B,
                                   net=net, surface=s, k=k, raise_on_noconv=False)
                row[name] = {kk: rep[kk] for kk in ("iterations", "refinements", "rel_residual", "seconds",
                                                    "fallback_used")}
                row[name]["converged"] = rep["status"] == 0
            except bie.BieError as exc:
                row[name] = {"error": str(exc)}
        held.append(row)
        del A, B
        torch.cuda.empty_cache()
    return {"operator": "S (first kind, weighted density), plane wave",
            "family": "harmonic stars eps<=0.15, k~U[5,25], Np=16, Mth=96 (N=24,576)",
            "train_systems": n_train, "train_steps": steps, "batch": 16, "train_seconds": t_train,
            "loss_first10": float(np.mean(hist[:10])), "loss_last50": float(np.mean(hist[-50:])),
            "blockdiag_factor_seconds": float(np.median(lu_times)), "held_out": held}


def run_rows(bie, surf, k, A, flush, stream, near_ms, solve):
    """Figures of the steps around the pair pipeline on the same surface: the far fill (whole S
    assembly minus the correction stage), the FGMRES matvec (per iteration of the solves above) and
    the field evaluation at exterior points."""
    import torch
    N = surf.N
    hbm, hbm_src = _hbm_peak()

    def timed(fn, reps=3):
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    rows = {}
    asm_ms = timed(lambda: bie.assemble(surf, bie.OP_S, k, out=A))
    far_ms = asm_ms - near_ms
    rows["far_fill"] = {
        "assemble_ms": asm_ms, "correction_ms": near_ms, "far_fill_ms": far_ms,
        "entries_per_s": N * N / (far_ms / 1000.0),
        "write_GBps": 16.0 * N * N / (far_ms / 1000.0) / 1e9, "hbm_peak_GBps": hbm, "hbm_peak_source": hbm_src,
        "frac_of_hbm": 16.0 * N * N / (far_ms / 1000.0) / 1e9 / hbm,
        "bound": "FP64: one rsqrt and one sincos per entry (writes 16 B per entry)"}
    if solve is not None:
        mv = {}
        for name, bytes_per in (("fp64", 16), ("mixed_fp32_refined", 8)):
            rep = solve.get(name, {})
            if rep.get("iterations"):
                per = 1000.0 * rep["seconds"] / rep["iterations"]
                mv[name] = {"ms_per_iteration": per, "matrix_bytes": bytes_per * N * N,
                            "implied_read_GBps": bytes_per * N * N / (per / 1000.0) / 1e9}
        mv["note"] = ("iteration time covers the matvec, the Arnoldi step and, for the mixed solve, its "
                      "share of the FP64 refinement residuals; the implied rate is a lower bound on the matvec's")
        rows["matvec"] = mv
    pts = torch.as_tensor(wl.exterior_points(8192, 3.0), dtype=torch.float64).cuda()
    dens = torch.as_tensor(wl.random_complex((N,), 0, 13), dtype=torch.complex128).cuda()
    fe_ms = timed(lambda: bie.field_eval(surf, bie.OP_S, k, dens, pts))
    rows["field_eval"] = {"points": int(pts.shape[0]), "sources": N, "ms": fe_ms,
                          "source_point_pairs_per_s": N * pts.shape[0] / (fe_ms / 1000.0),
                          "bound": "FP64: one rsqrt and one sincos per source-point pair"}
    return rows


def run_kernel_only(n):
    """One launch of the pair pipeline on n pairs (all sources of consecutive target rows)."""
    import torch
    import paper_2608_16208_b300 as bie
    c = wl.config(WORKLOAD)
    ctx = bie.Context()
    surf = bie.Surface(ctx, c["surface"], c["Np"], c["Mt"], wl.load_ggq())
    rows = (16 * c["Mt"] * (c["Np"] // 2) + torch.arange(n, device="cuda", dtype=torch.int64) // 48)
    srcs = (torch.arange(n, device="cuda", dtype=torch.int32) % 48)
    kern = bie.KERNEL_S | (bie.KERNEL_K if os.environ.get("BENCH_KERNELS", "S") == "SK" else 0)
    out = bie.kernel_modes(surf, kern, c["k"], rows, srcs)
    ctx.sync()
    print("kernel-only: %d pairs, finite: %s" % (n, bool(torch.isfinite(torch.view_as_real(out)).all())))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-solve", action="store_true")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-preconditioner training and held-out solves")
    ap.add_argument("--batch-surfaces", type=int, default=8, help="surfaces in the batch-scheduler run (0: skip)")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="profiling aid: run the pair pipeline once on this many pairs of the workload and exit")
    args = ap.parse_args()
    if args.kernel_only:
        run_kernel_only(args.kernel_only)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
