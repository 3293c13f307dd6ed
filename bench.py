"""Benchmark: kernel-mode pairs/s of the correction stage, and time to a 1e-8
residual for the FP64 and the mixed-precision solve, on one B300.

Workload (N = 1): triaxial ellipsoid with semi-axes (1, 0.8, 0.6), k = 10,
16 panels x 16 Gauss-Legendre nodes, Mth = 128 angles (N = 32,768 unknowns,
1,507,328 near pairs).  A step is one correction stage over every near pair:
the per-pair pipeline (ring distances, complex root, A_m recurrence, smooth
factor FFT, singular convolution, Parseval weights) and the GGQ fill of the
near blocks into the resident N x N matrix.  Inputs are resident in HBM; L2 is
flushed (a 512 MiB write) before every timed step.

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
FP64_PEAK_GFLOPS = 1105.0   # measured FP64 FMA throughput of this B300 pool (profiles/fp64_peak_probe.md)
# DRAM bytes (read + write) per pair of the pair kernel, from one ncu capture of 75,776 pairs of this
# workload (profiles/pair_kernel_ellipsoid_np16_m128_k10.md), valid only for the kernel source it was
# taken on: the report carries it while the sources hash to the same value, and null otherwise.
PAIR_TRAFFIC = {"bytes_per_pair": (68.090624e6 + 292.715776e6) / 75776, "sources": "be4bc295f36c51fe"}


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


def near_launches(Np, Mt, nk):
    """Kernel launches of one near-correction pass: the pair pipeline once per group of panels whose
    weights fit 4 GiB, and the near-band fill once per panel."""
    per_panel = 16 * (16 * 48 * Mt) * Mt * nk
    group = max(1, min(Np, (4 << 30) // per_panel))
    return -(-Np // group) + Np


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
    step_ms = float(np.mean(ms))
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    pairs = surf.near_pairs
    value = world * pairs / (step_ms / 1000.0)
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
    del modes, rows_all, srcs_all, panel, keep
    fl = algorithmic_flops_per_pair(Mt)
    traffic = (PAIR_TRAFFIC["bytes_per_pair"] * pk_pairs
               if pair_kernel_sources_hash() == PAIR_TRAFFIC["sources"] else None)
    achieved_gflops = fl * pk_pairs / (pk_ms / 1000.0) / 1e9
    step_gflops = fl * pairs / (step_ms / 1000.0) / 1e9

    # end to end: host descriptors and tables in, near-band entries out to pinned host memory
    band = 3 * 16 * Mt
    host_band = torch.empty((N, band), dtype=torch.complex128, pin_memory=True)
    e2e_ms = []
    for it in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = bie.Surface(ctx, c["surface"], Np, Mt, ggq)
        bie.assemble_near(s2, bie.KERNEL_S, k, A)
        for j in range(Np):
            lo = max(j - 1, 0) * 16 * Mt
            hi = min(j + 2, Np) * 16 * Mt
            r0, r1 = j * 16 * Mt, (j + 1) * 16 * Mt
            host_band[r0:r1, : hi - lo].copy_(A[r0:r1, lo:hi], non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        del s2
    e2e_value = world * pairs / (float(np.median(e2e_ms)) / 1000.0)
    d2h = sum((min(j + 2, Np) - max(j - 1, 0)) * 16 * Mt * 16 * Mt * 16 for j in range(Np))
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
        res["learned"] = None
        res["operator"] = "I + K - i k S (combined field, unweighted density), plane wave"
        solve = res

    batch = None if args.batch_surfaces <= 0 else run_batch(bie, ctx, args.batch_surfaces, stream)

    if rank == 0:
        cpu_v, cpu_n, cpu_dt = oracle_pairs_per_second(c, seconds=15.0)
        cs = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(c, {"parallelism": "replicas" if world > 1 else "single"}),
            "clocks": cs,
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved_gflops / FP64_PEAK_GFLOPS, "traffic": traffic,
                         "kernel": "pair_kernel<S>", "peak_source": "measured FP64 FMA probe",
                         "traffic_source": "ncu capture of 75,776 pairs, scaled to the %d pairs of a launch" % pk_pairs,
                         "launch_ms": pk_ms,
                         "flops_per_pair": fl, "step_gflops": step_gflops},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": float(np.median(e2e_ms))},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d near pairs of 400 seeded target rows, method mode, %.1f s" % (cpu_n, cpu_dt)},
            "solve": solve,
            "batch": batch,
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
