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
METRIC = "kernel-mode pairs/s (correction stage, S kernel)"
# what the headline's arithmetic is: the per-pair root, recurrences and samples in FP64; the
# transforms, products and unpacking in double-word FP32 pairs (about 48 significant bits)
PRECISION = {"root_newton": "f64", "a_m_recurrences": "f64", "samples_rho2_F_phases": "f64",
             "transforms_products_unpacking": "double-word f32x2 (about 2^-48 per operation)",
             "outputs": "f64", "parity_bound_per_pair": 1e-12}
UNIT = "pairs/s"
def _hbm_peak():
    """Measured copy bandwidth of the B300s (GB/s) and its source."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def fp64_peak_gflops():
    """FP64 throughput of this GPU measured now: cuBLAS DGEMM 4096^3 (2 n^3 flops), best of 3, CUDA
    events.  MEASURED_PEAKS.json has no FP64 figure, and the pair pipeline's roofline is FP64."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best / 1000.0) / 1e9


# DRAM bytes (read + write) per pair of the pair pipeline (root kernel + transform kernel: the kernel
# modes plus the per-pair records between the two), from one ncu capture of 75,776 pairs of this
# workload; valid only for the kernel sources it was taken on: the report carries it while the
# sources hash to the same value, and null otherwise.
PAIR_TRAFFIC = {"bytes_per_pair": (20.452608e6 + 288.863488e6 + 245.873408e6 + 124.057856e6) / 75776,
                "sources": "4623af80c9a2424d"}


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


def host_cores():
    """Host CPU threads this process may run on, and the CPU model (read at run time)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return n, model


def _oracle_worker(job):
    """One host process: the oracle's method mode on its own slice of pairs for a bounded time."""
    surface, Mt, k, t, th, ts, seconds = job
    from oracle import kernel_modes as km
    done = 0
    t0 = time.perf_counter()
    while done < len(t) and time.perf_counter() - t0 < seconds:
        sl = slice(done, done + 64)
        km.method_modes(surface, t[sl], th[sl], ts[sl], Mt, k, ("S",))
        done += len(t[sl])
    return done, time.perf_counter() - t0


def oracle_pairs_per_second(c, seconds=15.0, max_pairs=None, cores=None):
    """Oracle (method mode, S) on a bounded sample of the workload's near pairs, one single-threaded
    process per host core (spawned), each on its own slice of pairs; rate = all pairs / the longest
    process's time.  Returns (pairs/s, pairs, seconds, cores)."""
    import multiprocessing as mp
    from oracle import nystrom as ny
    cores = cores or host_cores()[0]
    gx = wl.load_ggq()[0]
    rows = wl.sample_rows(c["Np"], c["Mt"], max(400, 40 * cores), seed=1)
    pairs = ny.near_pairs(c["Np"], c["Mt"], rows, gx)
    if max_pairs:
        pairs = pairs[:max_pairs]
    t = np.array([p[3] for p in pairs])
    th = np.array([p[4] for p in pairs])
    ts = np.array([p[5] for p in pairs])
    per = -(-len(t) // cores)
    jobs = [(c["surface"], c["Mt"], c["k"], t[i * per:(i + 1) * per], th[i * per:(i + 1) * per],
             ts[i * per:(i + 1) * per], seconds) for i in range(cores) if i * per < len(t)]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"      # inherited by the spawned processes: one thread each
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_worker, jobs)
    done = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return done / dt, done, dt, len(jobs)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = wl.config(WORKLOAD)
    cores, model = host_cores()
    vals = []
    for _ in range(args.warmup):
        oracle_pairs_per_second(c, seconds=2.0, cores=cores)
    for _ in range(args.steps):
        v, n, dt, used = oracle_pairs_per_second(c, seconds=6.0, cores=cores)
        vals.append((v, n, dt))
    value = float(np.mean([v for v, _, _ in vals]))
    sample = ("%d steps, each up to 6 s of near pairs of seeded target rows on %d single-threaded processes "
              "(%s)" % (args.steps, used, model))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean([d for _, _, d in vals])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_json(c),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
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
    ctx.trace(True)    # per-kernel CUDA events inside the steps (the library's launch trace)
    with Clocks() as clk:
        for e0, e1 in events:
            flush.fill_(1.0)
            e0.record(stream)
            step()
            e1.record(stream)
        torch.cuda.synchronize()
    trace = ctx.trace_read()
    ctx.trace(False)
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
    # the same launch with the single layer's transforms in FP64 (context option): what the double-word
    # arithmetic buys, on the same pairs
    ctx.set_option(bie.OPT_FP64_TRANSFORMS, 1)
    bie.kernel_modes(surf, bie.KERNEL_S, k, rows_all, srcs_all, out=modes)
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bie.kernel_modes(surf, bie.KERNEL_S, k, rows_all, srcs_all, out=modes)
    e1.record(stream)
    torch.cuda.synchronize()
    f64_ms = e0.elapsed_time(e1)
    ctx.set_option(bie.OPT_FP64_TRANSFORMS, 0)
    pick64 = np.unique(wl.Stream(11, 5).integers(0, pk_pairs - 1, 128))
    pick64_d = torch.from_numpy(pick64).to(dev)
    f64_rows, f64_srcs = rows_all[pick64_d].cpu().numpy(), srcs_all[pick64_d].cpu().numpy()
    f64_got = modes[pick64_d, 0].cpu().numpy()
    # and again in double words, so that the accuracy sample below comes from the timed arithmetic
    bie.kernel_modes(surf, bie.KERNEL_S, k, rows_all, srcs_all, out=modes)
    torch.cuda.synchronize()
    # accuracy of the timed launch: 256 seeded pairs of its output against the oracle, one by one
    pick = np.unique(wl.Stream(11, 4).integers(0, pk_pairs - 1, 256))
    pick_d = torch.from_numpy(pick).to(dev)
    acc_rows, acc_srcs = rows_all[pick_d].cpu().numpy(), srcs_all[pick_d].cpu().numpy()
    acc_got = modes[pick_d, 0].cpu().numpy()
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
    del modes_sk
    banded = run_banded_route(bie, surf, k, rows_all, srcs_all, flush, stream)
    del rows_all, srcs_all, panel, keep
    fp64_peak = fp64_peak_gflops()
    fl = algorithmic_flops_per_pair(Mt)
    traffic = (PAIR_TRAFFIC["bytes_per_pair"] * pairs
               if pair_kernel_sources_hash() == PAIR_TRAFFIC["sources"] else None)
    # the dominant kernels: the pair pipeline (root + transform) inside the timed steps, per step
    pipe_ms = (trace["pair_root"][0] + trace["pair_transform"][0]) / args.steps
    achieved_gflops = fl * pairs / (pipe_ms / 1000.0) / 1e9
    step_gflops = fl * pairs / (step_ms / 1000.0) / 1e9
    launch_gflops = fl * pk_pairs / (pk_ms / 1000.0) / 1e9

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

    acc = accuracy_vs_oracle(c, acc_rows, acc_srcs, acc_got)
    acc64 = accuracy_vs_oracle(c, f64_rows, f64_srcs, f64_got)

    # time to a 1e-8 residual: FP64 vs the mixed solves, on this workload (4 plane waves + a point
    # source) and on the bumpy surface at k = 20 (N = 49,152; plane wave + point source)
    solve = None
    if not args.skip_solve:
        solve = {"ellipsoid_np16_m128_k10": run_solves(bie, ctx, surf, c, A)}
        mv_rows = solve["ellipsoid_np16_m128_k10"]
        rows = run_rows(bie, surf, k, A, flush, stream, step_ms, mv_rows)
        del A
        torch.cuda.empty_cache()
        c4 = wl.config("bumpy_np24_m128_k20")
        s4 = bie.Surface(ctx, c4["surface"], c4["Np"], c4["Mt"], ggq)
        solve["bumpy_np24_m128_k20"] = run_solves(bie, ctx, s4, c4, None)
        del s4
        torch.cuda.empty_cache()
        solve["learned"] = run_learned(bie) if args.learned else None
    else:
        rows = run_rows(bie, surf, k, A, flush, stream, step_ms, None)

    batch = None if args.batch_surfaces <= 0 else run_batch(bie, ctx, args.batch_surfaces, stream)

    if rank == 0:
        cpu_v, cpu_n, cpu_dt, cpu_cores = oracle_pairs_per_second(c, seconds=12.0)
        cpu_model = host_cores()[1]
        cs = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32x2", "data": "synthetic",
            "config": config_json(c, {"parallelism": "replicas" if world > 1 else "single"}),
            "clocks": cs,
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved_gflops, "peak": fp64_peak, "unit": "GFLOP/s",
                         "frac": achieved_gflops / fp64_peak, "traffic": traffic,
                         "kernel": "pair_root_kernel + pair_transform_kernel (S), as launched inside the timed "
                                   "steps (library launch trace: CUDA events on the context's stream)",
                         "pipeline_ms_per_step": pipe_ms,
                         "step_kernel_ms": {kk: v[0] / args.steps for kk, v in trace.items()},
                         "step_kernel_launches": {kk: v[1] / args.steps for kk, v in trace.items()},
                         "peak_source": "FP64 measured in this run: cuBLAS DGEMM 4096^3, best of 3 (the transforms "
                                        "run on the FP32 pipe, so this is an FP64-equivalent fraction)",
                         "traffic_source": "ncu capture of 75,776 pairs, scaled to the %d pairs of a step" % pairs,
                         "flops_per_pair": fl, "step_gflops": step_gflops,
                         "modes_launch": {"pairs": pk_pairs, "ms": pk_ms, "gflops": launch_gflops}},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": float(np.median(e2e_ms))},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_cores, "kind": "oracle",
                             "sample": "%d near pairs of seeded target rows, method mode, %.1f s on %d "
                                       "single-threaded processes (%s)" % (cpu_n, cpu_dt, cpu_cores, cpu_model)},
            "precision": PRECISION,
            "accuracy_vs_oracle": acc,
            "fp64_only": {"pairs_per_s": pk_pairs / (f64_ms / 1000.0), "ms": f64_ms, "pairs": pk_pairs,
                          "double_word_pairs_per_s": pk_pairs / (pk_ms / 1000.0),
                          "speedup_of_double_words": f64_ms / pk_ms, "accuracy_vs_oracle": acc64,
                          "path": "the same kernel-modes launch with the transforms, upsampling, products and "
                                  "unpacking in FP64 (BIE_OPT_FP64_TRANSFORMS)"},
            "solve": solve,
            "batch": batch,
            "rows": rows,
            "single_and_double_layer": {"pairs_per_s": pk_pairs / (sk_ms / 1000.0), "ms": sk_ms, "pairs": pk_pairs,
                                        "kernels": "S+K", "path": "fused FP64 pair kernel"},
            "banded_route": banded,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_banded_route(bie, surf, k, rows_all, srcs_all, flush, stream, n=75776):
    """The O(M) route to the single layer (Section 3.3, Eq. (Sphi:appr2) over the banded system
    Eq. (Axb)) on the first n pairs of the workload: its rate, one launch timed with events after a
    warm-up, and its normwise difference from the singularity-swapping route on the same pairs."""
    import torch
    n = min(n, rows_all.numel())
    r, c = rows_all[:n].contiguous(), srcs_all[:n].contiguous()
    out = bie.kernel_modes_banded(surf, k, r, c)
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bie.kernel_modes_banded(surf, k, r, c, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ref = bie.kernel_modes(surf, bie.KERNEL_S, k, r, c)[:, 0]
    surf.ctx.sync()
    diff = (out - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)
    return {"pairs": n, "ms": ms, "pairs_per_s": n / (ms / 1000.0),
            "vs_swapped_route": {"max_normwise": float(diff.max()), "median_normwise": float(diff.median())},
            "path": "bie_kernel_modes_banded: <rho^{-1}>_l by the banded system (m0 = 2 on the ellipsoid), "
                    "boundary modes by graded Gauss-Legendre quadrature, convolution with the grid modes "
                    "of cos(k rho)"}


def accuracy_vs_oracle(c, rows, srcs, got):
    """Normwise error, per pair, of sampled outputs of the timed launch against the oracle's method
    mode (max_m |gpu - oracle| / max_m |oracle|)."""
    from oracle import kernel_modes as km
    from oracle import nystrom as ny
    gx = wl.load_ggq()[0]
    Np, Mt = c["Np"], c["Mt"]
    t_nodes, h = ny.nodes(Np)
    tn, i, d, g = rows // Mt, rows % Mt, srcs // 16, srcs % 16
    ts = (tn // 16 + d - 1 + 0.5) * h + (h / 2) * gx[d, tn % 16, g]
    ref = np.concatenate([km.method_modes(c["surface"], t_nodes[tn[q:q + 128]], 2 * np.pi * i[q:q + 128] / Mt,
                                          ts[q:q + 128], Mt, c["k"], ("S",))["S"] for q in range(0, len(rows), 128)])
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return {"pairs": int(len(rows)), "max_normwise": float(err.max()), "median_normwise": float(np.median(err)),
            "kernel": "S", "sample": "seeded pairs of the timed kernel-modes launch over every near pair"}


def run_solves(bie, ctx, surf, c, A=None):
    """Time to a 1e-8 relative residual for the exterior sound-soft problem through the combined-field
    operator I + K - i k S (unweighted density), all right-hand sides in lockstep (plane waves along the
    workload's directions and the interior point source): FP64 products throughout; FP32 storage inside
    FGMRES; split-BF16 storage on the tensor cores inside FGMRES (both with FP64-accurate refinement).
    The matrix is assembled once; its FP32 and split-BF16 copies are made once (timed apart)."""
    import torch
    k = c["k"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A = bie.assemble(surf, bie.OP_CFIE | bie.UNWEIGHTED, k, out=A)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    B = torch.stack([bie.rhs(surf, 0, d, k) for d in c["dirs"]] + [bie.rhs(surf, 1, c["src"], k)])
    t0 = time.perf_counter()
    M = bie.Matrix(ctx, A, bie.STORE_FP32 | bie.STORE_BF16X2)
    torch.cuda.synchronize()
    t_copy = time.perf_counter() - t0
    dirs = wl.Stream(0, 21).directions(32)
    out = {"unknowns": surf.N, "rhs": int(B.shape[0]), "k": k, "tol": 1e-8,
           "operator": "I + K - i k S (combined field, unweighted density)",
           "assemble_s": t_asm, "low_precision_copies_s": t_copy, "far_field_directions": 32}
    ff = {}
    for name, prec in (("fp64", 0), ("mixed_fp32", 1), ("mixed_bf16x2_tensor_cores", 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            X, rep = M.solve(B, tol=1e-8, restart=200, maxit=3000, prec=prec)
            rep["wall_s"] = time.perf_counter() - t0
            rep["ms_per_iteration"] = 1000.0 * rep["seconds"] / max(1, rep["iterations"])
            ff[name] = np.stack([bie.field_eval(surf, bie.OP_CFIE | bie.UNWEIGHTED, k, X[j].contiguous(), dirs,
                                                far_field=True).cpu().numpy() for j in range(B.shape[0])])
        except bie.BieError as exc:
            rep = {"error": str(exc)}
        out[name] = rep
    # far-field errors: against the FP64 solve (every right-hand side) and, for the point source, against
    # its exact far field e^{-ik d.x_src} / (4 pi) (the manufactured solution)
    exact = np.exp(-1j * k * (dirs @ np.asarray(c["src"], float))) / (4 * np.pi)
    for name, u in ff.items():
        e = {"point_source_vs_exact": float(np.linalg.norm(u[-1] - exact) / np.linalg.norm(exact))}
        if name != "fp64" and "fp64" in ff:
            ref = ff["fp64"]
            e["vs_fp64_max_over_rhs"] = float(max(np.linalg.norm(u[j] - ref[j]) / np.linalg.norm(ref[j])
                                                  for j in range(len(u))))
        out[name]["far_field_error"] = e
    if "seconds" in out.get("fp64", {}):
        for name in ("mixed_fp32", "mixed_bf16x2_tensor_cores"):
            if "seconds" in out.get(name, {}):
                out[name]["speedup_vs_fp64"] = out["fp64"]["seconds"] / out[name]["seconds"]
    del M
    return out


def run_batch(bie, ctx, count, stream):
    """Uneven batch (harmonic stars, Np in 8..32, Mth in 64..256, k in [1, 20]) replayed from a CUDA graph
    (one class of equal grid size after another), against the same surfaces as single-surface plans run
    one after the other.  Throughput mode: the Parseval weights go to a ring of 2^20 pair rows and every
    target panel, once its pairs are done, is folded by the GGQ fill into a ring of near-band slots (the
    right-hand sides are not part of this measurement)."""
    import torch
    stream = torch.cuda.Stream()              # graph capture needs a non-default stream
    ctx = bie.Context(stream)
    all_specs = wl.batch_surfaces(seed=0, count=count)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    # sharding over ranks (one GPU each): the surfaces share no pairs, so each rank plans its own share
    # (longest-processing-time by near pairs x log2 Mth) and nothing moves between ranks
    costs = [16 * sp["Np"] * 48 * sp["Mt"] * np.log2(sp["Mt"]) for sp in all_specs]
    owner, load = bie.shard_surfaces(costs, world)
    specs = [sp for sp, o in zip(all_specs, owner) if o == rank]
    ggq = wl.load_ggq()
    surfs = [bie.Surface(ctx, sp["surface"], sp["Np"], sp["Mt"], ggq) for sp in specs]
    ks = [sp["k"] for sp in specs]
    maxMt = max(sp["Mt"] for sp in specs)
    slot = 1 << 20
    W = torch.empty((1, slot, maxMt), dtype=torch.complex128, device="cuda")
    # the GGQ fill of every target panel into a bounded ring of near-band slots (throughput mode)
    band_slots = 4
    band = torch.empty((band_slots, 16 * maxMt, 3, 16 * maxMt), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    plan = bie.Batch(ctx, surfs, ks, bie.KERNEL_S, W, slot)
    plan.set_fill(band, band_slots)
    plan.run()
    torch.cuda.synchronize()
    plan_pairs, plan_config, plan_keep = plan.pairs, plan.config, plan
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):           # replay() launches on the current stream
        e0.record(stream)
        graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del graph, plan, plan_keep
    job_ms, job_rate = ms, plan_pairs / (ms / 1000.0)
    if world > 1:
        # the job ends with its slowest rank; the pairs are every rank's
        import torch.distributed as dist
        t = torch.tensor([ms, float(plan_pairs)], dtype=torch.float64, device="cuda")
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        tp = t[1:].clone()
        dist.all_reduce(tp, op=dist.ReduceOp.SUM)
        job_ms, job_rate = float(tm.item()), float(tp.item()) / (float(tm.item()) / 1000.0)
        return {"surfaces": count, "ranks": world, "scaling": "strong (the 64 surfaces split over the ranks)",
                "shard_load": [float(v) for v in load], "pairs_per_s": job_rate, "ms": job_ms,
                "cuda_graph": True}
    # the same surfaces, one single-surface plan each (made, warmed by its autotuner, timed, freed), one
    # after the other; the sum of their run times
    ms_seq = 0.0
    for sf, k in zip(surfs, ks):
        sp = bie.Batch(ctx, [sf], [k], bie.KERNEL_S, W, slot)
        sp.set_fill(band, band_slots)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sp.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_seq += e0.elapsed_time(e1)
        del sp
    # the per-surface right-hand sides (nrhs plane waves each, seeded directions), timed apart
    maxN = max(sf.N for sf in surfs)
    rbuf = torch.empty((16, maxN), dtype=torch.complex128, device="cuda")
    dirs = [wl.Stream(i, 9).directions(sp["nrhs"]) for i, sp in enumerate(specs)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for sf, k, dd in zip(surfs, ks, dirs):
            for j, d in enumerate(dd):
                bie.rhs(sf, 0, d, k, out=rbuf[j, :sf.N])
        e1.record(stream)
    torch.cuda.synchronize()
    rhs = {"vectors": int(sum(len(dd) for dd in dirs)), "ms": e0.elapsed_time(e1),
           "kind": "plane waves -e^{ik d.x}, nrhs per surface as listed"}
    del rbuf
    mts = [sp["Mt"] for sp in specs]
    del surfs
    return {"surfaces": count, "pairs": plan_pairs, "pairs_per_s": job_rate, "ms": job_ms, "rhs": rhs,
            "sequential_ms": ms_seq, "sequential_pairs_per_s": plan_pairs / (ms_seq / 1000.0),
            "speedup_vs_sequential": ms_seq / ms,
            "single_surface_star": star_single_surface_rate(bie, ctx, ggq, stream), "autotuned": plan_config,
            "m_theta_counts": {str(m): mts.count(m) for m in sorted(set(mts))},
            "panels_range": [min(sp["Np"] for sp in specs), max(sp["Np"] for sp in specs)],
            "rhs_per_surface": [sp["nrhs"] for sp in specs],
            "output": "Parseval weights in a ring of %d pairs x %d angles; every target panel folded by the "
                      "GGQ fill into a ring of %d near-band slots (throughput mode)" % (slot, maxMt, band_slots),
            "cuda_graph": True}


def star_single_surface_rate(bie, ctx, ggq, stream):
    """The batch family's per-pair cost on the single-surface path at the bench workload's sizes: one
    harmonic star (eps = 0.15), Np = 16, Mth = 128, k = 10, every near pair through one kernel-modes
    launch (S), timed with events after a warm-up; the ellipsoid of the headline takes the same
    launch."""
    import torch
    Np, Mt, k = 16, 128, 10.0
    s = bie.Surface(ctx, wl.harmonic_star(0, 7, 0.15), Np, Mt, ggq)
    N = s.N
    rows = torch.arange(N, device="cuda", dtype=torch.int64).repeat_interleave(48)
    srcs = torch.arange(48, device="cuda", dtype=torch.int32).repeat(N)
    panel = rows // (16 * Mt) + srcs.to(torch.int64) // 16 - 1
    keep = (panel >= 0) & (panel < Np)
    rows, srcs = rows[keep].contiguous(), srcs[keep].contiguous()
    out = torch.empty((rows.numel(), 1, Mt + 1), dtype=torch.complex128, device="cuda")
    with torch.cuda.stream(stream):
        bie.kernel_modes(s, bie.KERNEL_S, k, rows, srcs, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bie.kernel_modes(s, bie.KERNEL_S, k, rows, srcs, out=out)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = rows.numel()
    del out, rows, srcs, s
    return {"surface": "harmonic star (35 terms), Np 16, Mth 128, k 10", "pairs": n, "ms": ms,
            "pairs_per_s": n / (ms / 1000.0)}


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
    systems with the block-diagonal preconditioner (the one the network must beat, and its fallback)
    and with the network on top of it.  Operator: the single layer S (first kind, weighted density),
    plane-wave data."""
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
    # block products alone (5 right-hand sides, one pass over the matrix each), timed with events
    M = bie.Matrix(surf.ctx, A, bie.STORE_FP32 | bie.STORE_BF16X2)
    X = torch.as_tensor(wl.random_complex((5, N), 3, 7), dtype=torch.complex128).cuda()
    mv = {}
    for name, prec, bytes_per in (("fp64", 0, 16), ("fp32", 1, 8), ("bf16x2_tensor_cores", 2, 8),
                                  ("fp64_storage_double_word", 3, 16)):
        ms_ = timed(lambda: M.matvec(X, prec))
        mv[name] = {"ms": ms_, "matrix_bytes": bytes_per * N * N, "rhs": 5,
                    "read_GBps": bytes_per * N * N / (ms_ / 1000.0) / 1e9,
                    "frac_of_hbm": bytes_per * N * N / (ms_ / 1000.0) / 1e9 / hbm}
    mv["hbm_peak_GBps"] = hbm
    rows["block_product"] = mv
    del M, X
    if solve is not None:
        it = {}
        for name in ("fp64", "mixed_fp32", "mixed_bf16x2_tensor_cores"):
            rep = solve.get(name, {})
            if rep.get("iterations"):
                it[name] = {"ms_per_iteration": 1000.0 * rep["seconds"] / rep["iterations"], "rhs": solve["rhs"]}
        it["note"] = ("iteration time covers the block product, the Arnoldi steps of every right-hand side and, for "
                      "the mixed solves, their share of the FP64-accurate refinement residuals")
        rows["fgmres_iteration"] = it
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


def run_profile_case(name):
    """Profiling aid: one small launch of a kernel family, sized for an ncu capture (inputs above the
    126 MB L2, a few GB on the device at most).  Prints what ran."""
    import torch
    import paper_2608_16208_b300 as bie
    ggq = wl.load_ggq()
    ctx = bie.Context()
    c = wl.config(WORKLOAD)
    if name == "assemble":        # far fill and near fill of S on Np = 4, Mth = 128 (N = 8,192; 1.07 GB)
        s = bie.Surface(ctx, c["surface"], 4, c["Mt"], ggq)
        A = bie.assemble(s, bie.OP_S, c["k"])
        ctx.sync()
        print("assemble: N = %d" % s.N)
    elif name == "products":      # block products, 5 right-hand sides, N = 8,192 (FP64 1.07 GB)
        s = bie.Surface(ctx, c["surface"], 4, c["Mt"], ggq)
        A = bie.assemble(s, bie.OP_CFIE | bie.UNWEIGHTED, c["k"])
        M = bie.Matrix(ctx, A, bie.STORE_FP32 | bie.STORE_BF16X2)
        X = torch.as_tensor(wl.random_complex((5, s.N), 3, 7), dtype=torch.complex128).cuda()
        for prec in (0, 1, 2, 3):
            M.matvec(X, prec)
        ctx.sync()
        print("products: N = %d, 5 right-hand sides, precisions 0-3" % s.N)
    elif name == "field":         # field evaluation, 32,768 sources x 1,024 points
        s = bie.Surface(ctx, c["surface"], c["Np"], c["Mt"], ggq)
        dens = torch.as_tensor(wl.random_complex((s.N,), 0, 13), dtype=torch.complex128).cuda()
        bie.field_eval(s, bie.OP_S, c["k"], dens, wl.exterior_points(1024, 3.0))
        ctx.sync()
        print("field: %d sources x 1024 points" % s.N)
    elif name == "batch":         # the split batch path with the GGQ fill: four harmonic stars, Mth 64..256
        specs = wl.batch_surfaces(seed=0, count=4)
        surfs = [bie.Surface(ctx, sp["surface"], sp["Np"], sp["Mt"], ggq) for sp in specs]
        W = torch.empty((1, 1 << 20, max(sp["Mt"] for sp in specs)), dtype=torch.complex128, device="cuda")
        plan = bie.Batch(ctx, surfs, [sp["k"] for sp in specs], bie.KERNEL_S, W, 1 << 20)
        maxMt = max(sp["Mt"] for sp in specs)
        band = torch.empty((2, 16 * maxMt, 3, 16 * maxMt), dtype=torch.complex128, device="cuda")
        plan.set_fill(band, 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run()
        e1.record()
        ctx.sync()
        print("batch: %d pairs, config %s, %.1f ms" % (plan.pairs, plan.config, e0.elapsed_time(e1)))
    elif name == "banded":        # the O(M) route to the single layer on 18,944 pairs of the workload
        s = bie.Surface(ctx, c["surface"], c["Np"], c["Mt"], ggq)
        n = 18944
        rows = 16 * c["Mt"] * (c["Np"] // 2) + torch.arange(n, device="cuda", dtype=torch.int64) // 48
        srcs = torch.arange(n, device="cuda", dtype=torch.int32) % 48
        out = bie.kernel_modes_banded(s, c["k"], rows, srcs)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bie.kernel_modes_banded(s, c["k"], rows, srcs, out=out)
        e1.record()
        ctx.sync()
        print("banded: %d pairs, finite: %s, %.3f ms" % (n, bool(torch.isfinite(torch.view_as_real(out)).all()),
                                                       e0.elapsed_time(e1)))
    elif name == "precond":       # block-diagonal factors and one training step of the network, N = 24,576
        desc, k, d = learned_family(1, 0)
        s = bie.Surface(ctx, desc, 16, 96, ggq)
        A = bie.assemble(s, bie.OP_S, k)
        B = bie.BlockDiag(ctx, A, 16 * 96)
        ts = bie.TrainSet(ctx, s, k, A, B)
        net = bie.Net(ctx, seed=1)
        net.train([ts], steps=2, batch=16, lr=1e-3, seed=2)
        ctx.sync()
        print("precond: N = %d" % s.N)
    else:
        raise SystemExit("unknown profile case %r" % name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-solve", action="store_true")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-preconditioner training and held-out solves")
    ap.add_argument("--batch-surfaces", type=int, default=64, help="surfaces in the batch-scheduler run (0: skip)")
    ap.add_argument("--profile-case", default="",
                    help="profiling aid: one small launch of a kernel family (assemble, products, field, batch, "
                         "banded, precond) and exit")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="profiling aid: run the pair pipeline once on this many pairs of the workload and exit")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
    elif args.kernel_only:
        run_kernel_only(args.kernel_only)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
