"""Benchmark: F-cycle time to a 1e-10 relative residual on the anisotropic 4097^2 problem.

One step = one complete solve (mg_solve) of -eps u_xx - u_yy = f on a 4097 x 4097
grid (h = 1/4096, 16.8 M unknowns, 12 grids, f uniform[-1, 1] from seed 1, zero
start vector) to ||b - A x|| / ||b|| <= 1e-10.  The default form is the GB300
mixed-precision solve (FP32 F-cycles, FP64 defect / refinement / coarsest solve);
--precision fp64 runs every step in FP64.

Prints one JSON line (rank 0).  Metric: milliseconds per solve (lower is better).
``--impl reference`` times the FP64 CPU oracle on the host instead (a bounded
sample: one oracle F-cycle per step, scaled by the cycle count to tolerance).
Under torchrun each rank solves its own instance (replicas, weak scaling).
"""
from __future__ import annotations

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

METRIC = "F-cycle time-to-1e-10-residual & smoother/defect HBM GB/s vs 8 TB/s peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4097)
    ap.add_argument("--eps", type=float, default=1.0)
    ap.add_argument("--smoother", default="rbgs")
    ap.add_argument("--omega", type=float, default=None)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nu", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="aniso",
                    choices=["aniso", "batched", "small", "annulus", "cylinder", "diff", "steps"],
                    help="aniso: the 4097^2 anisotropic solve (default); batched: 256 uneven instances in one "
                         "launch; small: 129^2 Poisson, Jacobi, FP64; annulus: 2049x2048 polar map; cylinder: "
                         "257x256x257 cylindrical map; diff: 1025^2 -div(k grad u) loss and gradient; steps: the "
                         "finest-level kernels of the aniso solve one step at a time (per-kernel timing, and a "
                         "short fixed launch sequence for profilers)")
    ap.add_argument("--count", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--levels", type=int, default=0,
                    help="grids of the hierarchy (0: as many as the grid allows); coarsest grids above 4096 "
                         "unknowns are solved by conjugate gradients")
    ap.add_argument("--flags", type=int, default=0,
                    help="extra MG_FLAG_* bits for the solver (1 = kernel-by-kernel launches, for profilers)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 FMA throughput of this GB300 pool, measured with an FMA-chain kernel
# (1.19-1.20 TFLOP/s = 0.6 T FMA instructions/s over 152 SMs at ~1.95 GHz).
FP64_TFLOPS_MEASURED = 1.197

# DRAM bytes (read + write) per launch of the finest-level red-black sweep of the 4097^2
# mixed solve, from one ncu capture of k_rb2d_tma: the mean of the cycle's four launches.  The
# record names the SHA-256 of the kernel's source file at the time of the capture; when the
# file has changed since, the counters no longer describe the kernel and traffic is reported
# as null.
FINEST_SWEEP_TRAFFIC = {"source": "paper_0805_3041_gb300/csrc/kernels_tma.cu",
                        "sha256": "2fdb2ea6bf718c3e68d5fd34865b1d796ef638a43e16641caf66cff68263f44a",
                        "bytes": 167.0e6,
                        "capture": "profiles/fcycle_mixed_rbgs_aniso4097.md"}


def finest_sweep_traffic():
    """The recorded DRAM traffic per launch, or None when the kernel's source has changed."""
    import hashlib
    rec = FINEST_SWEEP_TRAFFIC
    try:
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return rec["bytes"] if digest == rec["sha256"] else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def default_omega(smoother, omega=None):
    """The damping used unless --omega is given: 0.8 for point Jacobi, 0.7 for line Jacobi
    (and ADI), 1 for the Gauss-Seidel smoothers."""
    if omega is not None:
        return omega
    return 0.8 if smoother == "jacobi" else 0.7 if smoother.startswith("line") or smoother == "adi" else 1.0


def make_problem(args):
    from paper_0805_3041_gb300 import inputs
    sp = inputs.anisotropic(n=args.n, eps=args.eps, seed_f=1)
    levels = args.levels or inputs.max_levels(sp.n)
    return sp, levels, default_omega(args.smoother, args.omega)


def workload_config(args, levels, omega):
    return {"workload": f"anisotropic Poisson -eps u_xx - u_yy = f, {args.n}x{args.n} grid, eps={args.eps:g}, "
                        f"F-cycle over {levels} grids, {args.smoother} omega={omega:g} nu1=nu2={args.nu}, "
                        f"{args.precision}, f~U[-1,1] seed 1, x0=0, tol {args.tol:g}",
            "n": args.n, "eps": args.eps, "levels": levels, "smoother": args.smoother, "nu1": args.nu,
            "nu2": args.nu, "precision": args.precision, "tol": args.tol,
            "l2": "inputs larger than L2 (134 MB per FP64 field > 129 MB) and L2 flushed between steps"}


# --------------------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline key and the --impl reference arm)
# --------------------------------------------------------------------------------------
def oracle_cycles_to_tol(args, levels, omega):
    """Cycle count of the oracle to the tolerance on a 513^2 grid with the same eps,
    smoother and cycle (the F-cycle rate is mesh independent)."""
    from oracle import oracle as orc
    from paper_0805_3041_gb300 import inputs
    n = 513
    sp = inputs.anisotropic(n=n, eps=args.eps, seed_f=1)
    o = orc.Oracle(orc.Problem(dim=2, n=sp.n, kind=orc.CONST, h=sp.h, c=sp.c), levels=levels - 3,
                   smoother=args.smoother, omega=omega, nu1=args.nu, nu2=args.nu)
    x, st, cyc, rr, hist = o.solve(sp.b, tol=args.tol, maxit=200)
    return cyc


def host_cpu():
    """The host's CPU model (lscpu) and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count(), "arch": os.uname().machine}


def oracle_threads():
    """Threads of the oracle's threaded build (all host cores unless OMP_NUM_THREADS says
    otherwise); None when that build is not available."""
    from oracle import oracle as orc
    try:
        return orc.threads(True)
    except Exception:
        return None


def oracle_cycle_time(args, levels, omega, sp=None, reps=1, threaded=False):
    """Seconds for one oracle F-cycle plus its residual check on the full grid."""
    from oracle import oracle as orc
    if sp is None:
        sp, _, _ = make_problem(args)
    o = orc.Oracle(orc.Problem(dim=2, n=sp.n, kind=orc.CONST, h=sp.h, c=sp.c), levels=levels,
                   smoother=args.smoother, omega=omega, nu1=args.nu, nu2=args.nu, threaded=threaded)
    x = np.zeros_like(sp.b)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        x = o.cycle(x, sp.b)
        o.norm(o.defect(x, sp.b))
        ts.append(time.perf_counter() - t0)
    return ts


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sp, levels, omega = make_problem(args)
    cyc = oracle_cycles_to_tol(args, levels, omega)
    nthr = oracle_threads()
    threaded = nthr is not None
    # one oracle F-cycle per step on all host cores; the whole run is kept to about four
    # minutes of oracle time
    first = oracle_cycle_time(args, levels, omega, sp, reps=1, threaded=threaded)[0]
    budget = max(1, int(240.0 / max(first, 1e-3)) - 1)
    warm = min(args.warmup - 1, budget // 4) if args.warmup > 1 else 0
    timed = max(1, min(args.steps, budget - warm))
    ts = oracle_cycle_time(args, levels, omega, sp, reps=warm + timed, threaded=threaded)[warm:]
    per_cycle = float(np.mean(ts))
    value = per_cycle * cyc * 1e3
    cores = nthr if threaded else 1
    sample = (f"one oracle F-cycle + residual check on the full {args.n}^2 grid per step ({timed} timed) on "
              f"{cores} host threads, x{cyc} cycles (the oracle's cycle count to {args.tol:g} on 513^2, same "
              f"eps/smoother)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, levels, omega),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------
def max_over_ranks(value, device):
    """The largest per-rank time over the process group (every rank gets it): replicas finish
    together only when the slowest one does."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_0805_3041_gb300.binding import Solver, FLAG_TIMING

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sp, levels, omega = make_problem(args)
    b = torch.from_numpy(sp.b).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    # the measured solver runs the whole solve as one device-side graph loop; a second context
    # with CUDA events around every finest-level smoothing launch times the dominant kernel
    s = Solver(sp, levels=levels, smoother=args.smoother, omega=omega, nu1=args.nu, nu2=args.nu,
               precision=args.precision, max_cycles=100, flags=args.flags, device=dev)
    st = Solver(sp, levels=levels, smoother=args.smoother, omega=omega, nu1=args.nu, nu2=args.nu,
                precision=args.precision, max_cycles=100, flags=FLAG_TIMING | args.flags, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    infos = []
    for _ in range(args.warmup):
        x.zero_()
        s.solve_into(b, x, tol=args.tol)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = s.launch_count()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1)          # evict the previous solve from L2
        x.zero_()               # start vector
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = s.solve_into(b, x, tol=args.tol)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
        infos.append(info)
    barrier()
    launches = s.launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(total_ms / args.steps, dev) if world > 1 else total_ms / args.steps
    # dominant kernel: the finest-level smoothing sweeps, timed with CUDA events recorded on the
    # solver's stream around each launch, over the same number of solves
    for _ in range(max(1, args.warmup)):
        x.zero_()
        st.solve_into(b, x, tol=args.tol)
    st.kernel_timing()
    for _ in range(args.steps):
        flush.fill_(1)
        x.zero_()
        torch.cuda.synchronize(dev)
        st.solve_into(b, x, tol=args.tol)
    torch.cuda.synchronize(dev)
    kern_ms, kern_n, kern_bytes = st.kernel_timing()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    bh = torch.from_numpy(sp.b).pin_memory().numpy()
    xh = torch.zeros(sp.shape, dtype=torch.float64).pin_memory().numpy()
    e2e = []
    for r in range(max(2, args.steps // 2)):
        xh[...] = 0.0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.solve_host(bh, xh, tol=args.tol)
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = float(np.median(e2e))
    nbytes = sp.b.nbytes

    peaks, src = measured_peaks()
    if args.precision == "fp64":
        # FP64 smoothing is bound by GB300's FP64 pipe: report against the measured FMA rate
        unk = (args.n - 2) ** 2
        flops = 2.0 * 6 * unk   # 6 FMA per unknown and sweep (5-point residual + update)
        achieved = flops / (kern_ms * 1e-3) / 1e12 if kern_ms else None
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_TFLOPS_MEASURED, "unit": "TFLOP/s",
                "frac": achieved / FP64_TFLOPS_MEASURED if achieved else None, "traffic": None,
                "kernel": "finest-level smoothing sweep (FP64)", "peak_source": "measured FP64 FMA rate"}
    else:
        achieved = kern_bytes / (kern_ms * 1e-3) / 1e9 if kern_ms else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"] if achieved else None,
                "traffic": finest_sweep_traffic() if args.n == 4097 and args.smoother == "rbgs" else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, mean of the four "
                                  "finest-level sweeps of one refinement step (zero start, plain, correction "
                                  "folded in, plain)",
                "kernel": "finest-level smoothing sweep (FP32)", "peak_source": src,
                "launch_ms": kern_ms, "launches": kern_n, "bytes_per_launch": kern_bytes}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cyc = infos[-1]["cycles"]
        one = float(oracle_cycle_time(args, levels, omega, sp, reps=1)[0])
        nthr = oracle_threads()
        if nthr is not None:
            per = float(np.min(oracle_cycle_time(args, levels, omega, sp, reps=2, threaded=True)))
            cores = nthr
        else:
            per, cores = one, 1
        cpu = {"value": per * cyc * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": f"2 oracle F-cycles (+ residual check) on the full {args.n}^2 grid on {cores} host "
                         f"threads (rows and lines spread by OpenMP, results identical to the plain build); "
                         f"fastest x {cyc} cycles (the GPU's count to tolerance)",
               "single_thread_value": one * cyc * 1e3,
               "single_thread_sample": f"1 oracle F-cycle (+ residual check), plain build, one thread, x {cyc}",
               "host": host_cpu()}

    if rank == 0:
        last = infos[-1]
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(args, levels, omega),
                "cycles": last["cycles"], "relres": last["relres"], "rate": last["rate"],
                "solves_per_s": 1e3 / ms * world,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes},
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------------------
# batched workload: 256 independent instances of uneven size and anisotropy, one graph
# --------------------------------------------------------------------------------------
def run_batched(args):
    import torch
    from paper_0805_3041_gb300 import inputs
    from paper_0805_3041_gb300.autotune import Autotuner
    from paper_0805_3041_gb300.binding import Solver, Batch, BATCH_GRAPH

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    specs = inputs.batched(count=args.count, seed=4)
    tuner = Autotuner(path=os.path.join(ROOT, "paper_0805_3041_gb300", "tuned_gb300.json"))
    t0 = time.perf_counter()
    cfgs = [tuner.choose(sp) for sp in specs]
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    solvers = [Solver(sp, levels=inputs.max_levels(sp.n), precision="mixed", max_cycles=100, device=dev, **cfg)
               for sp, cfg in zip(specs, cfgs)]
    bs = [torch.from_numpy(sp.b).to(dev) for sp in specs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = Batch(solvers, bs, xs)   # small instances in the persistent kernel, the rest as a graph
    persistent, ctas, teams = batch.info()
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms)), out

    def batch_solve():
        for x in xs:
            x.zero_()
        return batch.solve(tol=args.tol)

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    launches0 = sum(s.launch_count() for s in solvers)
    ms, infos = timed(batch_solve, args.steps, args.warmup)
    launches = (sum(s.launch_count() for s in solvers) - launches0) // max(1, args.steps + args.warmup) * args.steps
    clk = clocks.stop()
    assert all(i["status"] == "MG_OK" for i in infos), [i["status"] for i in infos]

    def sequential(solver_list):
        out = []
        for s, b, x in zip(solver_list, bs, xs):
            x.zero_()
            out.append(s.solve_into(b, x, tol=args.tol))
        return out

    # the same batch as one CUDA graph with a branch per instance, for comparison
    gbatch = Batch(solvers, bs, xs, mode=BATCH_GRAPH)

    def graph_solve():
        for x in xs:
            x.zero_()
        return gbatch.solve(tol=args.tol)

    graph_ms, ginfos = timed(graph_solve, max(2, args.steps // 2), 1)
    gbatch.close()
    seq_ms, seq = timed(lambda: sequential(solvers), max(1, args.steps // 4), 1)
    fp64 = [Solver(sp, levels=inputs.max_levels(sp.n), precision="fp64", max_cycles=100, device=dev, **cfg)
            for sp, cfg in zip(specs, cfgs)]
    f64_ms, f64 = timed(lambda: sequential(fp64), max(1, args.steps // 4), 1)

    # end to end: host copies of every b and x around the batch solve
    bh = [torch.from_numpy(sp.b).pin_memory() for sp in specs]
    xh = [torch.zeros(sp.shape, dtype=torch.float64).pin_memory() for sp in specs]
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for b, h in zip(bs, bh):
            b.copy_(h, non_blocking=True)
        infos_e = batch_solve()
        for x, h in zip(xs, xh):
            h.copy_(x, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e.append((time.perf_counter() - t1) * 1e3)
    nbytes = sum(sp.b.nbytes for sp in specs)
    nodes = sum(sp.b.size for sp in specs)
    classes = {}
    for cfg in cfgs:
        k = f"{cfg['smoother']}/nu{cfg['nu1']}"
        classes[k] = classes.get(k, 0) + 1
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{args.count} independent 2-D anisotropic Poisson instances, N uniform over "
                                   f"{{65,129,257,513,1025}}, eps log-uniform [1e-3,1], f~U[-1,1] seed 4, x0=0, "
                                   f"mixed precision to {args.tol:g}, "
                                   + (f"{persistent} instances up to 257^2 in one persistent cooperative launch "
                                      f"({ctas} CTAs, {teams} teams), the other {args.count - persistent} in one "
                                      f"CUDA graph launch" if persistent else "one CUDA graph launch per batch")
                                   + ", autotuned schedule per class",
                       "instances": args.count, "nodes": int(nodes), "schedules": classes,
                       "l2": "L2 flushed between steps"},
            "cycles_max": max(i["cycles"] for i in infos), "relres_max": max(i["relres"] for i in infos),
            "form": ("persistent + graph" if persistent < args.count else "persistent") if persistent else "graph",
            "graph_form_ms": graph_ms,
            "sequential_mixed_ms": seq_ms, "sequential_fp64_ms": f64_ms,
            "fp64_relres_max": max(i["relres"] for i in f64),
            "setup_s": setup_s, "tune_s": tune_s, "roofline": None,
            "e2e": {"value": float(np.median(e2e)), "unit": "ms", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)
    batch.close()


# --------------------------------------------------------------------------------------
# the other study configurations: one step = one solve (diff: one loss + gradient)
# --------------------------------------------------------------------------------------
def config_problem(args):
    """(spec, levels, smoother, omega, description) of a study configuration."""
    from paper_0805_3041_gb300 import inputs
    if args.workload == "small":
        sp = inputs.poisson_sin(129)
        return sp, 6, "jacobi", 0.8, "2-D Poisson 129x129, f = 2 pi^2 sin sin, x0 = 0, 6 grids, damped Jacobi 0.8"
    if args.workload == "annulus":
        sp = inputs.annulus_2d()
        sm = args.smoother
        return (sp, inputs.max_levels(sp.n, periodic_y=True), sm, default_omega(sm, args.omega),
                "annulus r in [0.1, 1] x theta periodic mapped to 2049x2048 (separable weights), blob + noise "
                "seed 3, x0 = 0")
    if args.workload == "cylinder":
        sp = inputs.cylinder_3d()
        sm = args.smoother
        return (sp, inputs.max_levels(sp.n, periodic_y=True, dim=3), sm, default_omega(sm, args.omega),
                "cylinder shell (r, theta, z) mapped to 257x256x257 (separable weights), blob + noise seed 3, x0 = 0")
    sp = inputs.diffusion_cells(1025)
    return (sp, inputs.max_levels(sp.n), args.smoother, default_omega(args.smoother, args.omega),
            "-div(k grad u) = f on 1025x1025, k log-normal (correlation 16 cells, seed 5), blob source; "
            "step = forward solve + adjoint solve + gradient kernel (loss ||u - u_obs||^2)")


def run_config(args):
    import torch
    from oracle import oracle as orc
    from paper_0805_3041_gb300 import inputs
    from paper_0805_3041_gb300.binding import Solver

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    sp, levels, smoother, omega, desc = config_problem(args)
    if args.levels:
        levels = args.levels
    prec = "fp64" if args.workload == "small" else args.precision
    t0 = time.perf_counter()
    s = Solver(sp, levels=levels, smoother=smoother, omega=omega, nu1=args.nu, nu2=args.nu, precision=prec,
               max_cycles=200, flags=args.flags, device=dev)
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    b = torch.from_numpy(sp.b).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    diff = args.workload == "diff"
    if diff:   # u_obs: the solution for a reference field plus 1 % noise
        ref = Solver(inputs.ProblemSpec(name="ref", dim=2, n=sp.n, periodic_y=False, kind=inputs.CELL, h=sp.h,
                                        k=inputs.lognormal_cells(sp.n[0] - 1, seed=6)),
                     levels=levels, precision="fp64", max_cycles=200, device=dev)
        uref, _ = ref.solve(sp.b, tol=args.tol)
        noise = torch.from_numpy(inputs.observation_noise(sp.shape)).to(dev)
        uobs = uref + 0.01 * float(uref.pow(2).mean().sqrt()) * noise

    def step():
        x.zero_()
        info = s.solve_into(b, x, tol=args.tol)
        if diff:
            lam, ia = s.solve_adjoint(2.0 * (x - uobs), tol=args.tol)
            s.grad_coeff(x, lam)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    l0 = s.launch_count()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    launches = s.launch_count() - l0
    clk = clocks.stop()
    value = float(np.median(ms))
    # end to end: host buffers through mg_solve_host (copies inside the timed region)
    bh = torch.from_numpy(sp.b).pin_memory().numpy()
    xh = torch.zeros(sp.shape, dtype=torch.float64).pin_memory().numpy()
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        xh[...] = 0.0
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        s.solve_host(bh, xh, tol=args.tol)
        e2e.append((time.perf_counter() - t1) * 1e3)
    cpu = None
    if not args.no_cpu_baseline:   # one oracle F-cycle (+ residual) on the full grid, x the GPU's cycle count
        p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c, sx=sp.sx,
                        sy=sp.sy, sz=sp.sz, k=sp.k)
        nthr = oracle_threads()
        o = orc.Oracle(p, levels=levels, smoother=smoother, omega=omega, nu1=args.nu, nu2=args.nu, dense_max=4096,
                       threaded=nthr is not None)
        t1 = time.perf_counter()
        xo = o.cycle(np.zeros_like(sp.b), sp.b)
        o.norm(o.defect(xo, sp.b))
        per = time.perf_counter() - t1
        mult = 2 if diff else 1   # the adjoint solve costs what the forward does
        cores = nthr or 1
        cpu = {"value": per * info["cycles"] * mult * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": f"1 oracle F-cycle (+ residual check) on the full grid on {cores} host threads, x "
                         f"{info['cycles']} cycles" + (" x 2 (forward + adjoint)" if diff else ""),
               "host": host_cpu()}
    line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": desc + f", {smoother} omega={omega:g} nu1=nu2={args.nu}, {prec}, tol {args.tol:g}",
                       "levels": levels, "smoother": smoother, "precision": prec,
                       "l2": "L2 flushed between steps"},
            "cycles": info["cycles"], "relres": info["relres"], "rate": info["rate"], "setup_s": setup_s,
            "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": float(np.median(e2e)), "unit": "ms", "h2d_bytes_per_step": 2 * sp.b.nbytes,
                    "d2h_bytes_per_step": sp.b.nbytes},
            "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# the finest-level kernels of the solve, one step at a time
# --------------------------------------------------------------------------------------
def run_steps(args):
    """Each timed iteration runs, on the finest grid of the mixed context: one sweep (mode 0),
    the descending half of a visit from zero (mode 1, mode 0, defect + restriction), the ascending
    half (mode 2, mode 0) and the refinement loop's outer defect -- the single-step entry points,
    which also pack and unpack their FP64 arguments.  The step groups are timed with CUDA events;
    under a profiler each iteration is the same fixed sequence of kernels."""
    import torch
    from paper_0805_3041_gb300.binding import Solver
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    sp, levels, omega = make_problem(args)
    s = Solver(sp, levels=levels, smoother="rbgs", omega=omega, nu1=2, nu2=2, precision="mixed", max_cycles=4,
               flags=args.flags, device=dev)
    rng = np.random.default_rng(0)
    u = torch.tensor(rng.standard_normal(sp.shape) * 1e-3, device=dev)
    g = torch.tensor(sp.b, device=dev)
    ec = torch.tensor(rng.standard_normal(s.level_shape(levels - 1)) * 1e-3, device=dev)
    stream = torch.cuda.current_stream(dev)
    groups = {"sweep": lambda: s.smooth(u, g, 1, 0), "descend": lambda: s.descend(None, g),
              "ascend": lambda: s.ascend(ec, u, g), "outer_defect": lambda: s.outer_defect(u, g)}
    ms = {k: [] for k in groups}
    for it in range(args.warmup + args.steps):
        for k, fn in groups.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it >= args.warmup:
                ms[k].append(e0.elapsed_time(e1))
    line = {"workload": "steps", "n": args.n, "levels": levels, "steps": args.steps, "warmup": args.warmup,
            "ms_median": {k: float(np.median(v)) for k, v in ms.items()},
            "note": "each group includes the pack / unpack kernels of its FP64 arguments"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload in ("small", "annulus", "cylinder", "diff"):
        run_config(args)
    elif args.workload == "steps":
        run_steps(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
