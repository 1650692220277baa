"""Autotuner for the solver's schedule and kernel knobs.

For a problem class -- grid size and anisotropy -- it times candidate configurations on
the device and keeps the fastest one that reaches the tolerance:

1. the smoothing schedule: point red-black Gauss-Seidel, zebra y-line Gauss-Seidel, damped
   y-line Jacobi, or the alternating-direction GSADI / ADI, with nu1 = nu2 = 1 or 2 (for
   -eps u_xx - u_yy the point smoother slows down as eps falls, the y-line smoothers do
   not: Wallis 2008, section "Anisotropies");
2. then, for the chosen schedule, the kernel knobs that do not change the results: the
   single-CTA coarse-cycle cut-off (coarse_cut_nodes), the size below which the tile sweep
   replaces the row-streaming one (tile_nodes) and the rows per CTA of the streaming
   sweep (sweep_rows).

Results are cached per class in a JSON table (``Autotuner.save`` / ``load``).  The class
of a problem is (n0, n1, eps bucket) with eps = c_x / c_y of a constant-coefficient
operator rounded to half a decade.  The timing function is injectable, so the selection
logic is testable without a device.
"""
from __future__ import annotations

import json
import math
import os
import time

SCHEDULES = [
    dict(smoother="rbgs", omega=1.0, nu1=2, nu2=2),
    dict(smoother="rbgs", omega=1.0, nu1=1, nu2=1),
    dict(smoother="zebra_y", omega=1.0, nu1=1, nu2=1),
    dict(smoother="zebra_y", omega=1.0, nu1=2, nu2=2),
    dict(smoother="line_y", omega=0.7, nu1=2, nu2=2),
    dict(smoother="gsadi", omega=1.0, nu1=1, nu2=1),
    dict(smoother="adi", omega=0.8, nu1=2, nu2=2),
]
KNOBS = [
    dict(),
    dict(coarse_cut_nodes=5000),
    dict(tile_nodes=-1),
    dict(tile_nodes=1 << 30),
    dict(sweep_rows=16),
    dict(sweep_rows=64),
]
DEFAULT = dict(SCHEDULES[0])


def eps_of(spec):
    """Anisotropy c_x / c_y of a constant-coefficient problem (1 for other kinds)."""
    c = getattr(spec, "c", None)
    if c is None or not c[1]:
        return 1.0
    return float(c[0]) / float(c[1])


def class_key(spec):
    e = eps_of(spec)
    bucket = round(2.0 * math.log10(e)) / 2.0 if e > 0 else 0.0
    return f"{spec.n[0]}x{spec.n[1]}:eps1e{bucket:+.1f}"


def gpu_measure(spec, cfg, tol=1e-10, precision="mixed", reps=3, max_cycles=100):
    """Median seconds of `reps` solves of `spec` with configuration `cfg` (after one
    untimed solve); inf when the solve does not reach `tol`."""
    import torch
    from . import inputs
    from .binding import Solver
    s = Solver(spec, levels=inputs.max_levels(spec.n), precision=precision, max_cycles=max_cycles, **cfg)
    b = torch.from_numpy(spec.b).cuda()
    x = torch.zeros_like(b)
    info = s.solve_into(b, x, tol=tol)
    if info["status"] != "MG_OK":
        return math.inf
    ts = []
    for _ in range(reps):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = s.solve_into(b, x, tol=tol)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        if info["status"] != "MG_OK":
            return math.inf
    ts.sort()
    return ts[len(ts) // 2]


class Autotuner:
    """Per-class choice of schedule and knobs.  `measure(spec, cfg) -> seconds` (inf for a
    configuration that does not converge); the default times real solves on the GPU."""

    def __init__(self, path=None, measure=None, tol=1e-10, precision="mixed"):
        self.path = path
        self.measure = measure or (lambda spec, cfg: gpu_measure(spec, cfg, tol=tol, precision=precision))
        self.table = {}
        if path and os.path.exists(path):
            self.load(path)

    def load(self, path):
        with open(path) as f:
            data = json.load(f)
        self.table.update(data.get("classes", {}))

    def save(self, path=None):
        path = path or self.path
        with open(path, "w") as f:
            json.dump({"classes": self.table}, f, indent=1, sort_keys=True)

    def tune(self, spec):
        """Time the candidates for spec's class and record the winner."""
        trials = []
        best_s, best_t = None, math.inf
        for sc in SCHEDULES:
            t = self.measure(spec, dict(sc))
            trials.append((dict(sc), t))
            if t < best_t:
                best_s, best_t = dict(sc), t
        if best_s is None:   # nothing converged: keep the default schedule
            best_s = dict(DEFAULT)
        best_k, best_kt = {}, best_t
        for kn in KNOBS[1:]:
            t = self.measure(spec, {**best_s, **kn})
            trials.append(({**best_s, **kn}, t))
            if t < best_kt:
                best_k, best_kt = dict(kn), t
        cfg = {**best_s, **best_k}
        self.table[class_key(spec)] = {"config": cfg, "seconds": None if math.isinf(best_kt) else best_kt}
        return cfg, trials

    def choose(self, spec):
        """The configuration for spec's class: from the table, else tuned now."""
        k = class_key(spec)
        if k not in self.table:
            self.tune(spec)
        return dict(self.table[k]["config"])


def tune_batched_set(path, count=256, seed=4):
    """Tune every class of the batched workload (inputs.batched) and write the table."""
    from . import inputs
    tuner = Autotuner(path=path)
    seen = set()
    for sp in inputs.batched(count=count, seed=seed):
        k = class_key(sp)
        if k in seen or k in tuner.table:
            continue
        seen.add(k)
        cfg, _ = tuner.tune(sp)
        print(f"{k}: {cfg} {tuner.table[k]['seconds']}", flush=True)
    tuner.save(path)
    return tuner


if __name__ == "__main__":
    import sys
    tune_batched_set(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "tuned_gb300.json"))
