"""Thin Python binding of the C ABI in include/mg.h (argument marshalling only).

PyTorch provides device memory and the CUDA stream; every step of the solve
runs in the library's CUDA kernels.  There is no CPU path: if the shared
library cannot be loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

JACOBI, RBGS, LINE_X, LINE_Y, ZEBRA_X, ZEBRA_Y, ADI, GSADI = range(8)
SMOOTHERS = {"jacobi": JACOBI, "rbgs": RBGS, "line_x": LINE_X, "line_y": LINE_Y,
             "zebra_x": ZEBRA_X, "zebra_y": ZEBRA_Y, "adi": ADI, "gsadi": GSADI}
CONST, SEPARABLE, CELL, EDGE = 0, 1, 2, 3
FP64, MIXED = 0, 1
FLAG_NO_GRAPH, FLAG_TIMING, FLAG_NO_FUSED_COARSE, FLAG_NO_FUSED_SWEEP, FLAG_NO_TMA = 1, 2, 4, 8, 16
FLAG_FMG_START = 32
FLAG_ADAPTIVE_CORR = 64
FLAG_TEST_WAIT_TIMEOUT = 128
FLAG_GALERKIN = 256
FLAG_FP64_DEFECT = 512
FLAG_NO_PDL = 1024
FLAG_TEST_BOUNDS = 2048
FLAG_TRACE = 4096
STATUS = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV", 5: "MG_EDIVERGED",
          6: "MG_ETIMEOUT", 7: "MG_EBOUNDS"}
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EDIVERGED, ETIMEOUT, EBOUNDS = 0, 1, 2, 3, 4, 5, 6, 7

EXPORTS = ["mg_workspace_bytes", "mg_setup", "mg_solve", "mg_solve_host", "mg_solve_adjoint", "mg_grad_coeff", "mg_apply",
           "mg_residual_norm", "mg_residual_norm_noalloc", "mg_level_dims", "mg_step_smooth", "mg_step_defect", "mg_step_restrict", "mg_step_prolong",
           "mg_step_coarse", "mg_step_cycle", "mg_step_descend", "mg_step_ascend", "mg_step_outer_defect", "mg_kernel_timing", "mg_launch_count", "mg_destroy",
           "mg_status_str", "mg_last_error", "mg_batch_create", "mg_batch_create_ex", "mg_batch_info",
           "mg_batch_solve", "mg_batch_destroy", "mg_solve_batched", "mg_debug_build", "mg_trace_report"]
BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2


class Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("periodic_y", C.c_int), ("levels", C.c_int),
                ("smoother", C.c_int), ("omega", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
                ("omega_corr", C.c_double), ("precision", C.c_int), ("max_cycles", C.c_int),
                ("inner_cycles", C.c_int), ("stream", C.c_void_p), ("flags", C.c_uint),
                ("coarse_cut_nodes", C.c_int), ("sweep_rows", C.c_int), ("tile_nodes", C.c_int)]


class Coeffs(C.Structure):
    _fields_ = [("kind", C.c_int), ("h", C.c_double * 3), ("c", C.c_double * 3),
                ("sx", C.c_void_p), ("sy", C.c_void_p), ("sz", C.c_void_p), ("k", C.c_void_p),
                ("ex", C.c_void_p), ("ey", C.c_void_p), ("ez", C.c_void_p)]


class Report(C.Structure):
    _fields_ = [("cycles", C.c_int), ("relres", C.c_double), ("rate", C.c_double), ("status", C.c_int),
                ("history", C.c_void_p), ("history_cap", C.c_int), ("seconds", C.c_double)]


_libs = {}


def library_path(debug: bool = False) -> str:
    return _build.LIB_DEBUG if debug else _build.LIB


def load(build_if_missing: bool = True, debug: bool = False):
    """Load (building if needed) the shared library and declare its signatures.  debug=True: the
    checking build (device-side bounds checks, MG_EBOUNDS), a separate library file."""
    if debug in _libs:
        return _libs[debug]
    path = library_path(debug)
    if build_if_missing and not _build.up_to_date(debug):
        path = _build.build(debug=debug)
    if not os.path.exists(path):
        raise RuntimeError(f"solver library missing: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    L.mg_workspace_bytes.argtypes = [C.POINTER(Params), C.POINTER(Coeffs)]
    L.mg_workspace_bytes.restype = C.c_size_t
    L.mg_setup.argtypes = [C.POINTER(Params), C.POINTER(Coeffs), P, C.c_size_t, C.POINTER(P)]
    L.mg_setup.restype = I
    L.mg_solve.argtypes = [P, P, P, D, C.POINTER(Report)]
    L.mg_solve.restype = I
    L.mg_solve_host.argtypes = [P, P, P, D, C.POINTER(Report)]
    L.mg_solve_host.restype = I
    L.mg_solve_adjoint.argtypes = [P, P, P, D, C.POINTER(Report)]
    L.mg_solve_adjoint.restype = I
    L.mg_grad_coeff.argtypes = [P, P, P, P]
    L.mg_grad_coeff.restype = I
    L.mg_apply.argtypes = [P, I, P, P]
    L.mg_apply.restype = I
    L.mg_residual_norm.argtypes = [P, I, P, P, P]
    L.mg_residual_norm.restype = I
    L.mg_residual_norm_noalloc.argtypes = [C.POINTER(Params), C.POINTER(Coeffs), P, P, P]
    L.mg_residual_norm_noalloc.restype = I
    L.mg_level_dims.argtypes = [P, I, C.POINTER(C.c_int)]
    L.mg_level_dims.restype = I
    L.mg_step_smooth.argtypes = [P, I, P, P, P, I, I]
    L.mg_step_smooth.restype = I
    L.mg_step_defect.argtypes = [P, I, P, P, P]
    L.mg_step_defect.restype = I
    L.mg_step_restrict.argtypes = [P, I, P, P]
    L.mg_step_restrict.restype = I
    L.mg_step_prolong.argtypes = [P, I, P, P, P, D]
    L.mg_step_prolong.restype = I
    L.mg_step_coarse.argtypes = [P, P, P]
    L.mg_step_coarse.restype = I
    L.mg_step_cycle.argtypes = [P, P, P, P, I]
    L.mg_step_cycle.restype = I
    L.mg_step_descend.argtypes = [P, I, P, P, P, P, I]
    L.mg_step_descend.restype = I
    L.mg_step_ascend.argtypes = [P, I, P, P, P, P, I]
    L.mg_step_ascend.restype = I
    L.mg_step_outer_defect.argtypes = [P, P, P, P, C.POINTER(D)]
    L.mg_step_outer_defect.restype = I
    L.mg_kernel_timing.argtypes = [P, C.POINTER(D), C.POINTER(I), C.POINTER(D)]
    L.mg_kernel_timing.restype = I
    L.mg_launch_count.argtypes = [P]
    L.mg_launch_count.restype = C.c_longlong
    L.mg_destroy.argtypes = [P]
    L.mg_status_str.argtypes = [I]
    L.mg_status_str.restype = C.c_char_p
    L.mg_last_error.argtypes = [P]
    L.mg_last_error.restype = C.c_char_p
    L.mg_batch_create.argtypes = [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), C.POINTER(P)]
    L.mg_batch_create.restype = I
    L.mg_batch_create_ex.argtypes = [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), I, C.POINTER(P)]
    L.mg_batch_create_ex.restype = I
    L.mg_batch_info.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I)]
    L.mg_batch_info.restype = I
    L.mg_batch_solve.argtypes = [P, D, C.POINTER(Report)]
    L.mg_batch_solve.restype = I
    L.mg_batch_destroy.argtypes = [P]
    L.mg_solve_batched.argtypes = [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), D, C.POINTER(Report)]
    L.mg_solve_batched.restype = I
    L.mg_debug_build.argtypes = []
    L.mg_debug_build.restype = I
    L.mg_trace_report.argtypes = [P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
    L.mg_trace_report.restype = I
    _libs[debug] = L
    return L


class MGError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _torch():
    import torch
    return torch


class Solver:
    """One multigrid hierarchy on the GPU (mg_setup) with its caller-owned workspace.

    ``spec`` is an ``inputs.ProblemSpec``-like object with fields dim, n, periodic_y,
    kind, h, c, sx, sy, sz, k.  Arrays are numpy or torch; they are copied to the
    device once.
    """

    def __init__(self, spec, levels, smoother="rbgs", omega=1.0, nu1=2, nu2=2, omega_corr=1.0,
                 precision="fp64", max_cycles=100, inner_cycles=1, flags=0, device="cuda", stream=None,
                 coarse_cut_nodes=0, sweep_rows=0, tile_nodes=0, debug=False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("the multigrid solver needs a CUDA GPU; no CPU path exists")
        self.lib = load(debug=debug)
        self.device = torch.device(device)
        self.spec = spec
        self.dim = spec.dim
        self.n = tuple(spec.n)
        p = Params()
        p.dim = spec.dim
        p.n = (C.c_int * 3)(*[int(v) for v in spec.n])
        p.periodic_y = int(bool(spec.periodic_y))
        p.levels = int(levels)
        p.smoother = SMOOTHERS[smoother] if isinstance(smoother, str) else int(smoother)
        p.omega = float(omega)
        p.nu1, p.nu2 = int(nu1), int(nu2)
        p.omega_corr = float(omega_corr)
        p.precision = {"fp64": FP64, "mixed": MIXED}[precision] if isinstance(precision, str) else int(precision)
        p.max_cycles = int(max_cycles)
        p.inner_cycles = int(inner_cycles)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p.stream = self.stream.cuda_stream
        p.flags = int(flags)
        p.coarse_cut_nodes = int(coarse_cut_nodes)
        p.sweep_rows = int(sweep_rows)
        p.tile_nodes = int(tile_nodes)
        self.params = p
        k = Coeffs()
        k.kind = int(spec.kind)
        k.h = (C.c_double * 3)(*[float(v) for v in spec.h])
        k.c = (C.c_double * 3)(*[float(v) for v in (spec.c if spec.c is not None else (0, 0, 0))])
        self._coef_tensors = []
        for name in ("sx", "sy", "sz", "k", "ex", "ey", "ez"):
            arr = getattr(spec, name, None)
            if arr is not None:
                t = torch.as_tensor(np.ascontiguousarray(arr, dtype=np.float64) if isinstance(arr, np.ndarray)
                                    else arr, dtype=torch.float64, device=self.device).contiguous()
                self._coef_tensors.append(t)
                setattr(k, name, t.data_ptr())
        self.coeffs = k
        nbytes = self.lib.mg_workspace_bytes(C.byref(p), C.byref(k))
        if nbytes == 0:
            raise MGError(EINVAL, "invalid solver parameters")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        ctx = C.c_void_p()
        st = self.lib.mg_setup(C.byref(p), C.byref(k), C.c_void_p(aligned), nbytes, C.byref(ctx))
        if st != OK:
            msg = self.lib.mg_last_error(ctx).decode() if ctx.value else ""
            if ctx.value:
                self.lib.mg_destroy(ctx)
            raise MGError(st, msg)
        self.ctx = ctx
        self.levels = levels
        self.max_cycles = max_cycles
        del self._coef_tensors   # the library copied the coefficients

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value and self.lib is not None:
            self.lib.mg_destroy(ctx)
            self.ctx = None

    # -- helpers -------------------------------------------------------------------------
    def _dev(self, a):
        torch = _torch()
        if isinstance(a, np.ndarray):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)
        return a.to(device=self.device, dtype=torch.float64).contiguous()

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise MGError(st, self.lib.mg_last_error(self.ctx).decode())
        return st

    def level_shape(self, l):
        n = (C.c_int * 3)()
        self._check(self.lib.mg_level_dims(self.ctx, l, n))
        return (n[1], n[0]) if self.dim == 2 else (n[2], n[1], n[0])

    @property
    def shape(self):
        return self.level_shape(self.levels)

    def empty(self, l=None):
        return _torch().zeros(self.level_shape(self.levels if l is None else l), dtype=_torch().float64,
                              device=self.device)

    # -- solves --------------------------------------------------------------------------
    def _run(self, fn, rhs, x0, tol, history):
        rhs = self._dev(rhs)
        x = self.empty() if x0 is None else self._dev(x0).clone()
        hist = np.zeros(self.max_cycles + 2, dtype=np.float64)
        rep = Report()
        rep.history = hist.ctypes.data
        rep.history_cap = len(hist)
        st = fn(self.ctx, C.c_void_p(rhs.data_ptr()), C.c_void_p(x.data_ptr()), float(tol), C.byref(rep))
        self._check(st, allow=(OK, ENOCONV, EDIVERGED))
        info = dict(status=STATUS[st], cycles=rep.cycles, relres=rep.relres, rate=rep.rate,
                    seconds=rep.seconds, history=hist[:rep.cycles + 1].copy())
        return x, info

    def solve_into(self, b, x, tol=1e-10):
        """mg_solve on caller tensors: x (float64, on the device, contiguous) holds the start
        vector on entry and the solution on return.  Returns the info dict."""
        hist = np.zeros(self.max_cycles + 2, dtype=np.float64)
        rep = Report()
        rep.history = hist.ctypes.data
        rep.history_cap = len(hist)
        st = self.lib.mg_solve(self.ctx, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), float(tol),
                               C.byref(rep))
        self._check(st, allow=(OK, ENOCONV, EDIVERGED))
        return dict(status=STATUS[st], cycles=rep.cycles, relres=rep.relres, rate=rep.rate,
                    seconds=rep.seconds, history=hist[:rep.cycles + 1].copy())

    def solve(self, b, x0=None, tol=1e-10):
        """x with ||b - A x|| / ||b|| <= tol (F-cycles from x0); returns (x, info)."""
        return self._run(self.lib.mg_solve, b, x0, tol, True)

    def solve_host(self, b, x, tol=1e-10):
        """mg_solve_host: b, x are C-contiguous float64 numpy arrays (x: start vector in, solution out)."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        hist = np.zeros(self.max_cycles + 2, dtype=np.float64)
        rep = Report()
        rep.history = hist.ctypes.data
        rep.history_cap = len(hist)
        st = self.lib.mg_solve_host(self.ctx, C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data), float(tol),
                                    C.byref(rep))
        self._check(st, allow=(OK, ENOCONV, EDIVERGED))
        return dict(status=STATUS[st], cycles=rep.cycles, relres=rep.relres, rate=rep.rate,
                    seconds=rep.seconds, history=hist[:rep.cycles + 1].copy())

    def solve_adjoint(self, g, x0=None, tol=1e-10):
        """lambda with A^T lambda = g via the transposed F-cycle; returns (lambda, info)."""
        return self._run(self.lib.mg_solve_adjoint, g, x0, tol, True)

    def grad_coeff(self, u, lam):
        torch = _torch()
        cy = self.n[1] if self.spec.periodic_y else self.n[1] - 1
        shape = (cy, self.n[0] - 1) if self.dim == 2 else (self.n[2] - 1, cy, self.n[0] - 1)
        dk = torch.zeros(shape, dtype=torch.float64, device=self.device)
        u, lam = self._dev(u), self._dev(lam)
        self._check(self.lib.mg_grad_coeff(self.ctx, C.c_void_p(u.data_ptr()), C.c_void_p(lam.data_ptr()),
                                           C.c_void_p(dk.data_ptr())))
        return dk

    def residual_norm(self, u, b, l=None):
        """||b - A_l u||_2 over the unknowns (mg_residual_norm), as a 1-element float64 tensor."""
        l = self.levels if l is None else l
        u, b = self._dev(u), self._dev(b)
        out = _torch().zeros(1, dtype=_torch().float64, device=self.device)
        self._check(self.lib.mg_residual_norm(self.ctx, l, C.c_void_p(u.data_ptr()), C.c_void_p(b.data_ptr()),
                                              C.c_void_p(out.data_ptr())))
        return out

    def apply(self, u, l=None):
        l = self.levels if l is None else l
        u = self._dev(u)
        out = self.empty(l)
        self._check(self.lib.mg_apply(self.ctx, l, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    # -- single steps (the context's precision; FP64 in and out) --------------------------
    def smooth(self, u, g, sweeps=1, order=0, l=None):
        l = self.levels if l is None else l
        u, g = self._dev(u), self._dev(g)
        out = self.empty(l)
        self._check(self.lib.mg_step_smooth(self.ctx, l, C.c_void_p(u.data_ptr()), C.c_void_p(g.data_ptr()),
                                            C.c_void_p(out.data_ptr()), sweeps, order))
        return out

    def defect(self, u, g, l=None):
        l = self.levels if l is None else l
        u, g = self._dev(u), self._dev(g)
        out = self.empty(l)
        self._check(self.lib.mg_step_defect(self.ctx, l, C.c_void_p(u.data_ptr()), C.c_void_p(g.data_ptr()),
                                            C.c_void_p(out.data_ptr())))
        return out

    def restrict(self, r, l=None):
        l = self.levels if l is None else l
        r = self._dev(r)
        out = self.empty(l - 1)
        self._check(self.lib.mg_step_restrict(self.ctx, l, C.c_void_p(r.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def prolong_add(self, ec, u, w=1.0, l=None):
        l = self.levels if l is None else l
        ec, u = self._dev(ec), self._dev(u)
        out = self.empty(l)
        self._check(self.lib.mg_step_prolong(self.ctx, l, C.c_void_p(ec.data_ptr()), C.c_void_p(u.data_ptr()),
                                             C.c_void_p(out.data_ptr()), float(w)))
        return out

    def coarse_solve(self, g):
        g = self._dev(g)
        out = self.empty(1)
        self._check(self.lib.mg_step_coarse(self.ctx, C.c_void_p(g.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def cycle(self, x, b, transposed=False):
        x, b = self._dev(x), self._dev(b)
        out = self.empty()
        self._check(self.lib.mg_step_cycle(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                           C.c_void_p(out.data_ptr()), int(transposed)))
        return out

    def descend(self, u, g, l=None, transposed=False):
        """mg_step_descend: (S^nu1(u, g), R(g - A S^nu1(u, g))); u=None starts from zero."""
        l = self.levels if l is None else l
        g = self._dev(g)
        u = None if u is None else self._dev(u)
        uo, gc = self.empty(l), self.empty(l - 1)
        self._check(self.lib.mg_step_descend(self.ctx, l, None if u is None else C.c_void_p(u.data_ptr()),
                                             C.c_void_p(g.data_ptr()), C.c_void_p(uo.data_ptr()),
                                             C.c_void_p(gc.data_ptr()), int(transposed)))
        return uo, gc

    def ascend(self, ec, u, g, l=None, transposed=False):
        """mg_step_ascend: S^nu2(u + omega_l P ec, g)."""
        l = self.levels if l is None else l
        ec, u, g = self._dev(ec), self._dev(u), self._dev(g)
        uo = self.empty(l)
        self._check(self.lib.mg_step_ascend(self.ctx, l, C.c_void_p(ec.data_ptr()), C.c_void_p(u.data_ptr()),
                                            C.c_void_p(g.data_ptr()), C.c_void_p(uo.data_ptr()), int(transposed)))
        return uo

    def outer_defect(self, x, b):
        """mg_step_outer_defect (MG_MIXED): the refinement loop's defect (float-float or FP64) widened
        to FP64, and the sum of its squares."""
        x, b = self._dev(x), self._dev(b)
        r = self.empty()
        sq = C.c_double()
        self._check(self.lib.mg_step_outer_defect(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                                  C.c_void_p(r.data_ptr()), C.byref(sq)))
        return r, sq.value

    def kernel_timing(self):
        ms, n, by = C.c_double(), C.c_int(), C.c_double()
        self._check(self.lib.mg_kernel_timing(self.ctx, C.byref(ms), C.byref(n), C.byref(by)))
        return ms.value, n.value, by.value

    def trace_report(self):
        """mg_trace_report (contexts made with FLAG_TRACE): list of (kernel, level, launches, ms) since
        the last report, the most expensive first."""
        n = C.c_size_t()
        self._check(self.lib.mg_trace_report(self.ctx, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.mg_trace_report(self.ctx, buf, n.value, C.byref(n)))
        rows = []
        self.trace_header = buf.value.decode().splitlines()[0]
        for line in buf.value.decode().splitlines()[1:]:
            name, lev, cnt, ms = line.split()
            rows.append((name, int(lev), int(cnt), float(ms)))
        return rows

    def launch_count(self):
        return int(self.lib.mg_launch_count(self.ctx))


def _batch_args(solvers, bs, xs):
    n = len(solvers)
    if n < 1 or len(bs) != n or len(xs) != n:
        raise ValueError("solvers, bs and xs must have the same non-zero length")
    for s, b, x in zip(solvers, bs, xs):
        for t in (b, x):
            if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
                raise ValueError("b and x must be contiguous float64 CUDA tensors")
            if tuple(t.shape) != tuple(s.shape):
                raise ValueError(f"tensor shape {tuple(t.shape)} does not match the solver's {tuple(s.shape)}")
    cs = (C.c_void_p * n)(*[s.ctx for s in solvers])
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    return n, cs, bp, xp


def _batch_reports(solvers, n):
    hists = [np.zeros(s.max_cycles + 2, dtype=np.float64) for s in solvers]
    reps = (Report * n)()
    for r, h in zip(reps, hists):
        r.history = h.ctypes.data
        r.history_cap = len(h)
    return reps, hists


def _batch_infos(reps, hists):
    return [dict(status=STATUS[r.status], cycles=r.cycles, relres=r.relres, rate=r.rate, seconds=r.seconds,
                 history=h[:r.cycles + 1].copy()) for r, h in zip(reps, hists)]


class Batch:
    """Several independent solves in one launch (mg_batch_create_ex / mg_batch_solve):
    solvers[i] solves its problem with right-hand side bs[i] and start vector / solution
    xs[i] (contiguous float64 CUDA tensors of the solver's shape, kept by reference).
    mode: BATCH_AUTO (qualifying instances of up to 257^2 in the persistent kernel, the rest
    in one CUDA graph), BATCH_GRAPH or BATCH_PERSISTENT.  Built once; solve() launches it and returns
    one info dict per instance."""

    def __init__(self, solvers, bs, xs, mode=BATCH_AUTO):
        self.lib = list(solvers)[0].lib   # the contexts' library (normal or checking build)
        self.solvers, self.bs, self.xs = list(solvers), list(bs), list(xs)
        n, cs, bp, xp = _batch_args(self.solvers, self.bs, self.xs)
        self.n = n
        h = C.c_void_p()
        st = self.lib.mg_batch_create_ex(cs, n, bp, xp, int(mode), C.byref(h))
        if st != OK:
            raise MGError(st, self.lib.mg_last_error(self.solvers[0].ctx).decode())
        self.handle = h.value

    def info(self):
        """(instances in the persistent launch, its CTAs, its teams) of the batch (mg_batch_info)."""
        per, ctas, teams = C.c_int(), C.c_int(), C.c_int()
        self.lib.mg_batch_info(self.handle, C.byref(per), C.byref(ctas), C.byref(teams))
        return per.value, ctas.value, teams.value

    def solve(self, tol=1e-10):
        """Solve every instance; one info dict per instance, whose status says how that instance
        ended (an instance whose bounded device wait ran out reports MG_ETIMEOUT)."""
        reps, hists = _batch_reports(self.solvers, self.n)
        st = self.lib.mg_batch_solve(self.handle, float(tol), reps)
        if st not in (OK, ENOCONV, EDIVERGED, ETIMEOUT):
            raise MGError(st, self.lib.mg_last_error(self.solvers[0].ctx).decode())
        return _batch_infos(reps, hists)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(solvers, bs, xs, tol=1e-10):
    """mg_solve_batched: build, launch and free the batch graph in one call."""
    lib = list(solvers)[0].lib
    n, cs, bp, xp = _batch_args(solvers, bs, xs)
    reps, hists = _batch_reports(solvers, n)
    st = lib.mg_solve_batched(cs, n, bp, xp, float(tol), reps)
    if st not in (OK, ENOCONV, EDIVERGED):
        raise MGError(st, lib.mg_last_error(solvers[0].ctx).decode())
    return _batch_infos(reps, hists)
