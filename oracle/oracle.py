"""ctypes front end of the FP64 CPU oracle (``mg_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the solver package never imports it.

The oracle follows J. T. Wallis, "Methods toward better Multigrid Solver
Convergence" (2008): the preconditioned-Richardson smoothers of section
"Smoothers" / "The choice of C" and the recursive algorithm MG(l, u, g) of
section "The Multigrid Technique", run as the F-cycle named in the abstract.
See ``mg_oracle.c`` for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_HDR = os.path.join(_HERE, "mg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()

CONST, SEPARABLE, CELL, EDGE = 0, 1, 2, 3
JACOBI, RBGS, LINE_X, LINE_Y, ZEBRA_X, ZEBRA_Y, ADI, GSADI = range(8)
RED_FIRST, BLACK_FIRST = 0, 1
CYCLE_F, CYCLE_V = 0, 1
COARSE_EXACT, COARSE_SMOOTH = 0, 1
OK, EINVAL, ENOMEM, ENOCONV, EDIVERGED = 0, 1, 2, 4, 5

SMOOTHERS = {"jacobi": JACOBI, "rbgs": RBGS, "line_x": LINE_X, "line_y": LINE_Y,
             "zebra_x": ZEBRA_X, "zebra_y": ZEBRA_Y, "adi": ADI, "gsadi": GSADI}


_SO_MT = os.path.join(_BUILD, "liboracle_mt.so")


def build(force: bool = False, threaded: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FP contraction).  threaded=True builds the
    second library of the timed CPU baseline: the same source with -fopenmp -DOR_THREADED,
    whose grid loops run on all host cores with identical results."""
    with _LOCK:
        so = _SO_MT if threaded else _SO
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(so) and os.path.getmtime(so) >= newest:
            return so
        os.makedirs(_BUILD, exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        extra = ["-fopenmp", "-DOR_THREADED"] if threaded else []
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
        return so


class _Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("periodic_y", C.c_int), ("kind", C.c_int),
                ("h", C.c_double * 3), ("c", C.c_double * 3),
                ("sx", C.c_void_p), ("sy", C.c_void_p), ("sz", C.c_void_p), ("k", C.c_void_p),
                ("levels", C.c_int), ("smoother", C.c_int), ("omega", C.c_double),
                ("nu1", C.c_int), ("nu2", C.c_int), ("omega_corr", C.c_double),
                ("coarse_mode", C.c_int), ("coarse_sweeps", C.c_int), ("dense_max", C.c_int),
                ("adaptive_corr", C.c_int), ("ex", C.c_void_p), ("ey", C.c_void_p), ("ez", C.c_void_p),
                ("galerkin", C.c_int)]


_libs = {}


def lib(threaded: bool = False):
    """The oracle library (plain, or the threaded build of the timed CPU baseline)."""
    if threaded not in _libs:
        L = C.CDLL(build(threaded=threaded))
        P = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Config), C.POINTER(P)]
        L.or_create.restype = C.c_int
        L.or_destroy.argtypes = [P]
        L.or_levels.argtypes = [P]
        L.or_levels.restype = C.c_int
        L.or_level_dims.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
        L.or_level_nodes.argtypes = [P, C.c_int]
        L.or_level_nodes.restype = C.c_size_t
        L.or_level_unknowns.argtypes = [P, C.c_int]
        L.or_level_unknowns.restype = C.c_int
        L.or_level_coeffs.argtypes = [P, C.c_int, P]
        L.or_apply.argtypes = [P, C.c_int, P, P]
        L.or_diag.argtypes = [P, C.c_int, P]
        L.or_defect.argtypes = [P, C.c_int, P, P, P]
        L.or_norm2.argtypes = [P, C.c_int, P]
        L.or_norm2.restype = C.c_double
        L.or_smooth.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int]
        L.or_restrict.argtypes = [P, C.c_int, P, P]
        L.or_prolong_add.argtypes = [P, C.c_int, P, P, C.c_double]
        L.or_coarse_solve.argtypes = [P, P, P]
        L.or_cycle.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int]
        L.or_fmg_start.argtypes = [P, P, P, C.c_int]
        L.or_adaptive_omega.argtypes = [P, C.c_int, P, P, P]
        L.or_adaptive_omega.restype = C.c_double
        L.or_fmg_start.restype = None
        L.or_solve.argtypes = [P, P, P, C.c_double, C.c_int, C.c_int, P, C.c_int,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.or_solve.restype = C.c_int
        L.or_grad_k.argtypes = [P, P, P, P]
        L.or_thomas.argtypes = [C.c_int, P, P, P, P, P]
        L.or_cyclic_thomas.argtypes = [C.c_int, P, P, P, P, P]
        L.or_counts.argtypes = [P, P, C.POINTER(C.c_long)]
        L.or_reset_counts.argtypes = [P]
        L.or_level_stencil.argtypes = [P, C.c_int, P]
        L.or_level_stencil.restype = C.c_int
        L.or_threads.argtypes = []
        L.or_threads.restype = C.c_int
        _libs[threaded] = L
    return _libs[threaded]


def threads(threaded: bool = True) -> int:
    """Threads the oracle's grid loops run on in that build."""
    return int(lib(threaded).or_threads())


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


class Problem:
    """Operator description on the finest grid (see ``mg_oracle.h``)."""

    def __init__(self, dim=2, n=(129, 129, 1), periodic_y=False, kind=CONST, h=(1.0, 1.0, 1.0),
                 c=(1.0, 1.0, 1.0), sx=None, sy=None, sz=None, k=None, ex=None, ey=None, ez=None):
        self.dim = dim
        self.n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        if dim == 2:
            self.n = (self.n[0], self.n[1], 1)
        self.periodic_y = bool(periodic_y)
        self.kind = kind
        self.h = tuple(float(v) for v in h)
        self.c = tuple(float(v) for v in c)
        self.sx = None if sx is None else np.ascontiguousarray(sx, dtype=np.float64)
        self.sy = None if sy is None else np.ascontiguousarray(sy, dtype=np.float64)
        self.sz = None if sz is None else np.ascontiguousarray(sz, dtype=np.float64)
        self.k = None if k is None else np.ascontiguousarray(k, dtype=np.float64)
        # EDGE: full node arrays (numpy node shape), weight of the edge to the +x / +y / +z neighbour
        self.ex = None if ex is None else np.ascontiguousarray(ex, dtype=np.float64)
        self.ey = None if ey is None else np.ascontiguousarray(ey, dtype=np.float64)
        self.ez = None if ez is None else np.ascontiguousarray(ez, dtype=np.float64)

    @property
    def shape(self):
        """numpy shape of a node array: (n1, n0) in 2D, (n2, n1, n0) in 3D."""
        return (self.n[1], self.n[0]) if self.dim == 2 else (self.n[2], self.n[1], self.n[0])


class Oracle:
    """One multigrid hierarchy of the oracle."""

    def __init__(self, prob: Problem, levels=2, smoother="rbgs", omega=1.0, nu1=2, nu2=2,
                 omega_corr=1.0, coarse_mode=COARSE_EXACT, coarse_sweeps=2, dense_max=1024,
                 adaptive_corr=False, threaded=False, galerkin=False):
        self.prob = prob
        self._L = lib(threaded)
        cfg = _Config()
        cfg.dim = prob.dim
        cfg.n = (C.c_int * 3)(*prob.n)
        cfg.periodic_y = int(prob.periodic_y)
        cfg.kind = prob.kind
        cfg.h = (C.c_double * 3)(*prob.h)
        cfg.c = (C.c_double * 3)(*prob.c)
        self._keep = []
        for name in ("sx", "sy", "sz", "k", "ex", "ey", "ez"):
            arr = getattr(prob, name)
            if arr is not None:
                self._keep.append(arr)
                setattr(cfg, name, arr.ctypes.data)
        cfg.levels = levels
        cfg.smoother = SMOOTHERS[smoother] if isinstance(smoother, str) else int(smoother)
        cfg.omega = omega
        cfg.nu1, cfg.nu2 = nu1, nu2
        cfg.omega_corr = omega_corr
        cfg.coarse_mode = coarse_mode
        cfg.coarse_sweeps = coarse_sweeps
        cfg.dense_max = dense_max
        cfg.adaptive_corr = int(bool(adaptive_corr))
        cfg.galerkin = int(bool(galerkin))
        h = C.c_void_p()
        st = self._L.or_create(C.byref(cfg), C.byref(h))
        if st != OK:
            raise ValueError(f"oracle setup failed with status {st}")
        self._h = h
        self.levels = levels

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_L", None) is not None:
            self._L.or_destroy(h)
            self._h = None

    # -- level geometry ----------------------------------------------------------
    def dims(self, l):
        n = (C.c_int * 3)()
        self._L.or_level_dims(self._h, l, n)
        return tuple(n)

    def shape(self, l=None):
        n = self.dims(self.levels if l is None else l)
        return (n[1], n[0]) if self.prob.dim == 2 else (n[2], n[1], n[0])

    def zeros(self, l=None):
        return np.zeros(self.shape(l), dtype=np.float64)

    def unknown_mask(self, l=None):
        n = self.dims(self.levels if l is None else l)
        m = np.zeros(self.shape(l), dtype=bool)
        if self.prob.dim == 2:
            ys = slice(None) if self.prob.periodic_y else slice(1, n[1] - 1)
            m[ys, 1:n[0] - 1] = True
        else:
            ys = slice(None) if self.prob.periodic_y else slice(1, n[1] - 1)
            m[1:n[2] - 1, ys, 1:n[0] - 1] = True
        return m

    def unknowns(self, l=None):
        return self._L.or_level_unknowns(self._h, self.levels if l is None else l)

    # -- steps of the method -----------------------------------------------------
    def apply(self, u, l=None):
        l = self.levels if l is None else l
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = self.zeros(l)
        self._L.or_apply(self._h, l, _ptr(u), _ptr(out))
        return out

    def diag(self, l=None):
        l = self.levels if l is None else l
        out = self.zeros(l)
        self._L.or_diag(self._h, l, _ptr(out))
        return out

    def defect(self, u, g, l=None):
        l = self.levels if l is None else l
        u = np.ascontiguousarray(u, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = self.zeros(l)
        self._L.or_defect(self._h, l, _ptr(u), _ptr(g), _ptr(out))
        return out

    def norm(self, v, l=None):
        l = self.levels if l is None else l
        return self._L.or_norm2(self._h, l, _ptr(np.ascontiguousarray(v, dtype=np.float64)))

    def smooth(self, u, g, sweeps=1, order=RED_FIRST, l=None):
        l = self.levels if l is None else l
        u = np.array(u, dtype=np.float64, copy=True, order="C")
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._L.or_smooth(self._h, l, _ptr(u), _ptr(g), sweeps, order)
        return u

    def restrict(self, rf, lf=None):
        lf = self.levels if lf is None else lf
        rf = np.ascontiguousarray(rf, dtype=np.float64)
        out = self.zeros(lf - 1)
        self._L.or_restrict(self._h, lf, _ptr(rf), _ptr(out))
        return out

    def prolong_add(self, ec, uf, w=1.0, lf=None):
        lf = self.levels if lf is None else lf
        ec = np.ascontiguousarray(ec, dtype=np.float64)
        uf = np.array(uf, dtype=np.float64, copy=True, order="C")
        self._L.or_prolong_add(self._h, lf, _ptr(ec), _ptr(uf), w)
        return uf

    def coarse_solve(self, g):
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = self.zeros(1)
        self._L.or_coarse_solve(self._h, _ptr(g), _ptr(out))
        return out

    def cycle(self, u, g, l=None, cycle=CYCLE_F, transposed=False):
        l = self.levels if l is None else l
        u = np.array(u, dtype=np.float64, copy=True, order="C")
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._L.or_cycle(self._h, l, _ptr(u), _ptr(g), cycle, int(transposed))
        return u

    def adaptive_omega(self, u, g, e, l=None):
        """Energy-optimal correction weight at level l for iterate u, right-hand side g and
        coarse correction e (or_adaptive_omega)."""
        l = self.levels if l is None else l
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, g, e)]
        return self._L.or_adaptive_omega(self._h, l, *[_ptr(a) for a in arrs])

    def fmg_start(self, b, ncyc=1):
        """Nested-iteration start vector (or_fmg_start)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = self.zeros()
        self._L.or_fmg_start(self._h, _ptr(b), _ptr(x), int(ncyc))
        return x

    def solve(self, b, x0=None, tol=1e-10, maxit=100, transposed=False, start="given"):
        """F-cycles until ||b - A x|| / ||b|| <= tol from x0 (zero if None), or from the
        nested-iteration start when start == "fmg".  Returns (x, status, cycles, relres, history)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if start == "fmg":
            x0 = self.fmg_start(b)
        x = self.zeros() if x0 is None else np.array(x0, dtype=np.float64, copy=True, order="C")
        hist = np.zeros(maxit + 1, dtype=np.float64)
        cyc = C.c_int()
        rr = C.c_double()
        st = self._L.or_solve(self._h, _ptr(b), _ptr(x), tol, maxit, int(transposed), _ptr(hist), maxit + 1,
                            C.byref(cyc), C.byref(rr))
        return x, st, cyc.value, rr.value, hist[:cyc.value + 1].copy()

    def grad_k(self, u, lam):
        p = self.prob
        cx = p.n[0] - 1
        cy = p.n[1] if p.periodic_y else p.n[1] - 1
        shape = (cy, cx) if p.dim == 2 else (p.n[2] - 1, cy, cx)
        out = np.zeros(shape, dtype=np.float64)
        self._L.or_grad_k(self._h, _ptr(np.ascontiguousarray(u, dtype=np.float64)),
                        _ptr(np.ascontiguousarray(lam, dtype=np.float64)), _ptr(out))
        return out

    def level_coeffs(self, l):
        n = self.dims(l)
        p = self.prob
        if p.kind == CONST:
            out = np.zeros(3)
        elif p.kind == SEPARABLE:
            out = np.zeros(3 * n[0])
        elif p.kind == EDGE:
            out = np.zeros(3 * n[0] * n[1] * n[2])
        else:
            cy = n[1] if p.periodic_y else n[1] - 1
            out = np.zeros((n[0] - 1) * cy * (n[2] - 1 if p.dim == 3 else 1))
        self._L.or_level_coeffs(self._h, l, _ptr(out))
        return out

    def stencil(self, l):
        """The 9-point stencil of a Galerkin level: array (..., 3, 3) over the node shape with
        [.., b + 1, a + 1] = A(p, p + (a, b))."""
        out = np.zeros(self.shape(l) + (3, 3))
        if self._L.or_level_stencil(self._h, l, _ptr(out)) != OK:
            raise ValueError(f"level {l} has no 9-point stencil")
        return out

    def counts(self):
        sm = np.zeros(self.levels, dtype=np.int64)
        nc = C.c_long()
        self._L.or_counts(self._h, sm.ctypes.data_as(C.c_void_p), C.byref(nc))
        return sm, nc.value

    def reset_counts(self):
        self._L.or_reset_counts(self._h)


def thomas(lo, di, up, d):
    m = len(di)
    x = np.zeros(m)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (lo, di, up, d)]
    lib().or_thomas(m, *[_ptr(a) for a in arrs], _ptr(x))
    return x


def cyclic_thomas(lo, di, up, d):
    """Cyclic tridiagonal solve (or_cyclic_thomas): lo[0] couples row 0 to x[m-1], up[m-1] row m-1 to x[0]."""
    m = len(di)
    x = np.zeros(m)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (lo, di, up, d)]
    lib().or_cyclic_thomas(m, *[_ptr(a) for a in arrs], _ptr(x))
    return x
